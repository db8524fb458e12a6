// Internal declarations shared by the library's translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <vector>

#include "../../include/lat.h"

// The bulk-copy rings refill a shared-memory slot only after a block barrier that follows every
// thread's last read of it; build with -DLAT_RING_PROXY_FENCE=1 to also issue a generic-to-async
// proxy fence before each refill.
#ifndef LAT_RING_PROXY_FENCE
#define LAT_RING_PROXY_FENCE 0
#endif

namespace lat {

// Device status bits; translated to LAT_E* codes by the host.
enum : unsigned {
    ST_CFL = 1u,       // Eq. (cfl) violated by the evolving flow
    ST_NUMERIC = 2u,   // non-finite value in f
    ST_NOISE = 4u,     // noise table exhausted
    ST_OVERFLOW = 8u,  // reduced-precision scale overflow
    ST_TIMEOUT = 16u,  // a bounded wait gave up
};

// Device-resident step counter and status word of one context.
struct DevState {
    long long step;        // steps taken
    long long noise_base;  // step at which noise row 0 applies
    long long noise_rows;  // rows in the noise table
    unsigned status;
    unsigned stall;        // != 0: the bulk-copy producers issue nothing (lat_debug_stall)
};

// One 1D lattice instance as the kernels see it.
struct Inst1D {
    long long off;    // element offset of f[0][0] in the ensemble buffer
    long long xoff;   // offset of this instance's cells in per-cell arrays (sum of earlier nx)
    int nx;
    int pow2;         // 1 if nx is a power of two
    double g;         // dt / tau_p
    double inv_dv;    // 1 / dv
    double dv;
    double dx;
    double r;         // kappa dt / dv^2
    double ou_e;      // e^{-dt/tau_f}
    double ou_s;      // sigma sqrt(1 - e^2)
    double two_over_nx;
    double dt;
};

// Step kernel variants (1D).
enum { STEP1D_PLAIN = 0, STEP1D_RING = 1, STEP1D_PC = 2 };

constexpr int kMaxModes1D = 16;
constexpr int kMaxModes2D = 512;

// Arguments of the 1D step kernels.
struct Step1DArgs {
    void* f[2];              // ping-pong buffers: absolute step s reads f[s & 1], writes the other
    const Inst1D* inst;
    const int2* items;       // (instance, first x) of each tile
    int item_begin, item_end;
    int flow_kind;           // LAT_FLOW_*
    int nmodes;
    int k[kMaxModes1D];
    const double* amp;       // [2][n_inst][2M] parity-indexed amplitudes
    double* amp_w;           // same buffer, written (other parity)
    const float* ampf;       // FP32 copy of amp read by the FP32 kernels
    float* ampf_w;
    long long amp_stride;    // n_inst * 2M
    const double* noise;     // [rows][n_inst][2M]
    const void* field;       // FIELD flow, per-cell array over all instances
    DevState* st;
    int dry;                 // 1: do not advance the flow (autotuning)
    int frozen;              // 1: flow frozen (tau_f infinite)
    int scheme;              // LAT_SCHEME_UPWIND or LAT_SCHEME_KOREN (drag sub-step)
    double mu;               // limiter bound psi(theta) <= mu theta (KOREN)
    // moments of the new state, fused into the step (k_step1d_pc with moments); may be null
    double* m_rho;
    double* m_mv;
    double* m_mv2;
    double* m_partials;      // [item][consumer warp][M, P, E][sum, compensation]
};

constexpr int kPcConsumerWarps = 4;

// Arguments of the moment kernels (1D).
struct Mom1DArgs {
    const void* f;
    const Inst1D* inst;
    const int2* items;
    int nitems;
    int nv;
    double* rho;
    double* mean_v;
    double* mean_v2;
    double* partials;        // [nitems][3][2] (sum, compensation)
    DevState* st;
};

// Launchers (step1d.cu, moments.cu).
cudaError_t launch_step1d(int dtype, int nv, int variant, int block, int slots, int grid,
                          const Step1DArgs& a, int kstep, cudaStream_t s);
int step1d_max_block(int dtype, int nv, int variant);
bool step1d_ring_supported(int dtype, int nv);
bool step1d_limiter_supported(int nv);
int step1d_ring_tile();
int step1d_ring_min_nx();
int step1d_ring_occupancy(int nv, int slots, int variant);
// One producer/consumer step (2 slots) that also writes the moments of the new state.
cudaError_t launch_step1d_moments(int nv, int grid, const Step1DArgs& a, cudaStream_t s);
bool step1d_moments_supported(int dtype, int nv);
cudaError_t launch_moments1d(int dtype, int block, int tile_xpt, int grid, const Mom1DArgs& a,
                             cudaStream_t s);
// Fold per-instance partials: instance i owns partials [per_item begin[i], per_item begin[i+1]).
// Observables (observables.cu): <rho_r^2> and the Eulerian S1 from per-cell rho (FP64).
cudaError_t launch_coarse1d(const double* rho, const Inst1D* inst, int n_inst, long long total_x,
                            const int* widths, int nw, double* P, double* out, int sm_count,
                            cudaStream_t s);
cudaError_t launch_coarse2d(const double* rho, int nx, int ny, double dx, const int* widths,
                            int nw, double* S, double* out, int sm_count, cudaStream_t s);
cudaError_t launch_s1_1d(int dtype, const void* f, const Inst1D* inst, int n_inst, int nv,
                         const double* rho, const int* seps, int ns, double* num, double* den,
                         int sm_count, cudaStream_t s);

// State I/O (state_io.cu): element conversions between FP64 and FP32 arrays of n values, and
// the device step counter, noise window and status of a restored checkpoint.
cudaError_t launch_f64_to_f32(const double* src, float* dst, long long n, cudaStream_t s);
cudaError_t launch_f32_to_f64(const float* src, double* dst, long long n, cudaStream_t s);
cudaError_t launch_set_devstate(DevState* st, long long step, long long noise_base,
                                long long noise_rows, cudaStream_t s);
cudaError_t launch_set_stall(DevState* st, unsigned on, cudaStream_t s);

cudaError_t launch_finalize1d(const double* partials, const int* inst_item_begin,
                              const Inst1D* inst, int n_inst, double* glob, int per_item,
                              cudaStream_t s);
cudaError_t launch_advance_step(DevState* st, long long n, cudaStream_t s);

}  // namespace lat

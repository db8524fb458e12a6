// Internal declarations shared by the library's translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <vector>

#include "../../include/lat.h"

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
    unsigned pad;
};

// One 1D lattice instance as the kernels see it.
struct Inst1D {
    long long off;    // element offset of f[0][0] in the ensemble buffer
    long long xoff;   // offset of this instance's cells in per-cell arrays (sum of earlier nx)
    int nx;
    int pad;
    double g;         // dt / tau_p
    double inv_dv;    // 1 / dv
    double dv;
    double dx;
    double r;         // kappa dt / dv^2
    double ou_e;      // e^{-dt/tau_f}
    double ou_s;      // sigma sqrt(1 - e^2)
};

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
    long long amp_stride;    // n_inst * 2M
    const double* noise;     // [rows][n_inst][2M]
    const void* field;       // FIELD flow, per-cell array over all instances
    DevState* st;
    int dry;                 // 1: do not advance the flow (autotuning)
    int frozen;              // 1: flow frozen (tau_f infinite)
};

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
cudaError_t launch_step1d(int dtype, int nv, int block, int xpt, int grid, const Step1DArgs& a,
                          int kstep, cudaStream_t s);
bool step1d_supported(int dtype, int nv, int xpt);
int step1d_max_block(int dtype, int nv, int xpt);
cudaError_t launch_moments1d(int dtype, int block, int tile_xpt, int grid, const Mom1DArgs& a,
                             cudaStream_t s);
cudaError_t launch_finalize1d(const double* partials, const int* inst_item_begin,
                              const Inst1D* inst, int n_inst, double* glob, cudaStream_t s);
cudaError_t launch_advance_step(DevState* st, long long n, cudaStream_t s);

}  // namespace lat

// Internal interface of the 2D lattice context (step2d.cu), used by lat_api.cu.
#pragma once

#include "lat_internal.h"

namespace lat {

struct Ctx2D;

int ctx2d_create(Ctx2D** out, const lat_grid* g, DevState* st, int sm_count, cudaStream_t s);
int ctx2d_set_flow(Ctx2D* c, const lat_flow* fl, bool frozen, cudaStream_t s);
int ctx2d_set_noise(Ctx2D* c, const double* noise, long long rows, long long step,
                    cudaStream_t s);
int ctx2d_step(Ctx2D* c, void* const f[2], int n, cudaStream_t s);
int ctx2d_prepare(Ctx2D* c, void* const f[2], int n);
void ctx2d_geometry(const Ctx2D* c, int* nx, int* ny, int* nv, double* dx, double* dv);
int ctx2d_set_scheme(Ctx2D* c, int scheme, double mu);
// The moments of buffer f; the globals go to host memory, through a stream synchronisation
// (wait) or by an asynchronous copy into the caller's pinned buffer.
int ctx2d_moments(Ctx2D* c, const void* f, int cur, double* rho, double* mean_v,
                  double* mean_v2, double* globals, bool wait, cudaStream_t s);
// One step whose kernel also reduces the moments of the state it writes (FP32 storage, upwind,
// producer/consumer launch variants 4, 5 and 8-10); LAT_EINVAL otherwise
// (ctx2d_moments_fusable).  globals and wait as for ctx2d_moments.
bool ctx2d_moments_fusable(const Ctx2D* c);
int ctx2d_step_moments(Ctx2D* c, void* const f[2], double* rho, double* mean_v,
                       double* mean_v2, double* globals, bool wait, cudaStream_t s);
// 16-bit storage: line maxima of the caller's initial state (scales 1), encoding of an FP32
// state into the current buffer, decoding of the current buffer (dst and/or its line scales).
int ctx2d_init_state(Ctx2D* c, void* const f[2], int cur, cudaStream_t s);
int ctx2d_encode(Ctx2D* c, const float* src, void* const f[2], int cur, cudaStream_t s);
int ctx2d_decode(Ctx2D* c, void* const f[2], int cur, float* dst, float* scales, cudaStream_t s);
// Learned flux closure (FP32 contexts): parameters from host memory, mode 0 off, 1 FP32 network,
// 2 BF16 tensor-core network; the loss and gradient of an n-step rollout (FP32 network).
int ctx2d_learn_set(Ctx2D* c, const float* params, int mode, cudaStream_t s);
int ctx2d_learn_corr(Ctx2D* c, void* const f[2], int cur, float* G_out, int reuse,
                     cudaStream_t s);
int ctx2d_learn_grad(Ctx2D* c, void* const f[2], int cur, int n, const float* target,
                     double rho_weight, double* loss, float* grad, cudaStream_t s);
int ctx2d_set_launch(Ctx2D* c, int kernel, int block, int bps, int mode);
int ctx2d_autotune(Ctx2D* c, void* const f[2], int reps, double* best, cudaStream_t s);
void ctx2d_destroy(Ctx2D* c);

// Parts of a 2D context that a checkpoint saves and restores (pointers into its scratch).
struct Ctx2DDyn {
    long long nlines = 0;        // 16-bit line scales (and maxima) per parity; 0 otherwise
    float* sc = nullptr;         // [2][nlines]
    unsigned* mx = nullptr;      // [2][nlines]
    int flow_kind = 0, nmodes = 0;
    double* phase = nullptr;     // [2][nmodes], MODES flows
    double* noise = nullptr;     // noise table, [rows][nmodes]
    long long noise_cap = 0;     // doubles
    double g = 0, r = 0;         // dt / tau_p, kappa dt / dv^2
    bool frozen = true;          // the flow does not evolve (no noise consumed)
};
void ctx2d_dyn(const Ctx2D* c, Ctx2DDyn* out);
// Grow the noise table to at least `doubles` values (contents not kept).
int ctx2d_noise_reserve(Ctx2D* c, long long doubles, cudaStream_t s);
// Drop the cached step graphs (a restored state may have moved the noise table).
void ctx2d_drop_graphs(Ctx2D* c);

}  // namespace lat

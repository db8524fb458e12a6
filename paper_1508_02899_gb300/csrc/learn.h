// Internal interface of the learned flux closure on a coarse 2D lattice (learn.cu, learn_tc.cu),
// used by the 2D context in step2d.cu.
//
// One learned step: the streamed density rho* of every spatial cell; per phase-space cell the
// 16 features, the 16-64-64-2 ReLU network with tanh-bounded outputs y, and the correction
// fluxes y (f*_{j+1} - f*_j) on the interior velocity faces (G[0]: face jx + 1/2, G[1]: face
// jy + 1/2, zero on the walls); then the plain step with G added to the upwind drag fluxes.
#pragma once

#include <cuda_runtime.h>

#include "step2d_dev.h"

namespace lat {

constexpr int kLNF = 16, kLNH = 64, kLNO = 2;
// parameter vector: W1 [16][64], b1 [64], W2 [64][64], b2 [64], W3 [64][2], b3 [2] (x W + b)
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kLNF * kLNH;
constexpr int kOffW2 = kOffB1 + kLNH;
constexpr int kOffB2 = kOffW2 + kLNH * kLNH;
constexpr int kOffW3 = kOffB2 + kLNH;
constexpr int kOffB3 = kOffW3 + kLNH * kLNO;
constexpr int kLNParam = kOffB3 + kLNO;
constexpr float kYMax = 0.25f;   // output bound towards extra diffusion
constexpr float kTheta = 0.9f;   // share of the upwind numerical diffusivity y may take back

// Bound of an output for z > 0: kTheta |ca| (1 - |ca|) / 2, ca = c a_cell - g / 2 the face
// value of the cell's drag Courant number (the numerical diffusivity of the upwind flux).
__host__ __device__ __forceinline__ float anti_bound(float ca_cell, float g) {
    const float ca = fabsf(ca_cell - 0.5f * g);
    return kTheta * 0.5f * fmaxf(ca * (1.f - ca), 0.f);
}

struct LearnArgs {
    const float* f[2];     // state buffers; the step reads parity (st->step + k) & 1
    const float* u;        // flow [2][ny][nx]
    float* rho;            // streamed density [ny][nx]
    float4* feat;          // per spatial cell, two float4 (or null): [1/rho*, dt du_x/dx,
                           // dt du_x/dy, dt du_y/dx], [dt du_y/dy, u_x/dv, u_y/dv, 0]
    const float* params;   // FP32 parameters [kLNParam]
    float* G;              // corrections [2][N_v^2][ny][nx]
    const DevState* st;
    int nx, ny;
    float g;               // dt / tau_p
    float inv_dv;          // 1 / dv
    float dt_2dx;          // dt / (2 dx): centred differences of u times dt
};

// Periodic wrap of v = i + d with |d| < n (the learned step needs N_x, N_y > J).
__device__ __forceinline__ int wrap_near(int v, int n) {
    v += v < 0 ? n : 0;
    return v >= n ? v - n : v;
}

// Phase-cell index i (< 2^32) -> plane p and spatial cell (x, y), 32-bit divisions.
__device__ __forceinline__ void split_index(unsigned i, unsigned ncell, unsigned nx, int& p, int& x,
                                            int& y) {
    p = (int)(i / ncell);
    const unsigned c = i - (unsigned)p * ncell;
    y = (int)(c / nx);
    x = (int)(c - (unsigned)y * nx);
}

bool learn_nv_supported(int nv);
cudaError_t launch_rho_star(int nv, const LearnArgs& a, int k, cudaStream_t s);
cudaError_t launch_mlp_f32(int nv, const LearnArgs& a, int k, cudaStream_t s);
// The same network in BF16 on the tensor cores (tcgen05, FP32 accumulation in TMEM), from the
// parameter tiles that launch_learn_tc_pack builds from the FP32 parameters.  With `units` and
// N_x a multiple of 128 a CTA takes all planes of 128 x of one grid row in turn, sliding the
// velocity neighbourhood of f* from plane to plane; otherwise tiles of 128 phase cells in
// storage order.  Both give the same bits.
bool learn_tc_supported(int nv);
size_t learn_tc_bytes();
cudaError_t launch_learn_tc_pack(const float* params, void* wtc, cudaStream_t s);
cudaError_t launch_mlp_tc(int nv, const LearnArgs& a, const void* wtc, int sm_count, bool units,
                          int k, cudaStream_t s);
// The plain 2D FP32 step (Step2DArgs) with the corrections G added to the drag fluxes, on a
// persistent grid of as many blocks as are resident on sm_count SMs.
cudaError_t launch_step2d_corr(int nv, int sm_count, const k2d::Step2DArgs& a, const float* G,
                               int k, cudaStream_t s);

// ---- gradient of a rollout (FP32, CUDA cores) ---------------------------------------------
// Buffers of one backward step: lam_out = dL/df^{n+1} (in), lam_in = dL/df^n (out); f = f^n;
// work arrays: lss (dL/df**), lrho [ny][nx], dX9 [9][N_v^2][ny][nx]; grad [kLNParam] accumulates.
struct LearnBwdArgs {
    LearnArgs fw;          // f[0] = f[1] = f^n, u = u^n, rho = rho*^n (recomputed)
    const float* lam_out;
    float* lss;
    float* lrho;
    float* dX9;
    float* cxy;            // [2][N_v^2][ny][nx]: y lambda_F of faces jx + 1/2, jy + 1/2
    float* lfs;            // dL/df* without the neighbour-feature and density terms
    float* lam_in;
    float* grad;
    float r;               // kappa dt / dv^2
};
cudaError_t launch_diffuse_adjoint(int nv, const float* lam, float* out, float r, int nx, int ny,
                                   cudaStream_t s);
cudaError_t launch_mlp_bwd(int nv, const LearnBwdArgs& a, int sm_count, cudaStream_t s);
// The same outputs for the BF16 network on the tensor cores (forward again, network backward and
// the weight-gradient sums as tcgen05 MMAs), from the image launch_learn_tc_pack builds.
cudaError_t launch_mlp_bwd_tc(int nv, const LearnBwdArgs& a, const void* wtc, int sm_count,
                              cudaStream_t s);
cudaError_t launch_gather_adjoint(int nv, const LearnBwdArgs& a, cudaStream_t s);
// Fine 2D state (N_v = nvf, 4 k + 1) -> coarse state (N_v = (nvf - 1)/4 + 1), per velocity axis.
cudaError_t launch_restrict(const float* fine, int nvf, int nx, int ny, float* coarse,
                            cudaStream_t s);
// loss = mean (f - target)^2 + rho_weight mean_x r(x)^2, r = sum over the np velocity planes of
// (f - target) (FP64 sums); lam = dloss/df.  partials: 2 nblocks doubles; r: ncell floats.
cudaError_t launch_loss(const float* f, const float* target, int np, long long ncell,
                        double rho_weight, float* r, float* lam, double* partials, int nblocks,
                        double* loss, cudaStream_t s);

}  // namespace lat

// Internal interface of the reduced-precision (FP16 / BF16) 2D storage path (step2d_h.cu), used
// by the 2D context in step2d.cu.
//
// Storage: f[jy][jx][y][x] as 16-bit values h with one power-of-two scale S per x-line
// (velocity plane (jx, jy), row y): f = h * S.  Scales and line maxima are parity-indexed like
// the two state buffers (absolute step s reads parity s & 1) and stored per row, velocity row,
// then jx padded to N_vp = a multiple of 4, so that the N_v scales of one plane row at one
// source row are a single 16-byte aligned run (one bulk copy):
//   sc[par][(y N_v + jy) N_vp + jx]  FP32 scale 2^E of the lines of buffer par (1 in padding);
//   mx[par][(y N_v + jy) N_vp + jx]  bits of max |f| over the line (non-negative FP32, compared
//                                    as unsigned; 0 in padding).
// Before every step, the scales of the output lines come from a bound on their values (the
// step's growth bound over the 13-cell velocity stencil, see k_scale2d), and the step records
// the output's line maxima for the following step.
#pragma once

#include <cuda_runtime.h>

#include "step2d_dev.h"

namespace lat {

struct Step2DHArgs {
    k2d::Step2DArgs b;
    float* sc[2];
    unsigned* mx[2];
};

// Window of 16-bit values copied per plane row: 128 cells plus 16 bytes of alignment slack.
constexpr int kWinH = k2d::TW + 8;

__host__ __device__ constexpr int nv_padded(int nv) { return (nv + 3) & ~3; }
// Scales (or maxima) per buffer: N_y N_v N_vp.
inline long long scale_count(int nv, int ny) { return (long long)ny * nv * nv_padded(nv); }

bool h2d_supported(int nv);
bool h2d_ring_ok(int nx);
// pcv: 0 plain loads; 4 producer/consumer with a 4-slot ring; 5 with a 3-slot ring.
cudaError_t launch_step2d_h(int dtype, int nv, int pcv, int grid, const Step2DHArgs& a, int k,
                            cudaStream_t s);
int occupancy_step2d_h(int dtype, int nv, int pcv);
// Output-line scales of the step that reads parity (st->step + k) & 1, and zeroed output maxima.
cudaError_t launch_scale2d(int nv, int ny, const Step2DHArgs& a, int k, cudaStream_t s);
// Line maxima of the stored lines of buffer f (decoded with scales sc) into mx.
cudaError_t launch_linemax_h(int dtype, const void* f, const float* sc, unsigned* mx, int nv,
                             int nx, int ny, cudaStream_t s);
// Encode the FP32 state src into f with fresh line scales sc and maxima mx.
cudaError_t launch_encode_h(int dtype, const float* src, void* f, float* sc, unsigned* mx,
                            int nv, int nx, int ny, DevState* st, cudaStream_t s);
// Decode f (scales sc) into the FP32 array dst.
cudaError_t launch_decode_h(int dtype, const void* f, const float* sc, float* dst, int nv, int nx,
                            int ny, cudaStream_t s);
// Copy the scales sc to dst in the dense [jy][jx][y] order.
cudaError_t launch_scales_dense(const float* sc, float* dst, int nv, int ny, cudaStream_t s);
// Set every scale of both parities to 1.
cudaError_t launch_fill_scales(float* sc, long long n, cudaStream_t s);

}  // namespace lat

// State I/O of a context: FP64 <-> FP32 element conversions for the host density calls, and the
// device-side step counter, noise window and status word written when a checkpoint is restored.
#include <math.h>

#include "lat_internal.h"

namespace lat {
namespace {

__global__ void __launch_bounds__(256) k_f64_to_f32(const double* src, float* dst, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = __double2float_rn(src[i]);
}

__global__ void __launch_bounds__(256) k_f32_to_f64(const float* src, double* dst, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = (double)src[i];
}

__global__ void k_set_devstate(DevState* st, long long step, long long base, long long rows) {
    st->step = step;
    st->noise_base = base;
    st->noise_rows = rows;
    st->status = 0u;
    st->stall = 0u;
}

__global__ void k_set_stall(DevState* st, unsigned on) { st->stall = on; }

int grid_for(long long n) {
    const long long b = (n + 255) / 256;
    return (int)(b < 4096 ? (b < 1 ? 1 : b) : 4096);
}

}  // namespace

cudaError_t launch_f64_to_f32(const double* src, float* dst, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_f64_to_f32<<<grid_for(n), 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_f32_to_f64(const float* src, double* dst, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_f32_to_f64<<<grid_for(n), 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_set_devstate(DevState* st, long long step, long long noise_base,
                                long long noise_rows, cudaStream_t s) {
    k_set_devstate<<<1, 1, 0, s>>>(st, step, noise_base, noise_rows);
    return cudaGetLastError();
}

cudaError_t launch_set_stall(DevState* st, unsigned on, cudaStream_t s) {
    k_set_stall<<<1, 1, 0, s>>>(st, on);
    return cudaGetLastError();
}

}  // namespace lat

// ---- Adam update of a parameter vector on the device ----------------------------------------
namespace lat {
namespace {

__global__ void __launch_bounds__(256) k_adam(float* p, float* m, float* v, const float* g, int n,
                                              float gscale, float lr, float b1, float b2,
                                              float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = __fmul_rn(g[i], gscale);
        const float mi = __fmaf_rn(b1, m[i], __fmul_rn(1.f - b1, gi));
        const float vi = __fmaf_rn(b2, v[i], __fmul_rn(1.f - b2, __fmul_rn(gi, gi)));
        m[i] = mi;
        v[i] = vi;
        const float mh = __fdiv_rn(mi, c1), vh = __fdiv_rn(vi, c2);
        p[i] = __fsub_rn(p[i], __fdiv_rn(__fmul_rn(lr, mh), __fadd_rn(__fsqrt_rn(vh), eps)));
    }
}

}  // namespace
}  // namespace lat

extern "C" int lat_adam(float* params, float* m, float* v, const float* grad, int n, int t,
                        double lr, double beta1, double beta2, double eps, double grad_scale,
                        void* stream) {
    if (!params || !m || !v || !grad || n < 1 || t < 1 || !(lr > 0) || !(beta1 >= 0) ||
        !(beta1 < 1) || !(beta2 >= 0) || !(beta2 < 1) || !(eps > 0))
        return LAT_EINVAL;
    const float c1 = (float)(1.0 - pow(beta1, t)), c2 = (float)(1.0 - pow(beta2, t));
    const int grid = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
    lat::k_adam<<<grid, 256, 0, (cudaStream_t)stream>>>(params, m, v, grad, n, (float)grad_scale,
                                                        (float)lr, (float)beta1, (float)beta2,
                                                        (float)eps, c1, c2);
    return cudaGetLastError() == cudaSuccess ? LAT_OK : LAT_ECUDA;
}

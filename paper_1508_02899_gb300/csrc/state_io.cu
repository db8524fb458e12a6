// State I/O of a context: FP64 <-> FP32 element conversions for the host density calls, and the
// device-side step counter, noise window and status word written when a checkpoint is restored.
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

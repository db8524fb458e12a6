// The learned closure's network in BF16 on the fifth-generation tensor cores (tcgen05), FP32
// accumulation in tensor memory.  Same features and output as learn.cu's FP32 network.
//
// A CTA of 128 threads takes tiles of 128 phase-space cells (one cell per thread = one row of
// the M = 128 MMA tile).  Per tile: every thread builds its row of features (FP32 -> BF16) in
// shared memory; one thread issues layer 1 (K = 16, N = 64), the CTA waits on the commit's
// mbarrier, reads its accumulator rows (tcgen05.ld), adds the bias, applies ReLU and writes the
// BF16 activations back as the next A operand; layer 2 (K = 64, N = 64) and layer 3 (K = 64,
// N = 16 with two live outputs) the same way; the outputs y = kYMax tanh(z) times the density
// differences across the +jx and +jy faces are the corrections.
//
// Operand layout (no swizzle, K-major): a tile of R rows by K columns is stored as 8 x 8 core
// matrices of 128 contiguous bytes (8 rows of 8 BF16); the stride between core matrices along
// the rows (SBO) is 128 bytes, along K (LBO) is R/8 * 128 bytes.  Weights W [K][N] are stored
// as B operands B[n][k] = W[k][n] in the same layout, built once by k_pack.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "learn.h"

namespace lat {
namespace {

using namespace k2d;

// byte offsets inside the packed parameter image (global memory and shared memory alike)
constexpr int kW1T = 0;                       // B of layer 1: N 64 x K 16 (2 KB)
constexpr int kW2T = kW1T + 64 * 16 * 2;      // B of layer 2: N 64 x K 64 (8 KB)
constexpr int kW3T = kW2T + 64 * 64 * 2;      // B of layer 3: N 16 x K 64 (2 KB), rows >= 2 zero
constexpr int kBias = kW3T + 16 * 64 * 2;     // FP32 b1 [64], b2 [64], b3 [2] (+2 pad)
constexpr int kImage = kBias + (64 + 64 + 4) * 4;
// shared memory of the kernel: image, A1 (128 x 16), A2 (128 x 64), barrier, TMEM address
constexpr int kSA1 = (kImage + 1023) / 1024 * 1024;
constexpr int kSA2 = kSA1 + 128 * 16 * 2;
constexpr int kSBar = kSA2 + 128 * 64 * 2;
constexpr int kSmem = kSBar + 16;
// Requested per CTA: at most 4 CTAs per SM, so that their TMEM (4 x 128 columns) always fits.
constexpr int kSmemReq = kSmem > 48 * 1024 ? kSmem : 48 * 1024;
constexpr int kTmemCols = 128;                // D1 / D3 at columns 0.., D2 at 64..

__host__ __device__ constexpr unsigned tile_off(int r, int k, int rows) {
    // element (r, k) of a K-major no-swizzle tile with `rows` rows: SBO 128, LBO rows/8 * 128
    return (unsigned)((r & 7) * 16 + (k & 7) * 2 + (r >> 3) * 128 + (k >> 3) * (rows / 8) * 128);
}

__device__ __forceinline__ unsigned su32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t sdesc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, M = 128
__host__ __device__ constexpr unsigned idesc_n(unsigned n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void mma(unsigned dtmem, uint64_t ad, uint64_t bd, unsigned idesc,
                                    int accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     su32(bar))
                 : "memory");
}

__device__ __forceinline__ bool wait_parity(uint64_t* bar, unsigned parity) {
    const unsigned long long t0 = [] {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        return t;
    }();
    for (long long it = 0; it < (1ll << 26); ++it) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, q;\n\t}"
            : "=r"(ok)
            : "r"(su32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 255) == 0) {
            unsigned long long t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            if (t - t0 > 1000000000ull) break;
        }
    }
    return false;
}

// 16 consecutive accumulator columns of this thread's row
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld2(unsigned taddr, float& a, float& b) {
    unsigned r0, r1;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];"
                 : "=r"(r0), "=r"(r1)
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    a = __uint_as_float(r0);
    b = __uint_as_float(r1);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// bias + ReLU of 64 accumulator columns of this thread's row into row r of a 128 x 64 A tile
__device__ __forceinline__ void epilogue64(unsigned taddr, const float* bias, unsigned char* A,
                                           int r) {
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 16) {
        float v[16];
        tmem_ld16(taddr + c0, v);
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // two 8-column core-matrix chunks
            uint4 w;
            const int k = c0 + 8 * h;
            w.x = pack_bf16(fmaxf(v[8 * h + 0] + bias[k + 0], 0.f), fmaxf(v[8 * h + 1] + bias[k + 1], 0.f));
            w.y = pack_bf16(fmaxf(v[8 * h + 2] + bias[k + 2], 0.f), fmaxf(v[8 * h + 3] + bias[k + 3], 0.f));
            w.z = pack_bf16(fmaxf(v[8 * h + 4] + bias[k + 4], 0.f), fmaxf(v[8 * h + 5] + bias[k + 5], 0.f));
            w.w = pack_bf16(fmaxf(v[8 * h + 6] + bias[k + 6], 0.f), fmaxf(v[8 * h + 7] + bias[k + 7], 0.f));
            *reinterpret_cast<uint4*>(A + tile_off(r, k, 128)) = w;
        }
    }
}

__device__ __forceinline__ int vwrap(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

// Features of phase cell (jx, jy, x, y), as in learn.cu.
template <int NV>
__device__ __forceinline__ void features_tc(const LearnArgs& a, const float* f, int jx, int jy,
                                            int x, int y, float (&X)[kLNF], float& fc,
                                            float& fxp, float& fyp) {
    constexpr int J = (NV - 1) / 2;
    const size_t ncell = (size_t)a.nx * a.ny;
    const float rho = a.rho[(size_t)y * a.nx + x];
    const float inv = rho != 0.f ? __frcp_rn(rho) : 0.f;
    int q = 0;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            const int jx2 = jx + dx, jy2 = jy + dy;
            const bool in = jx2 >= 0 && jx2 < NV && jy2 >= 0 && jy2 < NV;
            float v = 0.f;
            if (in)
                v = f[(size_t)(jy2 * NV + jx2) * ncell + (size_t)vwrap(y - (jy2 - J), a.ny) * a.nx +
                      vwrap(x - (jx2 - J), a.nx)];
            if (dy == 0 && dx == 0) fc = v;
            if (dy == 0 && dx == 1) fxp = v;
            if (dy == 1 && dx == 0) fyp = v;
            X[q++] = __fmul_rn(v, inv);
        }
    const float* ux = a.u;
    const float* uy = a.u + ncell;
    const size_t c = (size_t)y * a.nx + x;
    const int xp = x + 1 == a.nx ? 0 : x + 1, xm = x == 0 ? a.nx - 1 : x - 1;
    const int yp = y + 1 == a.ny ? 0 : y + 1, ym = y == 0 ? a.ny - 1 : y - 1;
    X[9] = __fmul_rn(__fsub_rn(ux[(size_t)y * a.nx + xp], ux[(size_t)y * a.nx + xm]), a.dt_2dx);
    X[10] = __fmul_rn(__fsub_rn(ux[(size_t)yp * a.nx + x], ux[(size_t)ym * a.nx + x]), a.dt_2dx);
    X[11] = __fmul_rn(__fsub_rn(uy[(size_t)y * a.nx + xp], uy[(size_t)y * a.nx + xm]), a.dt_2dx);
    X[12] = __fmul_rn(__fsub_rn(uy[(size_t)yp * a.nx + x], uy[(size_t)ym * a.nx + x]), a.dt_2dx);
    X[13] = __fmul_rn(a.g, __fsub_rn(__fmul_rn(ux[c], a.inv_dv), (float)(jx - J)));
    X[14] = __fmul_rn(a.g, __fsub_rn(__fmul_rn(uy[c], a.inv_dv), (float)(jy - J)));
    X[15] = 1.f;
}

template <int NV>
__global__ void __launch_bounds__(128) k_mlp_tc(const LearnArgs a, const unsigned char* image,
                                                int kstep) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* W = sm;
    unsigned char* A1 = sm + kSA1;
    unsigned char* A2 = sm + kSA2;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kSBar);
    unsigned* tslot = reinterpret_cast<unsigned*>(sm + kSBar + 8);
    const int t = threadIdx.x, warp = t >> 5;
    for (int i = t; i < kImage / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(W)[i] = reinterpret_cast<const uint4*>(image)[i];
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         su32(tslot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *tslot;
    const unsigned trow = tmem + ((unsigned)(warp * 32) << 16);  // this warp's lanes
    const float* b1 = reinterpret_cast<const float*>(W + kBias);
    const float* b2 = b1 + 64;
    const float* b3 = b2 + 64;
    const unsigned wbase = su32(W), a1 = su32(A1), a2 = su32(A2);
    const float* f = a.f[(int)((a.st->step + kstep) & 1)];
    const long long ncell = (long long)a.nx * a.ny;
    const long long n = ncell * NV * NV;
    const long long ntiles = (n + 127) / 128;
    unsigned phase = 0;
    bool failed = false;
    for (long long tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
        const long long i = tile * 128 + t;
        const bool on = i < n;
        float X[kLNF], fc = 0.f, fxp = 0.f, fyp = 0.f;
        int jx = 0, jy = 0;
        if (on) {
            const int p = (int)(i / ncell);
            const long long c = i % ncell;
            jy = p / NV;
            jx = p % NV;
            features_tc<NV>(a, f, jx, jy, (int)(c % a.nx), (int)(c / a.nx), X, fc, fxp, fyp);
        } else {
#pragma unroll
            for (int q = 0; q < kLNF; ++q) X[q] = 0.f;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint4 w;
            w.x = pack_bf16(X[8 * h + 0], X[8 * h + 1]);
            w.y = pack_bf16(X[8 * h + 2], X[8 * h + 3]);
            w.z = pack_bf16(X[8 * h + 4], X[8 * h + 5]);
            w.w = pack_bf16(X[8 * h + 6], X[8 * h + 7]);
            *reinterpret_cast<uint4*>(A1 + tile_off(t, 8 * h, 128)) = w;
        }
        // layer 1: D[0..63] = A1 (128 x 16) W1^T
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (t == 0) {
            mma(tmem, sdesc(a1, 2048, 128), sdesc(wbase + kW1T, 1024, 128), idesc_n(64), 0);
            commit(bar);
        }
        bool ok = wait_parity(bar, phase);
        phase ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (ok) epilogue64(trow, b1, A2, t);
        // layer 2: D[64..127] = H1 (128 x 64) W2^T
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (t == 0) {
            for (int kk = 0; kk < 4; ++kk)
                mma(tmem + 64, sdesc(a2 + kk * 2 * 2048, 2048, 128),
                    sdesc(wbase + kW2T + kk * 2 * 1024, 1024, 128), idesc_n(64), kk);
            commit(bar);
        }
        ok = wait_parity(bar, phase);
        phase ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (ok) epilogue64(trow + 64, b2, A2, t);  // MMA 2 is done with A2: overwrite with H2
        // layer 3: D[0..15] = H2 (128 x 64) W3^T
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (t == 0) {
            for (int kk = 0; kk < 4; ++kk)
                mma(tmem, sdesc(a2 + kk * 2 * 2048, 2048, 128),
                    sdesc(wbase + kW3T + kk * 2 * 256, 256, 128), idesc_n(16), kk);
            commit(bar);
        }
        ok = wait_parity(bar, phase);
        phase ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (ok) {
            float y0, y1;
            tmem_ld2(trow, y0, y1);
            if (on) {
                const float z0 = y0 + b3[0], z1 = y1 + b3[1];
                y0 = __fmul_rn(z0 > 0.f ? anti_bound(X[13], a.g) : kYMax, tanhf(z0));
                y1 = __fmul_rn(z1 > 0.f ? anti_bound(X[14], a.g) : kYMax, tanhf(z1));
                a.G[i] = jx < NV - 1 ? __fmul_rn(y0, __fsub_rn(fxp, fc)) : 0.f;
                a.G[n + i] = jy < NV - 1 ? __fmul_rn(y1, __fsub_rn(fyp, fc)) : 0.f;
            }
        }
        // every thread is done with the accumulators and A2 before the next tile's MMAs
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (failed && t == 0) atomicOr(const_cast<unsigned*>(&a.st->status), ST_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
}

// Parameter image: BF16 B operands of the three layers and the FP32 biases.
__global__ void k_pack(const float* P, unsigned char* img) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 64 * 16 + 64 * 64 + 16 * 64;
         e += gridDim.x * blockDim.x) {
        if (e < 64 * 16) {  // W1T [n][k] = W1[k][n]
            const int nn = e / 16, k = e % 16;
            *reinterpret_cast<__nv_bfloat16*>(img + kW1T + tile_off(nn, k, 64)) =
                __float2bfloat16_rn(P[kOffW1 + k * kLNH + nn]);
        } else if (e < 64 * 16 + 64 * 64) {
            const int q = e - 64 * 16, nn = q / 64, k = q % 64;
            *reinterpret_cast<__nv_bfloat16*>(img + kW2T + tile_off(nn, k, 64)) =
                __float2bfloat16_rn(P[kOffW2 + k * kLNH + nn]);
        } else {
            const int q = e - 64 * 16 - 64 * 64, nn = q / 64, k = q % 64;
            *reinterpret_cast<__nv_bfloat16*>(img + kW3T + tile_off(nn, k, 16)) =
                __float2bfloat16_rn(nn < kLNO ? P[kOffW3 + k * kLNO + nn] : 0.f);
        }
    }
    float* bias = reinterpret_cast<float*>(img + kBias);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 64 + 64 + 4; e += gridDim.x * blockDim.x)
        bias[e] = e < 64 ? P[kOffB1 + e] : (e < 128 ? P[kOffB2 + e - 64] : (e < 130 ? P[kOffB3 + e - 128] : 0.f));
}

}  // namespace

#define LEARN_TC_NV_LIST(X) X(3) X(5) X(9) X(13) X(17)

bool learn_tc_supported(int nv) {
    switch (nv) {
#define X(n) case n:
        LEARN_TC_NV_LIST(X)
#undef X
        return true;
        default: return false;
    }
}

size_t learn_tc_bytes() { return (size_t)kImage; }

cudaError_t launch_learn_tc_pack(const float* params, void* wtc, cudaStream_t s) {
    k_pack<<<24, 256, 0, s>>>(params, static_cast<unsigned char*>(wtc));
    return cudaGetLastError();
}

cudaError_t launch_mlp_tc(int nv, const LearnArgs& a, const void* wtc, int sm_count, int k,
                          cudaStream_t s) {
    const long long n = (long long)a.nx * a.ny * nv * nv;
    const int grid = (int)std::max<long long>(1, std::min<long long>((n + 127) / 128, 4LL * sm_count));
    const unsigned char* img = static_cast<const unsigned char*>(wtc);
    switch (nv) {
#define X(nn)                                                                                   \
    case nn: {                                                                                  \
        static bool attr = false;                                                               \
        if (!attr) {                                                                            \
            cudaError_t e = cudaFuncSetAttribute(k_mlp_tc<nn>,                                  \
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                                 kSmemReq);                                     \
            if (e != cudaSuccess) return e;                                                     \
            attr = true;                                                                        \
        }                                                                                       \
        k_mlp_tc<nn><<<grid, 128, kSmemReq, s>>>(a, img, k);                                    \
        return cudaGetLastError();                                                              \
    }
        LEARN_TC_NV_LIST(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lat

// Device code shared by the 2D step kernels of every storage type (included by step2d.cu and
// step2d_h.cu only): PTX wrappers for mbarriers and bulk asynchronous copies, the column
// arithmetic of one velocity row, and the per-cell flow and CFL helpers.
#pragma once

#include <stdint.h>

#include "lat_internal.h"

namespace lat {
namespace k2d {

constexpr int TW = 128;  // cells per tile (= consumer threads per block)

struct Step2DArgs {
    void* f[2];
    int nx, ny;
    double g, r, inv_dv;
    const void* u;            // [2][ny][nx] of T, or null for u = 0
    DevState* st;
    int ntx, ntiles;
};

// ---- PTX helpers (mbarrier + bulk async copy) ----------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait on an mbarrier phase: gives up after ~1 s (then the caller raises ST_TIMEOUT).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (long long it = 0; it < (1ll << 26); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255) == 0 && globaltimer() - t0 > 1000000000ull) break;
    }
    return false;
}

__device__ __forceinline__ int wrap(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// ---- the row sweep shared by both kernels ---------------------------------------------------
// Processes velocity row index r (0..NV): computes f** of row r-1 (needs f* rows r-1 and r, the
// latter absent when r == NV) and, for r >= 2, writes the output row r-2.
// Column arithmetic with explicit rounding, so that every variant gives the same bits.
template <typename T>
struct Ops;
template <>
struct Ops<float> {
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
};
template <>
struct Ops<double> {
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
};
// c a_j = g (w - j);  c F_{j+1/2} = (c a_j)^+ f_j + (c a_{j+1})^- f_{j+1}
template <typename T>
__device__ __forceinline__ T cacc(T g, T w, int j) { return Ops<T>::mul(g, Ops<T>::sub(w, T(j))); }
template <typename T>
__device__ __forceinline__ T dflux(T caj, T can, T fj, T fn) {
    return Ops<T>::fma(fmax(caj, T(0)), fj, Ops<T>::mul(fmin(can, T(0)), fn));
}

// Processes velocity row index r (1..NV): computes f** of row rb = r-1 from f* rows rb (cur) and
// r (nxt, absent when r == NV) and, for r >= 2, writes output row r-2.
//   f**_{jx} = f*_{jx} - (cFx_{jx+1/2} - cFx_{jx-1/2}) - (cFy_{rb+1/2} - cFy_{rb-1/2})
//   out      = f** + (Dx_{jx+1/2} - Dx_{jx-1/2}) + (Dy_{+1/2} - Dy_{-1/2}),  D = r (f**_+ - f**)
// Opaque copy: keeps the compiler from hoisting per-jx invariants (drag coefficients, store
// offsets) out of the row loop into NV live registers each.
__device__ __forceinline__ float opaque(float v) {
    float r;
    asm volatile("mov.b32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ double opaque(double v) {
    double r;
    asm volatile("mov.b64 %0, %1;" : "=d"(r) : "d"(v));
    return r;
}

// Extra drag flux on the interior velocity faces (the learned closure); NoCorr adds nothing.
// Corr::gx(rb, jx): flux through face jx + 1/2 of velocity row rb; Corr::gy(rb, jx): flux
// through face rb + 1/2 of column jx.
struct NoCorr {
    static constexpr bool active = false;
    template <typename T>
    __device__ __forceinline__ T gx(int, int) const { return T(0); }
    template <typename T>
    __device__ __forceinline__ T gy(int, int) const { return T(0); }
};

// The learned closure's corrections of one cell, G [2][N_v^2][N_y][N_x] FP32: the vx faces at
// (plane, cell) from cx = G + cell, the vy faces from cy = G + N_v^2 N_x N_y + cell.
struct GlobCorr {
    static constexpr bool active = true;
    const float* cx;
    const float* cy;
    size_t ps;
    int nv;
    template <typename T>
    __device__ __forceinline__ T gx(int rb, int jx) const { return cx[(size_t)(rb * nv + jx) * ps]; }
    template <typename T>
    __device__ __forceinline__ T gy(int rb, int jx) const { return cy[(size_t)(rb * nv + jx) * ps]; }
};

// The output goes through `put`: put.begin(row) before output row `row`, then put(o) for
// jx = 0..NV-1 in order (StorePut for FP32/FP64 storage).  G (vy-drag flux row) and H
// (vy-diffusion flux row) are register arrays or per-thread shared-memory columns (SmemCol).
template <typename T, int NV, class Row, class GArr, class HArr, class Put, class Corr = NoCorr>
__device__ __forceinline__ void sweep_row(T (&A)[NV], GArr& G, HArr& H, int r,
                                          const Row& cur, const Row& nxt_row, T g_in, T wx_in,
                                          T wy, T rr, Put& put, const Corr& corr = Corr()) {
    using O = Ops<T>;
    constexpr int J = (NV - 1) / 2;
    const int rb = r - 1;
    const bool nxt = r < NV;
    const T g = opaque(g_in), wx = opaque(wx_in);
    const T ayp = fmax(cacc<T>(g, wy, rb - J), T(0));
    const T aym = nxt ? fmin(cacc<T>(g, wy, r - J), T(0)) : T(0);
    T Fprev = T(0), Dprev = T(0);
    T sc = cur.get(0);
    put.begin(r >= 2 ? r - 2 : 0);
#pragma unroll
    for (int jx = 0; jx < NV; ++jx) {
        T sn = T(0), Fnext = T(0);
        if (jx < NV - 1) {
            sn = cur.get(jx + 1);
            Fnext = dflux<T>(cacc<T>(g, wx, jx - J), cacc<T>(g, wx, jx + 1 - J), sc, sn);
            if constexpr (Corr::active) Fnext = O::add(Fnext, corr.template gx<T>(rb, jx));
        }
        T Gn = nxt ? O::fma(ayp, sc, O::mul(aym, nxt_row.get(jx))) : T(0);
        if constexpr (Corr::active) {
            if (nxt) Gn = O::add(Gn, corr.template gy<T>(rb, jx));
        }
        const T b = O::sub(O::sub(sc, O::sub(Fnext, Fprev)), O::sub(Gn, G[jx]));
        G[jx] = Gn;
        Fprev = Fnext;
        sc = sn;
        if (r >= 2) {
            const T a = A[jx];
            const T Dn = (jx < NV - 1) ? O::mul(rr, O::sub(A[jx + 1], a)) : T(0);
            const T Hn = O::mul(rr, O::sub(b, a));
            const T o = O::add(O::add(a, O::sub(Dn, Dprev)), O::sub(Hn, H[jx]));
            H[jx] = Hn;
            Dprev = Dn;
            put(o);
        }
        A[jx] = b;
    }
}

// Last output row (jy = J): no f** row above it, so the vy-diffusion flux there is zero.
template <typename T, int NV, class HArr, class Put>
__device__ __forceinline__ void final_row(T (&A)[NV], HArr& H, T rr, Put& put) {
    using O = Ops<T>;
    T Dprev = T(0);
    put.begin(NV - 1);
#pragma unroll
    for (int jx = 0; jx < NV; ++jx) {
        const T a = A[jx];
        const T Dn = (jx < NV - 1) ? O::mul(rr, O::sub(A[jx + 1], a)) : T(0);
        const T o = O::add(O::add(a, O::sub(Dn, Dprev)), O::sub(T(0), H[jx]));
        Dprev = Dn;
        put(o);
    }
}

// Steps an output pointer by one velocity plane through a volatile asm statement.  In the
// shared-memory sweeps this keeps the compiler from moving the row's loads ahead of earlier
// stores, which would hold many loaded values live across the row and spill the flux rows.
// Kernels that read f* from global memory need those loads in flight early: they step plainly.
template <typename T>
__device__ __forceinline__ T* next_plane(T* p, size_t pstride) {
    unsigned long long q = reinterpret_cast<unsigned long long>(p + pstride);
    asm volatile("mov.b64 %0, %0;" : "+l"(q));
    return reinterpret_cast<T*>(q);
}

// Plain store of every output value: out points at cell (x, y) of plane (0, 0).  OPAQUE: step
// the pointer with next_plane (shared-memory sweeps) instead of a plain addition.
template <typename T, int NV, bool OPAQUE = true>
struct StorePut {
    T* out;
    size_t pstride;
    bool active;
    T* p;
    __device__ __forceinline__ StorePut(T* out_, size_t ps, bool act)
        : out(out_), pstride(ps), active(act), p(out_) {}
    __device__ __forceinline__ void begin(int row) { p = out + (size_t)row * NV * pstride; }
    __device__ __forceinline__ void operator()(T o) {
        if (active) *p = o;
        if constexpr (OPAQUE) p = next_plane(p, pstride);
        else p += pstride;
    }
};

template <typename T>
__device__ __forceinline__ void load_w(const Step2DArgs& a, int x, int y, T& wx, T& wy) {
    if (a.u) {
        const T* u = static_cast<const T*>(a.u);
        const size_t c = (size_t)y * a.nx + x;
        wx = u[c] * T(a.inv_dv);
        wy = u[(size_t)a.nx * a.ny + c] * T(a.inv_dv);
    } else {
        wx = T(0);
        wy = T(0);
    }
}

template <typename T, int NV>
__device__ __forceinline__ void cfl_check(const Step2DArgs& a, T g, T wx, T wy, bool active) {
    constexpr int J = (NV - 1) / 2;
    if (active && g * (T(J) + fabs(wx)) + g * (T(J) + fabs(wy)) > T(1))
        atomicOr(&a.st->status, ST_CFL);
}

// Row jy of f* at one cell, read straight from global memory (periodic wrap in x and y).
template <typename T, int NV>
struct GlobalRow {
    const T* base;  // f + (jy NV ny + ys) nx: plane (jy, 0), source row ys = (y - jy) mod ny
    size_t pstride;
    int x, nx;
    __device__ __forceinline__ GlobalRow(const T* f, int row, int x_, int y, int nx_, int ny)
        : x(x_), nx(nx_) {
        constexpr int J = (NV - 1) / 2;
        pstride = (size_t)nx_ * ny;
        base = f + (size_t)row * NV * pstride + (size_t)wrap(y - (row - J), ny) * nx_;
    }
    __device__ __forceinline__ T get(int jx) const {
        constexpr int J = (NV - 1) / 2;
        return __ldg(base + jx * pstride + wrap(x - (jx - J), nx));
    }
};

struct SmemCol {  // one thread's column in a [NV][TW] shared array
    float* p;
    __device__ __forceinline__ float& operator[](int j) const { return p[j * TW]; }
};

}  // namespace k2d

// Flux-limited 2D step (limiter2d.cu): stage 1, stage 2 and the diffusion of step k of a batch.
// form 1: three passes, with `scratch` holding one state; 2: one fused kernel for the whole
// step (N_v with limiter2d_fused_supported; bps 1 or 2 the resident blocks per SM where both
// are built); 3: the fused kernel on cell pairs in FP32 register pairs (FP32 storage).
cudaError_t launch_step2d_limited(int dtype, const k2d::Step2DArgs& s2, int nv, double mu,
                                  void* scratch, int form, int bps, int k, int sm_count,
                                  cudaStream_t s);
bool limiter2d_fused_supported(int nv);

}  // namespace lat

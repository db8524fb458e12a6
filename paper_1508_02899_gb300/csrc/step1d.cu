// One fused time step of the 1D phase-space lattice (Section 2 of arXiv:1508.02899):
// exact streaming in x, first-order upwind Stokes-drag flux in v, velocity diffusion.
//
// Work decomposition: a work item is one x-tile of one instance; a persistent grid walks the
// item list.  Each thread owns one spatial column x and sweeps its velocity column
// j = -J..J once: the post-streaming value f*(x, j) = f(x - j, j) is gathered (the gather *is*
// the streaming step), the drag flux and the diffusion flux are carried along the sweep as
// scalars with a lag of two cells, and each output value is written once.  HBM traffic per
// cell: one read and one write of f.
//
// Three variants share the column arithmetic (bit-identical results):
//  * ring: the tile's N_v shifted plane windows are brought into a shared-memory ring by bulk
//    asynchronous copies (cp.async.bulk + mbarrier), several items ahead of the sweep, so the
//    loads in flight do not depend on registers or occupancy (FP32, N_x % 4 == 0, N_x >= 132);
//  * reg:  the column is gathered with plain coalesced loads into registers (fixed N_v);
//  * any:  plain loads through a sliding window (any odd N_v).
// The flow u(x, t_n) is evaluated in the same kernel from the mode amplitudes; the first tile
// of every instance also advances those amplitudes to t_{n+1} (parity ping-pong, so no tile
// reads what another tile of the same launch writes).
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "f32x2.h"
#include "lat_internal.h"
#include "lat_reduce.h"

namespace lat {
namespace {

constexpr int TW1 = 128;        // columns per tile of the ring kernel (= threads per block)
constexpr int WIN1 = TW1 + 4;   // floats copied per plane (x window rounded to 16 bytes)

// ---- column arithmetic with explicit rounding (identical in every variant) -----------------
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

// c a_j = (dt/dv) * (-(v_j - u)/tau_p) = g (w - j), g = dt/tau_p, w = u/dv
template <typename T>
__device__ __forceinline__ T cacc(T g, T w, int j) {
    return Ops<T>::mul(g, Ops<T>::sub(w, T(j)));
}
// c F_{j+1/2} = (c a_j)^+ f_j + (c a_{j+1})^- f_{j+1}   (cell-centred upwind)
template <typename T>
__device__ __forceinline__ T dflux(T caj, T can, T fj, T fn) {
    return Ops<T>::fma(fmax(caj, T(0)), fj, Ops<T>::mul(fmin(can, T(0)), fn));
}

// Sliding-window sweep of one column.  get(jj) returns f*(x, jj - J); put(jj, v) stores.
//   d_j   = f*_j - (cF_{j+1/2} - cF_{j-1/2})            (drag, zero flux at the walls)
//   out_j = d_j + (D_{j+1/2} - D_{j-1/2}),  D = r (d_{j+1} - d_j)   (diffusion)
template <typename T, int NV, class Get, class Put>
__device__ __forceinline__ void sweep_column(T w, T g, T r, const Get& get, const Put& put) {
    constexpr int J = (NV - 1) / 2;
    T s = get(0);
    T Fprev = T(0), Dprev = T(0), dprev = T(0);
#pragma unroll
    for (int jj = 0; jj < NV; ++jj) {
        T sn = T(0), Fn = T(0);
        if (jj < NV - 1) {
            sn = get(jj + 1);
            Fn = dflux<T>(cacc<T>(g, w, jj - J), cacc<T>(g, w, jj + 1 - J), s, sn);
        }
        const T d = Ops<T>::sub(s, Ops<T>::sub(Fn, Fprev));
        Fprev = Fn;
        if (jj > 0) {
            const T D = Ops<T>::mul(r, Ops<T>::sub(d, dprev));
            put(jj - 1, Ops<T>::add(dprev, Ops<T>::sub(D, Dprev)));
            Dprev = D;
        }
        dprev = d;
        s = sn;
    }
    put(NV - 1, Ops<T>::add(dprev, Ops<T>::sub(T(0), Dprev)));
}

// Packed two-lane form of sweep_column (FP32, N_v = 2h + 1 >= 5): lane 0 of an f32x2 pair
// sweeps cells 0 .. h, lane 1 cells h .. 2h, with exactly the operations of sweep_column in the
// same order, so the outputs have the same bits.  Lane 1 starts from the drag fluxes of faces
// h - 3/2 and h - 1/2 and the drag output of cell h - 1, which it computes from f*_{h-2..h}
// first.  put2(p, o) for p = 1..h stores lane 0's o at cell p - 1 and lane 1's at p - 1 + h;
// put_last(v) stores cell 2h.
template <int NV, class Get, class Put2, class PutLast>
__device__ __forceinline__ void sweep_column2(float w, float g, float r, const Get& get,
                                              const Put2& put2, const PutLast& put_last) {
    constexpr int J = (NV - 1) / 2, h = J;
    static_assert(NV >= 5, "packed sweep needs N_v >= 5");
    const f2 g2 = pk(g, g), w2 = pk(w, w), r2 = pk(r, r);
    const f2 one2 = opaque2(pk(1.f, 1.f));
    f2 kk = opaque2(pk(float(-J), 0.f));  // velocity indices of step p: (p - J, p)
    f2 cac = mul2(g2, sub2(w2, kk));
    // lane 1's entry state at cell h
    const float fm2 = get(h - 2), fm1 = get(h - 1), f0 = get(h);
    const float Fa = dflux<float>(cacc<float>(g, w, -2), cacc<float>(g, w, -1), fm2, fm1);
    const float Fb = dflux<float>(cacc<float>(g, w, -1), cacc<float>(g, w, 0), fm1, f0);
    const float dm1 = Ops<float>::sub(fm1, Ops<float>::sub(Fb, Fa));
    f2 s2 = pk(get(0), f0);
    f2 Fp = pk(0.f, Fb);
    f2 dp = pk(0.f, dm1);
    f2 Dp = 0ull;
#pragma unroll
    for (int p = 0; p <= h; ++p) {
        const f2 kn = add2(kk, one2);
        const f2 can = mul2(g2, sub2(w2, kn));
        const f2 sn = p < h ? pk(get(p + 1), get(p + 1 + h)) : pk(get(h + 1), 0.f);
        f2 Fn = fma2(max0(cac), s2, mul2(min0(can), sn));
        if (p == h) Fn = pk(lo(Fn), 0.f);  // lane 1 reached the wall
        const f2 d = sub2(s2, sub2(Fn, Fp));
        Fp = Fn;
        const f2 D = mul2(r2, sub2(d, dp));
        if (p == 0) {
            Dp = pk(0.f, hi(D));  // lane 0 has no face below cell 0; lane 1: face h - 1/2
        } else {
            put2(p, add2(dp, sub2s(D, Dp)));
            Dp = D;
        }
        dp = d;
        s2 = sn;
        cac = can;
        kk = kn;
    }
    put_last(Ops<float>::add(hi(dp), Ops<float>::sub(0.f, hi(Dp))));
}

// ---- flux-limited drag (scheme KOREN) -----------------------------------------------------------
// Limited increment psi(theta) dp of Koren's limiter in Hundsdorfer et al.'s form (Sec. 2, flux
// limiter): psi(theta) = max(0, min(1, 1/3 + theta/6, mu theta)), theta = dm / dp, written
// without the division: with s = sign(dp), psi(theta) dp = s max(0, min(|dp|, s (dp/3 + dm/6),
// s mu dm)); zero when dp = 0.
template <typename T>
__device__ __forceinline__ T lim_inc(T dp, T dm, T mu) {
    using O = Ops<T>;
    const T s = copysign(T(1), dp);
    const T b = O::mul(s, O::fma(dm, T(1.0 / 6.0), O::mul(dp, T(1.0 / 3.0))));
    const T c = O::mul(s, O::mul(mu, dm));
    return O::mul(s, fmax(T(0), fmin(fabs(dp), fmin(b, c))));
}

// Limited flux through interface i + 1/2 from the split fluxes P = (c a)^+ q, M = (c a)^- q of
// cells i - 1 .. i + 2 (cells beyond the walls count as empty):
//   F = P_i + psi(theta^P)(P_{i+1} - P_i) + M_{i+1} + psi(theta^M)(M_i - M_{i+1}).
template <typename T, int NV>
__device__ __forceinline__ T lim_face(const T (&P)[NV], const T (&M)[NV], int i, T mu) {
    using O = Ops<T>;
    const T Pm = i >= 1 ? P[i - 1] : T(0);
    const T Mpp = i + 2 < NV ? M[i + 2] : T(0);
    const T pos = O::add(P[i], lim_inc<T>(O::sub(P[i + 1], P[i]), O::sub(P[i], Pm), mu));
    const T neg = O::add(M[i + 1], lim_inc<T>(O::sub(M[i], M[i + 1]), O::sub(M[i + 1], Mpp), mu));
    return O::add(pos, neg);
}

// The limited drag sub-step by Heun's method, then the diffusion, for one column (scheme KOREN):
//   y = x - (F(x)_{j+1/2} - F(x)_{j-1/2}),  h = (x + y - (F(y)_{j+1/2} - F(y)_{j-1/2})) / 2,
//   out = h + (D_{j+1/2} - D_{j-1/2}),  D = r (h_{j+1} - h_j),  zero fluxes at the walls.
// One unrolled pass over k: cell k is read, stage-1 face and cell k - 2, stage-2 face and cell
// k - 4, output k - 5, so that every array element lives for a few iterations only.
template <typename T, int NV, class Get, class Put>
__device__ __forceinline__ void sweep_column_lim(T w, T g, T r, T mu, const Get& get,
                                                 const Put& put) {
    using O = Ops<T>;
    constexpr int J = (NV - 1) / 2;
    T x[NV], P0[NV], M0[NV], y[NV], P1[NV], M1[NV], h[NV], F0[NV + 1], F1[NV + 1];
    T Dprev = T(0);
#pragma unroll
    for (int k = 0; k < NV + 5; ++k) {
        if (k < NV) {
            x[k] = get(k);
            const T ca = cacc<T>(g, w, k - J);
            P0[k] = O::mul(fmax(ca, T(0)), x[k]);
            M0[k] = O::mul(fmin(ca, T(0)), x[k]);
        }
        if (k - 2 >= 0 && k - 2 <= NV - 2) F0[k - 1] = lim_face<T, NV>(P0, M0, k - 2, mu);
        if (k - 2 >= 0 && k - 2 < NV) {
            const int j = k - 2;
            const T Fl = j == 0 ? T(0) : F0[j];
            const T Fr = j == NV - 1 ? T(0) : F0[j + 1];
            y[j] = O::sub(x[j], O::sub(Fr, Fl));
            const T ca = cacc<T>(g, w, j - J);
            P1[j] = O::mul(fmax(ca, T(0)), y[j]);
            M1[j] = O::mul(fmin(ca, T(0)), y[j]);
        }
        if (k - 4 >= 0 && k - 4 <= NV - 2) F1[k - 3] = lim_face<T, NV>(P1, M1, k - 4, mu);
        if (k - 4 >= 0 && k - 4 < NV) {
            const int j = k - 4;
            const T Fl = j == 0 ? T(0) : F1[j];
            const T Fr = j == NV - 1 ? T(0) : F1[j + 1];
            h[j] = O::mul(T(0.5), O::add(x[j], O::sub(y[j], O::sub(Fr, Fl))));
        }
        if (k - 5 >= 0 && k - 5 < NV) {
            const int j = k - 5;
            const T D = j < NV - 1 ? O::mul(r, O::sub(h[j + 1], h[j])) : T(0);
            put(j, O::add(h[j], O::sub(D, Dprev)));
            Dprev = D;
        }
    }
}

// Drag scheme of one column: upwind, or the limited scheme (LIM, a separate kernel instance,
// so that the upwind kernels keep their own code and registers).
template <typename T, int NV, bool LIM, class Get, class Put>
__device__ __forceinline__ void sweep_scheme(const Step1DArgs& a, T w, T g, T r, const Get& get,
                                             const Put& put) {
    if constexpr (LIM) sweep_column_lim<T, NV>(w, g, r, T(a.mu), get, put);
    else sweep_column<T, NV>(w, g, r, get, put);
}

// Runtime-N_v version of the same sweep (identical operation order).
template <typename T, class Get, class Put>
__device__ __forceinline__ void sweep_column_any(int NV, T w, T g, T r, const Get& get,
                                                 const Put& put) {
    const int J = (NV - 1) / 2;
    T s = get(0);
    T Fprev = T(0), Dprev = T(0), dprev = T(0);
#pragma unroll 4
    for (int jj = 0; jj < NV; ++jj) {
        T sn = T(0), Fn = T(0);
        if (jj < NV - 1) {
            sn = get(jj + 1);
            Fn = dflux<T>(cacc<T>(g, w, jj - J), cacc<T>(g, w, jj + 1 - J), s, sn);
        }
        const T d = Ops<T>::sub(s, Ops<T>::sub(Fn, Fprev));
        Fprev = Fn;
        if (jj > 0) {
            const T D = Ops<T>::mul(r, Ops<T>::sub(d, dprev));
            put(jj - 1, Ops<T>::add(dprev, Ops<T>::sub(D, Dprev)));
            Dprev = D;
        }
        dprev = d;
        s = sn;
    }
    put(NV - 1, Ops<T>::add(dprev, Ops<T>::sub(T(0), Dprev)));
}

// ---- flow ------------------------------------------------------------------------------------
__device__ __forceinline__ void sincospi_t(float y, float* s, float* c) { sincospif(y, s, c); }
__device__ __forceinline__ void sincospi_t(double y, double* s, double* c) { sincospi(y, s, c); }

template <typename T>
__device__ __forceinline__ const T* amp_ptr(const Step1DArgs& a, int par, int inst);
template <>
__device__ __forceinline__ const float* amp_ptr<float>(const Step1DArgs& a, int par, int inst) {
    return a.ampf + par * a.amp_stride + (long long)inst * 2 * a.nmodes;
}
template <>
__device__ __forceinline__ const double* amp_ptr<double>(const Step1DArgs& a, int par, int inst) {
    return a.amp + par * a.amp_stride + (long long)inst * 2 * a.nmodes;
}

// u(x_i, t_n) = sum_m A_m cos(2 pi k_m i / N_x) + B_m sin(2 pi k_m i / N_x); the phase is
// reduced in integers (k_m i mod N_x) and evaluated as sin/cos of pi * (2 (k_m i mod N_x)/N_x).
// Explicit rounding, so that every kernel variant gets the same bits whatever the compiler
// contracts around it.
template <typename T>
__device__ __forceinline__ T flow_at(const Step1DArgs& a, const Inst1D& in, const T* amp, int x) {
    if (a.flow_kind == LAT_FLOW_FIELD) return static_cast<const T*>(a.field)[in.xoff + x];
    if (a.flow_kind != LAT_FLOW_MODES) return T(0);
    using O = Ops<T>;
    const int M = a.nmodes;
    const T two_over_nx = T(in.two_over_nx);
    T u = T(0);
    for (int m = 0; m < M; ++m) {
        int kx = a.k[m] * x;
        kx = in.pow2 ? (kx & (in.nx - 1)) : (kx % in.nx);
        if (kx < 0) kx += in.nx;
        T s, c;
        sincospi_t(O::mul(T(kx), two_over_nx), &s, &c);
        u = O::add(u, O::fma(__ldg(amp + m), c, O::mul(__ldg(amp + M + m), s)));
    }
    return u;
}

// Exact Ornstein-Uhlenbeck update of the instance's amplitudes (Eq. A1d), t_n -> t_{n+1}.
__device__ __forceinline__ void advance_amplitudes(const Step1DArgs& a, int inst,
                                                   const Inst1D& in, long long step, int par) {
    const int M2 = 2 * a.nmodes;
    const long long row = step - a.st->noise_base;
    const bool have = row >= 0 && row < a.st->noise_rows;
    for (int t = threadIdx.x; t < M2; t += blockDim.x) {
        const double old = a.amp[par * a.amp_stride + (long long)inst * M2 + t];
        double xi = 0.0;
        if (have) xi = a.noise[row * a.amp_stride + (long long)inst * M2 + t];
        const double nw = __dadd_rn(__dmul_rn(old, in.ou_e), __dmul_rn(in.ou_s, xi));
        a.amp_w[(1 - par) * a.amp_stride + (long long)inst * M2 + t] = nw;
        a.ampf_w[(1 - par) * a.amp_stride + (long long)inst * M2 + t] = (float)nw;
    }
    if (!have && threadIdx.x == 0) atomicOr(&a.st->status, ST_NOISE);
}

template <typename T, int J, bool LIM = false>
__device__ __forceinline__ void cfl_flag(const Step1DArgs& a, T g, T w) {
    // Eq. (cfl); each stage of the limited scheme (LIM) is positive for nu (1 + mu) <= 1
    const T f = LIM ? T(1) + T(a.mu) : T(1);
    if (g * (T(J) + fabs(w)) * f > T(1)) atomicOr(&a.st->status, ST_CFL);
}

// ---- reg / any variants (plain loads) ----------------------------------------------------------
template <typename T, int NV>
struct MaxThreads {
    static constexpr int words = NV * (int)(sizeof(T) / 4);
    static constexpr int value = words > 56 ? 256 : (words > 20 ? 512 : 1024);
};

template <typename T, int NV, bool LIM>
__global__ void __launch_bounds__(MaxThreads<T, NV>::value)
    k_step1d_reg(const Step1DArgs a, const int kstep) {
    constexpr int J = (NV - 1) / 2;
    const long long step = a.st->step + kstep;
    const int par = (int)(step & 1);
    for (int it = a.item_begin + blockIdx.x; it < a.item_end; it += gridDim.x) {
        const int2 item = a.items[it];
        const Inst1D in = a.inst[item.x];
        const int nx = in.nx;
        const int x = item.y + threadIdx.x;
        if (x < nx) {
            const T g = T(in.g), r = T(in.r);
            const T* __restrict__ src = static_cast<const T*>(a.f[par]) + in.off;
            T* __restrict__ dst = static_cast<T*>(a.f[par ^ 1]) + in.off + x;
            const T w = flow_at<T>(a, in, amp_ptr<T>(a, par, item.x), x) * T(in.inv_dv);
            T f[NV];
            if (nx >= J) {
#pragma unroll
                for (int jj = 0; jj < NV; ++jj) {
                    int xs = x - (jj - J);
                    xs += (xs < 0) ? nx : 0;
                    xs -= (xs >= nx) ? nx : 0;
                    f[jj] = __ldg(src + (size_t)jj * nx + xs);
                }
            } else {
#pragma unroll
                for (int jj = 0; jj < NV; ++jj) {
                    int xs = (x - (jj - J)) % nx;
                    xs += (xs < 0) ? nx : 0;
                    f[jj] = __ldg(src + (size_t)jj * nx + xs);
                }
            }
            sweep_scheme<T, NV, LIM>(
                a, w, g, r, [&](int jj) { return f[jj]; },
                [&](int jj, T v) { dst[(size_t)jj * nx] = v; });
            cfl_flag<T, J, LIM>(a, g, w);
        }
        if (!a.dry && !a.frozen && a.flow_kind == LAT_FLOW_MODES && item.y == 0)
            advance_amplitudes(a, item.x, in, step, par);
    }
}

template <typename T>
__global__ void __launch_bounds__(512) k_step1d_any(const Step1DArgs a, const int kstep,
                                                    const int NV) {
    const int J = (NV - 1) / 2;
    const long long step = a.st->step + kstep;
    const int par = (int)(step & 1);
    for (int it = a.item_begin + blockIdx.x; it < a.item_end; it += gridDim.x) {
        const int2 item = a.items[it];
        const Inst1D in = a.inst[item.x];
        const int nx = in.nx;
        const int x = item.y + threadIdx.x;
        if (x < nx) {
            const T g = T(in.g), r = T(in.r);
            const T* __restrict__ src = static_cast<const T*>(a.f[par]) + in.off;
            T* __restrict__ dst = static_cast<T*>(a.f[par ^ 1]) + in.off + x;
            const T w = flow_at<T>(a, in, amp_ptr<T>(a, par, item.x), x) * T(in.inv_dv);
            sweep_column_any<T>(
                NV, w, g, r,
                [&](int jj) {
                    int xs = (x - (jj - J)) % nx;
                    xs += (xs < 0) ? nx : 0;
                    return __ldg(src + (size_t)jj * nx + xs);
                },
                [&](int jj, T v) { dst[(size_t)jj * nx] = v; });
            if (g * (T(J) + fabs(w)) > T(1)) atomicOr(&a.st->status, ST_CFL);
        }
        if (!a.dry && !a.frozen && a.flow_kind == LAT_FLOW_MODES && item.y == 0)
            advance_amplitudes(a, item.x, in, step, par);
    }
}

// ---- ring variant (FP32, bulk async copies into a shared-memory ring) --------------------------
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
// Bounded wait on an mbarrier phase: gives up after ~1 s (the caller raises ST_TIMEOUT).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (long long it = 0; it < (1ll << 26); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255) == 0 && globaltimer() - t0 > 1000000000ull) break;
    }
    return false;
}
__device__ __forceinline__ int wrapi(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

// Copy the N_v shifted windows of item `it` into ring slot `slot` (warp 0 only): plane j needs
// columns [x0 - j, x0 - j + 128); the window starts at that offset rounded down to 16 bytes and
// is split in two at the periodic wrap.
template <int NV>
__device__ __forceinline__ void issue_item(const Step1DArgs& a, const float* fin, float* ring,
                                           uint64_t* bar, int slot, int it) {
    constexpr int J = (NV - 1) / 2;
    const int lane = threadIdx.x & 31;
    if (lane == 0) mbar_expect_tx(&bar[slot], (unsigned)(NV * WIN1 * sizeof(float)));
    __syncwarp();
    const int2 item = a.items[it];
    const Inst1D& in = a.inst[item.x];
    const float* base_ptr = fin + in.off;
    for (int jj = lane; jj < NV; jj += 32) {
        const float* prow = base_ptr + (size_t)jj * in.nx;
        const int s = item.y - (jj - J);
        const int b = wrapi(s - ((s % 4) + 4) % 4, in.nx);
        float* dst = ring + ((size_t)slot * NV + jj) * WIN1;
        if (b + WIN1 <= in.nx) {
            bulk_g2s(dst, prow + b, WIN1 * sizeof(float), &bar[slot]);
        } else {
            const int n1 = in.nx - b;
            bulk_g2s(dst, prow + b, n1 * sizeof(float), &bar[slot]);
            bulk_g2s(dst + n1, prow, (WIN1 - n1) * sizeof(float), &bar[slot]);
        }
    }
}

template <int NV, int NS, bool LIM>
__global__ void __launch_bounds__(TW1) k_step1d_ring(const Step1DArgs a, const int kstep) {
    constexpr int J = (NV - 1) / 2;
    extern __shared__ __align__(128) unsigned char smem[];
    float* ring = reinterpret_cast<float*>(smem);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + (size_t)NS * NV * WIN1 * sizeof(float));
    const long long step = a.st->step + kstep;
    const int par = (int)(step & 1);
    const float* fin = static_cast<const float*>(a.f[par]);
    float* fout = static_cast<float*>(a.f[par ^ 1]);
    const int tid = threadIdx.x;
    const int first = a.item_begin + blockIdx.x;
    const int nloc = first < a.item_end ? (a.item_end - 1 - first) / gridDim.x + 1 : 0;
    if (tid == 0) {
        for (int q = 0; q < NS; ++q) mbar_init(&bar[q], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid < 32)
        for (int k = 0; k < NS - 1 && k < nloc; ++k)
            issue_item<NV>(a, fin, ring, bar, k % NS, first + k * gridDim.x);
    int issued = std::min(NS - 1, nloc);
    bool failed = false;
    for (int k = 0; k < nloc; ++k) {
        if (__syncthreads_or(failed ? 1 : 0)) {
            failed = true;
            break;
        }
        // slot (k + NS - 1) % NS held item k - 1, which every thread has finished
        if (k + NS - 1 < nloc) {
            if (tid < 32) {
#if LAT_RING_PROXY_FENCE
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
#endif
                issue_item<NV>(a, fin, ring, bar, (k + NS - 1) % NS,
                               first + (k + NS - 1) * gridDim.x);
            }
            issued = k + NS;
        }
        const int it = first + k * gridDim.x;
        const int2 item = a.items[it];
        const Inst1D in = a.inst[item.x];
        const int x = item.y + tid;
        const float g = float(in.g), r = float(in.r);
        float w = 0.f;
        if (x < in.nx) w = flow_at<float>(a, in, amp_ptr<float>(a, par, item.x), x) * float(in.inv_dv);
        if (!mbar_wait_bounded(&bar[k % NS], (unsigned)((k / NS) & 1))) {
            failed = true;
            continue;
        }
        if (x < in.nx) {
            const float* col = ring + (size_t)(k % NS) * NV * WIN1 + tid;
            float* dst = fout + in.off + x;
            const int nx = in.nx;
            sweep_scheme<float, NV, LIM>(
                a, w, g, r,
                [&](int jj) { return col[jj * WIN1 + ((J - jj) % 4 + 4) % 4]; },
                [&](int jj, float v) { dst[(size_t)jj * nx] = v; });
            cfl_flag<float, J, LIM>(a, g, w);
        }
        if (!a.dry && !a.frozen && a.flow_kind == LAT_FLOW_MODES && item.y == 0)
            advance_amplitudes(a, item.x, in, step, par);
    }
    if (failed) {
        if (tid == 0) {
            atomicOr(&a.st->status, ST_TIMEOUT);
            // let the copies already issued land before the block's shared memory goes away
            for (int k = std::max(0, issued - NS); k < issued; ++k)
                mbar_wait_bounded(&bar[k % NS], (unsigned)((k / NS) & 1));
        }
        __syncthreads();
    }
}

// ---- producer/consumer variant: no block-wide barrier per item -------------------------------
// Four consumer warps own the 128 columns of an item; a fifth warp only produces: it refills a
// ring slot with the next item's plane windows once every consumer warp has released the slot
// (per-slot "empty" mbarrier, one arrival per consumer warp).  Consumers wait only on the
// per-slot "full" mbarrier that the bulk copies complete, so warps drift freely.
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

constexpr int PC1_CONSUMERS = TW1 / 32;
constexpr int PC1_THREADS = 32 * (PC1_CONSUMERS + 1);

template <int NV, int NS>
size_t pc1d_smem() {
    return (size_t)NS * NV * WIN1 * sizeof(float) + 2 * NS * sizeof(uint64_t);
}

// With MOM the consumers also reduce the moments of the columns they write (the same FP32
// column sums, in the same order, as the moment kernel; compensated across cells).
template <int NV, int NS, bool MOM, bool LIM>
__global__ void __launch_bounds__(PC1_THREADS) k_step1d_pc(const Step1DArgs a, const int kstep) {
    constexpr int J = (NV - 1) / 2;
    extern __shared__ __align__(128) unsigned char smem[];
    float* ring = reinterpret_cast<float*>(smem);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)NS * NV * WIN1 * sizeof(float));
    uint64_t* empty = full + NS;
    const long long step = a.st->step + kstep;
    const int par = (int)(step & 1);
    const float* fin = static_cast<const float*>(a.f[par]);
    float* fout = static_cast<float*>(a.f[par ^ 1]);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int first = a.item_begin + blockIdx.x;
    const int nloc = first < a.item_end ? (a.item_end - 1 - first) / gridDim.x + 1 : 0;
    if (threadIdx.x == 0) {
        for (int q = 0; q < NS; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], PC1_CONSUMERS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (warp == PC1_CONSUMERS) {
        // a stalled context issues no copies: every consumer's bounded wait runs out
        const int nfill = a.st->stall ? 0 : nloc;
        int k = 0;
        for (; k < nfill; ++k) {
            const int q = k % NS;
            if (k >= NS && !mbar_wait_bounded(&empty[q], (unsigned)(((k / NS) + 1) & 1))) {
                if (lane == 0) atomicOr(&a.st->status, ST_TIMEOUT);
                break;
            }
            issue_item<NV>(a, fin, ring, full, q, first + k * gridDim.x);
        }
        // the copies issued last must land before this warp leaves
        for (int d = std::max(0, k - NS); d < k; ++d)
            mbar_wait_bounded(&full[d % NS], (unsigned)((d / NS) & 1));
        return;
    }
    const int tid = threadIdx.x;
    for (int k = 0; k < nloc; ++k) {
        const int it = first + k * gridDim.x;
        const int2 item = a.items[it];
        const Inst1D in = a.inst[item.x];
        const int x = item.y + tid;
        const float g = float(in.g), r = float(in.r);
        float w = 0.f;
        if (x < in.nx) w = flow_at<float>(a, in, amp_ptr<float>(a, par, item.x), x) * float(in.inv_dv);
        if (!mbar_wait_bounded(&full[k % NS], (unsigned)((k / NS) & 1))) {
            if (lane == 0) atomicOr(&a.st->status, ST_TIMEOUT);
            break;
        }
        cs::ColumnSums sums;
        if (x < in.nx) {
            const float* col = ring + (size_t)(k % NS) * NV * WIN1 + tid;
            float* dst = fout + in.off + x;
            const int nx = in.nx;
            auto get = [&](int jj) { return col[jj * WIN1 + ((J - jj) % 4 + 4) % 4]; };
            if constexpr (!LIM && NV >= 5) {
                // packed two-lane sweep; the moments in ColumnSums2 order (lane 0: cells
                // 0 .. J - 1, lane 1: J .. 2J), the order of the moment kernel
                cs::ColumnSums2 s2;
                const f2 one2 = pk(1.f, 1.f);
                f2 jv = pk(float(-J), 0.f);
                sweep_column2<NV>(
                    w, g, r, get,
                    [&](int p, f2 o) {
                        dst[(size_t)(p - 1) * nx] = lo(o);
                        dst[(size_t)(p - 1 + J) * nx] = hi(o);
                        if constexpr (MOM) {
                            s2.add(jv, mul2(jv, jv), o);
                            jv = add2(jv, one2);
                        }
                    },
                    [&](float v) {
                        dst[(size_t)(NV - 1) * nx] = v;
                        if constexpr (MOM) s2.add_hi(float(J), v);
                    });
                if constexpr (MOM) sums = s2.collapse();
            } else {
                cs::ColumnSums2 s2;
                sweep_scheme<float, NV, LIM>(a, w, g, r, get, [&](int jj, float v) {
                    dst[(size_t)jj * nx] = v;
                    if constexpr (MOM) {
                        if (jj < J) s2.add_lo((float)(jj - J), v);
                        else s2.add_hi((float)(jj - J), v);
                    }
                });
                if constexpr (MOM) sums = s2.collapse();
            }
            cfl_flag<float, J, LIM>(a, g, w);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[k % NS]);
        if constexpr (MOM) {  // same per-warp partials as the moment kernel with 128 columns
            if (x < in.nx) {
                if (!isfinite(sums.a0.s) || !isfinite(sums.b2))
                    atomicOr(&a.st->status, ST_NUMERIC);
                // per-cell moments in FP64 only when asked for (FP64 is slow here)
                if (a.m_rho || a.m_mv || a.m_mv2) {
                    cs::Comp t0, t1, t2;
                    sums.result(in.dv, t0, t1, t2);
                    const double m0 = cs::nval(t0), m1 = cs::nval(t1), m2 = cs::nval(t2);
                    const long long cell = in.xoff + x;
                    if (a.m_rho) a.m_rho[cell] = m0 * in.dv;
                    if (a.m_mv) a.m_mv[cell] = (m0 != 0.0) ? m1 / m0 : 0.0;
                    if (a.m_mv2) a.m_mv2[cell] = (m0 != 0.0) ? m2 / m0 : 0.0;
                }
            }
            cs::warp_partial_1d(sums, in.dv,
                                a.m_partials + ((size_t)it * PC1_CONSUMERS + warp) * 6);
        }
        if (!a.dry && !a.frozen && a.flow_kind == LAT_FLOW_MODES && item.y == 0)
            advance_amplitudes(a, item.x, in, step, par);
    }
}

__global__ void k_advance_step(DevState* st, long long n) { st->step += n; }

template <int NV, int NS, bool MOM, bool LIM>
cudaError_t launch_pc1_t(int grid, const Step1DArgs& a, int kstep, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_step1d_pc<NV, NS, MOM, LIM>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)pc1d_smem<NV, NS>());
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_step1d_pc<NV, NS, MOM, LIM><<<grid, PC1_THREADS, pc1d_smem<NV, NS>(), s>>>(a, kstep);
    return cudaGetLastError();
}

// the scheme's instance of the kernel
template <int NV, int NS, bool MOM = false>
cudaError_t launch_pc1(int grid, const Step1DArgs& a, int kstep, cudaStream_t s) {
    if (a.scheme == LAT_SCHEME_KOREN) return launch_pc1_t<NV, NS, MOM, true>(grid, a, kstep, s);
    return launch_pc1_t<NV, NS, MOM, false>(grid, a, kstep, s);
}

// Occupancy of the upwind instance; the limited one holds the same shared memory, which is what
// limits the resident blocks.
template <int NV, int NS>
int occupancy_pc1() {
    int nb = 0;
    cudaFuncSetAttribute(k_step1d_pc<NV, NS, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)pc1d_smem<NV, NS>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step1d_pc<NV, NS, false, false>, PC1_THREADS,
                                                  pc1d_smem<NV, NS>());
    return nb;
}

template <int NV, int NS>
size_t ring1d_smem() {
    return (size_t)NS * NV * WIN1 * sizeof(float) + NS * sizeof(uint64_t);
}

template <int NV, int NS, bool LIM>
cudaError_t launch_ring_t(int grid, const Step1DArgs& a, int kstep, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_step1d_ring<NV, NS, LIM>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)ring1d_smem<NV, NS>());
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_step1d_ring<NV, NS, LIM><<<grid, TW1, ring1d_smem<NV, NS>(), s>>>(a, kstep);
    return cudaGetLastError();
}

template <int NV, int NS>
cudaError_t launch_ring(int grid, const Step1DArgs& a, int kstep, cudaStream_t s) {
    if (a.scheme == LAT_SCHEME_KOREN) return launch_ring_t<NV, NS, true>(grid, a, kstep, s);
    return launch_ring_t<NV, NS, false>(grid, a, kstep, s);
}

template <int NV, int NS>
int occupancy_ring() {
    int nb = 0;
    cudaFuncSetAttribute(k_step1d_ring<NV, NS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)ring1d_smem<NV, NS>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step1d_ring<NV, NS, false>, TW1,
                                                  ring1d_smem<NV, NS>());
    return nb;
}

template <typename T, int NV>
cudaError_t launch_reg(int block, int grid, const Step1DArgs& a, int kstep, cudaStream_t s) {
    if (block > MaxThreads<T, NV>::value) return cudaErrorInvalidValue;
    if (a.scheme == LAT_SCHEME_KOREN) k_step1d_reg<T, NV, true><<<grid, block, 0, s>>>(a, kstep);
    else k_step1d_reg<T, NV, false><<<grid, block, 0, s>>>(a, kstep);
    return cudaGetLastError();
}

#define LAT1D_NV_LIST(X) X(3) X(5) X(9) X(17) X(33) X(65)


template <typename T>
cudaError_t launch_plain(int nv, int block, int grid, const Step1DArgs& a, int kstep,
                         cudaStream_t s) {
    switch (nv) {
#define X(n) \
    case n: return launch_reg<T, n>(block, grid, a, kstep, s);
        LAT1D_NV_LIST(X)
#undef X
        default:
            if (block > 512) return cudaErrorInvalidValue;
            k_step1d_any<T><<<grid, block, 0, s>>>(a, kstep, nv);
            return cudaGetLastError();
    }
}

}  // namespace

int step1d_max_block(int dtype, int nv, int variant) {
    if (variant == STEP1D_RING || variant == STEP1D_PC) return TW1;
    bool reg = false;
#define X(n) reg |= nv == n;
    LAT1D_NV_LIST(X)
#undef X
    if (!reg) return 512;
    const int words = nv * (dtype == LAT_F64 ? 2 : 1);
    return words > 56 ? 256 : (words > 20 ? 512 : 1024);
}

// The limited scheme runs in the compiled-N_v kernels only (not k_step1d_any).
bool step1d_limiter_supported(int nv) {
    switch (nv) {
#define X(n) case n:
        LAT1D_NV_LIST(X)
#undef X
        return true;
        default: return false;
    }
}

bool step1d_ring_supported(int dtype, int nv) {
    if (dtype != LAT_F32) return false;
    bool ok = false;
#define X(n) ok |= nv == n;
    LAT1D_NV_LIST(X)
#undef X
    return ok;
}

int step1d_ring_tile() { return TW1; }
int step1d_ring_min_nx() { return WIN1; }

int step1d_ring_occupancy(int nv, int slots, int variant) {
    switch (nv) {
#define X(n)                                                                    \
    case n:                                                                     \
        if (variant == STEP1D_PC) {                                             \
            if (slots == 2) return occupancy_pc1<n, 2>();                       \
            if (slots == 3) return occupancy_pc1<n, 3>();                       \
            return occupancy_pc1<n, 4>();                                       \
        }                                                                       \
        if (slots == 2) return occupancy_ring<n, 2>();                          \
        if (slots == 3) return occupancy_ring<n, 3>();                          \
        return occupancy_ring<n, 4>();
        LAT1D_NV_LIST(X)
#undef X
        default: return 0;
    }
}

// the fused epilogue reduces in the two-lane order of ColumnSums2 (N_v >= 5)
bool step1d_moments_supported(int dtype, int nv) {
    return nv >= 5 && step1d_ring_supported(dtype, nv);
}

cudaError_t launch_step1d_moments(int nv, int grid, const Step1DArgs& a, cudaStream_t s) {
    if (grid <= 0) return cudaSuccess;
    switch (nv) {
#define X(n) \
    case n: return launch_pc1<n, 2, true>(grid, a, 0, s);
        LAT1D_NV_LIST(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step1d(int dtype, int nv, int variant, int block, int slots, int grid,
                          const Step1DArgs& a, int kstep, cudaStream_t s) {
    if (grid <= 0) return cudaSuccess;
    if (variant == STEP1D_PC) {
        if (dtype != LAT_F32 || block != TW1) return cudaErrorInvalidValue;
        switch (nv) {
#define X(n)                                                         \
    case n:                                                          \
        if (slots == 2) return launch_pc1<n, 2>(grid, a, kstep, s);  \
        if (slots == 3) return launch_pc1<n, 3>(grid, a, kstep, s);  \
        if (slots == 4) return launch_pc1<n, 4>(grid, a, kstep, s);  \
        return cudaErrorInvalidValue;
            LAT1D_NV_LIST(X)
#undef X
            default: return cudaErrorInvalidValue;
        }
    }
    if (variant == STEP1D_RING) {
        if (dtype != LAT_F32 || block != TW1) return cudaErrorInvalidValue;
        switch (nv) {
#define X(n)                                                         \
    case n:                                                          \
        if (slots == 2) return launch_ring<n, 2>(grid, a, kstep, s); \
        if (slots == 3) return launch_ring<n, 3>(grid, a, kstep, s); \
        if (slots == 4) return launch_ring<n, 4>(grid, a, kstep, s); \
        return cudaErrorInvalidValue;
            LAT1D_NV_LIST(X)
#undef X
            default: return cudaErrorInvalidValue;
        }
    }
    if (dtype == LAT_F32) return launch_plain<float>(nv, block, grid, a, kstep, s);
    if (dtype == LAT_F64) return launch_plain<double>(nv, block, grid, a, kstep, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_advance_step(DevState* st, long long n, cudaStream_t s) {
    k_advance_step<<<1, 1, 0, s>>>(st, n);
    return cudaGetLastError();
}

}  // namespace lat

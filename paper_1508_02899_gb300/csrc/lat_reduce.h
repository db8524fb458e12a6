// Compensated summation helpers shared by the moment reductions (device code only).
#pragma once

#include <cuda_runtime.h>

#include "f32x2.h"

namespace lat {
namespace cs {

// FP64 value with a Neumaier compensation term: the sum is s + c.
struct Comp {
    double s, c;
};

// Neumaier's compensated addition.
__device__ __forceinline__ void nadd(Comp& a, double x) {
    const double t = __dadd_rn(a.s, x);
    if (fabs(a.s) >= fabs(x)) a.c = __dadd_rn(a.c, __dadd_rn(__dsub_rn(a.s, t), x));
    else a.c = __dadd_rn(a.c, __dadd_rn(__dsub_rn(x, t), a.s));
    a.s = t;
}
__device__ __forceinline__ void nmerge(Comp& a, const Comp& b) {
    nadd(a, b.s);
    a.c = __dadd_rn(a.c, b.c);
}
__device__ __forceinline__ double nval(const Comp& a) { return __dadd_rn(a.s, a.c); }

__device__ __forceinline__ Comp shfl_down(const Comp& a, int off) {
    return Comp{__shfl_down_sync(0xffffffffu, a.s, off), __shfl_down_sync(0xffffffffu, a.c, off)};
}
__device__ __forceinline__ Comp shfl_up(const Comp& a, int off) {
    return Comp{__shfl_up_sync(0xffffffffu, a.s, off), __shfl_up_sync(0xffffffffu, a.c, off)};
}

// Kahan-compensated FP32 accumulator (c holds the negated running error: the sum is s - c).
struct FComp {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float y = __fsub_rn(x, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    // s + x by Knuth's branch-free TwoSum (t + e = s + x exactly), e folded into c: unlike add(),
    // no rounding of x is lost, so s - c keeps the sum to the roundings of c (about n u^2 of the
    // sum after n terms) where Kahan's add() can lose up to about 2u.
    __device__ __forceinline__ void add_exact(float x) {
        const float t = __fadd_rn(s, x);
        const float bb = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(x, bb));
        s = t;
        c = __fsub_rn(c, e);
    }
    // (s - c) + (o.s - o.c): s + o.s by Knuth's branch-free TwoSum (t + e exactly, whatever the
    // magnitudes), then both error terms and e fold into c.  Only the rounding of c is lost,
    // about u^2 of the partial sums per merge (u = 2^-24).
    __device__ __forceinline__ void merge(const FComp& o) {
        const float t = __fadd_rn(s, o.s);
        const float bb = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(o.s, bb));
        s = t;
        c = __fsub_rn(__fadd_rn(c, o.c), e);
    }
    __device__ __forceinline__ Comp to_comp(double scale) const {
        return Comp{__dmul_rn((double)s, scale), -__dmul_rn((double)c, scale)};
    }
};

__device__ __forceinline__ FComp shfl_down(const FComp& a, int off) {
    FComp r;
    r.s = __shfl_down_sync(0xffffffffu, a.s, off);
    r.c = __shfl_down_sync(0xffffffffu, a.c, off);
    return r;
}

// Butterfly reduction of an FP32 compensated sum over a warp, in a fixed order (lane 0).
__device__ __forceinline__ void warp_reduce(FComp& t) {
    for (int off = 16; off > 0; off >>= 1) t.merge(shfl_down(t, off));
}
__device__ __forceinline__ void warp_reduce(Comp& t) {
    for (int off = 16; off > 0; off >>= 1) nmerge(t, shfl_down(t, off));
}

// Column sums of one 1D column [sum f, sum j f, sum j^2 f] in FP32, returned as FP64
// compensated values scaled to [M0, M1 = sum v f, M2 = sum v^2 f] / dv.  The mass sum is exact
// up to the roundings of its compensation term (TwoSum, add_exact).  The two weighted sums take
// one FMA per value (the product j f or j^2 f exact inside it, one rounding of the running
// sum): error at most (N_v - 1) u of sum |j^k f| (u = 2^-24), the accuracy of the FP32 state
// itself, at far fewer instructions than compensating them too.
struct ColumnSums {
    FComp a0;
    float b1 = 0.f, b2 = 0.f;
    __device__ __forceinline__ void add(float j, float fv) {
        a0.add_exact(fv);
        b1 = __fmaf_rn(j, fv, b1);
        b2 = __fmaf_rn(j * j, fv, b2);
    }
    __device__ __forceinline__ FComp a1() const { return FComp{b1, 0.f}; }
    __device__ __forceinline__ FComp a2() const { return FComp{b2, 0.f}; }
    __device__ __forceinline__ void result(double dv, Comp& s0, Comp& s1, Comp& s2) const {
        const double dv2 = __dmul_rn(dv, dv);
        s0 = Comp{(double)a0.s, -(double)a0.c};
        s1 = Comp{__dmul_rn((double)b1, dv), 0.0};
        s2 = Comp{__dmul_rn((double)b2, dv2), 0.0};
    }
};

// The column sums of ColumnSums over two half-columns at once, one per f32x2 lane (the packed
// 1D sweep's lanes): lane 0 takes the column's values 0 .. h - 1 and lane 1 the values h .. 2h,
// each in ascending order; collapse() merges lane 1 into lane 0 (FComp merge for the mass, one
// addition for each weighted sum).  Every FP32 column reduction of the library that must give
// the bits of another uses this order.
struct ColumnSums2 {
    f2 s = 0ull, c = 0ull, b1 = 0ull, b2 = 0ull;
    // v: the two lanes' values; j, jsq: their velocity indices and squares (exact)
    __device__ __forceinline__ void add(f2 j, f2 jsq, f2 v) {
        const f2 t = add2(s, v);
        const f2 bb = sub2(t, s);
        const f2 e = add2(sub2(s, sub2(t, bb)), sub2(v, bb));
        s = t;
        c = sub2(c, e);
        b1 = fma2(j, v, b1);
        b2 = fma2(jsq, v, b2);
    }
    // lane 0 alone
    __device__ __forceinline__ void add_lo(float j, float v) {
        FComp a{lo(s), lo(c)};
        a.add_exact(v);
        s = pk(a.s, hi(s));
        c = pk(a.c, hi(c));
        b1 = pk(__fmaf_rn(j, v, lo(b1)), hi(b1));
        b2 = pk(__fmaf_rn(__fmul_rn(j, j), v, lo(b2)), hi(b2));
    }
    // lane 1 alone
    __device__ __forceinline__ void add_hi(float j, float v) {
        FComp a{hi(s), hi(c)};
        a.add_exact(v);
        s = pk(lo(s), a.s);
        c = pk(lo(c), a.c);
        b1 = pk(lo(b1), __fmaf_rn(j, v, hi(b1)));
        b2 = pk(lo(b2), __fmaf_rn(__fmul_rn(j, j), v, hi(b2)));
    }
    __device__ __forceinline__ ColumnSums collapse() const {
        ColumnSums r;
        r.a0 = FComp{lo(s), lo(c)};
        r.a0.merge(FComp{hi(s), hi(c)});
        r.b1 = __fadd_rn(lo(b1), hi(b1));
        r.b2 = __fadd_rn(lo(b2), hi(b2));
        return r;
    }
};

// Butterfly reduction of three compensated sums over a warp (result in lane 0).
__device__ __forceinline__ void warp_reduce3(Comp& t0, Comp& t1, Comp& t2) {
    for (int off = 16; off > 0; off >>= 1) {
        Comp o0 = shfl_down(t0, off), o1 = shfl_down(t1, off), o2 = shfl_down(t2, off);
        nmerge(t0, o0);
        nmerge(t1, o1);
        nmerge(t2, o2);
    }
}

// Per-warp partial of the 1D moments of FP32 columns: every lane holds the column sums of its
// column (zero for an inactive lane); lane 0 writes [M, P, E] (sum, compensation) scaled to
// [1, dv, dv^2] at p.  The cross-column part stays in FP32 Kahan form (FP64 is slow here).
__device__ __forceinline__ void warp_partial_1d(const ColumnSums& cs_, double dv, double* p) {
    FComp a0 = cs_.a0, a1 = cs_.a1(), a2 = cs_.a2();
    warp_reduce(a0);
    warp_reduce(a1);
    warp_reduce(a2);
    if ((threadIdx.x & 31) == 0) {
        const Comp t0 = a0.to_comp(1.0), t1 = a1.to_comp(dv), t2 = a2.to_comp(__dmul_rn(dv, dv));
        p[0] = t0.s; p[1] = t0.c;
        p[2] = t1.s; p[3] = t1.c;
        p[4] = t2.s; p[5] = t2.c;
    }
}

}  // namespace cs
}  // namespace lat

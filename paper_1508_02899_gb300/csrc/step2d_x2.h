// Packed two-lane form of the 2D velocity-row sweep (step2d_dev.h) for FP32 arithmetic.
//
// A thread still owns one spatial cell and sweeps its velocity column row by row, but holds a
// velocity row as two half-rows in the two 32-bit lanes of 64-bit register pairs: for
// N_v = 2h + 1, pair p (p = 0..h) carries column p in lane 0 and column p + h in lane 1.  Column h
// is in both lanes (lane 0 at p = h, lane 1 at p = 0); the two copies see the same inputs and
// give the same bits, and lane 1's copy is never stored.  The packed add/sub/mul/fma.rn.f32x2
// instructions do the arithmetic of both half-rows at once; every lane performs exactly the
// operations of sweep_row, in the same order and with the same rounding, so a packed kernel
// writes the same bits as the scalar ones.  The two lanes meet only at the seam: the x-drag and
// x-diffusion fluxes through faces h - 1/2 (entering lane 1) and h + 1/2 (leaving lane 0), which
// are formed from the other lane's values read at the start of the row.
#pragma once

#include "f32x2.h"
#include "step2d_dev.h"

namespace lat {
namespace k2d {

template <int NV>
struct Pairs {
    static constexpr int h = (NV - 1) / 2;  // = J
    static constexpr int n = h + 1;         // pairs per row
};

// Per-thread column of pairs in a [n][TW] shared array.
struct SmemCol2 {
    f2* p;
    __device__ __forceinline__ f2& operator[](int i) const { return p[i * TW]; }
};

// Row r of the sweep (1..NV), as sweep_row: f** of row r - 1 from f* rows r - 1 (cur) and r
// (nxt, absent when r == NV); for r >= 2 output row r - 2 goes to put(p, o2) for p = 0..h after
// put.begin(r - 2).  A, Hd: f** of the previous row and the vy-diffusion flux below it (pairs);
// G: vy-drag flux below the current row (pairs, registers or SmemCol2).
template <int NV, class Row, class GArr, class Put>
__device__ __forceinline__ void sweep_row2(f2 (&A)[Pairs<NV>::n], GArr& G,
                                           f2 (&Hd)[Pairs<NV>::n], int r, const Row& cur,
                                           const Row& nxt_row, float g_in, float wx_in,
                                           float wy, float rr, Put& put) {
    constexpr int J = (NV - 1) / 2, h = Pairs<NV>::h;
    const int rb = r - 1;
    const bool nxt = r < NV;
    const float g = opaque(g_in), wx = opaque(wx_in);
    const float ayp = fmaxf(cacc<float>(g, wy, rb - J), 0.f);
    const float aym = nxt ? fminf(cacc<float>(g, wy, r - J), 0.f) : 0.f;
    const f2 g2 = pk(g, g), wx2 = pk(wx, wx), rr2 = pk(rr, rr);
    const f2 ayp2 = pk(ayp, ayp), aym2 = pk(aym, aym);
    const f2 one2 = opaque2(pk(1.f, 1.f));
    f2 kk = opaque2(pk(float(-J), 0.f));  // velocity indices of pair p: (p - J, p)
    f2 cac = mul2(g2, sub2(wx2, kk));      // c a of the pair's columns
    f2 sc = pk(cur.get(0), cur.get(h));
    // seam: flux through face h - 1/2 entering lane 1's first column (column h)
    const float fhm = cur.get(h - 1);
    const float cahm = cacc<float>(g, wx, -1);
    f2 Fp = pk(0.f, dflux<float>(cahm, cacc<float>(g, wx, 0), fhm, hi(sc)));
    // seam of the diffusion: f** of columns h - 1, h, h + 1 in the previous row
    const float Ahm = lo(A[h - 1]), Ah = hi(A[0]), Ahp = hi(A[1]);
    f2 Dp = pk(0.f, Ops<float>::mul(rr, Ops<float>::sub(Ah, Ahm)));
    put.begin(r >= 2 ? r - 2 : 0);
#pragma unroll
    for (int p = 0; p <= h; ++p) {
        const f2 kn = add2(kk, one2);
        const f2 can = mul2(g2, sub2(wx2, kn));
        const f2 sn = p < h ? pk(cur.get(p + 1), cur.get(p + 1 + h)) : pk(cur.get(h + 1), 0.f);
        f2 Fn = fma2(max0(cac), sc, mul2(min0(can), sn));
        if (p == h) Fn = pk(lo(Fn), 0.f);  // lane 1 reached the wall
        const f2 Gn = nxt ? fma2(ayp2, sc, mul2(aym2, pk(nxt_row.get(p), nxt_row.get(p + h))))
                          : pk(0.f, 0.f);
        const f2 b = sub2(sub2(sc, sub2(Fn, Fp)), sub2(Gn, G[p]));
        G[p] = Gn;
        Fp = Fn;
        sc = sn;
        cac = can;
        kk = kn;
        if (r >= 2) {
            const f2 a = A[p];
            f2 Dn;
            if (p < h) Dn = mul2(rr2, sub2(A[p + 1], a));
            else Dn = pk(Ops<float>::mul(rr, Ops<float>::sub(Ahp, lo(a))), 0.f);
            const f2 Hn = mul2(rr2, sub2(b, a));
            const f2 o = add2(add2(a, sub2(Dn, Dp)), sub2(Hn, Hd[p]));
            Hd[p] = Hn;
            Dp = Dn;
            put(p, o);
        }
        A[p] = b;
    }
}

// Last output row (jy = J), as final_row.
template <int NV, class Put>
__device__ __forceinline__ void final_row2(f2 (&A)[Pairs<NV>::n], f2 (&Hd)[Pairs<NV>::n],
                                           float rr, Put& put) {
    constexpr int h = Pairs<NV>::h;
    const f2 rr2 = pk(rr, rr), z2 = pk(0.f, 0.f);
    const float Ahm = lo(A[h - 1]), Ah = hi(A[0]), Ahp = hi(A[1]);
    f2 Dp = pk(0.f, Ops<float>::mul(rr, Ops<float>::sub(Ah, Ahm)));
    put.begin(NV - 1);
#pragma unroll
    for (int p = 0; p <= h; ++p) {
        const f2 a = A[p];
        f2 Dn;
        if (p < h) Dn = mul2(rr2, sub2(A[p + 1], a));
        else Dn = pk(Ops<float>::mul(rr, Ops<float>::sub(Ahp, lo(a))), 0.f);
        const f2 o = add2(add2(a, sub2(Dn, Dp)), sub2(z2, Hd[p]));
        Dp = Dn;
        put(p, o);
    }
}

// Stores of a packed sweep: lane 0 of pair p to plane (row, p), lane 1 to plane (row, p + h),
// except lane 1 of pair 0 (the second copy of column h).
template <int NV>
struct StorePut2 {
    static constexpr int h = Pairs<NV>::h;
    float* out;
    size_t pstride;
    bool active;
    float* p0;
    float* p1;
    __device__ __forceinline__ StorePut2(float* out_, size_t ps, bool act)
        : out(out_), pstride(ps), active(act), p0(out_), p1(out_) {}
    __device__ __forceinline__ void begin(int row) {
        p0 = out + (size_t)row * NV * pstride;
        p1 = p0 + (size_t)h * pstride;
    }
    __device__ __forceinline__ void operator()(int p, f2 o) {
        if (active) {
            *p0 = lo(o);
            if (p > 0) *p1 = hi(o);
        }
        p0 = next_plane(p0, pstride);
        p1 = next_plane(p1, pstride);
    }
};

}  // namespace k2d
}  // namespace lat

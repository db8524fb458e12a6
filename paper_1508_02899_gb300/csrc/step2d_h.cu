// Reduced-precision storage of the 2D lattice: FP16 or BF16 values with one power-of-two scale
// per x-line, FP32 arithmetic.  Every step decodes f* = h * S_in, runs the same column arithmetic
// as the FP32 kernels (stream, unsplit upwind drag, five-point velocity diffusion; Section 2),
// and encodes the result with the output line's scale S_out.
//
// Scales.  Under the CFL condition of the unsplit drag (g (J + |w_x|) + g (J + |w_y|) <= 1) and
// 4 r <= 1, f** is a combination of f* at the cell and its four velocity neighbours with
// non-negative weights summing to at most 3, and the diffusion output a combination of f** over
// the same stencil with weights summing to at most 1.  So an output value is at most 3 times the
// largest input value on the 13-cell velocity diamond |djx| + |djy| <= 2 around it, and that
// input value lies on line (jx', jy', y - (jy' - J)) of the input.  k_scale2d takes the maxima
// of those input lines, B, and sets S_out = 2^(ilogb(B) - 12): every encoded output value is
// below 3 * 2^13 = 24576, inside FP16's range (65504), and FP16 stays normal down to 2^-27 of B.
// A value that still exceeds the format's range (CFL broken, or non-finite input) raises
// ST_OVERFLOW.
//
// Error feedback.  Each thread owns one spatial cell's whole velocity column and encodes it in
// (jy, jx) order; the rounding residual of each value, t - decode(encode(t)), is carried into
// the next value.  A value takes at most kCarryLim * S_out of the carry (2^14 in FP16, so that
// |code| < 24576 + 16384 even next to a line 2^14 times larger); the rest stays in the carry.
// The stored column sum then equals the FP32 column sum up to the carry left after the corner
// velocity cell, so the reduced-precision store does not drift the mass: the mass drift stays
// at the level of the FP32 arithmetic.
//
// Line maxima.  Every step records max |stored value| per output line.  The plain kernel takes a
// warp maximum (redux) per value and a global atomicMax per warp.  After the producer/consumer
// kernel, k_linemax_step reads the stored output once more (2 bytes per cell) and reduces each
// line; with |h S| = |h| S exactly for a power-of-two S, both give the same bits, and the
// separate pass costs a fraction of the in-sweep reduction.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "step2d_h.h"

namespace lat {
namespace {

using namespace k2d;

template <typename S>
struct HTraits;
template <>
struct HTraits<__half> {
    static __device__ __forceinline__ float dec(__half h) { return __half2float(h); }
    static __device__ __forceinline__ __half enc(float q) { return __float2half_rn(q); }
    static constexpr float kMax = 65504.f;
    static constexpr float kCarryLim = 16384.f;  // 2^14
};
template <>
struct HTraits<__nv_bfloat16> {
    static __device__ __forceinline__ float dec(__nv_bfloat16 h) { return __bfloat162float(h); }
    static __device__ __forceinline__ __nv_bfloat16 enc(float q) { return __float2bfloat16_rn(q); }
    static constexpr float kMax = 3.38953139e38f;
    static constexpr float kCarryLim = 1.2676506e30f;  // 2^100
};

// 2^-E from 2^E, for the normal exponents the scales use (|E| <= 120).
__device__ __forceinline__ float pow2_inv(float s) {
    return __int_as_float((254 << 23) - __float_as_int(s));
}

constexpr int kScaleDrop = 12;  // S = 2^(ilogb(bound) - kScaleDrop)

// Scale for lines bounded by the non-negative float with bits m (0: S = 1).
__device__ __forceinline__ float scale_for(unsigned m) {
    if (m == 0u || m >= 0x7f800000u) return 1.f;
    int E = (int)(m >> 23) - 127 - kScaleDrop;
    E = E < -120 ? -120 : (E > 120 ? 120 : E);
    return __int_as_float((E + 127) << 23);
}

// ---- output scales of one step --------------------------------------------------------------
template <int NV>
__global__ void __launch_bounds__(256) k_scale2d(const Step2DHArgs a, int kstep) {
    constexpr int J = (NV - 1) / 2;
    const long long step = a.b.st->step + kstep;
    const int par = (int)(step & 1);
    const unsigned* mxi = (par ? a.mx[1] : a.mx[0]);
    float* so = (par ? a.sc[0] : a.sc[1]);
    unsigned* mxo = (par ? a.mx[0] : a.mx[1]);
    constexpr int NVP = nv_padded(NV);
    const int ny = a.b.ny;
    const long long nl = (long long)ny * NV * NVP;
    unsigned flags = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nl;
         i += (long long)gridDim.x * blockDim.x) {
        const int jx = (int)(i % NVP);
        const int jy = (int)((i / NVP) % NV);
        const int y = (int)(i / ((long long)NVP * NV));
        if (jx >= NV) {  // padding
            so[i] = 1.f;
            mxo[i] = 0u;
            continue;
        }
        unsigned m = 0;
        for (int dy = -2; dy <= 2; ++dy) {
            const int jy2 = jy + dy;
            if (jy2 < 0 || jy2 >= NV) continue;
            const int ys = wrap(y - (jy2 - J), ny);
            const int rx = 2 - (dy < 0 ? -dy : dy);
            for (int dx = -rx; dx <= rx; ++dx) {
                const int jx2 = jx + dx;
                if (jx2 < 0 || jx2 >= NV) continue;
                m = max(m, mxi[((size_t)ys * NV + jy2) * NVP + jx2]);
            }
        }
        if (m > 0x7f800000u) flags |= ST_NUMERIC;
        else if (m == 0x7f800000u) flags |= ST_OVERFLOW;
        so[i] = scale_for(m);
        mxo[i] = 0u;
    }
    if (flags) atomicOr(&a.b.st->status, flags);
}

// ---- encoding with error feedback -----------------------------------------------------------
// Shared by both step kernels: encode o + carry with the multiplier inv = 1/S, keep the residual.
template <typename S>
struct Encoder {
    float carry = 0.f;
    bool bad = false;
    // returns the stored value; *back = its decoded value
    __device__ __forceinline__ S operator()(float o, float inv, float* back) {
        return code(o, inv, pow2_inv(inv), back, true);
    }
    // the same from the scale's biased exponent e (S = 2^(e - 127)), without the overflow test:
    // a value out of the format is an infinite code, which the line maxima of the stored
    // output show (k_linemax_step)
    __device__ __forceinline__ S from_exponent(float o, unsigned e, float* back) {
        const unsigned sb = e << 23;
        return code(o, __uint_as_float((254u << 23) - sb), __uint_as_float(sb), back, false);
    }
    __device__ __forceinline__ S code(float o, float inv, float sc, float* back, bool test) {
        const float lim = __fmul_rn(HTraits<S>::kCarryLim, sc);
        const float used = fminf(fmaxf(carry, -lim), lim);
        const float t = __fadd_rn(o, used);
        const S h = HTraits<S>::enc(__fmul_rn(t, inv));
        const float hd = HTraits<S>::dec(h);
        *back = __fmul_rn(hd, sc);
        carry = __fadd_rn(__fsub_rn(t, *back), __fsub_rn(carry, used));
        if (test) bad |= !(fabsf(hd) <= HTraits<S>::kMax);
        return h;
    }
};

__device__ __forceinline__ unsigned warp_max_abs(float v, bool active) {
    return __reduce_max_sync(0xffffffffu, active ? __float_as_uint(fabsf(v)) : 0u);
}

// ---- plain-load kernel (any N_x, N_y) ---------------------------------------------------------
template <typename S, int NV>
struct GlobalRowH {
    const S* base;      // plane (row, 0) at source row ys
    const float* sc;    // scales of the plane row's lines at source row ys
    size_t pstride;
    int x, nx;
    __device__ __forceinline__ GlobalRowH(const S* f, const float* scales, int row, int x_, int y,
                                          int nx_, int ny_)
        : x(x_), nx(nx_) {
        constexpr int J = (NV - 1) / 2;
        pstride = (size_t)nx_ * ny_;
        const int ys = wrap(y - (row - J), ny_);
        base = f + (size_t)row * NV * pstride + (size_t)ys * nx_;
        sc = scales + ((size_t)ys * NV + row) * nv_padded(NV);
    }
    __device__ __forceinline__ float get(int jx) const {
        constexpr int J = (NV - 1) / 2;
        return __fmul_rn(HTraits<S>::dec(base[jx * pstride + wrap(x - (jx - J), nx)]), sc[jx]);
    }
};

template <typename S, int NV>
struct HalfPutG {
    S* out;
    const float* sc;   // output scales of row y
    unsigned* mx;      // output line maxima of row y
    size_t pstride;
    bool active;
    Encoder<S> enc;
    S* p;
    const float* sp;
    unsigned* mp;
    __device__ __forceinline__ HalfPutG(S* out_, const float* sc_, unsigned* mx_, size_t ps,
                                        bool act)
        : out(out_), sc(sc_), mx(mx_), pstride(ps), active(act), p(out_), sp(sc_), mp(mx_) {}
    __device__ __forceinline__ void begin(int row) {
        p = out + (size_t)row * NV * pstride;
        sp = sc + row * nv_padded(NV);
        mp = mx + row * nv_padded(NV);
    }
    __device__ __forceinline__ void operator()(float o) {
        float back;
        const S h = enc(o, pow2_inv(*sp), &back);
        if (active) *p = h;
        p += pstride;  // global loads: plain steps
        const unsigned m = warp_max_abs(back, active);
        if ((threadIdx.x & 31) == 0 && m) atomicMax(mp, m);
        ++sp;
        ++mp;
    }
};

template <typename S, int NV>
__global__ void __launch_bounds__(TW) k_step2d_plain_h(const Step2DHArgs ha, int kstep) {
    const Step2DArgs& a = ha.b;
    const long long step = a.st->step + kstep;
    const int par = (int)(step & 1);
    const float g = float(a.g), rr = float(a.r);
    const S* fin = static_cast<const S*>(par ? a.f[1] : a.f[0]);
    S* fout = static_cast<S*>(par ? a.f[0] : a.f[1]);
    const float* s_in = (par ? ha.sc[1] : ha.sc[0]);
    const float* s_out = (par ? ha.sc[0] : ha.sc[1]);
    unsigned* m_out = (par ? ha.mx[0] : ha.mx[1]);
    const size_t ps = (size_t)a.nx * a.ny;
    bool bad = false;
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const int y = tile / a.ntx;
        const int xr = (tile % a.ntx) * TW + threadIdx.x;
        const bool active = xr < a.nx;
        const int x = active ? xr : 0;
        float wx, wy;
        load_w<float>(a, x, y, wx, wy);
        cfl_check<float, NV>(a, g, wx, wy, active);
        float A[NV], G[NV], H[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            A[j] = 0.f;
            G[j] = 0.f;
            H[j] = 0.f;
        }
        const size_t yrow = (size_t)y * NV * nv_padded(NV);
        HalfPutG<S, NV> put(fout + (size_t)y * a.nx + x, s_out + yrow, m_out + yrow, ps, active);
        for (int r = 1; r <= NV; ++r) {
            const GlobalRowH<S, NV> cur(fin, s_in, r - 1, x, y, a.nx, a.ny);
            const GlobalRowH<S, NV> nxt(fin, s_in, r < NV ? r : r - 1, x, y, a.nx, a.ny);
            sweep_row<float, NV>(A, G, H, r, cur, nxt, g, wx, wy, rr, put);
        }
        final_row<float, NV>(A, H, rr, put);
        bad |= put.enc.bad && active;
    }
    if (bad) atomicOr(&a.st->status, ST_OVERFLOW);
}

// ---- producer/consumer kernel (N_x % 8 == 0, N_x >= kWinH) ------------------------------------
// The FP32 producer/consumer design with 16-bit rows in the ring.  One producer warp bulk-copies,
// per f* row, the shifted plane windows (16-byte aligned, split at the periodic wrap) and the
// row's N_v decode scales (one aligned run); with the first row of a tile it also copies the
// scales of the tile's N_v^2 output lines.
// Every copy of a row completes on that row's "full" mbarrier.  Four consumer warps sweep the
// columns, the vy-drag flux row G in shared memory.
template <int NV, int NS>
struct PCHShape {
    static constexpr int consumers = TW / 32;
    static constexpr int threads = 32 * (consumers + 1);
    static constexpr int min_blocks = 3;
};

// HSM: the vy-diffusion flux row H in shared memory as well, right after G.
template <typename S, int NV, int NS, bool HSM = false>
struct PCHLayout {
    static constexpr int NVP = nv_padded(NV);
    static constexpr int NLP = NV * NVP;  // padded output lines of a tile
    static constexpr size_t ring = (size_t)NS * NV * kWinH * sizeof(S);
    static constexpr size_t gsm = (size_t)(HSM ? 2 : 1) * NV * TW * sizeof(float);
    static constexpr size_t dsc = (size_t)NS * NVP * sizeof(float);
    static constexpr size_t enc = ((size_t)2 * NLP + 15) / 16 * 16;  // exponent bytes
    static constexpr size_t mxs = 0;  // the line maxima come from k_linemax_step
    static constexpr size_t bars = (size_t)2 * NS * sizeof(uint64_t);
    static constexpr size_t o_gsm = ring;
    static constexpr size_t o_dsc = o_gsm + gsm;
    static constexpr size_t o_enc = o_dsc + dsc;
    static constexpr size_t o_mxs = o_enc + enc;
    static constexpr size_t o_bar = o_mxs + mxs;
    static constexpr size_t total = o_bar + bars;
    static_assert(ring % 16 == 0 && gsm % 16 == 0 && dsc % 16 == 0 && enc % 16 == 0 &&
                  mxs % 16 == 0, "bulk-copy destinations must stay 16-byte aligned");
};

template <typename S, int NV>
struct RingRowH {
    const S* p;        // ring + slot NV kWinH + cell
    const float* d;    // decode scales of the slot's NV planes
    __device__ __forceinline__ float get(int jx) const {
        constexpr int J = (NV - 1) / 2;
        return __fmul_rn(HTraits<S>::dec(p[jx * kWinH + ((J - jx) % 8 + 8) % 8]), d[jx]);
    }
};

// Output writer of the producer/consumer kernel.  The line maxima of what it writes are not
// reduced here (a warp maximum and a shared atomic per value cost a quarter of the step): the
// next launch, k_linemax_step, takes them from the stored output, the same values exactly.
template <typename S, int NV>
struct HalfPutS {
    S* out;
    size_t pstride;
    bool active;
    const unsigned char* sc_tab;  // biased exponents of the tile's output scales [NV][NVP]
                                  // (shared memory; the scales are powers of two)
    Encoder<S> enc;
    S* p;
    const unsigned char* sp;
    __device__ __forceinline__ HalfPutS(S* out_, size_t ps, bool act, const unsigned char* e)
        : out(out_), pstride(ps), active(act), sc_tab(e), p(out_), sp(e) {}
    __device__ __forceinline__ void begin(int row) {
        p = out + (size_t)row * NV * pstride;
        sp = sc_tab + row * nv_padded(NV);
    }
    __device__ __forceinline__ void operator()(float o) {
        float back;
        const S h = enc.from_exponent(o, *sp, &back);
        ++sp;
        if (active) *p = h;
        p = next_plane(p, pstride);
    }
};

// Issue the copies of f* row `row` of tile `tile` into ring slot `slot` (producer warp): the
// plane windows and the row's decode scales; with row 0 the warp first writes the biased
// exponents of the tile's output scales (powers of two) into enc_dst, one byte per line, which
// the row's mbarrier arrival releases to the consumers.
template <typename S, int NV>
__device__ __forceinline__ void issue_row_h(const Step2DArgs& a, const S* fin, S* ring,
                                            uint64_t* bar, float* dsc, const float* s_in,
                                            const float* s_out, unsigned char* enc_dst, int slot,
                                            int tile, int row) {
    constexpr int J = (NV - 1) / 2;
    constexpr int NVP = nv_padded(NV);
    constexpr int EL = 16 / (int)sizeof(S);  // elements per 16 bytes
    const int lane = threadIdx.x & 31;
    const int y = tile / a.ntx;
    const int x0 = (tile % a.ntx) * TW;
    const int ys = wrap(y - (row - J), a.ny);
    const unsigned bytes = (unsigned)(NV * kWinH * sizeof(S) + NVP * sizeof(float));
    if (row == 0) {
        const float* so = s_out + (size_t)y * NV * NVP;
        for (int i = lane; i < NV * NVP; i += 32)
            enc_dst[i] = (unsigned char)(__float_as_uint(so[i]) >> 23);
        __syncwarp();
    }
    if (lane == 0) mbar_expect_tx(&bar[slot], bytes);  // release: the exponents written above
    __syncwarp();
    if (lane == 0)
        bulk_g2s(dsc + slot * NVP, s_in + ((size_t)ys * NV + row) * NVP, NVP * sizeof(float),
                 &bar[slot]);
    for (int jx = lane; jx < NV; jx += 32) {
        const S* prow = fin + (((size_t)row * NV + jx) * a.ny + ys) * a.nx;
        const int s = x0 - (jx - J);
        const int base = wrap(s - ((s % EL) + EL) % EL, a.nx);
        S* dst = ring + ((size_t)slot * NV + jx) * kWinH;
        if (base + kWinH <= a.nx) {
            bulk_g2s(dst, prow + base, kWinH * sizeof(S), &bar[slot]);
        } else {
            const int n1 = a.nx - base;
            bulk_g2s(dst, prow + base, n1 * sizeof(S), &bar[slot]);
            bulk_g2s(dst + n1, prow, (kWinH - n1) * sizeof(S), &bar[slot]);
        }
    }
}

// Producer warp of the 16-bit producer/consumer kernels: fills the ring and copies the scales.
template <typename S, int NV, int NS, class TileOf>
__device__ __forceinline__ void produce_rows_h(const Step2DArgs& a, const S* fin, S* ring,
                                               uint64_t* full, uint64_t* empty, float* dsc,
                                               const float* s_in, const float* s_out,
                                               unsigned char* enc, int ntl,
                                               const TileOf& tile_of) {
    constexpr int NLP = NV * nv_padded(NV);
    const int lane = threadIdx.x & 31;
    // a stalled context issues no copies: every consumer's bounded wait runs out
    const long long total = a.st->stall ? 0 : (long long)ntl * NV;
    long long f = 0;
    for (; f < total; ++f) {
        const int q = (int)(f % NS);
        if (f >= NS && !mbar_wait_bounded(&empty[q], (unsigned)(((f / NS) + 1) & 1))) {
            if (lane == 0) atomicOr(&a.st->status, ST_TIMEOUT);
            break;
        }
        // the exponent table of tile t (written with its row 0) alternates between two
        // buffers: every consumer released fill f - NS, a row of tile t - 1, so all of them are
        // past tile t - 2, its previous user
        const int t = (int)(f / NV);
        issue_row_h<S, NV>(a, fin, ring, full, dsc, s_in, s_out, enc + (t & 1) * NLP, q,
                           tile_of(f), (int)(f % NV));
    }
    for (long long d = std::max(0ll, f - NS); d < f; ++d)
        mbar_wait_bounded(&full[d % NS], (unsigned)((d / NS) & 1));
}

template <typename S, int NV, int NS, bool HSM>
__global__ void __launch_bounds__(PCHShape<NV, NS>::threads, PCHShape<NV, NS>::min_blocks)
    k_step2d_pch(const Step2DHArgs ha, int kstep) {
    using Lay = PCHLayout<S, NV, NS, HSM>;
    constexpr int NC = PCHShape<NV, NS>::consumers;
    constexpr int NVP = Lay::NVP;
    constexpr int NLP = Lay::NLP;
    const Step2DArgs& a = ha.b;
    extern __shared__ __align__(128) unsigned char smem[];
    S* ring = reinterpret_cast<S*>(smem);
    float* gsm = reinterpret_cast<float*>(smem + Lay::o_gsm);
    float* dsc = reinterpret_cast<float*>(smem + Lay::o_dsc);
    unsigned char* enc = smem + Lay::o_enc;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + Lay::o_bar);
    uint64_t* empty = full + NS;
    const long long step = a.st->step + kstep;
    const int par = (int)(step & 1);
    const float g = float(a.g), rr = float(a.r);
    const S* fin = static_cast<const S*>(par ? a.f[1] : a.f[0]);
    S* fout = static_cast<S*>(par ? a.f[0] : a.f[1]);
    const float* s_in = (par ? ha.sc[1] : ha.sc[0]);
    const float* s_out = (par ? ha.sc[0] : ha.sc[1]);
    const size_t ps = (size_t)a.nx * a.ny;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntl = a.ntiles > (int)blockIdx.x ? (a.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    auto tile_of = [&](long long s) { return (int)(blockIdx.x + (s / NV) * gridDim.x); };
    if (threadIdx.x == 0) {
        for (int q = 0; q < NS; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], NC);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (warp == NC) {
        produce_rows_h<S, NV, NS>(a, fin, ring, full, empty, dsc, s_in, s_out, enc, ntl,
                                  tile_of);
        return;
    }
    const int cell = threadIdx.x;
    bool failed = false;
    for (int lt = 0; lt < ntl && !failed; ++lt) {
        const int tile = tile_of((long long)lt * NV);
        const int y = tile / a.ntx;
        const int xr = (tile % a.ntx) * TW + cell;
        const bool active = xr < a.nx;
        const int x = active ? xr : 0;
        float wx, wy;
        load_w<float>(a, x, y, wx, wy);
        cfl_check<float, NV>(a, g, wx, wy, active);
        float A[NV], Hreg[NV];
        SmemCol Gs{gsm + cell}, Hs{gsm + NV * TW + cell};
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            A[j] = 0.f;
            if constexpr (HSM) Hs[j] = 0.f;
            else Hreg[j] = 0.f;
            Gs[j] = 0.f;
        }
        HalfPutS<S, NV> put(fout + (size_t)y * a.nx + x, ps, active, enc + (lt & 1) * NLP);
        const long long s0 = (long long)lt * NV;
        for (int r = 0; r <= NV; ++r) {
            const long long s = s0 + r;
            if (r < NV && !mbar_wait_bounded(&full[s % NS], (unsigned)((s / NS) & 1))) {
                failed = true;
                break;
            }
            if (r >= 1) {
                const int qc = (int)((s - 1) % NS), qn = (int)(s % NS);
                const RingRowH<S, NV> cur{ring + (size_t)qc * NV * kWinH + cell, dsc + qc * NVP};
                const RingRowH<S, NV> nxt{ring + (size_t)qn * NV * kWinH + cell, dsc + qn * NVP};
                if constexpr (HSM) sweep_row<float, NV>(A, Gs, Hs, r, cur, nxt, g, wx, wy, rr, put);
                else sweep_row<float, NV>(A, Gs, Hreg, r, cur, nxt, g, wx, wy, rr, put);
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[qc]);  // row s - 1 is done
            }
        }
        if (!failed) {
            if constexpr (HSM) final_row<float, NV>(A, Hs, rr, put);
            else final_row<float, NV>(A, Hreg, rr, put);
        }
    }
    if (failed && lane == 0) atomicOr(&a.st->status, ST_TIMEOUT);
    // encoder overflows show as infinite line maxima: k_linemax_step reports them
}

// ---- state conversion -------------------------------------------------------------------------
// Index of line (plane p = jy N_v + jx, row y) in the scale layout.
__device__ __forceinline__ size_t scale_index(int p, int y, int nv) {
    const int jy = p / nv, jx = p - jy * nv;
    return ((size_t)y * nv + jy) * nv_padded(nv) + jx;
}

// One warp per line: max |value| (decoded with the line's scale when sc is given).  Lines are
// visited in the state's order, l = p N_y + y.
template <typename T>
__global__ void __launch_bounds__(256) k_linemax(const T* f, const float* sc, unsigned* mx,
                                                 float* scale_out, long long nlines, int nx,
                                                 int ny, int nv) {
    const int lane = threadIdx.x & 31;
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long l = w0; l < nlines; l += nw) {
        const T* row = f + (size_t)l * nx;
        const size_t si = scale_index((int)(l / ny), (int)(l % ny), nv);
        const float s = sc ? sc[si] : 1.f;
        unsigned m = 0;
        for (int x = lane; x < nx; x += 32)
            m = max(m, __float_as_uint(fabsf(__fmul_rn((float)row[x], s))));
        m = __reduce_max_sync(0xffffffffu, m);
        if (lane == 0) {
            if (mx) mx[si] = m;
            if (scale_out) scale_out[si] = scale_for(m);
        }
    }
}

// The line maxima of the output of step kstep of a batch (buffer, scales and maxima of parity
// (step + kstep + 1) & 1), one warp per line, 16-byte loads (N_x a multiple of 8): the values
// and bits of k_linemax.
template <typename S>
__global__ void __launch_bounds__(256) k_linemax_step(const Step2DHArgs ha, int kstep, int nv) {
    const Step2DArgs& a = ha.b;
    const bool par = ((a.st->step + kstep) & 1) != 0;
    const S* f = static_cast<const S*>(par ? a.f[0] : a.f[1]);
    const float* sc = par ? ha.sc[0] : ha.sc[1];
    unsigned* mx = par ? ha.mx[0] : ha.mx[1];
    const int nx = a.nx, ny = a.ny;
    const long long nlines = (long long)nv * nv * ny;
    constexpr int EL = 16 / (int)sizeof(S);
    const int lane = threadIdx.x & 31;
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long l = w0; l < nlines; l += nw) {
        const uint4* row = reinterpret_cast<const uint4*>(f + (size_t)l * nx);
        const size_t si = scale_index((int)(l / ny), (int)(l % ny), nv);
        const float s = sc[si];
        unsigned m = 0;
        for (int c = lane; c < nx / EL; c += 32) {
            const uint4 v = row[c];
            const S* h = reinterpret_cast<const S*>(&v);
#pragma unroll
            for (int e = 0; e < EL; ++e)
                m = max(m, __float_as_uint(fabsf(__fmul_rn(HTraits<S>::dec(h[e]), s))));
        }
        m = __reduce_max_sync(0xffffffffu, m);
        if (lane == 0) {
            mx[si] = m;
            // an infinite or NaN stored value on this line: the encoder's overflow (the test
            // the plain kernel's encoder makes per value)
            if (m >= 0x7f800000u) atomicOr(&a.st->status, ST_OVERFLOW);
        }
    }
}

// Line l of the [plane][y][x] layout is (plane, y) = (l / ny, l % ny), the scale index itself.
template <typename S>
__global__ void __launch_bounds__(256) k_encode(const float* src, S* f, const float* sc, int nv,
                                                int nx, int ny, DevState* st) {
    const long long ncell = (long long)nx * ny;
    const int np = nv * nv;
    bool bad = false;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(c / nx);
        Encoder<S> enc;
        for (int p = 0; p < np; ++p) {
            float back;
            f[(size_t)p * ncell + c] =
                enc(src[(size_t)p * ncell + c], pow2_inv(sc[scale_index(p, y, nv)]), &back);
        }
        bad |= enc.bad;
    }
    if (bad) atomicOr(&st->status, ST_OVERFLOW);
}

template <typename S>
__global__ void __launch_bounds__(256) k_decode(const S* f, const float* sc, float* dst,
                                                long long n, int nx, int ny, int nv) {
    const long long ncell = (long long)nx * ny;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(i / ncell);
        const int y = (int)((i % ncell) / nx);
        dst[i] = __fmul_rn(HTraits<S>::dec(f[i]), sc[scale_index(p, y, nv)]);
    }
}

__global__ void k_scales_dense(const float* sc, float* dst, int nv, int ny) {
    const long long n = (long long)nv * nv * ny;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = sc[scale_index((int)(i / ny), (int)(i % ny), nv)];
}

__global__ void k_fill(float* p, long long n, float v) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

int grid_for(long long n, int per_block) {
    return (int)std::max<long long>(1, std::min<long long>((n + per_block - 1) / per_block, 4096));
}

// ---- launch tables ----------------------------------------------------------------------------
#define LATH_NV_LIST(X) X(1) X(3) X(5) X(9) X(13) X(17) X(21) X(33)
#define LATH_PC(n) ((n) >= 9)

template <typename S, int NV, int NS, bool HSM = false>
cudaError_t launch_pch(int grid, const Step2DHArgs& a, int k, cudaStream_t s) {
    using Lay = PCHLayout<S, NV, NS, HSM>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_step2d_pch<S, NV, NS, HSM>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Lay::total);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_step2d_pch<S, NV, NS, HSM><<<grid, PCHShape<NV, NS>::threads, Lay::total, s>>>(a, k);
    return cudaGetLastError();
}

template <typename S, int NV, int NS, bool HSM = false>
int occupancy_pch() {
    using Lay = PCHLayout<S, NV, NS, HSM>;
    int nb = 0;
    cudaFuncSetAttribute(k_step2d_pch<S, NV, NS, HSM>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::total);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step2d_pch<S, NV, NS, HSM>,
                                                  PCHShape<NV, NS>::threads, Lay::total);
    return nb;
}

template <typename S>
cudaError_t launch_linemax_step(const Step2DHArgs& a, int k, int nv, cudaStream_t s) {
    const long long nl = (long long)nv * nv * a.b.ny;
    k_linemax_step<S><<<grid_for(nl * 32, 256), 256, 0, s>>>(a, k, nv);
    return cudaGetLastError();
}

// The producer/consumer kernels, each followed by the line maxima of what it wrote.
template <typename S, int NV>
cudaError_t launch_h_t(int pcv, int grid, const Step2DHArgs& a, int k, cudaStream_t s) {
    if constexpr (LATH_PC(NV)) {
        cudaError_t e = cudaErrorInvalidValue;
        if (pcv == 4) e = launch_pch<S, NV, 4>(grid, a, k, s);
        else if (pcv == 5) e = launch_pch<S, NV, 3>(grid, a, k, s);
        else if (pcv == 6) e = launch_pch<S, NV, 3, true>(grid, a, k, s);
        else if (pcv == 7) e = launch_pch<S, NV, 2, true>(grid, a, k, s);
        if (pcv >= 4 && pcv <= 7) {
            if (e != cudaSuccess) return e;
            return launch_linemax_step<S>(a, k, NV, s);
        }
    }
    if (pcv == 0) {
        k_step2d_plain_h<S, NV><<<grid, TW, 0, s>>>(a, k);
        return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
}

template <typename S, int NV>
int occupancy_h_t(int pcv) {
    if constexpr (LATH_PC(NV)) {
        if (pcv == 4) return occupancy_pch<S, NV, 4>();
        if (pcv == 5) return occupancy_pch<S, NV, 3>();
        if (pcv == 6) return occupancy_pch<S, NV, 3, true>();
        if (pcv == 7) return occupancy_pch<S, NV, 2, true>();
    }
    return 0;
}

}  // namespace

bool h2d_supported(int nv) {
    switch (nv) {
#define X(n) case n:
        LATH_NV_LIST(X)
#undef X
        return true;
        default: return false;
    }
}

bool h2d_ring_ok(int nx) { return nx % 8 == 0 && nx >= kWinH; }

cudaError_t launch_step2d_h(int dtype, int nv, int pcv, int grid, const Step2DHArgs& a, int k,
                            cudaStream_t s) {
    if (pcv != 0 && (nv < 9 || !h2d_ring_ok(a.b.nx))) return cudaErrorInvalidValue;
    switch (nv) {
#define X(n)                                                                      \
    case n:                                                                       \
        if (dtype == LAT_F16) return launch_h_t<__half, n>(pcv, grid, a, k, s);   \
        if (dtype == LAT_BF16) return launch_h_t<__nv_bfloat16, n>(pcv, grid, a, k, s); \
        return cudaErrorInvalidValue;
        LATH_NV_LIST(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

int occupancy_step2d_h(int dtype, int nv, int pcv) {
    switch (nv) {
#define X(n)                                                                       \
    case n:                                                                        \
        if (dtype == LAT_F16) return occupancy_h_t<__half, n>(pcv);                \
        if (dtype == LAT_BF16) return occupancy_h_t<__nv_bfloat16, n>(pcv);        \
        return 0;
        LATH_NV_LIST(X)
#undef X
        default: return 0;
    }
}

cudaError_t launch_scale2d(int nv, int ny, const Step2DHArgs& a, int k, cudaStream_t s) {
    const long long nl = scale_count(nv, ny);
    const int grid = grid_for(nl, 256);
    switch (nv) {
#define X(n)                                            \
    case n:                                             \
        k_scale2d<n><<<grid, 256, 0, s>>>(a, k);        \
        return cudaGetLastError();
        LATH_NV_LIST(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_linemax_h(int dtype, const void* f, const float* sc, unsigned* mx, int nv,
                             int nx, int ny, cudaStream_t s) {
    const long long nl = (long long)nv * nv * ny;
    const int grid = grid_for(nl * 32, 256);
    if (dtype == LAT_F16)
        k_linemax<__half><<<grid, 256, 0, s>>>(static_cast<const __half*>(f), sc, mx, nullptr, nl,
                                               nx, ny, nv);
    else if (dtype == LAT_BF16)
        k_linemax<__nv_bfloat16><<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(f), sc, mx,
                                                      nullptr, nl, nx, ny, nv);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_encode_h(int dtype, const float* src, void* f, float* sc, unsigned* mx,
                            int nv, int nx, int ny, DevState* st, cudaStream_t s) {
    const long long nl = (long long)nv * nv * ny;
    // scales from the line maxima of the input, then the encoding, then the stored maxima
    k_linemax<float><<<grid_for(nl * 32, 256), 256, 0, s>>>(src, nullptr, nullptr, sc, nl, nx,
                                                            ny, nv);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long ncell = (long long)nx * ny;
    const int grid = grid_for(ncell, 256);
    if (dtype == LAT_F16)
        k_encode<__half><<<grid, 256, 0, s>>>(src, static_cast<__half*>(f), sc, nv, nx, ny, st);
    else if (dtype == LAT_BF16)
        k_encode<__nv_bfloat16><<<grid, 256, 0, s>>>(src, static_cast<__nv_bfloat16*>(f), sc, nv,
                                                     nx, ny, st);
    else
        return cudaErrorInvalidValue;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_linemax_h(dtype, f, sc, mx, nv, nx, ny, s);
}

cudaError_t launch_decode_h(int dtype, const void* f, const float* sc, float* dst, int nv, int nx,
                            int ny, cudaStream_t s) {
    const long long n = (long long)nv * nv * nx * ny;
    const int grid = grid_for(n, 256);
    if (dtype == LAT_F16)
        k_decode<__half><<<grid, 256, 0, s>>>(static_cast<const __half*>(f), sc, dst, n, nx, ny,
                                              nv);
    else if (dtype == LAT_BF16)
        k_decode<__nv_bfloat16><<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(f), sc, dst,
                                                     n, nx, ny, nv);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_scales_dense(const float* sc, float* dst, int nv, int ny, cudaStream_t s) {
    k_scales_dense<<<grid_for((long long)nv * nv * ny, 256), 256, 0, s>>>(sc, dst, nv, ny);
    return cudaGetLastError();
}

cudaError_t launch_fill_scales(float* sc, long long n, cudaStream_t s) {
    k_fill<<<grid_for(n, 256), 256, 0, s>>>(sc, n, 1.f);
    return cudaGetLastError();
}

}  // namespace lat

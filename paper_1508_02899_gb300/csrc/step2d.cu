// Two-dimensional lattice context: flow evaluation, the fused 2D step and the 2D moments.
//
// Layout f[jy][jx][y][x] (x fastest).  One thread owns one spatial cell (x, y); a block owns a
// tile of 128 consecutive x cells of one row y.  The velocity column of a cell is swept row by
// row in jy.  Row jy of the post-streaming density, f*(x, y, jx, jy) = f(x - jx, y - jy, jx, jy)
// for all jx, is one velocity "row"; the drag (unsplit, first-order upwind in vx and vy) and the
// five-point velocity diffusion then need, per thread, only three register rows:
//   A = f** of the previous row, G = vy-drag flux between rows, H = vy-diffusion flux between
// rows; x-direction fluxes are carried as scalars along the jx sweep.
//
// Rows of f* reach shared memory by bulk asynchronous copies (cp.async.bulk, completion on an
// mbarrier) into a 4-slot ring, two rows ahead of the sweep: the streaming shift is applied by
// the copy's source address (x window rounded down to 16 bytes, split in two at the periodic
// wrap; y wraps by choosing the source row).  A plain-load variant with the same arithmetic
// serves FP64 and grids the copy path does not cover (N_x not a multiple of 4, or < 132).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include <algorithm>
#include <type_traits>
#include <map>

#include "lat2d.h"
#include "step2d_dev.h"
#include "step2d_x2.h"
#include "step2d_h.h"
#include "learn.h"
#include "lat_reduce.h"

namespace lat {

namespace {

using namespace k2d;
using namespace cs;

constexpr int WIN = TW + 4;   // floats copied per plane row (x window rounded to 16 bytes)
#ifndef LAT_RING2D_SLOTS
#define LAT_RING2D_SLOTS 4
#endif
constexpr int NSLOT = LAT_RING2D_SLOTS;  // ring slots of f* rows
constexpr int LOOK = NSLOT - 2;          // rows in flight ahead of the one being waited for

struct Flow2DArgs {
    const int2* k;            // [M] (kx, ky)
    const double* cx;         // [M] coefficient of sin(theta) in u_x
    const double* cy;         // [M] coefficient of sin(theta) in u_y
    double* phase;            // [2][M] parity-indexed phases
    const double* noise;      // [rows][M] in the caller's mode order
    const int* perm;          // [M] caller's index of mode m (modes are kept sorted by kx)
    const int* runs;          // [nruns + 1][2]: first mode and kx of each run of equal kx
    double walk;              // sqrt(2 dt / tau_f)
    const void* xtab;         // [2 kmax+1][nx][2] of T
    const void* ytab;         // [2 kmax+1][ny][2] of T
    int kmax;
    int nmodes, nx, ny, nruns;
    void* u;                  // [2][ny][nx] of T
    DevState* st;
    int frozen, dry;
};

// ---- plain-load kernel (any N_x, N_y; FP32 or FP64) -----------------------------------------
template <typename T, int NV>
__global__ void __launch_bounds__(TW) k_step2d_plain(const Step2DArgs a, int kstep) {
    const long long step = a.st->step + kstep;
    const int par = (int)(step & 1);
    const T g = T(a.g), rr = T(a.r);
    const T* fin = static_cast<const T*>(par ? a.f[1] : a.f[0]);
    T* fout = static_cast<T*>(par ? a.f[0] : a.f[1]);
    const size_t ps = (size_t)a.nx * a.ny;
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const int y = tile / a.ntx;
        const int xr = (tile % a.ntx) * TW + threadIdx.x;
        const bool active = xr < a.nx;
        const int x = active ? xr : 0;
        T wx, wy;
        load_w<T>(a, x, y, wx, wy);
        cfl_check<T, NV>(a, g, wx, wy, active);
        T A[NV], G[NV], H[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            A[j] = T(0);
            G[j] = T(0);
            H[j] = T(0);
        }
        StorePut<T, NV, false> put(fout + (size_t)y * a.nx + x, ps, active);  // global loads
        for (int r = 1; r <= NV; ++r) {
            const GlobalRow<T, NV> cur(fin, r - 1, x, y, a.nx, a.ny);
            const GlobalRow<T, NV> nxt(fin, r < NV ? r : r - 1, x, y, a.nx, a.ny);
            sweep_row<T, NV>(A, G, H, r, cur, nxt, g, wx, wy, rr, put);
        }
        final_row<T, NV>(A, H, rr, put);
    }
}

// ---- bulk-copy ring kernel (FP32; N_x % 4 == 0, N_x >= WIN) -----------------------------------
// Row of f* held in one ring slot: plane jx starts at p + jx WIN, shifted by the 16-byte
// rounding of its window, (x0 - (jx - J)) mod 4 with x0 % 4 == 0.
template <int NV>
struct RingRow {
    const float* p;  // ring + slot NV WIN + tid
    __device__ __forceinline__ float get(int jx) const {
        constexpr int J = (NV - 1) / 2;
        return p[jx * WIN + ((J - jx) % 4 + 4) % 4];
    }
};

// Issue the bulk copies of f* row `row` of tile `tile` into ring slot `slot` (warp 0 only).
// A slot holds NV windows of WIN floats, then GX floats more.  With corrections (gcorr, GX =
// 2 NV TW): the row's learned-closure corrections G[c][row][jx] at the tile's cells, unshifted,
// as rows of TW floats ([c][jx][cell]); the tile's cells only (N_x a multiple of 4 keeps every
// piece a multiple of 16 bytes).
template <int NV, int GX = 0>
__device__ __forceinline__ void issue_row(const Step2DArgs& a, const float* fin, float* ring,
                                          uint64_t* bar, int slot, int tile, int row,
                                          const float* gcorr = nullptr) {
    constexpr int J = (NV - 1) / 2;
    constexpr size_t SL = (size_t)NV * WIN + GX;  // floats per slot
    const int lane = threadIdx.x & 31;
    const int y = tile / a.ntx;
    const int x0 = (tile % a.ntx) * TW;
    const int ncx = min(TW, a.nx - x0);  // cells of the tile
    unsigned bytes = (unsigned)(NV * WIN * sizeof(float));
    if constexpr (GX > 0) bytes += (unsigned)(2 * NV * ncx * sizeof(float));
    if (lane == 0) mbar_expect_tx(&bar[slot], bytes);
    __syncwarp();
    const int ys = wrap(y - (row - J), a.ny);
    if constexpr (GX > 0) {
        const size_t ps = (size_t)a.nx * a.ny;
        float* gdst = ring + (size_t)slot * SL + (size_t)NV * WIN;
        for (int i = lane; i < 2 * NV; i += 32) {  // i = c NV + jx
            const int cmp = i / NV, jx = i - cmp * NV;
            const float* src =
                gcorr + (size_t)cmp * NV * NV * ps + ((size_t)row * NV + jx) * ps + (size_t)y * a.nx + x0;
            bulk_g2s(gdst + (size_t)i * TW, src, (unsigned)(ncx * sizeof(float)), &bar[slot]);
        }
    }
    for (int jx = lane; jx < NV; jx += 32) {
        const float* prow = fin + (((size_t)row * NV + jx) * a.ny + ys) * a.nx;
        const int s = x0 - (jx - J);
        const int base = wrap(s - ((s % 4) + 4) % 4, a.nx);
        float* dst = ring + (size_t)slot * SL + (size_t)jx * WIN;
        if (base + WIN <= a.nx) {
            bulk_g2s(dst, prow + base, WIN * sizeof(float), &bar[slot]);
        } else {
            const int n1 = a.nx - base;
            bulk_g2s(dst, prow + base, n1 * sizeof(float), &bar[slot]);
            bulk_g2s(dst + n1, prow, (WIN - n1) * sizeof(float), &bar[slot]);
        }
    }
}

// ---- split-column sweep: chunk [J0, J1) of the jx range of one cell ----------------------------
// Same operations, in the same order, as sweep_row restricted to jx in [J0, J1): the x-drag flux
// entering at J0 - 1/2 is recomputed from the shared-memory row; the x-diffusion flux there needs
// the neighbouring chunk's f** of the previous row (xl, left) and, at J1 - 1/2, xr (right).
template <int NV, int J0, int J1, int WM>
__device__ __forceinline__ void sweep_chunk(float (&A)[WM], float (&G)[WM], float (&H)[WM], int r,
                                            const RingRow<NV>& cur, const RingRow<NV>& nxt_row,
                                            float g, float wx, float wy, float rr, float xl,
                                            float xr, float* __restrict__ out, size_t pstride,
                                            bool active) {
    using O = Ops<float>;
    constexpr int J = (NV - 1) / 2, W = J1 - J0;
    const int rb = r - 1;
    const bool nxt = r < NV;
    const float ayp = fmax(cacc<float>(g, wy, rb - J), 0.f);
    const float aym = nxt ? fmin(cacc<float>(g, wy, r - J), 0.f) : 0.f;
    float Fprev = 0.f, Dprev = 0.f;
    if (J0 > 0) {
        Fprev = dflux<float>(cacc<float>(g, wx, J0 - 1 - J), cacc<float>(g, wx, J0 - J),
                             cur.get(J0 - 1), cur.get(J0));
        if (r >= 2) Dprev = O::mul(rr, O::sub(A[0], xl));
    }
    float sc = cur.get(J0);
#pragma unroll
    for (int k = 0; k < W; ++k) {
        const int jx = J0 + k;
        float sn = 0.f, Fnext = 0.f;
        if (jx < NV - 1) {
            sn = cur.get(jx + 1);
            Fnext = dflux<float>(cacc<float>(g, wx, jx - J), cacc<float>(g, wx, jx + 1 - J), sc, sn);
        }
        const float Gn = nxt ? O::fma(ayp, sc, O::mul(aym, nxt_row.get(jx))) : 0.f;
        const float b = O::sub(O::sub(sc, O::sub(Fnext, Fprev)), O::sub(Gn, G[k]));
        G[k] = Gn;
        Fprev = Fnext;
        sc = sn;
        if (r >= 2) {
            const float a = A[k];
            const float an = (k + 1 < W) ? A[k + 1] : xr;
            const float Dn = (jx < NV - 1) ? O::mul(rr, O::sub(an, a)) : 0.f;
            const float Hn = O::mul(rr, O::sub(b, a));
            const float o = O::add(O::add(a, O::sub(Dn, Dprev)), O::sub(Hn, H[k]));
            H[k] = Hn;
            Dprev = Dn;
            if (active) out[((size_t)(r - 2) * NV + jx) * pstride] = o;
        }
        A[k] = b;
    }
}

template <int NV, int J0, int J1, int WM>
__device__ __forceinline__ void final_chunk(float (&A)[WM], float (&H)[WM], float rr, float xl,
                                            float xr, float* __restrict__ out, size_t pstride,
                                            bool active) {
    using O = Ops<float>;
    constexpr int W = J1 - J0;
    float Dprev = (J0 > 0) ? O::mul(rr, O::sub(A[0], xl)) : 0.f;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        const int jx = J0 + k;
        const float a = A[k];
        const float an = (k + 1 < W) ? A[k + 1] : xr;
        const float Dn = (jx < NV - 1) ? O::mul(rr, O::sub(an, a)) : 0.f;
        const float o = O::add(O::add(a, O::sub(Dn, Dprev)), O::sub(0.f, H[k]));
        Dprev = Dn;
        if (active) out[((size_t)(NV - 1) * NV + jx) * pstride] = o;
    }
}

// Compile-time dispatch of the calling warp's chunk (the chunk index is warp-uniform).
template <int NV, int C, int WM, int c = 0>
__device__ __forceinline__ void chunk_sweep(int chunk, float (&A)[WM], float (&G)[WM],
                                            float (&H)[WM], int r, const RingRow<NV>& cur,
                                            const RingRow<NV>& nxt, float g, float wx, float wy,
                                            float rr, float xl, float xr, float* out, size_t ps,
                                            bool active, float* pub_first, float* pub_last) {
    if constexpr (c < C) {
        constexpr int J0 = c * NV / C, J1 = (c + 1) * NV / C;
        if (chunk == c) {
            sweep_chunk<NV, J0, J1, WM>(A, G, H, r, cur, nxt, g, wx, wy, rr, xl, xr, out, ps,
                                        active);
            if (C > 1) {  // publish this chunk's edges of the new f** row
                *pub_first = A[0];
                *pub_last = A[J1 - J0 - 1];
            }
            return;
        }
        chunk_sweep<NV, C, WM, c + 1>(chunk, A, G, H, r, cur, nxt, g, wx, wy, rr, xl, xr, out, ps,
                                      active, pub_first, pub_last);
    }
}
template <int NV, int C, int WM, int c = 0>
__device__ __forceinline__ void chunk_final(int chunk, float (&A)[WM], float (&H)[WM], float rr,
                                            float xl, float xr, float* out, size_t ps, bool active) {
    if constexpr (c < C) {
        if (chunk == c) {
            final_chunk<NV, c * NV / C, (c + 1) * NV / C, WM>(A, H, rr, xl, xr, out, ps, active);
            return;
        }
        chunk_final<NV, C, WM, c + 1>(chunk, A, H, rr, xl, xr, out, ps, active);
    }
}
template <int NV, int C>
struct RingShape {
    static constexpr int threads = TW * C;
    static constexpr int min_blocks = C == 1 ? (NV > 17 ? 2 : 3) : (C == 2 ? 2 : 1);
    static constexpr int wmax = (NV + C - 1) / C;
};

// Bulk-copy ring kernel: a block of 128 C threads owns 128 cells; the C warp groups split each
// cell's jx range into chunks and exchange one f** value per chunk boundary per row.
template <int NV, int C>
__global__ void __launch_bounds__(RingShape<NV, C>::threads, RingShape<NV, C>::min_blocks)
    k_step2d_ring(const Step2DArgs a, int kstep) {
    constexpr int WM = RingShape<NV, C>::wmax;
    extern __shared__ __align__(128) unsigned char smem[];
    float* ring = reinterpret_cast<float*>(smem);
    float* xch = ring + (size_t)NSLOT * NV * WIN;  // [2][C][2][TW]
    uint64_t* bar = reinterpret_cast<uint64_t*>(xch + 2 * C * 2 * TW);
    const long long step = a.st->step + kstep;
    const int par = (int)(step & 1);
    const float g = float(a.g), rr = float(a.r);
    const float* fin = static_cast<const float*>(par ? a.f[1] : a.f[0]);
    float* fout = static_cast<float*>(par ? a.f[0] : a.f[1]);
    const size_t ps = (size_t)a.nx * a.ny;
    const int tid = threadIdx.x;
    const int cell = tid % TW;
    const int chunk = tid / TW;
    auto xch_at = [&](int parity, int c, int side) -> float& {
        return xch[((parity * C + c) * 2 + side) * TW + cell];
    };
    const int ntl = a.ntiles > (int)blockIdx.x ? (a.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const long long total = (long long)ntl * NV;  // rows this block consumes
    if (tid == 0) {
        for (int q = 0; q < NSLOT; ++q) mbar_init(&bar[q], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto tile_of = [&](long long s) { return (int)(blockIdx.x + (s / NV) * gridDim.x); };
    if (tid < 32) {
        for (long long s = 0; s < LOOK && s < total; ++s)
            issue_row<NV>(a, fin, ring, bar, (int)(s % NSLOT), tile_of(s), (int)(s % NV));
    }
    long long issued = std::min<long long>(LOOK, total);
    bool failed = false;
    for (int lt = 0; lt < ntl && !failed; ++lt) {
        const int tile = tile_of((long long)lt * NV);
        const int y = tile / a.ntx;
        const int xr = (tile % a.ntx) * TW + cell;
        const bool active = xr < a.nx;
        const int x = active ? xr : 0;
        float wx, wy;
        load_w<float>(a, x, y, wx, wy);
        if (chunk == 0) cfl_check<float, NV>(a, g, wx, wy, active);
        float A[WM], G[WM], H[WM];
#pragma unroll
        for (int j = 0; j < WM; ++j) {
            A[j] = 0.f;
            G[j] = 0.f;
            H[j] = 0.f;
        }
        float* out = fout + (size_t)y * a.nx + x;
        const long long s0 = (long long)lt * NV;
        for (int r = 0; r <= NV; ++r) {
            const long long s = s0 + r;
            // every thread is done with row s-2's slot and with the exchange values of row r-2;
            // a timeout anywhere stops the block
            if (__syncthreads_or(failed ? 1 : 0)) {
                failed = true;
                break;
            }
            if (r < NV) {
                // slot (s + LOOK) % NSLOT last held row s - 2, released by the barrier above
                if (tid < 32 && s + LOOK < total) {
#if LAT_RING_PROXY_FENCE
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
#endif
                    issue_row<NV>(a, fin, ring, bar, (int)((s + LOOK) % NSLOT),
                                  tile_of(s + LOOK), (int)((s + LOOK) % NV));
                }
                if (s + LOOK < total) issued = s + LOOK + 1;
                if (!mbar_wait_bounded(&bar[s % NSLOT], (unsigned)((s / NSLOT) & 1))) {
                    failed = true;
                    continue;
                }
            }
            if (r >= 1) {
                const RingRow<NV> cur{ring + (size_t)((s - 1) % NSLOT) * NV * WIN + cell};
                const RingRow<NV> nxt{ring + (size_t)(s % NSLOT) * NV * WIN + cell};
                float xl = 0.f, xrgt = 0.f;  // neighbouring chunks' f** of row r-2
                if (C > 1 && r >= 2) {
                    if (chunk > 0) xl = xch_at((r - 1) & 1, chunk - 1, 1);
                    if (chunk < C - 1) xrgt = xch_at((r - 1) & 1, chunk + 1, 0);
                }
                chunk_sweep<NV, C, WM>(chunk, A, G, H, r, cur, nxt, g, wx, wy, rr, xl, xrgt, out,
                                       ps, active, &xch_at(r & 1, chunk, 0),
                                       &xch_at(r & 1, chunk, 1));
            }
        }
        if (failed) break;
        float xl = 0.f, xrgt = 0.f;
        if (C > 1) {
            __syncthreads();
            if (chunk > 0) xl = xch_at(NV & 1, chunk - 1, 1);
            if (chunk < C - 1) xrgt = xch_at(NV & 1, chunk + 1, 0);
        }
        chunk_final<NV, C, WM>(chunk, A, H, rr, xl, xrgt, out, ps, active);
    }
    if (failed) {
        if (tid == 0) {
            atomicOr(&a.st->status, ST_TIMEOUT);
            // let the copies already issued land before the block's shared memory goes away
            for (long long s = std::max(0ll, issued - NSLOT); s < issued; ++s)
                mbar_wait_bounded(&bar[s % NSLOT], (unsigned)((s / NSLOT) & 1));
        }
        __syncthreads();
    }
}

// ---- producer/consumer kernel: no block-wide barrier per row ------------------------------------
// Four consumer warps own 128 cells (one cell column per thread, as in the plain kernel); a fifth
// warp only produces: it refills a ring slot as soon as every consumer warp has released it
// (per-slot "empty" mbarrier, one arrival per consumer warp) and the consumers wait only on the
// per-slot "full" mbarrier the bulk copies complete.  Warps drift freely within the ring's slack.
// With GSM the vy-drag flux row G lives in shared memory (private per thread) instead of
// registers, which lowers register pressure and raises occupancy.
// Producer warp of the producer/consumer kernels: fill f (row f % NV of the block's tile f / NV)
// goes to slot f % NS once the consumers released that slot's previous content (fill f - NS).
template <int NV, int NS, class TileOf, int GX = 0>
__device__ __forceinline__ void produce_rows(const Step2DArgs& a, const float* fin, float* ring,
                                             uint64_t* full, uint64_t* empty, long long total,
                                             const TileOf& tile_of,
                                             const float* gcorr = nullptr) {
    const int lane = threadIdx.x & 31;
    // a stalled context issues no copies: every consumer's bounded wait runs out
    const long long nfill = a.st->stall ? 0 : total;
    long long f = 0;
    for (; f < nfill; ++f) {
        const int q = (int)(f % NS);
        if (f >= NS && !mbar_wait_bounded(&empty[q], (unsigned)(((f / NS) + 1) & 1))) {
            if (lane == 0) atomicOr(&a.st->status, ST_TIMEOUT);
            break;
        }
        issue_row<NV, GX>(a, fin, ring, full, q, tile_of(f), (int)(f % NV), gcorr);
    }
    // the copies issued last must land before this warp leaves (the block may finish early)
    for (long long d = std::max(0ll, f - NS); d < f; ++d)
        mbar_wait_bounded(&full[d % NS], (unsigned)((d / NS) & 1));
}

// Moment outputs of a step that also reduces the moments of the state it writes (the FP32
// producer/consumer kernel with MOM): per-cell arrays as lat_moments (any may be null) and one
// compensated partial [4][2] per consumer warp.
struct Mom2DOut {
    double* rho = nullptr;
    double* mv = nullptr;
    double* mv2 = nullptr;
    double* partials = nullptr;
    double dv = 0.0;
};

// Output writer that also sums the written values of one cell in the order and precision of
// k_moments2d<float> (velocity rows in order, TwoSum row masses, FMA-weighted sums), so that
// the per-cell moments come out with the same bits.
template <int NV>
struct MomPut {
    static constexpr int J = (NV - 1) / 2;
    StorePut<float, NV> st;
    FComp s0, ey;
    float s1 = 0.f, s2 = 0.f, s3 = 0.f, ex = 0.f, fy = 0.f, fy2 = 0.f;
    int row = -1, jx = 0;
    __device__ __forceinline__ MomPut(float* out, size_t ps, bool act) : st(out, ps, act) {}
    __device__ __forceinline__ void close() {
        s0.merge(ey);
        s1 = __fadd_rn(s1, ex);
        s2 = __fmaf_rn(fy, __fsub_rn(ey.s, ey.c), s2);
    }
    __device__ __forceinline__ void begin(int r) {
        if (r != row) {  // sweep_row opens row 0 once without values, then again with them
            if (row >= 0) close();
            row = r;
            fy = (float)(r - J);
            fy2 = fy * fy;
            ey = FComp{};
            ex = 0.f;
        }
        jx = 0;
        st.begin(r);
    }
    __device__ __forceinline__ void operator()(float o) {  // jx = 0 .. NV - 1 in order
        st(o);
        const float fx = (float)(jx - J);
        ey.add_exact(o);
        ex = __fmaf_rn(fx, o, ex);
        s3 = __fmaf_rn(__fmaf_rn(fx, fx, fy2), o, s3);
        ++jx;
    }
};

template <int NV, int NS, bool GSM, bool HSM = false>
struct PCShape {
    static constexpr int consumers = TW / 32;
    static constexpr int threads = 32 * (consumers + 1);
    static constexpr int min_blocks = HSM ? (NS == 2 ? 3 : 2) : ((GSM && NS == 3) ? 3 : 2);
};

template <int NV, int NS, bool GSM, bool HSM = false, int GX = 0>
size_t pc_smem() {
    return (size_t)NS * ((size_t)NV * WIN + GX) * sizeof(float) +
           (GSM ? (size_t)NV * TW * sizeof(float) : 0) +
           (HSM ? (size_t)NV * TW * sizeof(float) : 0) + 2 * NS * sizeof(uint64_t);
}

// The corrections of one cell's row rb in the ring slot of f* row rb ([c][jx][cell] rows of TW,
// see issue_row): gx(rb, jx) through face jx + 1/2, gy(rb, jx) through face rb + 1/2.
template <int NV>
struct RingCorr {
    static constexpr bool active = true;
    const float* p;  // slot's corrections + cell
    template <typename T>
    __device__ __forceinline__ T gx(int, int jx) const { return p[jx * TW]; }
    template <typename T>
    __device__ __forceinline__ T gy(int, int jx) const { return p[(NV + jx) * TW]; }
};

// HSM: the vy-diffusion flux row H in shared memory too (fewer registers, no spills).
// MOM: the consumers also reduce the moments of the cells they write (Mom2DOut).
// CORR: the learned closure's corrected step, the corrections G [2][N_v^2][N_y][N_x] added to
// the interior drag fluxes (register rows only).
template <int NV, int NS, bool GSM, bool HSM, bool MOM, bool CORR = false>
__global__ void __launch_bounds__(PCShape<NV, NS, GSM, HSM>::threads,
                                  PCShape<NV, NS, GSM, HSM>::min_blocks)
    k_step2d_pc(const Step2DArgs a, int kstep, const Mom2DOut m, const float* gcorr) {
    static_assert(!CORR || (!GSM && !HSM && !MOM), "corrections with register rows only");
    constexpr int NC = PCShape<NV, NS, GSM, HSM>::consumers;
    constexpr int GX = CORR ? 2 * NV * TW : 0;       // correction rows per ring slot
    constexpr size_t SL = (size_t)NV * WIN + GX;  // floats per slot
    extern __shared__ __align__(128) unsigned char smem[];
    float* ring = reinterpret_cast<float*>(smem);
    float* gsm = ring + (size_t)NS * SL;
    float* hsm = gsm + (GSM ? NV * TW : 0);
    uint64_t* full = reinterpret_cast<uint64_t*>(hsm + (HSM ? NV * TW : 0));
    uint64_t* empty = full + NS;
    const long long step = a.st->step + kstep;
    const int par = (int)(step & 1);
    const float g = float(a.g), rr = float(a.r);
    const float* fin = static_cast<const float*>(par ? a.f[1] : a.f[0]);
    float* fout = static_cast<float*>(par ? a.f[0] : a.f[1]);
    const size_t ps = (size_t)a.nx * a.ny;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntl = a.ntiles > (int)blockIdx.x ? (a.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const long long total = (long long)ntl * NV;
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
        produce_rows<NV, NS, decltype(tile_of), GX>(a, fin, ring, full, empty, total, tile_of,
                                                    gcorr);
        return;
    }
    const int cell = threadIdx.x;
    bool failed = false, bad = false;
    FComp t[4];  // MOM: this thread's cells
    for (int lt = 0; lt < ntl && !failed; ++lt) {
        const int tile = tile_of((long long)lt * NV);
        const int y = tile / a.ntx;
        const int xr = (tile % a.ntx) * TW + cell;
        const bool active = xr < a.nx;
        const int x = active ? xr : 0;
        float wx, wy;
        load_w<float>(a, x, y, wx, wy);
        cfl_check<float, NV>(a, g, wx, wy, active);
        float A[NV], Hreg[NV], Greg[NV];
        SmemCol Gs{gsm + cell}, Hs{hsm + cell};
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            A[j] = 0.f;
            if (HSM) Hs[j] = 0.f;
            else Hreg[j] = 0.f;
            if (GSM) Gs[j] = 0.f;
            else Greg[j] = 0.f;
        }
        std::conditional_t<MOM, MomPut<NV>, StorePut<float, NV>> put(
            fout + (size_t)y * a.nx + x, ps, active);
        const long long s0 = (long long)lt * NV;
        for (int r = 0; r <= NV; ++r) {
            const long long s = s0 + r;
            if (r < NV && !mbar_wait_bounded(&full[s % NS], (unsigned)((s / NS) & 1))) {
                failed = true;
                break;
            }
            if (r >= 1) {
                const RingRow<NV> cur{ring + (size_t)((s - 1) % NS) * SL + cell};
                const RingRow<NV> nxt{ring + (size_t)(s % NS) * SL + cell};
                if constexpr (CORR) {  // the corrections of row r - 1 came with its f* row
                    const RingCorr<NV> rc{ring + (size_t)((s - 1) % NS) * SL +
                                          (size_t)NV * WIN + cell};
                    sweep_row<float, NV>(A, Greg, Hreg, r, cur, nxt, g, wx, wy, rr, put, rc);
                } else if constexpr (HSM) {
                    sweep_row<float, NV>(A, Gs, Hs, r, cur, nxt, g, wx, wy, rr, put);
                } else if constexpr (GSM) {
                    sweep_row<float, NV>(A, Gs, Hreg, r, cur, nxt, g, wx, wy, rr, put);
                } else {
                    sweep_row<float, NV>(A, Greg, Hreg, r, cur, nxt, g, wx, wy, rr, put);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[(s - 1) % NS]);  // row s - 1 is done
            }
        }
        if (!failed) {
            if constexpr (HSM) final_row<float, NV>(A, Hs, rr, put);
            else final_row<float, NV>(A, Hreg, rr, put);
            if constexpr (MOM) {
                if (active) {
                    put.close();
                    bad |= !isfinite(put.s0.s) || !isfinite(put.s3);
                    const long long c = (long long)y * a.nx + x, ncell = (long long)a.nx * a.ny;
                    if (m.rho || m.mv || m.mv2) {  // FP64 per cell only when asked for
                        const double dv2 = __dmul_rn(m.dv, m.dv);
                        const double m0 = nval(put.s0.to_comp(1.0));
                        if (m.rho) m.rho[c] = m0 * dv2;
                        if (m.mv) {
                            m.mv[c] = m0 != 0.0 ? __dmul_rn((double)put.s1, m.dv) / m0 : 0.0;
                            m.mv[ncell + c] = m0 != 0.0 ? __dmul_rn((double)put.s2, m.dv) / m0 : 0.0;
                        }
                        if (m.mv2) m.mv2[c] = m0 != 0.0 ? __dmul_rn((double)put.s3, dv2) / m0 : 0.0;
                    }
                    t[0].merge(put.s0);
                    t[1].merge(FComp{put.s1, 0.f});
                    t[2].merge(FComp{put.s2, 0.f});
                    t[3].merge(FComp{put.s3, 0.f});
                }
            }
        }
    }
    if (failed && lane == 0) atomicOr(&a.st->status, ST_TIMEOUT);
    if constexpr (MOM) {  // one partial per consumer warp, lanes folded in butterfly order
        if (bad) atomicOr(&a.st->status, ST_NUMERIC);
        for (int q = 0; q < 4; ++q) warp_reduce(t[q]);
        if (lane == 0) {
            const double sc[4] = {1.0, m.dv, m.dv, __dmul_rn(m.dv, m.dv)};
            double* p = m.partials + ((size_t)blockIdx.x * NC + warp) * 8;
            for (int q = 0; q < 4; ++q) {
                const Comp cq = t[q].to_comp(sc[q]);
                p[2 * q] = cq.s;
                p[2 * q + 1] = cq.c;
            }
        }
    }
}

// ---- flow: u = (d_y psi, -d_x psi) of psi = sum a_m cos(theta_m) --------------------------------

// Per-mode terms of the flow at step `step` into shared memory, sh = [M] cos phi, [M] sin phi
// (phases in FP64, terms stored as T), by threads t = t0, t0 + nt, ...; the writer also stores
// the next step's phases (unless the flow is frozen or the run is dry) and flags a missing
// noise row.  The caller synchronises the threads that read sh afterwards.
template <typename T>
__device__ __forceinline__ void flow_modes_prepare(const Flow2DArgs& a, long long step, T* sh,
                                                   int t, int nt, bool writer) {
    const int M = a.nmodes;
    const int par = (int)(step & 1);
    const double* ph = a.phase + (size_t)par * M;
    for (int m = t; m < M; m += nt) {
        if constexpr (sizeof(T) == 4) {
            // FP32 terms: the FP64 phase reduced to [-pi, pi] in FP64, then sincosf (FP64
            // arithmetic runs at a small fraction of FP32's here)
            constexpr double kTwoPi = 6.283185307179586;
            const double q = rint(__dmul_rn(ph[m], 1.0 / kTwoPi));
            float sf, cf;
            sincosf((float)__fma_rn(-q, kTwoPi, ph[m]), &sf, &cf);
            sh[m] = T(cf);
            sh[M + m] = T(sf);
        } else {
            double sd, cd;
            sincos(ph[m], &sd, &cd);
            sh[m] = T(cd);
            sh[M + m] = T(sd);
        }
    }
    if (writer && !a.frozen && !a.dry) {
        const long long row = step - a.st->noise_base;
        const bool have = row >= 0 && row < a.st->noise_rows;
        for (int m = t; m < M; m += nt) {
            const double xi = have ? a.noise[row * M + a.perm[m]] : 0.0;
            a.phase[(size_t)(par ^ 1) * M + m] = __dadd_rn(ph[m], __dmul_rn(a.walk, xi));
        }
        if (!have && t == 0) atomicOr(&a.st->status, ST_NOISE);
    }
}

// u = (d_y psi, -d_x psi) = sum over the modes of (c_x, c_y) sin(theta_m), theta_m =
// 2 pi (kx x / nx + ky y / ny) + phi_m.  With e^{i theta} = X_kx(x) Y_ky(y) e^{i phi} from the
// separable tables, sin(theta) = Im(X w), w = Y e^{i phi}: one block per row y forms
// W_m = (c_x w, c_y w) for every mode in shared memory, then each thread sums over the modes for
// its cells with four FMAs per mode.  Modes are sorted by kx and taken run by run (runs of equal
// kx), so a thread loads X_kx(x) once per run.  Explicit rounding throughout.
template <typename T>
__global__ void __launch_bounds__(256) k_flow2d(const Flow2DArgs a, int kstep) {
    using O = Ops<T>;
    extern __shared__ double sh_raw[];
    const int M = a.nmodes;
    T* sh = reinterpret_cast<T*>(sh_raw);   // [M] cos phi, [M] sin phi
    T* W = sh + 2 * M;                      // [M][4]: c_x w_re, c_x w_im, c_y w_re, c_y w_im
    const long long step = a.st->step + kstep;
    flow_modes_prepare<T>(a, step, sh, threadIdx.x, blockDim.x, blockIdx.x == 0);
    __syncthreads();
    const long long ncell = (long long)a.nx * a.ny;
    const T* xt = static_cast<const T*>(a.xtab);  // [kx + kmax][x][cos, sin] of 2 pi kx x / nx
    const T* yt = static_cast<const T*>(a.ytab);  // [ky + kmax][y][cos, sin] of 2 pi ky y / ny
    T* u = static_cast<T*>(a.u);
    for (int y = blockIdx.x; y < a.ny; y += gridDim.x) {
        for (int m = threadIdx.x; m < M; m += blockDim.x) {
            const int2 k = a.k[m];
            const T* Y = yt + 2 * ((size_t)(k.y + a.kmax) * a.ny + y);
            const T c = sh[m], s = sh[M + m];
            const T w0 = O::fma(Y[0], c, -O::mul(Y[1], s));
            const T w1 = O::fma(Y[0], s, O::mul(Y[1], c));
            const T cx = T(a.cx[m]), cy = T(a.cy[m]);
            W[4 * m] = O::mul(cx, w0);
            W[4 * m + 1] = O::mul(cx, w1);
            W[4 * m + 2] = O::mul(cy, w0);
            W[4 * m + 3] = O::mul(cy, w1);
        }
        __syncthreads();
        for (int x = threadIdx.x; x < a.nx; x += blockDim.x) {
            T ux = T(0), uy = T(0);
            for (int q = 0; q < a.nruns; ++q) {
                const int m0 = a.runs[2 * q], m1 = a.runs[2 * q + 2], kx = a.runs[2 * q + 1];
                const T* X = xt + 2 * ((size_t)(kx + a.kmax) * a.nx + x);
                const T X0 = X[0], X1 = X[1];
#pragma unroll 4
                for (int m = m0; m < m1; ++m) {
                    // Im(X w) (c_x, c_y) = X_re (c w_im) + X_im (c w_re)
                    ux = O::fma(X0, W[4 * m + 1], O::fma(X1, W[4 * m], ux));
                    uy = O::fma(X0, W[4 * m + 3], O::fma(X1, W[4 * m + 2], uy));
                }
            }
            u[(size_t)y * a.nx + x] = ux;
            u[ncell + (size_t)y * a.nx + x] = uy;
        }
        __syncthreads();
    }
}

// ---- packed producer/consumer kernel -----------------------------------------------------------
// The producer/consumer design with the packed two-lane sweep (step2d_x2.h): one producer warp
// fills the ring, four consumer warps sweep one cell each, holding a velocity row as two
// half-rows in f32x2 register pairs.  Same bits as every other FP32 launch variant.  GSM: the
// vy-drag flux pairs in shared memory instead of registers.
template <int NV, int NS, bool GSM>
struct PC2Shape {
    static constexpr int consumers = TW / 32;
    static constexpr int threads = 32 * (consumers + 1);
    static constexpr int min_blocks = GSM ? 3 : 2;
};

template <int NV, int NS, bool GSM>
size_t pc2_smem() {
    return (size_t)NS * NV * WIN * sizeof(float) +
           (GSM ? (size_t)Pairs<NV>::n * TW * sizeof(f2) : 0) + 2 * NS * sizeof(uint64_t);
}

template <int NV, int NS, bool GSM>
__global__ void __launch_bounds__(PC2Shape<NV, NS, GSM>::threads,
                                  PC2Shape<NV, NS, GSM>::min_blocks)
    k_step2d_pc2(const Step2DArgs a, int kstep) {
    constexpr int NC = PC2Shape<NV, NS, GSM>::consumers;
    constexpr int NP = Pairs<NV>::n;
    extern __shared__ __align__(128) unsigned char smem[];
    float* ring = reinterpret_cast<float*>(smem);
    f2* gsm = reinterpret_cast<f2*>(ring + (size_t)NS * NV * WIN);
    uint64_t* full = reinterpret_cast<uint64_t*>(gsm + (GSM ? NP * TW : 0));
    uint64_t* empty = full + NS;
    const long long step = a.st->step + kstep;
    const int par = (int)(step & 1);
    const float g = float(a.g), rr = float(a.r);
    const float* fin = static_cast<const float*>(par ? a.f[1] : a.f[0]);
    float* fout = static_cast<float*>(par ? a.f[0] : a.f[1]);
    const size_t ps = (size_t)a.nx * a.ny;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntl = a.ntiles > (int)blockIdx.x ? (a.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const long long total = (long long)ntl * NV;
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
        produce_rows<NV, NS>(a, fin, ring, full, empty, total, tile_of);
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
        f2 A[NP], Hd[NP], Greg[NP];
        SmemCol2 Gs{gsm + cell};
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            A[p] = 0ull;
            Hd[p] = 0ull;
            if (GSM) Gs[p] = 0ull;
            else Greg[p] = 0ull;
        }
        StorePut2<NV> put(fout + (size_t)y * a.nx + x, ps, active);
        const long long s0 = (long long)lt * NV;
        for (int r = 0; r <= NV; ++r) {
            const long long s = s0 + r;
            if (r < NV && !mbar_wait_bounded(&full[s % NS], (unsigned)((s / NS) & 1))) {
                failed = true;
                break;
            }
            if (r >= 1) {
                const RingRow<NV> cur{ring + (size_t)((s - 1) % NS) * NV * WIN + cell};
                const RingRow<NV> nxt{ring + (size_t)(s % NS) * NV * WIN + cell};
                if constexpr (GSM) sweep_row2<NV>(A, Gs, Hd, r, cur, nxt, g, wx, wy, rr, put);
                else sweep_row2<NV>(A, Greg, Hd, r, cur, nxt, g, wx, wy, rr, put);
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[(s - 1) % NS]);  // row s - 1 is done
            }
        }
        if (!failed) final_row2<NV>(A, Hd, rr, put);
    }
    if (failed && lane == 0) atomicOr(&a.st->status, ST_TIMEOUT);
}

// ---- moments ----------------------------------------------------------------------------------
using namespace cs;

template <typename T>
__device__ __forceinline__ double to_d(T v) { return (double)v; }

constexpr int kMom2DWarps = 8;  // warps per moment block (256 threads)

// Per cell: sums over the N_v^2 velocity cells of f, jx f, jy f, (jx^2 + jy^2) f; per-cell moments
// and one compensated partial per block: partials[block][4][2] (warps fold in warp order).
//   FP64 storage: Neumaier FP64 throughout.
//   FP32 / FP16 / BF16 storage: FP32 Kahan sums per cell and across a thread's cells and the
//   warp (exact integer weights); FP64 from the warp partials on (FP64 is slow on this GPU).
template <typename T>
__global__ void __launch_bounds__(256) k_moments2d(const void* fv, const float* scales, int nv,
                                                   int nx, int ny, double dv, double* rho,
                                                   double* mv, double* mv2, double* partials,
                                                   DevState* st) {
    const T* f = static_cast<const T*>(fv);
    const int J = (nv - 1) / 2;
    const long long ncell = (long long)nx * ny;
    const double dv2 = __dmul_rn(dv, dv);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double* p = partials + (size_t)blockIdx.x * 8;  // one partial per block
    bool bad = false;
    if constexpr (sizeof(T) == sizeof(double)) {
        Comp t[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
        for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
             c += (long long)gridDim.x * blockDim.x) {
            Comp s[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
            for (int jy = 0; jy < nv; ++jy) {
                const double vy = __dmul_rn((double)(jy - J), dv);
                for (int jx = 0; jx < nv; ++jx) {
                    const double vx = __dmul_rn((double)(jx - J), dv);
                    const size_t plane = (size_t)jy * nv + jx;
                    const double fvv = to_d(f[plane * ncell + c]);
                    bad |= !isfinite(fvv);
                    nadd(s[0], fvv);
                    nadd(s[1], __dmul_rn(vx, fvv));
                    nadd(s[2], __dmul_rn(vy, fvv));
                    nadd(s[3], __dmul_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)), fvv));
                }
            }
            const double m0 = nval(s[0]);
            if (rho) rho[c] = m0 * dv * dv;
            if (mv) {
                mv[c] = m0 != 0.0 ? nval(s[1]) / m0 : 0.0;
                mv[ncell + c] = m0 != 0.0 ? nval(s[2]) / m0 : 0.0;
            }
            if (mv2) mv2[c] = m0 != 0.0 ? nval(s[3]) / m0 : 0.0;
            for (int q = 0; q < 4; ++q) nmerge(t[q], s[q]);
        }
        for (int q = 0; q < 4; ++q) warp_reduce(t[q]);
        __shared__ Comp wsum[kMom2DWarps][4];
        if (lane == 0)
            for (int q = 0; q < 4; ++q) wsum[warp][q] = t[q];
        __syncthreads();
        if (threadIdx.x == 0)
            for (int q = 0; q < 4; ++q) {
                Comp z = wsum[0][q];
                for (int w = 1; w < kMom2DWarps; ++w) nmerge(z, wsum[w][q]);
                p[2 * q] = z.s;
                p[2 * q + 1] = z.c;
            }
    } else {
        // per cell: the mass exact up to the roundings of its compensation (TwoSum per velocity
        // row, rows merged); the weighted sums one FMA per value (the integer weights exact, the
        // product exact inside the FMA), error at most (N_v^2 - 1) u of the sum of
        // |weight f|, u = 2^-24
        FComp t[4];
        for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
             c += (long long)gridDim.x * blockDim.x) {
            FComp s0;
            float s1 = 0.f, s2 = 0.f, s3 = 0.f;
            // scales of this cell's row: [jy][jx padded]
            const float* sc_c = scales ? scales + (size_t)(c / nx) * nv * nv_padded(nv) : nullptr;
            for (int jy = 0; jy < nv; ++jy) {
                const float fy = (float)(jy - J);
                const float fy2 = fy * fy;
                FComp ey;         // sum f of the velocity row
                float ex = 0.f;   // sum jx f of the velocity row
#pragma unroll 4
                for (int jx = 0; jx < nv; ++jx) {
                    const float fx = (float)(jx - J);
                    const size_t plane = (size_t)jy * nv + jx;
                    float fvv = (float)f[plane * ncell + c];
                    if (sc_c) fvv = fvv * sc_c[jy * nv_padded(nv) + jx];  // exact: powers of two
                    ey.add_exact(fvv);
                    ex = __fmaf_rn(fx, fvv, ex);
                    s3 = __fmaf_rn(__fmaf_rn(fx, fx, fy2), fvv, s3);
                }
                s0.merge(ey);
                s1 = __fadd_rn(s1, ex);
                s2 = __fmaf_rn(fy, __fsub_rn(ey.s, ey.c), s2);
            }
            bad |= !isfinite(s0.s) || !isfinite(s3);
            if (rho || mv || mv2) {  // FP64 per cell only when asked for (FP64 is slow here)
                const double m0 = nval(s0.to_comp(1.0));
                if (rho) rho[c] = m0 * dv2;
                if (mv) {
                    mv[c] = m0 != 0.0 ? __dmul_rn((double)s1, dv) / m0 : 0.0;
                    mv[ncell + c] = m0 != 0.0 ? __dmul_rn((double)s2, dv) / m0 : 0.0;
                }
                if (mv2) mv2[c] = m0 != 0.0 ? __dmul_rn((double)s3, dv2) / m0 : 0.0;
            }
            t[0].merge(s0);
            t[1].merge(FComp{s1, 0.f});
            t[2].merge(FComp{s2, 0.f});
            t[3].merge(FComp{s3, 0.f});
        }
        for (int q = 0; q < 4; ++q) warp_reduce(t[q]);
        __shared__ FComp wsum[kMom2DWarps][4];
        if (lane == 0)
            for (int q = 0; q < 4; ++q) wsum[warp][q] = t[q];
        __syncthreads();
        if (threadIdx.x == 0) {
            const double sc[4] = {1.0, dv, dv, dv2};
            for (int q = 0; q < 4; ++q) {
                FComp z = wsum[0][q];
                for (int w = 1; w < kMom2DWarps; ++w) z.merge(wsum[w][q]);
                const Comp cq = z.to_comp(sc[q]);
                p[2 * q] = cq.s;
                p[2 * q + 1] = cq.c;
            }
        }
    }
    if (bad) atomicOr(&st->status, ST_NUMERIC);
}

// One block of kFin2DThreads folds the block partials: thread i takes partials i, i + 256, ...,
// then warp butterflies and warp 0 folds the warps in order.
constexpr int kFin2DThreads = 256;
__global__ void __launch_bounds__(kFin2DThreads)
    k_finalize2d(const double* partials, int npart, double w, double* glob) {
    __shared__ Comp wsum[kFin2DThreads / 32][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Comp t[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (int b = threadIdx.x; b < npart; b += kFin2DThreads)
        for (int q = 0; q < 4; ++q) nmerge(t[q], Comp{partials[b * 8 + 2 * q], partials[b * 8 + 2 * q + 1]});
    for (int q = 0; q < 4; ++q) warp_reduce(t[q]);
    if (lane == 0)
        for (int q = 0; q < 4; ++q) wsum[warp][q] = t[q];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int q = 0; q < 4; ++q) {
            Comp z = wsum[0][q];
            for (int v = 1; v < kFin2DThreads / 32; ++v) nmerge(z, wsum[v][q]);
            glob[q] = nval(z) * w;
        }
}

__global__ void k_set_noise2d(DevState* st, long long base, long long rows) {
    st->noise_base = base;
    st->noise_rows = rows;
}

__global__ void k_advance2d(DevState* st, long long n) { st->step += n; }

// ---- launch tables ----------------------------------------------------------------------------
template <int NV, int C>
size_t ring_smem() {
    return (size_t)NSLOT * NV * WIN * sizeof(float) + (size_t)2 * C * 2 * TW * sizeof(float) +
           NSLOT * sizeof(uint64_t);
}

template <typename T, int NV>
cudaError_t launch_plain(int grid, const Step2DArgs& a, int k, cudaStream_t s) {
    k_step2d_plain<T, NV><<<grid, TW, 0, s>>>(a, k);
    return cudaGetLastError();
}

template <int NV, int C>
cudaError_t launch_ring(int grid, const Step2DArgs& a, int k, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_step2d_ring<NV, C>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)ring_smem<NV, C>());
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_step2d_ring<NV, C><<<grid, RingShape<NV, C>::threads, ring_smem<NV, C>(), s>>>(a, k);
    return cudaGetLastError();
}

template <int NV, int C>
int occupancy_ring_t() {
    int nb = 0;
    cudaFuncSetAttribute(k_step2d_ring<NV, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)ring_smem<NV, C>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step2d_ring<NV, C>,
                                                  RingShape<NV, C>::threads, ring_smem<NV, C>());
    return nb;
}

#define LAT2D_NV_LIST(X) X(1) X(3) X(5) X(9) X(13) X(17) X(19) X(21) X(33)
// velocity lattices whose columns may be split over several warp groups
#define LAT2D_SPLIT(n) ((n) >= 17)

bool nv2d_supported(int nv) {
    switch (nv) {
#define X(n) case n:
        LAT2D_NV_LIST(X)
#undef X
        return true;
        default: return false;
    }
}

bool chunks_supported(int nv, int chunks) {
    return chunks == 1 || (chunks >= 2 && chunks <= 4 && LAT2D_SPLIT(nv));
}

template <int NV>
cudaError_t launch_ring_c(int chunks, int grid, const Step2DArgs& a, int k, cudaStream_t s) {
    if constexpr (LAT2D_SPLIT(NV)) {
        if (chunks == 2) return launch_ring<NV, 2>(grid, a, k, s);
        if (chunks == 3) return launch_ring<NV, 3>(grid, a, k, s);
        if (chunks == 4) return launch_ring<NV, 4>(grid, a, k, s);
    }
    if (chunks == 1) return launch_ring<NV, 1>(grid, a, k, s);
    return cudaErrorInvalidValue;
}

template <int NV>
int occupancy_ring_c(int chunks) {
    if constexpr (LAT2D_SPLIT(NV)) {
        if (chunks == 2) return occupancy_ring_t<NV, 2>();
        if (chunks == 3) return occupancy_ring_t<NV, 3>();
        if (chunks == 4) return occupancy_ring_t<NV, 4>();
    }
    if (chunks == 1) return occupancy_ring_t<NV, 1>();
    return 0;
}

// Producer/consumer variants: 3 = G in registers, 4-slot ring; 4 = G in shared memory, 4 slots;
// 5 = G in shared memory, 3 slots; 6 = G and H in shared memory, 3 slots; 7 = the same, 2 slots.
#define LAT2D_PC(n) ((n) >= 9)

template <int NV, int NS, bool GSM, bool HSM = false, bool MOM = false>
cudaError_t launch_pc(int grid, const Step2DArgs& a, int k, cudaStream_t s,
                      const Mom2DOut& m = Mom2DOut()) {
    static bool attr = false;
    const size_t bytes = pc_smem<NV, NS, GSM, HSM>();
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_step2d_pc<NV, NS, GSM, HSM, MOM>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)bytes);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_step2d_pc<NV, NS, GSM, HSM, MOM>
        <<<grid, PCShape<NV, NS, GSM, HSM>::threads, bytes, s>>>(a, k, m, nullptr);
    return cudaGetLastError();
}

// The learned closure's corrected step on the bulk-copy ring (kernel 3's shape: four slots,
// register rows), as many resident blocks as fit.
template <int NV>
cudaError_t launch_pc_corr_t(int sm_count, const Step2DArgs& a, const float* G, int k,
                             cudaStream_t s) {
    static int occ = 0;
    const size_t bytes = pc_smem<NV, 4, false, false, 2 * NV * TW>();
    if (occ == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_step2d_pc<NV, 4, false, false, false, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)bytes);
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &nb, k_step2d_pc<NV, 4, false, false, false, true>, PCShape<NV, 4, false, false>::threads,
            bytes);
        if (e != cudaSuccess) return e;
        occ = nb > 0 ? nb : 1;
    }
    const int grid = std::max(1, std::min(a.ntiles, occ * sm_count));
    k_step2d_pc<NV, 4, false, false, false, true>
        <<<grid, PCShape<NV, 4, false, false>::threads, bytes, s>>>(a, k, Mom2DOut(), G);
    return cudaGetLastError();
}

// The corrected step on the ring for the learned lattices it is built for (N_v = 9, 13, 17);
// cudaErrorNotSupported otherwise.
cudaError_t launch_corr_ring(int nv, int sm_count, const Step2DArgs& a, const float* G, int k,
                             cudaStream_t s) {
    switch (nv) {
        case 9: return launch_pc_corr_t<9>(sm_count, a, G, k, s);
        case 13: return launch_pc_corr_t<13>(sm_count, a, G, k, s);
        case 17: return launch_pc_corr_t<17>(sm_count, a, G, k, s);
        default: return cudaErrorNotSupported;
    }
}

template <int NV, int NS, bool GSM, bool HSM = false, bool MOM = false>
int occupancy_pc_t() {
    int nb = 0;
    const size_t bytes = pc_smem<NV, NS, GSM, HSM>();
    cudaFuncSetAttribute(k_step2d_pc<NV, NS, GSM, HSM, MOM>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step2d_pc<NV, NS, GSM, HSM, MOM>,
                                                  PCShape<NV, NS, GSM, HSM>::threads, bytes);
    return nb;
}

// Variants 4 and 5 with the moment epilogue: the grid of its own resident blocks (at most bps
// per SM when bps > 0), so that no block waits for a free slot.
template <int NV>
cudaError_t launch_pc_mom(int v, int bps, int sm_count, const Step2DArgs& a, int k,
                          const Mom2DOut& m, int* grid_out, cudaStream_t s) {
    if constexpr (LAT2D_PC(NV)) {
        if (v == 4 || v == 5) {
            int occ = v == 4 ? occupancy_pc_t<NV, 4, true, false, true>()
                             : occupancy_pc_t<NV, 3, true, false, true>();
            occ = std::max(1, bps > 0 ? std::min(bps, occ) : occ);
            const int grid = std::max(1, std::min(a.ntiles, occ * sm_count));
            *grid_out = grid;
            return v == 4 ? launch_pc<NV, 4, true, false, true>(grid, a, k, s, m)
                          : launch_pc<NV, 3, true, false, true>(grid, a, k, s, m);
        }
    }
    return cudaErrorInvalidValue;
}

template <int NV, int NS, bool GSM>
cudaError_t launch_pc2(int grid, const Step2DArgs& a, int k, cudaStream_t s) {
    static bool attr = false;
    const size_t bytes = pc2_smem<NV, NS, GSM>();
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_step2d_pc2<NV, NS, GSM>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)bytes);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_step2d_pc2<NV, NS, GSM><<<grid, PC2Shape<NV, NS, GSM>::threads, bytes, s>>>(a, k);
    return cudaGetLastError();
}

template <int NV, int NS, bool GSM>
int occupancy_pc2_t() {
    int nb = 0;
    const size_t bytes = pc2_smem<NV, NS, GSM>();
    cudaFuncSetAttribute(k_step2d_pc2<NV, NS, GSM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)bytes);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step2d_pc2<NV, NS, GSM>,
                                                  PC2Shape<NV, NS, GSM>::threads, bytes);
    return nb;
}

template <int NV>
cudaError_t launch_pc_v(int v, int grid, const Step2DArgs& a, int k, cudaStream_t s) {
    if constexpr (LAT2D_PC(NV)) {
        if (v == 8) return launch_pc2<NV, 3, false>(grid, a, k, s);
        if (v == 9) return launch_pc2<NV, 3, true>(grid, a, k, s);
        if (v == 10) return launch_pc2<NV, 2, true>(grid, a, k, s);
        if (v == 3) return launch_pc<NV, 4, false>(grid, a, k, s);
        if (v == 4) return launch_pc<NV, 4, true>(grid, a, k, s);
        if (v == 5) return launch_pc<NV, 3, true>(grid, a, k, s);
        if (v == 6) return launch_pc<NV, 3, true, true>(grid, a, k, s);
        if (v == 7) return launch_pc<NV, 2, true, true>(grid, a, k, s);
    }
    return cudaErrorInvalidValue;
}

template <int NV>
int occupancy_pc_v(int v) {
    if constexpr (LAT2D_PC(NV)) {
        if (v == 8) return occupancy_pc2_t<NV, 3, false>();
        if (v == 9) return occupancy_pc2_t<NV, 3, true>();
        if (v == 10) return occupancy_pc2_t<NV, 2, true>();
        if (v == 3) return occupancy_pc_t<NV, 4, false>();
        if (v == 4) return occupancy_pc_t<NV, 4, true>();
        if (v == 5) return occupancy_pc_t<NV, 3, true>();
        if (v == 6) return occupancy_pc_t<NV, 3, true, true>();
        if (v == 7) return occupancy_pc_t<NV, 2, true, true>();
    }
    return 0;
}

bool pc_supported(int nv) {
    switch (nv) {
#define X(n) \
    case n: return LAT2D_PC(n);
        LAT2D_NV_LIST(X)
#undef X
        default: return false;
    }
}

cudaError_t launch_step2d(int dtype, int nv, bool ring, int chunks, int pcv, int grid,
                          const Step2DArgs& a, int k, cudaStream_t s) {
    switch (nv) {
#define X(n)                                                                   \
    case n:                                                                    \
        if (dtype == LAT_F64) return launch_plain<double, n>(grid, a, k, s);   \
        if (ring && pcv) return launch_pc_v<n>(pcv, grid, a, k, s);            \
        if (ring) return launch_ring_c<n>(chunks, grid, a, k, s);              \
        return launch_plain<float, n>(grid, a, k, s);
        LAT2D_NV_LIST(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step2d_mom(int nv, int pcv, int bps, int sm_count, const Step2DArgs& a, int k,
                              const Mom2DOut& m, int* grid_out, cudaStream_t s) {
    switch (nv) {
#define X(n) \
    case n: return launch_pc_mom<n>(pcv, bps, sm_count, a, k, m, grid_out, s);
        LAT2D_NV_LIST(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

int occupancy_ring(int nv, int chunks, int pcv) {
    switch (nv) {
#define X(n) \
    case n: return pcv ? occupancy_pc_v<n>(pcv) : occupancy_ring_c<n>(chunks);
        LAT2D_NV_LIST(X)
#undef X
        default: return 0;
    }
}

}  // namespace

// ---- context ----------------------------------------------------------------------------------
struct Ctx2D {
    int nx, ny, nv, dtype;
    double L, dx, dv, g, r, dt;
    DevState* st;
    int sm_count;
    // flow
    int flow_kind = LAT_FLOW_NONE;
    const void* field = nullptr;
    int nmodes = 0;
    int2* d_k = nullptr;      // modes sorted by kx (see k_flow2d)
    int* d_perm = nullptr;    // caller's index of each mode (noise columns)
    int* d_runs = nullptr;    // runs of equal kx among the sorted modes ([nruns + 1][2])
    int nruns = 0;
    double* d_cx = nullptr;
    double* d_cy = nullptr;
    double* d_phase = nullptr;
    void* d_xtab = nullptr;   // separable flow tables (see k_flow2d)
    void* d_ytab = nullptr;
    int kmax = 0;
    double* d_noise = nullptr;
    long long noise_cap = 0;
    double walk = 0.0;
    bool frozen = true;
    void* d_u = nullptr;
    // launch
    bool ring = false;
    int chunks = 1;    // warp groups per cell column in the ring kernel
    int pcv = 0;       // 0: ring kernel; 3..7: producer/consumer variant
    int bps = 0;       // 0 = occupancy limit
    int mode = 0;      // 0 graph, 2 direct launches
    // reduced-precision storage: per-line scales and maxima, [2][N_v^2 N_y] each
    bool half = false;
    long long nlines = 0;  // scales (or maxima) per buffer, padded layout
    float* d_sc = nullptr;
    unsigned* d_mx = nullptr;
    // learned flux closure: 0 off, 1 FP32 network on CUDA cores, 2 BF16 network on tensor cores
    int learn = 0;
    float* d_params = nullptr;   // [kLNParam] FP32
    void* d_wtc = nullptr;       // tensor-core weight tiles (BF16) and biases
    float* d_rho = nullptr;      // [ny][nx]
    float4* d_feat = nullptr;    // [ny][nx][2]: spatial parts of the features (BF16 network)
    // drag scheme: upwind (the fused kernels) or flux-limited (limiter2d.cu: one fused kernel,
    // or three passes with the scratch state d_lim)
    int scheme = LAT_SCHEME_UPWIND;
    double mu = 2.0 / 3.0;
    int lim_kernel = 0;  // limited step: 0 the fastest form, 1 three passes, 2 fused, 3 packed
    int lim_bps = 2;     // blocks per SM of the fused limited kernel, where two shapes exist
    void* d_lim = nullptr;
    float* d_G = nullptr;        // [2][N_v^2][ny][nx]
    DevState* d_st0 = nullptr;   // step 0, no flags: explicit-buffer rollouts
    // moments
    double* d_partials = nullptr;
    double* d_glob = nullptr;
    double* h_glob = nullptr;
    int mom_blocks = 0;
    std::map<int, cudaGraphExec_t> graphs;
};

namespace {

int cuda_err(cudaError_t e, const char* what) {
    fprintf(stderr, "lat(2d): %s failed: %s\n", what, cudaGetErrorString(e));
    return LAT_ECUDA;
}
#define CK2(call)                                               \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_err(e_, #call);      \
    } while (0)

void drop(Ctx2D* c) {
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
}

bool ring_ok(const Ctx2D* c) {
    if (c->half) return h2d_ring_ok(c->nx);
    return c->dtype == LAT_F32 && c->nx % 4 == 0 && c->nx >= WIN;
}

bool pc_ok(const Ctx2D* c) { return c->half ? c->nv >= 9 : pc_supported(c->nv); }

// Launch form of the flux-limited step (1 three passes, 2 fused, 3 fused on FP32 register
// pairs): the caller's choice, else the packed form for FP32 and the fused one for FP64 where
// the kernels are built for N_v, else the three passes.
int lim_form(const Ctx2D* c) {
    if (!limiter2d_fused_supported(c->nv)) return 1;
    if (c->lim_kernel) return c->lim_kernel;
    return c->dtype == LAT_F32 ? 3 : 2;
}

// The three passes' scratch state, allocated while they are the limited scheme's launch form.
int lim_scratch(Ctx2D* c) {
    if (c->scheme != LAT_SCHEME_KOREN || lim_form(c) != 1 || c->d_lim) return LAT_OK;
    const size_t bytes =
        (size_t)c->nx * c->ny * c->nv * c->nv * (c->dtype == LAT_F64 ? 8 : 4);
    if (cudaMalloc(&c->d_lim, bytes) != cudaSuccess) {
        c->d_lim = nullptr;
        return LAT_ENOMEM;
    }
    return LAT_OK;
}

Step2DHArgs half_args(const Ctx2D* c, const Step2DArgs& a) {
    Step2DHArgs h;
    h.b = a;
    h.sc[0] = c->d_sc;
    h.sc[1] = c->d_sc + c->nlines;
    h.mx[0] = c->d_mx;
    h.mx[1] = c->d_mx + c->nlines;
    return h;
}

Step2DArgs step_args(const Ctx2D* c, void* const f[2]) {
    Step2DArgs a;
    memset(&a, 0, sizeof(a));
    a.f[0] = f[0];
    a.f[1] = f[1];
    a.nx = c->nx;
    a.ny = c->ny;
    a.g = c->g;
    a.r = c->r;
    a.inv_dv = 1.0 / c->dv;
    a.u = c->flow_kind == LAT_FLOW_FIELD ? c->field : (c->flow_kind == LAT_FLOW_MODES ? c->d_u : nullptr);
    a.st = c->st;
    a.ntx = (c->nx + TW - 1) / TW;
    a.ntiles = a.ntx * c->ny;
    return a;
}

int grid_of(const Ctx2D* c, int ntiles) {
    int per_sm = c->bps;
    if (c->ring) {
        const int occ = c->half ? occupancy_step2d_h(c->dtype, c->nv, c->pcv)
                                : occupancy_ring(c->nv, c->chunks, c->pcv);
        if (per_sm <= 0 || per_sm > occ) per_sm = std::max(1, occ);
    } else if (per_sm <= 0) {
        per_sm = 8;
    }
    return std::max(1, std::min(ntiles, per_sm * c->sm_count));
}

// Enqueue n steps.  Dry runs (autotuning) repeat step 0 n times: every repetition reads the
// current buffer and writes the other one, so the state and the flow are left as they were.
// Flow of step st->step + k into d_u (modal flow only); the phases of the following step are
// written unless dry.
Flow2DArgs flow_args(const Ctx2D* c, int dry) {
    Flow2DArgs fa;
    fa.k = c->d_k;
    fa.perm = c->d_perm;
    fa.runs = c->d_runs;
    fa.nruns = c->nruns;
    fa.cx = c->d_cx;
    fa.cy = c->d_cy;
    fa.phase = c->d_phase;
    fa.noise = c->d_noise;
    fa.walk = c->walk;
    fa.xtab = c->d_xtab;
    fa.ytab = c->d_ytab;
    fa.kmax = c->kmax;
    fa.nmodes = c->nmodes;
    fa.nx = c->nx;
    fa.ny = c->ny;
    fa.u = c->d_u;
    fa.st = c->st;
    fa.frozen = c->frozen ? 1 : 0;
    fa.dry = dry;
    return fa;
}

int launch_flow(Ctx2D* c, int k, int dry, cudaStream_t s) {
    const Flow2DArgs fa = flow_args(c, dry);
    const int fg = std::max(1, std::min(c->ny, 4 * c->sm_count));  // rows per block: grid stride
    const size_t sh = 6 * sizeof(double) * c->nmodes;
    if (c->dtype == LAT_F64) k_flow2d<double><<<fg, 256, sh, s>>>(fa, k);
    else k_flow2d<float><<<fg, 256, sh, s>>>(fa, k);
    CK2(cudaGetLastError());
    return LAT_OK;
}

LearnArgs learn_args(const Ctx2D* c, const void* f0, const void* f1, const DevState* st) {
    LearnArgs la;
    la.f[0] = static_cast<const float*>(f0);
    la.f[1] = static_cast<const float*>(f1);
    la.u = c->flow_kind == LAT_FLOW_FIELD ? static_cast<const float*>(c->field)
                                          : static_cast<const float*>(c->d_u);
    la.rho = c->d_rho;
    la.feat = c->d_feat;
    la.params = c->d_params;
    la.G = c->d_G;
    la.st = st;
    la.nx = c->nx;
    la.ny = c->ny;
    la.g = (float)c->g;
    la.inv_dv = (float)(1.0 / c->dv);
    la.dt_2dx = (float)(c->dt / (2.0 * c->dx));
    return la;
}

// The corrected step of the learned closure: on the bulk-copy ring when the context's launch
// uses the ring and the kernel is built for N_v, else with plain loads (the same bits).
cudaError_t launch_corrected(const Ctx2D* c, const Step2DArgs& a, int k, cudaStream_t s) {
    if (c->ring && ring_ok(c) && (c->nv == 9 || c->nv == 13 || c->nv == 17))
        return launch_corr_ring(c->nv, c->sm_count, a, c->d_G, k, s);
    return launch_step2d_corr(c->nv, c->sm_count, a, c->d_G, k, s);
}

// One learned step from the buffers of a (parity from a.st): flow, density, network, step.
int enqueue_learned(Ctx2D* c, const Step2DArgs& a, int k, cudaStream_t s) {
    const LearnArgs la = learn_args(c, a.f[0], a.f[1], a.st);
    CK2(launch_rho_star(c->nv, la, k, s));
    if (c->learn == 2) CK2(launch_mlp_tc(c->nv, la, c->d_wtc, c->sm_count, c->ring, k, s));
    else CK2(launch_mlp_f32(c->nv, la, k, s));
    CK2(launch_corrected(c, a, k, s));
    return LAT_OK;
}

int enqueue2d(Ctx2D* c, void* const f[2], int n, cudaStream_t s, int dry) {
    const Step2DArgs a = step_args(c, f);
    const int grid = grid_of(c, a.ntiles);
    for (int kk = 0; kk < n; ++kk) {
        const int k = dry ? 0 : kk;
        if (c->flow_kind == LAT_FLOW_MODES) {
            const int rc = launch_flow(c, k, dry, s);
            if (rc != LAT_OK) return rc;
        }
        if (c->learn) {
            const int rc = enqueue_learned(c, a, k, s);
            if (rc != LAT_OK) return rc;
        } else if (c->scheme == LAT_SCHEME_KOREN) {
            CK2(launch_step2d_limited(c->dtype, a, c->nv, c->mu, c->d_lim, lim_form(c),
                                      c->lim_bps, k, c->sm_count, s));
        } else if (c->half) {
            const Step2DHArgs ha = half_args(c, a);
            CK2(launch_scale2d(c->nv, c->ny, ha, k, s));
            CK2(launch_step2d_h(c->dtype, c->nv, c->ring ? c->pcv : 0, grid, ha, k, s));
        } else {
            CK2(launch_step2d(c->dtype, c->nv, c->ring, c->chunks, c->pcv, grid, a, k, s));
        }
    }
    if (!dry) {
        k_advance2d<<<1, 1, 0, s>>>(c->st, n);
        CK2(cudaGetLastError());
    }
    return LAT_OK;
}

int graph2d(Ctx2D* c, void* const f[2], int n, cudaGraphExec_t* out) {
    auto it = c->graphs.find(n);
    if (it == c->graphs.end()) {
        cudaStream_t cap;
        CK2(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cap);
            return cuda_err(e, "cudaStreamBeginCapture");
        }
        int rc = enqueue2d(c, f, n, cap, 0);
        e = cudaStreamEndCapture(cap, &g);
        cudaStreamDestroy(cap);
        if (rc != LAT_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_err(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_err(e, "cudaGraphInstantiate");
        if (c->graphs.size() >= 8) drop(c);
        it = c->graphs.emplace(n, ge).first;
    }
    *out = it->second;
    return LAT_OK;
}

}  // namespace

int ctx2d_create(Ctx2D** out, const lat_grid* g, DevState* st, int sm_count, cudaStream_t s) {
    *out = nullptr;
    if (!nv2d_supported(g->nv)) return LAT_EINVAL;
    const bool half = g->dtype == LAT_F16 || g->dtype == LAT_BF16;
    if (g->dtype != LAT_F32 && g->dtype != LAT_F64 && !half) return LAT_EINVAL;
    if (half && !h2d_supported(g->nv)) return LAT_EINVAL;
    Ctx2D* c = new Ctx2D();
    c->half = half;
    c->nx = g->nx;
    c->ny = g->ny;
    c->nv = g->nv;
    c->dtype = g->dtype;
    c->L = g->L;
    c->dx = g->L / g->nx;
    c->dt = g->dt;
    c->dv = c->dx / g->dt;
    c->g = isinf(g->tau_p) ? 0.0 : g->dt / g->tau_p;
    c->r = g->kappa * g->dt / (c->dv * c->dv);
    c->st = st;
    c->sm_count = sm_count;
    c->ring = ring_ok(c);
    c->chunks = chunks_supported(c->nv, 3) ? 3 : 1;
    c->pcv = c->ring && pc_ok(c) ? (half ? 6 : 9) : 0;
    if (half && !c->pcv) c->ring = false;
    const long long ncell = (long long)c->nx * c->ny;
    c->mom_blocks = (int)std::min<long long>((ncell + 255) / 256, 8LL * sm_count);
    // room for the moment kernel's block partials or the fused step's warp partials
    const size_t npart = std::max<size_t>(c->mom_blocks, (size_t)8 * sm_count * (TW / 32));
    if (cudaMalloc(&c->d_partials, sizeof(double) * 8 * npart) != cudaSuccess ||
        cudaMalloc(&c->d_glob, sizeof(double) * 4) != cudaSuccess ||
        cudaMallocHost(&c->h_glob, sizeof(double) * 4) != cudaSuccess) {
        ctx2d_destroy(c);
        return LAT_ENOMEM;
    }
    if (half) {
        c->nlines = scale_count(c->nv, c->ny);
        if (cudaMalloc(&c->d_sc, sizeof(float) * 2 * c->nlines) != cudaSuccess ||
            cudaMalloc(&c->d_mx, sizeof(unsigned) * 2 * c->nlines) != cudaSuccess) {
            ctx2d_destroy(c);
            return LAT_ENOMEM;
        }
        cudaError_t e = launch_fill_scales(c->d_sc, 2 * c->nlines, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->d_mx, 0, sizeof(unsigned) * 2 * c->nlines, s);
        if (e != cudaSuccess) {
            ctx2d_destroy(c);
            return cuda_err(e, "scale initialisation");
        }
    }
    *out = c;
    return LAT_OK;
}

int ctx2d_set_flow(Ctx2D* c, const lat_flow* fl, bool frozen, cudaStream_t s) {
    drop(c);
    if (fl->kind == LAT_FLOW_NONE) {
        c->flow_kind = LAT_FLOW_NONE;
    } else if (fl->kind == LAT_FLOW_FIELD) {
        if (!fl->field) return LAT_EINVAL;
        c->flow_kind = LAT_FLOW_FIELD;
        c->field = fl->field;
    } else if (fl->kind == LAT_FLOW_MODES) {
        const int M = fl->nmodes;
        if (M < 1 || M > kMaxModes2D || !fl->k || !fl->amp0 || !fl->phase0) return LAT_EINVAL;
        // modes in ascending kx (stable), so that the flow kernel loads each x table row once
        std::vector<int> perm(M);
        for (int m = 0; m < M; ++m) perm[m] = m;
        std::stable_sort(perm.begin(), perm.end(),
                         [&](int i, int j) { return fl->k[2 * i] < fl->k[2 * j]; });
        std::vector<int2> k(M);
        std::vector<double> cx(M), cy(M), ph(2 * M);
        const double Lx = c->nx * c->dx, Ly = c->ny * c->dx;
        for (int m = 0; m < M; ++m) {
            const int q = perm[m];
            k[m] = make_int2(fl->k[2 * q], fl->k[2 * q + 1]);
            cx[m] = -fl->amp0[q] * (2.0 * M_PI * k[m].y / Ly);
            cy[m] = fl->amp0[q] * (2.0 * M_PI * k[m].x / Lx);
            ph[m] = fl->phase0[q];
            ph[M + m] = fl->phase0[q];
        }
        cudaFree(c->d_k);
        cudaFree(c->d_cx);
        cudaFree(c->d_cy);
        cudaFree(c->d_phase);
        c->d_k = nullptr;
        c->d_cx = c->d_cy = c->d_phase = nullptr;
        cudaFree(c->d_perm);
        c->d_perm = nullptr;
        if (cudaMalloc(&c->d_perm, sizeof(int) * M) != cudaSuccess) return LAT_ENOMEM;
        CK2(cudaMemcpy(c->d_perm, perm.data(), sizeof(int) * M, cudaMemcpyHostToDevice));
        // runs of equal kx: [first mode, kx] per run, then [M, 0]
        std::vector<int> runs;
        for (int m = 0; m < M; ++m)
            if (m == 0 || k[m].x != k[m - 1].x) {
                runs.push_back(m);
                runs.push_back(k[m].x);
            }
        c->nruns = (int)runs.size() / 2;
        runs.push_back(M);
        runs.push_back(0);
        cudaFree(c->d_runs);
        c->d_runs = nullptr;
        if (cudaMalloc(&c->d_runs, sizeof(int) * runs.size()) != cudaSuccess) return LAT_ENOMEM;
        CK2(cudaMemcpy(c->d_runs, runs.data(), sizeof(int) * runs.size(), cudaMemcpyHostToDevice));
        if (cudaMalloc(&c->d_k, sizeof(int2) * M) != cudaSuccess ||
            cudaMalloc(&c->d_cx, sizeof(double) * M) != cudaSuccess ||
            cudaMalloc(&c->d_cy, sizeof(double) * M) != cudaSuccess ||
            cudaMalloc(&c->d_phase, sizeof(double) * 2 * M) != cudaSuccess)
            return LAT_ENOMEM;
        CK2(cudaMemcpy(c->d_k, k.data(), sizeof(int2) * M, cudaMemcpyHostToDevice));
        CK2(cudaMemcpy(c->d_cx, cx.data(), sizeof(double) * M, cudaMemcpyHostToDevice));
        CK2(cudaMemcpy(c->d_cy, cy.data(), sizeof(double) * M, cudaMemcpyHostToDevice));
        CK2(cudaMemcpy(c->d_phase, ph.data(), sizeof(double) * 2 * M, cudaMemcpyHostToDevice));
        const size_t es = c->dtype == LAT_F64 ? sizeof(double) : sizeof(float);
        if (!c->d_u) {
            if (cudaMalloc(&c->d_u, es * 2 * (size_t)c->nx * c->ny) != cudaSuccess)
                return LAT_ENOMEM;
        }
        // separable tables of e^{i 2 pi k x / n}: the phase k x mod n is reduced in integers and
        // evaluated in FP64, then stored in the flow's precision
        int kmax = 0;
        for (int m = 0; m < M; ++m) kmax = std::max(kmax, std::max(abs(k[m].x), abs(k[m].y)));
        auto table = [&](int n, void** dst) -> int {
            const size_t cnt = (size_t)(2 * kmax + 1) * n * 2;
            std::vector<double> t(cnt);
            for (int kk = -kmax; kk <= kmax; ++kk)
                for (int i = 0; i < n; ++i) {
                    long long p = ((long long)kk * i) % n;
                    if (p < 0) p += n;
                    const double th = 2.0 * M_PI * (double)p / (double)n;
                    t[2 * ((size_t)(kk + kmax) * n + i)] = cos(th);
                    t[2 * ((size_t)(kk + kmax) * n + i) + 1] = sin(th);
                }
            cudaFree(*dst);
            *dst = nullptr;
            if (cudaMalloc(dst, es * cnt) != cudaSuccess) return LAT_ENOMEM;
            if (es == sizeof(double)) {
                CK2(cudaMemcpy(*dst, t.data(), es * cnt, cudaMemcpyHostToDevice));
            } else {
                std::vector<float> tf(t.begin(), t.end());
                CK2(cudaMemcpy(*dst, tf.data(), es * cnt, cudaMemcpyHostToDevice));
            }
            return LAT_OK;
        };
        int trc = table(c->nx, &c->d_xtab);
        if (trc == LAT_OK) trc = table(c->ny, &c->d_ytab);
        if (trc != LAT_OK) return trc;
        c->kmax = kmax;
        c->nmodes = M;
        c->flow_kind = LAT_FLOW_MODES;
        c->walk = frozen ? 0.0 : sqrt(2.0 * c->dt / fl->tau_f);
    } else {
        return LAT_EINVAL;
    }
    c->frozen = frozen || fl->kind != LAT_FLOW_MODES;
    k_set_noise2d<<<1, 1, 0, s>>>(c->st, 0, 0);
    CK2(cudaGetLastError());
    return LAT_OK;
}

int ctx2d_set_noise(Ctx2D* c, const double* noise, long long rows, long long step,
                    cudaStream_t s) {
    if (c->flow_kind != LAT_FLOW_MODES) return LAT_EINVAL;
    const long long need = rows * c->nmodes;
    if (need > c->noise_cap) {
        CK2(cudaStreamSynchronize(s));
        double* p = nullptr;
        if (cudaMalloc(&p, sizeof(double) * need) != cudaSuccess) return LAT_ENOMEM;
        cudaFree(c->d_noise);
        c->d_noise = p;
        c->noise_cap = need;
        drop(c);
    }
    if (need > 0)
        CK2(cudaMemcpyAsync(c->d_noise, noise, sizeof(double) * need, cudaMemcpyHostToDevice, s));
    k_set_noise2d<<<1, 1, 0, s>>>(c->st, step, rows);
    CK2(cudaGetLastError());
    return LAT_OK;
}

int ctx2d_prepare(Ctx2D* c, void* const f[2], int n) {
    if (c->mode != 0) return LAT_OK;
    cudaGraphExec_t ge;
    return graph2d(c, f, n, &ge);
}

int ctx2d_step(Ctx2D* c, void* const f[2], int n, cudaStream_t s) {
    if (c->mode != 0) return enqueue2d(c, f, n, s, 0);
    cudaGraphExec_t ge;
    int rc = graph2d(c, f, n, &ge);
    if (rc != LAT_OK) return rc;
    CK2(cudaGraphLaunch(ge, s));
    return LAT_OK;
}

int ctx2d_set_scheme(Ctx2D* c, int scheme, double mu) {
    if (scheme == LAT_SCHEME_KOREN) {
        if (c->half || c->learn || (c->dtype != LAT_F32 && c->dtype != LAT_F64)) return LAT_EINVAL;
        const long long n = (long long)c->nx * c->ny * c->nv * c->nv;
        const int Jv = (c->nv - 1) / 2;
        // 32-bit indices, one-step periodic wraps of the streaming shifts, grid.y = plane
        if (n >= (1ll << 32) || c->nx <= Jv || c->ny <= Jv)
            return LAT_EINVAL;
        // each Heun stage is positive for (dt/dv)(max|a_x| + max|a_y|)(1 + mu) <= 1; at rest
        // that is 2 g J (1 + mu)
        const int J = (c->nv - 1) / 2;
        if (2.0 * c->g * J * (1.0 + mu) > 1.0) return LAT_ECFL;
        c->mu = mu;
        c->scheme = scheme;
        const int rc = lim_scratch(c);
        if (rc != LAT_OK) {
            c->scheme = LAT_SCHEME_UPWIND;
            return rc;
        }
    } else {
        cudaFree(c->d_lim);
        c->d_lim = nullptr;
    }
    c->scheme = scheme;
    drop(c);
    return LAT_OK;
}

void ctx2d_geometry(const Ctx2D* c, int* nx, int* ny, int* nv, double* dx, double* dv) {
    *nx = c->nx;
    *ny = c->ny;
    *nv = c->nv;
    *dx = c->dx;
    *dv = c->dv;
}

// The four globals of the last reduction to host memory: through the context's pinned buffer
// and a stream synchronisation (wait), or copied straight into the caller's (pinned) buffer
// without waiting.
int copy_globals(Ctx2D* c, double* globals, bool wait, cudaStream_t s) {
    if (!globals) return LAT_OK;
    if (!wait) {
        CK2(cudaMemcpyAsync(globals, c->d_glob, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
        return LAT_OK;
    }
    CK2(cudaMemcpyAsync(c->h_glob, c->d_glob, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
    CK2(cudaStreamSynchronize(s));
    memcpy(globals, c->h_glob, sizeof(double) * 4);
    return LAT_OK;
}

int ctx2d_moments(Ctx2D* c, const void* f, int cur, double* rho, double* mean_v,
                  double* mean_v2, double* globals, bool wait, cudaStream_t s) {
    const float* sc = c->half ? c->d_sc + (size_t)cur * c->nlines : nullptr;
    if (c->dtype == LAT_F16)
        k_moments2d<__half><<<c->mom_blocks, 32 * kMom2DWarps, 0, s>>>(f, sc, c->nv, c->nx, c->ny, c->dv,
                                                         rho, mean_v, mean_v2, c->d_partials, c->st);
    else if (c->dtype == LAT_BF16)
        k_moments2d<__nv_bfloat16><<<c->mom_blocks, 32 * kMom2DWarps, 0, s>>>(f, sc, c->nv, c->nx, c->ny, c->dv,
                                                         rho, mean_v, mean_v2, c->d_partials, c->st);
    else if (c->dtype == LAT_F64)
        k_moments2d<double><<<c->mom_blocks, 32 * kMom2DWarps, 0, s>>>(f, nullptr, c->nv, c->nx, c->ny, c->dv,
                                                         rho, mean_v, mean_v2, c->d_partials, c->st);
    else
        k_moments2d<float><<<c->mom_blocks, 32 * kMom2DWarps, 0, s>>>(f, nullptr, c->nv, c->nx, c->ny, c->dv,
                                                        rho, mean_v, mean_v2, c->d_partials, c->st);
    CK2(cudaGetLastError());
    k_finalize2d<<<1, kFin2DThreads, 0, s>>>(c->d_partials, c->mom_blocks,
                                             c->dx * c->dx * c->dv * c->dv, c->d_glob);
    CK2(cudaGetLastError());
    return copy_globals(c, globals, wait, s);
}

bool ctx2d_moments_fusable(const Ctx2D* c) {
    return c->dtype == LAT_F32 && !c->half && !c->learn && c->scheme == LAT_SCHEME_UPWIND &&
           c->ring && (c->pcv == 4 || c->pcv == 5 || c->pcv >= 8) && pc_supported(c->nv);
}

int ctx2d_step_moments(Ctx2D* c, void* const f[2], double* rho, double* mean_v,
                       double* mean_v2, double* globals, bool wait, cudaStream_t s) {
    if (!ctx2d_moments_fusable(c)) return LAT_EINVAL;
    const Step2DArgs a = step_args(c, f);
    if (c->flow_kind == LAT_FLOW_MODES) {
        const int rc = launch_flow(c, 0, 0, s);
        if (rc != LAT_OK) return rc;
    }
    Mom2DOut m;
    m.rho = rho;
    m.mv = mean_v;
    m.mv2 = mean_v2;
    m.partials = c->d_partials;
    m.dv = c->dv;
    int grid = 0;
    // the packed kernels write the same bits as kernel 5, which also reduces the moments
    const int v = c->pcv >= 8 ? 5 : c->pcv;
    CK2(launch_step2d_mom(c->nv, v, c->pcv >= 8 ? 0 : c->bps, c->sm_count, a, 0, m, &grid, s));
    k_advance2d<<<1, 1, 0, s>>>(c->st, 1);
    CK2(cudaGetLastError());
    k_finalize2d<<<1, kFin2DThreads, 0, s>>>(c->d_partials, grid * (TW / 32),
                                             c->dx * c->dx * c->dv * c->dv, c->d_glob);
    CK2(cudaGetLastError());
    return copy_globals(c, globals, wait, s);
}

int ctx2d_set_launch(Ctx2D* c, int kernel, int block, int bps, int mode) {
    // kernel: 0 keep, 1 plain loads (128 threads), >= 2 bulk-copy ring; for the ring, block =
    // 128 C threads splits every cell's jx range over C warp groups (C = 1..4)
    // kernel 3..7: producer/consumer variants, 8..10 the packed two-lane sweep (160 threads)
    if (c->scheme == LAT_SCHEME_KOREN) {  // 1 three passes, 2 fused, 3 fused on FP32 pairs
        if (kernel < 0 || kernel > 3) return LAT_EINVAL;
        if (kernel >= 2 && !limiter2d_fused_supported(c->nv)) return LAT_EINVAL;
        if (kernel == 3 && c->dtype != LAT_F32) return LAT_EINVAL;
        if (mode == 1 || mode > 2) return LAT_EINVAL;
        if (bps < 0 || bps > 2) return LAT_EINVAL;
        const int was = c->lim_kernel;
        if (kernel) c->lim_kernel = kernel;
        if (bps) c->lim_bps = bps;
        const int rc = lim_scratch(c);
        if (rc != LAT_OK) {
            c->lim_kernel = was;
            return rc;
        }
        if (mode == 0 || mode == 2) c->mode = mode;
        drop(c);
        return LAT_OK;
    }
    if (kernel < 0 || kernel > 10) return LAT_EINVAL;
    if (c->half && (kernel == 2 || kernel == 3 || kernel >= 8)) return LAT_EINVAL;
    if (kernel >= 2 && !ring_ok(c)) return LAT_EINVAL;
    if (c->half && kernel >= 4 && !pc_ok(c)) return LAT_EINVAL;
    if (kernel >= 3 && !pc_supported(c->nv)) return LAT_EINVAL;
    const bool ring = kernel == 0 ? c->ring : kernel >= 2;
    const int pcv = kernel == 0 ? c->pcv : (kernel >= 3 ? kernel : 0);
    int chunks = c->chunks;
    if (block && !pcv) {
        if (block % TW != 0) return LAT_EINVAL;
        if (!ring && block != TW) return LAT_EINVAL;
        if (ring) chunks = block / TW;
    }
    if (ring && !pcv && !chunks_supported(c->nv, chunks)) return LAT_EINVAL;
    if (mode == 1 || mode > 2) return LAT_EINVAL;
    c->ring = ring;
    c->chunks = chunks;
    c->pcv = pcv;
    if (bps > 0) c->bps = bps;
    if (mode == 0 || mode == 2) c->mode = mode;
    drop(c);
    return LAT_OK;
}

int ctx2d_autotune(Ctx2D* c, void* const f[2], int reps, double* best, cudaStream_t s) {
    if (c->learn || c->scheme == LAT_SCHEME_KOREN) {  // one launch shape
        if (best) {
            best[0] = 1;
            best[1] = TW;
            best[2] = 0;
            best[3] = 0;
        }
        return LAT_OK;
    }
    cudaEvent_t e0, e1;
    CK2(cudaEventCreate(&e0));
    CK2(cudaEventCreate(&e1));
    double best_us = 1e300;
    bool best_ring = c->ring;
    int best_bps = c->bps, best_chunks = c->chunks, best_pcv = c->pcv;
    // variant 0: plain loads; 1..4: ring with that many chunks; 5..12: producer/consumer 3..10
    for (int variant = 0; variant <= 12; ++variant) {
        if (variant > 0 && !ring_ok(c)) continue;
        if (variant >= 1 && variant <= 4 && !chunks_supported(c->nv, variant)) continue;
        if (variant >= 5 && !pc_ok(c)) continue;
        if (c->half && ((variant >= 1 && variant <= 5) || variant >= 10)) continue;  // 16-bit: plain, pc 4..7
        for (int bps : {1, 2, 3, 4, 6, 8}) {
            c->ring = variant > 0;
            c->chunks = (variant >= 1 && variant <= 4) ? variant : 1;
            c->pcv = variant >= 5 ? variant - 2 : 0;
            c->bps = bps;
            const int occ = c->half ? occupancy_step2d_h(c->dtype, c->nv, c->pcv)
                                    : occupancy_ring(c->nv, c->chunks, c->pcv);
            if (c->ring && bps > occ) continue;
            int rc = enqueue2d(c, f, 1, s, 1);
            if (rc != LAT_OK) return rc;
            CK2(cudaEventRecord(e0, s));
            rc = enqueue2d(c, f, reps, s, 1);
            if (rc != LAT_OK) return rc;
            CK2(cudaEventRecord(e1, s));
            CK2(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK2(cudaEventElapsedTime(&ms, e0, e1));
            const double us = 1000.0 * ms / reps;
            if (us < best_us) {
                best_us = us;
                best_ring = c->ring;
                best_chunks = c->chunks;
                best_pcv = c->pcv;
                best_bps = bps;
            }
        }
    }
    c->ring = best_ring;
    c->chunks = best_chunks;
    c->pcv = best_pcv;
    c->bps = best_bps;
    drop(c);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best) {
        best[0] = best_pcv ? best_pcv : (best_ring ? 2 : 1);
        best[1] = best_pcv ? TW + 32 : (best_ring ? TW * best_chunks : TW);
        best[2] = best_bps;
        best[3] = best_us;
    }
    return LAT_OK;
}

int ctx2d_init_state(Ctx2D* c, void* const f[2], int cur, cudaStream_t s) {
    if (!c->half) return LAT_OK;
    // the caller's initial 16-bit values are taken with scale 1
    CK2(launch_linemax_h(c->dtype, f[cur], c->d_sc + (size_t)cur * c->nlines,
                         c->d_mx + (size_t)cur * c->nlines, c->nv, c->nx, c->ny, s));
    return LAT_OK;
}

void ctx2d_dyn(const Ctx2D* c, Ctx2DDyn* o) {
    o->nlines = c->half ? c->nlines : 0;
    o->sc = c->d_sc;
    o->mx = c->d_mx;
    o->flow_kind = c->flow_kind;
    o->nmodes = c->flow_kind == LAT_FLOW_MODES ? c->nmodes : 0;
    o->phase = c->d_phase;
    o->noise = c->d_noise;
    o->noise_cap = c->noise_cap;
    o->g = c->g;
    o->r = c->r;
    o->frozen = c->frozen;
}

int ctx2d_noise_reserve(Ctx2D* c, long long need, cudaStream_t s) {
    if (need <= c->noise_cap) return LAT_OK;
    CK2(cudaStreamSynchronize(s));
    double* p = nullptr;
    if (cudaMalloc(&p, sizeof(double) * need) != cudaSuccess) return LAT_ENOMEM;
    cudaFree(c->d_noise);
    c->d_noise = p;
    c->noise_cap = need;
    drop(c);
    return LAT_OK;
}

void ctx2d_drop_graphs(Ctx2D* c) { drop(c); }

int ctx2d_encode(Ctx2D* c, const float* src, void* const f[2], int cur, cudaStream_t s) {
    if (!c->half || !src) return LAT_EINVAL;
    CK2(launch_encode_h(c->dtype, src, f[cur], c->d_sc + (size_t)cur * c->nlines,
                        c->d_mx + (size_t)cur * c->nlines, c->nv, c->nx, c->ny, c->st, s));
    return LAT_OK;
}

int ctx2d_decode(Ctx2D* c, void* const f[2], int cur, float* dst, float* scales,
                 cudaStream_t s) {
    if (!c->half) return LAT_EINVAL;
    const float* sc = c->d_sc + (size_t)cur * c->nlines;
    if (dst) CK2(launch_decode_h(c->dtype, f[cur], sc, dst, c->nv, c->nx, c->ny, s));
    if (scales) CK2(launch_scales_dense(sc, scales, c->nv, c->ny, s));
    return LAT_OK;
}

int ctx2d_learn_set(Ctx2D* c, const float* params, int mode, cudaStream_t s) {
    if (mode == 0) {
        c->learn = 0;
        drop(c);
        return LAT_OK;
    }
    if ((mode != 1 && mode != 2) || !params || c->dtype != LAT_F32 || !learn_nv_supported(c->nv))
        return LAT_EINVAL;
    const int J = (c->nv - 1) / 2;
    // the kernels wrap streamed indices with one conditional add; nv^2 nx ny indexes in 32 bits
    if (c->nx <= J + 1 || c->ny <= J + 1 ||
        (long long)c->nx * c->ny * c->nv * c->nv >= (1ll << 32) - 256)
        return LAT_EINVAL;
    if (mode == 2 && !learn_tc_supported(c->nv)) return LAT_EINVAL;
    const long long ncell = (long long)c->nx * c->ny;
    if (!c->d_params) {
        if (cudaMalloc(&c->d_params, sizeof(float) * kLNParam) != cudaSuccess ||
            cudaMalloc(&c->d_rho, sizeof(float) * ncell) != cudaSuccess ||
            cudaMalloc(&c->d_feat, sizeof(float4) * 2 * ncell) != cudaSuccess ||
            cudaMalloc(&c->d_G, sizeof(float) * 2 * c->nv * c->nv * ncell) != cudaSuccess ||
            cudaMalloc(&c->d_wtc, learn_tc_bytes()) != cudaSuccess ||
            cudaMalloc(&c->d_st0, sizeof(DevState)) != cudaSuccess)
            return LAT_ENOMEM;
        CK2(cudaMemsetAsync(c->d_st0, 0, sizeof(DevState), s));
    }
    CK2(cudaMemcpyAsync(c->d_params, params, sizeof(float) * kLNParam, cudaMemcpyHostToDevice, s));
    CK2(launch_learn_tc_pack(c->d_params, c->d_wtc, s));
    CK2(cudaStreamSynchronize(s));
    c->learn = mode;
    drop(c);
    return LAT_OK;
}

// Correction fluxes of the current state (flow of the current step, not advanced): rho*, the
// network, G; copied to G_out ([2][N_v^2][ny][nx] floats, device) when given.
int ctx2d_learn_corr(Ctx2D* c, void* const f[2], int cur, float* G_out, int reuse,
                     cudaStream_t s) {
    if (!c->learn) return LAT_EINVAL;
    if (c->flow_kind == LAT_FLOW_MODES && !reuse) {
        const int rc = launch_flow(c, 0, 1, s);
        if (rc != LAT_OK) return rc;
    }
    const LearnArgs la = learn_args(c, f[cur], f[cur], c->d_st0);
    if (!reuse) CK2(launch_rho_star(c->nv, la, 0, s));
    if (c->learn == 2) CK2(launch_mlp_tc(c->nv, la, c->d_wtc, c->sm_count, c->ring, 0, s));
    else CK2(launch_mlp_f32(c->nv, la, 0, s));
    if (G_out) {
        const size_t n = (size_t)2 * c->nv * c->nv * c->nx * c->ny;
        CK2(cudaMemcpyAsync(G_out, c->d_G, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
    }
    return LAT_OK;
}

// Loss of an n-step rollout of the learned step (FP32 network) from the current state against
// target, and its gradient with respect to the parameters.  The state, the flow phases and the
// step counter are left as they were.
int ctx2d_learn_grad(Ctx2D* c, void* const f[2], int cur, int n, const float* target,
                     double rho_weight, double* loss, float* grad, cudaStream_t s) {
    if (!c->learn || n < 1 || n > 64 || !target || c->flow_kind == LAT_FLOW_NONE) return LAT_EINVAL;
    const long long ncell = (long long)c->nx * c->ny;
    const long long nst = ncell * c->nv * c->nv;
    float* buf = nullptr;
    // F[0..n], U[0..n-1], lam x2, lss, lfs, lrho, dX9, cxy, grad; loss partials
    const size_t nfl = (size_t)(n + 1) * nst + (size_t)n * 2 * ncell + 4 * (size_t)nst + ncell +
                       11 * (size_t)nst + kLNParam;
    const int nb = 256;
    double* dpart = nullptr;
    if (cudaMalloc(&buf, sizeof(float) * nfl) != cudaSuccess) return LAT_ENOMEM;
    if (cudaMalloc(&dpart, sizeof(double) * (2 * nb + 1)) != cudaSuccess) {
        cudaFree(buf);
        return LAT_ENOMEM;
    }
    double* dphase = nullptr;
    const bool modes = c->flow_kind == LAT_FLOW_MODES;
    int rc = LAT_OK;
    auto fail = [&](int code) {
        rc = code;
        return code;
    };
    do {
        float* F = buf;
        float* U = F + (size_t)(n + 1) * nst;
        float* lamA = U + (size_t)n * 2 * ncell;
        float* lamB = lamA + nst;
        float* lss = lamB + nst;
        float* lfs = lss + nst;
        float* lrho = lfs + nst;
        float* dX9 = lrho + ncell;
        float* cxy = dX9 + 9 * nst;
        float* g = cxy + 2 * nst;
        if (modes) {
            if (cudaMalloc(&dphase, sizeof(double) * 2 * c->nmodes) != cudaSuccess) {
                fail(LAT_ENOMEM);
                break;
            }
            if (cudaMemcpyAsync(dphase, c->d_phase, sizeof(double) * 2 * c->nmodes,
                                cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
                fail(LAT_ECUDA);
                break;
            }
        }
        if (cudaMemcpyAsync(F, f[cur], sizeof(float) * nst, cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess) {
            fail(LAT_ECUDA);
            break;
        }
        // forward rollout on explicit buffers F[k] -> F[k+1] (zero step counter: parity 0)
        Step2DArgs a = step_args(c, f);
        a.st = c->d_st0;
        for (int k = 0; k < n && rc == LAT_OK; ++k) {
            if (modes && launch_flow(c, k, 0, s) != LAT_OK) fail(LAT_ECUDA);
            const float* u = c->flow_kind == LAT_FLOW_FIELD ? static_cast<const float*>(c->field)
                                                            : static_cast<const float*>(c->d_u);
            if (cudaMemcpyAsync(U + (size_t)k * 2 * ncell, u, sizeof(float) * 2 * ncell,
                                cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                fail(LAT_ECUDA);
            a.f[0] = F + (size_t)k * nst;
            a.f[1] = F + (size_t)(k + 1) * nst;
            LearnArgs la = learn_args(c, a.f[0], a.f[1], c->d_st0);
            la.u = U + (size_t)k * 2 * ncell;
            a.u = la.u;
            // the network of the context's mode: FP32 on CUDA cores, or BF16 on tensor cores
            if (launch_rho_star(c->nv, la, 0, s) != cudaSuccess ||
                (c->learn == 2 ? launch_mlp_tc(c->nv, la, c->d_wtc, c->sm_count, c->ring, 0, s)
                               : launch_mlp_f32(c->nv, la, 0, s)) != cudaSuccess ||
                launch_corrected(c, a, 0, s) != cudaSuccess)
                fail(LAT_ECUDA);
        }
        if (rc != LAT_OK) break;
        // lrho holds the density error r(x) until the backward steps reuse it
        if (launch_loss(F + (size_t)n * nst, target, c->nv * c->nv, ncell, rho_weight, lrho, lamA,
                        dpart, nb, dpart + 2 * nb, s) != cudaSuccess ||
            cudaMemsetAsync(g, 0, sizeof(float) * kLNParam, s) != cudaSuccess) {
            fail(LAT_ECUDA);
            break;
        }
        for (int k = n - 1; k >= 0 && rc == LAT_OK; --k) {
            LearnBwdArgs b;
            b.fw = learn_args(c, F + (size_t)k * nst, F + (size_t)k * nst, c->d_st0);
            b.fw.u = U + (size_t)k * 2 * ncell;
            b.lam_out = lamA;
            b.lss = lss;
            b.lrho = lrho;
            b.dX9 = dX9;
            b.cxy = cxy;
            b.lfs = lfs;
            b.lam_in = lamB;
            b.grad = g;
            b.r = (float)c->r;
            if (launch_diffuse_adjoint(c->nv, lamA, lss, (float)c->r, c->nx, c->ny, s) != cudaSuccess ||
                cudaMemsetAsync(lrho, 0, sizeof(float) * ncell, s) != cudaSuccess ||
                launch_rho_star(c->nv, b.fw, 0, s) != cudaSuccess ||
                (c->learn == 2 ? launch_mlp_bwd_tc(c->nv, b, c->d_wtc, c->sm_count, s)
                               : launch_mlp_bwd(c->nv, b, c->sm_count, s)) != cudaSuccess ||
                launch_gather_adjoint(c->nv, b, s) != cudaSuccess)
                fail(LAT_ECUDA);
            std::swap(lamA, lamB);
        }
        if (rc != LAT_OK) break;
        if (cudaMemcpyAsync(grad, g, sizeof(float) * kLNParam, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(loss, dpart + 2 * nb, sizeof(double), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess)
            fail(LAT_ECUDA);
    } while (false);
    if (dphase) {
        cudaMemcpyAsync(c->d_phase, dphase, sizeof(double) * 2 * c->nmodes,
                        cudaMemcpyDeviceToDevice, s);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == LAT_OK) rc = LAT_ECUDA;
    cudaFree(dphase);
    cudaFree(dpart);
    cudaFree(buf);
    return rc;
}

void ctx2d_destroy(Ctx2D* c) {
    if (!c) return;
    drop(c);
    cudaFree(c->d_k);
    cudaFree(c->d_perm);
    cudaFree(c->d_runs);
    cudaFree(c->d_cx);
    cudaFree(c->d_cy);
    cudaFree(c->d_phase);
    cudaFree(c->d_xtab);
    cudaFree(c->d_ytab);
    cudaFree(c->d_noise);
    cudaFree(c->d_u);
    cudaFree(c->d_partials);
    cudaFree(c->d_sc);
    cudaFree(c->d_mx);
    cudaFree(c->d_params);
    cudaFree(c->d_wtc);
    cudaFree(c->d_rho);
    cudaFree(c->d_feat);
    cudaFree(c->d_lim);
    cudaFree(c->d_G);
    cudaFree(c->d_st0);
    cudaFree(c->d_glob);
    if (c->h_glob) cudaFreeHost(c->h_glob);
    delete c;
}

}  // namespace lat

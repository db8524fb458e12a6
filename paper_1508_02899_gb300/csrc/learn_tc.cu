// The learned closure's network in BF16 on the fifth-generation tensor cores (tcgen05), FP32
// accumulation in tensor memory.  Same features and output as learn.cu's FP32 network.
//
// A CTA of 128 threads takes tiles of 128 phase-space cells (one cell per thread = one row of
// the M = 128 MMA tile).  Per tile: every thread builds its row of features (FP32 -> BF16) in
// shared memory; one thread issues layer 1 (K = 16, N = 64), the CTA waits on the commit's
// mbarrier, reads its accumulator row (tcgen05.ld) and writes relu(.) as BF16 (one
// cvt.rn.relu.bf16x2 per pair) back as the next A operand; layer 2 (K = 80, N = 64) and layer 3
// (K = 80, N = 16 with two live outputs) the same way; the bounded outputs y = b tanh(z) times
// the density differences across the +jx and +jy faces are the corrections.
//
// Tile order: with N_x a multiple of 128 a CTA takes units of 128 x of one grid row, all N_v^2
// planes of a unit in turn, and keeps the 3 x 3 velocity neighbourhood of f* in registers as it
// slides from plane to plane (UnitFeed); otherwise tiles of 128 phase cells in storage order,
// each gathering its nine neighbours (StorageFeed).
//
// Biases ride in the products: feature 15 is the constant 1, so b1 joins row 15 of W1; the
// activation tiles carry a constant 1 in column 64 (columns 65..79 zero, K padded to a multiple
// of 16), so b2 and b3 join row 64 of W2 and W3.  The three layers share one 64-column TMEM
// accumulator (each is read before the next MMA writes), so five CTAs fit an SM.
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
constexpr int kK2 = 80;                       // K of layers 2 and 3: 64 activations, 1, zeros
constexpr int kW1T = 0;                       // B of layer 1: N 64 x K 16 (2 KB), b1 in k = 15
constexpr int kW2T = kW1T + 64 * 16 * 2;      // B of layer 2: N 64 x K 80 (10 KB), b2 in k = 64
constexpr int kW3T = kW2T + 64 * kK2 * 2;     // B of layer 3: N 16 x K 80 (2.5 KB), b3 in k = 64
constexpr int kImage = kW3T + 16 * kK2 * 2;
// shared memory of the kernel: image, A1 (128 x 16), A2 (128 x 80), barrier, TMEM address
constexpr int kSA1 = (kImage + 1023) / 1024 * 1024;
constexpr int kSA2 = kSA1 + 128 * 16 * 2;
constexpr int kSBar = kSA2 + 128 * kK2 * 2;
constexpr int kSmem = kSBar + 16;
constexpr int kSmemReq = kSmem;
constexpr int kTmemCols = 64;                 // D1, D2, D3 in turn (D3: columns 0..15)
static_assert(kImage % 16 == 0, "image copied in 16-byte pieces");
static_assert((228 * 1024) / (kSmemReq + 1024) * kTmemCols <= 512,
              "the CTAs that fit an SM by shared memory must also fit its TMEM");

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

// 16 consecutive accumulator columns of this thread's row (completion: tmem_wait)
__device__ __forceinline__ void tmem_ld16(unsigned taddr, unsigned (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
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

// relu(lo), relu(hi) rounded to BF16 and packed (lo in the low half)
__device__ __forceinline__ uint32_t pack_relu_bf16(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// ReLU of 64 accumulator columns of this thread's row into row r of a 128-row A tile; the
// columns come in two groups of 32 (two loads in flight per wait)
__device__ __forceinline__ void epilogue64(unsigned taddr, unsigned char* A, int r) {
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 32) {
        unsigned v[2][16];
        tmem_ld16(taddr + c0, v[0]);
        tmem_ld16(taddr + c0 + 16, v[1]);
        tmem_wait();
#pragma unroll
        for (int g = 0; g < 4; ++g) {  // four 8-column core-matrix chunks
            const unsigned* u = v[g >> 1] + 8 * (g & 1);
            uint4 w;
            w.x = pack_relu_bf16(__uint_as_float(u[0]), __uint_as_float(u[1]));
            w.y = pack_relu_bf16(__uint_as_float(u[2]), __uint_as_float(u[3]));
            w.z = pack_relu_bf16(__uint_as_float(u[4]), __uint_as_float(u[5]));
            w.w = pack_relu_bf16(__uint_as_float(u[6]), __uint_as_float(u[7]));
            *reinterpret_cast<uint4*>(A + tile_off(r, c0 + 8 * g, 128)) = w;
        }
    }
}

// tanh on the special-function unit (tanh.approx.f32: relative error about 2^-11, far below the
// BF16 rounding the network already carries)
__device__ __forceinline__ float tanh_fast(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ int vwrap(int v, int n) { return wrap_near(v, n); }

// Raw inputs of one phase cell's features (learn.cu's features, split so that the global loads
// can be issued early and consumed after other work): f* over the 3 x 3 velocity neighbourhood,
// and the spatial parts of the features, which the density kernel formed once per spatial cell
// (1/rho*, the four velocity gradients times dt, u / dv).  Element indices are 32-bit (the
// learned step keeps N_v^2 N_x N_y below 2^32) and periodic wraps are one conditional add.
struct Raw {
    float fs[9];
    float4 fa, fb;
};

template <int NV>
__device__ __forceinline__ void load_raw(const LearnArgs& a, const float* f, int jx, int jy, int x,
                                         int y, Raw& r) {
    constexpr int J = (NV - 1) / 2;
    const unsigned nx = (unsigned)a.nx, ncell = (unsigned)a.nx * (unsigned)a.ny;
    const unsigned c = (unsigned)y * nx + (unsigned)x;
    r.fa = a.feat[2 * c];
    r.fb = a.feat[2 * c + 1];
    int q = 0;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
        const int jy2 = jy + dy;
        const bool iny = jy2 >= 0 && jy2 < NV;
        const unsigned row = (unsigned)vwrap(y - (jy2 - J), a.ny) * nx;  // source row of plane row jy2
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            const int jx2 = jx + dx;
            const bool in = iny && jx2 >= 0 && jx2 < NV;
            r.fs[q++] = in ? f[(unsigned)(jy2 * NV + jx2) * ncell + row +
                               (unsigned)vwrap(x - (jx2 - J), a.nx)]
                           : 0.f;
        }
    }
}

template <int NV>
__device__ __forceinline__ void features_of(const LearnArgs& a, const Raw& r, int jx, int jy,
                                            float (&X)[kLNF]) {
    constexpr int J = (NV - 1) / 2;
    const float inv = r.fa.x;
#pragma unroll
    for (int q = 0; q < 9; ++q) X[q] = __fmul_rn(r.fs[q], inv);
    X[9] = r.fa.y;
    X[10] = r.fa.z;
    X[11] = r.fa.w;
    X[12] = r.fb.x;
    X[13] = __fmul_rn(a.g, __fsub_rn(r.fb.y, (float)(jx - J)));
    X[14] = __fmul_rn(a.g, __fsub_rn(r.fb.z, (float)(jy - J)));
    X[15] = 1.f;
}

// The corrections of one phase cell: the outputs y = b tanh(z), with b the bound for z's sign,
// times the differences of f* across the cell's +jx and +jy faces (zero at the upper walls).
template <int NV>
__device__ __forceinline__ void write_corrections(const LearnArgs& a, unsigned n, unsigned i,
                                                  int jx, int jy, float c13, float c14, float f0,
                                                  float fx, float fy, float z0, float z1) {
    const float y0 = __fmul_rn(z0 > 0.f ? anti_bound(c13, a.g) : kYMax, tanh_fast(z0));
    const float y1 = __fmul_rn(z1 > 0.f ? anti_bound(c14, a.g) : kYMax, tanh_fast(z1));
    a.G[i] = jx < NV - 1 ? __fmul_rn(y0, __fsub_rn(fx, f0)) : 0.f;
    a.G[(size_t)n + i] = jy < NV - 1 ? __fmul_rn(y1, __fsub_rn(fy, f0)) : 0.f;
}

// ---- tile sources -----------------------------------------------------------------------------
// A feed hands a CTA its tiles in order.  load() issues the global loads of the next tile (while
// the tensor cores work on the current one); features() forms that tile's 16 features, which
// run_network stores into A1; out() writes the corrections of a finished tile.  A Slot carries
// one tile from load() to out(); `valid` (the tile exists) is the same for every thread of the
// CTA.

// Tiles of 128 phase cells in storage order: tile b, b + G, b + 2G, ... for CTA b of G.  Any N_x;
// the last tile may be ragged.
template <int NV>
struct StorageFeed {
    struct Slot {
        Raw r;
        unsigned i;
        int jx, jy;
        bool valid, on;
        float c13, c14;  // features 13 and 14, which bound the outputs
    };
    const LearnArgs& a;
    const float* f;
    unsigned n, ncell;
    long long tile, ntiles;  // the next tile to load
    int t;

    __device__ StorageFeed(const LearnArgs& a_, const float* f_, int t_)
        : a(a_), f(f_), t(t_) {
        ncell = (unsigned)a.nx * (unsigned)a.ny;
        n = ncell * (unsigned)(NV * NV);
        ntiles = ((long long)n + 127) / 128;
        tile = blockIdx.x;
    }
    __device__ __forceinline__ void load(Slot& q) {
        const long long i = tile * 128 + t;
        q.valid = tile < ntiles;
        q.on = q.valid && i < (long long)n;
        q.jx = q.jy = 0;
        q.i = (unsigned)i;
        if (q.on) {
            int p, x, y;
            split_index((unsigned)i, ncell, (unsigned)a.nx, p, x, y);
            q.jy = p / NV;
            q.jx = p % NV;
            load_raw<NV>(a, f, q.jx, q.jy, x, y, q.r);
        }
        tile += gridDim.x;
    }
    __device__ __forceinline__ void features(Slot& q, float (&X)[kLNF]) {
        if (q.on) {
            features_of<NV>(a, q.r, q.jx, q.jy, X);
        } else {
#pragma unroll
            for (int k = 0; k < kLNF; ++k) X[k] = 0.f;
        }
        q.c13 = X[13];
        q.c14 = X[14];
    }
    __device__ __forceinline__ void out(const Slot& q, float z0, float z1) {
        // f* of the cell and of its +jx, +jy neighbours: entries 4, 5 and 7 of the 3 x 3 block
        if (q.on) write_corrections<NV>(a, n, q.i, q.jx, q.jy, q.c13, q.c14, q.r.fs[4],
                                        q.r.fs[5], q.r.fs[7], z0, z1);
    }
};

// With N_x a multiple of 128: units of 128 consecutive x of one grid row, unit b, b + G, ... for
// CTA b of G, each taken as its N_v^2 planes in storage order (jx fastest), one tile per plane.
// Along a plane row the 3 x 3 velocity neighbourhood of f* slides by one column per tile, so a
// tile loads one new column (three values; two columns at the start of a row) where a tile in
// storage order gathers all nine, and the spatial part of the features is loaded once per unit.
// The features, and so every correction, have the same bits as in storage order.
template <int NV>
struct UnitFeed {
    static constexpr int J = (NV - 1) / 2;
    static constexpr int NN = NV * NV;
    struct Slot {
        unsigned i;
        int jx, jy;
        bool valid;
        float c13, c14;    // features 13 and 14, which bound the outputs
        float f0, fx, fy;  // f* of the cell and of its +jx and +jy neighbours
    };
    const LearnArgs& a;
    const float* f;
    unsigned nx, ny, ncell, n, nbx, nunits;
    unsigned unit;     // unit of the next tile to load
    int p;             // its plane
    unsigned x, y;     // this thread's spatial cell in that unit
    unsigned roff[3];  // source rows y - (jy2 - J), wrapped, times N_x, for jy2 = jy - 1 .. jy + 1
    float w[3][3];     // f* at (jy - 1 .. jy + 1, jx - 1 .. jx + 1) of the tile staged last
    float in[2][3];    // columns loaded for the next tile: jx and jx + 1 at a row start, else jx + 1
    float4 fa, fb;     // spatial features of this thread's cell in the unit loaded last
    int t;

    __device__ UnitFeed(const LearnArgs& a_, const float* f_, int t_) : a(a_), f(f_), t(t_) {
        nx = (unsigned)a.nx;
        ny = (unsigned)a.ny;
        ncell = nx * ny;
        n = ncell * (unsigned)NN;
        nbx = nx / 128;
        nunits = ny * nbx;
        unit = blockIdx.x;
        p = 0;
        x = y = 0;
    }
    // column jx2 of the 3 x 3 block of plane row jy (zero outside the velocity box)
    __device__ __forceinline__ void column(int jy, int jx2, float (&v)[3]) const {
        const unsigned xs = (unsigned)wrap_near((int)x - (jx2 - J), (int)nx);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int jy2 = jy - 1 + r;
            v[r] = (jx2 < NV && jy2 >= 0 && jy2 < NV)
                       ? f[(unsigned)(jy2 * NV + jx2) * ncell + roff[r] + xs]
                       : 0.f;
        }
    }
    __device__ __forceinline__ void load(Slot& q) {
        q.valid = unit < nunits;
        if (!q.valid) return;
        const int jy = p / NV, jx = p - jy * NV;
        q.jx = jx;
        q.jy = jy;
        if (p == 0) {  // a new unit: its spatial cell and features
            y = unit / nbx;
            x = (unit - y * nbx) * 128u + (unsigned)t;
            const unsigned c = y * nx + x;
            fa = a.feat[2 * c];
            fb = a.feat[2 * c + 1];
        }
        if (jx == 0) {  // a new plane row: its source rows and the first two columns
#pragma unroll
            for (int r = 0; r < 3; ++r)
                roff[r] = (unsigned)wrap_near((int)y - (jy - 1 + r - J), (int)ny) * nx;
            column(jy, 0, in[0]);
            column(jy, 1, in[1]);
        } else {
            column(jy, jx + 1, in[1]);
        }
        q.i = (unsigned)p * ncell + y * nx + x;
        if (++p == NN) {
            p = 0;
            unit += gridDim.x;
        }
    }
    __device__ __forceinline__ void features(Slot& q, float (&X)[kLNF]) {
        if (!q.valid) {
#pragma unroll
            for (int k = 0; k < kLNF; ++k) X[k] = 0.f;
            return;
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            if (q.jx == 0) {
                w[r][0] = 0.f;
                w[r][1] = in[0][r];
            } else {
                w[r][0] = w[r][1];
                w[r][1] = w[r][2];
            }
            w[r][2] = in[1][r];
        }
        Raw raw;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) raw.fs[3 * r + c] = w[r][c];
        raw.fa = fa;
        raw.fb = fb;
        features_of<NV>(a, raw, q.jx, q.jy, X);
        q.c13 = X[13];
        q.c14 = X[14];
        q.f0 = w[1][1];
        q.fx = w[1][2];
        q.fy = w[2][1];
    }
    __device__ __forceinline__ void out(const Slot& q, float z0, float z1) {
        if (q.valid)
            write_corrections<NV>(a, n, q.i, q.jx, q.jy, q.c13, q.c14, q.f0, q.fx, q.fy, z0, z1);
    }
};

// The network over a CTA's tiles from a feed.  Per tile, the MMAs of the current tile (features
// already in A1) run while the feed loads and stages the next; two slots alternate, so nothing
// is copied between tiles.
template <class Feed>
__device__ __forceinline__ void run_network(Feed& feed, unsigned char* sm,
                                            const unsigned char* image, const LearnArgs& a) {
    unsigned char* W = sm;
    unsigned char* A1 = sm + kSA1;
    unsigned char* A2 = sm + kSA2;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kSBar);
    unsigned* tslot = reinterpret_cast<unsigned*>(sm + kSBar + 8);
    const int t = threadIdx.x, warp = t >> 5;
    for (int i = t; i < kImage / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(W)[i] = reinterpret_cast<const uint4*>(image)[i];
    {   // the constant columns 64..79 of this thread's activation row: 1, then zeros
        uint4 one;
        one.x = pack_bf16(1.f, 0.f);
        one.y = one.z = one.w = 0u;
        *reinterpret_cast<uint4*>(A2 + tile_off(t, 64, 128)) = one;
        *reinterpret_cast<uint4*>(A2 + tile_off(t, 72, 128)) = make_uint4(0u, 0u, 0u, 0u);
    }
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
    const unsigned wbase = su32(W), a1 = su32(A1), a2 = su32(A2);
    unsigned phase = 0;
    // features of q into row t of A1 (zeros past the end)
    auto stage = [&](typename Feed::Slot& q) {
        float X[kLNF];
        feed.features(q, X);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint4 v;
            v.x = pack_bf16(X[8 * h + 0], X[8 * h + 1]);
            v.y = pack_bf16(X[8 * h + 2], X[8 * h + 3]);
            v.z = pack_bf16(X[8 * h + 4], X[8 * h + 5]);
            v.w = pack_bf16(X[8 * h + 6], X[8 * h + 7]);
            *reinterpret_cast<uint4*>(A1 + tile_off(t, 8 * h, 128)) = v;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    };
    // Wait for the MMAs committed last: warp 0 polls the mbarrier, the others block in the CTA
    // barrier (no issue slots spent spinning); false on a timeout, for every thread.
    auto wait_mma = [&]() -> bool {
        bool ok = true;
        if (warp == 0) ok = wait_parity(bar, phase);
        phase ^= 1;
        const bool bad = __syncthreads_or(!ok);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        return !bad;
    };
    auto sync_for_mma = [&]() {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    };
    auto one_tile = [&](const typename Feed::Slot& cur, typename Feed::Slot& nxt) -> bool {
        // layer 1: D = A1 (128 x 16) W1^T, while the next tile's inputs load
        sync_for_mma();
        if (t == 0) {
            mma(tmem, sdesc(a1, 2048, 128), sdesc(wbase + kW1T, 1024, 128), idesc_n(64), 0);
            commit(bar);
        }
        feed.load(nxt);
        if (!wait_mma()) return false;
        epilogue64(trow, A2, t);
        // layer 2: D = [H1 1 0] (128 x 80) W2^T; A1 is free again: stage the next features
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        sync_for_mma();
        if (t == 0) {
            for (int kk = 0; kk < kK2 / 16; ++kk)
                mma(tmem, sdesc(a2 + kk * 2 * 2048, 2048, 128),
                    sdesc(wbase + kW2T + kk * 2 * 1024, 1024, 128), idesc_n(64), kk);
            commit(bar);
        }
        stage(nxt);
        if (!wait_mma()) return false;
        epilogue64(trow, A2, t);  // MMA 2 is done with A2: overwrite with H2
        // layer 3: D[0..15] = [H2 1 0] (128 x 80) W3^T
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        sync_for_mma();
        if (t == 0) {
            for (int kk = 0; kk < kK2 / 16; ++kk)
                mma(tmem, sdesc(a2 + kk * 2 * 2048, 2048, 128),
                    sdesc(wbase + kW3T + kk * 2 * 256, 256, 128), idesc_n(16), kk);
            commit(bar);
        }
        if (!wait_mma()) return false;
        float z0, z1;
        tmem_ld2(trow, z0, z1);
        feed.out(cur, z0, z1);
        // the next layer-1 MMA (after sync_for_mma) overwrites D only once every thread has read it
        return true;
    };
    typename Feed::Slot s0, s1;
    bool failed = false;
    feed.load(s0);
    stage(s0);
    while (s0.valid) {
        if (!one_tile(s0, s1)) {
            failed = true;
            break;
        }
        if (!s1.valid) break;
        if (!one_tile(s1, s0)) {
            failed = true;
            break;
        }
    }
    if (failed && t == 0) atomicOr(const_cast<unsigned*>(&a.st->status), ST_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
}

// the state buffer a step reads: parity (st->step + kstep) & 1, chosen without indexing the
// kernel's parameters
__device__ __forceinline__ const float* state_in(const LearnArgs& a, int kstep) {
    return ((a.st->step + kstep) & 1) ? a.f[1] : a.f[0];
}

template <int NV>
__global__ void __launch_bounds__(128) k_mlp_tc(const LearnArgs a, const unsigned char* image,
                                                int kstep) {
    extern __shared__ __align__(1024) unsigned char sm[];
    StorageFeed<NV> feed(a, state_in(a, kstep), threadIdx.x);
    run_network(feed, sm, image, a);
}

template <int NV>
__global__ void __launch_bounds__(128) k_mlp_tc_units(const LearnArgs a,
                                                      const unsigned char* image, int kstep) {
    extern __shared__ __align__(1024) unsigned char sm[];
    UnitFeed<NV> feed(a, state_in(a, kstep), threadIdx.x);
    run_network(feed, sm, image, a);
}

// Parameter image: the BF16 B operands of the three layers, biases folded in (b1 into row 15 of
// W1, which meets the constant feature 1; b2 and b3 into row 64 of W2 and W3, which meets the
// constant activation column).
__global__ void k_pack(const float* P, unsigned char* img) {
    const int n1 = 64 * 16, n2 = 64 * kK2, n3 = 16 * kK2;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n1 + n2 + n3;
         e += gridDim.x * blockDim.x) {
        if (e < n1) {  // W1T [n][k] = W1[k][n] (+ b1[n] at k = 15)
            const int nn = e / 16, k = e % 16;
            float w = P[kOffW1 + k * kLNH + nn];
            if (k == 15) w += P[kOffB1 + nn];
            *reinterpret_cast<__nv_bfloat16*>(img + kW1T + tile_off(nn, k, 64)) = __float2bfloat16_rn(w);
        } else if (e < n1 + n2) {
            const int q = e - n1, nn = q / kK2, k = q % kK2;
            const float w = k < 64 ? P[kOffW2 + k * kLNH + nn] : (k == 64 ? P[kOffB2 + nn] : 0.f);
            *reinterpret_cast<__nv_bfloat16*>(img + kW2T + tile_off(nn, k, 64)) = __float2bfloat16_rn(w);
        } else {
            const int q = e - n1 - n2, nn = q / kK2, k = q % kK2;
            float w = 0.f;
            if (nn < kLNO) w = k < 64 ? P[kOffW3 + k * kLNO + nn] : (k == 64 ? P[kOffB3 + nn] : 0.f);
            *reinterpret_cast<__nv_bfloat16*>(img + kW3T + tile_off(nn, k, 16)) = __float2bfloat16_rn(w);
        }
    }
}

// ---- backward pass on the tensor cores ------------------------------------------------------
// The gradient of a learned step with respect to the network's parameters, for the BF16
// network: per tile of 128 phase cells the forward again (layers 1-3 as in k_mlp_tc, the ReLU
// masks and activations kept), the adjoint of the corrected drag fluxes (CUDA cores, as in
// learn.cu's k_mlp_bwd), then three more MMAs for the network's backward, each with M = 128
// cells:
//   dz2 = (dz3 W3^T) [h2 > 0]  (K = 16, N = 64),   dz1 = (dz2 W2^T) [h1 > 0]  (K = 64, N = 64),
//   dX = dz1 W1^T  (K = 64, N = 16),
// and three for the weight gradients, which sum over the tile's cells (K = 128 cells) into
// accumulators that stay in tensor memory across all of a CTA's tiles:
//   [dz2 | dz1]^T [h1 1 0]  -> rows 0..63: dW2^T with db2 in column 64   (M = 128, N = 80),
//   [dz2 | dz1]^T X         -> rows 64..127: dW1^T, db1 = column 15      (M = 128, N = 16),
//   [h2 1 0]^T dz3          -> rows 0..63: dW3, row 64: db3               (M = 128, N = 16).
// The weight-gradient operands are the tile's values transposed (rows = features, K = cells):
// every thread scatters its cell's BF16 values into column `cell` of those K-major tiles.
// Backward B operands, packed from the FP32 parameters after the forward image:
//   B4 [n = i][k = o] = W3[i][o] (o < 2),  B5 [n = i][k = j] = W2[i][j],  B6 [n = q][k = i] = W1[q][i].
constexpr int kB4 = kImage;                   // N 64 x K 16 (2 KB)
constexpr int kB5 = kB4 + 64 * 16 * 2;        // N 64 x K 64 (8 KB)
constexpr int kB6 = kB5 + 64 * 64 * 2;        // N 16 x K 64 (2 KB)
constexpr int kImageAll = kB6 + 16 * 64 * 2;
static_assert(kImageAll % 16 == 0, "image copied in 16-byte pieces");

__global__ void k_pack_bwd(const float* P, unsigned char* img) {
    const int n4 = 64 * 16, n5 = 64 * 64, n6 = 16 * 64;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n4 + n5 + n6;
         e += gridDim.x * blockDim.x) {
        if (e < n4) {
            const int i = e / 16, o = e % 16;
            const float w = o < kLNO ? P[kOffW3 + i * kLNO + o] : 0.f;
            *reinterpret_cast<__nv_bfloat16*>(img + kB4 + tile_off(i, o, 64)) = __float2bfloat16_rn(w);
        } else if (e < n4 + n5) {
            const int q = e - n4, i = q / 64, j = q % 64;
            *reinterpret_cast<__nv_bfloat16*>(img + kB5 + tile_off(i, j, 64)) =
                __float2bfloat16_rn(P[kOffW2 + i * kLNH + j]);
        } else {
            const int q = e - n4 - n5, qq = q / 64, i = q % 64;
            *reinterpret_cast<__nv_bfloat16*>(img + kB6 + tile_off(qq, i, 16)) =
                __float2bfloat16_rn(P[kOffW1 + qq * kLNH + i]);
        }
    }
}

// Shared memory of the backward kernel (byte offsets; every tile 1024-byte aligned).
constexpr int kBW = 0;                                  // forward + backward images
constexpr int kBA1 = (kImageAll + 1023) / 1024 * 1024;  // X        [128][16]
constexpr int kBA2 = kBA1 + 128 * 16 * 2;               // [h1 1 0] [128][80]
constexpr int kBA3 = kBA2 + 128 * kK2 * 2;              // [h2 1 0] [128][80]
constexpr int kBZ3 = kBA3 + 128 * kK2 * 2;              // dz3      [128][16]
constexpr int kBZ2 = kBZ3 + 128 * 16 * 2;               // dz2      [128][64]
constexpr int kBZ1 = kBZ2 + 128 * 64 * 2;               // dz1      [128][64]
constexpr int kTDZ = kBZ1 + 128 * 64 * 2;               // [dz2 | dz1]^T [128][128 cells]
constexpr int kTH1 = kTDZ + 128 * 128 * 2;              // [h1 1 0]^T    [80][128]
constexpr int kTX = kTH1 + 80 * 128 * 2;                // X^T           [16][128]
constexpr int kTH2 = kTX + 16 * 128 * 2;                // [h2 1 0]^T    [128][128]
constexpr int kTZ3 = kTH2 + 128 * 128 * 2;              // dz3^T         [16][128]
constexpr int kBBar = kTZ3 + 16 * 128 * 2;
constexpr int kBSmem = kBBar + 16;
static_assert(kBSmem <= 227 * 1024, "backward kernel's shared memory");
// tensor memory: per-tile accumulator, then the three weight-gradient accumulators
constexpr int kBTmemCols = 256;
constexpr int kTD = 0, kTW2 = 64, kTW1 = 144, kTW3 = 160;

__device__ __forceinline__ void put_bf16(unsigned char* tile, unsigned off, float v) {
    *reinterpret_cast<__nv_bfloat16*>(tile + off) = __float2bfloat16_rn(v);
}
__device__ __forceinline__ void put_bits(unsigned char* tile, unsigned off, unsigned short b) {
    *reinterpret_cast<unsigned short*>(tile + off) = b;
}

// ReLU of 64 accumulator columns of this thread's row (cell r) into row r of A (as epilogue64)
// and into column r of the transposed tile T (rows = features, `trows` rows); bit k of mask is
// set where column k was positive.
__device__ __forceinline__ void epilogue64_t(unsigned taddr, unsigned char* A, unsigned char* T,
                                             int trows, int r, unsigned (&mask)[2]) {
    mask[0] = mask[1] = 0u;
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 32) {
        unsigned v[2][16];
        tmem_ld16(taddr + c0, v[0]);
        tmem_ld16(taddr + c0 + 16, v[1]);
        tmem_wait();
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const unsigned* u = v[g >> 1] + 8 * (g & 1);
            unsigned w[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float a = __uint_as_float(u[2 * e]), b = __uint_as_float(u[2 * e + 1]);
                w[e] = pack_relu_bf16(a, b);
                const int col = c0 + 8 * g + 2 * e;
                mask[col >> 5] |= (a > 0.f ? 1u : 0u) << (col & 31);
                mask[col >> 5] |= (b > 0.f ? 1u : 0u) << ((col + 1) & 31);
                put_bits(T, tile_off(col, r, trows), (unsigned short)(w[e] & 0xffffu));
                put_bits(T, tile_off(col + 1, r, trows), (unsigned short)(w[e] >> 16));
            }
            *reinterpret_cast<uint4*>(A + tile_off(r, c0 + 8 * g, 128)) =
                make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// The masked product of a backward MMA (64 accumulator columns of cell r) as BF16 into row r
// of D and into rows row0 .. row0 + 63 of column r of the transposed tile T (128 rows).
__device__ __forceinline__ void epilogue64_mask(unsigned taddr, const unsigned (&mask)[2],
                                                bool on, unsigned char* D, unsigned char* T,
                                                int row0, int r) {
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 32) {
        unsigned v[2][16];
        tmem_ld16(taddr + c0, v[0]);
        tmem_ld16(taddr + c0 + 16, v[1]);
        tmem_wait();
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const unsigned* u = v[g >> 1] + 8 * (g & 1);
            unsigned w[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int col = c0 + 8 * g + 2 * e;
                const bool ma = on && ((mask[col >> 5] >> (col & 31)) & 1u);
                const bool mb = on && ((mask[(col + 1) >> 5] >> ((col + 1) & 31)) & 1u);
                w[e] = pack_bf16(ma ? __uint_as_float(u[2 * e]) : 0.f,
                                 mb ? __uint_as_float(u[2 * e + 1]) : 0.f);
                put_bits(T, tile_off(row0 + col, r, 128), (unsigned short)(w[e] & 0xffffu));
                put_bits(T, tile_off(row0 + col + 1, r, 128), (unsigned short)(w[e] >> 16));
            }
            *reinterpret_cast<uint4*>(D + tile_off(r, c0 + 8 * g, 128)) =
                make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// n MMAs over K = 16 n: D (+)= A B^T, A [128][16 n] and B [N][16 n] K-major tiles.
__device__ __forceinline__ void mma_k(unsigned dt, unsigned a, unsigned a_lbo, unsigned b,
                                      unsigned b_lbo, unsigned n_out, int nk, bool acc) {
    for (int kk = 0; kk < nk; ++kk)
        mma(dt, sdesc(a + kk * 2 * a_lbo, a_lbo, 128), sdesc(b + kk * 2 * b_lbo, b_lbo, 128),
            idesc_n(n_out), (acc || kk > 0) ? 1 : 0);
}

// One CTA of 128 threads per SM (about 199 KB of shared memory) walks tiles of 128 phase cells
// in storage order; thread t owns cell t of the tile.  Outputs as learn.cu's k_mlp_bwd: cxy,
// lfs, dX9 per cell, lrho (atomic per spatial cell) and the parameter gradient (atomic, once per
// CTA at the end).
template <int NV>
__global__ void __launch_bounds__(128, 1) k_mlp_bwd_tc(const LearnBwdArgs b,
                                                      const unsigned char* image) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const LearnArgs& a = b.fw;
    unsigned char* W = sm + kBW;
    unsigned char* A1 = sm + kBA1;
    unsigned char* A2 = sm + kBA2;
    unsigned char* A3 = sm + kBA3;
    unsigned char* Z3 = sm + kBZ3;
    unsigned char* Z2 = sm + kBZ2;
    unsigned char* Z1 = sm + kBZ1;
    unsigned char* TDZ = sm + kTDZ;
    unsigned char* TH1 = sm + kTH1;
    unsigned char* TX = sm + kTX;
    unsigned char* TH2 = sm + kTH2;
    unsigned char* TZ3 = sm + kTZ3;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kBBar);
    unsigned* tslot = reinterpret_cast<unsigned*>(sm + kBBar + 8);
    const int t = threadIdx.x, warp = t >> 5;
    for (int i = t; i < kImageAll / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(W)[i] = reinterpret_cast<const uint4*>(image)[i];
    {   // constant parts of the operand tiles (never overwritten)
        const uint4 one = make_uint4(pack_bf16(1.f, 0.f), 0u, 0u, 0u);
        const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(A2 + tile_off(t, 64, 128)) = one;
        *reinterpret_cast<uint4*>(A2 + tile_off(t, 72, 128)) = zero;
        *reinterpret_cast<uint4*>(A3 + tile_off(t, 64, 128)) = one;
        *reinterpret_cast<uint4*>(A3 + tile_off(t, 72, 128)) = zero;
        *reinterpret_cast<uint4*>(Z3 + tile_off(t, 8, 128)) = zero;
        for (int rr = 64; rr < 80; ++rr) put_bf16(TH1, tile_off(rr, t, 80), rr == 64 ? 1.f : 0.f);
        for (int rr = 64; rr < 128; ++rr) put_bf16(TH2, tile_off(rr, t, 128), rr == 64 ? 1.f : 0.f);
        for (int rr = 2; rr < 16; ++rr) put_bf16(TZ3, tile_off(rr, t, 16), 0.f);
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         su32(tslot)),
                     "r"(kBTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *tslot;
    const unsigned trow = tmem + ((unsigned)(warp * 32) << 16);
    const unsigned w = su32(W);
    const float* f = a.f[0];
    const long long ncell = (long long)a.nx * a.ny;
    const long long n = ncell * NV * NV;
    const long long ntiles = (n + 127) / 128;
    unsigned phase = 0;
    bool failed = false, first = true;
    auto wait_mma = [&]() -> bool {
        bool ok = true;
        if (warp == 0) ok = wait_parity(bar, phase);
        phase ^= 1;
        const bool bad = __syncthreads_or(!ok);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        return !bad;
    };
    auto sync_for_mma = [&]() {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    };
    for (long long tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
        const long long i = tile * 128 + t;
        const bool on = i < n;
        int p = 0, x = 0, y = 0, jx = 0, jy = 0;
        Raw r;
        float X[kLNF];
        if (on) {
            split_index((unsigned)i, (unsigned)ncell, (unsigned)a.nx, p, x, y);
            jy = p / NV;
            jx = p % NV;
            load_raw<NV>(a, f, jx, jy, x, y, r);
            features_of<NV>(a, r, jx, jy, X);
        } else {
#pragma unroll
            for (int q = 0; q < kLNF; ++q) X[q] = 0.f;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint4 v;
            v.x = pack_bf16(X[8 * h + 0], X[8 * h + 1]);
            v.y = pack_bf16(X[8 * h + 2], X[8 * h + 3]);
            v.z = pack_bf16(X[8 * h + 4], X[8 * h + 5]);
            v.w = pack_bf16(X[8 * h + 6], X[8 * h + 7]);
            *reinterpret_cast<uint4*>(A1 + tile_off(t, 8 * h, 128)) = v;
        }
#pragma unroll
        for (int q = 0; q < kLNF; ++q) put_bf16(TX, tile_off(q, t, 16), X[q]);
        // forward: layers 1-3, keeping the activations (rows and transposed) and ReLU masks
        unsigned m1[2], m2[2];
        sync_for_mma();
        if (t == 0) {
            mma_k(tmem + kTD, su32(A1), 2048, w + kW1T, 1024, 64, 1, false);
            commit(bar);
        }
        if (!wait_mma()) { failed = true; break; }
        epilogue64_t(trow + kTD, A2, TH1, 80, t, m1);
        sync_for_mma();
        if (t == 0) {
            mma_k(tmem + kTD, su32(A2), 2048, w + kW2T, 1024, 64, kK2 / 16, false);
            commit(bar);
        }
        if (!wait_mma()) { failed = true; break; }
        epilogue64_t(trow + kTD, A3, TH2, 128, t, m2);
        sync_for_mma();
        if (t == 0) {
            mma_k(tmem + kTD, su32(A3), 2048, w + kW3T, 256, 16, kK2 / 16, false);
            commit(bar);
        }
        if (!wait_mma()) { failed = true; break; }
        float z0, z1;
        tmem_ld2(trow + kTD, z0, z1);
        // adjoint of the corrected drag fluxes (learn.cu's k_mlp_bwd, same operations)
        float dz30 = 0.f, dz31 = 0.f, lf = 0.f, inv = 0.f;
        if (on) {
            const float t0 = tanh_fast(z0), t1 = tanh_fast(z1);
            const float b0 = z0 > 0.f ? anti_bound(X[13], a.g) : kYMax;
            const float b1 = z1 > 0.f ? anti_bound(X[14], a.g) : kYMax;
            const float y0 = __fmul_rn(b0, t0), y1 = __fmul_rn(b1, t1);
            const float* L = b.lss;
            const float l0 = L[i];
            const float lxp = jx < NV - 1 ? __fsub_rn(L[i + ncell], l0) : 0.f;
            const float lxm = jx > 0 ? __fsub_rn(l0, L[i - ncell]) : 0.f;
            const float lyp = jy < NV - 1 ? __fsub_rn(L[i + NV * ncell], l0) : 0.f;
            const float lym = jy > 0 ? __fsub_rn(l0, L[i - NV * ncell]) : 0.f;
            const float cax = X[13], cay = X[14];
            lf = l0;
            lf = __fmaf_rn(fmaxf(cax, 0.f), lxp, lf);
            lf = __fmaf_rn(fminf(cax, 0.f), lxm, lf);
            lf = __fmaf_rn(fmaxf(cay, 0.f), lyp, lf);
            lf = __fmaf_rn(fminf(cay, 0.f), lym, lf);
            const float cx = __fmul_rn(y0, lxp), cy = __fmul_rn(y1, lyp);
            lf = __fsub_rn(__fsub_rn(lf, cx), cy);
            b.cxy[i] = cx;
            b.cxy[n + i] = cy;
            const float dy0 = __fmul_rn(lxp, __fsub_rn(r.fs[5], r.fs[4]));
            const float dy1 = __fmul_rn(lyp, __fsub_rn(r.fs[7], r.fs[4]));
            dz30 = __fmul_rn(dy0, __fmul_rn(b0, __fsub_rn(1.f, __fmul_rn(t0, t0))));
            dz31 = __fmul_rn(dy1, __fmul_rn(b1, __fsub_rn(1.f, __fmul_rn(t1, t1))));
            inv = r.fa.x;
        }
        *reinterpret_cast<uint4*>(Z3 + tile_off(t, 0, 128)) =
            make_uint4(pack_bf16(dz30, dz31), 0u, 0u, 0u);
        put_bf16(TZ3, tile_off(0, t, 16), dz30);
        put_bf16(TZ3, tile_off(1, t, 16), dz31);
        // network backward: dz2 = (dz3 W3^T)[h2 > 0], dz1 = (dz2 W2^T)[h1 > 0], dX = dz1 W1^T
        sync_for_mma();
        if (t == 0) {
            mma_k(tmem + kTD, su32(Z3), 2048, w + kB4, 1024, 64, 1, false);
            commit(bar);
        }
        if (!wait_mma()) { failed = true; break; }
        epilogue64_mask(trow + kTD, m2, on, Z2, TDZ, 0, t);
        sync_for_mma();
        if (t == 0) {
            mma_k(tmem + kTD, su32(Z2), 2048, w + kB5, 1024, 64, 4, false);
            commit(bar);
        }
        if (!wait_mma()) { failed = true; break; }
        epilogue64_mask(trow + kTD, m1, on, Z1, TDZ, 64, t);
        sync_for_mma();
        if (t == 0) {
            mma_k(tmem + kTD, su32(Z1), 2048, w + kB6, 256, 16, 4, false);
            // weight gradients, summed over the tile's cells into the CTA's accumulators
            mma_k(tmem + kTW2, su32(TDZ), 2048, su32(TH1), 1280, 80, 8, !first);
            mma_k(tmem + kTW1, su32(TDZ), 2048, su32(TX), 256, 16, 8, !first);
            mma_k(tmem + kTW3, su32(TH2), 2048, su32(TZ3), 256, 16, 8, !first);
            commit(bar);
        }
        if (!wait_mma()) { failed = true; break; }
        first = false;
        unsigned dx[16];
        tmem_ld16(trow + kTD, dx);
        tmem_wait();
        if (on) {
            float lr = 0.f;
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const float d = __uint_as_float(dx[q]);
                b.dX9[(size_t)q * n + i] = __fmul_rn(d, inv);
                lr = __fsub_rn(lr, __fmul_rn(__fmul_rn(d, X[q]), inv));
            }
            b.lfs[i] = lf;
            atomicAdd(&b.lrho[(long long)y * a.nx + x], lr);
        }
    }
    if (!failed && !first) {
        // rows 0..63 of the W2 accumulator: dW2^T[j][i] (i < 64) and db2[j] (i = 64)
        if (t < 64) {
#pragma unroll 1
            for (int c0 = 0; c0 < 80; c0 += 16) {
                unsigned v[16];
                tmem_ld16(trow + kTW2 + c0, v);
                tmem_wait();
                for (int e = 0; e < 16; ++e) {
                    const int col = c0 + e;
                    const float g = __uint_as_float(v[e]);
                    if (col < 64) atomicAdd(&b.grad[kOffW2 + col * kLNH + t], g);
                    else if (col == 64) atomicAdd(&b.grad[kOffB2 + t], g);
                }
            }
        } else {  // rows 64..127 of the W1 accumulator: dW1^T[i][q]; q = 15 meets the constant 1
            unsigned v[16];
            tmem_ld16(trow + kTW1, v);
            tmem_wait();
            const int ii = t - 64;
            for (int q = 0; q < kLNF; ++q) {
                const float g = __uint_as_float(v[q]);
                atomicAdd(&b.grad[kOffW1 + q * kLNH + ii], g);
                if (q == kLNF - 1) atomicAdd(&b.grad[kOffB1 + ii], g);
            }
        }
        // rows 0..64 of the W3 accumulator: dW3[i][o], row 64 (the constant) db3[o]
        float g0, g1;
        tmem_ld2(trow + kTW3, g0, g1);
        if (t < 64) {
            atomicAdd(&b.grad[kOffW3 + t * kLNO], g0);
            atomicAdd(&b.grad[kOffW3 + t * kLNO + 1], g1);
        } else if (t == 64) {
            atomicAdd(&b.grad[kOffB3], g0);
            atomicAdd(&b.grad[kOffB3 + 1], g1);
        }
    }
    if (failed && t == 0) atomicOr(const_cast<unsigned*>(&a.st->status), ST_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kBTmemCols)
                     : "memory");
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

size_t learn_tc_bytes() { return (size_t)kImageAll; }

cudaError_t launch_learn_tc_pack(const float* params, void* wtc, cudaStream_t s) {
    k_pack<<<24, 256, 0, s>>>(params, static_cast<unsigned char*>(wtc));
    k_pack_bwd<<<24, 256, 0, s>>>(params, static_cast<unsigned char*>(wtc));
    return cudaGetLastError();
}

cudaError_t launch_mlp_bwd_tc(int nv, const LearnBwdArgs& b, const void* wtc, int sm_count,
                              cudaStream_t s) {
    const long long n = (long long)b.fw.nx * b.fw.ny * nv * nv;
    const int grid = (int)std::max<long long>(1, std::min<long long>((n + 127) / 128, sm_count));
    const unsigned char* img = static_cast<const unsigned char*>(wtc);
    switch (nv) {
#define X(nn)                                                                                   \
    case nn: {                                                                                  \
        static bool attr = false;                                                               \
        if (!attr) {                                                                            \
            cudaError_t e = cudaFuncSetAttribute(k_mlp_bwd_tc<nn>,                              \
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                                 kBSmem);                                       \
            if (e != cudaSuccess) return e;                                                     \
            attr = true;                                                                        \
        }                                                                                       \
        k_mlp_bwd_tc<nn><<<grid, 128, kBSmem, s>>>(b, img);                                     \
        return cudaGetLastError();                                                              \
    }
        LEARN_TC_NV_LIST(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_mlp_tc(int nv, const LearnArgs& a, const void* wtc, int sm_count, bool units,
                          int k, cudaStream_t s) {
    const long long n = (long long)a.nx * a.ny * nv * nv;
    const bool by_units = units && a.nx % 128 == 0;
    const long long work = by_units ? (long long)a.ny * (a.nx / 128) : (n + 127) / 128;
    // five resident CTAs per SM: 5 x 64 TMEM columns and 5 x 40 KB of shared memory
    const int grid = (int)std::max<long long>(1, std::min<long long>(work, 5LL * sm_count));
    const unsigned char* img = static_cast<const unsigned char*>(wtc);
    switch (nv) {
#define X(nn)                                                                                   \
    case nn: {                                                                                  \
        static bool attr = false;                                                               \
        if (!attr) {                                                                            \
            cudaError_t e = cudaFuncSetAttribute(k_mlp_tc<nn>,                                  \
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                                 kSmemReq);                                     \
            if (e == cudaSuccess)                                                               \
                e = cudaFuncSetAttribute(k_mlp_tc_units<nn>,                                    \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemReq); \
            if (e != cudaSuccess) return e;                                                     \
            attr = true;                                                                        \
        }                                                                                       \
        if (by_units) k_mlp_tc_units<nn><<<grid, 128, kSmemReq, s>>>(a, img, k);                \
        else k_mlp_tc<nn><<<grid, 128, kSmemReq, s>>>(a, img, k);                               \
        return cudaGetLastError();                                                              \
    }
        LEARN_TC_NV_LIST(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lat

// Velocity moments of the 1D lattice state (density by summing over v, Sec. 4.2; mass
// normalisation sum f dx dv = N_p, Sec. 3.2) with compensated FP64 sums in a fixed order.
//
// Pass 1: one thread per column x sums its N_v values (Neumaier), writes the per-cell
// moments, and the block folds its columns into one compensated partial per work item
// (warp shuffles in a fixed butterfly order, then shared memory).  Pass 2: one block per
// instance folds that instance's item partials in item order.  Both passes are deterministic.
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "lat_internal.h"
#include "lat_reduce.h"

namespace lat {
namespace {

using namespace cs;

// One block (one thread per column of a work item's tile, blockDim = tile width) per item,
// grid-stride over items.  Every warp writes one partial per item: partials[item][warp][6].
//  FP32 storage: column sums in FP32 (ColumnSums: mass compensated, weights j, j^2 by FMA),
//    cross-column sums per warp in FP32 compensated form, FP64 from the warp partials on (FP64
//    is slow here).
//  FP64 storage: Neumaier FP64 throughout.
template <typename T>
__global__ void __launch_bounds__(1024) k_moments1d(const Mom1DArgs a, const int xpt) {
    const int nv = a.nv;
    const int J = (nv - 1) / 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    for (int it = blockIdx.x; it < a.nitems; it += gridDim.x) {
        const int2 item = a.items[it];
        const Inst1D in = a.inst[item.x];
        const T* f = static_cast<const T*>(a.f) + in.off;
        const int x = item.y + threadIdx.x;
        const bool on = x < in.nx;
        bool bad = false;
        double* p = a.partials + ((size_t)it * nwarps + warp) * 6;
        (void)xpt;
        if (sizeof(T) == sizeof(double)) {
            Comp s0{0, 0}, s1{0, 0}, s2{0, 0};
            if (on) {
                for (int jj = 0; jj < nv; ++jj) {
                    const double v = __dmul_rn((double)(jj - J), in.dv);
                    const double fv = (double)f[(size_t)jj * in.nx + x];
                    bad |= !isfinite(fv);
                    nadd(s0, fv);
                    nadd(s1, __dmul_rn(v, fv));
                    nadd(s2, __dmul_rn(__dmul_rn(v, v), fv));
                }
                const double m0 = nval(s0), m1 = nval(s1), m2 = nval(s2);
                const long long cell = in.xoff + x;
                if (a.rho) a.rho[cell] = m0 * in.dv;
                if (a.mean_v) a.mean_v[cell] = (m0 != 0.0) ? m1 / m0 : 0.0;
                if (a.mean_v2) a.mean_v2[cell] = (m0 != 0.0) ? m2 / m0 : 0.0;
            }
            warp_reduce3(s0, s1, s2);
            if (lane == 0) {
                p[0] = s0.s; p[1] = s0.c;
                p[2] = s1.s; p[3] = s1.c;
                p[4] = s2.s; p[5] = s2.c;
            }
        } else {
            ColumnSums sums;
            if (on && nv >= 5) {
                // two half-columns, as the fused step epilogue sums them (ColumnSums2)
                ColumnSums2 s2;
                for (int p = 1; p <= J; ++p) {
                    const float f0 = (float)f[(size_t)(p - 1) * in.nx + x];
                    const float f1 = (float)f[(size_t)(p - 1 + J) * in.nx + x];
                    bad |= !isfinite(f0) || !isfinite(f1);
                    const f2 jv = pk((float)(p - 1 - J), (float)(p - 1));
                    s2.add(jv, mul2(jv, jv), pk(f0, f1));
                }
                const float fl = (float)f[(size_t)(nv - 1) * in.nx + x];
                bad |= !isfinite(fl);
                s2.add_hi((float)J, fl);
                sums = s2.collapse();
            } else if (on) {
                for (int jj = 0; jj < nv; ++jj) {
                    const float fv = (float)f[(size_t)jj * in.nx + x];
                    bad |= !isfinite(fv);
                    sums.add((float)(jj - J), fv);
                }
            }
            if (on) {
                if (a.rho || a.mean_v || a.mean_v2) {  // FP64 per cell only when asked for
                    Comp s0, s1, s2;
                    sums.result(in.dv, s0, s1, s2);
                    const double m0 = nval(s0), m1 = nval(s1), m2 = nval(s2);
                    const long long cell = in.xoff + x;
                    if (a.rho) a.rho[cell] = m0 * in.dv;
                    if (a.mean_v) a.mean_v[cell] = (m0 != 0.0) ? m1 / m0 : 0.0;
                    if (a.mean_v2) a.mean_v2[cell] = (m0 != 0.0) ? m2 / m0 : 0.0;
                }
            }
            warp_partial_1d(sums, in.dv, p);
        }
        if (bad) atomicOr(&a.st->status, ST_NUMERIC);
    }
}

// Eight lanes per instance (four instances per warp) fold that instance's partials (per_item
// partials per work item): lane l of the group takes partials l, l + 8, ... in order, then a
// fixed three-level butterfly; glob[i] = [M, P, E].  (FP64 is slow on this part: eight lanes
// keep the butterfly's share of the merges small, and the order stays fixed.)
constexpr int kFinLanes = 8;

__global__ void k_finalize1d(const double* partials, const int* begin, const Inst1D* inst,
                             int n_inst, double* glob, int per_item) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (32 / kFinLanes) + lane / kFinLanes;
    const int l = lane % kFinLanes;
    const bool on = i < n_inst;
    Comp t0{0, 0}, t1{0, 0}, t2{0, 0};
    if (on) {
        for (long long it = (long long)begin[i] * per_item + l;
             it < (long long)begin[i + 1] * per_item; it += kFinLanes) {
            nmerge(t0, Comp{partials[it * 6 + 0], partials[it * 6 + 1]});
            nmerge(t1, Comp{partials[it * 6 + 2], partials[it * 6 + 3]});
            nmerge(t2, Comp{partials[it * 6 + 4], partials[it * 6 + 5]});
        }
    }
    for (int off = kFinLanes / 2; off > 0; off >>= 1) {  // within the group of eight lanes
        const Comp o0 = shfl_down(t0, off), o1 = shfl_down(t1, off), o2 = shfl_down(t2, off);
        nmerge(t0, o0);
        nmerge(t1, o1);
        nmerge(t2, o2);
    }
    if (on && l == 0) {
        const double w = inst[i].dx * inst[i].dv;
        glob[i * 3 + 0] = nval(t0) * w;
        glob[i * 3 + 1] = nval(t1) * w;
        glob[i * 3 + 2] = nval(t2) * w;
    }
}

// ---- allocation-free variant: global moments of one FP32 lattice, static scratch ------------
constexpr int kNoAllocTile = 128;

// Per-tile compensated partials of lat_moments1d_noalloc: [tile][M, P, E][sum, compensation].
// Every GPU that loads this library holds this array until the process exits.
static __device__ __align__(256) double g_noalloc_partials[LAT_NOALLOC_MAX_TILES * 6];

// One block per 128-column tile: FP32 column sums (ColumnSums), Neumaier over the tile's columns.
__global__ void __launch_bounds__(kNoAllocTile)
    k_moments1d_noalloc(const float* f, int nv, int nx, double dv, double* partials) {
    __shared__ Comp red[3][kNoAllocTile / 32];
    const int J = (nv - 1) / 2;
    const int x = blockIdx.x * kNoAllocTile + threadIdx.x;
    Comp t0{0, 0}, t1{0, 0}, t2{0, 0};
    if (x < nx) {
        ColumnSums sums;
        if (nv >= 5) {  // the two half-columns of lat_moments (ColumnSums2 order)
            ColumnSums2 s2;
            for (int p = 1; p <= J; ++p) {
                const f2 jv = pk((float)(p - 1 - J), (float)(p - 1));
                s2.add(jv, mul2(jv, jv),
                       pk(f[(size_t)(p - 1) * nx + x], f[(size_t)(p - 1 + J) * nx + x]));
            }
            s2.add_hi((float)J, f[(size_t)(nv - 1) * nx + x]);
            sums = s2.collapse();
        } else {
            for (int jj = 0; jj < nv; ++jj) sums.add((float)(jj - J), f[(size_t)jj * nx + x]);
        }
        sums.result(dv, t0, t1, t2);
    }
    for (int off = 16; off > 0; off >>= 1) {
        Comp o0 = shfl_down(t0, off), o1 = shfl_down(t1, off), o2 = shfl_down(t2, off);
        nmerge(t0, o0);
        nmerge(t1, o1);
        nmerge(t2, o2);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][warp] = t0;
        red[1][warp] = t1;
        red[2][warp] = t2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Comp z[3] = {{0, 0}, {0, 0}, {0, 0}};
        for (int w = 0; w < kNoAllocTile / 32; ++w)
            for (int q = 0; q < 3; ++q) nmerge(z[q], red[q][w]);
        double* p = partials + (size_t)blockIdx.x * 6;
        for (int q = 0; q < 3; ++q) {
            p[2 * q] = z[q].s;
            p[2 * q + 1] = z[q].c;
        }
    }
}

// Fold the tile partials in tile order: out = [M, P, E] * dx dv.
__global__ void k_finalize_noalloc(const double* partials, int ntiles, double w, double* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    Comp t[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int b = 0; b < ntiles; ++b)
        for (int q = 0; q < 3; ++q) nmerge(t[q], Comp{partials[b * 6 + 2 * q], partials[b * 6 + 2 * q + 1]});
    for (int q = 0; q < 3; ++q) out[q] = nval(t[q]) * w;
}

// Device address of the static scratch, looked up once per device (with that device current).
int noalloc_scratch(double** out) {
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static double* addr[kMaxDevices] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LAT_ECUDA;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) {
            fprintf(stderr, "lat_moments1d_noalloc: cudaGetSymbolAddress failed: %s\n",
                    cudaGetErrorString(e));
            return LAT_ECUDA;
        }
        addr[dev] = static_cast<double*>(p);
    }
    *out = addr[dev];
    return LAT_OK;
}

}  // namespace

cudaError_t launch_moments1d(int dtype, int block, int xpt, int grid, const Mom1DArgs& a,
                             cudaStream_t s) {
    if (grid <= 0) return cudaSuccess;
    if (dtype == LAT_F32) k_moments1d<float><<<grid, block, 0, s>>>(a, xpt);
    else if (dtype == LAT_F64) k_moments1d<double><<<grid, block, 0, s>>>(a, xpt);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_finalize1d(const double* partials, const int* inst_item_begin,
                              const Inst1D* inst, int n_inst, double* glob, int per_item,
                              cudaStream_t s) {
    if (n_inst <= 0) return cudaSuccess;
    const int groups = 32 / kFinLanes;
    k_finalize1d<<<(n_inst + groups - 1) / groups, 32, 0, s>>>(partials, inst_item_begin, inst,
                                                               n_inst, glob, per_item);
    return cudaGetLastError();
}

}  // namespace lat

extern "C" int lat_moments1d_noalloc(const float* f, int nv, int nx, double dx, double dv,
                                     double* globals, void* stream) {
    if (!f || !globals || nv < 1 || nv % 2 == 0 || nx < 1 || !(dx > 0) || !(dv > 0))
        return LAT_EINVAL;
    const int ntiles = (nx + lat::kNoAllocTile - 1) / lat::kNoAllocTile;
    if (ntiles > LAT_NOALLOC_MAX_TILES) {
        fprintf(stderr,
                "lat_moments1d_noalloc: N_x = %d exceeds the static scratch limit of %d columns\n",
                nx, LAT_NOALLOC_MAX_TILES * lat::kNoAllocTile);
        return LAT_EINVAL;
    }
    double* scratch = nullptr;
    const int rc = lat::noalloc_scratch(&scratch);
    if (rc != LAT_OK) return rc;
    const cudaStream_t s = (cudaStream_t)stream;
    lat::k_moments1d_noalloc<<<ntiles, lat::kNoAllocTile, 0, s>>>(f, nv, nx, dv, scratch);
    lat::k_finalize_noalloc<<<1, 32, 0, s>>>(scratch, ntiles, dx * dv, globals);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        fprintf(stderr, "lat_moments1d_noalloc: launch failed: %s\n", cudaGetErrorString(e));
        return LAT_ECUDA;
    }
    return LAT_OK;
}

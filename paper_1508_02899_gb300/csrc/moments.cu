// Velocity moments of the 1D lattice state (density by summing over v, Sec. 4.2; mass
// normalisation sum f dx dv = N_p, Sec. 3.2) with compensated FP64 sums in a fixed order.
//
// Pass 1: one thread per column x sums its N_v values (Neumaier), writes the per-cell
// moments, and the block folds its columns into one compensated partial per work item
// (warp shuffles in a fixed butterfly order, then shared memory).  Pass 2: one block per
// instance folds that instance's item partials in item order.  Both passes are deterministic.
#include <math.h>

#include "lat_internal.h"

namespace lat {
namespace {

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

// Kahan-compensated FP32 accumulator (c holds the negated running error).
struct FComp {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float y = __fsub_rn(x, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
};

__device__ __forceinline__ Comp shfl_down(const Comp& a, int off) {
    return Comp{__shfl_down_sync(0xffffffffu, a.s, off), __shfl_down_sync(0xffffffffu, a.c, off)};
}

template <typename T>
__global__ void __launch_bounds__(1024) k_moments1d(const Mom1DArgs a, const int xpt) {
    __shared__ Comp red[3][32];
    const int nv = a.nv;
    const int J = (nv - 1) / 2;
    for (int it = blockIdx.x; it < a.nitems; it += gridDim.x) {
        const int2 item = a.items[it];
        const Inst1D in = a.inst[item.x];
        const T* f = static_cast<const T*>(a.f) + in.off;
        Comp t0{0, 0}, t1{0, 0}, t2{0, 0};
        bool bad = false;
        for (int p = 0; p < xpt; ++p) {
            const int x = item.y + threadIdx.x + p * blockDim.x;
            if (x >= in.nx) continue;
            Comp s0{0, 0}, s1{0, 0}, s2{0, 0};
            if (sizeof(T) == sizeof(double)) {
                for (int jj = 0; jj < nv; ++jj) {
                    const double v = __dmul_rn((double)(jj - J), in.dv);
                    const double fv = (double)f[(size_t)jj * in.nx + x];
                    bad |= !isfinite(fv);
                    nadd(s0, fv);
                    nadd(s1, __dmul_rn(v, fv));
                    nadd(s2, __dmul_rn(__dmul_rn(v, v), fv));
                }
            } else {
                // FP32 storage: the column sums run in FP32 with Kahan compensation (exact
                // integer weights j, j^2), which keeps them at the storage precision; only the
                // reduction over cells is FP64 (FP64 throughput is low on this GPU).
                FComp a0, a1, a2;
                for (int jj = 0; jj < nv; ++jj) {
                    const float fv = (float)f[(size_t)jj * in.nx + x];
                    const float j = (float)(jj - J);
                    bad |= !isfinite(fv);
                    a0.add(fv);
                    a1.add(j * fv);
                    a2.add(j * j * fv);
                }
                // Kahan's c is the negated lost part: the sum is s - c
                s0 = Comp{(double)a0.s, -(double)a0.c};
                s1 = Comp{__dmul_rn((double)a1.s, in.dv), -__dmul_rn((double)a1.c, in.dv)};
                const double dv2 = __dmul_rn(in.dv, in.dv);
                s2 = Comp{__dmul_rn((double)a2.s, dv2), -__dmul_rn((double)a2.c, dv2)};
            }
            const double m0 = nval(s0), m1 = nval(s1), m2 = nval(s2);
            const long long cell = in.xoff + x;
            if (a.rho) a.rho[cell] = m0 * in.dv;
            if (a.mean_v) a.mean_v[cell] = (m0 != 0.0) ? m1 / m0 : 0.0;
            if (a.mean_v2) a.mean_v2[cell] = (m0 != 0.0) ? m2 / m0 : 0.0;
            nmerge(t0, s0);
            nmerge(t1, s1);
            nmerge(t2, s2);
        }
        if (bad) atomicOr(&a.st->status, ST_NUMERIC);
        // fixed-order reduction: butterfly within warps, then warp 0 over the warp results
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
        if (warp == 0) {
            const int nw = (blockDim.x + 31) >> 5;
            Comp z{0, 0};
            t0 = lane < nw ? red[0][lane] : z;
            t1 = lane < nw ? red[1][lane] : z;
            t2 = lane < nw ? red[2][lane] : z;
            for (int off = 16; off > 0; off >>= 1) {
                Comp o0 = shfl_down(t0, off), o1 = shfl_down(t1, off), o2 = shfl_down(t2, off);
                nmerge(t0, o0);
                nmerge(t1, o1);
                nmerge(t2, o2);
            }
            if (lane == 0) {
                double* p = a.partials + (size_t)it * 6;
                p[0] = t0.s; p[1] = t0.c;
                p[2] = t1.s; p[3] = t1.c;
                p[4] = t2.s; p[5] = t2.c;
            }
        }
        __syncthreads();
    }
}

// One block per instance: fold the item partials in item order; glob[i] = [M, P, E].
__global__ void k_finalize1d(const double* partials, const int* begin, const Inst1D* inst,
                             int n_inst, double* glob) {
    const int i = blockIdx.x;
    if (i >= n_inst || threadIdx.x != 0) return;
    Comp t[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int it = begin[i]; it < begin[i + 1]; ++it)
        for (int q = 0; q < 3; ++q) nmerge(t[q], Comp{partials[it * 6 + 2 * q], partials[it * 6 + 2 * q + 1]});
    const double w = inst[i].dx * inst[i].dv;
    for (int q = 0; q < 3; ++q) glob[i * 3 + q] = nval(t[q]) * w;
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
                              const Inst1D* inst, int n_inst, double* glob, cudaStream_t s) {
    if (n_inst <= 0) return cudaSuccess;
    k_finalize1d<<<n_inst, 32, 0, s>>>(partials, inst_item_begin, inst, n_inst, glob);
    return cudaGetLastError();
}

}  // namespace lat

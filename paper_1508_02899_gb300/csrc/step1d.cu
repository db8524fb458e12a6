// One fused time step of the 1D phase-space lattice (Section 2 of arXiv:1508.02899):
// exact streaming in x, first-order upwind Stokes-drag flux in v, velocity diffusion.
//
// Work decomposition: a work item is one x-tile of one instance; a persistent grid walks the
// item list.  Each thread owns one spatial column x (XPT columns per thread), gathers its
// post-streaming column f*(x, j) = f(x - j, j) with one coalesced load per velocity plane
// (the gather *is* the streaming step, so it costs no extra pass), applies the drag and the
// diffusion in registers and writes the column once.  HBM traffic per cell: one read and one
// write of f.  The flow u(x, t_n) is evaluated in the same kernel from the mode amplitudes;
// the first tile of every instance also advances those amplitudes to t_{n+1} (parity
// ping-pong, so no tile reads what another tile of the same launch writes).
#include <math.h>

#include "lat_internal.h"

namespace lat {
namespace {

__device__ __forceinline__ void sincospi_t(float y, float* s, float* c) { sincospif(y, s, c); }
__device__ __forceinline__ void sincospi_t(double y, double* s, double* c) { sincospi(y, s, c); }

template <typename T>
__device__ __forceinline__ T ldg_t(const T* p) { return __ldg(p); }

// Fluid velocity at column x of an instance at time t_n.
template <typename T>
__device__ __forceinline__ T flow_at(const Step1DArgs& a, const Inst1D& in, const double* amp,
                                     int x) {
    if (a.flow_kind == LAT_FLOW_FIELD) return static_cast<const T*>(a.field)[in.xoff + x];
    if (a.flow_kind != LAT_FLOW_MODES) return T(0);
    const int M = a.nmodes;
    T u = T(0);
    for (int m = 0; m < M; ++m) {
        // phase 2 pi k x / N_x reduced exactly in integers, then sin/cos of pi * (2 kx / N_x)
        long long kx = ((long long)a.k[m] * x) % in.nx;
        if (kx < 0) kx += in.nx;
        T s, c;
        sincospi_t(T(2 * kx) / T(in.nx), &s, &c);
        u += T(amp[m]) * c + T(amp[M + m]) * s;
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
        a.amp_w[(1 - par) * a.amp_stride + (long long)inst * M2 + t] =
            __dadd_rn(__dmul_rn(old, in.ou_e), __dmul_rn(in.ou_s, xi));
    }
    if (!have && threadIdx.x == 0) atomicOr(&a.st->status, ST_NOISE);
}

// Drag then diffusion on a register-resident column (Section 2, flux form).
//   drag:  c F_{j+1/2} = max(g (w - j), 0) f_j + min(g (w - j - 1), 0) f_{j+1},  zero at walls,
//          f_j <- f_j - (c F_{j+1/2} - c F_{j-1/2}),  g = dt/tau_p, w = u/dv, c = dt/dv;
//   diffusion: D_{j+1/2} = r (f_{j+1} - f_j), zero at walls, f_j <- f_j + D_{j+1/2} - D_{j-1/2}.
template <typename T, int NV>
__device__ __forceinline__ void column_update(T (&f)[NV], T w, T g, T r) {
    constexpr int J = (NV - 1) / 2;
    T Fprev = T(0);
#pragma unroll
    for (int jj = 0; jj < NV; ++jj) {
        T Fnext = T(0);
        if (jj < NV - 1) {
            const T caj = g * (w - T(jj - J));
            const T can = g * (w - T(jj + 1 - J));
            Fnext = fmax(caj, T(0)) * f[jj] + fmin(can, T(0)) * f[jj + 1];
        }
        f[jj] = f[jj] - (Fnext - Fprev);
        Fprev = Fnext;
    }
    T Dprev = T(0);
#pragma unroll
    for (int jj = 0; jj < NV; ++jj) {
        const T Dnext = (jj < NV - 1) ? r * (f[jj + 1] - f[jj]) : T(0);
        f[jj] = f[jj] + (Dnext - Dprev);
        Dprev = Dnext;
    }
}

// Largest block that still leaves each thread enough registers for its XPT columns.
template <typename T, int NV, int XPT>
struct MaxThreads {
    static constexpr int words = NV * XPT * (int)(sizeof(T) / 4);
    static constexpr int value = words > 56 ? 256 : (words > 20 ? 512 : 1024);
};

template <typename T, int NV, int XPT>
__global__ void __launch_bounds__(MaxThreads<T, NV, XPT>::value)
    k_step1d_reg(const Step1DArgs a, const int kstep) {
    constexpr int J = (NV - 1) / 2;
    const long long step = a.st->step + kstep;
    const int par = (int)(step & 1);
    for (int it = a.item_begin + blockIdx.x; it < a.item_end; it += gridDim.x) {
        const int2 item = a.items[it];
        const Inst1D in = a.inst[item.x];
        const int nx = in.nx;
        const T g = T(in.g), r = T(in.r), inv_dv = T(in.inv_dv);
        const T* __restrict__ src = static_cast<const T*>(a.f[par]) + in.off;
        T* __restrict__ dst = static_cast<T*>(a.f[par ^ 1]) + in.off;
        const double* amp = a.amp + par * a.amp_stride + (long long)item.x * 2 * a.nmodes;
#pragma unroll
        for (int p = 0; p < XPT; ++p) {
            const int x = item.y + threadIdx.x + p * blockDim.x;
            if (x < nx) {
                const T w = flow_at<T>(a, in, amp, x) * inv_dv;
                T f[NV];
                if (nx >= J) {
#pragma unroll
                    for (int jj = 0; jj < NV; ++jj) {
                        int xs = x - (jj - J);
                        xs += (xs < 0) ? nx : 0;
                        xs -= (xs >= nx) ? nx : 0;
                        f[jj] = ldg_t(src + (size_t)jj * nx + xs);
                    }
                } else {
#pragma unroll
                    for (int jj = 0; jj < NV; ++jj) {
                        int xs = (x - (jj - J)) % nx;
                        xs += (xs < 0) ? nx : 0;
                        f[jj] = ldg_t(src + (size_t)jj * nx + xs);
                    }
                }
                column_update<T, NV>(f, w, g, r);
#pragma unroll
                for (int jj = 0; jj < NV; ++jj) dst[(size_t)jj * nx + x] = f[jj];
                if (g * (T(J) + fabs(w)) > T(1)) atomicOr(&a.st->status, ST_CFL);
            }
        }
        if (!a.dry && !a.frozen && a.flow_kind == LAT_FLOW_MODES && item.y == 0)
            advance_amplitudes(a, item.x, in, step, par);
    }
}

// Any odd N_v: the column is streamed through a sliding window of registers
// (s_j, s_{j+1} for the drag flux; d_{j-1}, d_j for the diffusion flux).
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
        const T g = T(in.g), r = T(in.r), inv_dv = T(in.inv_dv);
        const T* __restrict__ src = static_cast<const T*>(a.f[par]) + in.off;
        T* __restrict__ dst = static_cast<T*>(a.f[par ^ 1]) + in.off;
        const double* amp = a.amp + par * a.amp_stride + (long long)item.x * 2 * a.nmodes;
        const int x = item.y + threadIdx.x;
        if (x < nx) {
            const T w = flow_at<T>(a, in, amp, x) * inv_dv;
            auto load = [&](int jj) -> T {
                int xs = (x - (jj - J)) % nx;
                xs += (xs < 0) ? nx : 0;
                return ldg_t(src + (size_t)jj * nx + xs);
            };
            T s = load(0);
            T Fprev = T(0), Dprev = T(0), dprev = T(0);
#pragma unroll 4
            for (int jj = 0; jj < NV; ++jj) {
                T snext = T(0), Fnext = T(0);
                if (jj < NV - 1) {
                    snext = load(jj + 1);
                    Fnext = fmax(g * (w - T(jj - J)), T(0)) * s +
                            fmin(g * (w - T(jj + 1 - J)), T(0)) * snext;
                }
                const T d = s - (Fnext - Fprev);
                Fprev = Fnext;
                if (jj > 0) {
                    const T D = r * (d - dprev);
                    dst[(size_t)(jj - 1) * nx + x] = dprev + (D - Dprev);
                    Dprev = D;
                }
                dprev = d;
                s = snext;
            }
            dst[(size_t)(NV - 1) * nx + x] = dprev + (T(0) - Dprev);
            if (g * (T(J) + fabs(w)) > T(1)) atomicOr(&a.st->status, ST_CFL);
        }
        if (!a.dry && !a.frozen && a.flow_kind == LAT_FLOW_MODES && item.y == 0)
            advance_amplitudes(a, item.x, in, step, par);
    }
}

__global__ void k_advance_step(DevState* st, long long n) { st->step += n; }

template <typename T, int NV>
cudaError_t launch_reg(int block, int xpt, int grid, const Step1DArgs& a, int kstep,
                       cudaStream_t s) {
    if (xpt == 1) {
        if (block > MaxThreads<T, NV, 1>::value) return cudaErrorInvalidValue;
        k_step1d_reg<T, NV, 1><<<grid, block, 0, s>>>(a, kstep);
    } else if (xpt == 2) {
        if (block > MaxThreads<T, NV, 2>::value) return cudaErrorInvalidValue;
        k_step1d_reg<T, NV, 2><<<grid, block, 0, s>>>(a, kstep);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_t(int nv, int block, int xpt, int grid, const Step1DArgs& a, int kstep,
                     cudaStream_t s) {
    switch (nv) {
        case 3: return launch_reg<T, 3>(block, xpt, grid, a, kstep, s);
        case 5: return launch_reg<T, 5>(block, xpt, grid, a, kstep, s);
        case 9: return launch_reg<T, 9>(block, xpt, grid, a, kstep, s);
        case 17: return launch_reg<T, 17>(block, xpt, grid, a, kstep, s);
        case 33: return launch_reg<T, 33>(block, xpt, grid, a, kstep, s);
        case 65: return launch_reg<T, 65>(block, xpt, grid, a, kstep, s);
        default:
            if (xpt != 1 || block > 512) return cudaErrorInvalidValue;
            k_step1d_any<T><<<grid, block, 0, s>>>(a, kstep, nv);
            return cudaGetLastError();
    }
}

}  // namespace

int step1d_max_block(int dtype, int nv, int xpt) {
    const bool reg = nv == 3 || nv == 5 || nv == 9 || nv == 17 || nv == 33 || nv == 65;
    if (!reg) return xpt == 1 ? 512 : 0;
    const int words = nv * xpt * (dtype == LAT_F64 ? 2 : 1);
    return words > 56 ? 256 : (words > 20 ? 512 : 1024);
}

bool step1d_supported(int dtype, int nv, int xpt) {
    if (dtype != LAT_F32 && dtype != LAT_F64) return false;
    if (nv < 1 || (nv % 2) == 0 || nv > 129) return false;
    return step1d_max_block(dtype, nv, xpt) > 0;
}

cudaError_t launch_step1d(int dtype, int nv, int block, int xpt, int grid, const Step1DArgs& a,
                          int kstep, cudaStream_t s) {
    if (grid <= 0) return cudaSuccess;
    if (dtype == LAT_F32) return launch_t<float>(nv, block, xpt, grid, a, kstep, s);
    if (dtype == LAT_F64) return launch_t<double>(nv, block, xpt, grid, a, kstep, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_advance_step(DevState* st, long long n, cudaStream_t s) {
    k_advance_step<<<1, 1, 0, s>>>(st, n);
    return cudaGetLastError();
}

}  // namespace lat

// Observables of the phase-space density that the paper uses to benchmark the method (Sec. 3.2):
// the second moment of the coarse-grained density, Eq. (def_coarse), and the Eulerian first-order
// velocity structure function, Eq. (def_eulS1).  They start from the per-cell density rho that the
// moment kernels produce (FP64) and, for S1, from the state itself.
//
// Lattice forms: r = w dx for whole numbers w of cells, the window of cell i covering cells
// i .. i + w - 1 (periodic; w x w squares in 2D); separations s dx; velocity differences
// |j - j'| dv.  All reductions are compensated FP64 sums in a fixed order (deterministic).
#include "lat_internal.h"
#include "lat_reduce.h"

namespace lat {
namespace {

using namespace cs;

constexpr int kObsThreads = 256;

// Fixed-order block reduction of one compensated sum per thread (result in thread 0).
__device__ __forceinline__ Comp block_reduce(Comp t) {
    __shared__ Comp wsum[kObsThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    warp_reduce(t);
    __syncthreads();  // wsum may still be read by an earlier call
    if (lane == 0) wsum[warp] = t;
    __syncthreads();
    Comp z{0, 0};
    if (threadIdx.x == 0)
        for (int w = 0; w < kObsThreads / 32; ++w) nmerge(z, wsum[w]);
    return z;
}

// Exclusive prefix sums of rho per instance, compensated (hi + lo): instance k's n + 1 sums
// start at xoff_k + k.  One block per instance; chunks of the block width in order, a warp scan
// per chunk.  Window sums are then differences of prefix sums, accurate to about u of the window
// (u = 2^-53) however long the instance.
__global__ void __launch_bounds__(kObsThreads)
    k_prefix1d(const double* rho, const Inst1D* inst, int n_inst, double* Ph, double* Pl) {
    __shared__ Comp wtot[kObsThreads / 32];
    __shared__ Comp carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = blockIdx.x; k < n_inst; k += gridDim.x) {
        const Inst1D in = inst[k];
        const double* r = rho + in.xoff;
        double* ph = Ph + in.xoff + k;
        double* pl = Pl + in.xoff + k;
        if (threadIdx.x == 0) carry = Comp{0, 0};
        __syncthreads();
        for (int base = 0; base < in.nx; base += kObsThreads) {
            const int i = base + threadIdx.x;
            Comp incl{i < in.nx ? r[i] : 0.0, 0.0};
            for (int off = 1; off < 32; off <<= 1) {  // inclusive scan, predecessors first
                const Comp o = shfl_up(incl, off);
                if (lane >= off) {
                    Comp t = o;
                    nmerge(t, incl);
                    incl = t;
                }
            }
            Comp excl = shfl_up(incl, 1);
            if (lane == 0) excl = Comp{0, 0};
            if (lane == 31) wtot[warp] = incl;
            __syncthreads();
            Comp before = carry;
            for (int w = 0; w < warp; ++w) nmerge(before, wtot[w]);
            if (i < in.nx) {
                Comp v = before;
                nmerge(v, excl);
                ph[i] = v.s;
                pl[i] = v.c;
            }
            __syncthreads();
            if (threadIdx.x == kObsThreads - 1) {
                nmerge(before, incl);
                carry = before;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            ph[in.nx] = carry.s;
            pl[in.nx] = carry.c;
        }
        __syncthreads();
    }
}

// <rho_r^2> per (instance, width): block per pair, threads over cells.
__global__ void __launch_bounds__(kObsThreads)
    k_coarse1d(const double* Ph, const double* Pl, const Inst1D* inst, int n_inst,
               const int* widths, int nw, double* out) {
    for (int b = blockIdx.x; b < n_inst * nw; b += gridDim.x) {
        const int k = b / nw, q = b % nw;
        const Inst1D in = inst[k];
        const double* ph = Ph + in.xoff + k;
        const double* pl = Pl + in.xoff + k;
        const int w = widths[q], n = in.nx;
        Comp t{0, 0};
        for (int i = threadIdx.x; i < n; i += kObsThreads) {
            double m;
            if (i + w <= n) {
                m = (ph[i + w] - ph[i]) + (pl[i + w] - pl[i]);
            } else {
                const int e = i + w - n;
                m = ((ph[n] - ph[i]) + ph[e]) + ((pl[n] - pl[i]) + pl[e]);
            }
            const double r = m * in.dx;
            nadd(t, r * r);
        }
        const Comp z = block_reduce(t);
        if (threadIdx.x == 0) out[b] = nval(z) / n;
    }
}

// Compensated summed-area table of rho (ny x nx): S[y (nx + 1) + x] = the sum of rho over rows
// < y and columns < x, as hi + lo.
__global__ void k_sat_rows(const double* rho, int nx, int ny, double* Sh, double* Sl) {
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y > ny) return;
    double* sh = Sh + (size_t)y * (nx + 1);
    double* sl = Sl + (size_t)y * (nx + 1);
    Comp acc{0, 0};
    sh[0] = 0.0;
    sl[0] = 0.0;
    for (int x = 0; x < nx; ++x) {
        if (y > 0) nadd(acc, rho[(size_t)(y - 1) * nx + x]);
        sh[x + 1] = acc.s;
        sl[x + 1] = acc.c;
    }
}
__global__ void k_sat_cols(int nx, int ny, double* Sh, double* Sl) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x > nx) return;
    Comp acc{0, 0};
    for (int y = 1; y <= ny; ++y) {
        const size_t c = (size_t)y * (nx + 1) + x;
        nmerge(acc, Comp{Sh[c], Sl[c]});
        Sh[c] = acc.s;
        Sl[c] = acc.c;
    }
}

// sum over rows [y0, y1), columns [x0, x1), from the compensated table
__device__ __forceinline__ double rect(const double* Sh, const double* Sl, int nx1, int y0,
                                       int y1, int x0, int x1) {
    const size_t a = (size_t)y0 * nx1 + x0, b = (size_t)y0 * nx1 + x1;
    const size_t c = (size_t)y1 * nx1 + x0, d = (size_t)y1 * nx1 + x1;
    return ((Sh[d] - Sh[b]) - (Sh[c] - Sh[a])) + ((Sl[d] - Sl[b]) - (Sl[c] - Sl[a]));
}

// 2D <rho_r^2> per width: w x w windows with periodic wrap (up to four rectangles).
__global__ void __launch_bounds__(kObsThreads)
    k_coarse2d(const double* Sh, const double* Sl, int nx, int ny, double dx, const int* widths,
               int nw, double* out) {
    const int nx1 = nx + 1;
    const long long ncell = (long long)nx * ny;
    for (int q = blockIdx.x; q < nw; q += gridDim.x) {
        const int w = widths[q];
        Comp t{0, 0};
        for (long long c = threadIdx.x; c < ncell; c += kObsThreads) {
            const int y = (int)(c / nx), x = (int)(c % nx);
            const int ye = y + w, xe = x + w;
            const int ya = ye <= ny ? ye : ny, xa = xe <= nx ? xe : nx;
            double m = rect(Sh, Sl, nx1, y, ya, x, xa);
            if (ye > ny) m += rect(Sh, Sl, nx1, 0, ye - ny, x, xa);
            if (xe > nx) m += rect(Sh, Sl, nx1, y, ya, 0, xe - nx);
            if (ye > ny && xe > nx) m += rect(Sh, Sl, nx1, 0, ye - ny, 0, xe - nx);
            const double r = m * dx * dx;
            nadd(t, r * r);
        }
        const Comp z = block_reduce(t);
        if (threadIdx.x == 0) out[q] = nval(z) / (double)ncell;
    }
}

// Eq. (def_eulS1) per (instance, separation): the pair sum over velocity cells of cell i and
// cell i + s, sum_j a_j sum_j' b_j' |j - j'|, by two running sums without cancellation:
//   T_j = sum_{j' < j} b_j' (j - j'),  T_{j+1} = T_j + sum_{j' <= j} b_j'   (forward),
//   U_j = sum_{j' > j} b_j' (j' - j),  U_{j-1} = U_j + sum_{j' >= j} b_j'   (backward),
// then times dv^3; the denominator rho_i rho_{i+s}.  T = float for FP32 states (errors about
// N_v u of the positive sums), double for FP64 states.
template <typename T>
__global__ void __launch_bounds__(kObsThreads)
    k_s1_1d(const T* f, const Inst1D* inst, int n_inst, int nv, const double* rho,
            const int* seps, int ns, double* num, double* den) {
    for (int b = blockIdx.x; b < n_inst * ns; b += gridDim.x) {
        const int k = b / ns, q = b % ns;
        const Inst1D in = inst[k];
        const int n = in.nx, s = seps[q];
        const T* fk = f + in.off;
        Comp tn{0, 0}, td{0, 0};
        for (int i = threadIdx.x; i < n; i += kObsThreads) {
            const int i2 = i + s < n ? i + s : i + s - n;
            T acc = T(0), B = T(0), run = T(0);
            for (int j = 0; j < nv; ++j) {
                const T a = fk[(size_t)j * n + i];
                acc += a * run;
                B += fk[(size_t)j * n + i2];
                run += B;
            }
            B = T(0);
            run = T(0);
            for (int j = nv - 1; j >= 0; --j) {
                const T a = fk[(size_t)j * n + i];
                acc += a * run;
                B += fk[(size_t)j * n + i2];
                run += B;
            }
            nadd(tn, (double)acc);
            nadd(td, rho[in.xoff + i] * rho[in.xoff + i2]);
        }
        const Comp zn = block_reduce(tn);
        const Comp zd = block_reduce(td);
        if (threadIdx.x == 0) {
            num[b] = nval(zn) * in.dv * in.dv * in.dv / n;
            den[b] = nval(zd) / n;
        }
    }
}

int obs_grid(long long blocks, int sm_count) {
    return (int)std::max(1ll, std::min(blocks, (long long)sm_count * 16));
}

}  // namespace

// P: 2 (total_x + n_inst) doubles of scratch.
cudaError_t launch_coarse1d(const double* rho, const Inst1D* inst, int n_inst, long long total_x,
                            const int* widths, int nw, double* P, double* out, int sm_count,
                            cudaStream_t s) {
    double* Pl = P + total_x + n_inst;
    k_prefix1d<<<obs_grid(n_inst, sm_count), kObsThreads, 0, s>>>(rho, inst, n_inst, P, Pl);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_coarse1d<<<obs_grid((long long)n_inst * nw, sm_count), kObsThreads, 0, s>>>(
        P, Pl, inst, n_inst, widths, nw, out);
    return cudaGetLastError();
}

// S: 2 (ny + 1)(nx + 1) doubles of scratch.
cudaError_t launch_coarse2d(const double* rho, int nx, int ny, double dx, const int* widths,
                            int nw, double* S, double* out, int sm_count, cudaStream_t s) {
    double* Sl = S + (size_t)(ny + 1) * (nx + 1);
    k_sat_rows<<<(ny + 1 + 127) / 128, 128, 0, s>>>(rho, nx, ny, S, Sl);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sat_cols<<<(nx + 1 + 127) / 128, 128, 0, s>>>(nx, ny, S, Sl);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_coarse2d<<<obs_grid(nw, sm_count), kObsThreads, 0, s>>>(S, Sl, nx, ny, dx, widths, nw,
                                                             out);
    return cudaGetLastError();
}

cudaError_t launch_s1_1d(int dtype, const void* f, const Inst1D* inst, int n_inst, int nv,
                         const double* rho, const int* seps, int ns, double* num, double* den,
                         int sm_count, cudaStream_t s) {
    const int grid = obs_grid((long long)n_inst * ns, sm_count);
    if (dtype == LAT_F32)
        k_s1_1d<float><<<grid, kObsThreads, 0, s>>>(static_cast<const float*>(f), inst, n_inst,
                                                    nv, rho, seps, ns, num, den);
    else if (dtype == LAT_F64)
        k_s1_1d<double><<<grid, kObsThreads, 0, s>>>(static_cast<const double*>(f), inst,
                                                     n_inst, nv, rho, seps, ns, num, den);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace lat

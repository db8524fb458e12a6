// Flux-limited drag sub-step on the 2D lattice (Sec. 2 flux limiter, Sec. 4: the scheme of the
// paper's 2D runs): Koren's limiter on the split fluxes P = (c a)^+ q and M = (c a)^- q of both
// velocity axes, unsplit, integrated by Heun's method, then the five-point diffusion.
//
// Three passes over the state, one thread per phase cell (x fastest, so that every stencil load
// is coalesced along x):
//   1. y1 = q - dFx(q) - dFy(q),  q = f* gathered from the input buffer (streaming)  -> output buffer
//   2. h = (q + y1 - dFx(y1) - dFy(y1)) / 2                                          -> scratch
//   3. out = h + (Dx_{+} - Dx_{-}) + (Dy_{+} - Dy_{-}),  D = r (h_next - h)           -> output buffer
// Each flux through face i + 1/2 needs the cells i - 1 .. i + 2 of its axis (cells beyond the
// walls count as empty; the wall fluxes are zero), so a cell reads 9 values per stage.  The
// passes trade the fused kernels' single read and write for simplicity: about three reads and
// three writes of the state per step.
#include "lat_internal.h"
#include "step2d_dev.h"

namespace lat {
namespace {

using namespace k2d;

constexpr int kLimThreads = 256;

// psi(theta) dp with psi(theta) = max(0, min(1, 1/3 + theta/6, mu theta)), theta = dm / dp,
// written without the division (zero when dp = 0)
template <typename T>
__device__ __forceinline__ T lim_inc2(T dp, T dm, T mu) {
    using O = Ops<T>;
    const T s = copysign(T(1), dp);
    const T b = O::mul(s, O::fma(dm, T(1.0 / 6.0), O::mul(dp, T(1.0 / 3.0))));
    const T c = O::mul(s, O::mul(mu, dm));
    return O::mul(s, fmax(T(0), fmin(fabs(dp), fmin(b, c))));
}

// Flux through face i + 1/2 of one axis from the split fluxes of cells i - 1 .. i + 2
// (P[k], M[k] for k = 0..3 standing for cells i - 1 + k).
template <typename T>
__device__ __forceinline__ T face_flux(const T (&P)[4], const T (&M)[4], T mu) {
    using O = Ops<T>;
    const T pos = O::add(P[1], lim_inc2<T>(O::sub(P[2], P[1]), O::sub(P[1], P[0]), mu));
    const T neg = O::add(M[2], lim_inc2<T>(O::sub(M[1], M[2]), O::sub(M[2], M[3]), mu));
    return O::add(pos, neg);
}

// Limited flux difference F_{j+1/2} - F_{j-1/2} along one axis at index j, given the values of
// cells j - 2 .. j + 2 (v[k] for cell j - 2 + k, zero beyond the walls) and c a at those cells.
template <typename T>
__device__ __forceinline__ T flux_diff(const T (&v)[5], const T (&ca)[5], int j, int nv, T mu) {
    using O = Ops<T>;
    T P[5], M[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        P[k] = O::mul(fmax(ca[k], T(0)), v[k]);
        M[k] = O::mul(fmin(ca[k], T(0)), v[k]);
    }
    const T Pl[4] = {P[0], P[1], P[2], P[3]}, Ml[4] = {M[0], M[1], M[2], M[3]};
    const T Pr[4] = {P[1], P[2], P[3], P[4]}, Mr[4] = {M[1], M[2], M[3], M[4]};
    const T Fl = j > 0 ? face_flux<T>(Pl, Ml, mu) : T(0);        // face j - 1/2
    const T Fr = j < nv - 1 ? face_flux<T>(Pr, Mr, mu) : T(0);   // face j + 1/2
    return O::sub(Fr, Fl);
}

struct Lim2DArgs {
    void* f[2];        // state buffers: step s reads f[s & 1] (f before streaming) and writes
                       // f[(s + 1) & 1] (stage 1's result first, then the step's result)
    void* scr;         // scratch: Heun's average before the diffusion
    const void* u;     // [2][ny][nx] or null
    DevState* st;
    int nx, ny, nv;
    double g, r, inv_dv, mu;
};

// Periodic wrap of v with -n <= v < 2n (N_x, N_y > J, checked by lat_set_scheme).
__device__ __forceinline__ int wrap1(int v, int n) {
    v += v < 0 ? n : 0;
    return v >= n ? v - n : v;
}

// f*(jx, jy, x, y) from the input buffer (streaming: j moves mass by j cells), or y1 values from
// a post-streaming buffer; zero outside the velocity box.  32-bit indices (N_v^2 N_x N_y < 2^32).
template <typename T, bool STREAMED>
__device__ __forceinline__ T qval(const T* q, int jx, int jy, int x, int y, int nx, int ny,
                                  int nv) {
    if (jx < 0 || jx >= nv || jy < 0 || jy >= nv) return T(0);
    const unsigned ncell = (unsigned)nx * (unsigned)ny;
    if (STREAMED) {
        const int J = (nv - 1) / 2;
        return q[(unsigned)(jy * nv + jx) * ncell + (unsigned)wrap1(y - (jy - J), ny) * nx +
                 (unsigned)wrap1(x - (jx - J), nx)];
    }
    return q[(unsigned)(jy * nv + jx) * ncell + (unsigned)y * nx + x];
}

// c a_j = g (w - j) along one axis at velocity index j (offset J), for the five stencil cells
template <typename T>
__device__ __forceinline__ void speeds(T g, T w, int j, int J, T (&ca)[5]) {
#pragma unroll
    for (int k = 0; k < 5; ++k) ca[k] = Ops<T>::mul(g, Ops<T>::sub(w, T(j - 2 + k - J)));
}

// Stage 1 (STAGE = 1): y1 = q - dFx - dFy with q = f* -> fout.  Stage 2: h = (q + y1 - dFx(y1) -
// dFy(y1)) / 2 with y1 from fout -> scr.
template <typename T, int STAGE>
__global__ void __launch_bounds__(kLimThreads) k_lim2d_stage(const Lim2DArgs a, int kstep) {
    using O = Ops<T>;
    const int nx = a.nx, ny = a.ny, nv = a.nv, J = (nv - 1) / 2;
    const long long ncell = (long long)nx * ny;
    const long long n = ncell * nv * nv;
    const T g = T(a.g), mu = T(a.mu);
    const int par = (int)((a.st->step + kstep) & 1);
    const T* fin = static_cast<const T*>(a.f[par]);
    const T* y1 = static_cast<const T*>(a.f[par ^ 1]);
    T* dst = STAGE == 1 ? static_cast<T*>(a.f[par ^ 1]) : static_cast<T*>(a.scr);
    const T cflf = O::mul(g, O::add(T(1), mu));
    const T* ux = static_cast<const T*>(a.u);
    bool cfl = false;
    // grid.x = velocity plane, grid.y over the plane's cells: consecutive blocks take the same
    // cells in all planes, so that the stencil's other planes are still in L2.  N_v^2 N_x N_y
    // < 2^32 (checked by lat_set_scheme): 32-bit index arithmetic
    (void)n;
    const int p = blockIdx.x;
    const int jy = p / nv, jx = p - jy * nv;
    for (unsigned cc = blockIdx.y * blockDim.x + threadIdx.x; cc < (unsigned)ncell;
         cc += gridDim.y * blockDim.x) {
        const unsigned i = (unsigned)p * (unsigned)ncell + cc;
        const int y = (int)(cc / (unsigned)nx), x = (int)(cc - (unsigned)y * (unsigned)nx);
        T wx = T(0), wy = T(0);
        if (ux) {
            wx = O::mul(ux[cc], T(a.inv_dv));
            wy = O::mul(ux[ncell + cc], T(a.inv_dv));
        }
        if (STAGE == 1 && cflf * (T(2 * J) + fabs(wx) + fabs(wy)) > T(1)) cfl = true;
        T cax[5], cay[5], vx[5], vy[5];
        speeds<T>(g, wx, jx, J, cax);
        speeds<T>(g, wy, jy, J, cay);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            if (STAGE == 1) {
                vx[k] = qval<T, true>(fin, jx - 2 + k, jy, x, y, nx, ny, nv);
                vy[k] = qval<T, true>(fin, jx, jy - 2 + k, x, y, nx, ny, nv);
            } else {
                vx[k] = qval<T, false>(y1, jx - 2 + k, jy, x, y, nx, ny, nv);
                vy[k] = qval<T, false>(y1, jx, jy - 2 + k, x, y, nx, ny, nv);
            }
        }
        const T dfx = flux_diff<T>(vx, cax, jx, nv, mu);
        const T dfy = flux_diff<T>(vy, cay, jy, nv, mu);
        const T c = vx[2];  // the cell itself
        const T stage = O::sub(O::sub(c, dfx), dfy);
        if (STAGE == 1) {
            dst[i] = stage;
        } else {
            const T q0 = qval<T, true>(fin, jx, jy, x, y, nx, ny, nv);
            dst[i] = O::mul(T(0.5), O::add(q0, stage));
        }
    }
    if (cfl) atomicOr(&a.st->status, ST_CFL);
}

// out = h + (Dx_{+} - Dx_{-}) + (Dy_{+} - Dy_{-}), D = r (h_next - h), zero at the walls
template <typename T>
__global__ void __launch_bounds__(kLimThreads) k_lim2d_diffuse(const Lim2DArgs a, int kstep) {
    using O = Ops<T>;
    const int nx = a.nx, ny = a.ny, nv = a.nv;
    const long long ncell = (long long)nx * ny;
    const long long n = ncell * nv * nv;
    const T r = T(a.r);
    const int par = (int)((a.st->step + kstep) & 1);
    const T* h = static_cast<const T*>(a.scr);
    T* out = static_cast<T*>(a.f[par ^ 1]);
    (void)n;
    const int p = blockIdx.x;
    const int jy = p / nv, jx = p - jy * nv;
    for (unsigned cc = blockIdx.y * blockDim.x + threadIdx.x; cc < (unsigned)ncell;
         cc += gridDim.y * blockDim.x) {
        const unsigned i = (unsigned)p * (unsigned)ncell + cc;
        const T hc = h[i];
        const T Dxr = jx < nv - 1 ? O::mul(r, O::sub(h[i + ncell], hc)) : T(0);
        const T Dxl = jx > 0 ? O::mul(r, O::sub(hc, h[i - ncell])) : T(0);
        const T Dyr = jy < nv - 1 ? O::mul(r, O::sub(h[i + ncell * nv], hc)) : T(0);
        const T Dyl = jy > 0 ? O::mul(r, O::sub(hc, h[i - ncell * nv])) : T(0);
        out[i] = O::add(O::add(hc, O::sub(Dxr, Dxl)), O::sub(Dyr, Dyl));
    }
}

template <typename T>
cudaError_t launch_lim2d_t(const Lim2DArgs& a, int k, int sm_count, cudaStream_t s) {
    const long long ncell = (long long)a.nx * a.ny;
    (void)sm_count;
    const dim3 grid((unsigned)(a.nv * a.nv),
                    (unsigned)std::min((ncell + kLimThreads - 1) / kLimThreads, 65535ll));
    k_lim2d_stage<T, 1><<<grid, kLimThreads, 0, s>>>(a, k);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_lim2d_stage<T, 2><<<grid, kLimThreads, 0, s>>>(a, k);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_lim2d_diffuse<T><<<grid, kLimThreads, 0, s>>>(a, k);
    return cudaGetLastError();
}

}  // namespace

// One limited 2D step k of an enqueued batch: input buffer f[par], output f[par ^ 1] (par from
// the device step counter plus k), scratch of the state's size.
cudaError_t launch_step2d_limited(int dtype, const Step2DArgs& s2, int nv, double mu, void* scratch,
                                  int k, int sm_count, cudaStream_t s) {
    Lim2DArgs a;
    a.f[0] = s2.f[0];
    a.f[1] = s2.f[1];
    a.scr = scratch;
    a.u = s2.u;
    a.st = s2.st;
    a.nx = s2.nx;
    a.ny = s2.ny;
    a.nv = nv;
    a.g = s2.g;
    a.r = s2.r;
    a.inv_dv = s2.inv_dv;
    a.mu = mu;
    if (dtype == LAT_F32) return launch_lim2d_t<float>(a, k, sm_count, s);
    if (dtype == LAT_F64) return launch_lim2d_t<double>(a, k, sm_count, s);
    return cudaErrorInvalidValue;
}

}  // namespace lat

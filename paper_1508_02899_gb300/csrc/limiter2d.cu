// Flux-limited drag sub-step on the 2D lattice (Sec. 2 flux limiter, Sec. 4: the scheme of the
// paper's 2D runs): Koren's limiter on the split fluxes P = (c a)^+ q and M = (c a)^- q of both
// velocity axes, unsplit, integrated by Heun's method, then the five-point diffusion.
//
// Three passes over the state (x fastest within every thread block, so that every stencil load
// is coalesced along x):
//   1. y1 = q - dFx(q) - dFy(q),  q = f* gathered from the input buffer (streaming)  -> output buffer
//   2. h = (q + y1 - dFx(y1) - dFy(y1)) / 2                                          -> scratch
//   3. out = h + (Dx_{+} - Dx_{-}) + (Dy_{+} - Dy_{-}),  D = r (h_next - h)           -> output buffer
// Each flux through face i + 1/2 needs the cells i - 1 .. i + 2 of its axis (cells beyond the
// walls count as empty; the wall fluxes are zero).  The stages sweep pairs of velocity rows, so
// a pair of cells reads 6 values of its column per stage.  The passes trade the fused kernels'
// single read and write for simplicity: about three reads and three writes of the state per
// step.
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

// Stage 1 (STAGE = 1): y1 = q - dFx - dFy with q = f* -> f[par ^ 1].  Stage 2: h = (q + y1 -
// dFx(y1) - dFy(y1)) / 2 with y1 from f[par ^ 1] -> scratch.
// A thread takes one spatial cell and the velocity rows jy0 = 2 blockIdx.x and jy0 + 1 and
// sweeps jx = 0 .. N_v - 1: the vx split fluxes and faces of each row slide along it (each face
// once), and the three vy faces jy0 - 1/2, jy0 + 1/2, jy0 + 3/2 of the column come from the
// values of rows jy0 - 2 .. jy0 + 3 (the middle face serves both rows).  grid.x = row pairs,
// grid.y over the spatial cells (consecutive blocks take the same cells in every row pair, so
// the other rows are still in L2).  Every face is formed by the same operations as in a sweep
// of one row, so the result does not depend on the pairing.
// NVT > 0: N_v known at compile time (the velocity loop unrolled); 0: any N_v.
template <typename T, int STAGE, int NVT = 0>
__global__ void __launch_bounds__(kLimThreads) k_lim2d_stage(const Lim2DArgs a, int kstep) {
    using O = Ops<T>;
    const int nx = a.nx, ny = a.ny, nv = NVT > 0 ? NVT : a.nv, J = (nv - 1) / 2;
    const unsigned ncell = (unsigned)nx * (unsigned)ny;
    const T g = T(a.g), mu = T(a.mu);
    const int par = (int)((a.st->step + kstep) & 1);
    const T* fin = static_cast<const T*>(a.f[par]);
    const T* y1 = static_cast<const T*>(a.f[par ^ 1]);
    T* dst = STAGE == 1 ? static_cast<T*>(a.f[par ^ 1]) : static_cast<T*>(a.scr);
    const T* src = STAGE == 1 ? fin : y1;  // the values the fluxes act on
    const T cflf = O::mul(g, O::add(T(1), mu));
    const T* ux = static_cast<const T*>(a.u);
    const int jy0 = 2 * (int)blockIdx.x, jy1 = jy0 + 1;
    const bool two = jy1 < nv;  // the last pair of an odd N_v holds one row
    bool cfl = false;
    for (unsigned cc = blockIdx.y * blockDim.x + threadIdx.x; cc < ncell;
         cc += gridDim.y * blockDim.x) {
        const int y = (int)(cc / (unsigned)nx), x = (int)(cc - (unsigned)y * (unsigned)nx);
        T wx = T(0), wy = T(0);
        if (ux) {
            wx = O::mul(ux[cc], T(a.inv_dv));
            wy = O::mul(ux[ncell + cc], T(a.inv_dv));
        }
        if (STAGE == 1 && jy0 == 0 && cflf * (T(2 * J) + fabs(wx) + fabs(wy)) > T(1)) cfl = true;
        // rows jy0 - 2 .. jy0 + 3: plane-row offsets (rowin false outside the box) and c a_y
        unsigned rowoff[6];
        bool rowin[6];
        T cay[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int jr = jy0 - 2 + k;
            rowin[k] = jr >= 0 && jr < nv;
            const int yr = STAGE == 1 ? wrap1(y - (jr - J), ny) : y;
            rowoff[k] = rowin[k] ? (unsigned)(jr * nv) * ncell + (unsigned)yr * nx : 0u;
            cay[k] = O::mul(g, O::sub(wy, T(jr - J)));
        }
        // value of (jx', row k) for the stencil (0 outside the box)
        auto val = [&](int jxp, int k) -> T {
            if (!rowin[k] || jxp < 0 || jxp >= nv) return T(0);
            const int xc = STAGE == 1 ? wrap1(x - (jxp - J), nx) : x;
            return src[rowoff[k] + (unsigned)jxp * ncell + (unsigned)xc];
        };
        auto cax = [&](int jxp) { return O::mul(g, O::sub(wx, T(jxp - J))); };
        // stage 2 averages with f* of the cell, read streamed from the input buffer
        const unsigned rowq0 =
            (unsigned)(jy0 * nv) * ncell + (unsigned)wrap1(y - (jy0 - J), ny) * (unsigned)nx;
        const unsigned rowq1 =
            (unsigned)(jy1 * nv) * ncell + (unsigned)wrap1(y - (jy1 - J), ny) * (unsigned)nx;
        // x windows of rows jy0 (A, stencil row 2) and jy1 (B, row 3): values and split fluxes
        // of cells jx - 1 .. jx + 2 (index 0 .. 3)
        T VA[4], PA[4], MA[4], VB[4], PB[4], MB[4];
        VA[0] = PA[0] = MA[0] = VB[0] = PB[0] = MB[0] = T(0);  // cell -1, beyond the wall
#pragma unroll
        for (int k = 1; k < 4; ++k) {
            const T ca = cax(k - 1);
            VA[k] = val(k - 1, 2);
            PA[k] = O::mul(fmax(ca, T(0)), VA[k]);
            MA[k] = O::mul(fmin(ca, T(0)), VA[k]);
            VB[k] = val(k - 1, 3);
            PB[k] = O::mul(fmax(ca, T(0)), VB[k]);
            MB[k] = O::mul(fmin(ca, T(0)), VB[k]);
        }
        T FxlA = T(0), FxlB = T(0);  // faces jx - 1/2 (the wall face for jx = 0)
#pragma unroll(NVT > 0 ? NVT : 1)
        for (int jx = 0; jx < nv; ++jx) {
            // faces jx + 1/2 from cells jx - 1 .. jx + 2
            T FxrA = T(0), FxrB = T(0);
            if (jx < nv - 1) {
                const T P4[4] = {PA[0], PA[1], PA[2], PA[3]}, M4[4] = {MA[0], MA[1], MA[2], MA[3]};
                FxrA = face_flux<T>(P4, M4, mu);
                if (two) {
                    const T Q4[4] = {PB[0], PB[1], PB[2], PB[3]};
                    const T N4[4] = {MB[0], MB[1], MB[2], MB[3]};
                    FxrB = face_flux<T>(Q4, N4, mu);
                }
            }
            // the column jx: rows jy0 - 2 .. jy0 + 3 and their split fluxes
            T P[6], M[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const T v = k == 2 ? VA[1] : (k == 3 ? VB[1] : val(jx, k));
                P[k] = O::mul(fmax(cay[k], T(0)), v);
                M[k] = O::mul(fmin(cay[k], T(0)), v);
            }
            const T Pm[4] = {P[0], P[1], P[2], P[3]}, Mm[4] = {M[0], M[1], M[2], M[3]};
            const T Pc[4] = {P[1], P[2], P[3], P[4]}, Mc[4] = {M[1], M[2], M[3], M[4]};
            const T Fm = jy0 > 0 ? face_flux<T>(Pm, Mm, mu) : T(0);       // face jy0 - 1/2
            const T F0 = jy0 < nv - 1 ? face_flux<T>(Pc, Mc, mu) : T(0);  // face jy0 + 1/2
            const T stageA = O::sub(O::sub(VA[1], O::sub(FxrA, FxlA)), O::sub(F0, Fm));
            const unsigned oA = (unsigned)(jy0 * nv + jx) * ncell + cc;
            if (STAGE == 1) {
                dst[oA] = stageA;
            } else {
                const T q0 = fin[rowq0 + (unsigned)jx * ncell + (unsigned)wrap1(x - (jx - J), nx)];
                dst[oA] = O::mul(T(0.5), O::add(q0, stageA));
            }
            if (two) {
                const T Pp[4] = {P[2], P[3], P[4], P[5]}, Mp[4] = {M[2], M[3], M[4], M[5]};
                const T Fp = jy1 < nv - 1 ? face_flux<T>(Pp, Mp, mu) : T(0);  // face jy1 + 1/2
                const T stageB = O::sub(O::sub(VB[1], O::sub(FxrB, FxlB)), O::sub(Fp, F0));
                const unsigned oB = oA + (unsigned)nv * ncell;
                if (STAGE == 1) {
                    dst[oB] = stageB;
                } else {
                    const T q1 =
                        fin[rowq1 + (unsigned)jx * ncell + (unsigned)wrap1(x - (jx - J), nx)];
                    dst[oB] = O::mul(T(0.5), O::add(q1, stageB));
                }
            }
            // slide the windows to cells jx .. jx + 3
            FxlA = FxrA;
            FxlB = FxrB;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                VA[k] = VA[k + 1];
                PA[k] = PA[k + 1];
                MA[k] = MA[k + 1];
                VB[k] = VB[k + 1];
                PB[k] = PB[k + 1];
                MB[k] = MB[k + 1];
            }
            const T ca = cax(jx + 3);
            VA[3] = val(jx + 3, 2);
            PA[3] = O::mul(fmax(ca, T(0)), VA[3]);
            MA[3] = O::mul(fmin(ca, T(0)), VA[3]);
            VB[3] = val(jx + 3, 3);
            PB[3] = O::mul(fmax(ca, T(0)), VB[3]);
            MB[3] = O::mul(fmin(ca, T(0)), VB[3]);
        }
    }
    if (cfl) atomicOr(&a.st->status, ST_CFL);
}

// out = h + (Dx_{+} - Dx_{-}) + (Dy_{+} - Dy_{-}), D = r (h_next - h), zero at the walls.
// A thread takes one spatial cell and the velocity rows jy0 = 2 blockIdx.x and jy0 + 1 and sweeps
// jx: the row values slide along jx (one new load per row and step), the rows jy0 - 1 and
// jy0 + 2 give the vy neighbours, so a pair of cells loads four values.  grid as the stages.
template <typename T, int NVT = 0>
__global__ void __launch_bounds__(kLimThreads) k_lim2d_diffuse(const Lim2DArgs a, int kstep) {
    using O = Ops<T>;
    const int nv = NVT > 0 ? NVT : a.nv;
    const unsigned ncell = (unsigned)a.nx * (unsigned)a.ny;
    const T r = T(a.r);
    const int par = (int)((a.st->step + kstep) & 1);
    const T* h = static_cast<const T*>(a.scr);
    T* out = static_cast<T*>(a.f[par ^ 1]);
    const int jy0 = 2 * (int)blockIdx.x, jy1 = jy0 + 1;
    const bool two = jy1 < nv;
    for (unsigned cc = blockIdx.y * blockDim.x + threadIdx.x; cc < ncell;
         cc += gridDim.y * blockDim.x) {
        const T* r0 = h + (unsigned)(jy0 * nv) * ncell + cc;  // row jy0, column 0
        const T* r1 = r0 + (unsigned)nv * ncell;              // row jy1
        const unsigned ps = ncell;
        // row values at jx - 1, jx, jx + 1 (index 0 .. 2)
        T a0 = T(0), a1 = r0[0], b0 = T(0), b1 = two ? r1[0] : T(0);
#pragma unroll(NVT > 0 ? NVT : 1)
        for (int jx = 0; jx < nv; ++jx) {
            const T a2 = jx < nv - 1 ? r0[(unsigned)(jx + 1) * ps] : T(0);
            const T b2 = (two && jx < nv - 1) ? r1[(unsigned)(jx + 1) * ps] : T(0);
            const T dn = jy0 > 0 ? *(r0 + (unsigned)jx * ps - (unsigned)nv * ps) : T(0);
            const T hc = a1;
            const T Dxr = jx < nv - 1 ? O::mul(r, O::sub(a2, hc)) : T(0);
            const T Dxl = jx > 0 ? O::mul(r, O::sub(hc, a0)) : T(0);
            const T Dyr = jy0 < nv - 1 ? O::mul(r, O::sub(b1, hc)) : T(0);
            const T Dyl = jy0 > 0 ? O::mul(r, O::sub(hc, dn)) : T(0);
            out[(unsigned)(jy0 * nv + jx) * ps + cc] = O::add(O::add(hc, O::sub(Dxr, Dxl)), O::sub(Dyr, Dyl));
            if (two) {
                const T up = jy1 < nv - 1 ? r1[(unsigned)jx * ps + (unsigned)nv * ps] : T(0);
                const T hd = b1;
                const T Exr = jx < nv - 1 ? O::mul(r, O::sub(b2, hd)) : T(0);
                const T Exl = jx > 0 ? O::mul(r, O::sub(hd, b0)) : T(0);
                const T Eyr = jy1 < nv - 1 ? O::mul(r, O::sub(up, hd)) : T(0);
                const T Eyl = O::mul(r, O::sub(hd, hc));
                out[(unsigned)(jy1 * nv + jx) * ps + cc] =
                    O::add(O::add(hd, O::sub(Exr, Exl)), O::sub(Eyr, Eyl));
            }
            a0 = a1;
            a1 = a2;
            b0 = b1;
            b1 = b2;
        }
    }
}

template <typename T, int NVT>
void launch_stages(const Lim2DArgs& a, int k, dim3 grow, cudaStream_t s) {
    k_lim2d_stage<T, 1, NVT><<<grow, kLimThreads, 0, s>>>(a, k);
    k_lim2d_stage<T, 2, NVT><<<grow, kLimThreads, 0, s>>>(a, k);
    k_lim2d_diffuse<T, NVT><<<grow, kLimThreads, 0, s>>>(a, k);
}

template <typename T>
cudaError_t launch_lim2d_t(const Lim2DArgs& a, int k, int sm_count, cudaStream_t s) {
    const long long ncell = (long long)a.nx * a.ny;
    (void)sm_count;
    const unsigned chunks = (unsigned)std::min((ncell + kLimThreads - 1) / kLimThreads, 65535ll);
    const dim3 grow((unsigned)(a.nv + 1) / 2, chunks);
    // FP32 lattices of the common sizes take the unrolled stages
    bool done = false;
    if constexpr (sizeof(T) == 4) {
        done = true;
        if (a.nv == 9) launch_stages<T, 9>(a, k, grow, s);
        else if (a.nv == 17) launch_stages<T, 17>(a, k, grow, s);
        else if (a.nv == 19) launch_stages<T, 19>(a, k, grow, s);
        else if (a.nv == 33) launch_stages<T, 33>(a, k, grow, s);
        else done = false;
    }
    if (!done) launch_stages<T, 0>(a, k, grow, s);
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

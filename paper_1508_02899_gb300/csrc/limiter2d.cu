// Flux-limited drag sub-step on the 2D lattice (Sec. 2 flux limiter, Sec. 4: the scheme of the
// paper's 2D runs): Koren's limiter on the split fluxes P = (c a)^+ q and M = (c a)^- q of both
// velocity axes, unsplit, integrated by Heun's method, then the five-point diffusion.
//
// The step, with q = f* (the streamed values):
//   1. y1 = q - dFx(q) - dFy(q)
//   2. h = (q + y1 - dFx(y1) - dFy(y1)) / 2
//   3. out = h + (Dx_{+} - Dx_{-}) + (Dy_{+} - Dy_{-}),  D = r (h_next - h)
// Each flux through face i + 1/2 needs the cells i - 1 .. i + 2 of its axis (cells beyond the
// walls count as empty; the wall fluxes are zero).  Three launch forms give the same values:
//   - three passes over the state, one per line above (stage 1 gathers q from the input buffer
//     and writes y1 to the output buffer, stage 2 writes h to a scratch state, the diffusion
//     writes the output): about three reads and three writes of the state per step; any N_v.
//   - k_lim2d_fused: one kernel per step with a tile of cells and all its velocities staged in
//     shared memory, one read and one write of the state (FP32 and FP64).
//   - k_lim2d_packed: the same on cell pairs in FP32 register pairs (FP32, the default).
// Steps 1-3 act on each cell's velocity plane only (streaming is the gather of q), which is what
// lets one block finish a tile of cells without touching its neighbours.
#include "f32x2.h"
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

// ---- fused form: one read and one write of the state per step ---------------------------------
//
// A block takes a tile of TC consecutive cells of one grid row and stages their streamed values
// f* for all N_v^2 velocities in shared memory (plane A).  Stage 1 writes y1 to plane B, stage 2
// writes h over f* in plane A, and the diffusion reads h and stores the step's result.  Thread
// (c, jx) owns cell c of the tile and the velocity column jx, and sweeps the rows jy: the vy
// faces slide along its column (each formed once), and the vx faces jx -/+ 1/2 of a row come
// from the columns jx - 2 .. jx + 2 (each formed by both columns it separates).  The planes
// carry two zero columns on either side, so the stencil loads need no bounds tests; the wall
// faces are still set to zero explicitly.  While the diffusion runs, the next tile's f* is
// copied (cp.async) into plane B, and the planes swap roles.
//
// Zero parts.  The limited flux of a face is the sum of a part built from P = (c a)^+ q and a
// part built from M = (c a)^- q of its four cells.  When c a >= 0 on all four cells, every M is
// zero and so is the M part; likewise the P part when c a <= 0 on all four.  Such parts are not
// formed.  c a_j = g (w - (j - J)) has the sign of w - (j - J) (g > 0, and the rounded
// difference keeps the sign of the exact one), so the test compares cell indices with
// floor(w) + J and ceil(w) + J, taken over the 32 lanes of a warp so that the branch is uniform.
// Up to the sign of a zero flux, every face has the bits of face_flux, and the step those of
// the three-pass form.
template <typename T, int NV, int TC>
struct LimFused {
    static constexpr int J = (NV - 1) / 2;
    static constexpr int CPW = 32 / TC;              // velocity columns per warp
    static constexpr int NW = (NV + CPW - 1) / CPW;  // warps per block
    static constexpr int kThreads = 32 * NW;
    static constexpr int PW = NV + 4;                // plane row: columns -2 .. NV + 1
    static constexpr int kRow = PW * TC;             // elements of one plane row
    static constexpr int kPlane = NV * kRow;
    static constexpr size_t kSmem = 2 * (size_t)kPlane * sizeof(T);
    static_assert(32 % TC == 0 && kThreads <= 1024, "tile shape");
};

enum { kBothParts = 0, kPosPart = 1, kNegPart = 2 };

// Lane bounds of the sign test: c a_j >= 0 for every j <= kp, c a_j <= 0 for every j >= kn.
template <typename T>
__device__ __forceinline__ void sign_bounds(T w, int J, int& kp, int& kn) {
    if (fabs(w) < T(1 << 20)) {  // false for NaN
        kp = (int)floor(w) + J;
        kn = (int)ceil(w) + J;
    } else {
        kp = -(1 << 28);
        kn = 1 << 28;
    }
}

// Parts of the face whose cells are a .. a + 3.
__device__ __forceinline__ int face_kind(int a, int kp, int kn) {
    return a + 3 <= kp ? kPosPart : (a >= kn ? kNegPart : kBothParts);
}

// The kind of every lane of the warp if they agree, both parts otherwise.
__device__ __forceinline__ int uniform_kind(int kind) {
    if (__all_sync(0xffffffffu, kind == kPosPart)) return kPosPart;
    if (__all_sync(0xffffffffu, kind == kNegPart)) return kNegPart;
    return kBothParts;
}

// P part: P1 + psi dP;  M part: M2 + psi dM (the two halves of face_flux)
template <typename T>
__device__ __forceinline__ T pos_part(T P0, T P1, T P2, T mu) {
    using O = Ops<T>;
    return O::add(P1, lim_inc2<T>(O::sub(P2, P1), O::sub(P1, P0), mu));
}
template <typename T>
__device__ __forceinline__ T neg_part(T M1, T M2, T M3, T mu) {
    using O = Ops<T>;
    return O::add(M2, lim_inc2<T>(O::sub(M1, M2), O::sub(M2, M3), mu));
}

// Face flux from the split fluxes of its four cells, forming only the parts `kind` names.
template <typename T>
__device__ __forceinline__ T face_parts(int kind, T P0, T P1, T P2, T M1, T M2, T M3, T mu) {
    if (kind == kPosPart) return pos_part<T>(P0, P1, P2, mu);
    if (kind == kNegPart) return neg_part<T>(M1, M2, M3, mu);
    return Ops<T>::add(pos_part<T>(P0, P1, P2, mu), neg_part<T>(M1, M2, M3, mu));
}

// The same from the cells' values x0..x3 and coefficients (c a)^+ (cp) and (c a)^- (cm): only
// the products a formed part uses are taken.
template <typename T>
__device__ __forceinline__ T face_vals(int kind, T x0, T x1, T x2, T x3, T cp0, T cp1, T cp2,
                                       T cm1, T cm2, T cm3, T mu) {
    using O = Ops<T>;
    if (kind == kPosPart) return pos_part<T>(O::mul(cp0, x0), O::mul(cp1, x1), O::mul(cp2, x2), mu);
    if (kind == kNegPart) return neg_part<T>(O::mul(cm1, x1), O::mul(cm2, x2), O::mul(cm3, x3), mu);
    return O::add(pos_part<T>(O::mul(cp0, x0), O::mul(cp1, x1), O::mul(cp2, x2), mu),
                  neg_part<T>(O::mul(cm1, x1), O::mul(cm2, x2), O::mul(cm3, x3), mu));
}

__device__ __forceinline__ void cp_async_elem(float* dst, const float* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_elem(double* dst, const double* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// f* of cell x of grid row y, column jx, all rows jy, into a plane:
// f*(x, y; jx, jy) = f(x - (jx - J), y - (jy - J); jx, jy) (periodic; N_x, N_y > J).
template <typename T, int NV, int TC>
__device__ __forceinline__ void lim_fused_load(const T* fin, T* plane, int nx, int ny, int y,
                                               int x, int jx, int c) {
    using L = LimFused<T, NV, TC>;
    T* d = plane + (jx + 2) * TC + c;
    if (x >= nx) {  // beyond a ragged edge: zeros
#pragma unroll
        for (int jy = 0; jy < NV; ++jy) d[jy * L::kRow] = T(0);
        return;
    }
    const size_t ncell = (size_t)nx * (size_t)ny;
    const T* src = fin + (size_t)jx * ncell + (size_t)wrap1(x - (jx - L::J), nx);
    int yr = wrap1(y + L::J, ny);  // the source row of jy = 0
#pragma unroll
    for (int jy = 0; jy < NV; ++jy) {
        cp_async_elem(d + jy * L::kRow, src + (size_t)yr * nx);
        src += (size_t)NV * ncell;
        yr = yr == 0 ? ny - 1 : yr - 1;
    }
}

// One Heun stage on column jx of the tile: STAGE 1 reads q from `src` and writes
// y1 = q - dFx(q) - dFy(q) to `dst`; STAGE 2 reads y1 from `src` and replaces q in `dst` by
// h = (q + y1 - dFx(y1) - dFy(y1)) / 2.  cxp/cxm: (c a_x)^+/- of the columns jx - 2 .. jx + 2;
// kl, kr: parts of the faces jx - 1/2 and jx + 1/2; kyp, kyn: the warp's vy sign bounds.
template <typename T, int NV, int TC, int STAGE, int UNR>
__device__ __forceinline__ void lim_fused_stage(const T* src, T* dst, int jx, int c, bool store,
                                                T g, T wy, T mu, const T (&cxp)[5],
                                                const T (&cxm)[5], int kl, int kr, int kyp,
                                                int kyn) {
    using L = LimFused<T, NV, TC>;
    using O = Ops<T>;
    constexpr int J = L::J, R = L::kRow;
    const T* col = src + (jx + 2) * TC + c;
    T* out = dst + (jx + 2) * TC + c;
    // values and split vy fluxes of the rows jy - 1 .. jy + 2 (zero outside the lattice)
    T v[4], P[4], M[4];
    v[0] = P[0] = M[0] = T(0);
#pragma unroll
    for (int k = 1; k < 4; ++k) {
        const int jr = k - 1;
        v[k] = jr < NV ? col[jr * R] : T(0);
        const T ca = O::mul(g, O::sub(wy, T(jr - J)));
        P[k] = O::mul(fmax(ca, T(0)), v[k]);
        M[k] = O::mul(fmin(ca, T(0)), v[k]);
    }
    T Fyl = T(0);  // the wall face jy = -1/2
#pragma unroll(UNR)
    for (int jy = 0; jy < NV; ++jy) {
        // face jy + 1/2 from the rows jy - 1 .. jy + 2 (the wall face NV - 1/2 is zero)
        T Fyr = T(0);
        if (jy < NV - 1)
            Fyr = face_parts<T>(face_kind(jy - 1, kyp, kyn), P[0], P[1], P[2], M[1], M[2], M[3],
                                mu);
        // faces jx - 1/2 (cells jx - 2 .. jx + 1) and jx + 1/2 (cells jx - 1 .. jx + 2)
        const T* rp = col + jy * R;
        const T xm2 = rp[-2 * TC], xm1 = rp[-TC], x0 = v[1], xp1 = rp[TC], xp2 = rp[2 * TC];
        T Fxl = face_vals<T>(kl, xm2, xm1, x0, xp1, cxp[0], cxp[1], cxp[2], cxm[1], cxm[2],
                             cxm[3], mu);
        T Fxr = face_vals<T>(kr, xm1, x0, xp1, xp2, cxp[1], cxp[2], cxp[3], cxm[2], cxm[3],
                             cxm[4], mu);
        if (jx == 0) Fxl = T(0);
        if (jx == NV - 1) Fxr = T(0);
        const T sv = O::sub(O::sub(x0, O::sub(Fxr, Fxl)), O::sub(Fyr, Fyl));
        if (store) {
            if (STAGE == 1) out[jy * R] = sv;
            else out[jy * R] = O::mul(T(0.5), O::add(out[jy * R], sv));
        }
        Fyl = Fyr;
        // slide the column window to the rows jy .. jy + 3
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            v[k] = v[k + 1];
            P[k] = P[k + 1];
            M[k] = M[k + 1];
        }
        const int jn = jy + 3;
        const T vn = col[(jn < NV ? jn : NV - 1) * R];
        v[3] = jn < NV ? vn : T(0);
        const T ca = O::mul(g, O::sub(wy, T(jn - J)));
        P[3] = O::mul(fmax(ca, T(0)), v[3]);
        M[3] = O::mul(fmin(ca, T(0)), v[3]);
    }
}

// Diffusion of column jx: out = h + (Dx+ - Dx-) + (Dy+ - Dy-), D = r (h_next - h), zero at the
// walls (the operations of k_lim2d_diffuse); `gout` points at row jy = 0 of the column's cell.
template <typename T, int NV, int TC, int UNR>
__device__ __forceinline__ void lim_fused_diffuse(const T* plane, T* gout, size_t ncell, int jx,
                                                  int c, bool store, T r) {
    using L = LimFused<T, NV, TC>;
    using O = Ops<T>;
    constexpr int R = L::kRow;
    const T* col = plane + (jx + 2) * TC + c;
    T hm = T(0), h0 = col[0];
#pragma unroll(UNR)
    for (int jy = 0; jy < NV; ++jy) {
        const T hnext = col[(jy < NV - 1 ? jy + 1 : jy) * R];
        const T hp = jy < NV - 1 ? hnext : T(0);
        const T hl = col[jy * R - TC], hr = col[jy * R + TC];
        const T Dxr = jx < NV - 1 ? O::mul(r, O::sub(hr, h0)) : T(0);
        const T Dxl = jx > 0 ? O::mul(r, O::sub(h0, hl)) : T(0);
        const T Dyr = jy < NV - 1 ? O::mul(r, O::sub(hp, h0)) : T(0);
        const T Dyl = jy > 0 ? O::mul(r, O::sub(h0, hm)) : T(0);
        if (store) gout[(size_t)jy * NV * ncell] = O::add(O::add(h0, O::sub(Dxr, Dxl)), O::sub(Dyr, Dyl));
        hm = h0;
        h0 = hp;
    }
}

template <typename T, int NV, int TC, int MINB, int UNR>
__global__ void __launch_bounds__(LimFused<T, NV, TC>::kThreads, MINB)
    k_lim2d_fused(const Lim2DArgs a, int kstep) {
    using L = LimFused<T, NV, TC>;
    using O = Ops<T>;
    constexpr int J = L::J;
    extern __shared__ __align__(16) unsigned char lim_smem[];
    T* pa = reinterpret_cast<T*>(lim_smem);
    T* pb = pa + L::kPlane;
    const int nx = a.nx, ny = a.ny;
    const size_t ncell = (size_t)nx * (size_t)ny;
    const bool par = ((a.st->step + kstep) & 1) != 0;
    const T* fin = static_cast<const T*>(par ? a.f[1] : a.f[0]);
    T* fout = static_cast<T*>(par ? a.f[0] : a.f[1]);
    const T* u = static_cast<const T*>(a.u);
    const T g = T(a.g), mu = T(a.mu), r = T(a.r), inv_dv = T(a.inv_dv);
    const T cflf = O::mul(g, O::add(T(1), mu));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = lane % TC;
    const int jx_raw = warp * L::CPW + lane / TC;
    const bool active = jx_raw < NV;  // the spare columns of the last warp compute column NV - 1
    const int jx = active ? jx_raw : NV - 1;
    const int ntx = (nx + TC - 1) / TC;
    const long long ntiles = (long long)ntx * ny;
    // the pad columns -2, -1, NV, NV + 1 of both planes stay zero
    for (int i = threadIdx.x; i < 2 * NV * 4 * TC; i += blockDim.x) {
        const int e = i % TC, k = (i / TC) % 4, row = (i / (4 * TC)) % NV, p = i / (4 * TC * NV);
        (p ? pb : pa)[row * L::kRow + (k < 2 ? k : NV + k) * TC + e] = T(0);
    }
    long long t = blockIdx.x;
    if (t < ntiles && active) {
        const int y = (int)(t / ntx);
        lim_fused_load<T, NV, TC>(fin, pa, nx, ny, y, (int)(t - (long long)y * ntx) * TC + c, jx, c);
    }
    bool cfl = false;
    for (; t < ntiles; t += gridDim.x) {
        const int y = (int)(t / ntx);
        const int x = (int)(t - (long long)y * ntx) * TC + c;
        const bool in = x < nx;
        T wx = T(0), wy = T(0);
        if (u && in) {
            wx = O::mul(u[(size_t)y * nx + x], inv_dv);
            wy = O::mul(u[ncell + (size_t)y * nx + x], inv_dv);
        }
        if (jx_raw == 0 && in && cflf * (T(2 * J) + fabs(wx) + fabs(wy)) > T(1)) cfl = true;
        T cxp[5], cxm[5];  // (c a_x)^+/- of the columns jx - 2 .. jx + 2
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const T ca = O::mul(g, O::sub(wx, T(jx - 2 + k - J)));
            cxp[k] = fmax(ca, T(0));
            cxm[k] = fmin(ca, T(0));
        }
        int kxp, kxn, kyp, kyn;
        sign_bounds<T>(wx, J, kxp, kxn);
        sign_bounds<T>(wy, J, kyp, kyn);
        const int kl = uniform_kind(face_kind(jx - 2, kxp, kxn));
        const int kr = uniform_kind(face_kind(jx - 1, kxp, kxn));
        kyp = __reduce_min_sync(0xffffffffu, kyp);
        kyn = __reduce_max_sync(0xffffffffu, kyn);
        cp_async_wait_all();
        __syncthreads();  // f* of the tile in pa; every warp is done with the previous tile
        lim_fused_stage<T, NV, TC, 1, UNR>(pa, pb, jx, c, active, g, wy, mu, cxp, cxm, kl, kr, kyp,
                                           kyn);
        __syncthreads();
        lim_fused_stage<T, NV, TC, 2, UNR>(pb, pa, jx, c, active, g, wy, mu, cxp, cxm, kl, kr, kyp,
                                           kyn);
        __syncthreads();
        const long long tn = t + gridDim.x;
        if (tn < ntiles && active) {
            const int yn = (int)(tn / ntx);
            lim_fused_load<T, NV, TC>(fin, pb, nx, ny, yn, (int)(tn - (long long)yn * ntx) * TC + c,
                                      jx, c);
        }
        T* gout = fout + ((size_t)jx * ny + y) * nx + (in ? x : 0);
        lim_fused_diffuse<T, NV, TC, UNR>(pa, gout, ncell, jx, c, active && in, r);
        T* tmp = pa;
        pa = pb;
        pb = tmp;
    }
    cp_async_wait_all();
    if (cfl) atomicOr(&a.st->status, ST_CFL);
}

template <typename T, int NV, int TC, int MINB, int UNR = 4>
cudaError_t launch_fused_t(const Lim2DArgs& a, int k, int sm_count, cudaStream_t s) {
    using L = LimFused<T, NV, TC>;
    static bool attr = false;
    static int per_sm = 0;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_lim2d_fused<T, NV, TC, MINB, UNR>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)L::kSmem);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lim2d_fused<T, NV, TC, MINB, UNR>,
                                                          L::kThreads, L::kSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const long long ntiles = (long long)((a.nx + TC - 1) / TC) * a.ny;
    const int grid = (int)std::min<long long>(ntiles, (long long)std::max(per_sm, 1) * sm_count);
    k_lim2d_fused<T, NV, TC, MINB, UNR><<<grid, L::kThreads, L::kSmem, s>>>(a, k);
    return cudaGetLastError();
}

// ---- packed FP32 form of the fused kernel ----------------------------------------------------
// As k_lim2d_fused with a thread on two neighbouring cells of the tile (one velocity column):
// their values travel as pairs (8-byte shared-memory accesses) and the arithmetic of both cells
// runs in the two lanes of the f32x2 instructions; min/max and the sign tests stay per lane.
// Every lane performs the scalar kernel's operations in the same order, so the bits are the
// same.  LPC = TC / 2 lanes per column, CPW = 32 / LPC columns per warp.
template <int NV, int TC>
struct LimPacked {
    static constexpr int J = (NV - 1) / 2;
    static constexpr int LPC = TC / 2;
    static constexpr int CPW = 32 / LPC;
    static constexpr int NW = (NV + CPW - 1) / CPW;
    static constexpr int kThreads = 32 * NW;
    static constexpr int PW = NV + 4;
    static constexpr int kRow = PW * TC;
    static constexpr int kPlane = NV * kRow;
    static constexpr size_t kSmem = 2 * (size_t)kPlane * sizeof(float);
    static_assert(TC % 2 == 0 && 32 % LPC == 0 && kThreads <= 1024, "tile shape");
};

// a * b lane by lane with scalar instructions (the rounding of mul2), for a product whose only
// use is a packed add or subtract (see sub2s in f32x2.h and face_vals_x2 below).
__device__ __forceinline__ f2 mul2s(f2 a, f2 b) {
    return pk(__fmul_rn(lo(a), lo(b)), __fmul_rn(hi(a), hi(b)));
}
__device__ __forceinline__ f2 ld2s(const float* p) { return *reinterpret_cast<const f2*>(p); }
__device__ __forceinline__ void st2s(float* p, f2 v) { *reinterpret_cast<f2*>(p) = v; }
__device__ __forceinline__ f2 splat(float a) { return pk(a, a); }

// lim_inc2<float> lane by lane
__device__ __forceinline__ f2 lim_inc2_x2(f2 dp, f2 dm, f2 mu2) {
    const float dp0 = lo(dp), dp1 = hi(dp);
    const f2 s = pk(copysignf(1.f, dp0), copysignf(1.f, dp1));
    const f2 b = mul2(s, fma2(dm, splat((float)(1.0 / 6.0)), mul2(dp, splat((float)(1.0 / 3.0)))));
    const f2 c = mul2(s, mul2(mu2, dm));
    const float m0 = fmaxf(0.f, fminf(fabsf(dp0), fminf(lo(b), lo(c))));
    const float m1 = fmaxf(0.f, fminf(fabsf(dp1), fminf(hi(b), hi(c))));
    return mul2(s, pk(m0, m1));
}
__device__ __forceinline__ f2 pos_part_x2(f2 P0, f2 P1, f2 P2, f2 mu2) {
    return add2(P1, lim_inc2_x2(sub2(P2, P1), sub2(P1, P0), mu2));
}
__device__ __forceinline__ f2 neg_part_x2(f2 M1, f2 M2, f2 M3, f2 mu2) {
    return add2(M2, lim_inc2_x2(sub2(M1, M2), sub2(M2, M3), mu2));
}
__device__ __forceinline__ f2 face_parts_x2(int kind, f2 P0, f2 P1, f2 P2, f2 M1, f2 M2, f2 M3,
                                            f2 mu2) {
    if (kind == kPosPart) return pos_part_x2(P0, P1, P2, mu2);
    if (kind == kNegPart) return neg_part_x2(M1, M2, M3, mu2);
    return add2(pos_part_x2(P0, P1, P2, mu2), neg_part_x2(M1, M2, M3, mu2));
}
// The split fluxes of a vx face are formed lane by lane (mul2s): each is used by this face
// only, and with mul.rn.f32x2 the kernels built by this toolchain differed from the scalar
// kernel by one unit in the last place in some faces, while every packed instruction on its own
// rounds exactly.
__device__ __forceinline__ f2 face_vals_x2(int kind, f2 x0, f2 x1, f2 x2, f2 x3, f2 cp0, f2 cp1,
                                           f2 cp2, f2 cm1, f2 cm2, f2 cm3, f2 mu2) {
    if (kind == kPosPart) return pos_part_x2(mul2s(cp0, x0), mul2s(cp1, x1), mul2s(cp2, x2), mu2);
    if (kind == kNegPart) return neg_part_x2(mul2s(cm1, x1), mul2s(cm2, x2), mul2s(cm3, x3), mu2);
    return add2(pos_part_x2(mul2s(cp0, x0), mul2s(cp1, x1), mul2s(cp2, x2), mu2),
                neg_part_x2(mul2s(cm1, x1), mul2s(cm2, x2), mul2s(cm3, x3), mu2));
}

// f* of cells x and x + 1 (column jx, all rows) into a plane; zeros beyond N_x.
template <int NV, int TC>
__device__ __forceinline__ void limp_load(const float* fin, float* plane, int nx, int ny, int y,
                                          int x, int jx, int c) {
    using L = LimPacked<NV, TC>;
    float* d = plane + (jx + 2) * TC + c;
    const size_t ncell = (size_t)nx * (size_t)ny;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        if (x + e >= nx) {
#pragma unroll
            for (int jy = 0; jy < NV; ++jy) d[jy * L::kRow + e] = 0.f;
            continue;
        }
        const float* src = fin + (size_t)jx * ncell + (size_t)wrap1(x + e - (jx - L::J), nx);
        int yr = wrap1(y + L::J, ny);
#pragma unroll
        for (int jy = 0; jy < NV; ++jy) {
            cp_async_elem(d + jy * L::kRow + e, src + (size_t)yr * nx);
            src += (size_t)NV * ncell;
            yr = yr == 0 ? ny - 1 : yr - 1;
        }
    }
}

// One Heun stage on column jx for the cell pair at offset c (as lim_fused_stage).
template <int NV, int TC, int STAGE, int UNR>
__device__ __forceinline__ void limp_stage(const float* src, float* dst, int jx, int c, bool store,
                                           f2 g2, f2 wy2, f2 mu2, const f2 (&cxp)[5],
                                           const f2 (&cxm)[5], int kl, int kr, int kyp, int kyn) {
    using L = LimPacked<NV, TC>;
    constexpr int J = L::J, R = L::kRow;
    const float* col = src + (jx + 2) * TC + c;
    float* out = dst + (jx + 2) * TC + c;
    const f2 z = pk(0.f, 0.f);
    f2 v[4], P[4], M[4];
    v[0] = P[0] = M[0] = z;
#pragma unroll
    for (int k = 1; k < 4; ++k) {
        const int jr = k - 1;
        v[k] = jr < NV ? ld2s(col + jr * R) : z;
        const f2 ca = mul2(g2, sub2(wy2, splat((float)(jr - J))));
        P[k] = mul2(max0(ca), v[k]);
        M[k] = mul2(min0(ca), v[k]);
    }
    f2 Fyl = z;
#pragma unroll(UNR)
    for (int jy = 0; jy < NV; ++jy) {
        f2 Fyr = z;
        if (jy < NV - 1)
            Fyr = face_parts_x2(face_kind(jy - 1, kyp, kyn), P[0], P[1], P[2], M[1], M[2], M[3],
                                mu2);
        const float* rp = col + jy * R;
        const f2 xm2 = ld2s(rp - 2 * TC), xm1 = ld2s(rp - TC), x0 = v[1], xp1 = ld2s(rp + TC),
                 xp2 = ld2s(rp + 2 * TC);
        f2 Fxl = face_vals_x2(kl, xm2, xm1, x0, xp1, cxp[0], cxp[1], cxp[2], cxm[1], cxm[2],
                              cxm[3], mu2);
        f2 Fxr = face_vals_x2(kr, xm1, x0, xp1, xp2, cxp[1], cxp[2], cxp[3], cxm[2], cxm[3],
                              cxm[4], mu2);
        if (jx == 0) Fxl = z;
        if (jx == NV - 1) Fxr = z;
        const f2 sv = sub2(sub2(x0, sub2(Fxr, Fxl)), sub2(Fyr, Fyl));
        if (store) {
            if (STAGE == 1) st2s(out + jy * R, sv);
            else st2s(out + jy * R, mul2(splat(0.5f), add2(ld2s(out + jy * R), sv)));
        }
        Fyl = Fyr;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            v[k] = v[k + 1];
            P[k] = P[k + 1];
            M[k] = M[k + 1];
        }
        const int jn = jy + 3;
        const f2 vn = ld2s(col + (jn < NV ? jn : NV - 1) * R);
        v[3] = jn < NV ? vn : z;
        const f2 ca = mul2(g2, sub2(wy2, splat((float)(jn - J))));
        P[3] = mul2(max0(ca), v[3]);
        M[3] = mul2(min0(ca), v[3]);
    }
}

// Diffusion of column jx for the cell pair (as lim_fused_diffuse); st0/st1: the cells to store.
template <int NV, int TC, int UNR>
__device__ __forceinline__ void limp_diffuse(const float* plane, float* gout, size_t ncell, int jx,
                                             int c, bool st0, bool st1, bool vec, f2 r2) {
    using L = LimPacked<NV, TC>;
    constexpr int R = L::kRow;
    const float* col = plane + (jx + 2) * TC + c;
    const f2 z = pk(0.f, 0.f);
    f2 hm = z, h0 = ld2s(col);
#pragma unroll(UNR)
    for (int jy = 0; jy < NV; ++jy) {
        const f2 hnext = ld2s(col + (jy < NV - 1 ? jy + 1 : jy) * R);
        const f2 hp = jy < NV - 1 ? hnext : z;
        const f2 hl = ld2s(col + jy * R - TC), hr = ld2s(col + jy * R + TC);
        const f2 Dxr = jx < NV - 1 ? mul2(r2, sub2(hr, h0)) : z;
        const f2 Dxl = jx > 0 ? mul2(r2, sub2(h0, hl)) : z;
        const f2 Dyr = jy < NV - 1 ? mul2(r2, sub2(hp, h0)) : z;
        const f2 Dyl = jy > 0 ? mul2(r2, sub2(h0, hm)) : z;
        // the differences of two products by r lane by lane (sub2s): with sub.rn.f32x2 there,
        // a few cells came out one unit in the last place away from the scalar kernel's
        const f2 o = add2(add2(h0, sub2s(Dxr, Dxl)), sub2s(Dyr, Dyl));
        float* gp = gout + (size_t)jy * NV * ncell;
        if (vec) {
            st2s(gp, o);
        } else {
            if (st0) gp[0] = lo(o);
            if (st1) gp[1] = hi(o);
        }
        hm = h0;
        h0 = hp;
    }
}

template <int NV, int TC, int MINB, int UNR>
__global__ void __launch_bounds__(LimPacked<NV, TC>::kThreads, MINB)
    k_lim2d_packed(const Lim2DArgs a, int kstep) {
    using L = LimPacked<NV, TC>;
    using O = Ops<float>;
    constexpr int J = L::J;
    extern __shared__ __align__(16) unsigned char limp_smem[];
    float* pa = reinterpret_cast<float*>(limp_smem);
    float* pb = pa + L::kPlane;
    const int nx = a.nx, ny = a.ny;
    const size_t ncell = (size_t)nx * (size_t)ny;
    const bool par = ((a.st->step + kstep) & 1) != 0;
    const float* fin = static_cast<const float*>(par ? a.f[1] : a.f[0]);
    float* fout = static_cast<float*>(par ? a.f[0] : a.f[1]);
    const float* u = static_cast<const float*>(a.u);
    const float g = (float)a.g, mu = (float)a.mu, inv_dv = (float)a.inv_dv;
    const float cflf = O::mul(g, O::add(1.f, mu));
    const f2 g2 = splat(g), mu2 = splat(mu), r2 = splat((float)a.r);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = 2 * (lane % L::LPC);
    const int jx_raw = warp * L::CPW + lane / L::LPC;
    const bool active = jx_raw < NV;  // spare columns of the last warp compute column NV - 1
    const int jx = active ? jx_raw : NV - 1;
    const int ntx = (nx + TC - 1) / TC;
    const long long ntiles = (long long)ntx * ny;
    // pairs of cells 8-byte aligned in the output buffer: one 8-byte store per pair
    const bool even = (nx & 1) == 0 && (reinterpret_cast<uintptr_t>(fout) & 7) == 0;
    for (int i = threadIdx.x; i < 2 * NV * 4 * TC; i += blockDim.x) {
        const int e = i % TC, k = (i / TC) % 4, row = (i / (4 * TC)) % NV, p = i / (4 * TC * NV);
        (p ? pb : pa)[row * L::kRow + (k < 2 ? k : NV + k) * TC + e] = 0.f;
    }
    long long t = blockIdx.x;
    if (t < ntiles && active) {
        const int y = (int)(t / ntx);
        limp_load<NV, TC>(fin, pa, nx, ny, y, (int)(t - (long long)y * ntx) * TC + c, jx, c);
    }
    bool cfl = false;
    for (; t < ntiles; t += gridDim.x) {
        const int y = (int)(t / ntx);
        const int x = (int)(t - (long long)y * ntx) * TC + c;
        const bool in0 = x < nx, in1 = x + 1 < nx;
        float wx0 = 0.f, wy0 = 0.f, wx1 = 0.f, wy1 = 0.f;
        if (u) {
            const float* ur = u + (size_t)y * nx + x;
            if (in0) {
                wx0 = O::mul(ur[0], inv_dv);
                wy0 = O::mul(ur[ncell], inv_dv);
            }
            if (in1) {
                wx1 = O::mul(ur[1], inv_dv);
                wy1 = O::mul(ur[ncell + 1], inv_dv);
            }
        }
        if (jx_raw == 0 && ((in0 && cflf * (float(2 * J) + fabsf(wx0) + fabsf(wy0)) > 1.f) ||
                            (in1 && cflf * (float(2 * J) + fabsf(wx1) + fabsf(wy1)) > 1.f)))
            cfl = true;
        const f2 wx2 = pk(wx0, wx1), wy2 = pk(wy0, wy1);
        f2 cxp[5], cxm[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const f2 ca = mul2(g2, sub2(wx2, splat((float)(jx - 2 + k - J))));
            cxp[k] = max0(ca);
            cxm[k] = min0(ca);
        }
        int kxp, kxn, kyp, kyn, kp1, kn1;
        sign_bounds<float>(wx0, J, kxp, kxn);
        sign_bounds<float>(wx1, J, kp1, kn1);
        kxp = min(kxp, kp1);
        kxn = max(kxn, kn1);
        sign_bounds<float>(wy0, J, kyp, kyn);
        sign_bounds<float>(wy1, J, kp1, kn1);
        kyp = __reduce_min_sync(0xffffffffu, min(kyp, kp1));
        kyn = __reduce_max_sync(0xffffffffu, max(kyn, kn1));
        const int kl = uniform_kind(face_kind(jx - 2, kxp, kxn));
        const int kr = uniform_kind(face_kind(jx - 1, kxp, kxn));
        cp_async_wait_all();
        __syncthreads();
        limp_stage<NV, TC, 1, UNR>(pa, pb, jx, c, active, g2, wy2, mu2, cxp, cxm, kl, kr, kyp, kyn);
        __syncthreads();
        limp_stage<NV, TC, 2, UNR>(pb, pa, jx, c, active, g2, wy2, mu2, cxp, cxm, kl, kr, kyp, kyn);
        __syncthreads();
        const long long tn = t + gridDim.x;
        if (tn < ntiles && active) {
            const int yn = (int)(tn / ntx);
            limp_load<NV, TC>(fin, pb, nx, ny, yn, (int)(tn - (long long)yn * ntx) * TC + c, jx, c);
        }
        float* gout = fout + ((size_t)jx * ny + y) * nx + (in0 ? x : 0);
        limp_diffuse<NV, TC, UNR>(pa, gout, ncell, jx, c, active && in0, active && in1,
                                  active && in1 && even, r2);
        float* tmp = pa;
        pa = pb;
        pb = tmp;
    }
    cp_async_wait_all();
    if (cfl) atomicOr(&a.st->status, ST_CFL);
}

template <int NV, int TC, int MINB, int UNR = 4>
cudaError_t launch_packed_t(const Lim2DArgs& a, int k, int sm_count, cudaStream_t s) {
    using L = LimPacked<NV, TC>;
    static bool attr = false;
    static int per_sm = 0;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_lim2d_packed<NV, TC, MINB, UNR>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)L::kSmem);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, k_lim2d_packed<NV, TC, MINB, UNR>, L::kThreads, L::kSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const long long ntiles = (long long)((a.nx + TC - 1) / TC) * a.ny;
    const int grid = (int)std::min<long long>(ntiles, (long long)std::max(per_sm, 1) * sm_count);
    k_lim2d_packed<NV, TC, MINB, UNR><<<grid, L::kThreads, L::kSmem, s>>>(a, k);
    return cudaGetLastError();
}

cudaError_t launch_packed(const Lim2DArgs& a, int k, int sm_count, cudaStream_t s) {
    switch (a.nv) {
        case 5: return launch_packed_t<5, 32, 4>(a, k, sm_count, s);
        case 9: return launch_packed_t<9, 32, 4>(a, k, sm_count, s);
        case 13: return launch_packed_t<13, 32, 3>(a, k, sm_count, s);
        case 17: return launch_packed_t<17, 32, 2>(a, k, sm_count, s);
        case 19: return launch_packed_t<19, 32, 2>(a, k, sm_count, s);
        case 21: return launch_packed_t<21, 16, 3>(a, k, sm_count, s);
        case 33: return launch_packed_t<33, 16, 1>(a, k, sm_count, s);
        default: return cudaErrorNotSupported;
    }
}

// The fused form for the lattices it is built for (N_v = 5, 9, 13, 17, 19, 21, 33);
// cudaErrorNotSupported for the others, which take the three passes.  bps: blocks per SM the FP32 kernels of N_v = 17
// and 19 are compiled for (1: registers for the whole sweep; 2, the default: 48 registers).
template <typename T>
cudaError_t launch_fused(const Lim2DArgs& a, int bps, int k, int sm_count, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        switch (a.nv) {
            case 5: return launch_fused_t<T, 5, 32, 1>(a, k, sm_count, s);
            case 9: return launch_fused_t<T, 9, 32, 1>(a, k, sm_count, s);
            case 13: return launch_fused_t<T, 13, 32, 1>(a, k, sm_count, s);
            case 17:
                return bps == 1 ? launch_fused_t<T, 17, 32, 1>(a, k, sm_count, s)
                                : launch_fused_t<T, 17, 32, 2>(a, k, sm_count, s);
            case 19:
                return bps == 1 ? launch_fused_t<T, 19, 32, 1>(a, k, sm_count, s)
                                : launch_fused_t<T, 19, 32, 2>(a, k, sm_count, s);
            case 21: return launch_fused_t<T, 21, 32, 1>(a, k, sm_count, s);
            case 33: return launch_fused_t<T, 33, 16, 1>(a, k, sm_count, s);
            default: return cudaErrorNotSupported;
        }
    } else {
        switch (a.nv) {
            case 5: return launch_fused_t<T, 5, 32, 1>(a, k, sm_count, s);
            case 9: return launch_fused_t<T, 9, 32, 1>(a, k, sm_count, s);
            case 13: return launch_fused_t<T, 13, 32, 1>(a, k, sm_count, s);
            case 17: return launch_fused_t<T, 17, 16, 1>(a, k, sm_count, s);
            case 19: return launch_fused_t<T, 19, 16, 1>(a, k, sm_count, s);
            case 21: return launch_fused_t<T, 21, 16, 1>(a, k, sm_count, s);
            case 33: return launch_fused_t<T, 33, 8, 1>(a, k, sm_count, s);
            default: return cudaErrorNotSupported;
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

bool limiter2d_fused_supported(int nv) {
    return nv == 5 || nv == 9 || nv == 13 || nv == 17 || nv == 19 || nv == 21 || nv == 33;
}

// One limited 2D step k of an enqueued batch: input buffer f[par], output f[par ^ 1] (par from
// the device step counter plus k).  form 1: three passes (a scratch of the state's size);
// 2: the fused kernel; 3: its packed FP32 form.
cudaError_t launch_step2d_limited(int dtype, const Step2DArgs& s2, int nv, double mu, void* scratch,
                                  int form, int bps, int k, int sm_count, cudaStream_t s) {
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
    if (form == 3 && dtype == LAT_F32 && limiter2d_fused_supported(nv))
        return launch_packed(a, k, sm_count, s);
    if (form >= 2 && limiter2d_fused_supported(nv)) {
        if (dtype == LAT_F32) return launch_fused<float>(a, bps, k, sm_count, s);
        if (dtype == LAT_F64) return launch_fused<double>(a, bps, k, sm_count, s);
        return cudaErrorInvalidValue;
    }
    if (dtype == LAT_F32) return launch_lim2d_t<float>(a, k, sm_count, s);
    if (dtype == LAT_F64) return launch_lim2d_t<double>(a, k, sm_count, s);
    return cudaErrorInvalidValue;
}

}  // namespace lat

// Learned flux closure on a coarse 2D lattice, FP32 on CUDA cores: the streamed density, the
// per-cell network and correction fluxes, the corrected step, and the exact gradient of a
// rollout's loss with respect to the network's parameters (the adjoint of every step).
//
// Features of phase-space cell (x, j) after streaming, in order: f*(x, j + d) / rho*(x) for
// d = (dy, dx) in {-1, 0, 1}^2 row-major (0 outside the velocity box), dt du_x/dx, dt du_x/dy,
// dt du_y/dx, dt du_y/dy (centred differences on the periodic grid), the drag Courant numbers
// c a_x = g (w_x - (jx - J)) and c a_y = g (w_y - (jy - J)), and 1.  Network: 16 -> 64 -> 64 -> 2
// with ReLU, outputs y = b tanh(z) (b = kYMax towards extra diffusion, at most kTheta times the
// face's upwind numerical diffusivity towards anti-diffusion); correction fluxes
// y_0 (f*_{jx+1} - f*_{jx}) through face
// jx + 1/2 and y_1 (f*_{jy+1} - f*_{jy}) through face jy + 1/2 on interior faces only (a learned
// face diffusivity), so mass is kept exactly.  The paper suggests large-eddy closures for the
// lattice (Section 5); this is one, trained against a restricted fine lattice.
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "learn.h"

namespace lat {
namespace {

using namespace k2d;

__device__ __forceinline__ int vwrap(int v, int n) { return wrap_near(v, n); }

// f*(x, y, jx, jy) of buffer f = f(x - (jx - J), y - (jy - J), jx, jy)
template <int NV>
__device__ __forceinline__ float fstar(const float* f, int jx, int jy, int x, int y, int nx,
                                       int ny) {
    constexpr int J = (NV - 1) / 2;
    const size_t ncell = (size_t)nx * ny;
    return f[(size_t)(jy * NV + jx) * ncell + (size_t)vwrap(y - (jy - J), ny) * nx +
             vwrap(x - (jx - J), nx)];
}

template <int NV>
__global__ void __launch_bounds__(256) k_rho_star(const LearnArgs a, int kstep) {
    const float* f = a.f[(int)((a.st->step + kstep) & 1)];
    const long long ncell = (long long)a.nx * a.ny;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const int y = (int)((unsigned)c / (unsigned)a.nx), x = (int)((unsigned)c - (unsigned)y * a.nx);
        float s = 0.f;
        for (int jy = 0; jy < NV; ++jy)
            for (int jx = 0; jx < NV; ++jx) s = __fadd_rn(s, fstar<NV>(f, jx, jy, x, y, a.nx, a.ny));
        a.rho[c] = s;
        if (a.feat) {
            // the spatial parts of the features, formed once per cell with the same operations
            // as features(): 1/rho*, dt times the centred velocity gradients, u / dv
            const float* ux = a.u;
            const float* uy = a.u + ncell;
            const int xp = x + 1 == a.nx ? 0 : x + 1, xm = x == 0 ? a.nx - 1 : x - 1;
            const int yp = y + 1 == a.ny ? 0 : y + 1, ym = y == 0 ? a.ny - 1 : y - 1;
            const size_t yr = (size_t)y * a.nx;
            float4 fa, fb;
            fa.x = s != 0.f ? __frcp_rn(s) : 0.f;
            fa.y = __fmul_rn(__fsub_rn(ux[yr + xp], ux[yr + xm]), a.dt_2dx);
            fa.z = __fmul_rn(__fsub_rn(ux[(size_t)yp * a.nx + x], ux[(size_t)ym * a.nx + x]), a.dt_2dx);
            fa.w = __fmul_rn(__fsub_rn(uy[yr + xp], uy[yr + xm]), a.dt_2dx);
            fb.x = __fmul_rn(__fsub_rn(uy[(size_t)yp * a.nx + x], uy[(size_t)ym * a.nx + x]), a.dt_2dx);
            fb.y = __fmul_rn(ux[c], a.inv_dv);
            fb.z = __fmul_rn(uy[c], a.inv_dv);
            fb.w = 0.f;
            a.feat[2 * c] = fa;
            a.feat[2 * c + 1] = fb;
        }
    }
}

// f* of the cell and of its +jx and +jy neighbours (0 outside the box): the correction's factors
struct Nbr {
    float c, xp, yp;
};

// Features of phase cell (jx, jy, x, y); returns 1 / rho* (0 where rho* = 0).
template <int NV>
__device__ __forceinline__ float features(const LearnArgs& a, const float* f, int jx, int jy,
                                          int x, int y, float (&X)[kLNF], Nbr& nb) {
    constexpr int J = (NV - 1) / 2;
    const float rho = a.rho[(size_t)y * a.nx + x];
    const float inv = rho != 0.f ? __frcp_rn(rho) : 0.f;
    int q = 0;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            const int jx2 = jx + dx, jy2 = jy + dy;
            const bool in = jx2 >= 0 && jx2 < NV && jy2 >= 0 && jy2 < NV;
            const float v = in ? fstar<NV>(f, jx2, jy2, x, y, a.nx, a.ny) : 0.f;
            if (dy == 0 && dx == 0) nb.c = v;
            if (dy == 0 && dx == 1) nb.xp = v;
            if (dy == 1 && dx == 0) nb.yp = v;
            X[q++] = __fmul_rn(v, inv);
        }
    const size_t ncell = (size_t)a.nx * a.ny;
    const float* ux = a.u;
    const float* uy = a.u + ncell;
    const size_t c = (size_t)y * a.nx + x;
    const int xp = x + 1 == a.nx ? 0 : x + 1, xm = x == 0 ? a.nx - 1 : x - 1;
    const int yp = y + 1 == a.ny ? 0 : y + 1, ym = y == 0 ? a.ny - 1 : y - 1;
    X[9] = __fmul_rn(__fsub_rn(ux[(size_t)y * a.nx + xp], ux[(size_t)y * a.nx + xm]), a.dt_2dx);
    X[10] = __fmul_rn(__fsub_rn(ux[(size_t)yp * a.nx + x], ux[(size_t)ym * a.nx + x]), a.dt_2dx);
    X[11] = __fmul_rn(__fsub_rn(uy[(size_t)y * a.nx + xp], uy[(size_t)y * a.nx + xm]), a.dt_2dx);
    X[12] = __fmul_rn(__fsub_rn(uy[(size_t)yp * a.nx + x], uy[(size_t)ym * a.nx + x]), a.dt_2dx);
    X[13] = __fmul_rn(a.g, __fsub_rn(__fmul_rn(ux[c], a.inv_dv), (float)(jx - J)));
    X[14] = __fmul_rn(a.g, __fsub_rn(__fmul_rn(uy[c], a.inv_dv), (float)(jy - J)));
    X[15] = 1.f;
    return inv;
}

__device__ __forceinline__ void load_params(const float* params, float* sp) {
    for (int i = threadIdx.x; i < kLNParam; i += blockDim.x) sp[i] = params[i];
    __syncthreads();
}

// h1 = relu(X W1 + b1), z1 kept for the backward mask
__device__ __forceinline__ void layer1(const float* P, const float (&X)[kLNF], float (&h1)[kLNH]) {
#pragma unroll
    for (int n = 0; n < kLNH; ++n) h1[n] = P[kOffB1 + n];
#pragma unroll
    for (int k = 0; k < kLNF; ++k)
#pragma unroll
        for (int n = 0; n < kLNH; ++n) h1[n] = __fmaf_rn(X[k], P[kOffW1 + k * kLNH + n], h1[n]);
}

__device__ __forceinline__ void layer2(const float* P, const float (&h1)[kLNH], float (&z2)[kLNH]) {
#pragma unroll
    for (int n = 0; n < kLNH; ++n) z2[n] = P[kOffB2 + n];
    for (int k = 0; k < kLNH; ++k) {
        const float hk = fmaxf(h1[k], 0.f);
#pragma unroll
        for (int n = 0; n < kLNH; ++n) z2[n] = __fmaf_rn(hk, P[kOffW2 + k * kLNH + n], z2[n]);
    }
}

// y = b tanh(h2 W3 + b3), b = anti_bound(.) for z > 0 and kYMax otherwise; t = tanh(.) and the
// bounds kept for the backward
struct Out3 {
    float y0, y1, t0, t1, b0, b1;
};
__device__ __forceinline__ Out3 layer3(const float* P, const float (&z2)[kLNH],
                                       const float (&X)[kLNF], float g) {
    float z0 = P[kOffB3], z1 = P[kOffB3 + 1];
#pragma unroll
    for (int k = 0; k < kLNH; ++k) {
        const float hk = fmaxf(z2[k], 0.f);
        z0 = __fmaf_rn(hk, P[kOffW3 + 2 * k], z0);
        z1 = __fmaf_rn(hk, P[kOffW3 + 2 * k + 1], z1);
    }
    Out3 o;
    o.t0 = tanhf(z0);
    o.t1 = tanhf(z1);
    o.b0 = z0 > 0.f ? anti_bound(X[13], g) : kYMax;
    o.b1 = z1 > 0.f ? anti_bound(X[14], g) : kYMax;
    o.y0 = __fmul_rn(o.b0, o.t0);
    o.y1 = __fmul_rn(o.b1, o.t1);
    return o;
}

template <int NV>
__global__ void __launch_bounds__(128) k_mlp_f32(const LearnArgs a, int kstep) {
    __shared__ float P[kLNParam];
    load_params(a.params, P);
    const float* f = a.f[(int)((a.st->step + kstep) & 1)];
    const long long ncell = (long long)a.nx * a.ny;
    const long long n = ncell * NV * NV;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        int p, x, y;
        split_index((unsigned)i, (unsigned)ncell, (unsigned)a.nx, p, x, y);
        const int jy = p / NV, jx = p % NV;
        float X[kLNF], h1[kLNH], z2[kLNH];
        Nbr nb;
        features<NV>(a, f, jx, jy, x, y, X, nb);
        layer1(P, X, h1);
        layer2(P, h1, z2);
        const Out3 o = layer3(P, z2, X, a.g);
        a.G[i] = jx < NV - 1 ? __fmul_rn(o.y0, __fsub_rn(nb.xp, nb.c)) : 0.f;
        a.G[n + i] = jy < NV - 1 ? __fmul_rn(o.y1, __fsub_rn(nb.yp, nb.c)) : 0.f;
    }
}


template <int NV>
__global__ void __launch_bounds__(TW) k_step2d_corr(const Step2DArgs a, const float* G, int kstep) {
    const long long step = a.st->step + kstep;
    const int par = (int)(step & 1);
    const float g = float(a.g), rr = float(a.r);
    const float* fin = static_cast<const float*>(par ? a.f[1] : a.f[0]);
    float* fout = static_cast<float*>(par ? a.f[0] : a.f[1]);
    const size_t ps = (size_t)a.nx * a.ny;
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const int y = tile / a.ntx;
        const int xr = (tile % a.ntx) * TW + threadIdx.x;
        const bool active = xr < a.nx;
        const int x = active ? xr : 0;
        float wx, wy;
        load_w<float>(a, x, y, wx, wy);
        cfl_check<float, NV>(a, g, wx, wy, active);
        float A[NV], Gr[NV], H[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            A[j] = 0.f;
            Gr[j] = 0.f;
            H[j] = 0.f;
        }
        const size_t c = (size_t)y * a.nx + x;
        const GlobCorr corr{G + c, G + (size_t)NV * NV * ps + c, ps, NV};
        StorePut<float, NV, false> put(fout + c, ps, active);  // global loads: plain steps
        for (int r = 1; r <= NV; ++r) {
            const GlobalRow<float, NV> cur(fin, r - 1, x, y, a.nx, a.ny);
            const GlobalRow<float, NV> nxt(fin, r < NV ? r : r - 1, x, y, a.nx, a.ny);
            sweep_row<float, NV>(A, Gr, H, r, cur, nxt, g, wx, wy, rr, put, corr);
        }
        final_row<float, NV>(A, H, rr, put);
    }
}

// ---- backward -------------------------------------------------------------------------------
// lss = Diff(lam): the zero-flux five-point velocity Laplacian step is symmetric.
template <int NV>
__global__ void __launch_bounds__(256) k_diffuse_adjoint(const float* lam, float* out, float r,
                                                         int nx, int ny) {
    const long long ncell = (long long)nx * ny;
    const long long n = ncell * NV * NV;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(i / ncell);
        const int jy = p / NV, jx = p % NV;
        const float v = lam[i];
        float s = 0.f;
        if (jx > 0) s = __fadd_rn(s, __fsub_rn(lam[i - ncell], v));
        if (jx < NV - 1) s = __fadd_rn(s, __fsub_rn(lam[i + ncell], v));
        if (jy > 0) s = __fadd_rn(s, __fsub_rn(lam[i - NV * ncell], v));
        if (jy < NV - 1) s = __fadd_rn(s, __fsub_rn(lam[i + NV * ncell], v));
        out[i] = __fadd_rn(v, __fmul_rn(r, s));
    }
}

constexpr int kBT = 128;  // phase cells per backward tile (= threads per block)
// per-cell vectors kept in shared memory, rows of kBT (cell fastest): X 16, dz1 64, h1 64,
// dz2 64, h2 64, dz3 2 (rows kRDY); h1 and h2 are after the ReLU, so h > 0 is the ReLU's
// derivative mask
constexpr int kRX = 0, kRDZ1 = kLNF, kRH1 = kRDZ1 + kLNH, kRDZ2 = kRH1 + kLNH,
              kRH2 = kRDZ2 + kLNH, kRDY = kRH2 + kLNH, kVec = kRDY + kLNO;
constexpr int kPerThread = (kLNParam + kBT - 1) / kBT;

// One block per SM loops over tiles of kBT phase cells.  Per cell: the forward again, the adjoint
// of the corrected drag fluxes, the network's backward; per tile the weight gradients as sums over
// the tile's cells (thread t owns parameters t, t + kBT, ...), kept in registers across tiles and
// added to grad once per block.
template <int NV>
__global__ void __launch_bounds__(kBT, 1) k_mlp_bwd(const LearnBwdArgs b) {
    extern __shared__ float sh[];
    float* P = sh;                       // parameters
    float* V = sh + kLNParam;            // [kVec][kBT]
    float* ACC = V + kVec * kBT;         // [kPerThread][kBT] this block's gradient sums
    const LearnArgs& a = b.fw;
    load_params(a.params, P);
    const float* f = a.f[0];
    const long long ncell = (long long)a.nx * a.ny;
    const long long n = ncell * NV * NV;
    const long long ntiles = (n + kBT - 1) / kBT;
    const int t = threadIdx.x;
    auto v = [&](int row) -> float& { return V[row * kBT + t]; };
    for (int m = 0; m < kPerThread; ++m) ACC[m * kBT + t] = 0.f;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long i = tile * kBT + t;
        if (i < n) {
            int p, x, y;
            split_index((unsigned)i, (unsigned)ncell, (unsigned)a.nx, p, x, y);
            const long long c = (long long)y * a.nx + x;
            const int jy = p / NV, jx = p % NV;
            float X[kLNF];
            Nbr nb;
            const float inv = features<NV>(a, f, jx, jy, x, y, X, nb);
#pragma unroll
            for (int q = 0; q < kLNF; ++q) v(kRX + q) = X[q];
            Out3 o;
            {
                float h1[kLNH];
                layer1(P, X, h1);
#pragma unroll
                for (int k = 0; k < kLNH; ++k) v(kRH1 + k) = fmaxf(h1[k], 0.f);
            }
            {
                float z2[kLNH];
#pragma unroll
                for (int nn = 0; nn < kLNH; ++nn) z2[nn] = P[kOffB2 + nn];
                for (int k = 0; k < kLNH; ++k) {
                    const float hk = v(kRH1 + k);
#pragma unroll
                    for (int nn = 0; nn < kLNH; ++nn) z2[nn] = __fmaf_rn(hk, P[kOffW2 + k * kLNH + nn], z2[nn]);
                }
#pragma unroll
                for (int k = 0; k < kLNH; ++k) v(kRH2 + k) = fmaxf(z2[k], 0.f);
                o = layer3(P, z2, X, a.g);
            }
            // adjoint of f** = f* - (F_{j+1/2} - F_{j-1/2}) in x and y, F = upwind + correction
            const float* L = b.lss;
            const float l0 = L[i];
            const float lxp = jx < NV - 1 ? __fsub_rn(L[i + ncell], l0) : 0.f;   // face jx + 1/2
            const float lxm = jx > 0 ? __fsub_rn(l0, L[i - ncell]) : 0.f;       // face jx - 1/2
            const float lyp = jy < NV - 1 ? __fsub_rn(L[i + NV * ncell], l0) : 0.f;
            const float lym = jy > 0 ? __fsub_rn(l0, L[i - NV * ncell]) : 0.f;
            const float cax = X[13], cay = X[14];
            float lf = l0;
            lf = __fmaf_rn(fmaxf(cax, 0.f), lxp, lf);
            lf = __fmaf_rn(fminf(cax, 0.f), lxm, lf);
            lf = __fmaf_rn(fmaxf(cay, 0.f), lyp, lf);
            lf = __fmaf_rn(fminf(cay, 0.f), lym, lf);
            // correction G_{j+1/2} = y (f*_{j+1} - f*_j): -y lambda_F to this cell, +y lambda_F
            // to the +jx / +jy neighbour (gathered there), dL/dy = lambda_F (f*_{j+1} - f*_j)
            const float cx = __fmul_rn(o.y0, lxp), cy = __fmul_rn(o.y1, lyp);
            lf = __fsub_rn(__fsub_rn(lf, cx), cy);
            b.cxy[i] = cx;
            b.cxy[n + i] = cy;
            const float dy0 = __fmul_rn(lxp, __fsub_rn(nb.xp, nb.c));
            const float dy1 = __fmul_rn(lyp, __fsub_rn(nb.yp, nb.c));
            // through y = b tanh(z3)
            const float dz30 = __fmul_rn(dy0, __fmul_rn(o.b0, __fsub_rn(1.f, __fmul_rn(o.t0, o.t0))));
            const float dz31 = __fmul_rn(dy1, __fmul_rn(o.b1, __fsub_rn(1.f, __fmul_rn(o.t1, o.t1))));
            v(kRDY) = dz30;
            v(kRDY + 1) = dz31;
            float lr = 0.f;
            // network backward: dz2 = (dz3 W3^T) [h2 > 0], dz1 = (dz2 W2^T) [h1 > 0], dX = dz1 W1^T
#pragma unroll
            for (int k = 0; k < kLNH; ++k) {
                const float d = __fmaf_rn(dz30, P[kOffW3 + 2 * k], __fmul_rn(dz31, P[kOffW3 + 2 * k + 1]));
                v(kRDZ2 + k) = v(kRH2 + k) > 0.f ? d : 0.f;
            }
            {
                float dz1[kLNH];
#pragma unroll
                for (int k = 0; k < kLNH; ++k) dz1[k] = 0.f;
                for (int nn = 0; nn < kLNH; ++nn) {
                    const float d = v(kRDZ2 + nn);
#pragma unroll
                    for (int k = 0; k < kLNH; ++k) dz1[k] = __fmaf_rn(d, P[kOffW2 + k * kLNH + nn], dz1[k]);
                }
#pragma unroll
                for (int k = 0; k < kLNH; ++k) v(kRDZ1 + k) = v(kRH1 + k) > 0.f ? dz1[k] : 0.f;
            }
            // neighbour features X_q = f*_q / rho*: d/df*_q = dX_q / rho*, d/drho* = -dX_q X_q / rho*
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                float d = 0.f;
                for (int k = 0; k < kLNH; ++k) d = __fmaf_rn(v(kRDZ1 + k), P[kOffW1 + q * kLNH + k], d);
                b.dX9[(size_t)q * n + i] = __fmul_rn(d, inv);
                lr = __fsub_rn(lr, __fmul_rn(__fmul_rn(d, X[q]), inv));
            }
            b.lfs[i] = lf;
            atomicAdd(&b.lrho[c], lr);
        } else {
            for (int row = 0; row < kVec; ++row) v(row) = 0.f;
        }
        __syncthreads();
        // parameter e = t + kBT m: gradient = sum over the tile's cells of (left) * (right)
#pragma unroll 1
        for (int m = 0; m < kPerThread; ++m) {
            const int e = t + kBT * m;
            if (e < kLNParam) {
                int lo, ro;  // rows of V: left factor (-1 for the constant 1) and right factor
                if (e < kOffB1) { lo = kRX + e / kLNH; ro = kRDZ1 + e % kLNH; }
                else if (e < kOffW2) { lo = -1; ro = kRDZ1 + (e - kOffB1); }
                else if (e < kOffB2) { lo = kRH1 + (e - kOffW2) / kLNH; ro = kRDZ2 + (e - kOffW2) % kLNH; }
                else if (e < kOffW3) { lo = -1; ro = kRDZ2 + (e - kOffB2); }
                else if (e < kOffB3) { lo = kRH2 + (e - kOffW3) / kLNO; ro = kRDY + (e - kOffW3) % kLNO; }
                else { lo = -1; ro = kRDY + (e - kOffB3); }
                const float* R = V + (size_t)ro * kBT;
                float s = 0.f;
                if (lo < 0) {
                    for (int cc = 0; cc < kBT; ++cc) s = __fadd_rn(s, R[cc]);
                } else {
                    const float* Lf = V + (size_t)lo * kBT;
                    for (int cc = 0; cc < kBT; ++cc) s = __fmaf_rn(Lf[cc], R[cc], s);
                }
                ACC[m * kBT + t] = __fadd_rn(ACC[m * kBT + t], s);
            }
        }
        __syncthreads();
    }
    for (int m = 0; m < kPerThread; ++m) {
        const int e = t + kBT * m;
        if (e < kLNParam) atomicAdd(&b.grad[e], ACC[m * kBT + t]);
    }
}

// lam_in(x, j) = lambda_f*(x + (j - J), j): the identity/upwind part, the neighbour features
// (dX9 of the cells whose features read this plane) and the streamed density's adjoint.
template <int NV>
__global__ void __launch_bounds__(256) k_gather_adjoint(const LearnBwdArgs b) {
    constexpr int J = (NV - 1) / 2;
    const int nx = b.fw.nx, ny = b.fw.ny;
    const long long ncell = (long long)nx * ny;
    const long long n = ncell * NV * NV;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        int p, x, y;
        split_index((unsigned)i, (unsigned)ncell, (unsigned)nx, p, x, y);
        const int jy = p / NV, jx = p % NV;
        // f^n at (x, y) of plane p streams to (x + jx - J, y + jy - J)
        const long long cs = (long long)vwrap(y + (jy - J), ny) * nx + vwrap(x + (jx - J), nx);
        const long long is = (long long)p * ncell + cs;
        float v = b.lfs[is];
        // corrections through faces jx - 1/2 and jy - 1/2, owned by the -jx / -jy neighbours
        if (jx > 0) v = __fadd_rn(v, b.cxy[is - ncell]);
        if (jy > 0) v = __fadd_rn(v, b.cxy[n + is - (long long)NV * ncell]);
        int q = 0;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx, ++q) {
                // cell (jx - dx, jy - dy) read this plane as its feature q
                const int jx2 = jx - dx, jy2 = jy - dy;
                if (jx2 < 0 || jx2 >= NV || jy2 < 0 || jy2 >= NV) continue;
                v = __fadd_rn(v, b.dX9[(size_t)q * n + (size_t)(jy2 * NV + jx2) * ncell + cs]);
            }
        b.lam_in[i] = __fadd_rn(v, b.lrho[cs]);
    }
}

// coarse[kc_y][kc_x][y][x] = sum over the fine cells j = 4 k + d, d in -2..2 per axis, of
// w(d_y) w(d_x) / 16 fine[j_y][j_x][y][x] with w = (1/2, 1, 1, 1, 1/2): the restriction that
// keeps the mass sum f dv^2 when dv grows fourfold.
__global__ void __launch_bounds__(256) k_restrict(const float* fine, int nvf, int nx, int ny,
                                                  float* coarse) {
    const int nvc = (nvf - 1) / 4 + 1;
    const int Jf = (nvf - 1) / 2, Jc = (nvc - 1) / 2;
    const long long ncell = (long long)nx * ny;
    const long long n = ncell * nvc * nvc;
    const float w[5] = {0.5f, 1.f, 1.f, 1.f, 0.5f};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(i / ncell);
        const long long c = i % ncell;
        const int ky = p / nvc - Jc, kx = p % nvc - Jc;
        float s = 0.f;
        for (int dy = -2; dy <= 2; ++dy) {
            const int jy = 4 * ky + dy;
            if (jy < -Jf || jy > Jf) continue;
            for (int dx = -2; dx <= 2; ++dx) {
                const int jx = 4 * kx + dx;
                if (jx < -Jf || jx > Jf) continue;
                const float v = fine[(size_t)((jy + Jf) * nvf + (jx + Jf)) * ncell + c];
                s = __fmaf_rn(__fmul_rn(w[dy + 2], w[dx + 2]), v, s);
            }
        }
        coarse[i] = __fmul_rn(s, 0.0625f);
    }
}

// Density error per spatial cell r(x) = sum_j (f - target), and sums of r^2 per block.
__global__ void __launch_bounds__(256) k_rho_err(const float* f, const float* target, int np,
                                                 long long ncell, float* r, double* partials) {
    __shared__ double red[8];
    double s = 0.0;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        double d = 0.0;
        for (int p = 0; p < np; ++p) d += (double)f[p * ncell + c] - (double)target[p * ncell + c];
        r[c] = (float)d;
        s += d * d;
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double z = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) z += red[q];
        partials[blockIdx.x] = z;
    }
}

// lam = 2 (f - target) / n + rho_weight 2 r(x) / ncell, and sums of (f - target)^2 per block.
__global__ void __launch_bounds__(256) k_loss(const float* f, const float* target, long long n,
                                              long long ncell, const float* r, double rho_weight,
                                              float* lam, double* partials) {
    __shared__ double red[8];
    double s = 0.0;
    const double w = 2.0 / (double)n, wr = 2.0 * rho_weight / (double)ncell;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double d = (double)f[i] - (double)target[i];
        s += d * d;
        lam[i] = (float)(w * d + wr * (double)r[i % ncell]);
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double z = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) z += red[q];
        partials[blockIdx.x] = z;
    }
}

__global__ void k_loss_final(const double* partials, const double* partials_r, int nb, long long n,
                             long long ncell, double rho_weight, double* loss) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double z = 0.0, zr = 0.0;
    for (int q = 0; q < nb; ++q) {
        z += partials[q];
        zr += partials_r[q];
    }
    *loss = z / (double)n + rho_weight * zr / (double)ncell;
}

int grid_n(long long n, int block) {
    return (int)std::max<long long>(1, std::min<long long>((n + block - 1) / block, 8192));
}

}  // namespace

#define LEARN_NV_LIST(X) X(3) X(5) X(9) X(13) X(17)

bool learn_nv_supported(int nv) {
    switch (nv) {
#define X(n) case n:
        LEARN_NV_LIST(X)
#undef X
        return true;
        default: return false;
    }
}

cudaError_t launch_rho_star(int nv, const LearnArgs& a, int k, cudaStream_t s) {
    const int grid = grid_n((long long)a.nx * a.ny, 256);
    switch (nv) {
#define X(n) case n: k_rho_star<n><<<grid, 256, 0, s>>>(a, k); return cudaGetLastError();
        LEARN_NV_LIST(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_mlp_f32(int nv, const LearnArgs& a, int k, cudaStream_t s) {
    const int grid = grid_n((long long)a.nx * a.ny * nv * nv, 128);
    switch (nv) {
#define X(n) case n: k_mlp_f32<n><<<grid, 128, 0, s>>>(a, k); return cudaGetLastError();
        LEARN_NV_LIST(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

// Persistent grid of k_step2d_corr<NV>: its resident blocks on sm_count SMs.  A larger grid
// would leave its last blocks to run their whole tile loops after the others finish.
template <int NV>
int corr_grid(int sm_count, int ntiles) {
    static int occ = 0;
    if (occ == 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step2d_corr<NV>, TW, 0) !=
            cudaSuccess)
            nb = 1;
        occ = nb > 0 ? nb : 1;
    }
    return std::max(1, std::min(ntiles, occ * sm_count));
}

cudaError_t launch_step2d_corr(int nv, int sm_count, const Step2DArgs& a, const float* G, int k,
                               cudaStream_t s) {
    switch (nv) {
#define X(n)                                                                                 \
    case n:                                                                                  \
        k_step2d_corr<n><<<corr_grid<n>(sm_count, a.ntiles), TW, 0, s>>>(a, G, k);           \
        return cudaGetLastError();
        LEARN_NV_LIST(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_diffuse_adjoint(int nv, const float* lam, float* out, float r, int nx, int ny,
                                   cudaStream_t s) {
    const int grid = grid_n((long long)nx * ny * nv * nv, 256);
    switch (nv) {
#define X(n) case n: k_diffuse_adjoint<n><<<grid, 256, 0, s>>>(lam, out, r, nx, ny); return cudaGetLastError();
        LEARN_NV_LIST(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_mlp_bwd(int nv, const LearnBwdArgs& b, int sm_count, cudaStream_t s) {
    const size_t sh = sizeof(float) * ((size_t)kLNParam + (size_t)(kVec + kPerThread) * kBT);
    switch (nv) {
#define X(n)                                                                                 \
    case n: {                                                                                \
        cudaError_t e = cudaFuncSetAttribute(k_mlp_bwd<n>,                                   \
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                             (int)sh);                                       \
        if (e != cudaSuccess) return e;                                                      \
        k_mlp_bwd<n><<<sm_count, kBT, sh, s>>>(b);                                           \
        return cudaGetLastError();                                                           \
    }
        LEARN_NV_LIST(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_gather_adjoint(int nv, const LearnBwdArgs& b, cudaStream_t s) {
    const int grid = grid_n((long long)b.fw.nx * b.fw.ny * nv * nv, 256);
    switch (nv) {
#define X(n) case n: k_gather_adjoint<n><<<grid, 256, 0, s>>>(b); return cudaGetLastError();
        LEARN_NV_LIST(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_restrict(const float* fine, int nvf, int nx, int ny, float* coarse,
                            cudaStream_t s) {
    const int nvc = (nvf - 1) / 4 + 1;
    k_restrict<<<grid_n((long long)nx * ny * nvc * nvc, 256), 256, 0, s>>>(fine, nvf, nx, ny,
                                                                           coarse);
    return cudaGetLastError();
}

cudaError_t launch_loss(const float* f, const float* target, int np, long long ncell,
                        double rho_weight, float* r, float* lam, double* partials, int nblocks,
                        double* loss, cudaStream_t s) {
    const long long n = ncell * np;
    k_rho_err<<<nblocks, 256, 0, s>>>(f, target, np, ncell, r, partials + nblocks);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_loss<<<nblocks, 256, 0, s>>>(f, target, n, ncell, r, rho_weight, lam, partials);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_loss_final<<<1, 32, 0, s>>>(partials, partials + nblocks, nblocks, n, ncell, rho_weight,
                                  loss);
    return cudaGetLastError();
}

}  // namespace lat

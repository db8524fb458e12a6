// Two FP32 lanes in one 64-bit register pair, and the packed IEEE arithmetic of sm_100 and
// later (add/sub/mul/fma.rn.f32x2: each lane rounded exactly as the scalar instruction), used by
// the packed two-lane sweeps of the 1D and 2D steps.
#pragma once

namespace lat {

typedef unsigned long long f2;  // lane 0 in the low word

__device__ __forceinline__ f2 pk(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float lo(f2 v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return a;
}
__device__ __forceinline__ float hi(f2 v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return b;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
// a - b lane by lane with scalar instructions (same rounding as sub2).  The packed 1D sweep
// uses it for the difference of consecutive diffusion fluxes: with sub.rn.f32x2 there, the
// kernels built by this toolchain differed from the scalar sweep by one unit in the last
// place in a few cells, while every packed instruction on its own rounds exactly.
__device__ __forceinline__ f2 sub2s(f2 a, f2 b) {
    return pk(__fsub_rn(lo(a), lo(b)), __fsub_rn(hi(a), hi(b)));
}
__device__ __forceinline__ f2 max0(f2 v) { return pk(fmaxf(lo(v), 0.f), fmaxf(hi(v), 0.f)); }
__device__ __forceinline__ f2 min0(f2 v) { return pk(fminf(lo(v), 0.f), fminf(hi(v), 0.f)); }
// Hides a value from the compiler's constant folding and hoisting.
__device__ __forceinline__ f2 opaque2(f2 v) {
    asm volatile("mov.b64 %0, %0;" : "+l"(v));
    return v;
}

}  // namespace lat

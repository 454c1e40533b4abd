// Double-float ("df64") arithmetic on the FP32 pipe.
//
// A df64 value is an unevaluated pair of floats hi + lo with |lo| <= ulp(hi)
// (hi = RN(x), lo = RN(x - hi)): 48 significant bits, relative representation
// error below 2^-48.  The Krylov basis of the solver is stored this way (same
// 8 bytes per element as a double) because on this GPU the FP64 pipe is far
// narrower than HBM: an FP64 Gram-Schmidt pass is bound by FP64 issue, the
// same pass in df64 by memory.
//
// Error-free transformations (Knuth's TwoSum, Dekker's Fast2Sum, the FMA form
// of TwoProd) use the _rn intrinsics so that the compiler never contracts a
// product and a sum into one FMA, which would break exactness.
//
// Vectors of n elements are planar: hi [n] floats, then lo [n] floats.
#pragma once

#include <cuda_runtime.h>

namespace rte {
namespace df {

// s + e = a + b exactly (TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
}

// p + e = (ah + al)(bh + bl) up to about 2^-47 relative: ah bh exactly
// (TwoProd by FMA), the cross terms rounded, al bl dropped.
__device__ __forceinline__ void mul(float ah, float al, float bh, float bl, float& p, float& e) {
    p = __fmul_rn(ah, bh);
    e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
}

// running sum S + C += p + e (S exact by TwoSum, the small parts summed in C)
__device__ __forceinline__ void acc(float& S, float& C, float p, float e) {
    float s, t;
    two_sum(S, p, s, t);
    S = s;
    C = __fadd_rn(C, __fadd_rn(t, e));
}

// renormalise S + C so that |C| <= ulp(S) / 2
__device__ __forceinline__ void renorm(float& S, float& C) {
    float s, t;
    two_sum(S, C, s, t);
    S = s;
    C = t;
}

// (ah + al) - (bh + bl), normalised
__device__ __forceinline__ void sub(float ah, float al, float bh, float bl, float& rh, float& rl) {
    float s, t;
    two_sum(ah, -bh, s, t);
    t = __fadd_rn(t, __fsub_rn(al, bl));
    two_sum(s, t, rh, rl);
}

// df64 -> double (exact: 48 significant bits fit in 53); two conversions and
// one FP64 add, for outputs written once per element
__device__ __forceinline__ double to_double(float h, float l) { return (double)h + (double)l; }

// double -> df64 (hi = RN(x), lo = RN(x - hi)); FP64 work, for inputs split
// once per element
__device__ __forceinline__ void from_double(double x, float& h, float& l) {
    h = __double2float_rn(x);
    l = __double2float_rn(x - (double)h);
}

// Packed pairs (two independent df64 lanes per register pair) with the
// .f32x2 instructions of sm_100+: one issue slot for two FP32 operations.
// Every instruction rounds to nearest and is never contracted.
using f2 = unsigned long long;      // two floats: x in the low word, y in the high word

__device__ __forceinline__ f2 pk(float x, float y) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
    return r;
}
__device__ __forceinline__ void upk(f2 a, float& x, float& y) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a));
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// S + C += (ah + al)(bh + bl) on both lanes, given nbh = -bh and nbl = -bl:
// p = ah bh and q = p - ah bh - al bh - ah bl (so p - q is the product to
// about 2^-47), then TwoSum(S, p) with its error and -q added to C.
__device__ __forceinline__ void mac2(f2& S, f2& C, f2 ah, f2 al, f2 nbh, f2 nbl, f2 bh) {
    const f2 p = mul2(ah, bh);
    f2 q = fma2(ah, nbh, p);
    q = fma2(al, nbh, q);
    q = fma2(ah, nbl, q);
    const f2 s = add2(S, p);
    const f2 bv = sub2(s, S);
    const f2 av = sub2(s, bv);
    const f2 t = add2(sub2(S, av), sub2(p, bv));
    C = add2(C, sub2(t, q));
    S = s;
}

// s + e = a + b exactly on both lanes (TwoSum)
__device__ __forceinline__ void two_sum2(f2 a, f2 b, f2& s, f2& e) {
    s = add2(a, b);
    const f2 bv = sub2(s, a);
    const f2 av = sub2(s, bv);
    e = add2(sub2(a, av), sub2(b, bv));
}

// S + C renormalised on both lanes (TwoSum)
__device__ __forceinline__ void renorm2(f2& S, f2& C) {
    const f2 s = add2(S, C);
    const f2 bv = sub2(s, S);
    const f2 av = sub2(s, bv);
    C = add2(sub2(S, av), sub2(C, bv));
    S = s;
}

}  // namespace df
}  // namespace rte

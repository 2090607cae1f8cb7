// dfloat.cuh -- double-float accumulation (an unevaluated sum hi + lo of two fp32 words,
// about 48 significant bits) for the vector work around the product when the vectors are
// fp32.  The fp64 pipe of this GPU issues at a small fraction of the fp32 rate, so sums
// of millions of fp32 products are carried in pairs of fp32 words and only the per-thread
// totals are converted to fp64 for the final (fixed-order) reductions.
//
// Building blocks (Knuth's TwoSum for the sum; the FMA gives the exact rounding error of
// a product, so a product of two fp32 numbers is held exactly as p + e).  The _rn
// intrinsics keep the compiler from contracting or reassociating these operations.
#pragma once

// (hi, lo) += p
__device__ __forceinline__ void df_add(float &hi, float &lo, float p) {
  const float t = __fadd_rn(hi, p);
  const float bb = __fsub_rn(t, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  hi = t;
  lo = __fadd_rn(lo, err);
}

// (hi, lo) += a * b, with the product's rounding error kept
__device__ __forceinline__ void df_add_prod(float &hi, float &lo, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  df_add(hi, lo, p);
  lo = __fadd_rn(lo, e);
}

// (hi, lo) -= (ch + cl) * u for a coefficient split into two fp32 words
__device__ __forceinline__ void df_sub_scaled(float &hi, float &lo, float ch, float cl, float u) {
  const float p = __fmul_rn(ch, u);
  const float e = __fmaf_rn(ch, u, -p);
  df_add(hi, lo, -p);
  lo = __fsub_rn(lo, __fmaf_rn(cl, u, e));
}

// a double as two fp32 words whose sum holds about 48 of its bits
__device__ __forceinline__ void df_split(double c, float &ch, float &cl) {
  ch = (float)c;
  cl = (float)(c - (double)ch);
}

__device__ __forceinline__ double df_value(float hi, float lo) { return (double)hi + (double)lo; }

// the fp32 word nearest to hi + lo
__device__ __forceinline__ float df_round(float hi, float lo) { return __fadd_rn(hi, lo); }

// the pair (hi, lo) as the fp32 word o nearest to it plus the fp32 word r nearest to the
// rest, and the square of o + r added to (nh, nl)
__device__ __forceinline__ void df_store(float hi, float lo, float &o, float &r) {
  o = __fadd_rn(hi, lo);
  r = __fadd_rn(__fsub_rn(hi, o), lo);
}

__device__ __forceinline__ void df_add_sq(float &nh, float &nl, float o, float r) {
  df_add_prod(nh, nl, o, o);
  df_add_prod(nh, nl, __fadd_rn(o, o), r);
}

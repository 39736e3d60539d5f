// Double-word ("float-float") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2, about 48 significant bits.  GB300 runs FP64 at 1/73 of
// the FP32 rate, and a warp-wide FP64 instruction holds a sub-partition's FP64
// unit for tens of cycles, so short dependent chains that need more than FP32
// (the Gram inverse of CP-ALS) run faster in double-word FP32 than in FP64.
//
// The building blocks are the error-free transformations of Knuth (TwoSum),
// Dekker (Fast2Sum) and the FMA product error, combined as in Joldes, Muller
// and Popescu, "Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic", ACM TOMS 44(2), 2017: the sum (AccurateDWPlusDW)
// has relative error at most 3u^2 + 13u^3 and the product (DWTimesDW2, with the
// lo * lo term) at most 5u^2, u = 2^-24.  The reciprocal
// is Newton's iteration from the hardware approximation, its residual 1 - y r
// formed with an FMA (Markstein 1990; Karp and Markstein 1997).  Every
// operation is an explicitly rounded intrinsic, so the compiler can neither
// contract nor reassociate them.
#pragma once

namespace rcp {

struct dwf {
  float hi, lo;
};

__device__ __forceinline__ dwf dw_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float t = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, t)), __fsub_rn(b, t));
  return {s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ dwf dw_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dwf dw_add(dwf x, dwf y) {
  const dwf s = dw_two_sum(x.hi, y.hi);
  const dwf t = dw_two_sum(x.lo, y.lo);
  const dwf v = dw_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return dw_fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}

__device__ __forceinline__ dwf dw_neg(dwf x) { return {-x.hi, -x.lo}; }

__device__ __forceinline__ dwf dw_mul(dwf x, dwf y) {
  const float ch = __fmul_rn(x.hi, y.hi);
  const float cl1 = __fmaf_rn(x.hi, y.hi, -ch);
  const float tl0 = __fmul_rn(x.lo, y.lo);
  const float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
  const float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
  return dw_fast_two_sum(ch, __fadd_rn(cl1, cl2));
}

// 1 / y for y > 0 normal: the hardware approximation (relative error about
// 2^-23), one FP32 Newton step, then one double-word Newton step whose residual
// 1 - y r is formed with FMAs.  Relative error a few u^2.
__device__ __forceinline__ dwf dw_rcp(dwf y) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y.hi));
  r = __fmaf_rn(r, __fmaf_rn(-y.hi, r, 1.0f), r);
  const float e = __fmaf_rn(-y.lo, r, __fmaf_rn(-y.hi, r, 1.0f));
  return dw_fast_two_sum(r, __fmul_rn(r, e));
}

// sqrt of a positive double word s: the FP32 square root r of s.hi and one
// correction (s - r^2) / (2 r) formed with the exact square of r (the
// Karp-Markstein form of a Newton step); relative error about 2^-46.
__device__ __forceinline__ dwf dw_sqrt(dwf s) {
  const float r = __fsqrt_rn(s.hi);
  const float r2 = __fmul_rn(r, r);
  const float r2l = __fmaf_rn(r, r, -r2);
  const float d = __fadd_rn(__fsub_rn(__fsub_rn(s.hi, r2), r2l), s.lo);
  float q;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(q) : "f"(r));
  q = __fmaf_rn(q, __fmaf_rn(-r, q, 1.0f), q);  // 1 / r, one Newton step
  return dw_fast_two_sum(r, __fmul_rn(d, __fmul_rn(0.5f, q)));
}

// Nearest double-word of a double inside the FP32 exponent range.
__device__ __forceinline__ dwf dw_from_double(double v) {
  const float h = __double2float_rn(v);
  return {h, __double2float_rn(v - (double)h)};
}

__device__ __forceinline__ double dw_to_double(dwf x) { return (double)x.hi + (double)x.lo; }

// Inverse of the R x R symmetric positive definite V (R <= 32) by
// Gauss-Jordan elimination without pivoting (every pivot of an SPD matrix is a
// Schur-complement diagonal, hence positive), in double-word arithmetic by all
// NT threads of the CTA.  The augmented matrix [V | I] lives twice, A0 and A1
// (32 x 64 float2 each, row pitch 64): step k reads one copy and writes the
// other, so a step costs one barrier.  At step k only columns k+1 .. R+k
// change, and the identity columns beyond them are still intact in both
// copies when their turn comes.  The element update is
//   a_ij <- a_ij - (a_ik a_kj) / a_kk,   a_kj <- a_kj / a_kk,
// with the product a_ik a_kj formed while the pivot's reciprocal is; each
// thread's (at most four) elements are computed without branches so that
// their dependent chains overlap.
//
// On entry A0[i][j], i, j < R, holds V in double-word form (the caller's
// choice of how to form it), visible to the CTA (a barrier after the writes).
// On success V^{-1} is written in FP64 to Zd (row pitch 32), which aliases the
// copy not holding the result, and true is returned.  false (returned by every
// thread at the same point) means that the trace of V is outside
// (1e-18, 1e18), that a pivot fell to R 2^-44 trace(V) or below, or that an
// element of the inverse is not finite.
template <int NT, int KE>
__device__ bool cta_gj_inverse_dw_k(int R, float2* A0, float2* A1, double** Zd) {
  const int tid = threadIdx.x, lane = tid & 31;
  for (int e = tid; e < R * R; e += NT) {
    const int i = e / R, c = e - i * R;
    const float2 v = make_float2(c == i ? 1.0f : 0.0f, 0.0f);
    A0[i * 64 + R + c] = v;
    A1[i * 64 + R + c] = v;
  }
  float tr = lane < R ? A0[lane * 64 + lane].x : 0.0f;
  for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
  int row[KE], col[KE];
  bool own[KE];
#pragma unroll
  for (int u = 0; u < KE; ++u) {
    const int e = tid + u * NT;
    own[u] = e < R * R;
    row[u] = own[u] ? e / R : 0;
    col[u] = own[u] ? e - (e / R) * R : 0;
  }
  __syncthreads();
  // |v_ij| <= trace for SPD V: with the trace inside (1e-18, 1e18) the FP32
  // products a_ik a_kj of the first steps stay finite and the pivot floor
  // below stays a normal number (rcp.approx.ftz flushes subnormals)
  if (!(tr > 1e-18f && tr < 1e18f)) return false;
  const float floor_ = (float)R * 5.684342e-14f * tr;
  const float2* cur = A0;
  float2* nxt = A1;
  for (int k = 0; k < R; ++k) {
    const float2 p = cur[k * 64 + k];
    if (!(p.x > floor_)) return false;
    dwf fc[KE], ac[KE], rk[KE];
#pragma unroll
    for (int u = 0; u < KE; ++u) {
      const int j = k + 1 + col[u];
      const float2 c = cur[k * 64 + j], f = cur[row[u] * 64 + k], a = cur[row[u] * 64 + j];
      rk[u].hi = c.x;
      rk[u].lo = c.y;
      ac[u].hi = a.x;
      ac[u].lo = a.y;
      fc[u] = dw_mul({f.x, f.y}, rk[u]);
    }
    const dwf pinv = dw_rcp({p.x, p.y});
#pragma unroll
    for (int u = 0; u < KE; ++u) {
      const bool pivrow = row[u] == k;
      const dwf q = dw_mul(pivrow ? rk[u] : fc[u], pinv);
      const dwf o = pivrow ? q : dw_add(ac[u], dw_neg(q));
      if (own[u]) nxt[row[u] * 64 + k + 1 + col[u]] = make_float2(o.hi, o.lo);
    }
    __syncthreads();
    float2* t = (float2*)cur;
    cur = nxt;
    nxt = t;
  }
  double* z = (double*)nxt;
  int bad = 0;
  for (int e = tid; e < R * R; e += NT) {
    const int i = e / R, c = e - i * R;
    const float2 v = cur[i * 64 + R + c];
    const double d = dw_to_double({v.x, v.y});
    bad |= !isfinite(d);
    z[i * 32 + c] = d;
  }
  // an element growth that overflowed FP32 on the way (a nearly singular V whose
  // pivots still passed the floor) sends the caller to its FP64 path
  if (__syncthreads_or(bad)) return false;
  *Zd = z;
  return true;
}

// Dispatch on the number of window elements per thread, ceil(R^2 / NT), so
// that each instantiation computes its elements without branches.
template <int NT>
__device__ bool cta_gj_inverse_dw(int R, float2* A0, float2* A1, double** Zd) {
  const int ke = (R * R + NT - 1) / NT;
  if (ke <= 1) return cta_gj_inverse_dw_k<NT, 1>(R, A0, A1, Zd);
  if (ke == 2) return cta_gj_inverse_dw_k<NT, 2>(R, A0, A1, Zd);
  if (ke == 3) return cta_gj_inverse_dw_k<NT, 3>(R, A0, A1, Zd);
  return cta_gj_inverse_dw_k<NT, 4>(R, A0, A1, Zd);
}

}  // namespace rcp

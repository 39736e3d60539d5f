// Warp-level dense linear algebra on small matrices in shared memory:
// Cholesky factorisation and triangular solves; and the FP64 reciprocal
// square root of the factorisations.
#pragma once

namespace rcp {

// 1 / sqrt(d) for a positive normal d: the FP32 hardware estimate and two
// Newton steps y <- y + y (1 - d y^2) / 2 in FP64 (each doubles the correct
// bits; the result is within a few ulp).  Outside the FP32 exponent range the
// FP64 library square root is used instead.
__device__ __forceinline__ double rsqrt64(double d) {
  // range test on the exponent bits (integer compares keep it off the FP64 pipe)
  const int ex = (__double2hiint(d) >> 20) & 0x7ff;
  if (ex < 1023 - 99 || ex > 1023 + 99) return 1.0 / sqrt(d);
  double y = (double)rsqrtf(__double2float_rn(d));
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double t = d * y;
    y = fma(0.5 * y, fma(-t, y, 1.0), y);
  }
  return y;
}


// One warp factors V = U^T U in place (upper triangle, row pitch R + 1),
// left-looking: row k of U is V[k, :] minus the dot products with the rows
// above, so every inner loop only reads shared memory (no read-after-write
// chains); false on a pivot <= floor.
template <typename T>
__device__ bool warp_chol(T* U, int R, T floor_) {
  const int lane = threadIdx.x & 31;
  const int P = R + 1;
  for (int k = 0; k < R; ++k) {
    T part = (T)0;
    for (int i = lane; i < k; i += 32) part += U[i * P + k] * U[i * P + k];
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    const T d = U[k * P + k] - part;
    if (!(d > floor_)) return false;  // warp-uniform: every lane holds the same d
    const T inv = (T)1 / sqrt(d);
    for (int j = k + 1 + lane; j < R; j += 32) {
      T s0 = U[k * P + j], s1 = (T)0;
      int i = 0;
      for (; i + 1 < k; i += 2) {
        s0 -= U[i * P + k] * U[i * P + j];
        s1 -= U[(i + 1) * P + k] * U[(i + 1) * P + j];
      }
      if (i < k) s0 -= U[i * P + k] * U[i * P + j];
      U[k * P + j] = (s0 + s1) * inv;
    }
    if (lane == 0) U[k * P + k] = d * inv;
    __syncwarp();
  }
  return true;
}

// Solve U^T U x = b in place for one right-hand side held two entries per
// lane (entry c in lane c % 32, slot c / 32): column-oriented substitutions,
// one broadcast and one fused multiply-add per step.
template <typename T>
__device__ void warp_solve(const T* U, const T* invd, int R, double (&b)[2]) {
  const int lane = threadIdx.x & 31;
  const int P = R + 1;
  T y[2] = {(T)b[0], (T)b[1]};
  for (int k = 0; k < R; ++k) {  // U^T y = b
    const int owner = k & 31, hk = k >> 5;
    const T yk = __shfl_sync(0xffffffffu, (hk ? y[1] : y[0]) * invd[k], owner);
    if (lane == owner) {
      if (hk) y[1] = yk; else y[0] = yk;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = lane + 32 * h;
      if (j > k && j < R) y[h] -= U[k * P + j] * yk;
    }
  }
  for (int k = R - 1; k >= 0; --k) {  // U x = y
    const int owner = k & 31, hk = k >> 5;
    const T xk = __shfl_sync(0xffffffffu, (hk ? y[1] : y[0]) * invd[k], owner);
    if (lane == owner) {
      if (hk) y[1] = xk; else y[0] = xk;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = lane + 32 * h;
      if (i < k) y[h] -= U[i * P + k] * xk;
    }
  }
  b[0] = (double)y[0];
  b[1] = (double)y[1];
}

}  // namespace rcp

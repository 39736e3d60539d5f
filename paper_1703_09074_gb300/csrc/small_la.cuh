// Dense linear algebra on small matrices in shared memory: warp-level
// Cholesky factorisation and triangular solves, the CTA-wide Cholesky with
// R^{-1} of CholeskyQR (FP32 or FP64), and the FP64 reciprocal square root.
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

__device__ __forceinline__ float rsqrt_t(float d) { return rsqrtf(d); }
__device__ __forceinline__ double rsqrt_t(double d) { return rsqrt64(d); }

// d > floor_ >= 0 and finite, as integer compares (positive IEEE numbers order
// like their bit patterns), which keeps the test off the FP64 pipe
__device__ __forceinline__ bool pivot_ok(double d, double floor_) {
  const long long db = __double_as_longlong(d);
  return db > __double_as_longlong(floor_) && db > 0 && db < 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool pivot_ok(float d, float floor_) {
  const int db = __float_as_int(d);
  return db > __float_as_int(floor_) && db > 0 && db < 0x7f800000;
}

// Cholesky G = R^T R of the SPD matrix in the upper triangle of S (l x l, with
// the strict lower triangle zero) by one CTA, together with R^{-1}.
// Elimination on [G | I] by rows: step k scales row k by 1 / sqrt(pivot)
// (giving row k of R, and of R^{-T} on the right) and subtracts R[k][i] times
// it from every later row i, so the left part ends as R and the right part as
// R^{-T} (the row operations E satisfy E G = R, hence E = R^{-T}).  S keeps
// the Schur complement in its upper triangle and receives R^{-T} in its strict
// lower triangle (diagonal in tdiag).  The pivot chain (update of row k+1, its
// reciprocal square root, the scaling) runs on warp 0 one step ahead, while
// warps 1-3 and 5-7 (warp 4 shares warp 0's sub-partition, whose FP64 unit
// issues one warp instruction per 64 cycles) update rows k+2.. of step k: one
// barrier per step.  Returns false, uniformly, when a pivot is not above
// floor_ (>= 0); 256 threads.
template <typename T>
__device__ bool chol_elim(T (*S)[kMaxL + 1], T* tdiag, T (*rowb)[kMaxL], T (*tb)[kMaxL], int l,
                          T floor_, int* fail_sh) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // update warps 1-3, 5-7 as uw = 0..5: column lane (l <= 32) or lane + 32 (uw & 1),
  // rows k+2+r0, k+2+r0+rstep, ...
  const int uw = warp == 0 || warp == 4 ? -1 : (warp < 4 ? warp - 1 : warp - 2);
  const int jcol = l <= 32 ? lane : lane + 32 * (uw & 1);
  const int r0 = l <= 32 ? uw : uw >> 1, rstep = l <= 32 ? 6 : 3;
  if (tid == 0) *fail_sh = 0;
  __syncthreads();
  if (warp == 0) {
    const T d = S[0][0];
    const bool good = pivot_ok(d, floor_);
    const T rs = good ? rsqrt_t(d) : T(0);
    for (int j = lane; j < l; j += 32) rowb[0][j] = S[0][j] * rs;
    if (lane == 0) {
      tb[0][0] = rs;
      tdiag[0] = rs;
      if (!good) *fail_sh = 1;
    }
  }
  __syncthreads();
  bool ok = *fail_sh == 0;
  for (int k = 0; ok && k + 1 < l; ++k) {
    const T* rk = rowb[k & 1];
    const T* tk = tb[k & 1];
    if (warp == 0) {
      // row k+1: its update by row k, the pivot, the scaling
      const int i = k + 1;
      const T f = rk[i];
      T v[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = lane + 32 * h;
        v[h] = T(0);
        if (j < l) v[h] = fma(-f, j >= i ? rk[j] : tk[j], S[i][j]);
      }
      const T d = __shfl_sync(0xffffffffu, (i >> 5) ? v[1] : v[0], i & 31);
      const bool good = pivot_ok(d, floor_);
      const T rs = good ? rsqrt_t(d) : T(0);
      T* rn = rowb[(k + 1) & 1];
      T* tn = tb[(k + 1) & 1];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = lane + 32 * h;
        if (j < l) {
          const T w = v[h] * rs;
          if (j > i) {
            rn[j] = w;
          } else if (j < i) {
            tn[j] = w;
            S[i][j] = w;
          }
        }
      }
      if (lane == 0) {
        tn[i] = rs;
        tdiag[i] = rs;
        if (!good) *fail_sh = 1;
      }
    } else if (uw >= 0 && jcol < l) {
      // rows k+2..: S[i][j] -= R[k][i] R[k][j] (j >= i), T[i][j] -= R[k][i] T[k][j] (j <= k)
      const int j = jcol;
      for (int i = k + 2 + r0; i < l; i += rstep) {
        if (j >= i) S[i][j] = fma(-rk[i], rk[j], S[i][j]);
        else if (j <= k) S[i][j] = fma(-rk[i], tk[j], S[i][j]);
      }
    }
    __syncthreads();
    ok = *fail_sh == 0;
  }
  return ok;
}

// R^{-1} = (R^{-T})^T to Rinv (l x l column-major): (R^{-1})[i][c] = T[c][i], i <= c
template <typename T>
__device__ void write_rinv(const T (*S)[kMaxL + 1], const T* tdiag, int l, double* Rinv) {
  for (int q = threadIdx.x; q < l * l; q += blockDim.x) {
    const int i = q % l, c = q / l;
    Rinv[q] = i < c ? (double)S[c][i] : (i == c ? (double)tdiag[c] : 0.0);
  }
}

}  // namespace rcp

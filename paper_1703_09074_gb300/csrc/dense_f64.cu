// Small dense FP64 linear algebra on the device: deterministic split reductions,
// the Gram matrix of a tall-skinny Y, Cholesky with the shifted fallback, and
// the triangular right-multiplication Q = Y R^{-1}.
//
// Orthonormalisation of each sketch (Algorithm 1 step 12, and the normalised
// power iterations of steps 7-11) uses CholeskyQR2: G = Y^T Y = R^T R,
// Q = Y R^{-1}, repeated once.  When the first Cholesky meets a pivot below the
// shift of shifted CholeskyQR3 (Fukaya, Kannan, Nakatsukasa, Zhang & Yamamoto,
// SIAM J. Sci. Comput. 2020: s = 11 (m n + n (n + 1)) u |Y|^2) the first round
// factors G + s I instead and a third round runs.  Every R has a positive
// diagonal, so Q equals the thin QR factor with positive diag(R).
#include <math.h>

#include <algorithm>

#include "rcp_internal.cuh"
#include "small_la.cuh"

namespace rcp {
namespace {

constexpr int kRedChunks = 16;

__global__ void k_reduce(const double* __restrict__ part, int64_t nsplit, int64_t n,
                         int64_t s0, int64_t s1_stride, double* __restrict__ out) {
  // out[chunk * n + e] = sum over s in this chunk of part[s * n + e], fixed order
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int64_t c = blockIdx.y;
  const int64_t sa = c * s1_stride, sb = min(nsplit, sa + s1_stride);
  double acc = 0.0;
  for (int64_t s = sa; s < sb; ++s) acc += part[s * n + e];
  out[c * n + e] = acc;
  (void)s0;
}

__device__ double block_sum(double v, double* red) {
  const int tid = threadIdx.x;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (tid == 0) {
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) s += red[w];
  }
  __syncthreads();
  return s;  // valid in thread 0
}

// One CTA per packed upper-triangular pair (c1 <= c2): G = Y^T Y.
__global__ void k_gram_pairs(const double* __restrict__ Y, int64_t I, int l,
                             double* __restrict__ Gp) {
  __shared__ double red[32];
  const int p = blockIdx.x;
  int c1 = 0, rem = p;
  while (rem >= l - c1) { rem -= l - c1; ++c1; }
  const int c2 = c1 + rem;
  const double* y1 = Y + I * c1;
  const double* y2 = Y + I * c2;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < I; i += blockDim.x) acc = fma(y1[i], y2[i], acc);
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) Gp[p] = s;
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

// The FP64 factorisation of one CholeskyQR round (chol_elim in FP64).
// shift_rows: the row count m entering the shifted-CholeskyQR3 shift; 0 forbids the shift.
// round < 0: unconditional; round == 2: only when an earlier round was shifted.
// after32 != 0: runs only when the FP32 attempt of the same round failed.
__global__ void __launch_bounds__(256) k_chol(const double* __restrict__ Gp, int l,
                                              double* __restrict__ Rinv, DevState* st,
                                              double shift_rows, int round, int als_mode,
                                              int after32) {
  __shared__ double S[kMaxL][kMaxL + 1];
  __shared__ double tdiag[kMaxL];
  __shared__ double rowb[2][kMaxL];
  __shared__ double tb[2][kMaxL];
  __shared__ double red[32];
  __shared__ int bad_sh, fail_sh;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (after32 && !st->chol32_fail) return;
  if (round == 2 && !st->extra_round) return;
  if (round == 0 && tid == 0) st->extra_round = 0;
  const int np = l * (l + 1) / 2;

  // trace and finiteness, all threads
  if (tid == 0) bad_sh = 0;
  __syncthreads();
  double tr = 0.0;
  for (int p = tid; p < np; p += nt) {
    const double g = Gp[p];
    if (!isfinite(g)) bad_sh = 1;
  }
  for (int i = tid; i < l; i += nt) tr += Gp[i * l - i * (i - 1) / 2];
  tr = block_sum(tr, red);
  if (tid == 0) red[31] = tr;
  __syncthreads();
  tr = red[31];
  if (bad_sh) {
    if (tid == 0) set_status(st, RCP_ENAN);
    return;
  }
  const double u = 1.1102230246251565e-16;
  const double shift = 11.0 * (shift_rows * l + (double)l * (l + 1)) * u * tr;

  bool ok = false;
  for (int attempt = 0; attempt < 2 && !ok; ++attempt) {
    for (int e = tid; e < l * l; e += nt) {
      const int i = e / l, j = e - (e / l) * l;  // packed upper triangle: row i starts at i l - i (i - 1) / 2
      if (j >= i) S[i][j] = Gp[i * l - i * (i - 1) / 2 + (j - i)] + ((attempt == 1 && j == i) ? shift : 0.0);
      else S[i][j] = 0.0;
    }
    const double floor_ = (attempt == 0 && shift_rows > 0.0) ? shift : 0.0;
    ok = chol_elim<double>(S, tdiag, rowb, tb, l, floor_, &fail_sh);
    if (!ok && attempt == 0 && shift_rows > 0.0) {
      if (tid == 0) {
        atomicOr(&st->info, als_mode ? RCP_INFO_ALS_REGULARISED : RCP_INFO_SHIFTED_QR);
        if (round == 0) st->extra_round = 1;
      }
      __syncthreads();
      continue;
    }
    if (!ok) {
      if (tid == 0) set_status(st, RCP_ESINGULAR);
      return;
    }
  }
  write_rinv<double>(S, tdiag, l, Rinv);
}

// The same factorisation in FP32 for the rounds that tolerate it: the
// normalisations inside the power iterations (any well-conditioned basis of
// the span serves) and the first round of each final CholeskyQR2 (whose second
// round, in FP64, restores orthonormality to FP64 rounding; Q is the unique
// qr+ factor whatever R the first round used).  A pivot at or below
// 64 l u_32 trace(G), or a non-finite entry, sets chol32_fail and the FP64
// kernel that follows redoes the round (with its shifted fallback) -- except
// for a normalisation inside the power iterations (span_only != 0), which
// instead factors G + s I with s = 64 l u_32 trace(G): every pivot then stays
// above FP32 rounding, Y R^{-1} spans the same space as Y, and its condition
// number is at most about sqrt(trace(G) / s), which is all the next product
// needs (the final CholeskyQR2 of the mode, in FP64, orthonormalises).
__global__ void __launch_bounds__(256) k_chol32(const double* __restrict__ Gp, int l,
                                                double* __restrict__ Rinv, DevState* st,
                                                int round, int span_only) {
  __shared__ float S[kMaxL][kMaxL + 1];
  __shared__ float tdiag[kMaxL];
  __shared__ float rowb[2][kMaxL];
  __shared__ float tb[2][kMaxL];
  __shared__ double red[32];
  __shared__ int bad_sh, fail_sh;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (round == 0 && tid == 0) st->extra_round = 0;
  if (tid == 0) bad_sh = 0;
  __syncthreads();
  double tr = 0.0;
  for (int e = tid; e < l * l; e += nt) {
    const int i = e / l, j = e - (e / l) * l;
    if (j >= i) {
      const double g = Gp[i * l - i * (i - 1) / 2 + (j - i)];
      if (!isfinite(g)) bad_sh = 1;
      if (j == i) tr += g;
      S[i][j] = (float)g;
    } else {
      S[i][j] = 0.0f;
    }
  }
  tr = block_sum(tr, red);
  if (tid == 0) red[31] = tr;
  __syncthreads();
  const float floor_ = 64.0f * (float)l * 5.9604645e-08f * (float)red[31];
  bool ok = !bad_sh && chol_elim<float>(S, tdiag, rowb, tb, l, floor_, &fail_sh);
  if (!ok && !bad_sh && span_only) {
    __syncthreads();
    for (int e = tid; e < l * l; e += nt) {
      const int i = e / l, j = e - (e / l) * l;
      S[i][j] = j >= i ? (float)Gp[i * l - i * (i - 1) / 2 + (j - i)] + (j == i ? floor_ : 0.0f) : 0.0f;
    }
    ok = chol_elim<float>(S, tdiag, rowb, tb, l, 0.0f, &fail_sh);
  }
  if (!ok) {
    if (tid == 0) st->chol32_fail = 1;
    return;
  }
  write_rinv<float>(S, tdiag, l, Rinv);
  if (tid == 0) st->chol32_fail = 0;
}

// out[i, c] = sum_{k <= c} Y[i, k] Rinv[k, c] (in place allowed).  A CTA owns
// kTrRows rows: it stages them in shared memory, then one thread per (row,
// column) forms the product, so the FP64 work spreads over I * l / 256 CTAs.
constexpr int kTrRows = 8;
template <int LMAX>
__global__ void __launch_bounds__(256) k_trmm(const double* Y, int64_t I, int l,
                                              const double* __restrict__ Rinv, double* out,
                                              const DevState* st, int only_if_extra) {
  __shared__ double Rs[LMAX * LMAX];
  __shared__ double Ys[kTrRows][LMAX];
  if (only_if_extra && !st->extra_round) return;
  if (st->status) return;
  const int tid = threadIdx.x;
  for (int q = tid; q < l * l; q += blockDim.x) Rs[(q % l) + LMAX * (q / l)] = Rinv[q];
  const int64_t i0 = (int64_t)blockIdx.x * kTrRows;
  for (int q = tid; q < kTrRows * l; q += blockDim.x) {
    const int r = q % kTrRows, k = q / kTrRows;
    const int64_t i = i0 + r;
    Ys[r][k] = (i < I) ? Y[i + I * k] : 0.0;
  }
  __syncthreads();
  for (int q = tid; q < kTrRows * l; q += blockDim.x) {
    const int r = q % kTrRows, c = q / kTrRows;
    const int64_t i = i0 + r;
    if (i >= I) continue;
    double acc = 0.0;
    for (int k = 0; k <= c; ++k) acc = fma(Ys[r][k], Rs[k + LMAX * c], acc);
    out[i + I * c] = acc;
  }
}

__global__ void k_sum_to(const double* __restrict__ x, int64_t n, double* dst) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += x[i];
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) *dst = s;
}

__global__ void k_sumsq_part(const double* __restrict__ x, int64_t n, double* __restrict__ part) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc = fma(x[i], x[i], acc);
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

template <typename T>
__global__ void k_to_f64(const T* __restrict__ src, int64_t n, double* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}

}  // namespace

cudaError_t launch_reduce(const double* part, int64_t nsplit, int64_t n, double* out, double* tmp,
                          int64_t tmp_elems, cudaStream_t s) {
  const int threads = 256;
  const unsigned gx = (unsigned)((n + threads - 1) / threads);
  if (nsplit > 2 * kRedChunks && tmp && tmp_elems >= kRedChunks * n) {
    const int64_t stride = (nsplit + kRedChunks - 1) / kRedChunks;
    count_launches(2);
    k_reduce<<<dim3(gx, kRedChunks), threads, 0, s>>>(part, nsplit, n, 0, stride, tmp);
    k_reduce<<<dim3(gx, 1), threads, 0, s>>>(tmp, kRedChunks, n, 0, kRedChunks, out);
  } else {
    count_launches(1);
    k_reduce<<<dim3(gx, 1), threads, 0, s>>>(part, nsplit, n, 0, nsplit, out);
  }
  return cudaGetLastError();
}

cudaError_t launch_gram(const double* Y, int64_t I, int l, double* Gp, cudaStream_t s) {
  count_launches(1);
  k_gram_pairs<<<l * (l + 1) / 2, 128, 0, s>>>(Y, I, l, Gp);
  return cudaGetLastError();
}

cudaError_t launch_chol(const double* Gp, int l, double* Rinv, DevState* st, double shift_rows,
                        int round, int als_mode, cudaStream_t s) {
  count_launches(1);
  k_chol<<<1, 256, 0, s>>>(Gp, l, Rinv, st, shift_rows, round, als_mode, 0);
  return cudaGetLastError();
}

cudaError_t launch_trmm(const double* Y, int64_t I, int l, const double* Rinv, double* out,
                        const DevState* st, int only_if_extra, cudaStream_t s) {
  const int threads = 256;
  const unsigned grid = (unsigned)((I + kTrRows - 1) / kTrRows);
  count_launches(1);
  if (l <= 16) k_trmm<16><<<grid, threads, 0, s>>>(Y, I, l, Rinv, out, st, only_if_extra);
  else if (l <= 32) k_trmm<32><<<grid, threads, 0, s>>>(Y, I, l, Rinv, out, st, only_if_extra);
  else if (l <= 48) k_trmm<48><<<grid, threads, 0, s>>>(Y, I, l, Rinv, out, st, only_if_extra);
  else k_trmm<64><<<grid, threads, 0, s>>>(Y, I, l, Rinv, out, st, only_if_extra);
  return cudaGetLastError();
}

cudaError_t launch_cholqr(double* Y, int64_t I, int l, double* Gp, double* Rinv, DevState* st,
                          cudaStream_t s, bool final_qr) {
  // round 0 (shift allowed), round 1, round 2 (only after a shifted round); in place on Y.
  // A normalisation inside the power iterations needs a well-conditioned basis
  // of the same span, not an orthonormal one: one round (CholeskyQR) serves it,
  // and the final QR of each mode (CholeskyQR2) removes the difference.
  // Round 0 is factored in FP32 first (FP64 only when that fails); the later
  // rounds of the final QR in FP64.
  const int rounds = final_qr ? 3 : 1;
  for (int round = 0; round < rounds; ++round) {
    cudaError_t e = launch_gram(Y, I, l, Gp, s);
    if (e != cudaSuccess) return e;
    if (round == 0 && l <= kMaxL) {
      count_launches(2);
      k_chol32<<<1, 256, 0, s>>>(Gp, l, Rinv, st, round, final_qr ? 0 : 1);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      k_chol<<<1, 256, 0, s>>>(Gp, l, Rinv, st, (double)I, round, 0, 1);
      e = cudaGetLastError();
    } else {
      e = launch_chol(Gp, l, Rinv, st, round == 0 ? (double)I : 0.0, round, 0, s);
    }
    if (e != cudaSuccess) return e;
    e = launch_trmm(Y, I, l, Rinv, Y, st, round == 2, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_sum_to(const double* part, int64_t n, double* dst, cudaStream_t s) {
  count_launches(1);
  k_sum_to<<<1, 256, 0, s>>>(part, n, dst);
  return cudaGetLastError();
}

cudaError_t launch_sumsq(const double* x, int64_t n, double* part, int nblocks, double* dst,
                         cudaStream_t s) {
  count_launches(2);
  k_sumsq_part<<<nblocks, 256, 0, s>>>(x, n, part);
  k_sum_to<<<1, 256, 0, s>>>(part, nblocks, dst);
  return cudaGetLastError();
}

cudaError_t launch_to_f64(const void* src, int src_dtype, int64_t n, double* dst, cudaStream_t s) {
  const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
  count_launches(1);
  if (src_dtype == RCP_DTYPE_F32)
    k_to_f64<float><<<grid, 256, 0, s>>>((const float*)src, n, dst);
  else
    k_to_f64<double><<<grid, 256, 0, s>>>((const double*)src, n, dst);
  return cudaGetLastError();
}

}  // namespace rcp

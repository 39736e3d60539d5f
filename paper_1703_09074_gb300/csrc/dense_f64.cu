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

// The FP64 factorisation of one CholeskyQR round (chol_elim in FP64).
// shift_rows: the row count m entering the shifted-CholeskyQR3 shift; 0 forbids the shift.
// round < 0: unconditional; round == 2: only when an earlier round was shifted.
// after32 != 0: runs only when the FP32 attempt of the same round failed.
// no_shift != 0: a Gram that would need the shift (a pivot at or below it)
// records RCP_ESINGULAR instead of being factored with it.
__global__ void __launch_bounds__(256) k_chol(const double* __restrict__ Gp, int l,
                                              double* __restrict__ Rinv, DevState* st,
                                              double shift_rows, int round, int als_mode,
                                              int after32, int no_shift) {
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
    if (!ok && attempt == 0 && shift_rows > 0.0 && !no_shift) {
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

template <typename T>
__global__ void k_sumsq_part(const T* __restrict__ x, int64_t n, double* __restrict__ part) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)x[i];
    acc = fma(v, v, acc);
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// Q = the I x I identity (column-major): the basis of a mode left uncompressed.
__global__ void k_identity(double* __restrict__ Q, int64_t I) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < I * I;
       e += (int64_t)gridDim.x * blockDim.x)
    Q[e] = (e % (I + 1)) == 0 ? 1.0 : 0.0;
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
                        int round, int als_mode, cudaStream_t s, bool no_shift) {
  count_launches(1);
  k_chol<<<1, 256, 0, s>>>(Gp, l, Rinv, st, shift_rows, round, als_mode, 0, no_shift ? 1 : 0);
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
                          cudaStream_t s, bool final_qr, bool no_shift) {
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
      k_chol32<<<1, 256, 0, s>>>(Gp, l, Rinv, st, round, (final_qr || no_shift) ? 0 : 1);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      k_chol<<<1, 256, 0, s>>>(Gp, l, Rinv, st, (double)I, round, 0, 1, no_shift ? 1 : 0);
      e = cudaGetLastError();
    } else {
      e = launch_chol(Gp, l, Rinv, st, round == 0 ? (double)I : 0.0, round, 0, s, no_shift);
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
  k_sumsq_part<double><<<nblocks, 256, 0, s>>>(x, n, part);
  k_sum_to<<<1, 256, 0, s>>>(part, nblocks, dst);
  return cudaGetLastError();
}

cudaError_t launch_sumsq_any(const void* x, int dtype, int64_t n, double* part, int nblocks,
                             double* dst, cudaStream_t s) {
  count_launches(2);
  if (dtype == RCP_DTYPE_F32) k_sumsq_part<float><<<nblocks, 256, 0, s>>>((const float*)x, n, part);
  else k_sumsq_part<double><<<nblocks, 256, 0, s>>>((const double*)x, n, part);
  k_sum_to<<<1, 256, 0, s>>>(part, nblocks, dst);
  return cudaGetLastError();
}

cudaError_t launch_identity(double* Q, int64_t I, cudaStream_t s) {
  count_launches(1);
  const unsigned grid = (unsigned)std::min<int64_t>((I * I + 255) / 256, 1024);
  k_identity<<<grid, 256, 0, s>>>(Q, I);
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

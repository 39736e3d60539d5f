// CP-ALS on the compressed tensor B (Algorithm 2 steps 3-11) and the recovery
// of the full factors (Algorithm 2 steps 12-13, Eq. qbs), FP64.
//
// One ALS sweep updates modes n = 1..N in order:
//   M   = B_(n) (KR of Atilde_m, m != n)        -- MTTKRP, split row sweep (sweeps_f64.cu)
//   V   = Hadamard product of Atilde_m^T Atilde_m, m != n
//   X   = M V^{-1}                              -- Definition 2 (Khatri-Rao pseudo-inverse);
//                                                  V is SPD, solved through its Cholesky factor
//   Atilde_n = X / colnorm(X); lambda = colnorm(X) for n = N (steps 5, 7, 9, 10)
// after which the fit of Section 3.3 is evaluated without forming Bhat:
//   |Bhat|^2 = lambda^T (Hadamard product of all Grams) lambda,
//   <Bhat, B> = sum_r lambda_r sum_i M_N[i, r] Atilde_N[i, r],
//   rho = 1 - (|B|^2 + |Bhat|^2 - 2 <Bhat, B>) / |B|^2,
// and ALS stops once |rho_j - rho_{j-1}| < tol (rho_0 = 0) or j = max_iters.
// Every ALS kernel returns at once after the stop, so the host can enqueue
// max_iters sweeps without reading anything back.
#include <math.h>

#include "rcp_internal.cuh"

namespace rcp {
namespace {

struct AlsArgs {
  int N, n0, R, ln;
  int nsplit;
  const double* part;
  double* At[kMaxN];
  double* Gm[kMaxN];
  int dims[kMaxN];
  double* lam;
  double* M;
  DevState* st;
  double tol;
  int max_iters;
};

__global__ void k_als_init(AlsArgs a, uint64_t seed, int user_init) {
  // seeded N(0,1) factors for modes 2..N (row-major l_m x R in the stream,
  // stored column-major), then their Grams; state reset.
  const int tid = threadIdx.x, nt = blockDim.x;
  const int R = a.R;
  for (int m = 1; m < a.N; ++m) {
    const int lm = a.dims[m];
    if (!user_init) {
      for (int e = tid; e < lm * R; e += nt) {
        const int i = e / R, r = e - i * R;
        const double2 z = normal_pair_f64(seed, (uint32_t)(m + 1), kPurposeAlsInit, (uint64_t)(e >> 1));
        a.At[m][i + lm * r] = (e & 1) ? z.y : z.x;
      }
    }
  }
  __syncthreads();
  for (int m = 1; m < a.N; ++m) {
    const int lm = a.dims[m];
    for (int e = tid; e < R * R; e += nt) {
      const int r = e % R, s = e / R;
      double acc = 0.0;
      for (int i = 0; i < lm; ++i) acc = fma(a.At[m][i + lm * r], a.At[m][i + lm * s], acc);
      a.Gm[m][e] = acc;
    }
  }
  if (tid == 0) {
    a.st->als_done = 0;
    a.st->als_iters = 0;
    a.st->fit = 0.0;
    a.st->fit_prev = 0.0;
    a.st->ip = 0.0;
  }
}

__global__ void k_als_update(AlsArgs a) {
  extern __shared__ double sm[];
  DevState* st = a.st;
  if (st->als_done || st->status) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int R = a.R, ln = a.ln, n0 = a.n0;
  double* Ms = sm;                 // ln x R (col-major)
  double* Xs = Ms + ln * R;        // ln x R
  double* V = Xs + ln * R;         // R x (R + 1): Cholesky factor in the upper triangle
  double* Ui = V + R * (R + 1);    // R x R: inverse of the factor, then V^{-1}
  double* nu = Ui + R * R;         // R
  __shared__ int fail;
  __shared__ double scal[4];

  // 1. M: fixed-order reduction of the MTTKRP split partials
  const int64_t n = (int64_t)ln * R;
  for (int e = tid; e < n; e += nt) {
    double acc = 0.0;
    for (int s = 0; s < a.nsplit; ++s) acc += a.part[(int64_t)s * n + e];
    Ms[e] = acc;
  }
  // 2. V = Hadamard product of the other modes' Grams
  for (int e = tid; e < R * R; e += nt) {
    const int r = e % R, c = e / R;
    double v = 1.0;
    for (int m = 0; m < a.N; ++m)
      if (m != n0) v *= a.Gm[m][e];
    V[r * (R + 1) + c] = v;
  }
  __syncthreads();
  // 3. Cholesky V = U^T U (upper U in place); on breakdown shift by R u trace(V)
  for (int attempt = 0; attempt < 2; ++attempt) {
    if (tid == 0) {
      fail = 0;
      double tr = 0.0;
      for (int c = 0; c < R; ++c) tr += V[c * (R + 1) + c];
      scal[0] = (double)R * 1.1102230246251565e-16 * tr;
      if (!isfinite(tr)) fail = 2;
    }
    __syncthreads();
    if (fail == 2) {
      if (tid == 0) set_status(st, RCP_ENAN);
      return;
    }
    if (attempt == 1) {
      // rebuild V and shift its diagonal
      for (int e = tid; e < R * R; e += nt) {
        const int r = e % R, c = e / R;
        double v = 1.0;
        for (int m = 0; m < a.N; ++m)
          if (m != n0) v *= a.Gm[m][e];
        V[r * (R + 1) + c] = v + (r == c ? scal[0] : 0.0);
      }
      __syncthreads();
    }
    for (int k = 0; k < R; ++k) {
      if (tid == 0) {
        const double d = V[k * (R + 1) + k];
        if (!(d > (attempt == 0 ? scal[0] : 0.0))) fail = 1;
        V[k * (R + 1) + k] = d > 0.0 ? sqrt(d) : 1.0;
      }
      __syncthreads();
      if (fail) break;
      const double ukk = V[k * (R + 1) + k];
      for (int j = k + 1 + tid; j < R; j += nt) V[k * (R + 1) + j] /= ukk;
      __syncthreads();
      const int m = R - k - 1;
      for (int q = tid; q < m * m; q += nt) {
        const int i = k + 1 + q / m, j = k + 1 + q % m;
        if (j >= i) V[i * (R + 1) + j] -= V[k * (R + 1) + i] * V[k * (R + 1) + j];
      }
      __syncthreads();
    }
    if (!fail) break;
    if (attempt == 0) {
      if (tid == 0) atomicOr(&st->info, RCP_INFO_ALS_REGULARISED);
      __syncthreads();
      continue;
    }
    if (tid == 0) set_status(st, RCP_ESINGULAR);
    return;
  }
  // 4. U^{-1} (upper) by back substitution, thread per column; then V^{-1} = U^{-1} U^{-T}
  for (int c = tid; c < R; c += nt) {
    for (int i = R - 1; i >= 0; --i) {
      double v = 0.0;
      if (i <= c) {
        v = (i == c) ? 1.0 : 0.0;
        for (int k = i + 1; k <= c; ++k) v -= V[i * (R + 1) + k] * Ui[k + R * c];
        v /= V[i * (R + 1) + i];
      }
      Ui[i + R * c] = v;
    }
  }
  __syncthreads();
  // V^{-1}[r, c] = sum_k Ui[r, k] Ui[c, k], k >= max(r, c); written over the factor's storage
  for (int e = tid; e < R * R; e += nt) {
    const int r = e % R, c = e / R;
    double acc = 0.0;
    for (int k = (r > c ? r : c); k < R; ++k) acc = fma(Ui[r + R * k], Ui[c + R * k], acc);
    V[r * (R + 1) + c] = acc;
  }
  __syncthreads();
  // X = M V^{-1}
  for (int e = tid; e < n; e += nt) {
    const int i = e % ln, r = e / ln;
    double acc = 0.0;
    for (int k = 0; k < R; ++k) acc = fma(Ms[i + ln * k], V[k * (R + 1) + r], acc);
    Xs[e] = acc;
  }
  __syncthreads();
  // 5. column norms
  for (int r = tid; r < R; r += nt) {
    double acc = 0.0;
    for (int i = 0; i < ln; ++i) acc = fma(Xs[i + ln * r], Xs[i + ln * r], acc);
    nu[r] = sqrt(acc);
  }
  __syncthreads();
  // 6. normalise (a zero column stays zero)
  for (int e = tid; e < n; e += nt) {
    const int r = e / ln;
    a.At[n0][e] = nu[r] > 0.0 ? Xs[e] / nu[r] : 0.0;
  }
  __syncthreads();
  // 7. Gram of the normalised factor
  for (int e = tid; e < R * R; e += nt) {
    const int r = e % R, c = e / R;
    double acc = 0.0;
    for (int i = 0; i < ln; ++i) acc = fma(a.At[n0][i + ln * r], a.At[n0][i + ln * c], acc);
    a.Gm[n0][e] = acc;
  }
  if (n0 != a.N - 1) return;
  __syncthreads();
  // 8. lambda, fit and the stop rule (after the last mode of the sweep)
  for (int r = tid; r < R; r += nt) a.lam[r] = nu[r];
  if (tid == 0) {
    double ip = 0.0;
    for (int e = 0; e < n; ++e) ip = fma(Ms[e], Xs[e], ip);
    double bh = 0.0;
    for (int e = 0; e < R * R; ++e) {
      const int r = e % R, c = e / R;
      double v = nu[r] * nu[c];
      for (int m = 0; m < a.N; ++m) v *= a.Gm[m][e];
      bh += v;
    }
    const double nb = st->norm_b2;
    const double rho = 1.0 - (nb + bh - 2.0 * ip) / nb;
    st->ip = ip;
    st->fit = rho;
    st->als_iters += 1;
    const bool conv = fabs(rho - st->fit_prev) < a.tol;
    st->fit_prev = rho;
    if (!isfinite(rho)) set_status(st, RCP_ENAN);
    if (conv || st->als_iters >= a.max_iters) st->als_done = conv ? 1 : 2;
  }
}

// A_n[i, r] = sum_c Q_n[i, c] Atilde_n[c, r] (unnormalised), one thread per
// output: each is an l-term FP64 chain, and I R of them spread over the GPU
// (consecutive threads take consecutive rows i, so the loads of Q coalesce).
__global__ void k_backproject(const double* __restrict__ Q, int64_t I, int l,
                              const double* __restrict__ At, int R, double* __restrict__ A) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= I * R) return;
  const int64_t r = e / I, i = e - r * I;
  const double* a = At + (int64_t)l * r;
  double acc = 0.0;
  for (int c = 0; c < l; ++c) acc = fma(Q[i + I * c], a[c], acc);
  A[e] = acc;
}

struct ProjArgs {
  int N, R;
  int64_t I[kMaxN];
  double* A[kMaxN];
  double* nu;          // N x R
  const double* lam_t;
  double* lam_out;
};

// Column norms of every A_n and the updated lambda (Algorithm 2 step 13).
__global__ void k_colnorms(ProjArgs p) {
  __shared__ double red[32];
  const int col = blockIdx.x;  // n * R + r
  const int n = col / p.R, r = col % p.R;
  const double* a = p.A[n] + p.I[n] * r;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < p.I[n]; i += blockDim.x) acc = fma(a[i], a[i], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)blockDim.x / 32; ++w) s += red[w];
    p.nu[col] = sqrt(s);
  }
}

__global__ void k_normalise(ProjArgs p) {
  const int n = blockIdx.y;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < p.I[n] * p.R) {
    const int r = (int)(e / p.I[n]);
    const double v = p.nu[n * p.R + r];
    p.A[n][e] = v > 0.0 ? p.A[n][e] / v : 0.0;
  }
  if (n == 0 && blockIdx.x == 0 && threadIdx.x < (unsigned)p.R) {
    const int r = threadIdx.x;
    double lam = p.lam_t[r];
    for (int m = 0; m < p.N; ++m) lam *= p.nu[m * p.R + r];
    p.lam_out[r] = lam;
  }
}

AlsArgs make_args(rcp_plan_s* p, int n0) {
  AlsArgs a{};
  a.N = p->N;
  a.n0 = n0;
  a.R = p->R;
  a.ln = p->l[n0];
  for (int m = 0; m < p->N; ++m) {
    a.At[m] = p->At[m];
    a.Gm[m] = p->Gm[m];
    a.dims[m] = p->l[m];
  }
  a.lam = p->lam;
  a.M = p->M;
  a.st = p->dstate;
  a.tol = p->cfg.tol;
  a.max_iters = p->cfg.max_iters;
  a.part = p->part;
  return a;
}

}  // namespace

cudaError_t launch_als_init(rcp_plan_s* p, cudaStream_t s) {
  AlsArgs a = make_args(p, 0);
  count_launches(1);
  k_als_init<<<1, 256, 0, s>>>(a, p->cfg.seed, p->user_init ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_als_sweep(rcp_plan_s* p, int n0, cudaStream_t s) {
  const ModeView v{[&] {
                     int64_t L = 1;
                     for (int m = 0; m < n0; ++m) L *= p->l[m];
                     return L;
                   }(),
                   p->l[n0],
                   [&] {
                     int64_t Rt = 1;
                     for (int m = n0 + 1; m < p->N; ++m) Rt *= p->l[m];
                     return Rt;
                   }(),
                   0};
  ModeView vv = v;
  vv.J = vv.L * vv.Rt;
  KrDims kr{};
  kr.N = p->N;
  kr.n = n0;
  for (int m = 0; m < p->N; ++m) {
    kr.dims[m] = p->l[m];
    kr.A[m] = p->At[m];
  }
  const int nsplit = sketch_splits(vv, p->nsm);
  cudaError_t e = launch_mttkrp_f64(p->Bcore64, vv, p->R, kr, nsplit, p->part, s);
  if (e != cudaSuccess) return e;
  AlsArgs a = make_args(p, n0);
  a.nsplit = nsplit;
  const int R = p->R, ln = p->l[n0];
  const size_t smem = (size_t)(2 * ln * R + R * (R + 1) + R * R + R) * sizeof(double);
  e = cudaFuncSetAttribute(k_als_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  count_launches(1);
  k_als_update<<<1, 256, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_backproject(rcp_plan_s* p, double* const* A_dev, double* lambda_dev,
                               cudaStream_t s) {
  ProjArgs pa{};
  pa.N = p->N;
  pa.R = p->R;
  int64_t maxe = 0;
  for (int n = 0; n < p->N; ++n) {
    pa.I[n] = p->dims[n];
    pa.A[n] = A_dev[n];
    const int64_t I = p->dims[n];
    count_launches(1);
    k_backproject<<<(unsigned)((I * p->R + 255) / 256), 256, 0, s>>>(p->Q[n], I, p->l[n],
                                                                      p->At[n], p->R, A_dev[n]);
    if (I * p->R > maxe) maxe = I * p->R;
  }
  pa.nu = p->tmp;
  pa.lam_t = p->lam;
  pa.lam_out = lambda_dev;
  count_launches(2);
  k_colnorms<<<p->N * p->R, 256, 0, s>>>(pa);
  k_normalise<<<dim3((unsigned)((maxe + 255) / 256), p->N), 256, 0, s>>>(pa);
  return cudaGetLastError();
}

}  // namespace rcp

// rCP-BCD on the compressed tensor B (Algorithm 3 steps 3-15, Section 3.2.2):
// CP by successive rank-one deflation, one CTA, every component and sweep in
// one launch.
//
// Component r = 1..R starts from column r of the initial factors of modes
// 2..N and repeats sweeps over n = 1..N of
//     a_n = Y_(n) (KR of the other a_m) / prod_{m != n} a_m^T a_m,
// normalising a_n (lambda_r = |a_N| at n = N), where Y = B - [[lambda_{1..r-1};
// A_{:,1..r-1}, ...]] is the residual of the components already found.  Y is
// never formed ("residual-free", Section 3.2.2): the rank-one MTTKRP is taken
// of B and the earlier components' contribution subtracted,
//     Y_(n) (KR a_m) = B_(n) (KR a_m) - sum_{s < r} lambda_s A_n[:, s]
//                      prod_{m != n} (A_m[:, s]^T a_m).
// The products A_m[:, s]^T a_m are kept per mode and refreshed when a_m
// changes.  B_(n) (KR a_m) is a chain of tensor-times-vector contractions, the
// highest remaining mode first: contracting mode m of the current tensor
// (viewed as L x l_m x Rt with L the product of the lower modes and Rt = l_n
// when n > m, else 1) gives out[a + L b] = sum_d T[a + L (d + l_m b)] v[d],
// one thread per output and coalesced across a.
//
// Fit and stop rule per component: after each sweep rho = 1 - (|Y|^2 -
// lambda_r^2) / |B|^2, the fit of the rank-r model (|Y - lambda_r a_1 o ... o
// a_N|^2 = |Y|^2 - lambda_r^2 once a_N is the least-squares update for unit
// a_1..a_{N-1}); the component ends when rho changes by less than tol from the
// previous sweep (before the first sweep: 1 - |Y|^2 / |B|^2) or after
// max_iters sweeps; then |Y|^2 drops by lambda_r^2.  TB is the element type of
// B: double (the plain path) or float (the precision form, whose first
// contraction sums in FP32 per output); everything else is FP64.
#include <math.h>

#include "rcp_internal.cuh"
#include "small_la.cuh"

namespace rcp {
namespace {

constexpr int kBT = 512;

struct BcdArgs {
  int N, R;
  int l[kMaxN];
  const void* B;
  double* At[kMaxN];     // in (user_init): initial factors l_n x R; out: the components
  double* lam;           // out: lambda (R)
  double* buf0;          // scratch: two contraction buffers of core / min l_n doubles
  double* buf1;
  DevState* st;
  uint64_t seed;
  double tol;
  int max_iters;
  int user_init;
  const int* user_init_dev;  // when set, a device word that replaces user_init
};

__device__ double block_sum_bcd(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < kBT / 32; ++w) s += red[w];
  return s;
}

template <typename TB>
__global__ void __launch_bounds__(kBT, 1) k_bcd(BcdArgs a) {
  __shared__ double vec[kMaxN][kMaxL];      // a_m of the current component
  __shared__ double gam[kMaxN][RCP_MAX_RANK];  // A_m[:, s]^T a_m, s < r
  __shared__ double nrm2[kMaxN];
  __shared__ double xs[kMaxL];
  __shared__ double red[kBT / 32];
  const int tid = threadIdx.x;
  const int N = a.N, R = a.R;
  const TB* B = (const TB*)a.B;
  int64_t core = 1;
  for (int m = 0; m < N; ++m) core *= a.l[m];

  // |B|^2
  double acc = 0.0;
  for (int64_t e = tid; e < core; e += kBT) {
    const double b = (double)B[e];
    acc = fma(b, b, acc);
  }
  const double nB = block_sum_bcd(acc, red);
  double nY = nB;
  double rho = 1.0 - nY / nB;
  int total = 0;
  bool bad = !(nB > 0.0) || !isfinite(nB);
  const int user_init = a.user_init_dev ? *a.user_init_dev : a.user_init;

  for (int r = 0; r < R && !bad; ++r) {
    // starting vectors of modes 2..N: column r of the initial factors
    for (int m = 1; m < N; ++m) {
      const int lm = a.l[m];
      for (int i = tid; i < lm; i += kBT) {
        double v;
        if (user_init) {
          v = a.At[m][i + (int64_t)lm * r];
        } else {
          const int g = i * R + r;  // the row-major l_m x R stream of the seeded start
          const double2 z = normal_pair_f64(a.seed, (uint32_t)(m + 1), kPurposeAlsInit,
                                            (uint64_t)(g >> 1));
          v = (g & 1) ? z.y : z.x;
        }
        vec[m][i] = v;
      }
    }
    __syncthreads();
    // squared norms and the products with the earlier components
    for (int m = 1; m < N; ++m) {
      const int lm = a.l[m];
      double s2 = 0.0;
      for (int i = tid; i < lm; i += kBT) s2 = fma(vec[m][i], vec[m][i], s2);
      s2 = block_sum_bcd(s2, red);
      if (tid == 0) nrm2[m] = s2;
      for (int s = tid; s < r; s += kBT) {
        double g = 0.0;
        for (int i = 0; i < lm; ++i) g = fma(a.At[m][i + (int64_t)lm * s], vec[m][i], g);
        gam[m][s] = g;
      }
    }
    __syncthreads();
    double rho_prev = 1.0 - nY / nB;
    double lam_r = 0.0;
    for (int it = 0; it < a.max_iters; ++it) {
      for (int n = 0; n < N; ++n) {
        const int ln = a.l[n];
        // ---- B_(n) (KR of the other a_m): contractions, highest mode first
        const double* src = nullptr;
        double* dst = a.buf0;
        bool first = true;
        for (int m = N - 1; m >= 0; --m) {
          if (m == n) continue;
          int64_t L = 1;
          for (int k = 0; k < m; ++k) L *= a.l[k];
          const int lm = a.l[m];
          const int64_t Rt = n > m ? ln : 1;
          const int64_t nout = L * Rt;
          for (int64_t o = tid; o < nout; o += kBT) {
            const int64_t b = o / L, aa = o - b * L;
            const int64_t base = aa + L * (int64_t)lm * b;
            double v;
            if (first) {
              TB s = (TB)0;
              for (int d = 0; d < lm; ++d) s = fma(B[base + L * d], (TB)vec[m][d], s);
              v = (double)s;
            } else {
              double s = 0.0;
              for (int d = 0; d < lm; ++d) s = fma(src[base + L * d], vec[m][d], s);
              v = s;
            }
            dst[o] = v;
          }
          __syncthreads();
          src = dst;
          dst = dst == a.buf0 ? a.buf1 : a.buf0;
          first = false;
        }
        // ---- minus the earlier components, over the product of the other norms
        double denom = 1.0;
        for (int m = 0; m < N; ++m)
          if (m != n) denom *= nrm2[m];
        for (int i = tid; i < ln; i += kBT) {
          double x = src ? src[i] : (double)B[i];  // N = 1 never occurs (N >= 2)
          for (int s = 0; s < r; ++s) {
            double w = a.lam[s] * a.At[n][i + (int64_t)ln * s];
            for (int m = 0; m < N; ++m)
              if (m != n) w *= gam[m][s];
            x -= w;
          }
          xs[i] = denom > 0.0 ? x / denom : 0.0;
        }
        __syncthreads();
        double s2 = 0.0;
        for (int i = tid; i < ln; i += kBT) s2 = fma(xs[i], xs[i], s2);
        s2 = block_sum_bcd(s2, red);
        const double nu = sqrt(s2);
        const double inv = nu > 0.0 ? 1.0 / nu : 0.0;
        double t2 = 0.0;
        for (int i = tid; i < ln; i += kBT) {
          const double v = xs[i] * inv;
          vec[n][i] = v;
          t2 = fma(v, v, t2);
        }
        t2 = block_sum_bcd(t2, red);  // also orders the vec[n] writes before the reads below
        if (tid == 0) nrm2[n] = t2;
        if (n == N - 1) lam_r = nu;
        for (int s = tid; s < r; s += kBT) {
          double g = 0.0;
          for (int i = 0; i < ln; ++i) g = fma(a.At[n][i + (int64_t)ln * s], vec[n][i], g);
          gam[n][s] = g;
        }
        __syncthreads();
      }
      ++total;
      rho = 1.0 - (nY - lam_r * lam_r) / nB;
      if (!isfinite(rho)) {
        bad = true;
        break;
      }
      const bool conv = fabs(rho - rho_prev) < a.tol;
      rho_prev = rho;
      if (conv) break;
    }
    // keep the component; the residual loses lambda_r^2
    for (int m = 0; m < N; ++m)
      for (int i = tid; i < a.l[m]; i += kBT) a.At[m][i + (int64_t)a.l[m] * r] = vec[m][i];
    if (tid == 0) a.lam[r] = lam_r;
    nY -= lam_r * lam_r;
    __syncthreads();
  }
  if (tid == 0) {
    a.st->fit = rho;
    a.st->fit_prev = rho;
    a.st->als_iters = total;
    a.st->norm_b2 = nB;
    a.st->als_done = 1;
    if (bad) set_status(a.st, RCP_ENAN);
  }
}

}  // namespace

// Scratch: two buffers of core / min_n l_n doubles each (the first contraction's output).
int64_t bcd_scratch_elems(const rcp_plan_s* p) {
  int lmin = p->l[0];
  for (int m = 1; m < p->N; ++m) lmin = lmin < p->l[m] ? lmin : p->l[m];
  return 2 * (p->core_elems / lmin + 1);
}

cudaError_t launch_bcd(rcp_plan_s* p, const void* B, bool f32, double* scratch,
                       const int* user_init_dev, cudaStream_t s) {
  BcdArgs a{};
  a.user_init_dev = user_init_dev;
  a.N = p->N;
  a.R = p->R;
  for (int m = 0; m < p->N; ++m) {
    a.l[m] = p->l[m];
    a.At[m] = p->At[m];
  }
  a.B = B;
  a.lam = p->lam;
  const int64_t half = bcd_scratch_elems(p) / 2;
  a.buf0 = scratch;
  a.buf1 = scratch + half;
  a.st = p->dstate;
  a.seed = p->cfg.seed;
  a.tol = p->cfg.tol;
  a.max_iters = p->cfg.max_iters;
  a.user_init = p->user_init ? 1 : 0;
  count_launches(1);
  if (f32) k_bcd<float><<<1, kBT, 0, s>>>(a);
  else k_bcd<double><<<1, kBT, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace rcp

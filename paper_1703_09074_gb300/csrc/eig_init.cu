// Eigenvector initialisation of the stage-2 solvers (Algorithm 2 step 2,
// Algorithm 3 step 2; Section 3.2.1 names it the standard initial guess):
// for every mode n = 2..N, the eigenvectors of B_(n) B_(n)^T belonging to its
// R largest eigenvalues, in descending order, each with its largest-magnitude
// entry positive (the first such entry on a tie).  Everything in FP64.
//
//   k_mode_grams  G_n = B_(n) B_(n)^T, one CTA per entry (i <= i') of one mode,
//                 the sum over the J_n columns split over the CTA's threads.
//   k_jacobi_eig  the cyclic Jacobi method on G_n, one CTA per mode (Golub &
//                 Van Loan, "Matrix Computations", Section 8.5): each sweep runs
//                 the l - 1 rounds of a round-robin ordering, in which the
//                 l / 2 disjoint pairs (p, q) are rotated at once; the rotation
//                 zeroing a_pq is the symmetric 2 x 2 Schur decomposition
//                 (tau = (a_qq - a_pp) / (2 a_pq), t = sign(tau) / (|tau| +
//                 sqrt(1 + tau^2)), c = 1 / sqrt(1 + t^2), s = t c).  Sweeps stop
//                 when the off-diagonal mass falls below (2^-53 |G|_F)^2 or after
//                 40 sweeps.  Then the eigenvalues are ranked, and the leading R
//                 eigenvectors are sign-fixed and written as the initial factor.
#include <math.h>

#include "rcp_internal.cuh"
#include "small_la.cuh"

namespace rcp {
namespace {

constexpr int kEigThreads = 256;
constexpr int kEigMax = kMaxL;          // l_n <= 64

struct GramArgs {
  const double* B;       // Kolda layout, l_1 x ... x l_N
  int N;
  int l[kMaxN];
  double* G[kMaxN];      // out: l_n x l_n row-major for n >= 1 (0-based mode index)
};

// blockIdx.y = mode index n - 1 (0-based mode n >= 1); blockIdx.x = packed pair (i <= i2)
__global__ void __launch_bounds__(kEigThreads) k_mode_grams(GramArgs a) {
  __shared__ double red[kEigThreads / 32];
  const int n = blockIdx.y + 1;
  const int ln = a.l[n];
  int rem = blockIdx.x, i = 0;
  while (i < ln && rem >= ln - i) {  // row i of the packed upper triangle holds ln - i pairs
    rem -= ln - i;
    ++i;
  }
  if (i >= ln) return;  // uniform per CTA
  const int i2 = i + rem;
  int64_t L = 1, Rt = 1;
  for (int m = 0; m < n; ++m) L *= a.l[m];
  for (int m = n + 1; m < a.N; ++m) Rt *= a.l[m];
  const int64_t J = L * Rt;
  double acc = 0.0;
  for (int64_t j = threadIdx.x; j < J; j += kEigThreads) {
    const int64_t b = j / L, aa = j - b * L;
    const int64_t base = aa + L * (int64_t)ln * b;
    acc = fma(a.B[base + L * i], a.B[base + L * i2], acc);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kEigThreads / 32; ++w) s += red[w];
    a.G[n][i * ln + i2] = s;
    a.G[n][i2 * ln + i] = s;
  }
}

struct EigArgs {
  int N, R;
  int l[kMaxN];
  const double* G[kMaxN];
  double* At[kMaxN];     // out: l_n x R column-major, n >= 1
  DevState* st;
};

__global__ void __launch_bounds__(kEigThreads) k_jacobi_eig(EigArgs a) {
  extern __shared__ double eig_smem[];   // A and V, m x (m + 1) each
  __shared__ double cs[kEigMax / 2], sn[kEigMax / 2];
  __shared__ int pp[kEigMax / 2], qq[kEigMax / 2];
  __shared__ double red[kEigThreads / 32];
  __shared__ int rank_of[kEigMax];
  __shared__ double off_sh, fro_sh;
  const int n = blockIdx.x + 1;
  const int ln = a.l[n], R = a.R;
  const int tid = threadIdx.x;
  const int m = ln + (ln & 1);  // even count: an odd l_n gets a dummy index that never rotates
  const int kEigPitch = m + 1;
  double* A = eig_smem;
  double* V = eig_smem + m * kEigPitch;
  for (int e = tid; e < m * m; e += kEigThreads) {
    const int r = e / m, c = e - r * m;
    A[r * kEigPitch + c] = (r < ln && c < ln) ? a.G[n][r * ln + c] : 0.0;
    V[r * kEigPitch + c] = r == c ? 1.0 : 0.0;
  }
  __syncthreads();
  // |G|_F^2
  double f = 0.0;
  for (int e = tid; e < ln * ln; e += kEigThreads) {
    const double g = a.G[n][e];
    f = fma(g, g, f);
  }
  for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
  if ((tid & 31) == 0) red[tid >> 5] = f;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < kEigThreads / 32; ++w) s += red[w];
    fro_sh = s;
  }
  __syncthreads();
  const double thresh = fro_sh * 1.2325951644078310e-32;  // (2^-53)^2 |G|_F^2
  const int npair = m / 2;
  for (int sweep = 0; sweep < 40; ++sweep) {
    // off-diagonal mass
    double o2 = 0.0;
    for (int e = tid; e < ln * ln; e += kEigThreads) {
      const int r = e / ln, c = e - r * ln;
      if (r != c) {
        const double v = A[r * kEigPitch + c];
        o2 = fma(v, v, o2);
      }
    }
    for (int o = 16; o > 0; o >>= 1) o2 += __shfl_xor_sync(0xffffffffu, o2, o);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = o2;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < kEigThreads / 32; ++w) s += red[w];
      off_sh = s;
    }
    __syncthreads();
    if (!(off_sh > thresh)) break;  // uniform (also stops on a non-finite mass)
    for (int round = 0; round < m - 1; ++round) {
      // round-robin pairs: slot k pairs positions k and m-1-k of the list
      // (m-1 fixed, the rest rotated by `round`)
      if (tid < npair) {
        auto pos = [&](int k) { return k == m - 1 ? m - 1 : (k + round) % (m - 1); };
        int p = pos(tid), q = pos(m - 1 - tid);
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        double c = 1.0, s = 0.0;
        const double apq = A[p * kEigPitch + q];
        if (q < ln && apq != 0.0) {
          const double tau = (A[q * kEigPitch + q] - A[p * kEigPitch + p]) / (2.0 * apq);
          const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(fma(tau, tau, 1.0)));
          c = rsqrt64(fma(t, t, 1.0));
          s = t * c;
        }
        pp[tid] = p;
        qq[tid] = q;
        cs[tid] = c;
        sn[tid] = s;
      }
      __syncthreads();
      // rows p, q of A: A <- J^T A
      for (int e = tid; e < npair * m; e += kEigThreads) {
        const int k = e / m, j = e - k * m;
        const int p = pp[k], q = qq[k];
        const double c = cs[k], s = sn[k];
        const double x = A[p * kEigPitch + j], y = A[q * kEigPitch + j];
        A[p * kEigPitch + j] = c * x - s * y;
        A[q * kEigPitch + j] = s * x + c * y;
      }
      __syncthreads();
      // columns p, q of A and of V: A <- A J, V <- V J
      for (int e = tid; e < npair * m; e += kEigThreads) {
        const int k = e / m, i = e - k * m;
        const int p = pp[k], q = qq[k];
        const double c = cs[k], s = sn[k];
        const double x = A[i * kEigPitch + p], y = A[i * kEigPitch + q];
        A[i * kEigPitch + p] = c * x - s * y;
        A[i * kEigPitch + q] = s * x + c * y;
        const double u = V[i * kEigPitch + p], w = V[i * kEigPitch + q];
        V[i * kEigPitch + p] = c * u - s * w;
        V[i * kEigPitch + q] = s * u + c * w;
      }
      __syncthreads();
    }
  }
  // rank of each eigenvalue, descending, ties by index (a stable sort)
  for (int i = tid; i < ln; i += kEigThreads) {
    const double di = A[i * kEigPitch + i];
    int rk = 0;
    for (int j = 0; j < ln; ++j) {
      const double dj = A[j * kEigPitch + j];
      rk += (dj > di) || (dj == di && j < i);
    }
    rank_of[i] = rk;
    if (!isfinite(di)) set_status(a.st, RCP_ENAN);
  }
  __syncthreads();
  // leading R eigenvectors, largest-magnitude entry positive (first on a tie)
  for (int col = tid; col < ln; col += kEigThreads) {
    const int r = rank_of[col];
    if (r >= R) continue;
    int piv = 0;
    double best = -1.0;
    for (int i = 0; i < ln; ++i) {
      const double v = fabs(V[i * kEigPitch + col]);
      if (v > best) {
        best = v;
        piv = i;
      }
    }
    const double sg = V[piv * kEigPitch + col] < 0.0 ? -1.0 : 1.0;
    for (int i = 0; i < ln; ++i) a.At[n][i + (int64_t)ln * r] = sg * V[i * kEigPitch + col];
  }
}

}  // namespace

// G_n for n = 2..N into `gram` (packed one l_n x l_n block per mode, l_max^2
// doubles each), then the eigenvector factors into At[1..N-1].
cudaError_t launch_eig_init(rcp_plan_s* p, const double* B, double* gram, cudaStream_t s) {
  int lmax = 1;
  for (int m = 0; m < p->N; ++m) lmax = lmax > p->l[m] ? lmax : p->l[m];
  GramArgs g{};
  g.B = B;
  g.N = p->N;
  EigArgs e{};
  e.N = p->N;
  e.R = p->R;
  e.st = p->dstate;
  for (int m = 0; m < p->N; ++m) {
    g.l[m] = e.l[m] = p->l[m];
    g.G[m] = gram + (size_t)m * lmax * lmax;
    e.G[m] = g.G[m];
    e.At[m] = p->At[m];
  }
  if (p->N < 2) return cudaSuccess;
  count_launches(2);
  k_mode_grams<<<dim3(lmax * (lmax + 1) / 2, p->N - 1), kEigThreads, 0, s>>>(g);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const int me = lmax + (lmax & 1);
  const size_t smem = (size_t)2 * me * (me + 1) * sizeof(double);
  err = cudaFuncSetAttribute(k_jacobi_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k_jacobi_eig<<<p->N - 1, kEigThreads, smem, s>>>(e);
  return cudaGetLastError();
}

}  // namespace rcp

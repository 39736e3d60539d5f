// Data path of the learned warm start for CP-ALS on the compressed tensor B.
//
// The network sees B in a canonical basis: for each mode n the eigenvectors
// U_n of the Gram B_(n) B_(n)^T (descending eigenvalues, each vector's
// largest-magnitude entry positive), i.e. the core G = B x_1 U_1^T x_2 U_2^T
// x_3 U_3^T of the higher-order SVD, scaled to unit Frobenius norm and
// zero-padded to 24^3.  Its output Y (3 x 24 x 16) is read as a correction in
// that basis: the initial factors are A_n = U_n (E + Y_n) restricted to l_n
// rows and R columns, where E holds the first R unit vectors.  With Y = 0 this
// is the eigenvector initialisation that Section 3.2 names as the ALS default.
//
// Training compares the columns of E + Y_n with the converged ALS factors of
// the same tensor expressed in the canonical basis, after matching the R
// components one to one (the CP model is invariant to their order) with the
// assignment that minimises sum_r sum_n (1 - cos^2); the per-column loss is
// invariant to the scale and sign of each component as well.
#include <math.h>

#include "mlp_internal.cuh"

namespace rcp {

namespace {

constexpr int L = kWsL;
constexpr int L2 = L * L;
constexpr int L3 = L * L * L;

// ---------------------------------------------------------------- gather
// Bpad[b] <- the compressed tensor of item b (Kolda l1 x l2 x l3), zero-padded
// to 24^3 with index i1 + 24 i2 + 576 i3; meta[b] = (l1, l2, l3, R), or zeros
// when the item is not eligible.
__global__ void __launch_bounds__(256) k_ws_gather(const WsItem* __restrict__ items,
                                                   float* __restrict__ Bpad, int* __restrict__ meta) {
  const WsItem it = items[blockIdx.x];
  float* out = Bpad + (int64_t)blockIdx.x * L3;
  const bool ok = it.core != nullptr;
  const int l1 = ok ? it.l[0] : 0, l2 = ok ? it.l[1] : 0, l3 = ok ? it.l[2] : 0;
  for (int e = threadIdx.x; e < L3; e += blockDim.x) {
    const int i1 = e % L, i2 = (e / L) % L, i3 = e / L2;
    float v = 0.0f;
    if (i1 < l1 && i2 < l2 && i3 < l3) v = it.core[i1 + l1 * (i2 + l2 * i3)];
    out[e] = v;
  }
  if (threadIdx.x == 0) {
    int* m = meta + 4 * blockIdx.x;
    m[0] = l1;
    m[1] = l2;
    m[2] = l3;
    m[3] = ok ? it.R : 0;
  }
}

// ---------------------------------------------------------------- canonical basis
// Parallel-order Jacobi (Golub & Van Loan, Section 8.5; round-robin ordering
// after Brent & Luk) on the symmetric l x l matrix A (row pitch L, FP64, shared
// memory) by one warp.  A sweep is n - 1 rounds (n = l rounded up to even); a
// round rotates n / 2 disjoint pairs at once: lane i forms the rotation of pair
// i from the round's A, then the lanes apply all of them to the columns (and to
// V) and then to the rows, A <- J^T A J, V <- V J.  FP64 keeps the eigenvectors
// of the small, clustered noise eigenvalues reproducible to the oracle's
// eigensolver.  Stops when the off-diagonal part is negligible or after 30
// sweeps.
__device__ void warp_jacobi(double* A, double* V, int l) {
  const int lane = threadIdx.x & 31;
  __shared__ double cs_sh[3][kWsL / 2][2];  // per calling warp (warps 0-2): c, s of each pair
  __shared__ int pq_sh[3][kWsL / 2][2];
  const int w = (threadIdx.x >> 5) % 3;
  double (*cs)[2] = cs_sh[w];
  int (*pq)[2] = pq_sh[w];
  for (int k = lane; k < L2; k += 32) V[k] = ((k / L) == (k % L)) ? 1.0 : 0.0;
  __syncwarp();
  const int n = (l + 1) & ~1, np = n / 2;  // player n - 1 is a dummy when l is odd
  for (int sweep = 0; sweep < 30; ++sweep) {
    // stop once every |a_pq| <= 1e-14 max_k a_kk (a threshold relative to the
    // largest eigenvalue: the small, clustered noise eigenvalues would never meet
    // one relative to sqrt(a_pp a_qq) in FP64)
    double worst = 0.0, dmax = 0.0;
    for (int e = lane; e < l * l; e += 32) {
      const int p = e / l, q = e % l;
      if (p < q) worst = fmax(worst, fabs(A[p * L + q]));
      if (p == q) dmax = fmax(dmax, A[p * L + p]);
    }
    for (int o = 16; o > 0; o >>= 1) {
      worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
      dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    }
    if (!(worst > 1e-14 * dmax)) break;
    const double skip = 1e-17 * dmax;  // rotations below this change nothing representable
    for (int r = 0; r < n - 1; ++r) {
      if (lane < np) {
        // circle method: position 0 holds player 0, position k >= 1 player (k - 1 + r) mod (n - 1) + 1
        const int pa = lane == 0 ? 0 : (lane - 1 + r) % (n - 1) + 1;
        const int pb = (n - 1 - lane - 1 + r) % (n - 1) + 1;
        int p = min(pa, pb), q = max(pa, pb);
        double c = 1.0, sn = 0.0;
        if (q < l) {
          const double apq = A[p * L + q];
          if (fabs(apq) > skip) {
            const double tau = (A[q * L + q] - A[p * L + p]) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            sn = t * c;
          }
        } else {
          p = q = -1;  // the dummy's partner sits out this round
        }
        cs[lane][0] = c;
        cs[lane][1] = sn;
        pq[lane][0] = p;
        pq[lane][1] = q;
      }
      __syncwarp();
      for (int task = lane; task < l * np; task += 32) {  // columns p, q of A and V
        const int i = task % np, k = task / np;
        const int p = pq[i][0], q = pq[i][1];
        if (p < 0 || cs[i][1] == 0.0) continue;
        const double c = cs[i][0], sn = cs[i][1];
        const double akp = A[k * L + p], akq = A[k * L + q];
        A[k * L + p] = c * akp - sn * akq;
        A[k * L + q] = sn * akp + c * akq;
        const double vkp = V[k * L + p], vkq = V[k * L + q];
        V[k * L + p] = c * vkp - sn * vkq;
        V[k * L + q] = sn * vkp + c * vkq;
      }
      __syncwarp();
      for (int task = lane; task < l * np; task += 32) {  // rows p, q of A
        const int i = task % np, k = task / np;
        const int p = pq[i][0], q = pq[i][1];
        if (p < 0 || cs[i][1] == 0.0) continue;
        const double c = cs[i][0], sn = cs[i][1];
        const double apk = A[p * L + k], aqk = A[q * L + k];
        A[p * L + k] = c * apk - sn * aqk;
        A[q * L + k] = sn * apk + c * aqk;
      }
      __syncwarp();
    }
  }
}

// One CTA per sample: Grams of the three unfoldings, their eigenvectors
// (sorted, sign-fixed) into U[b] (3 x 24 x 24, column j = vector j), and the
// unit-norm core G into x[b].
__global__ void __launch_bounds__(256) k_ws_canon(const float* __restrict__ Bpad,
                                                  const int* __restrict__ meta,
                                                  float* __restrict__ x, float* __restrict__ Uout) {
  extern __shared__ __align__(16) unsigned char sm[];
  float* Bs = (float*)sm;                        // L^3
  double* A = (double*)(Bs + L3);                // 3 x L x L
  double* V = A + 3 * L2;                        // 3 x L x L
  float* Uf = (float*)(V + 3 * L2);              // 3 x L x L
  __shared__ double red[8];
  __shared__ int perm[3][L];
  const int b = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int* mt = meta + 4 * b;
  const int ln[3] = {mt[0], mt[1], mt[2]};
  const float* src = Bpad + (int64_t)b * L3;
  for (int e = tid; e < 3 * L2; e += 256) Uf[e] = 0.0f;
  double nrm = 0.0;
  for (int e = tid; e < L3; e += 256) {
    const float v = src[e];
    Bs[e] = v;
    nrm += (double)v * v;
  }
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  if (lane == 0) red[warp] = nrm;
  __syncthreads();
  // Grams S_n[i][k] = sum over the other two indices (FP32 products, FP64 sum per entry)
  for (int e = tid; e < 3 * L2; e += 256) {
    const int n = e / L2, i = (e % L2) / L, k = e % L;
    double s = 0.0;
    if (i < ln[n] && k < ln[n] && i <= k) {
      const int st1 = n == 0 ? L : 1, st2 = n == 2 ? L : L2;  // strides of the other two modes
      const int sn = n == 0 ? 1 : (n == 1 ? L : L2);
      for (int u = 0; u < L; ++u) {
        float acc = 0.0f;
        for (int w = 0; w < L; ++w) {
          const int base = u * st1 + w * st2;
          acc = fmaf(Bs[base + i * sn], Bs[base + k * sn], acc);
        }
        s += acc;
      }
    }
    A[e] = s;
  }
  __syncthreads();
  for (int e = tid; e < 3 * L2; e += 256) {
    const int n = e / L2, i = (e % L2) / L, k = e % L;
    if (i > k) A[e] = A[n * L2 + k * L + i];
  }
  __syncthreads();
  if (warp < 3 && ln[warp] > 0) {
    const int n = warp, l = ln[n];
    double* An = A + n * L2;
    double* Vn = V + n * L2;
    warp_jacobi(An, Vn, l);
    __syncwarp();
    if (lane == 0) {  // descending eigenvalues (stable selection order)
      bool used[L];
      for (int k = 0; k < L; ++k) used[k] = false;
      for (int j = 0; j < l; ++j) {
        int best = -1;
        for (int k = 0; k < l; ++k)
          if (!used[k] && (best < 0 || An[k * L + k] > An[best * L + best])) best = k;
        used[best] = true;
        perm[n][j] = best;
      }
    }
    __syncwarp();
    for (int j = 0; j < L; ++j) {
      // column j of U_n: eigenvector perm[j], largest |entry| (first on ties) made positive
      double v = 0.0;
      if (j < l && lane < l) v = Vn[lane * L + perm[n][j]];
      double a = (lane < l && j < l) ? fabs(v) : -1.0;
      int idx = lane;
      for (int o = 16; o > 0; o >>= 1) {
        const double oa = __shfl_xor_sync(0xffffffffu, a, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (oa > a || (oa == a && oi < idx)) {
          a = oa;
          idx = oi;
        }
      }
      const double piv = __shfl_sync(0xffffffffu, v, idx);
      if (piv < 0.0) v = -v;
      if (lane < L) Uf[n * L2 + lane * L + j] = (float)v;
    }
  }
  __syncthreads();
  for (int e = tid; e < 3 * L2; e += 256) Uout[(int64_t)b * 3 * L2 + e] = Uf[e];
  // G = B x_1 U_1^T x_2 U_2^T x_3 U_3^T, one fibre per thread and mode, in place
  for (int n = 0; n < 3; ++n) {
    const int sn = n == 0 ? 1 : (n == 1 ? L : L2);
    for (int f = tid; f < L2; f += 256) {
      const int u = f % L, w = f / L;
      int base;
      if (n == 0) base = u * L + w * L2;
      else if (n == 1) base = u + w * L2;
      else base = u + w * L;
      float xin[L];
#pragma unroll
      for (int i = 0; i < L; ++i) xin[i] = Bs[base + i * sn];
#pragma unroll 4
      for (int j = 0; j < L; ++j) {
        float acc = 0.0f;
#pragma unroll
        for (int i = 0; i < L; ++i) acc = fmaf(Uf[n * L2 + i * L + j], xin[i], acc);
        Bs[base + j * sn] = acc;
      }
    }
    __syncthreads();
  }
  double tot = 0.0;
  for (int w = 0; w < 8; ++w) tot += red[w];
  const float sc = tot > 0.0 ? (float)(1.0 / sqrt(tot)) : 0.0f;
  float* xo = x + (int64_t)b * L3;
  for (int e = tid; e < L3; e += 256) xo[e] = Bs[e] * sc;
}

// ---------------------------------------------------------------- matching loss
// Minimum-cost perfect matching of an n x n cost matrix (row pitch kWsR) by the
// Hungarian method with row/column potentials (Kuhn 1955; the O(n^3)
// shortest-augmenting-path form).  match[r] = column assigned to row r.
// Non-finite costs must be replaced by the caller.  Every loop is bounded by n.
__device__ void hungarian(const float* cost, int n, int* match) {
  double u[kWsR + 1], v[kWsR + 1], minv[kWsR + 1];
  int p[kWsR + 1], way[kWsR + 1];
  bool used[kWsR + 1];
  for (int j = 0; j <= n; ++j) {
    u[j] = v[j] = 0.0;
    p[j] = 0;
    way[j] = 0;
  }
  for (int i = 1; i <= n; ++i) {
    p[0] = i;
    int j0 = 0;
    for (int j = 0; j <= n; ++j) {
      minv[j] = 1e300;
      used[j] = false;
    }
    for (int guard = 0; guard <= n; ++guard) {  // at most n + 1 columns become used
      used[j0] = true;
      const int i0 = p[j0];
      double delta = 1e300;
      int j1 = 0;
      for (int j = 1; j <= n; ++j) {
        if (used[j]) continue;
        const double cur = (double)cost[(i0 - 1) * kWsR + (j - 1)] - u[i0] - v[j];
        if (cur < minv[j]) {
          minv[j] = cur;
          way[j] = j0;
        }
        if (minv[j] < delta) {
          delta = minv[j];
          j1 = j;
        }
      }
      for (int j = 0; j <= n; ++j) {
        if (used[j]) {
          u[p[j]] += delta;
          v[j] -= delta;
        } else {
          minv[j] -= delta;
        }
      }
      j0 = j1;
      if (j0 == 0 || p[j0] == 0) break;
    }
    for (int guard = 0; guard <= n && j0 != 0; ++guard) {  // augment along the path
      const int j1 = way[j0];
      p[j0] = p[j1];
      j0 = j1;
    }
  }
  for (int j = 1; j <= n; ++j)
    if (p[j] >= 1) match[p[j] - 1] = j - 1;
}

// One CTA (128 threads) per sample.  F_n = E + Y_n on l_n rows and R columns;
// D[r][s] = sum_n (1 - (F_n[:, r] . T_n[:, s])^2 / |F_n[:, r]|^2) with unit
// target columns; loss = (1/R) sum_r D[r][match r]; dY = scale d loss / d Y.
__global__ void __launch_bounds__(128) k_ws_loss(const float* __restrict__ Y,
                                                 const float* __restrict__ T,
                                                 const int* __restrict__ meta, float scale,
                                                 float* __restrict__ dY, float* __restrict__ loss) {
  __shared__ float F[kMlpOut], Ts[kMlpOut];
  __shared__ float ff[3][kWsR], ft[3][kWsR][kWsR];
  __shared__ float D[kWsR * kWsR];
  __shared__ int match[kWsR];
  const int b = blockIdx.x, tid = threadIdx.x;
  const int* mt = meta + 4 * b;
  const int R = mt[3];
  const int ln[3] = {mt[0], mt[1], mt[2]};
  for (int e = tid; e < kMlpOut; e += 128) {
    const int n = e / (L * kWsR), i = (e / kWsR) % L, r = e % kWsR;
    const bool in = i < ln[n] && r < R;
    F[e] = in ? Y[(int64_t)b * kMlpOut + e] + (i == r ? 1.0f : 0.0f) : 0.0f;
    Ts[e] = in ? T[(int64_t)b * kMlpOut + e] : 0.0f;
  }
  __syncthreads();
  for (int e = tid; e < 3 * kWsR * (kWsR + 1); e += 128) {
    const int n = e / (kWsR * (kWsR + 1)), q = e % (kWsR * (kWsR + 1));
    const int r = q / (kWsR + 1), s = q % (kWsR + 1);
    const float* Fn = F + n * L * kWsR;
    const float* Tn = Ts + n * L * kWsR;
    float acc = 0.0f;
    if (s == kWsR) {
      for (int i = 0; i < L; ++i) acc = fmaf(Fn[i * kWsR + r], Fn[i * kWsR + r], acc);
      ff[n][r] = acc;
    } else {
      for (int i = 0; i < L; ++i) acc = fmaf(Fn[i * kWsR + r], Tn[i * kWsR + s], acc);
      ft[n][r][s] = acc;
    }
  }
  __syncthreads();
  for (int e = tid; e < kWsR * kWsR; e += 128) {
    const int r = e / kWsR, s = e % kWsR;
    float d = 0.0f;
    for (int n = 0; n < 3; ++n) d += 1.0f - ft[n][r][s] * ft[n][r][s] / fmaxf(ff[n][r], 1e-12f);
    D[e] = isfinite(d) ? d : 1e30f;
  }
  __syncthreads();
  if (tid == 0) {
    if (R > 0) hungarian(D, R, match);
    float s = 0.0f;
    for (int r = 0; r < R; ++r) s += D[r * kWsR + match[r]];
    loss[b] = R > 0 ? s / R : 0.0f;
  }
  __syncthreads();
  for (int e = tid; e < kMlpOut; e += 128) {
    const int n = e / (L * kWsR), i = (e / kWsR) % L, r = e % kWsR;
    float g = 0.0f;
    if (i < ln[n] && r < R) {
      const int s = match[r];
      const float f2 = fmaxf(ff[n][r], 1e-12f), c = ft[n][r][s];
      const float fi = F[e], ti = Ts[n * L * kWsR + i * kWsR + s];
      g = (scale / R) * (-2.0f * c * ti / f2 + 2.0f * c * c * fi / (f2 * f2));
    }
    dY[(int64_t)b * kMlpOut + e] = g;
  }
}

// ---------------------------------------------------------------- initial factors
// A_n = U_n (E + Y_n) on l_n rows and R columns, FP64 column-major into the
// item's ALS factors; the item's init word is set only when every column is
// finite and nonzero (else ALS keeps its random initialisation).
__global__ void __launch_bounds__(128) k_ws_init(const float* __restrict__ Y,
                                                 const float* __restrict__ U,
                                                 const int* __restrict__ meta,
                                                 const WsItem* __restrict__ items) {
  __shared__ float F[kMlpOut];
  __shared__ int bad;
  const int b = blockIdx.x, tid = threadIdx.x;
  const WsItem it = items[b];
  const int* mt = meta + 4 * b;
  const int R = mt[3];
  if (tid == 0) bad = (it.core == nullptr || R == 0) ? 1 : 0;
  for (int e = tid; e < kMlpOut; e += 128) {
    const int n = e / (L * kWsR), i = (e / kWsR) % L, r = e % kWsR;
    F[e] = (i < mt[n] && r < R) ? Y[(int64_t)b * kMlpOut + e] + (i == r ? 1.0f : 0.0f) : 0.0f;
  }
  __syncthreads();
  if (!bad) {
    for (int n = 1; n < 3; ++n) {
      const int l = mt[n];
      const float* Un = U + ((int64_t)b * 3 + n) * L2;
      for (int e = tid; e < l * R; e += 128) {
        const int i = e % l, r = e / l;
        double s = 0.0;
        for (int k = 0; k < l; ++k) s += (double)Un[i * L + k] * F[n * L * kWsR + k * kWsR + r];
        if (!isfinite(s)) atomicExch(&bad, 1);
        it.At[n][i + l * r] = s;
      }
      __syncthreads();
      if (tid < R) {
        double c = 0.0;
        for (int i = 0; i < l; ++i) c += it.At[n][i + l * tid] * it.At[n][i + l * tid];
        if (!(c > 0.0)) atomicExch(&bad, 1);
      }
      __syncthreads();
    }
  }
  __syncthreads();
  if (tid == 0) {
    if (it.user_init) *it.user_init = bad ? 0 : 1;
    if (!bad && it.st) atomicOr(&it.st->info, RCP_INFO_LEARNED_INIT);
  }
}

// Training targets: T_n = U_n^T A_n with unit columns (A_n: the item's
// converged ALS factors), zero outside l_n x R.
__global__ void __launch_bounds__(128) k_ws_targets(const WsItem* __restrict__ items,
                                                    const float* __restrict__ U,
                                                    float* __restrict__ T) {
  __shared__ float nrm[kWsR];
  const int b = blockIdx.x, tid = threadIdx.x;
  const WsItem it = items[b];
  float* Tb = T + (int64_t)b * kMlpOut;
  for (int e = tid; e < kMlpOut; e += 128) Tb[e] = 0.0f;
  if (it.core == nullptr) return;
  const int R = it.R;
  __syncthreads();
  for (int n = 0; n < 3; ++n) {
    const int l = it.l[n];
    const float* Un = U + ((int64_t)b * 3 + n) * L2;
    for (int e = tid; e < l * R; e += 128) {
      const int j = e / R, r = e % R;
      double s = 0.0;
      for (int i = 0; i < l; ++i) s += (double)Un[i * L + j] * it.At[n][i + l * r];
      Tb[n * L * kWsR + j * kWsR + r] = (float)s;
    }
    __syncthreads();
    if (tid < R) {
      float c = 0.0f;
      for (int j = 0; j < l; ++j) {
        const float v = Tb[n * L * kWsR + j * kWsR + tid];
        c += v * v;
      }
      nrm[tid] = c > 0.0f ? rsqrtf(c) : 0.0f;
    }
    __syncthreads();
    for (int e = tid; e < l * R; e += 128) {
      const int j = e / R, r = e % R;
      Tb[n * L * kWsR + j * kWsR + r] *= nrm[r];
    }
    __syncthreads();
  }
}

constexpr size_t kCanonSmem = (size_t)L3 * 4 + (size_t)6 * L2 * 8 + (size_t)3 * L2 * 4;

}  // namespace

cudaError_t launch_ws_gather(const WsItem* items, int count, float* Bpad, int* meta, cudaStream_t s) {
  count_launches(1);
  k_ws_gather<<<count, 256, 0, s>>>(items, Bpad, meta);
  return cudaGetLastError();
}

cudaError_t prepare_ws() {
  return cudaFuncSetAttribute(k_ws_canon, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kCanonSmem);
}

cudaError_t launch_ws_canon(const float* Bpad, const int* meta, int count, float* x, float* U,
                            cudaStream_t s) {
  count_launches(1);
  k_ws_canon<<<count, 256, kCanonSmem, s>>>(Bpad, meta, x, U);
  return cudaGetLastError();
}

cudaError_t launch_ws_loss(const float* Y, const float* T, const int* meta, int count, float scale,
                           float* dY, float* loss, cudaStream_t s) {
  count_launches(1);
  k_ws_loss<<<count, 128, 0, s>>>(Y, T, meta, scale, dY, loss);
  return cudaGetLastError();
}

cudaError_t launch_ws_init(const float* Y, const float* U, const int* meta, const WsItem* items,
                           int count, cudaStream_t s) {
  count_launches(1);
  k_ws_init<<<count, 128, 0, s>>>(Y, U, meta, items);
  return cudaGetLastError();
}

cudaError_t launch_ws_targets(const WsItem* items, const float* U, int count, float* T,
                              cudaStream_t s) {
  count_launches(1);
  k_ws_targets<<<count, 128, 0, s>>>(items, U, T);
  return cudaGetLastError();
}

}  // namespace rcp

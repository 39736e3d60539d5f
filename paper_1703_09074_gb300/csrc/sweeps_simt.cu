// Sweeps over the working tensor T_n on the CUDA cores: FP64 (the plain
// method) and FP32 (later modes of the mixed-precision form).
//
// Row sweep   : P[i, c] = sum_j T_(n)[i, j] V[j, c]          (split over j)
//   V = Omega_n  -> the sketch Y = T_(n) Omega_n             (Algorithm 1 step 6, Eq. sampleMatrix)
//   V = W        -> Y = T_(n) W of a power iteration         (Algorithm 1 step 10)
//   V = KR rows  -> the MTTKRP B_(n) (KR of the factors)     (Algorithm 2 steps 4, 6, 8)
// Column sweep: W[j, c] = sum_i T_(n)[i, j] Q[i, c]          (no split)
//   Q = Q of the sketch -> W = T_(n)^T Q                     (Algorithm 1 step 9), with the
//                          Gram W^T W of its normalisation accumulated per CTA
//   Q = Q_n             -> T_{n+1} = T_n x_n Q_n^T          (Algorithm 1 step 13, Definition 1)
// W is written in the Kolda layout of T_{n+1}: W[a + L (c + l b)] for column j = a + L b.
#include "rcp_internal.cuh"

namespace rcp {
namespace {

constexpr int kRowTile = 32;      // columns j staged per step of the row sweep
constexpr int kProjThreads = 256; // columns j per CTA step of the column sweep
static_assert(kProjThreads == kBColBlock, "batched column items count blocks of kProjThreads");
constexpr int kProjRows = 32;     // rows of Q staged per step of the column sweep
constexpr int kBatchQRows = 256;  // the same for the batched column sweep (FP32 Q)

enum { kSrcOmega = 0, kSrcW = 1, kSrcKr = 2 };

}  // namespace

// Row sweep body for block (bx, by) of a (gx, gy) grid: rows bx * rows_per_cta +
// [0, rows_per_cta), columns by * jchunk + [0, jchunk).
template <int LMAX, typename TIn, typename TA, int SRC, bool NORM>
__device__ __forceinline__ void row_sweep_body(const TIn* __restrict__ T, ModeView v,
                                               int64_t rows_per_cta, int l, uint64_t seed,
                                               uint32_t sid, const TA* __restrict__ W,
                                               const KrDims& kr, int64_t jchunk,
                                               double* __restrict__ part,
                                               double* __restrict__ normpart, int bx, int by,
                                               int gx) {
  __shared__ TA Vs[kRowTile][LMAX];
  __shared__ int64_t offs[kRowTile];   // column j of the tile: its offset in T
  __shared__ int64_t offw[kRowTile];   // and in W (SRC == kSrcW)
  const int tid = threadIdx.x;
  const int64_t i = (int64_t)bx * rows_per_cta + tid;
  const bool row_ok = (tid < rows_per_cta) && (i < v.I);
  const int64_t j0 = (int64_t)by * jchunk;
  const int64_t j1 = min(v.J, j0 + jchunk);

  TA acc[LMAX];
#pragma unroll
  for (int c = 0; c < LMAX; ++c) acc[c] = (TA)0;
  double nrm = 0.0;

  for (int k = tid; k < kRowTile * LMAX; k += blockDim.x) (&Vs[0][0])[k] = (TA)0;
  __syncthreads();

  for (int64_t jt = j0; jt < j1; jt += kRowTile) {
    const int nj = (int)min((int64_t)kRowTile, j1 - jt);
    if (tid < nj) {
      // the only 64-bit divisions of the tile: one per column
      const int64_t j = jt + tid;
      const int64_t b = v.L == 1 ? j : j / v.L, a = j - b * v.L;
      offs[tid] = a + v.L * v.I * b;
      if (SRC == kSrcW) offw[tid] = a + v.L * (int64_t)l * b;
    }
    // the stream elements of the tile are e = jt l + t, t < nj l local (32-bit)
    const int nt = nj * l;
    if (SRC == kSrcOmega && sizeof(TA) == 8) {
      // Omega_n[j, c] is element e = j * l + c of the FP64 stream; pairs g = e / 2.
      const int64_t e0 = jt * l;
      const int64_t g0 = e0 >> 1;
      const int lead = (int)(e0 - 2 * g0);
      for (int q = tid; 2 * q - lead < nt; q += blockDim.x) {
        const double2 z = normal_pair_f64(seed, sid, kPurposeSketch, (uint64_t)(g0 + q));
        int t = 2 * q - lead;
        if (t >= 0) Vs[t / l][t - (t / l) * l] = (TA)z.x;
        ++t;
        if (t < nt) Vs[t / l][t - (t / l) * l] = (TA)z.y;
      }
    } else if (SRC == kSrcOmega) {
      // reduced-precision stream: quads g = e / 4
      const int64_t e0 = jt * l;
      const int64_t g0 = e0 >> 2;
      const int lead = (int)(e0 - 4 * g0);
      for (int q = tid; 4 * q - lead < nt; q += blockDim.x) {
        const float4 z = normal_quad_f32(seed, sid, kPurposeSketch, (uint64_t)(g0 + q));
        const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int t = 4 * q + u - lead;
          if (t >= 0 && t < nt) Vs[t / l][t - (t / l) * l] = (TA)zz[u];
        }
      }
    } else if (SRC == kSrcW) {
      __syncthreads();  // offw of this tile
      for (int k = tid; k < nt; k += blockDim.x) {
        const int jj = k / l, c = k - jj * l;
        Vs[jj][c] = W[offw[jj] + v.L * c];
      }
    } else {
      // Khatri-Rao row of the factors of every mode but kr.n, mode 1 fastest.
      for (int k = tid; k < nj * l; k += blockDim.x) {
        const int jj = k / l, r = k - jj * l;
        int64_t jr = jt + jj;
        double prod = 1.0;
        for (int m = 0; m < kr.N; ++m) {
          if (m == kr.n) continue;
          const int d = kr.dims[m];
          const int im = (int)(jr % d);
          jr /= d;
          prod *= kr.A[m][im + (int64_t)d * r];
        }
        Vs[jj][r] = (TA)prod;
      }
    }
    __syncthreads();
    if (row_ok) {
      // U loads in flight per thread before their products (latency, not FMAs, bounds
      // this loop); the |X|^2 of the mixed form is summed per tile in FP32
      constexpr int U = sizeof(TA) == 4 ? 8 : 4;
      TA tn = (TA)0;
      int jj = 0;
      for (; jj + U <= nj; jj += U) {
        TA xs[U];
#pragma unroll
        for (int u = 0; u < U; ++u) xs[u] = (TA)__ldg(T + offs[jj + u] + v.L * i);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (NORM) tn = fma(xs[u], xs[u], tn);
#pragma unroll
          for (int c = 0; c < LMAX; ++c) acc[c] = fma(xs[u], Vs[jj + u][c], acc[c]);
        }
      }
      for (; jj < nj; ++jj) {
        const TA x = (TA)__ldg(T + offs[jj] + v.L * i);
        if (NORM) tn = fma(x, x, tn);
#pragma unroll
        for (int c = 0; c < LMAX; ++c) acc[c] = fma(x, Vs[jj][c], acc[c]);
      }
      if (NORM) nrm += (double)tn;
    }
    __syncthreads();
  }
  if (row_ok) {
#pragma unroll
    for (int c = 0; c < LMAX; ++c)
      if (c < l) part[((int64_t)by * l + c) * v.I + i] = (double)acc[c];
  }
  if (NORM) {
    __shared__ double red[256];
    red[tid] = nrm;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
      if (tid < s && tid + s < (int)blockDim.x) red[tid] += red[tid + s];
      __syncthreads();
    }
    if (tid == 0) normpart[(int64_t)by * gx + bx] = red[0];
  }
}

// Column sweep body for CTA bx of nb persistent CTAs of NT threads (columns j) each;
// Q is staged QR rows at a time.
template <int LMAX, typename TIn, typename TA, bool GRAM, int NT = kProjThreads,
          int QR = kProjRows>
__device__ __forceinline__ void col_sweep_body(const TIn* __restrict__ T, ModeView v, int l,
                                               const double* __restrict__ Q, TA* __restrict__ W,
                                               double* __restrict__ gpart, int bx, int nb);

namespace {

template <int LMAX, typename TIn, typename TA, int SRC, bool NORM>
__global__ void __launch_bounds__(256)
k_row_sweep(const TIn* __restrict__ T, ModeView v, int64_t rows_per_cta, int l, uint64_t seed,
            uint32_t sid, const TA* __restrict__ W, KrDims kr, int64_t jchunk,
            double* __restrict__ part, double* __restrict__ normpart) {
  row_sweep_body<LMAX, TIn, TA, SRC, NORM>(T, v, rows_per_cta, l, seed, sid, W, kr, jchunk, part,
                                           normpart, blockIdx.x, blockIdx.y, gridDim.x);
}

}  // namespace

template <int LMAX, typename TIn, typename TA, bool GRAM, int NT, int QR>
__device__ __forceinline__ void col_sweep_body(const TIn* __restrict__ T, ModeView v, int l,
                                               const double* __restrict__ Q, TA* __restrict__ W,
                                               double* __restrict__ gpart, int bx, int nb) {
  extern __shared__ double sm[];
  TA* Qs = (TA*)sm;                                 // QR x LMAX
  double* Ws = sm + QR * LMAX;                      // NT x (LMAX + 1), GRAM only
  __shared__ unsigned short pairs[kMaxL * (kMaxL + 1) / 2];
  constexpr int kSlots = (LMAX * (LMAX + 1) / 2 + NT - 1) / NT;
  const int tid = threadIdx.x;
  const int npairs = l * (l + 1) / 2;
  double gacc[GRAM ? kSlots : 1];
#pragma unroll
  for (int s = 0; s < (GRAM ? kSlots : 1); ++s) gacc[s] = 0.0;
  if (GRAM && tid < l) {
    int base = tid * l - tid * (tid - 1) / 2;
    for (int c2 = tid; c2 < l; ++c2) pairs[base + c2 - tid] = (unsigned short)((tid << 8) | c2);
  }

  for (int64_t jb = bx; jb * NT < v.J; jb += nb) {
    const int64_t j = jb * NT + tid;
    const bool ok = j < v.J;
    const int64_t a = ok ? j % v.L : 0, b = ok ? j / v.L : 0;
    const int64_t base = a + v.L * v.I * b;
    TA acc[LMAX];
#pragma unroll
    for (int c = 0; c < LMAX; ++c) acc[c] = (TA)0;
    for (int64_t i0 = 0; i0 < v.I; i0 += QR) {
      const int ni = (int)min((int64_t)QR, v.I - i0);
      __syncthreads();
      for (int k = tid; k < QR * LMAX; k += NT) {
        const int ii = k / LMAX, c = k - ii * LMAX;
        Qs[k] = (ii < ni && c < l) ? (TA)Q[(i0 + ii) + v.I * c] : (TA)0;
      }
      __syncthreads();
      if (ok) {
        constexpr int U = sizeof(TA) == 4 ? 8 : 4;  // loads in flight per thread
        int ii = 0;
        for (; ii + U <= ni; ii += U) {
          TA xs[U];
#pragma unroll
          for (int u = 0; u < U; ++u) xs[u] = (TA)__ldg(T + base + v.L * (i0 + ii + u));
#pragma unroll
          for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < LMAX; ++c) acc[c] = fma(xs[u], Qs[(ii + u) * LMAX + c], acc[c]);
        }
        for (; ii < ni; ++ii) {
          const TA x = (TA)__ldg(T + base + v.L * (i0 + ii));
#pragma unroll
          for (int c = 0; c < LMAX; ++c) acc[c] = fma(x, Qs[ii * LMAX + c], acc[c]);
        }
      }
    }
    if (ok) {
#pragma unroll
      for (int c = 0; c < LMAX; ++c)
        if (c < l) W[a + v.L * (c + (int64_t)l * b)] = acc[c];
    }
    if (GRAM) {
#pragma unroll
      for (int c = 0; c < LMAX; ++c) Ws[tid * (LMAX + 1) + c] = ok ? (double)acc[c] : 0.0;
      __syncthreads();
#pragma unroll
      for (int s = 0; s < kSlots; ++s) {
        const int p = tid + s * NT;
        if (p < npairs) {
          const int c1 = pairs[p] >> 8, c2 = pairs[p] & 0xff;
          double sum = 0.0;
          for (int t = 0; t < NT; ++t)
            sum = fma(Ws[t * (LMAX + 1) + c1], Ws[t * (LMAX + 1) + c2], sum);
          gacc[s] += sum;
        }
      }
    }
  }
  if (GRAM) {
#pragma unroll
    for (int s = 0; s < kSlots; ++s) {
      const int p = tid + s * NT;
      if (p < npairs) gpart[(int64_t)bx * npairs + p] = gacc[s];
    }
  }
}

namespace {

template <int LMAX, typename TIn, typename TA, bool GRAM, int NT>
__global__ void __launch_bounds__(NT)
k_col_sweep(const TIn* __restrict__ T, ModeView v, int l, const double* __restrict__ Q,
            TA* __restrict__ W, double* __restrict__ gpart) {
  col_sweep_body<LMAX, TIn, TA, GRAM, NT>(T, v, l, Q, W, gpart, blockIdx.x, gridDim.x);
}


int lmax_bucket(int l) { return l <= 16 ? 16 : l <= 32 ? 32 : l <= 48 ? 48 : 64; }

template <int LMAX, typename TIn, typename TA>
cudaError_t row_sweep_typed(const TIn* T, ModeView v, int l, uint64_t seed, uint32_t sid,
                            const TA* W, const KrDims* kr, int src, int nsplit, double* part,
                            double* normpart, cudaStream_t s) {
  const int64_t nib = (v.I + 255) / 256;
  const int64_t rpc = (v.I + nib - 1) / nib;
  const int threads = (int)((rpc + 31) / 32 * 32);
  const int64_t jchunk = (v.J + nsplit - 1) / nsplit;
  dim3 grid((unsigned)nib, (unsigned)nsplit);
  KrDims k{};
  if (kr) k = *kr;
  count_launches(1);
  if (src == kSrcOmega) {
    if (normpart)
      k_row_sweep<LMAX, TIn, TA, kSrcOmega, true><<<grid, threads, 0, s>>>(
          T, v, rpc, l, seed, sid, W, k, jchunk, part, normpart);
    else
      k_row_sweep<LMAX, TIn, TA, kSrcOmega, false><<<grid, threads, 0, s>>>(
          T, v, rpc, l, seed, sid, W, k, jchunk, part, normpart);
  } else if (src == kSrcW) {
    k_row_sweep<LMAX, TIn, TA, kSrcW, false><<<grid, threads, 0, s>>>(T, v, rpc, l, seed, sid, W, k,
                                                                    jchunk, part, normpart);
  } else {
    k_row_sweep<LMAX, TIn, TA, kSrcKr, false><<<grid, threads, 0, s>>>(T, v, rpc, l, seed, sid, W, k,
                                                                     jchunk, part, normpart);
  }
  return cudaGetLastError();
}

template <typename TIn, typename TA>
cudaError_t row_sweep_any(const TIn* T, ModeView v, int l, uint64_t seed, uint32_t sid,
                          const TA* W, const KrDims* kr, int src, int nsplit, double* part,
                          double* normpart, cudaStream_t s) {
  switch (lmax_bucket(l)) {
    case 16: return row_sweep_typed<16>(T, v, l, seed, sid, W, kr, src, nsplit, part, normpart, s);
    case 32: return row_sweep_typed<32>(T, v, l, seed, sid, W, kr, src, nsplit, part, normpart, s);
    case 48: return row_sweep_typed<48>(T, v, l, seed, sid, W, kr, src, nsplit, part, normpart, s);
    default: return row_sweep_typed<64>(T, v, l, seed, sid, W, kr, src, nsplit, part, normpart, s);
  }
}

template <int LMAX, typename TIn, typename TA>
cudaError_t col_sweep_typed(const TIn* T, ModeView v, int l, const double* Q, TA* W,
                            double* gpart, int nblocks, cudaStream_t s) {
  const size_t smem_q = (size_t)kProjRows * LMAX * sizeof(double);
  count_launches(1);
  if (gpart) {
    const size_t smem = smem_q + (size_t)kProjThreads * (LMAX + 1) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_col_sweep<LMAX, TIn, TA, true, kProjThreads>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_col_sweep<LMAX, TIn, TA, true, kProjThreads>
        <<<nblocks, kProjThreads, smem, s>>>(T, v, l, Q, W, gpart);
  } else {
    k_col_sweep<LMAX, TIn, TA, false, kProjThreads>
        <<<nblocks, kProjThreads, smem_q, s>>>(T, v, l, Q, W, gpart);
  }
  return cudaGetLastError();
}

template <typename TIn, typename TA>
cudaError_t col_sweep_any(const TIn* T, ModeView v, int l, const double* Q, TA* W,
                          double* gpart, int nblocks, cudaStream_t s) {
  switch (lmax_bucket(l)) {
    case 16: return col_sweep_typed<16>(T, v, l, Q, W, gpart, nblocks, s);
    case 32: return col_sweep_typed<32>(T, v, l, Q, W, gpart, nblocks, s);
    case 48: return col_sweep_typed<48>(T, v, l, Q, W, gpart, nblocks, s);
    default: return col_sweep_typed<64>(T, v, l, Q, W, gpart, nblocks, s);
  }
}

// Column sweep of the precision form for the later modes, whose tensors are
// small: W[a + L (c + l b)] = sum_i T[a + L (i + I b)] Q[i][c] (Q in FP64,
// staged once per CTA as FP32).  A thread owns one column j = (a, b) of a block
// of 64 and one block of 8 outputs c, and S threads split the rows i of each
// (column, output block) for small J; their partial sums meet in shared
// memory in a fixed order.  Thread tid: column jj = tid % 64, output block
// cb = (tid / 64) % NCB, row split s = tid / (64 NCB); a warp is 32
// consecutive columns of one (cb, s), so its loads of T coalesce and its
// reads of Q are broadcasts.
template <int NCB>
__global__ void __launch_bounds__(1024)
k_col_sweep_cb(const float* __restrict__ T, ModeView v, int l, const double* __restrict__ Q,
               float* __restrict__ W, int S) {
  extern __shared__ float4 smq[];
  constexpr int P = NCB * 8;  // padded row of Q in shared memory
  float* Qs = (float*)smq;
  float* red = Qs + (size_t)v.I * P;  // (S - 1) x 64 x P partial sums
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int64_t e = tid; e < v.I * P; e += nt) {
    const int64_t i = e / P;
    const int c = (int)(e - i * P);
    Qs[e] = c < l ? (float)Q[i + v.I * c] : 0.0f;
  }
  __syncthreads();
  const int jj = tid & 63, cb = (tid >> 6) % NCB, sp = (tid >> 6) / NCB;
  const int64_t rps = (v.I + S - 1) / S;
  const int64_t i_lo = min(v.I, sp * rps), i_hi = min(v.I, i_lo + rps);
  for (int64_t jb = blockIdx.x; jb * 64 < v.J; jb += gridDim.x) {
    const int64_t j = jb * 64 + jj;
    const bool ok = j < v.J;
    const int64_t a = ok ? j % v.L : 0, b = ok ? j / v.L : 0;
    const float* t = T + a + v.L * v.I * b;
    float acc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = 0.0f;
    if (ok) {
      int64_t i = i_lo;
      for (; i + 8 <= i_hi; i += 8) {
        float x[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) x[q] = __ldg(t + v.L * (i + q));
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 q0 = *(const float4*)(Qs + (i + q) * P + cb * 8);
          const float4 q1 = *(const float4*)(Qs + (i + q) * P + cb * 8 + 4);
          acc[0] = fmaf(x[q], q0.x, acc[0]);
          acc[1] = fmaf(x[q], q0.y, acc[1]);
          acc[2] = fmaf(x[q], q0.z, acc[2]);
          acc[3] = fmaf(x[q], q0.w, acc[3]);
          acc[4] = fmaf(x[q], q1.x, acc[4]);
          acc[5] = fmaf(x[q], q1.y, acc[5]);
          acc[6] = fmaf(x[q], q1.z, acc[6]);
          acc[7] = fmaf(x[q], q1.w, acc[7]);
        }
      }
      for (; i < i_hi; ++i) {
        const float x = __ldg(t + v.L * i);
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] = fmaf(x, Qs[i * P + cb * 8 + u], acc[u]);
      }
    }
    if (S > 1) {
      __syncthreads();
      if (sp > 0)
#pragma unroll
        for (int u = 0; u < 8; ++u) red[((sp - 1) * 64 + jj) * P + cb * 8 + u] = acc[u];
      __syncthreads();
      if (sp == 0)
        for (int s2 = 1; s2 < S; ++s2)
#pragma unroll
          for (int u = 0; u < 8; ++u) acc[u] += red[((s2 - 1) * 64 + jj) * P + cb * 8 + u];
    }
    if (ok && sp == 0) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int c = cb * 8 + u;
        if (c < l) W[a + v.L * (c + (int64_t)l * b)] = acc[u];
      }
    }
  }
}

template <int NCB>
cudaError_t col_sweep_cb_typed(const float* T, ModeView v, int l, const double* Q, float* W,
                               int nsm, cudaStream_t s) {
  // row splits S until the threads fill the SMs (2048 each), within 1024 per CTA;
  // at 64 registers a thread, an SM holds 1024 / (64 NCB S) CTAs of this shape
  const int64_t nb = (v.J + 63) / 64;
  const int smax = 1024 / (64 * NCB);
  const int64_t per_s = nb * 64 * NCB;
  int S = (int)((2048LL * nsm + per_s - 1) / per_s);
  S = S < 1 ? 1 : (S > smax ? smax : S);
  const int per_sm = 1024 / (64 * NCB * S) > 0 ? 1024 / (64 * NCB * S) : 1;
  const int grid = (int)(nb < (int64_t)per_sm * nsm ? nb : (int64_t)per_sm * nsm);
  const size_t smem = ((size_t)v.I * NCB * 8 + (size_t)(S - 1) * 64 * NCB * 8) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_col_sweep_cb<NCB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  count_launches(1);
  k_col_sweep_cb<NCB><<<grid, 64 * NCB * S, smem, s>>>(T, v, l, Q, W, S);
  return cudaGetLastError();
}

}  // namespace

// True when the blocked column sweep applies: Q (I x 8 ceil(l / 8) FP32) and
// the row-split partial sums fit in shared memory.
bool col_sweep_cb_fits(const ModeView& v, int l) {
  const int ncb = (l + 7) / 8;
  return l >= 1 && ncb <= 8 && ((size_t)v.I * ncb * 8 + (size_t)7 * 64 * ncb * 8) * 4 <= 200 * 1024;
}

int sketch_splits(const ModeView& v, int nsm) {
  const int64_t nib = (v.I + 255) / 256;
  int64_t want = (2LL * nsm + nib - 1) / nib;            // about two CTAs per SM
  const int64_t maxs = (v.J + kRowTile - 1) / kRowTile;  // at least one tile per split
  if (want > maxs) want = maxs;
  if (want < 1) want = 1;
  if (want > 65535) want = 65535;
  return (int)want;
}

int project_grid(const ModeView& v, int nsm) {
  const int64_t blocks = (v.J + kProjThreads - 1) / kProjThreads;
  const int64_t cap = 4LL * nsm;
  return (int)(blocks < cap ? (blocks < 1 ? 1 : blocks) : cap);
}

// ---------------------------------------------------------------- batched sweeps
// One launch covers the same sweep of every tensor of a batch: persistent CTAs
// pull work items (tensor b, block coordinates) from an atomic counter; the
// host orders the items largest tensor first.

namespace {

// acc[c] += x v[c] for c < LB, two columns per packed FP32 FMA (each lane is an
// fmaf: the sums are those of the scalar loop).  v is 16-byte aligned, LB % 4 == 0.
template <int LB>
__device__ __forceinline__ void fma_row2(float2 (&acc)[LB / 2], float x, const float* v) {
  const float2 xx = make_float2(x, x);
#pragma unroll
  for (int c = 0; c < LB; c += 4) {
    const float4 q = *reinterpret_cast<const float4*>(v + c);
    acc[c / 2] = __ffma2_rn(xx, make_float2(q.x, q.y), acc[c / 2]);
    acc[c / 2 + 1] = __ffma2_rn(xx, make_float2(q.z, q.w), acc[c / 2 + 1]);
  }
}

constexpr int kRowGroups = 8;  // column groups of the batched row sweep

// Row sweep of the batched form (FP32, l <= LB <= 32).  A block of few rows would
// leave most of a 256-thread CTA idle with one thread per row, so the threads form
// G groups of ceil32(rows) threads: one staging round fills G tiles of kRowTile
// columns, group g multiplies tile g, and the G partial sums of each row meet in
// shared memory in a fixed order.  The outputs are those of row_sweep_body.  Vs
// (kRowGroups kRowTile x LB floats), offs, offw and nred are the kernel's shared
// buffers, so that one launch can run several widths LB.
template <int LB, int SRC, int U>
__device__ __forceinline__ void row_sweep_body_grouped(const float* __restrict__ T, ModeView v,
                                                       int64_t rows_per_cta, int l,
                                                       uint64_t seed, uint32_t sid,
                                                       const float* __restrict__ W,
                                                       int64_t jchunk, double* __restrict__ part,
                                                       double* __restrict__ normpart, int bx,
                                                       int by, int gx, float* vs, int64_t* offs,
                                                       int64_t* offw, double* nred) {
  const bool NORM = normpart != nullptr;  // mode 1 of the sketch also sums X^2
  float(*Vs)[LB] = reinterpret_cast<float(*)[LB]>(vs);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int rpc = (int)rows_per_cta;
  const int rpc32 = (rpc + 31) & ~31;
  const int G = max(1, min(kRowGroups, nthr / rpc32));
  const int grp = tid / rpc32, r = tid - grp * rpc32;
  const int64_t i = (int64_t)bx * rows_per_cta + r;
  const bool row_ok = grp < G && r < rpc && i < v.I;
  const int64_t j0 = (int64_t)by * jchunk;
  const int64_t j1 = min(v.J, j0 + jchunk);
  const int TW = G * kRowTile;  // columns per staging round

  float2 acc[LB / 2];
#pragma unroll
  for (int c = 0; c < LB / 2; ++c) acc[c] = make_float2(0.0f, 0.0f);
  double nrm = 0.0;
  for (int k = tid; k < kRowGroups * kRowTile * LB; k += nthr) vs[k] = 0.0f;
  __syncthreads();

  for (int64_t jt = j0; jt < j1; jt += TW) {
    const int nj = (int)min((int64_t)TW, j1 - jt);
    for (int jj = tid; jj < nj; jj += nthr) {
      const int64_t j = jt + jj;
      const int64_t b = v.L == 1 ? j : j / v.L, a = j - b * v.L;
      offs[jj] = a + v.L * v.I * b;
      if (SRC == kSrcW) offw[jj] = a + v.L * (int64_t)l * b;
    }
    const int nt = nj * l;
    if (SRC == kSrcOmega) {
      const int64_t e0 = jt * l;
      const int64_t g0 = e0 >> 2;
      const int lead = (int)(e0 - 4 * g0);
      for (int q = tid; 4 * q - lead < nt; q += nthr) {
        const float4 z = normal_quad_f32(seed, sid, kPurposeSketch, (uint64_t)(g0 + q));
        const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int t = 4 * q + u - lead;
          if (t >= 0 && t < nt) Vs[t / l][t - (t / l) * l] = zz[u];
        }
      }
    } else {
      __syncthreads();  // offw of this round
      for (int k = tid; k < nt; k += nthr) {
        const int jj = k / l, c = k - jj * l;
        Vs[jj][c] = W[offw[jj] + v.L * c];
      }
    }
    __syncthreads();
    if (row_ok) {
      // group grp's tile: columns grp kRowTile .. of the round; U loads in flight
      const int c0 = grp * kRowTile, c1 = min(nj, c0 + kRowTile);
      float tn = 0.0f;
      int jj = c0;
      for (; jj + U <= c1; jj += U) {
        float xs[U];
#pragma unroll
        for (int u = 0; u < U; ++u) xs[u] = __ldg(T + offs[jj + u] + v.L * i);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (NORM) tn = fmaf(xs[u], xs[u], tn);
          fma_row2<LB>(acc, xs[u], Vs[jj + u]);
        }
      }
      for (; jj < c1; ++jj) {
        const float x = __ldg(T + offs[jj] + v.L * i);
        if (NORM) tn = fmaf(x, x, tn);
        fma_row2<LB>(acc, x, Vs[jj]);
      }
      if (NORM) nrm += (double)tn;
    }
    __syncthreads();
  }
  // groups 1..G-1 hand their sums to group 0 through Vs (G rpc32 LB <= its size)
  float2* red = reinterpret_cast<float2*>(vs);
  if (grp > 0 && grp < G)
#pragma unroll
    for (int c = 0; c < LB / 2; ++c) red[(grp * rpc32 + r) * (LB / 2) + c] = acc[c];
  __syncthreads();
  if (grp == 0 && row_ok) {
    for (int g2 = 1; g2 < G; ++g2)
#pragma unroll
      for (int c = 0; c < LB / 2; ++c) {
        const float2 o = red[(g2 * rpc32 + r) * (LB / 2) + c];
        acc[c].x += o.x;
        acc[c].y += o.y;
      }
#pragma unroll
    for (int c = 0; c < LB / 2; ++c) {
      if (2 * c < l) part[((int64_t)by * l + 2 * c) * v.I + i] = (double)acc[c].x;
      if (2 * c + 1 < l) part[((int64_t)by * l + 2 * c + 1) * v.I + i] = (double)acc[c].y;
    }
  }
  if (NORM) {
    nred[tid] = nrm;
    __syncthreads();
    for (int s2 = 128; s2 > 0; s2 >>= 1) {
      if (tid < s2 && tid + s2 < nthr) nred[tid] += nred[tid + s2];
      __syncthreads();
    }
    if (tid == 0) normpart[(int64_t)by * gx + bx] = nred[0];
  }
}
// U: loads in flight per thread (a tile-shape choice of the autotuner; the FMA
// order, and so every sum, is the same for each U).
template <int LMAX, int SRC, int U>
__global__ void __launch_bounds__(256, 3)
k_b_row_sweep(const BRowSweep* __restrict__ P, const BItem* __restrict__ items, int nitems,
              unsigned* counter, const float* const* __restrict__ xptrs) {
  __shared__ int item_sh;
  __shared__ __align__(16) float vs[kRowGroups * kRowTile * LMAX];
  __shared__ int64_t offs[kRowGroups * kRowTile];
  __shared__ int64_t offw[kRowGroups * kRowTile];
  __shared__ double nred[256];
  for (;;) {
    if (threadIdx.x == 0) item_sh = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int it = item_sh;
    __syncthreads();
    if (it >= nitems) break;
    const BItem w = items[it];
    const BRowSweep p = P[w.b];
    const float* T = p.T ? p.T : xptrs[w.b];  // mode 1 reads the caller's tensor
    // each tensor runs at its own padded width (FMAs on padding are wasted work)
    if (LMAX > 16 && p.l <= 16)
      row_sweep_body_grouped<16, SRC, U>(T, p.v, p.rows_per_cta, p.l, p.seed, p.sid, p.W,
                                         p.jchunk, p.part, p.normpart, w.bx, w.by, p.gx, vs,
                                         offs, offw, nred);
    else if (LMAX > 24 && p.l <= 24)
      row_sweep_body_grouped<24, SRC, U>(T, p.v, p.rows_per_cta, p.l, p.seed, p.sid, p.W,
                                         p.jchunk, p.part, p.normpart, w.bx, w.by, p.gx, vs,
                                         offs, offw, nred);
    else
      row_sweep_body_grouped<LMAX, SRC, U>(T, p.v, p.rows_per_cta, p.l, p.seed, p.sid, p.W,
                                           p.jchunk, p.part, p.normpart, w.bx, w.by, p.gx, vs,
                                           offs, offw, nred);
    __syncthreads();
  }
}

// Column sweep over the mode-1 unfolding of an FP32 tensor (L = 1: column j is
// the contiguous fibre X[:, j]): W[j, c] = sum_i X[i, j] Q[i, c] for the
// kProjThreads columns of block jb.  Q is staged in shared memory as FP32 rows
// of LB, once per call when I <= kBatchQRows, else kBatchQRows rows at a time.
// Rows of X are taken 16 at a time: each warp load covers the 16-row segments
// (64 contiguous bytes) of two columns; a thread holds the next chunk's 16
// values in registers while the current chunk, stored in a padded shared tile,
// is multiplied: thread t reads column t of the tile against the staged rows of
// Q, two columns of Q per packed FMA.  Each W[j, c] is one FMA chain over
// i = 0, 1, ...  sm holds kBatchQRows x LB floats of Q and the 16 x
// (kProjThreads + 1) tile.
constexpr int kFibRows = 16;
template <int LB>
__device__ __forceinline__ void col_sweep_fibres(const float* __restrict__ T, ModeView v, int l,
                                                 const double* __restrict__ Q,
                                                 float* __restrict__ W, int bx, int nb,
                                                 float* sm) {
  constexpr int NT = kProjThreads, TP = kProjThreads + 1, NW = NT / 32;
  constexpr int RC = kFibRows, NU = NT * RC / NT;  // values staged per thread per chunk
  float* Qs = sm;                     // kBatchQRows x LB
  float* Xt = Qs + kBatchQRows * LB;  // RC x TP
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int xr_row = lane & (RC - 1), xr_col = 2 * warp + (lane >> 4);  // + 2 NW u
  const int I = (int)v.I;
  // rows [p0, p0 + np) of Q into Qs (columns l..LB-1 zero)
  auto stage_q = [&](int p0, int np) {
    for (int k = tid; k < np * LB; k += NT) {
      const int c = k / np, ii = k - c * np;
      Qs[ii * LB + c] = c < l ? (float)Q[(p0 + ii) + (int64_t)I * c] : 0.0f;
    }
  };
  const bool qall = I <= kBatchQRows;
  if (qall) {
    __syncthreads();
    stage_q(0, I);
  }
  for (int64_t jb = bx; jb * NT < v.J; jb += nb) {
    const int64_t j0 = jb * NT, j = j0 + tid;
    float2 acc[LB / 2];
#pragma unroll
    for (int c = 0; c < LB / 2; ++c) acc[c] = make_float2(0.0f, 0.0f);
    auto load_x = [&](int i0, int iend, float (&xr)[NU]) {
      const bool row_ok = i0 + xr_row < iend;
#pragma unroll
      for (int u = 0; u < NU; ++u) {
        const int64_t col = j0 + xr_col + 2 * NW * u;
        xr[u] = (col < v.J && row_ok) ? __ldg(T + col * v.I + i0 + xr_row) : 0.0f;
      }
    };
    for (int p0 = 0; p0 < I; p0 += kBatchQRows) {
      const int np = min(kBatchQRows, I - p0);
      if (!qall) {
        __syncthreads();
        stage_q(p0, np);
      }
      float xr[NU];
      load_x(p0, p0 + np, xr);
      for (int i0 = 0; i0 < np; i0 += RC) {
        const int ni = min(RC, np - i0);
        __syncthreads();  // the previous chunk's tile reads (and Qs) are done
#pragma unroll
        for (int u = 0; u < NU; ++u) Xt[xr_row * TP + xr_col + 2 * NW * u] = xr[u];
        __syncthreads();
        if (i0 + RC < np) load_x(p0 + i0 + RC, p0 + np, xr);  // next chunk in flight
        const float* qrow = Qs + (qall ? p0 + i0 : i0) * LB;
        for (int ii = 0; ii < ni; ++ii) fma_row2<LB>(acc, Xt[ii * TP + tid], qrow + ii * LB);
      }
    }
    if (j < v.J) {
#pragma unroll
      for (int c = 0; c < LB / 2; ++c) {
        if (2 * c < l) W[2 * c + (int64_t)l * j] = acc[c].x;
        if (2 * c + 1 < l) W[2 * c + 1 + (int64_t)l * j] = acc[c].y;
      }
    }
  }
}

// One launch covers one mode of every tensor.  Mode 1 (FIB) reads contiguous fibres,
// each tensor at its own padded width; the other modes take the staged-Q column
// body (any L).
template <int LMAX, bool FIB>
__global__ void __launch_bounds__(kProjThreads, FIB ? 2 : 3)
k_b_col_sweep(const BColSweep* __restrict__ P, const BItem* __restrict__ items, int nitems,
              unsigned* counter, const float* const* __restrict__ xptrs) {
  extern __shared__ __align__(16) double b_col_sm[];
  __shared__ int item_sh;
  for (;;) {
    if (threadIdx.x == 0) item_sh = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int it = item_sh;
    __syncthreads();
    if (it >= nitems) break;
    const BItem w = items[it];
    const BColSweep p = P[w.b];
    const float* T = p.T ? p.T : xptrs[w.b];
    float* sm = reinterpret_cast<float*>(b_col_sm);
    if (FIB) {
      if (LMAX > 16 && p.l <= 16)
        col_sweep_fibres<16>(T, p.v, p.l, p.Q, p.W, w.bx, w.by, sm);
      else if (LMAX > 24 && p.l <= 24)
        col_sweep_fibres<24>(T, p.v, p.l, p.Q, p.W, w.bx, w.by, sm);
      else
        col_sweep_fibres<LMAX>(T, p.v, p.l, p.Q, p.W, w.bx, w.by, sm);
    } else {
      // Q staged 256 rows at a time: once per column block for I <= 256
      col_sweep_body<LMAX, float, float, false, kProjThreads, kBatchQRows>(
          T, p.v, p.l, p.Q, p.W, nullptr, w.bx, w.by);
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_b_row_sweep(const BRowSweep* P, const BItem* items, int nitems, unsigned* counter,
                               int lmax, bool use_w, int depth, const float* const* xptrs,
                               int grid, cudaStream_t s) {
  count_launches(1);
  // the batch's widths l <= 32 in buckets of 16, 24 and 32 columns (each thread
  // multiplies every staged column, so padding costs FMAs); depth 4 or 8 loads
  // in flight per thread
  const int b = lmax <= 16 ? 16 : lmax <= 24 ? 24 : lmax <= 32 ? 32 : 0;
  if (b == 0 || (depth != 4 && depth != 8)) return cudaErrorInvalidValue;
#define RCP_B_ROW(BB, SRC, U) k_b_row_sweep<BB, SRC, U><<<grid, 256, 0, s>>>(P, items, nitems, counter, xptrs)
#define RCP_B_ROW_U(BB, SRC)      \
  if (depth == 4) RCP_B_ROW(BB, SRC, 4); \
  else RCP_B_ROW(BB, SRC, 8);
  if (use_w) {
    if (b == 16) { RCP_B_ROW_U(16, kSrcW) }
    else if (b == 24) { RCP_B_ROW_U(24, kSrcW) }
    else { RCP_B_ROW_U(32, kSrcW) }
  } else {
    if (b == 16) { RCP_B_ROW_U(16, kSrcOmega) }
    else if (b == 24) { RCP_B_ROW_U(24, kSrcOmega) }
    else { RCP_B_ROW_U(32, kSrcOmega) }
  }
#undef RCP_B_ROW_U
#undef RCP_B_ROW
  return cudaGetLastError();
}

cudaError_t launch_b_col_sweep(const BColSweep* P, const BItem* items, int nitems, unsigned* counter,
                               int lmax, bool mode1, const float* const* xptrs, int grid,
                               cudaStream_t s) {
  count_launches(1);
  const int b = lmax <= 16 ? 16 : lmax <= 24 ? 24 : lmax <= 32 ? 32 : 0;
  // dynamic shared memory: the staged rows of Q (kBatchQRows x b) and, for the
  // fibre path, a kFibRows x (kProjThreads + 1) tile of X
  auto smem_for = [](int bb) {
    return ((size_t)kBatchQRows * bb + (size_t)kFibRows * (kProjThreads + 1)) * sizeof(float);
  };
  cudaError_t e = cudaSuccess;
#define RCP_B_COL(BB)                                                                          \
  do {                                                                                         \
    const size_t sm = smem_for(BB);                                                            \
    if (mode1) {                                                                               \
      e = cudaFuncSetAttribute(k_b_col_sweep<BB, true>,                                        \
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);          \
      if (e == cudaSuccess)                                                                    \
        k_b_col_sweep<BB, true><<<grid, kProjThreads, sm, s>>>(P, items, nitems, counter, xptrs); \
    } else {                                                                                   \
      e = cudaFuncSetAttribute(k_b_col_sweep<BB, false>,                                       \
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);          \
      if (e == cudaSuccess)                                                                    \
        k_b_col_sweep<BB, false><<<grid, kProjThreads, sm, s>>>(P, items, nitems, counter, xptrs); \
    }                                                                                          \
  } while (0)
  if (b == 16) RCP_B_COL(16);
  else if (b == 24) RCP_B_COL(24);
  else if (b == 32) RCP_B_COL(32);
  else return cudaErrorInvalidValue;
#undef RCP_B_COL
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

int sweep_rows_per_cta(int64_t I) {
  const int64_t nib = (I + 255) / 256;
  return (int)((I + nib - 1) / nib);
}

int sweep_row_blocks(int64_t I) { return (int)((I + 255) / 256); }

cudaError_t launch_sketch_f64(const void* T, int in_dtype, ModeView v, int l, uint64_t seed,
                              uint32_t stream_id, const double* W, int nsplit, double* part,
                              double* normpart, cudaStream_t s) {
  const int src = W ? kSrcW : kSrcOmega;
  if (in_dtype == RCP_DTYPE_F32)
    return row_sweep_any((const float*)T, v, l, seed, stream_id, W, nullptr, src, nsplit, part,
                         normpart, s);
  return row_sweep_any((const double*)T, v, l, seed, stream_id, W, nullptr, src, nsplit, part,
                       normpart, s);
}

cudaError_t launch_sketch_f32(const float* T, ModeView v, int l, uint64_t seed, uint32_t stream_id,
                              const float* W, int nsplit, double* part, double* normpart,
                              cudaStream_t s) {
  const int src = W ? kSrcW : kSrcOmega;
  return row_sweep_any(T, v, l, seed, stream_id, W, nullptr, src, nsplit, part, normpart, s);
}

cudaError_t launch_mttkrp_f64(const double* B, ModeView v, int R, const KrDims& kr, int nsplit,
                              double* part, cudaStream_t s) {
  return row_sweep_any(B, v, R, 0, 0, (const double*)nullptr, &kr, kSrcKr, nsplit, part, nullptr,
                       s);
}

cudaError_t launch_project_f64(const void* T, int in_dtype, ModeView v, int l, const double* Q,
                               double* W, double* gpart, int nblocks, cudaStream_t s) {
  if (in_dtype == RCP_DTYPE_F32)
    return col_sweep_any((const float*)T, v, l, Q, W, gpart, nblocks, s);
  return col_sweep_any((const double*)T, v, l, Q, W, gpart, nblocks, s);
}

cudaError_t launch_project_f32(const float* T, ModeView v, int l, const double* Q, float* W,
                               int nblocks, cudaStream_t s) {
  if (col_sweep_cb_fits(v, l)) {
    // nblocks counts CTAs of 256 columns; about nblocks / 4 * 4 >= SMs here
    int nsm = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return cudaErrorUnknown;
    switch ((l + 7) / 8) {
      case 1: return col_sweep_cb_typed<1>(T, v, l, Q, W, nsm, s);
      case 2: return col_sweep_cb_typed<2>(T, v, l, Q, W, nsm, s);
      case 3: return col_sweep_cb_typed<3>(T, v, l, Q, W, nsm, s);
      case 4: return col_sweep_cb_typed<4>(T, v, l, Q, W, nsm, s);
      case 5: return col_sweep_cb_typed<5>(T, v, l, Q, W, nsm, s);
      case 6: return col_sweep_cb_typed<6>(T, v, l, Q, W, nsm, s);
      case 7: return col_sweep_cb_typed<7>(T, v, l, Q, W, nsm, s);
      default: return col_sweep_cb_typed<8>(T, v, l, Q, W, nsm, s);
    }
  }
  return col_sweep_any(T, v, l, Q, W, (double*)nullptr, nblocks, s);
}

}  // namespace rcp

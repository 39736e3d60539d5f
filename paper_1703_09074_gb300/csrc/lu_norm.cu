// The pivoted-LU normalisation of Algorithm 1 steps 8-9, [Q, ~] = lu(Y): Q is
// the permuted unit lower-trapezoidal factor P L of the partial-pivoting
// factorisation Y = P L U (M x l, FP64, in place).  Element (j, c) sits at
// (j mod L) + L c + L l (j div L): L = M is the column-major sketch Y, L = 1 the
// row-major power-iteration W of mode 1, and in general the layout in which
// the project sweep writes W (the Kolda layout of T_{n+1}).  Its columns
// span the same space as Y's; the final QR of step 12 turns either basis into
// the same Q_n up to an l x l rotation, so this is the paper-literal variant of
// the CholeskyQR normalisation used by default.
//
// Rows are never swapped.  Step k picks the pivot among the rows not yet
// chosen (the largest |Y[i, k]|, the first on a tie, as LAPACK's getf2 does in
// its own row order), then every other unchosen row i takes the multiplier
// m_i = Y[i, k] / Y[p, k] (formed, as getf2 does, with the reciprocal of the
// pivot) into column k and subtracts m_i times the pivot row from its columns
// > k; the pivot row keeps its earlier multipliers, a 1 in column k and zeros
// to the right.  What is left is P L in the original row order.
//
//   k_lu_update  one launch per step over all rows (grid-stride): the update of
//                step k fused with each CTA's candidate pivot of step k + 1;
//   k_lu_pick    one CTA: the pivot of step k from the CTAs' candidates, and
//                the pivot row's entries k..l-1 for the update.
#include <math.h>

#include <algorithm>

#include "rcp_internal.cuh"

namespace rcp {
namespace {

constexpr int kLuT = 256;

struct LuArgs {
  double* Y;
  int64_t M;
  int l;
  int64_t L;         // inner block of the row index (see the layout above)
  uint8_t* used;     // M flags: row already chosen as a pivot
  double* cval;      // per-CTA candidate |value|
  int64_t* cidx;     // per-CTA candidate row
  double* prow;      // pivot row entries k..l-1 (prow[j]), and the pivot's row index at prow[l]
  DevState* st;
};

// keep (v, i) if it beats (bv, bi): larger |value|, the smaller row on a tie
__device__ __forceinline__ void better(double v, int64_t i, double& bv, int64_t& bi) {
  if (v > bv || (v == bv && i < bi)) {
    bv = v;
    bi = i;
  }
}

__device__ void cta_candidate(double bv, int64_t bi, double* cval, int64_t* cidx) {
  __shared__ double sv[kLuT / 32];
  __shared__ int64_t si[kLuT / 32];
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
    const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
    better(ov, oi, bv, bi);
  }
  if ((threadIdx.x & 31) == 0) {
    sv[threadIdx.x >> 5] = bv;
    si[threadIdx.x >> 5] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kLuT / 32; ++w) better(sv[w], si[w], bv, bi);
    cval[blockIdx.x] = bv;
    cidx[blockIdx.x] = bi;
  }
}

// k < 0: only the candidates of column 0 (all rows unchosen).
__global__ void __launch_bounds__(kLuT) k_lu_update(LuArgs a, int k) {
  const int l = a.l;
  const int64_t M = a.M;
  double rp = 0.0;
  int64_t p = -1;
  if (k >= 0) {
    p = (int64_t)a.prow[l];
    rp = 1.0 / a.prow[k];
  }
  double bv = -1.0;
  int64_t bi = INT64_MAX;
  const int64_t L = a.L;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ih = i / L;
    double* row = a.Y + (i - ih * L) + L * (int64_t)l * ih;  // column c at row[L c]
    if (k >= 0) {
      if (i == p) {
        row[L * k] = 1.0;
        for (int j = k + 1; j < l; ++j) row[L * j] = 0.0;
        continue;
      }
      if (a.used[i]) continue;
      const double m = row[L * k] * rp;
      row[L * k] = m;
      for (int j = k + 1; j < l; ++j) row[L * j] = fma(-m, a.prow[j], row[L * j]);
    } else if (a.used[i]) {
      continue;
    }
    if (k + 1 < l) better(fabs(row[L * (k + 1)]), i, bv, bi);
  }
  if (k + 1 < l) cta_candidate(bv, bi, a.cval, a.cidx);
}

__global__ void __launch_bounds__(kLuT) k_lu_pick(LuArgs a, int k, int nparts) {
  __shared__ int64_t piv_sh;
  double bv = -1.0;
  int64_t bi = INT64_MAX;
  for (int c = threadIdx.x; c < nparts; c += blockDim.x) better(a.cval[c], a.cidx[c], bv, bi);
  __shared__ double sv[kLuT / 32];
  __shared__ int64_t si[kLuT / 32];
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
    const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
    better(ov, oi, bv, bi);
  }
  if ((threadIdx.x & 31) == 0) {
    sv[threadIdx.x >> 5] = bv;
    si[threadIdx.x >> 5] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kLuT / 32; ++w) better(sv[w], si[w], bv, bi);
    if (!(bv > 0.0) || bi < 0 || bi >= a.M) {
      // no nonzero pivot left: Y is rank-deficient (or not finite)
      set_status(a.st, isfinite(bv) ? RCP_ESINGULAR : RCP_ENAN);
      bi = 0;
    }
    a.used[bi] = 1;
    piv_sh = bi;
    a.prow[a.l] = (double)bi;
  }
  __syncthreads();
  const int64_t p = piv_sh, ph = p / a.L;
  const double* row = a.Y + (p - ph * a.L) + a.L * (int64_t)a.l * ph;
  for (int j = k + threadIdx.x; j < a.l; j += blockDim.x) a.prow[j] = row[a.L * j];
}

}  // namespace

// In-place P L of Y (M x l FP64 in the layout above).  Scratch: used (M bytes),
// cval / cidx (2 nsm entries each), prow (l + 1 doubles).
cudaError_t launch_lu_norm(double* Y, int64_t M, int l, int64_t L, uint8_t* used, double* cval,
                           int64_t* cidx, double* prow, DevState* st, int nsm, cudaStream_t s) {
  LuArgs a{Y, M, l, L, used, cval, cidx, prow, st};
  const int grid = (int)std::min<int64_t>((M + kLuT - 1) / kLuT, 2 * (int64_t)nsm);
  cudaError_t e = cudaMemsetAsync(used, 0, (size_t)M, s);
  if (e != cudaSuccess) return e;
  count_launches(1);
  k_lu_update<<<grid, kLuT, 0, s>>>(a, -1);
  for (int k = 0; k < l; ++k) {
    count_launches(2);
    k_lu_pick<<<1, kLuT, 0, s>>>(a, k, grid);
    k_lu_update<<<grid, kLuT, 0, s>>>(a, k);
  }
  return cudaGetLastError();
}

}  // namespace rcp

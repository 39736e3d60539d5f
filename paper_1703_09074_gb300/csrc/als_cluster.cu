// CP-ALS on a small compressed tensor (Algorithm 2 steps 3-11) as ONE
// thread-block cluster, for the precision form (B in FP32, l_n <= 32, R <= 32,
// the whole core resident in shared memory).
//
// Every CTA of the cluster keeps its own copy of B (loaded once) and of every
// factor, so the mode-n update needs no cross-CTA reduction: CTA c owns the
// rows i = c, c + C, c + 2C, ... of the factor being updated.  Per mode update:
//
//   phase 1  nine warps (sub-partitions 1-3): MTTKRP rows M[i, :] = B_(n)[i, :]
//            (KR of the other factors) for the owned rows, in two stages
//            (Section 3.2.1): the inner sum over the first other mode a,
//              s[i, p, r] = sum_{i_a} B[.., i, .., i_a, .., p] A_a[i_a, r],
//            with one lane per multi-index p of the remaining modes, times the
//            remaining factors' Khatri-Rao row KR_p[r]; the 32 lanes' vectors
//            are then summed by a reduce-scatter so that lane r ends with
//            M[i, r].  FP32 products and sums (at most 32 terms per stage),
//            double-word accumulation across work items.
//            warp 0 (concurrently, alone on sub-partition 0): Z = V^{-1} by
//            Gauss-Jordan in FP32 registers, one row per lane, V the Hadamard
//            product of the other modes' Grams (Definition 2), built in double
//            word by the whole CTA at the end of the previous update.  V is
//            symmetric positive definite: no pivoting.  A pivot at or below
//            64 R u_32 trace(V) repeats it on V + s I with that shift s
//            (RCP_INFO_ALS_REGULARISED).
//   phase 2  warp j solves owned row j of x V = M (Definition 2): x0 = M Z,
//            then two steps of iterative refinement x <- x + (M - x V) Z whose
//            residual is a compensated dot product (Ogita, Rump & Oishi 2005)
//            over double-word x, V and M: each step multiplies the error by
//            about kappa(V) u_32, so the solve ends within about
//            (kappa u_32)^3 + kappa 2^-44 of the exact solution.
//   phase 3  each row (double word) goes to every CTA's shared memory through
//            distributed shared memory; one cluster barrier.
//   phase 4  every CTA, identically: column norms in double word, the column
//            normalisation of Algorithm 2 (lambda = the norms at n = N), the
//            FP32 copy for the next MTTKRPs, its Gram, V of the next update;
//            after mode N the fit of Section 3.3 and the stop rule.
//
// The receive buffers alternate between updates, so one cluster barrier per
// update orders every remote store after the readers of the buffer's previous
// contents.  Every CTA runs the same loop on the same data in the same order,
// so the stop decision is identical in all of them and every CTA reaches every
// cluster barrier: there is no spin-wait and no early exit.
#include <math.h>
#include <string.h>

#include "dw_arith.cuh"
#include "rcp_internal.cuh"

namespace rcp {
namespace {

// Twelve warps.  Warp w runs on sub-partition w % 4.  In phase 1 warp 0 (the
// latency-bound Gauss-Jordan chain) has sub-partition 0 to itself: warps 4 and
// 8 idle there, and the nine warps of sub-partitions 1-3 run the MTTKRP.
constexpr int kWarps = 12;
constexpr int kCThreads = kWarps * 32;
constexpr int kMW = 9;                       // MTTKRP warps
constexpr int kGP = 33;                      // row pitch of the FP32 Grams and of Z
constexpr int kFP = 33;                      // row pitch (float2) of the receive buffers
constexpr unsigned kFull = 0xffffffffu;

struct ClusterArgs {
  int N, R, C;
  int l[kMaxN];
  int S[kMaxN];          // shared-memory stride of each mode in the padded core
  int core_smem;         // floats of the padded core
  const float* B;        // compressed tensor, Kolda layout, FP32
  double* At[kMaxN];     // in: the caller's initial factors (user_init); out: final factors
  double* lam;           // out: lambda (R)
  float2* facdw;         // scratch: N x 32 x 32 double-word factors (written by CTA 0)
  DevState* st;
  uint64_t seed;
  double tol;
  int max_iters;
  int user_init;
  const int* user_init_dev;  // when set, a device word that replaces user_init
  int max_items;         // MTTKRP work items of the busiest mode (partial-result slots)
};

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// every thread of every CTA of the cluster; stores to shared memory (local or
// remote) made before the barrier are visible to every thread after it
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// the address of the same shared-memory location in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t remote_addr(uint32_t local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}

__device__ __forceinline__ void st_remote_f2(uint32_t addr, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y)
               : "memory");
}

__device__ __forceinline__ float fast_rcp(float p) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(p));
  return fmaf(r, fmaf(-p, r, 1.0f), r);  // one Newton step
}

__device__ __forceinline__ dwf ld_dw(const float2* p) {
  const float2 v = *p;
  return {v.x, v.y};
}

__device__ __forceinline__ void st_dw(float2* p, dwf v) { *p = make_float2(v.hi, v.lo); }

// Sum over the 32 lanes of v[0..31] with lane L receiving the total of v[L]:
// a reduce-scatter of five butterfly steps (31 shuffles).
template <int KR>
__device__ __forceinline__ float reduce_scatter32(const float (&acc)[KR], int lane) {
  float v[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = k < KR ? acc[k] : 0.0f;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < o; ++k) {
      const float send = up ? v[k] : v[k + o];
      const float keep = up ? v[k + o] : v[k];
      v[k] = keep + __shfl_xor_sync(kFull, send, o);
    }
  }
  return v[0];
}

// Double-word warp sum (every lane receives the total).
__device__ __forceinline__ dwf warp_sum_dw(dwf s) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const dwf t = {__shfl_xor_sync(kFull, s.hi, o), __shfl_xor_sync(kFull, s.lo, o)};
    s = dw_add(s, t);
  }
  return s;
}

// Shared-memory layout of one CTA (floats unless noted); identical on the host.
struct Layout {
  int F32, G32, Z, Vdw, Fdw, Macc, ipb, lamd, red, total;  // offsets in floats
};

__host__ __device__ inline Layout make_layout(int core_smem, int N, int KR, int max_items) {
  Layout L;
  int o = (core_smem + 3) & ~3;
  L.F32 = o;  o += N * 32 * KR;                 // FP32 factor copies, [i][r], pitch KR
  L.G32 = o;  o += N * 32 * kGP;                // FP32 Grams
  L.Z = o;    o += 32 * kGP;                    // FP32 V^{-1}
  o = (o + 3) & ~3;
  L.Vdw = o;  o += 2 * 32 * kFP;                // V, double word (row pitch kFP)
  L.Fdw = o;  o += 2 * 2 * 32 * kFP;            // two receive buffers of the new factor rows
  L.Macc = o; o += max_items * 32;              // one FP32 partial row per MTTKRP work item
  L.ipb = o;  o += 2 * 2 * 16;                  // <M, x> partial of each CTA, two buffers
  L.lamd = o; o += 2 * 32;                      // lambda, double word
  L.red = o;  o += 2 * 64;                      // 64 doubles of scratch
  L.total = o;
  return L;
}

// Work items of the MTTKRP of mode n for a CTA owning nrows rows: per row, PC
// chunks of 32 multi-indices p times S segments of the inner mode's range (S > 1
// only while there are fewer items than MTTKRP warps).
__host__ __device__ inline void mttkrp_items(const int* l, int N, int n, int nrows, int* PC,
                                             int* S) {
  const int am = n == 0 ? 1 : 0;
  int P = 1;
  for (int m = 0; m < N; ++m)
    if (m != n && m != am) P *= l[m];
  *PC = (P + 31) >> 5;
  const int base = nrows * *PC;
  const int la = l[am];
  *S = 1;
  if (base > 0 && base < kMW) {
    const int s1 = kMW / base, s2 = la >> 2;
    *S = s1 < (s2 > 1 ? s2 : 1) ? s1 : (s2 > 1 ? s2 : 1);
  }
}

// Phase 1, MTTKRP warps: rows crank + j C (j < nrows) of M = B_(n) KR.  Work
// items (row slot j, chunk of 32 multi-indices p, segment of the inner mode's
// range) are spread over the kMW MTTKRP warps; item t leaves its partial row
// (lane r: its part of M[i, r]) in slot t of Mpart; the items of row j are the
// PC S consecutive slots from j PC S.
// The item shape of mode n for this CTA (mttkrp_items: PC, S; P = the count of
// multi-indices p; seglen = ceil(l_am / S)) comes precomputed in mi.
template <int KR>
__device__ void mttkrp_rows(const ClusterArgs& a, int n, int nrows, int crank, const float* Bs,
                            const float* F32, float* Mpart, int warp, int lane, const int* mi) {
  const int N = a.N, C = a.C;
  const int am = n == 0 ? 1 : 0;  // the inner (first other) mode
  const int la = a.l[am];
  const int PC = mi[0], S = mi[1], P = mi[2], seglen = mi[3];
  const int nitems = nrows * PC * S;
  const int sa = a.S[am];
  for (int item = warp; item < nitems; item += kMW) {
    const int j = item / (PC * S);
    const int rem = item - j * (PC * S);
    const int pc = rem / S, seg = rem - pc * S;
    const int i = crank + j * C;
    const int p = pc * 32 + lane;
    const bool pv = p < P;
    int off = i * a.S[n];
    {
      int q = pv ? p : 0;
      for (int m = 0; m < N; ++m) {
        if (m == n || m == am) continue;
        const int lm = a.l[m];
        const int d = q % lm;
        q /= lm;
        off += d * a.S[m];
      }
    }
    float acc[KR];
#pragma unroll
    for (int r = 0; r < KR; ++r) acc[r] = 0.0f;
    const int ia0 = seg * seglen, ia1 = min(la, ia0 + seglen);
    const float* fa = F32 + am * 32 * KR;
    for (int ia = ia0; ia < ia1; ++ia) {
      const float b = pv ? Bs[off + ia * sa] : 0.0f;
      const float4* Ar = (const float4*)(fa + ia * KR);
#pragma unroll
      for (int q = 0; q < KR / 4; ++q) {
        const float4 v = Ar[q];
        acc[4 * q] = fmaf(b, v.x, acc[4 * q]);
        acc[4 * q + 1] = fmaf(b, v.y, acc[4 * q + 1]);
        acc[4 * q + 2] = fmaf(b, v.z, acc[4 * q + 2]);
        acc[4 * q + 3] = fmaf(b, v.w, acc[4 * q + 3]);
      }
    }
    // times the Khatri-Rao row of the remaining modes at p (digits formed again,
    // which keeps them out of a dynamically indexed array)
    int q = pv ? p : 0;
    for (int m = 0; m < N; ++m) {
      if (m == n || m == am) continue;
      const int lm = a.l[m];
      const int d = q % lm;
      q /= lm;
      const float4* Fr = (const float4*)(F32 + (m * 32 + d) * KR);
#pragma unroll
      for (int q = 0; q < KR / 4; ++q) {
        const float4 v = Fr[q];
        acc[4 * q] *= v.x;
        acc[4 * q + 1] *= v.y;
        acc[4 * q + 2] *= v.z;
        acc[4 * q + 3] *= v.w;
      }
    }
    Mpart[item * 32 + lane] = reduce_scatter32<KR>(acc, lane);
  }
}

// Gauss-Jordan inverse of the SPD matrix V held one row per lane (a[c]; lanes
// and columns >= R hold the identity), FP32, no pivoting (every pivot of an SPD
// matrix is a positive Schur-complement diagonal).  z receives the rows of
// V^{-1}.  Step k broadcasts the pivot row (lane k) by shuffles and updates
// every row at once: row_i -= f_i row_k with f_k = 1 - 1/a_kk, which scales the
// pivot row itself (no select).  The steps are instantiated recursively so
// that every register index is a constant; gj_warp returns false if a pivot is
// at or below floor_ or not finite (the same answer in every lane).
template <int KR, int K>
__device__ __forceinline__ void gj_steps(float (&a)[KR], float (&z)[KR], int R, float floor_,
                                         int lane, bool& ok) {
  if constexpr (K < KR) {
    // Steps K >= R (at most 3: KR is R rounded up to a multiple of 4) act on the
    // identity padding with every multiplier forced to zero: exact no-ops.  Running
    // them unguarded keeps the steps one straight line, so the shuffles of step K + 1
    // can issue while step K finishes.
    const float piv = __shfl_sync(kFull, a[K], K);
    ok = ok && (K >= R || piv > floor_);
    const float rp = fast_rcp(piv);
    const float f = K >= R ? 0.0f : (lane == K ? 1.0f - rp : a[K] * rp);
#pragma unroll
    for (int c = K + 1; c < KR; ++c) a[c] = fmaf(-f, __shfl_sync(kFull, a[c], K), a[c]);
#pragma unroll
    for (int c = 0; c <= K; ++c) z[c] = fmaf(-f, __shfl_sync(kFull, z[c], K), z[c]);
    gj_steps<KR, K + 1>(a, z, R, floor_, lane, ok);
  }
}

template <int KR>
__device__ bool gj_warp(float (&a)[KR], float (&z)[KR], int R, float floor_, int lane) {
#pragma unroll
  for (int c = 0; c < KR; ++c) z[c] = c == lane ? 1.0f : 0.0f;
  bool ok = true;
  gj_steps<KR, 0>(a, z, R, floor_, lane, ok);
  return ok;
}

// V for mode n, the Hadamard product of the other modes' FP32 Grams
// (Definition 2), in double word (exact for N = 3) into Vdw (row pitch kFP).
// Run by the whole CTA as soon as the last of those Grams is known, so the
// solver warp of the next phase 1 starts from it.
__device__ __forceinline__ void build_V(int N, int R, int n, const float* G32, float2* Vdw,
                                        int tid) {
  // the Grams are exactly symmetric (gram_f32), so V is: its upper triangle (at most
  // 528 entries: one or two per thread), each entry stored twice
  for (int e = tid; e < R * (R + 1) / 2; e += kCThreads) {
    int c = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while (c * (c + 1) / 2 > e) --c;
    while ((c + 1) * (c + 2) / 2 <= e) ++c;
    const int r = e - c * (c + 1) / 2;  // r <= c
    dwf w = {1.0f, 0.0f};
    bool first = true;
    for (int m = 0; m < N; ++m) {
      if (m == n) continue;
      const float g = G32[m * 32 * kGP + r * kGP + c];
      w = first ? dwf{g, 0.0f} : dw_mul(w, {g, 0.0f});
      first = false;
    }
    st_dw(&Vdw[r * kFP + c], w);
    if (r != c) st_dw(&Vdw[c * kFP + r], w);
  }
}

// Phase 1, solver warp: the FP32 inverse Z of V (Vdw, built beforehand).  Returns the RCP_INFO bits to add (regularised) or -1 when V
// is not finite.
template <int KR>
__device__ int build_and_invert(const ClusterArgs& a, int n, const float* G32, float* Z,
                                float2* Vdw, int lane) {
  const int R = a.R;
  float v[KR];
  float diag = 0.0f;
#pragma unroll
  for (int c = 0; c < KR; ++c) {
    v[c] = (lane < R && c < R) ? Vdw[lane * kFP + c].x : (c == lane ? 1.0f : 0.0f);
    if (c == lane && lane < R) diag = v[c];
  }
  float tr = diag;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) tr += __shfl_xor_sync(kFull, tr, o);
  if (!isfinite(tr)) return -1;
  const float floor_ = 64.0f * (float)R * 5.9604645e-08f * tr;
  float z[KR];
  int info = 0;
  float keep[KR];
#pragma unroll
  for (int c = 0; c < KR; ++c) keep[c] = v[c];
  bool ok = gj_warp<KR>(v, z, R, floor_, lane);
  if (!__all_sync(kFull, ok)) {
    // numerically singular at FP32: invert V + s I; the refinement against V
    // itself still converges (its error factor is s / (lambda_i + s) < 1)
#pragma unroll
    for (int c = 0; c < KR; ++c) v[c] = keep[c] + ((c == lane && lane < R) ? floor_ : 0.0f);
    ok = gj_warp<KR>(v, z, R, 0.0f, lane);
    info = RCP_INFO_ALS_REGULARISED;
    if (!__all_sync(kFull, ok)) return -1;
  }
  if (lane < R) {
#pragma unroll
    for (int c = 0; c < KR; ++c)
      if (c < R) Z[lane * kGP + c] = z[c];
  }
  return info;
}

// Phase 2 for one owned row, by one warp (lane c holds column c; lanes >= R
// hold zeros): x V = m with m the row of M, Z ~ V^{-1} (FP32) and V in double
// word.  x0 = m Z; then twice x <- x + (m - x V) Z, the residual formed as a
// compensated dot product (Ogita, Rump & Oishi 2005): the leading products
// x.hi V.hi are split exactly (FMA) and summed with TwoSum, their errors and
// the cross terms collect in FP32.  Every operand of another lane comes by a
// shuffle, so the row needs no CTA barrier.
template <int KR>
__device__ __forceinline__ dwf solve_row(dwf m, const float* Z, const float2* Vdw, int R,
                                         int lane) {
  const bool on = lane < R;
  const int cz = on ? lane : 0;  // lanes >= R read a valid column and are zeroed below
  // The k loops run to the compile-time bound KR with no guard, so that their
  // shuffles and shared loads issue ahead of the dependent arithmetic (one solving
  // warp per sub-partition leaves nothing else to hide their latency).  For k >= R
  // every operand is zero (lanes >= R hold zeros; rows >= R of Z and V are zeroed
  // at the start), and the sums are unchanged.
  float xa = 0.0f, xb = 0.0f;
#pragma unroll
  for (int k = 0; k < KR; ++k) {
    const float mk = __shfl_sync(kFull, m.hi, k);
    if (k & 1) xb = fmaf(mk, Z[k * kGP + cz], xb);
    else xa = fmaf(mk, Z[k * kGP + cz], xa);
  }
  dwf x = on ? dw_fast_two_sum(xa, xb) : dwf{0.0f, 0.0f};
#pragma unroll 1
  for (int step = 0; step < 2; ++step) {
    float s = m.hi, c0 = m.lo, c1 = 0.0f;
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      const float xh = __shfl_sync(kFull, x.hi, k);
      const float xl = __shfl_sync(kFull, x.lo, k);
      const float2 v = Vdw[k * kFP + cz];
      const float ph = __fmul_rn(xh, v.x);
      const float pl = __fmaf_rn(xh, v.x, -ph);
      const dwf t = dw_two_sum(s, -ph);
      s = t.hi;
      const float e = __fsub_rn(t.lo, __fadd_rn(pl, __fmaf_rn(xh, v.y, __fmul_rn(xl, v.x))));
      if (k & 1) c1 = __fadd_rn(c1, e);
      else c0 = __fadd_rn(c0, e);
    }
    const dwf r = on ? dw_two_sum(s, __fadd_rn(c0, c1)) : dwf{0.0f, 0.0f};  // s may have cancelled below c
    float da = 0.0f, db = 0.0f;
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      const float rk = __shfl_sync(kFull, r.hi, k);
      if (k & 1) db = fmaf(rk, Z[k * kGP + cz], db);
      else da = fmaf(rk, Z[k * kGP + cz], da);
    }
    x = on ? dw_add(x, {__fadd_rn(da, db), 0.0f}) : dwf{0.0f, 0.0f};
  }
  return x;
}

// Gram of mode m's FP32 factor copy: thread t forms the 2 x 2 block (rows 2 br,
// 2 br + 1; columns 2 bc, 2 bc + 1) from two 8-byte loads per row of the factor
// (columns >= R of the copy are zero).  Both halves are formed with the same
// products in the same order, so the matrix is exactly symmetric.
template <int KR>
__device__ __forceinline__ void gram_f32(const float* F32, float* G32, int m, int lm, int R,
                                         int tid) {
  const float* F = F32 + m * 32 * KR;
  float* G = G32 + m * 32 * kGP;
  const int nb = (R + 1) >> 1;
  for (int e = tid; e < nb * nb; e += kCThreads) {
    const int br = e / nb, bc = e - br * nb;
    float s00 = 0.0f, s01 = 0.0f, s10 = 0.0f, s11 = 0.0f;
    // all 32 rows, unguarded: rows >= lm are zero, so the sums are unchanged, and the
    // loads of later rows issue ahead of the dependent FMAs
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const float2 u = *(const float2*)(F + i * KR + 2 * br);
      const float2 v = *(const float2*)(F + i * KR + 2 * bc);
      s00 = fmaf(u.x, v.x, s00);
      s01 = fmaf(u.x, v.y, s01);
      s10 = fmaf(u.y, v.x, s10);
      s11 = fmaf(u.y, v.y, s11);
    }
    const int r = 2 * br, c = 2 * bc;
    G[r * kGP + c] = s00;
    if (c + 1 < R) G[r * kGP + c + 1] = s01;
    if (r + 1 < R) {
      G[(r + 1) * kGP + c] = s10;
      if (c + 1 < R) G[(r + 1) * kGP + c + 1] = s11;
    }
  }
}

template <int KR>
__device__ __forceinline__ void als_cluster_body(const ClusterArgs& a) {
  extern __shared__ __align__(16) float smem[];
  __shared__ int sh_info, sh_bad, sh_done;
  __shared__ float2 ipr[32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = a.N, R = a.R, C = a.C;
  const int crank = (int)cluster_rank();
  const Layout Ly = make_layout(a.core_smem, N, KR, a.max_items);
  float* Bs = smem;
  float* F32 = smem + Ly.F32;
  float* G32 = smem + Ly.G32;
  float* Z = smem + Ly.Z;
  float2* Vdw = (float2*)(smem + Ly.Vdw);
  float2* Fdw = (float2*)(smem + Ly.Fdw);
  float* Mpart = smem + Ly.Macc;
  float2* ipb = (float2*)(smem + Ly.ipb);
  float2* lamd = (float2*)(smem + Ly.lamd);
  double* red = (double*)(smem + Ly.red);
  DevState* st = a.st;
  // MTTKRP warps: the nine warps of sub-partitions 1-3
  const int mw = (warp & 3) ? (warp >> 2) * 3 + (warp & 3) - 1 : -1;

  // rows and columns of Z and V at or beyond R stay zero (the row solves run over them)
  for (int e = tid; e < 32 * kGP; e += kCThreads) Z[e] = 0.0f;
  for (int e = tid; e < 32 * kFP; e += kCThreads) Vdw[e] = make_float2(0.0f, 0.0f);
  // remote stores below need every CTA of the cluster to be running
  cluster_sync();

  // per mode, this CTA's owned rows and MTTKRP item shape (mttkrp_rows), formed once
  __shared__ int mish[kMaxN][5];  // PC, S, P, seglen, nrows
  if (tid < N) {
    const int n = tid, ln = a.l[n];
    const int nrows = ln > crank ? (ln - crank + C - 1) / C : 0;
    int PC, S;
    mttkrp_items(a.l, N, n, nrows, &PC, &S);
    const int am = n == 0 ? 1 : 0;
    int P = 1;
    for (int m = 0; m < N; ++m)
      if (m != n && m != am) P *= a.l[m];
    mish[n][0] = PC;
    mish[n][1] = S;
    mish[n][2] = P;
    mish[n][3] = (a.l[am] + S - 1) / S;
    mish[n][4] = nrows;
  }
  // ---- the core, into the padded layout; |B|^2 in double word
  int total = 1;
  for (int m = 0; m < N; ++m) total *= a.l[m];
  dwf nb = {0.0f, 0.0f};
  for (int e = tid; e < total; e += kCThreads) {
    int q = e, off = 0;
    for (int m = 0; m < N; ++m) {
      const int d = q % a.l[m];
      q /= a.l[m];
      off += d * a.S[m];
    }
    const float b = a.B[e];
    Bs[off] = b;
    const float bb = __fmul_rn(b, b);
    nb = dw_add(nb, {bb, __fmaf_rn(b, b, -bb)});
  }
  // ---- initial factors of modes 2..N: the caller's, or the seeded N(0,1)
  // stream drawn row-major (l_m x R), as FP32 copies (entries r >= R zero;
  // mode 1 starts at zero and is computed first)
  // (rows i >= l_m of every mode stay zero too: the Gram runs over all 32 rows)
  for (int e = tid; e < N * 32 * KR; e += kCThreads) F32[e] = 0.0f;
  __syncthreads();
  const int user_init = a.user_init_dev ? *a.user_init_dev : a.user_init;
  for (int m = 1; m < N; ++m) {
    const int lm = a.l[m];
    for (int e = tid; e < lm * KR; e += kCThreads) {
      const int i = e / KR, r = e - i * KR;
      float v = 0.0f;
      if (r < R) {
        double d;
        if (user_init) {
          d = a.At[m][i + lm * r];
        } else {
          const int g = i * R + r;
          const double2 zz = normal_pair_f64(a.seed, (uint32_t)(m + 1), kPurposeAlsInit,
                                             (uint64_t)(g >> 1));
          d = (g & 1) ? zz.y : zz.x;
        }
        v = (float)d;
      }
      F32[(m * 32 + i) * KR + r] = v;
    }
  }
  nb = warp_sum_dw(nb);
  if (lane == 0) {
    red[2 * warp] = (double)nb.hi;
    red[2 * warp + 1] = (double)nb.lo;
  }
  if (tid == 0) {
    sh_info = 0;
    sh_bad = 0;
    sh_done = 0;
  }
  __syncthreads();
  for (int m = 1; m < N; ++m) gram_f32<KR>(F32, G32, m, a.l[m], R, tid);
  double nb2 = 0.0;
  for (int w = 0; w < kWarps; ++w) nb2 += red[2 * w] + red[2 * w + 1];
  // |B|^2 and its reciprocal in double word for the per-sweep fit (FP64
  // instructions are long-latency on this part; the fit's chain stays in FP32)
  const dwf nb2_dw = dw_from_double(nb2);
  const dwf inv_nb2 = dw_rcp(nb2_dw);
  __syncthreads();
  build_V(N, R, 0, G32, Vdw, tid);
  __syncthreads();

  dwf rho_prev = {0.0f, 0.0f};
  int buf = 0, done = 0;
  for (int it = 1; it <= a.max_iters && !done; ++it) {
    for (int n = 0; n < N; ++n) {
      const int ln = a.l[n];
      const int nrows = mish[n][4];
      // ---- phase 1: MTTKRP of the owned rows || V and its inverse
      if (mw >= 0) {
        mttkrp_rows<KR>(a, n, nrows, crank, Bs, F32, Mpart, mw, lane, mish[n]);
      } else if (warp == 0) {
        const int inf = build_and_invert<KR>(a, n, G32, Z, Vdw, lane);
        if (lane == 0) {
          if (inf < 0) sh_bad = 1;
          else sh_info |= inf;
        }
      }
      __syncthreads();
      // ---- phase 2 + 3: warp w solves owned rows w, w + 12, ... and stores them into every CTA
      float2* fd = Fdw + buf * 32 * kFP;
      const int per_row = mish[n][0] * mish[n][1];
      for (int j = warp; j < nrows; j += kWarps) {
        const int i = crank + j * C;
        dwf m = {0.0f, 0.0f};
        if (lane < R)  // the row's partials in slot order, summed in double word
          for (int q = 0; q < per_row; ++q) {
            const float v = Mpart[(j * per_row + q) * 32 + lane];
            m = q == 0 ? dwf{v, 0.0f} : dw_add(m, {v, 0.0f});
          }
        const dwf x = solve_row<KR>(m, Z, Vdw, R, lane);
        if (lane < R) {
          const uint32_t loc = smem_addr(&fd[i * kFP + lane]);
          for (int d = 0; d < C; ++d) st_remote_f2(remote_addr(loc, (uint32_t)d), make_float2(x.hi, x.lo));
        }
        if (n == N - 1) {
          const dwf ipv = warp_sum_dw(lane < R ? dw_mul(m, x) : dwf{0.0f, 0.0f});
          if (lane == 0) ipr[j] = make_float2(ipv.hi, ipv.lo);
        }
      }
      if (n == N - 1) {
        // <M, x> of this CTA's rows into every CTA
        __syncthreads();
        if (warp == 0) {
          dwf ip = {0.0f, 0.0f};
          for (int j = 0; j < nrows; ++j) ip = dw_add(ip, ld_dw(&ipr[j]));
          const uint32_t loc = smem_addr(ipb + buf * 16 + crank);
          if (lane < C) st_remote_f2(remote_addr(loc, (uint32_t)lane), make_float2(ip.hi, ip.lo));
        }
      }
      cluster_sync();
      // ---- phase 4 (identical in every CTA): column norms, normalisation, FP32 copy
      {
        // warp w: columns w, w + 12, w + 24 (those below R; the count is warp-uniform)
        const int ncol = warp < R ? (R - warp + kWarps - 1) / kWarps : 0;
        dwf xv[3], nu2[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          const int r = warp + kWarps * t;
          xv[t] = (t < ncol && lane < ln) ? ld_dw(&fd[lane * kFP + r]) : dwf{0.0f, 0.0f};
          nu2[t] = dw_mul(xv[t], xv[t]);
        }
        if (ncol > 2) {
          nu2[0] = warp_sum_dw(nu2[0]);
          nu2[1] = warp_sum_dw(nu2[1]);
          nu2[2] = warp_sum_dw(nu2[2]);
        } else if (ncol == 2) {
          nu2[0] = warp_sum_dw(nu2[0]);
          nu2[1] = warp_sum_dw(nu2[1]);
        } else if (ncol == 1) {
          nu2[0] = warp_sum_dw(nu2[0]);
        }
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          const int r = warp + kWarps * t;
          if (t < ncol) {
            const bool pos = nu2[t].hi > 0.0f;
            const dwf nu = pos ? dw_sqrt(nu2[t]) : dwf{0.0f, 0.0f};
            const dwf inv = pos ? dw_rcp(nu) : dwf{0.0f, 0.0f};   // a zero column stays zero
            if (lane < ln) {
              const dwf av = dw_mul(xv[t], inv);
              F32[(n * 32 + lane) * KR + r] = av.hi;
              if (crank == 0) a.facdw[(n * 32 + lane) * 32 + r] = make_float2(av.hi, av.lo);
            }
            if (n == N - 1 && lane == 0) st_dw(&lamd[r], nu);
          }
        }
      }
      __syncthreads();
      gram_f32<KR>(F32, G32, n, ln, R, tid);
      __syncthreads();
      // V of the next mode update: every Gram it needs is final now
      build_V(N, R, n + 1 < N ? n + 1 : 0, G32, Vdw, tid);
      __syncthreads();
      if (n == N - 1) {
        // ---- fit of Section 3.3 on B: |Bhat|^2 = lambda^T (Hadamard product of
        // the Grams) lambda, <Bhat, B> = sum over rows of <M_N, x>
        dwf bh = {0.0f, 0.0f};
        for (int e = tid; e < R * R; e += kCThreads) {
          const int r = e / R, c = e - r * R;
          dwf g = {G32[r * kGP + c], 0.0f};
          for (int m = 1; m < N; ++m) g = dw_mul(g, {G32[m * 32 * kGP + r * kGP + c], 0.0f});
          bh = dw_add(bh, dw_mul(g, dw_mul(ld_dw(&lamd[r]), ld_dw(&lamd[c]))));
        }
        bh = warp_sum_dw(bh);
        float2* red2 = (float2*)red;
        if (lane == 0) red2[warp] = make_float2(bh.hi, bh.lo);
        __syncthreads();
        if (warp == 0) {
          // rho = 1 - (|B|^2 + |Bhat|^2 - 2 <Bhat, B>) / |B|^2, in double word
          const dwf bhat = warp_sum_dw(lane < kWarps ? ld_dw(&red2[lane]) : dwf{0.0f, 0.0f});
          const dwf ip = warp_sum_dw(lane < C ? ld_dw(&ipb[buf * 16 + lane]) : dwf{0.0f, 0.0f});
          if (lane == 0) {
            const dwf resid = dw_add(dw_add(nb2_dw, bhat), {-2.0f * ip.hi, -2.0f * ip.lo});
            const dwf rho = dw_add({1.0f, 0.0f}, dw_neg(dw_mul(resid, inv_nb2)));
            const dwf drho = dw_add(rho, dw_neg(rho_prev));
            const bool fin = isfinite(rho.hi) && isfinite(rho.lo);
            const bool conv = fabs((double)drho.hi + (double)drho.lo) < a.tol;
            int dn = conv ? 1 : (it >= a.max_iters ? 2 : 0);
            if (!fin || sh_bad) dn = 3;
            rho_prev = rho;
            sh_done = dn;
            if (crank == 0) {
              const double rhod = dw_to_double(rho);
              st->fit = rhod;
              st->ip = dw_to_double(ip);
              st->fit_prev = rhod;
              st->als_iters = it;
              st->norm_b2 = nb2;
              if (!fin || sh_bad) set_status(st, RCP_ENAN);
              if (dn) st->als_done = dn == 3 ? 2 : dn;
            }
          }
        }
        __syncthreads();
        done = sh_done;
      }
      buf ^= 1;
    }
  }
  // ---- results (CTA 0): FP64 factors, lambda, information bits
  if (crank == 0) {
    for (int m = 0; m < N; ++m) {
      const int lm = a.l[m];
      for (int e = tid; e < lm * R; e += kCThreads) {
        const int r = e / lm, i = e - r * lm;
        const float2 v = a.facdw[(m * 32 + i) * 32 + r];
        a.At[m][i + lm * r] = (double)v.x + (double)v.y;
      }
    }
    for (int r = tid; r < R; r += kCThreads) a.lam[r] = dw_to_double(ld_dw(&lamd[r]));
    if (tid == 0 && sh_info) atomicOr(&st->info, sh_info);
  }
}

template <int KR>
__global__ void __launch_bounds__(kCThreads, 1) k_als_cluster(ClusterArgs a) {
  als_cluster_body<KR>(a);
}

// the core's padded strides: S_1 = 1, S_{m+1} = S_m l_m rounded up to odd, so
// that lanes stepping along any one mode hit distinct banks
int pad_strides(const int* l, int N, int* S) {
  int s = 1;
  for (int m = 0; m < N; ++m) {
    S[m] = s;
    s *= l[m];
    if (m + 1 < N && !(s & 1)) s += 1;
  }
  return s;
}

// Width KR of the register blocks over the rank (every loop over r runs to KR): R
// rounded up to a multiple of 4 (the float4 loads), at least 8.  The batched kernel
// keeps buckets of 8, for fewer instantiations.
int kr_for(int R) { return R <= 8 ? 8 : (R + 3) & ~3; }
int kr_batched(int R) { return R <= 8 ? 8 : R <= 16 ? 16 : R <= 24 ? 24 : 32; }

// Shape-dependent fields of the arguments (widths, cluster size, padded
// strides, work-item slots) and the dynamic shared memory for KR accumulators.
size_t cluster_shape(int N, int R, const int* l, int cmax, ClusterArgs* a, int KR) {
  ClusterArgs t{};
  ClusterArgs* q = a ? a : &t;
  q->N = N;
  q->R = R;
  int lmax = 1;
  for (int m = 0; m < N; ++m) {
    q->l[m] = l[m];
    lmax = lmax > l[m] ? lmax : l[m];
  }
  q->C = lmax < cmax ? lmax : cmax;
  q->core_smem = pad_strides(l, N, q->S);
  int items = 1;
  for (int n = 0; n < N; ++n) {
    const int nrows = (l[n] + q->C - 1) / q->C;  // CTA 0 owns the most rows
    int PC, S;
    mttkrp_items(l, N, n, nrows, &PC, &S);
    items = items > nrows * PC * S ? items : nrows * PC * S;
  }
  q->max_items = items;
  const Layout L = make_layout(q->core_smem, N, KR, items);
  return (size_t)L.total * sizeof(float);
}

template <int KR>
cudaError_t launch_kr(const ClusterArgs& a, size_t smem, cudaStream_t s) {
  const void* kern = (const void*)k_als_cluster<KR>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.C);
  cfg.blockDim = dim3(kCThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = a.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launches(1);
  return cudaLaunchKernelEx(&cfg, k_als_cluster<KR>, a);
}

// Batched form: CTA b runs the whole ALS of problem b as a cluster of one CTA
// (C = 1: every row owned, the "remote" stores land in its own shared memory).
template <int KR>
__global__ void __launch_bounds__(kCThreads, 1) k_als_cluster_batched(const ClusterArgs* args) {
  als_cluster_body<KR>(args[blockIdx.x]);
}

}  // namespace

// True when the one-cluster kernel serves this plan: the precision form, every
// l_n <= 32, R <= 32 and the padded core with the rest in one CTA's shared memory.
bool als_cluster_fits(const rcp_plan_s* p) {
  if (p->prec != RCP_PREC_MIXED || p->N < 2 || p->R > 32) return false;
  for (int m = 0; m < p->N; ++m)
    if (p->l[m] > 32) return false;
  if (p->core_elems >= (1LL << 20)) return false;
  return cluster_shape(p->N, p->R, p->l, 8, nullptr, kr_for(p->R)) <= 220 * 1024;
}

cudaError_t launch_als_cluster(rcp_plan_s* p, const float* B, const int* user_init_dev,
                               cudaStream_t s) {
  ClusterArgs a{};
  const size_t smem = cluster_shape(p->N, p->R, p->l, 8, &a, kr_for(p->R));
  a.user_init_dev = user_init_dev;
  for (int m = 0; m < p->N; ++m) a.At[m] = p->At[m];
  a.B = B;
  a.lam = p->lam;
  a.facdw = (float2*)p->part;
  a.st = p->dstate;
  a.seed = p->cfg.seed;
  a.tol = p->cfg.tol;
  a.max_iters = p->cfg.max_iters;
  a.user_init = p->user_init ? 1 : 0;
  switch (kr_for(p->R)) {
    case 8: return launch_kr<8>(a, smem, s);
    case 12: return launch_kr<12>(a, smem, s);
    case 16: return launch_kr<16>(a, smem, s);
    case 20: return launch_kr<20>(a, smem, s);
    case 24: return launch_kr<24>(a, smem, s);
    case 28: return launch_kr<28>(a, smem, s);
    default: return launch_kr<32>(a, smem, s);
  }
}

// Arguments of problem b of a batch for k_als_cluster_batched: written into
// *out (host); returns its shared-memory need for KR = kr_batched(rmax), or 0 when
// the problem is beyond the kernel (some l_n > 32).
size_t cluster_batched_args(int N, int R, const int* l, int rmax, const float* B,
                            double* const* At, double* lam, float2* facdw, DevState* st,
                            uint64_t seed, double tol, int max_iters, const int* user_init_dev,
                            void* out) {
  for (int m = 0; m < N; ++m)
    if (l[m] > 32) return 0;
  ClusterArgs a{};
  const size_t smem = cluster_shape(N, R, l, 1, &a, kr_batched(rmax));
  for (int m = 0; m < N; ++m) a.At[m] = At[m];
  a.B = B;
  a.lam = lam;
  a.facdw = facdw;
  a.st = st;
  a.seed = seed;
  a.tol = tol;
  a.max_iters = max_iters;
  a.user_init = 0;
  a.user_init_dev = user_init_dev;
  memcpy(out, &a, sizeof(a));
  return smem;
}

size_t cluster_args_bytes() { return sizeof(ClusterArgs); }

// Shared-memory limit of the batched kernel for this batch (once, at plan time:
// the launch below may be captured into a graph).
cudaError_t prepare_als_cluster_batched(int rmax, size_t smem) {
  const int kr = kr_batched(rmax);
  const void* kern = kr == 8 ? (const void*)k_als_cluster_batched<8>
                   : kr == 16 ? (const void*)k_als_cluster_batched<16>
                   : kr == 24 ? (const void*)k_als_cluster_batched<24>
                              : (const void*)k_als_cluster_batched<32>;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_als_cluster_batched(const void* dev_args, int count, int rmax, size_t smem,
                                       cudaStream_t s) {
  const ClusterArgs* args = (const ClusterArgs*)dev_args;
  const int kr = kr_batched(rmax);
  count_launches(1);
  if (kr == 8) k_als_cluster_batched<8><<<count, kCThreads, smem, s>>>(args);
  else if (kr == 16) k_als_cluster_batched<16><<<count, kCThreads, smem, s>>>(args);
  else if (kr == 24) k_als_cluster_batched<24><<<count, kCThreads, smem, s>>>(args);
  else k_als_cluster_batched<32><<<count, kCThreads, smem, s>>>(args);
  return cudaGetLastError();
}

}  // namespace rcp

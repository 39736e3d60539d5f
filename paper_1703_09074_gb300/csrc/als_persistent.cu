// CP-ALS on the compressed tensor B (Algorithm 2 steps 3-11) as one persistent
// cooperative kernel: every sweep of every mode runs without a host round trip.
//
// Per mode n (1-based in the paper, n0 = n - 1 here):
//   phase A (all CTAs): MTTKRP partials  M_g = B_(n)[:, cols of g] KR[cols of g, :]
//             where KR is the Khatri-Rao product of the other factors (built per
//             column tile from the factor copies in shared memory);
//   barrier;
//   phase B (row owners): M[i, :] = sum_g M_g[i, :] in fixed order, then the
//             row of Definition 2's solve x = M[i, :] V^{-1} with V the Hadamard
//             product of the other Grams.  R <= 32: V^{-1} by Gauss-Jordan in
//             double-word FP32 arithmetic (prepared by the row owners while the
//             others compute MTTKRP partials), x0 = m V^{-1} in FP64 and one
//             step of FP64 iterative refinement x = x0 + (m - x0 V) V^{-1}.
//             R > 32: an FP32 Cholesky factor of V and up to six FP64
//             refinement steps.  If a pivot is too small, an FP64 Cholesky
//             (with a diagonal shift as last resort) is used instead;
//   barrier;
//   phase C (every CTA, identically): column norms of the new factor,
//             normalisation (lambda = the norms at n = N), its Gram, and after
//             mode N the fit of Section 3.3 and the stop rule.
// Every CTA holds the same factors and Grams, so no third barrier is needed.
// Serial FP64 chains are kept short on purpose: one FP64 warp instruction
// occupies a GB300 sub-partition for about 76 cycles (FP64 runs at 1/73 of
// FP32), so substitutions and factorisations run in FP32 and only the
// refinement residuals, the reductions and the Grams of the FP64 path are FP64.
// Grid barriers spin with a clock budget and record RCP_ETIMEOUT instead of
// hanging.  TM is the MTTKRP type (double for the FP64 path, float for the
// mixed form, whose factor Grams are also accumulated in FP32).
#include <math.h>

#include "dw_arith.cuh"
#include "rcp_internal.cuh"
#include "small_la.cuh"

namespace rcp {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kTileJ = 32;  // the tile loads and the Khatri-Rao rows map lanes / tid / 8 onto 32 columns
constexpr int kBP = kTileJ + 1;                   // padded pitch of the B tile
constexpr long long kBarrierBudget = 1LL << 31;  // default clock-cycle budget (about 1 s)


// Grid barrier over nblocks CTAs on a monotonic arrival counter (zeroed before
// the launch): barrier number e completes when the counter reaches e nblocks.
// Thread 0 publishes its CTA's writes (ordered before it by __syncthreads) with
// one release add and waits with acquire loads, so a single L2 round trip
// follows the last arrival.  The wait has a clock budget; on expiry the CTA
// raises the abort flag and returns false.  The other CTAs then run out their
// own budgets at this barrier or the next, neither of which can complete, so
// every CTA leaves.
__device__ bool grid_sync(unsigned* bar, unsigned nblocks, int* abort_flag, unsigned& epoch,
                          long long budget) {
  __syncthreads();
  __shared__ int ok_sh;
  if (threadIdx.x == 0) {
    epoch += 1u;
    const unsigned target = epoch * nblocks;
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
    int ok = 1;
    const long long t0 = clock64();
    while (true) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
      if ((int)(v - target) >= 0) break;
      if (clock64() - t0 > budget) {
        ok = 0;
        break;
      }
    }
    if (!ok) atomicExch(abort_flag, 1);
    ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

// Block-wide barrier for the G CTAs of one problem (a plain __syncthreads when G == 1).
__device__ __forceinline__ bool phase_sync(const PersArgs& a, int G, unsigned& epoch) {
  if (G == 1) {
    __syncthreads();
    return true;
  }
  return grid_sync(a.bar, (unsigned)G, a.abort_flag, epoch,
                   a.budget > 0 ? a.budget : kBarrierBudget);
}

// KACC: MTTKRP outputs (l_n x R) per thread, at most KACC * kThreads.
template <typename TM, int KACC>
__device__ void als_body(const PersArgs& a, int g) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = a.N, R = a.R, G = a.G;
  int lmax = 1, ftot = 0;
  int foff[kMaxN];
  for (int m = 0; m < N; ++m) {
    lmax = max(lmax, a.dims[m]);
    foff[m] = ftot;
    ftot += a.dims[m] * R;
  }

  // shared-memory carve-up
  double* Gr = (double*)smem;                   // N x R x R Grams
  double* V = Gr + N * R * R;                   // R x (R + 1): V, or its FP64 factor
  double* invd64 = V + R * (R + 1);             // R
  double* Xs = invd64 + R;                      // lmax x R new factor (FP64)
  double* nu = Xs + lmax * R;                   // R
  double* red = nu + R;                         // 64 scalars
  double* wsum = red + 64;                      // kWarps x 64 row / norm partials
  float* U32 = (float*)(wsum + kWarps * 64);    // R x (R + 1) FP32 copy of V / its factor
  float* invd32 = U32 + max(R * (R + 1), 1024); // R
  TM* Fac = (TM*)(((uintptr_t)(invd32 + R) + 15) & ~(uintptr_t)15);  // factor copies
  TM* Bs = Fac + ftot;                          // lmax x kBP
  TM* Ks = Bs + lmax * kBP;                     // kTileJ x R
  // the double-word Gauss-Jordan copies, 32 x 64 float2 each; after the inverse
  // one holds V^{-1} in FP64 (Zd, row pitch 32) and the other is scratch (Sx)
  float2* A0 = (float2*)(((uintptr_t)(Ks + kTileJ * R) + 15) & ~(uintptr_t)15);
  float2* A1 = A0 + 32 * 64;
  float* Gr32 = (float*)(A1 + 32 * 64);         // N x R x R FP32 Grams (mixed form)
  double* Zd = (double*)((R & 1) ? A0 : A1);
  double* Sx = (double*)((R & 1) ? A1 : A0);
  DevState* st = a.st;

  // ---- initial factors (modes 2..N) and their Grams, identical in every CTA
  const int user_init = a.user_init_dev ? *a.user_init_dev : a.user_init;
  for (int m = 1; m < N; ++m) {
    const int lm = a.dims[m];
    for (int e = tid; e < lm * R; e += kThreads) {
      const int i = e / R, r = e - i * R;
      double v;
      if (user_init) {
        v = a.At[m][i + lm * r];
      } else {
        const double2 z = normal_pair_f64(a.seed, (uint32_t)(m + 1), kPurposeAlsInit, (uint64_t)(e >> 1));
        v = (e & 1) ? z.y : z.x;
      }
      Fac[foff[m] + i + lm * r] = (TM)v;
      Xs[i + lm * r] = v;
    }
    __syncthreads();
    for (int e = tid; e < R * R; e += kThreads) {
      const int r = e % R, c = e / R;
      if (sizeof(TM) == 4) {
        // mixed form: from the FP32 copies, as after every update
        float acc = 0.0f;
        for (int i = 0; i < lm; ++i)
          acc = fmaf((float)Fac[foff[m] + i + lm * r], (float)Fac[foff[m] + i + lm * c], acc);
        Gr32[m * R * R + e] = acc;
        Gr[m * R * R + e] = (double)acc;
      } else {
        double acc = 0.0;
        for (int i = 0; i < lm; ++i) acc = fma(Xs[i + lm * r], Xs[i + lm * c], acc);
        Gr[m * R * R + e] = acc;
      }
    }
    __syncthreads();
  }

  // V = Hadamard product of the Grams of every mode but n0 (FP64) and the
  // solve it needs: path 3 (R <= 32) V^{-1} by double-word Gauss-Jordan into Zd,
  // path 1 (R > 32) an FP32 Cholesky factor plus FP64 refinement, path 0 the
  // FP64 Cholesky of V itself (with a diagonal shift as last resort).  The path
  // goes to red[0].
  auto prepare_solve = [&](int n0) {
        // (with one CTA per problem the path-3 solve keeps l_n x R outputs in 8 KB)
        const bool dw = !a.direct64 && R <= 32 && (G > 1 || lmax * R <= 1024);
        for (int e = tid; e < R * R; e += kThreads) {
          const int r = e % R, c = e / R;
          double v = Gr[(n0 == 0 ? 1 : 0) * R * R + e];
          for (int m = (n0 == 0 ? 2 : 1); m < N; ++m)
            if (m != n0) v *= Gr[m * R * R + e];
          V[r * (R + 1) + c] = v;
          if (!dw) {
            U32[r * (R + 1) + c] = (float)v;
          } else if (sizeof(TM) == 4) {
            // the FP32 Grams' product in double-word form (exact for N = 3)
            dwf w = {1.0f, 0.0f};
            bool first = true;
            for (int m = 0; m < N; ++m) {
              if (m == n0) continue;
              const float gm = Gr32[m * R * R + e];
              if (first) {
                w = {gm, 0.0f};
                first = false;
              } else {
                w = dw_mul(w, {gm, 0.0f});
              }
            }
            A0[r * 64 + c] = make_float2(w.hi, w.lo);
          } else {
            const dwf w = dw_from_double(v);
            A0[r * 64 + c] = make_float2(w.hi, w.lo);
          }
        }
        __syncthreads();
        bool gj = false;
        if (dw) {
          double* zd = nullptr;
          gj = cta_gj_inverse_dw<kThreads>(R, A0, A1, &zd);
          // FP32 copy of V^{-1} (the double-word high parts, row pitch 32) in U32,
          // unused by path 3: the one-CTA solve forms its refinement correction in FP32
          if (gj && G == 1)
            for (int e = tid; e < R * R; e += kThreads) {
              const int i = e / R, c = e - i * R;
              U32[i * 32 + c] = ((const float2*)Sx)[i * 64 + R + c].x;
            }
        }
        if (warp == 0) {
          int path = 0;
          if (gj) {
            path = 3;
          } else if (dw || a.direct64) {
            // path 0 below (a failed path-3 pivot means V is nearly singular)
          } else {
            float tr = 0.0f;
            for (int c = 0; c < R; ++c) tr += U32[c * (R + 1) + c];
            const float floor32 = 64.0f * 5.9604645e-08f * tr;
            bool f32ok = warp_chol(U32, R, floor32);
            if (f32ok)
              for (int k = lane; k < R; k += 32) invd32[k] = 1.0f / U32[k * (R + 1) + k];
            if (__all_sync(0xffffffffu, f32ok)) path = 1;
          }
          path = __shfl_sync(0xffffffffu, path, 0);
          if (path == 0) {
            // FP64 Cholesky of V itself; a diagonal shift R u trace(V) as last resort
            double trd = 0.0;
            for (int c = 0; c < R; ++c) trd += V[c * (R + 1) + c];
            const double shift = (double)R * 1.1102230246251565e-16 * trd;
            bool ok64 = warp_chol(V, R, shift);
            if (!ok64) {
              for (int e = lane; e < R * R; e += 32) {
                const int r = e % R, c = e / R;
                double v = 1.0;
                for (int m = 0; m < N; ++m)
                  if (m != n0) v *= Gr[m * R * R + e];
                V[r * (R + 1) + c] = v + (r == c ? shift : 0.0);
              }
              __syncwarp();
              ok64 = warp_chol(V, R, 0.0);
              if (lane == 0) atomicOr(&st->info, RCP_INFO_ALS_REGULARISED);
            }
            if (!ok64 && lane == 0) set_status(st, RCP_ESINGULAR);
            for (int k = lane; k < R; k += 32) invd64[k] = 1.0 / V[k * (R + 1) + k];
          }
          if (lane == 0) red[0] = (double)path;
        }
        __syncthreads();
  };

  double rho_prev = 0.0, nb2 = 0.0;
  unsigned epoch = 0;  // grid barriers passed (thread 0)
  int done = 0;
  bool ok = true;
  // partial writers of mode 1 (the |B|^2 partials are written in its first phase A)
  const int GW0 = G - ((G > 1 && G >= 2 * a.dims[0]) ? a.dims[0] : 0);
  for (int it = 1; it <= a.max_iters && ok && !done; ++it) {
    for (int n0 = 0; n0 < N && ok; ++n0) {
      const int ln = a.dims[n0];
      int L = 1, Rt = 1;
      for (int m = 0; m < n0; ++m) L *= a.dims[m];
      for (int m = n0 + 1; m < N; ++m) Rt *= a.dims[m];
      const int J = L * Rt;
      const int nout = ln * R;
      // With at least two CTAs per row, the row owners (g < ln) skip the MTTKRP
      // and prepare the Gram solve during phase A; the others write partials.
      const int gw0 = (G > 1 && G >= 2 * ln) ? ln : 0;
      const int GW = G - gw0, gi = g - gw0;
      constexpr bool kMixed = sizeof(TM) == 4;
      if (kMixed && a.S != nullptr) {
        // ---- phase A, dimension tree (mixed form, N >= 3, R <= 32): mode n's
        // MTTKRP is M = S_c reduced over the modes other than n and c against
        // their factors, with S_c = B x_c A_c^T (l_c contracted, the other modes
        // kept, R columns).  c = 2 for mode 1 and c = 1 otherwise: S_1 is formed
        // once per sweep, after mode 1's update, and serves modes 2..N.
        const int c = n0 == 0 ? 1 : 0;
        if (n0 <= 1) {
          // S_c[rest, r] = sum_{i_c} B[a + Lc (i_c + l_c b)] A_c[i_c, r], rest = a + Lc b;
          // thread per rest index, all R columns in registers (FP32 products and sums
          // over l_c <= 64 terms), A_c in shared memory row by row
          const int lc = a.dims[c];
          int Lc = 1, Rc = 1;
          for (int m = 0; m < c; ++m) Lc *= a.dims[m];
          for (int m = c + 1; m < N; ++m) Rc *= a.dims[m];
          const int nrest = Lc * Rc;
          float* FcT = (float*)Bs;  // l_c x 32, row-major, zero beyond R
          for (int e = tid; e < lc * 32; e += kThreads) {
            const int i = e >> 5, r = e & 31;
            FcT[e] = r < R ? (float)Fac[foff[c] + i + lc * r] : 0.0f;
          }
          __syncthreads();
          double nbs = 0.0;
          const bool want_nb = it == 1 && n0 == 0;
          for (int rest = gi * kThreads + tid; gi >= 0 && rest < nrest; rest += GW * kThreads) {
            const int bq = rest / Lc, aq = rest - bq * Lc;
            const float* Bp = (const float*)a.B + aq + (int64_t)Lc * lc * bq;
            float* Sp = a.S + (int64_t)rest * 32;
            // all 32 columns in one pass: FP32 sums of 8 terms (packed FMAs, two
            // columns per instruction) carried into double-word accumulators (Knuth's
            // TwoSum), so each S entry is accurate to a few u; the next 8 values of
            // the fibre are loaded while the current 8 are multiplied
            float shi[32], slo[32];
#pragma unroll
            for (int r = 0; r < 32; ++r) shi[r] = slo[r] = 0.0f;
            float xc[8], xn[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) xc[u] = u < lc ? Bp[(int64_t)Lc * u] : 0.0f;
            for (int ic0 = 0; ic0 < lc; ic0 += 8) {
#pragma unroll
              for (int u = 0; u < 8; ++u)
                xn[u] = ic0 + 8 + u < lc ? Bp[(int64_t)Lc * (ic0 + 8 + u)] : 0.0f;
              float2 t[16];
#pragma unroll
              for (int r = 0; r < 16; ++r) t[r] = make_float2(0.0f, 0.0f);
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                if (ic0 + u < lc) {
                  const float x = xc[u];
                  if (want_nb) nbs = fma((double)x, (double)x, nbs);
                  const float2 xx = make_float2(x, x);
                  const float4* f = (const float4*)(FcT + (ic0 + u) * 32);
#pragma unroll
                  for (int q = 0; q < 8; ++q) {
                    const float4 v = f[q];
                    t[2 * q] = __ffma2_rn(xx, make_float2(v.x, v.y), t[2 * q]);
                    t[2 * q + 1] = __ffma2_rn(xx, make_float2(v.z, v.w), t[2 * q + 1]);
                  }
                }
              }
#pragma unroll
              for (int r = 0; r < 16; ++r) {
                const dwf u0 = dw_two_sum(shi[2 * r], t[r].x);
                shi[2 * r] = u0.hi;
                slo[2 * r] = __fadd_rn(slo[2 * r], u0.lo);
                const dwf u1 = dw_two_sum(shi[2 * r + 1], t[r].y);
                shi[2 * r + 1] = u1.hi;
                slo[2 * r + 1] = __fadd_rn(slo[2 * r + 1], u1.lo);
              }
#pragma unroll
              for (int u = 0; u < 8; ++u) xc[u] = xn[u];
            }
#pragma unroll
            for (int q = 0; q < 8; ++q)
              ((float4*)Sp)[q] = make_float4(shi[4 * q] + slo[4 * q], shi[4 * q + 1] + slo[4 * q + 1],
                                             shi[4 * q + 2] + slo[4 * q + 2],
                                             shi[4 * q + 3] + slo[4 * q + 3]);
          }
          if (want_nb && gi >= 0) {
            for (int o = 16; o > 0; o >>= 1) nbs += __shfl_down_sync(0xffffffffu, nbs, o);
            if (lane == 0) red[8 + warp] = nbs;
            __syncthreads();
            if (tid == 0) {
              double sb = 0.0;
              for (int w = 0; w < kWarps; ++w) sb += red[8 + w];
              a.nbp[gi] = sb;
            }
          }
          // the row owners write no part of S_c: they invert V (which needs only the
          // Grams) while the others form it
          if (gw0 > 0 && g < ln) prepare_solve(n0);
          // every CTA's part of S_c is written before any CTA reduces it
          if (!phase_sync(a, G, epoch)) { ok = false; break; }
        }
        // M partials: warp w takes rows i = w, w + 8, ... of mode n; the CTA takes a
        // range of the multi-indices p over the modes other than n and c; lane r
        // accumulates sum_p S_c[(i, p), r] prod_{m != n, c} A_m[p_m, r] in FP32 over
        // the CTA's range (fixed order; the partials are summed in FP64 after)
        if (gi >= 0) {
          int np_ = 1;
          for (int m = 0; m < N; ++m)
            if (m != n0 && m != c) np_ *= a.dims[m];
          // stride of mode n in S_c's index (Kolda order over the modes other than c)
          int sn = 1;
          for (int m = 0; m < n0; ++m)
            if (m != c) sn *= a.dims[m];
          const int per = (np_ + GW - 1) / GW;
          const int p0 = gi * per, p1 = min(np_, p0 + per);
          constexpr int kRowsPerWarp = 8;  // l_n <= 64
          // double-word accumulators of exact products (TwoProduct by FMA, TwoSum)
          float mhi[kRowsPerWarp], mlo[kRowsPerWarp];
#pragma unroll
          for (int k = 0; k < kRowsPerWarp; ++k) mhi[k] = mlo[k] = 0.0f;
          // kPQ multi-indices per step: their S loads are all in flight before the
          // first is accumulated (the accumulation order is that of pp)
          constexpr int kPQ = 4;
          for (int pp = p0; pp < p1; pp += kPQ) {
            int offv[kPQ];
            float wv[kPQ];
#pragma unroll
            for (int e = 0; e < kPQ; ++e) {
              // digits of pp + e over the modes other than n and c, the S_c offset and
              // weight (weight 0 past the range)
              int q = pp + e, off = 0, st_ = 1;
              float wgt = (lane < R && pp + e < p1) ? 1.0f : 0.0f;
              for (int m = 0; m < N; ++m) {
                if (m == c) continue;
                if (m != n0) {
                  const int d = q % a.dims[m];
                  q /= a.dims[m];
                  off += d * st_;
                  if (lane < R) wgt *= (float)Fac[foff[m] + d + a.dims[m] * lane];
                }
                st_ *= a.dims[m];
              }
              offv[e] = pp + e < p1 ? off : 0;
              wv[e] = wgt;
            }
            float sv[kPQ][kRowsPerWarp];
#pragma unroll
            for (int e = 0; e < kPQ; ++e)
#pragma unroll
              for (int k = 0; k < kRowsPerWarp; ++k) {
                const int i = warp + kWarps * k;
                sv[e][k] = i < ln ? a.S[(int64_t)(offv[e] + i * sn) * 32 + lane] : 0.0f;
              }
#pragma unroll
            for (int e = 0; e < kPQ; ++e) {
              if (pp + e < p1) {
#pragma unroll
                for (int k = 0; k < kRowsPerWarp; ++k) {
                  const int i = warp + kWarps * k;
                  if (i < ln) {
                    const float pv = __fmul_rn(sv[e][k], wv[e]);
                    const float pe = __fmaf_rn(sv[e][k], wv[e], -pv);
                    const dwf u2 = dw_two_sum(mhi[k], pv);
                    mhi[k] = u2.hi;
                    mlo[k] = __fadd_rn(mlo[k], __fadd_rn(u2.lo, pe));
                  }
                }
              }
            }
          }
#pragma unroll
          for (int k = 0; k < kRowsPerWarp; ++k) {
            const int i = warp + kWarps * k;
            if (i < ln && lane < R)
              a.part[(int64_t)gi * nout + i + ln * lane] = (double)mhi[k] + (double)mlo[k];
          }
        }
      } else {
      // ---- phase A: MTTKRP partial over this CTA's column tiles
      // Each thread owns register blocks of outputs (below) and forms their tile
      // sums with independent FMA chains.  The mixed form sums its FP32 tile sums
      // across tiles in double-word FP32 (Knuth's TwoSum), the FP64 path in FP64.
      double acc[kMixed ? 1 : KACC];
      float ahi[kMixed ? KACC : 1], alo[kMixed ? KACC : 1];
#pragma unroll
      for (int k = 0; k < (kMixed ? 1 : KACC); ++k) acc[k] = 0.0;
#pragma unroll
      for (int k = 0; k < (kMixed ? KACC : 1); ++k) ahi[k] = alo[k] = 0.0f;
      // register blocks of kBI rows x kBR columns of the l_n x R output: block
      // q = tid + kThreads bb (bb < kKB) covers rows ig + nig u and columns rg + nrg v
      constexpr int kBI = 2, kBR = KACC >= 8 ? 4 : 2, kKB = KACC / (kBI * kBR);
      const int nig = (ln + kBI - 1) / kBI, nrg = (R + kBR - 1) / kBR;
      int b_ig[kKB], b_rg[kKB];
#pragma unroll
      for (int bb = 0; bb < kKB; ++bb) {
        const int q = tid + kThreads * bb;
        b_rg[bb] = q / nig;
        b_ig[bb] = q - b_rg[bb] * nig;
      }
      double nbpart = 0.0;
      // column tiles of tj <= kTileJ columns, narrow enough to keep the GW writers busy
      const int tj = max(1, min(kTileJ, (J + GW - 1) / GW));
      // B tile: Bs[i][jj] = B[(j % L) + L (i + ln (j / L))], with lanes along the
      // contiguous index (i for mode 1, the column otherwise).  The next tile is
      // loaded into registers while the current one is multiplied: kPS slots per
      // thread, 8 for l_n <= 64, 4 for a small register budget (l_n <= 32).
      constexpr int kPS = KACC >= 8 ? 8 : 4;
      auto b_slot = [&](int s2, int& i, int& jj) {
        if (L == 1) {
          jj = kPS == 8 ? warp + kWarps * (s2 >> 1) : warp + kWarps * s2;
          i = kPS == 8 ? lane + 32 * (s2 & 1) : lane;
        } else {
          jj = lane;
          i = warp + kWarps * s2;
        }
      };
      auto b_load = [&](int t0x, TM (&v)[kPS]) {
        const int njx = min(tj, J - t0x);
        int64_t base = 0;
        if (L != 1) {
          const int j = t0x + lane;
          const int b = j / L;
          base = (int64_t)(j - b * L) + (int64_t)L * ln * b;
        }
#pragma unroll
        for (int s2 = 0; s2 < kPS; ++s2) {
          int i, jj;
          b_slot(s2, i, jj);
          TM x = (TM)0;
          if (i < ln && jj < njx)
            x = L == 1 ? ((const TM*)a.B)[i + (int64_t)ln * (t0x + jj)]
                       : ((const TM*)a.B)[base + (int64_t)L * i];
          v[s2] = x;
        }
      };
      TM pf[kPS];
      if (gi >= 0 && gi * tj < J) b_load(gi * tj, pf);
      for (int t0 = gi * tj; gi >= 0 && t0 < J; t0 += GW * tj) {
        const int nj = min(tj, J - t0);
#pragma unroll
        for (int s2 = 0; s2 < kPS; ++s2) {
          int i, jj;
          b_slot(s2, i, jj);
          if (i < ln) Bs[i * kBP + jj] = pf[s2];
        }
        // Khatri-Rao rows of the other factors, mode 1 fastest: thread (jj, rg),
        // jj = tid / 8 < 32 = kTileJ, forms column t0 + jj's digits once and the
        // products for r = rg, rg + 8, ...
        {
          const int jj = tid >> 3, rg = tid & 7;
          int dig[kMaxN];
          int jr = t0 + jj;
          for (int m = 0; m < N; ++m) {
            if (m == n0) continue;
            const int d = a.dims[m];
            const int q = jr / d;
            dig[m] = jr - q * d;
            jr = q;
          }
          for (int r = rg; r < R; r += 8) {
            TM prod = (TM)0;
            if (jj < nj) {
              prod = (TM)1;
              for (int m = 0; m < N; ++m)
                if (m != n0) prod *= Fac[foff[m] + dig[m] + a.dims[m] * r];
            }
            Ks[jj * R + r] = prod;
          }
        }
        __syncthreads();
        if (t0 + GW * tj < J) b_load(t0 + GW * tj, pf);
        if (it == 1 && n0 == 0) {
          for (int e = tid; e < ln * kTileJ; e += kThreads) {
            const double v = (double)Bs[(e / kTileJ) * kBP + e % kTileJ];
            nbpart = fma(v, v, nbpart);
          }
        }
#pragma unroll
        for (int bb = 0; bb < kKB; ++bb) {
          if (b_rg[bb] < nrg) {
            // rows and columns past the edge read row / column 0 and are not written
            int ib[kBI], rb[kBR];
#pragma unroll
            for (int u = 0; u < kBI; ++u) {
              const int i = b_ig[bb] + nig * u;
              ib[u] = (i < ln ? i : 0) * kBP;
            }
#pragma unroll
            for (int v = 0; v < kBR; ++v) {
              const int r = b_rg[bb] + nrg * v;
              rb[v] = r < R ? r : 0;
            }
            TM sacc[kBI * kBR];
#pragma unroll
            for (int q = 0; q < kBI * kBR; ++q) sacc[q] = (TM)0;
            // unrolled so that the shared-memory loads of later columns are in
            // flight while earlier FMAs run
#pragma unroll 8
            for (int jj = 0; jj < nj; ++jj) {
              TM x[kBI], kr[kBR];
#pragma unroll
              for (int u = 0; u < kBI; ++u) x[u] = Bs[ib[u] + jj];
#pragma unroll
              for (int v = 0; v < kBR; ++v) kr[v] = Ks[jj * R + rb[v]];
#pragma unroll
              for (int u = 0; u < kBI; ++u)
#pragma unroll
                for (int v = 0; v < kBR; ++v) sacc[u * kBR + v] = fma(x[u], kr[v], sacc[u * kBR + v]);
            }
#pragma unroll
            for (int q = 0; q < kBI * kBR; ++q) {
              const int k = bb * kBI * kBR + q;
              if constexpr (kMixed) {
                const dwf t = dw_two_sum(ahi[k], (float)sacc[q]);
                ahi[k] = t.hi;
                alo[k] += t.lo;
              } else {
                acc[k] += (double)sacc[q];
              }
            }
          }
        }
        __syncthreads();
      }
#pragma unroll
      for (int bb = 0; bb < kKB; ++bb)
#pragma unroll
        for (int u = 0; u < kBI; ++u)
#pragma unroll
          for (int v = 0; v < kBR; ++v) {
            const int i = b_ig[bb] + nig * u, r = b_rg[bb] + nrg * v;
            if (gi >= 0 && b_rg[bb] < nrg && i < ln && r < R) {
              const int k = bb * kBI * kBR + u * kBR + v;
              double val;
              if constexpr (kMixed) val = (double)ahi[k] + (double)alo[k];
              else val = acc[k];
              a.part[(int64_t)gi * nout + i + ln * r] = val;
            }
          }
      if (it == 1 && n0 == 0 && gi >= 0) {
        for (int o = 16; o > 0; o >>= 1) nbpart += __shfl_down_sync(0xffffffffu, nbpart, o);
        if (lane == 0) red[8 + warp] = nbpart;
        __syncthreads();
        if (tid == 0) {
          double s = 0.0;
          for (int w = 0; w < kWarps; ++w) s += red[8 + w];
          a.nbp[gi] = s;
        }
      }
      }
      if (gw0 > 0 && g < ln && !(kMixed && a.S != nullptr && n0 <= 1)) prepare_solve(n0);
      if (!phase_sync(a, G, epoch)) { ok = false; break; }

      // ---- phase B: rows owned by this CTA (rows i = g, g + G, ...)
      if (g < ln) {
        if (gw0 == 0) prepare_solve(n0);
        const int path = (int)red[0];
        const bool use32 = path == 1;  // FP32 factor: FP64 refinement follows
        const bool want_ip = n0 == N - 1;  // <Bhat, B> is needed after the last mode only
        // sum of the four partial vectors the split products leave in wsum
        auto sum4 = [&](int c) {
          return (wsum[c] + wsum[64 + c]) + (wsum[128 + c] + wsum[192 + c]);
        };
        // out_c = sum_k v_k Mt[k][c] (R <= 32, lane c), split over warps 0..3 (one
        // per sub-partition: FP64 issues at one warp instruction per 64 cycles
        // per sub-partition) into wsum[w][c]
        auto split_mv = [&](const double* v, const double* Mt, int ld) {
          if (warp < 4) {
            double d = 0.0;
            if (lane < R)
              for (int k = warp; k < R; k += 4) d = fma(v[k], Mt[k * ld + lane], d);
            wsum[warp * 64 + lane] = d;
          }
        };
        if (G == 1 && path == 3) {
          // one CTA per problem, R <= 32 and ln R <= 1024: outputs (i, c) over all
          // threads; m, x0 in Sx, the residual in Xs (free until phase C)
          double* Mm = Sx;
          double* X0 = Sx + 1024;
          for (int e = tid; e < nout; e += kThreads) {
            double sm_ = 0.0;
            for (int gg = 0; gg < GW; ++gg) sm_ += a.part[(int64_t)gg * nout + e];
            Mm[e] = sm_;
          }
          __syncthreads();
          for (int e = tid; e < nout; e += kThreads) {
            const int c = e / ln, i = e - c * ln;
            double d = 0.0;
            for (int k = 0; k < R; ++k) d = fma(Mm[i + ln * k], Zd[k * 32 + c], d);
            X0[e] = d;
          }
          __syncthreads();
          // the residual m - x0 V in FP64, kept in FP32: the correction it feeds is
          // about kappa 2^-46 of x, so its FP32 rounding stays far below FP64 rounding
          // of x, and the FP64 unit is this loop's bound
          float* Rf = (float*)Xs;
          for (int e = tid; e < nout; e += kThreads) {
            const int c = e / ln, i = e - c * ln;
            double d = 0.0;
            for (int k = 0; k < R; ++k) d = fma(X0[i + ln * k], V[k * (R + 1) + c], d);
            Rf[e] = (float)(Mm[e] - d);
          }
          __syncthreads();
          for (int e = tid; e < nout; e += kThreads) {
            const int c = e / ln, i = e - c * ln;
            float d = 0.0f;
            for (int k = 0; k < R; ++k) d = fmaf(Rf[i + ln * k], U32[k * 32 + c], d);
            const double x = X0[e] + (double)d;
            a.rows[e] = x;
            X0[e] = Mm[e] * x;
          }
          if (want_ip) {
            __syncthreads();
            for (int i = tid; i < ln; i += kThreads) {
              double ip = 0.0;
              for (int c = 0; c < R; ++c) ip += X0[i + ln * c];
              a.ipp[i] = ip;
            }
          }
          __syncthreads();
        } else if (G == 1) {
          // one CTA per problem, paths 0 and 1: warp w solves rows w, w + 8, ...
          for (int i = warp; i < ln; i += kWarps) {
            double m[2], x[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int r = lane + 32 * h;
              double sm_ = 0.0;
              if (r < R)
                for (int gg = 0; gg < GW; ++gg) sm_ += a.part[(int64_t)gg * nout + i + ln * r];
              m[h] = sm_;
              x[h] = sm_;
            }
            if (path == 1) warp_solve(U32, invd32, R, x);
            else warp_solve(V, invd64, R, x);
            for (int step = 0; use32 && step < 6; ++step) {
              double rr[2] = {m[0], m[1]};
              for (int k = 0; k < R; ++k) {
                const double xk = __shfl_sync(0xffffffffu, (k >> 5) ? x[1] : x[0], k & 31);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                  const int c = lane + 32 * h;
                  if (c < R) rr[h] = fma(-V[k * (R + 1) + c], xk, rr[h]);
                }
              }
#pragma unroll
              for (int h = 0; h < 2; ++h)
                if (lane + 32 * h >= R) rr[h] = 0.0;
              warp_solve(U32, invd32, R, rr);
              x[0] += rr[0];
              x[1] += rr[1];
              double dm = fmax(fabs(rr[0]), fabs(rr[1])), xm = fmax(fabs(x[0]), fabs(x[1]));
              for (int o = 16; o > 0; o >>= 1) {
                dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
                xm = fmax(xm, __shfl_xor_sync(0xffffffffu, xm, o));
              }
              if (dm <= 2.220446049250313e-16 * xm) break;
            }
            double ip = 0.0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int r = lane + 32 * h;
              if (r < R) {
                a.rows[i + ln * r] = x[h];
                ip += m[h] * x[h];
              }
            }
            if (want_ip) {
              for (int o = 16; o > 0; o >>= 1) ip += __shfl_xor_sync(0xffffffffu, ip, o);
              if (lane == 0) a.ipp[i] = ip;
            }
          }
          __syncthreads();
        } else
        {
        // all warps reduce one row's partials; path 3 splits its three FP64
        // products over warps 0..3; paths 0 and 1 solve on warp 0 and split the
        // FP64 residuals of the refinement over all warps
        double* xs = wsum + (kWarps - 1) * 64;  // x broadcast (the last warp's slot is read first)
        for (int i = g; i < ln; i += G) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int r = lane + 32 * h;
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
            if (r < R) {
              const double* src = a.part + i + (int64_t)ln * r;
              int gg = warp;
              for (; gg + 3 * kWarps < GW; gg += 4 * kWarps) {
                s0 += src[(int64_t)gg * nout];
                s1 += src[(int64_t)(gg + kWarps) * nout];
                s2 += src[(int64_t)(gg + 2 * kWarps) * nout];
                s3 += src[(int64_t)(gg + 3 * kWarps) * nout];
              }
              for (; gg < GW; gg += kWarps) s0 += src[(int64_t)gg * nout];
            }
            wsum[warp * 64 + r] = (s0 + s1) + (s2 + s3);
          }
          __syncthreads();
          double m[2] = {0.0, 0.0}, x[2] = {0.0, 0.0};
          if (path == 3) {
            // m, x0 and the residual in Sx[0..95]
            if (warp == 0) {
              double sm_ = 0.0;
              if (lane < R)
                for (int w = 0; w < kWarps; ++w) sm_ += wsum[w * 64 + lane];
              m[0] = sm_;
              Sx[lane] = sm_;
            }
            __syncthreads();
            split_mv(Sx, Zd, 32);  // x0 = m V^{-1}
            __syncthreads();
            if (warp == 0) {
              x[0] = lane < R ? sum4(lane) : 0.0;
              Sx[32 + lane] = x[0];
            }
            __syncthreads();
            split_mv(Sx + 32, V, R + 1);  // x0 V
            __syncthreads();
            if (warp == 0) Sx[64 + lane] = lane < R ? m[0] - sum4(lane) : 0.0;
            __syncthreads();
            split_mv(Sx + 64, Zd, 32);  // (m - x0 V) V^{-1}
            __syncthreads();
            if (warp == 0 && lane < R) x[0] += sum4(lane);
          } else {
          if (warp == 0) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int r = lane + 32 * h;
              double s = 0.0;
              if (r < R)
                for (int w = 0; w < kWarps; ++w) s += wsum[w * 64 + r];
              m[h] = s;
              x[h] = s;
            }
            if (path == 1) warp_solve(U32, invd32, R, x);
            else warp_solve(V, invd64, R, x);
          }
          if (use32) {
            for (int step = 0; step < 6; ++step) {
              __syncthreads();
              if (warp == 0) {
                xs[lane] = x[0];
                xs[lane + 32] = x[1];
              }
              __syncthreads();
              // warp w: partial residual over k = w, w + 8, ... (lanes own columns c)
              double pr[2] = {0.0, 0.0};
              for (int k = warp; k < R; k += kWarps) {
                const double xk = xs[k];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                  const int c = lane + 32 * h;
                  if (c < R) pr[h] = fma(V[k * (R + 1) + c], xk, pr[h]);
                }
              }
              __syncthreads();
              wsum[warp * 64 + lane] = pr[0];
              wsum[warp * 64 + lane + 32] = pr[1];
              __syncthreads();
              int stop = 0;
              if (warp == 0) {
                double rr[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                  double sum = 0.0;
                  for (int w = 0; w < kWarps; ++w) sum += wsum[w * 64 + lane + 32 * h];
                  rr[h] = (lane + 32 * h < R) ? m[h] - sum : 0.0;
                }
                warp_solve(U32, invd32, R, rr);
                x[0] += rr[0];
                x[1] += rr[1];
                // stop once max |correction| <= 2^-52 max |x| (warp-uniform)
                double dm = fmax(fabs(rr[0]), fabs(rr[1])), xm = fmax(fabs(x[0]), fabs(x[1]));
                for (int o = 16; o > 0; o >>= 1) {
                  dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
                  xm = fmax(xm, __shfl_xor_sync(0xffffffffu, xm, o));
                }
                stop = dm <= 2.220446049250313e-16 * xm;
                if (lane == 0) red[6] = stop ? 1.0 : 0.0;
              }
              __syncthreads();
              if (red[6] != 0.0) break;
            }
          }
          }
          if (warp == 0) {
            double ip = 0.0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int r = lane + 32 * h;
              if (r < R) {
                a.rows[i + ln * r] = x[h];
                ip += m[h] * x[h];
              }
            }
            if (want_ip) {
              for (int o = 16; o > 0; o >>= 1) ip += __shfl_xor_sync(0xffffffffu, ip, o);
              if (lane == 0) a.ipp[i] = ip;
            }
          }
          __syncthreads();
        }
        }
      }
      if (!phase_sync(a, G, epoch)) { ok = false; break; }
      // every CTA reads the status once, after the barrier, so all leave
      // together (the load overlaps the load of the new rows)
      {
        int stv = 0;
        if (tid == 0) stv = *(volatile int*)&st->status;
        for (int e = tid; e < nout; e += kThreads) Xs[e] = a.rows[e];
        if (tid == 0) red[3] = (double)stv;
      }
      __syncthreads();
      if (red[3] != 0.0) { ok = false; break; }

      // ---- phase C (every CTA): norms, normalisation, Gram
#pragma unroll
      for (int h = 0; h < 2; ++h) {  // column norms: warp w sums rows w, w + 8, ...
        const int r = lane + 32 * h;
        double s = 0.0;
        if (r < R)
          for (int i = warp; i < ln; i += kWarps) s = fma(Xs[i + ln * r], Xs[i + ln * r], s);
        wsum[warp * 64 + r] = s;
      }
      __syncthreads();
      for (int r = tid; r < R; r += kThreads) {
        double s = 0.0;
        for (int w = 0; w < kWarps; ++w) s += wsum[w * 64 + r];
        // the norm and its reciprocal from one reciprocal square root (a zero column stays zero)
        const double rs = __double_as_longlong(s) > 0 ? rsqrt64(s) : 0.0;
        nu[r] = s * rs;
        wsum[kWarps * 64 - 64 + r] = rs;  // last warp's row is free now
      }
      __syncthreads();
      for (int e = tid; e < nout; e += kThreads) {
        const int r = e / ln;
        const double v = Xs[e] * wsum[kWarps * 64 - 64 + r];
        Xs[e] = v;
        Fac[foff[n0] + e] = (TM)v;
        if (g == 0) a.At[n0][e] = v;
      }
      __syncthreads();
      if (sizeof(TM) == 4) {
        // mixed form: Gram of the normalised factor from the FP32 copies
        for (int e = tid; e < R * R; e += kThreads) {
          const int r = e % R, c = e / R;
          float s = 0.0f;
          const TM* fr = Fac + foff[n0] + ln * r;
          const TM* fc = Fac + foff[n0] + ln * c;
          for (int i = 0; i < ln; ++i) s = fmaf((float)fr[i], (float)fc[i], s);
          Gr32[n0 * R * R + e] = s;
          Gr[n0 * R * R + e] = (double)s;
        }
      } else {
        // symmetric: entries r <= c only
        for (int e = tid; e < R * (R + 1) / 2; e += kThreads) {
          int c = 0, rem = e;
          while (rem > c) { rem -= c + 1; ++c; }
          const int r = rem;
          double s = 0.0;
          for (int i = 0; i < ln; ++i) s = fma(Xs[i + ln * r], Xs[i + ln * c], s);
          Gr[n0 * R * R + r + R * c] = s;
          Gr[n0 * R * R + c + R * r] = s;
        }
      }
      __syncthreads();
      if (n0 == N - 1) {
        // |Bhat|^2 = lambda^T (Hadamard product of all Grams) lambda, <Bhat, B> = sum_i ipp[i]
        double bh = 0.0;
        for (int e = tid; e < R * R; e += kThreads) {
          const int r = e % R, c = e / R;
          double v = nu[r] * nu[c];
          for (int m = 0; m < N; ++m) v *= Gr[m * R * R + e];
          bh += v;
        }
        double sb = 0.0, si = 0.0;
        if (warp == 0) {
          if (it == 1)
            for (int gg = lane; gg < GW0; gg += 32) sb += a.nbp[gg];
          for (int i = lane; i < ln; i += 32) si += a.ipp[i];
        }
        for (int o = 16; o > 0; o >>= 1) {
          bh += __shfl_xor_sync(0xffffffffu, bh, o);
          sb += __shfl_xor_sync(0xffffffffu, sb, o);
          si += __shfl_xor_sync(0xffffffffu, si, o);
        }
        if (lane == 0) red[16 + warp] = bh;
        if (tid == 0) {
          red[4] = sb;
          red[5] = si;
        }
        __syncthreads();
        if (tid == 0) {
          if (it == 1) nb2 = red[4];
          double bhat = 0.0;
          for (int w = 0; w < kWarps; ++w) bhat += red[16 + w];
          const double ip = red[5];
          const double rho = 1.0 - (nb2 + bhat - 2.0 * ip) / nb2;
          const bool conv = fabs(rho - rho_prev) < a.tol;
          red[2] = (conv || it >= a.max_iters) ? (conv ? 1.0 : 2.0) : 0.0;
          rho_prev = rho;
          if (g == 0) {
            st->fit = rho;
            st->ip = ip;
            st->fit_prev = rho;
            st->als_iters = it;
            st->norm_b2 = nb2;
            if (!isfinite(rho)) set_status(st, RCP_ENAN);
          }
        }
        if (g == 0)
          for (int r = tid; r < R; r += kThreads) a.lam[r] = nu[r];
        __syncthreads();
        done = red[2] != 0.0 ? (int)red[2] : 0;
        if (done && g == 0 && tid == 0) st->als_done = done;
        __syncthreads();
      }
    }
  }
  if (!ok && g == 0 && tid == 0 && !*(volatile int*)&st->status) set_status(st, RCP_ETIMEOUT);
}

// KACC: MTTKRP outputs per thread, in 2 x 4 register blocks (8: one block per
// thread, for ceil(l_max / 2) ceil(R / 4) <= 256; 16: two)
template <typename TM, int KACC>
__global__ void __launch_bounds__(kThreads, 1) k_als_persistent(PersArgs a) {
  als_body<TM, KACC>(a, blockIdx.x);
}

template <typename TM>
size_t smem_bytes(const rcp_plan_s* p) {
  int lmax = 1, ftot = 0;
  for (int m = 0; m < p->N; ++m) {
    lmax = lmax > p->l[m] ? lmax : p->l[m];
    ftot += p->l[m] * p->R;
  }
  const size_t R = p->R, N = p->N;
  const size_t d = N * R * R + R * (R + 1) + R + (size_t)lmax * R + R + 64 + kWarps * 64;
  const size_t f = (R * (R + 1) > 1024 ? R * (R + 1) : 1024) + R;
  return d * sizeof(double) + f * sizeof(float) + 16 +
         ((size_t)ftot + (size_t)lmax * kBP + (size_t)kTileJ * R) * sizeof(TM) + 16 +
         (size_t)2 * 32 * 64 * sizeof(float2) + N * R * R * sizeof(float);
}

template <typename TM>
cudaError_t launch_typed(rcp_plan_s* p, const void* B, const int* user_init_dev, cudaStream_t s) {
  const size_t smem = smem_bytes<TM>(p);
  int lmax0 = 1;
  for (int m = 0; m < p->N; ++m) lmax0 = lmax0 > p->l[m] ? lmax0 : p->l[m];
  // 8 outputs per thread: 2 x 4 register blocks of the l x R output, one per thread
  const bool small = (int64_t)((lmax0 + 1) / 2) * ((p->R + 3) / 4) <= kThreads;
  const void* kern = small ? (const void*)k_als_persistent<TM, 8> : (const void*)k_als_persistent<TM, 16>;
  cudaError_t e = cudaFuncSetAttribute(kern,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  PersArgs a{};
  a.N = p->N;
  a.R = p->R;
  // CTAs: one per SM when the MTTKRP is large; for a small core, about two per
  // row of the largest factor (each row needs an owner) -- fewer CTAs mean fewer
  // partials to reduce per row and cheaper grid barriers
  int lmax = 1;
  for (int m = 0; m < p->N; ++m) lmax = lmax > p->l[m] ? lmax : p->l[m];
  const double work = (double)p->core_elems * p->R;
  a.G = work >= 16.0e6 ? p->nsm : (2 * lmax < p->nsm ? (2 * lmax > 32 ? 2 * lmax : 32) : p->nsm);
  if (a.G > p->nsm) a.G = p->nsm;
  a.GA = a.G;  // every CTA computes MTTKRP partials
  for (int m = 0; m < p->N; ++m) {
    a.dims[m] = p->l[m];
    a.At[m] = p->At[m];
  }
  a.B = B;
  a.lam = p->lam;
  a.part = p->part;
  a.rows = p->M;
  a.ipp = p->tmp;
  a.nbp = p->normpart;
  a.bar = p->bar;
  a.abort_flag = p->abort_flag;
  a.st = p->dstate;
  a.seed = p->cfg.seed;
  a.tol = p->cfg.tol;
  a.max_iters = p->cfg.max_iters;
  a.user_init = p->user_init ? 1 : 0;
  a.budget = p->cfg.wait_budget;
  a.user_init_dev = user_init_dev;
  // mixed form: the dimension-tree MTTKRP when the plan holds its scratch
  a.S = sizeof(TM) == 4 ? p->als_S : nullptr;
  // R <= 32: each row-owning CTA inverts V in double-word arithmetic (path 3)
  a.direct64 = 0;
  void* args[] = {&a};
  count_launches(1);
  return cudaLaunchCooperativeKernel(kern, dim3(a.G), dim3(kThreads),
                                     args, smem, s);
}

}  // namespace

// True when the persistent kernel fits this plan (shared memory, rank, 32-bit core indexing).
bool als_persistent_fits(const rcp_plan_s* p, bool f32) {
  if (p->R > 64) return false;
  int lmax = 1;
  for (int m = 0; m < p->N; ++m) lmax = lmax > p->l[m] ? lmax : p->l[m];
  if ((int64_t)lmax * p->R > 16 * kThreads) return false;
  if (p->core_elems >= (1LL << 31)) return false;
  const size_t smem = f32 ? smem_bytes<float>(p) : smem_bytes<double>(p);
  return smem <= 200 * 1024;
}

cudaError_t launch_als_persistent(rcp_plan_s* p, const void* B, bool f32, const int* user_init_dev,
                                  cudaStream_t s) {
  return f32 ? launch_typed<float>(p, B, user_init_dev, s)
             : launch_typed<double>(p, B, user_init_dev, s);
}

}  // namespace rcp

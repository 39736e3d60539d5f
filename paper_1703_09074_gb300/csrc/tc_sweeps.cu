// Tensor-core sweeps over X for mode 1 of the mixed-precision form
// (tcgen05 kind::tf32, FP32 accumulation in tensor memory).  Mode 1 reads the
// whole input X, 2q + 2 times, so these sweeps set the end-to-end time.
//
// Precision: every FP32 operand is split into hi = its TF32 truncation and
// lo = the exact remainder, and each product is formed as
// hi*hi + hi*lo + lo*hi (three MMAs), which keeps about 21 bits.  Plain TF32
// (10 fraction bits) loses the weak signal directions of unfoldings whose
// spectrum spans two decades (factor congruence 0.5 at R = 20).
//
// X_(1) is I x J with columns contiguous (column j = the mode-1 fibre at j).
//
// Row sweep (k_tc_rows): P = X_(1) V with V = Omega_1 (Algorithm 1 step 6,
//   Eq. sampleMatrix; Gaussian entries from the reduced-precision counter
//   stream) or V = W of a power iteration (step 10).  Tensor-core problem:
//   M = I (rows i), N = l, K = J.  The A operand needs K (= j) contiguous, the
//   transpose of X's layout, so each thread loads one row i for 16 of the 32
//   columns j of a chunk (coalesced across the warp) and writes them as half of
//   the row's 128-byte swizzled line.  (A variant that landed X in a six-chunk
//   cp.async ring in shared memory, one CTA per SM, measured slower: the
//   per-chunk split and hand-off, not the loads, bound these sweeps.)
//   Each CTA owns 128 rows and a contiguous range of j (split over J).  Two
//   shared-memory stages and two register buffers: the loads of chunk k + 2 are
//   in flight while chunk k + 1 is staged and the MMAs of chunk k run.  A ninth
//   warp only issues the MMAs, so no staging warp waits for the issue.
// Column sweep (k_tc_cols): W = X_(1)^T Q (Algorithm 1 step 9) or the mode
//   product T_2 = X x_1 Q_1^T (step 13).  M = J (128 columns j per block),
//   N = l, K = I: K is X's contiguous direction, so 16-byte loads go straight
//   into the swizzled tile.  Persistent CTAs walk j-blocks.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "rcp_internal.cuh"
#include "tc_ptx.cuh"

namespace rcp {
namespace {

constexpr int kATile = 16384;  // 128 rows x 128 bytes
constexpr int kTT = 256;       // staging threads per CTA: two per tile row, 8 warps
constexpr int kCTA = kTT + 32; // plus one warp that only issues the MMAs

// Barrier 1 between the staging warps and the issuing warp (every thread of the CTA).
__device__ __forceinline__ void stage_barrier() {
  asm volatile("bar.sync 1, %0;" ::"n"(kCTA) : "memory");
}
constexpr int kNB = 2;         // register buffers: chunk k + 2 loads while k + 1 waits to be staged
constexpr long long kWaitBudget = 1LL << 31;  // clock cycles (about 1 s)

// FP32 = hi + lo with hi = the value truncated to TF32 (10 fraction bits) and
// lo = the exact remainder; hi * hi + hi * lo + lo * hi keeps about 21 bits.
__device__ __forceinline__ float tf32_hi(float x) {
  return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}

// Stage layout shared by both kernels: [A hi | A lo | B hi | B lo], each tile
// K-major, 128-byte swizzled, 1024-byte aligned.
template <int NP>
struct Stage {
  static constexpr int kA = kATile;
  static constexpr int kB = NP * 128;
  static constexpr int kBytes = 2 * kA + 2 * kB;
  static constexpr int kSmem = 2 * kBytes + 1024;
};

__device__ __forceinline__ void issue_3xtf32(uint32_t d, uint32_t ahi, uint32_t alo, uint32_t bhi,
                                             uint32_t blo, uint32_t idesc, bool first) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t o = 32u * k;
    tc::mma_tf32(d, tc::desc_kmajor_sw128(ahi + o), tc::desc_kmajor_sw128(bhi + o), idesc,
                 (first && k == 0) ? 0u : 1u);
    tc::mma_tf32(d, tc::desc_kmajor_sw128(ahi + o), tc::desc_kmajor_sw128(blo + o), idesc, 1u);
    tc::mma_tf32(d, tc::desc_kmajor_sw128(alo + o), tc::desc_kmajor_sw128(bhi + o), idesc, 1u);
  }
}

// Row sweep, one M = 128 block of rows per CTA (256 threads, two per row).
template <int NP, int SRC, bool NORM>
__global__ void __launch_bounds__(kCTA, 2)
k_tc_rows(const float* __restrict__ X, int64_t I, int64_t J, int l, uint64_t seed, uint32_t sid,
          const float* __restrict__ WT, int64_t jchunk, float* __restrict__ part,
          double* __restrict__ normpart, DevState* st) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t mbar[2];   // stage s free: the MMAs that read it completed
  __shared__ uint32_t tbase_sh;
  __shared__ int abort_sh;
  __shared__ double red[8];
  __shared__ uint16_t boff[32 * 64];  // element t = jj * l + c of a chunk -> its byte offset in B
  using S = Stage<NP>;
  constexpr uint32_t NCOLS = NP;
  constexpr uint32_t IDESC = tc::idesc_tf32(128, NP);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t i0 = (int64_t)blockIdx.x * 128;
  const int64_t jb = (int64_t)blockIdx.y * jchunk;
  const int64_t je = min(J, jb + jchunk);

  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    abort_sh = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(&tbase_sh, NCOLS);
  const bool issuer = warp == kTT / 32;
  for (int k = issuer ? 2 * 2 * NP * 32 : tid; k < 2 * 2 * NP * 32; k += kTT) {  // B rows c >= l stay zero
    const int s = k / (2 * NP * 32), e = k % (2 * NP * 32);
    *(float*)(sm + s * S::kBytes + 2 * S::kA + 4 * e) = 0.0f;
  }
  for (int t = issuer ? 32 * l : tid; t < 32 * l; t += kTT) {
    const int jj = t / l, c = t - jj * l;
    boff[t] = (uint16_t)tc::sw128_offset((uint32_t)c, (uint32_t)jj);
  }
  tc::tc_fence_before_sync();
  __syncthreads();
  tc::tc_fence_after_sync();
  const uint32_t tbase = tbase_sh;

  const int rl = tid & 127, half = tid >> 7;  // tile row, and which 16 of the 32 columns
  const int64_t row = i0 + rl;
  const bool row_ok = row < I;
  const int nk = (int)((je - jb + 31) / 32);
  constexpr int WV = NP * 32 / kTT;  // W^T values per thread and chunk
  float xbuf[kNB][16];
  float wbuf[kNB][WV];  // SRC 1: this thread's W^T values of a chunk (t = tid + kTT k)
  double nrm = 0.0;  // |X|^2 of this thread's elements: FP32 per chunk, FP64 across chunks
  uint32_t par0 = 0, par1 = 0;
  auto load_w = [&](float (&wr)[WV], int kc) {
    const int64_t j0 = jb + 32LL * kc;
#pragma unroll
    for (int k = 0; k < WV; ++k) {
      const int t = tid + kTT * k;  // t = c * 32 + jj, covering NP x 32
      const int c = t >> 5, jj = t & 31;
      const int64_t j = j0 + jj;
      wr[k] = (c < l && j < je) ? __ldg(WT + (int64_t)c * J + j) : 0.0f;
    }
  };

  auto load = [&](float (&xr)[16], int kc) {
    const int64_t j0 = jb + 32LL * kc + 16 * half;
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) {
      const int64_t j = j0 + jj;
      xr[jj] = (row_ok && j < je) ? __ldg(X + row + I * j) : 0.0f;
    }
  };
  auto put_b = [&](uint8_t* Bh, uint8_t* Bl, uint32_t off, float v) {
    const float h = tf32_hi(v);
    *(float*)(Bh + off) = h;
    *(float*)(Bl + off) = v - h;
  };
  // one 32-column chunk: stage it, prefetch chunk kc + 2 into the same registers, issue MMAs
  auto step = [&](float (&xr)[16], float (&wr)[WV], int kc) -> bool {
    const int s = kc & 1;
    uint8_t* Ah = sm + s * S::kBytes;
    uint8_t* Al = Ah + S::kA;
    uint8_t* Bh = Al + S::kA;
    uint8_t* Bl = Bh + S::kB;
    if (kc >= 2) {
      const uint32_t par = s ? par1 : par0;
      if (!tc::mbar_wait(&mbar[s], par, kWaitBudget)) atomicExch(&abort_sh, 1);
      if (s) par1 ^= 1; else par0 ^= 1;
    }
    const uint32_t rr = (uint32_t)rl;
    float cn = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float4 h, lo;
      h.x = tf32_hi(xr[4 * c]);     lo.x = xr[4 * c] - h.x;
      h.y = tf32_hi(xr[4 * c + 1]); lo.y = xr[4 * c + 1] - h.y;
      h.z = tf32_hi(xr[4 * c + 2]); lo.z = xr[4 * c + 2] - h.z;
      h.w = tf32_hi(xr[4 * c + 3]); lo.w = xr[4 * c + 3] - h.w;
      if (NORM)
        cn += xr[4 * c] * xr[4 * c] + xr[4 * c + 1] * xr[4 * c + 1] +
              xr[4 * c + 2] * xr[4 * c + 2] + xr[4 * c + 3] * xr[4 * c + 3];
      const uint32_t cc = (uint32_t)(4 * half + c);  // 16-byte chunk of the 128-byte row
      const uint32_t off = rr * 128 + (((cc ^ (rr & 7u)) & 7u) << 4);
      *(float4*)(Ah + off) = h;
      *(float4*)(Al + off) = lo;
    }
    if (NORM) nrm += (double)cn;
    const int64_t j0 = jb + 32LL * kc;
    if (SRC == 0) {
      if (kc + kNB < nk) load(xr, kc + kNB);
      // Omega_1[j, c] = element e = j l + c of the reduced-precision stream; local
      // index t = e - j0 l in [0, 32 l), counters g = e / 4 from g0 = (j0 l) / 4
      const int64_t e0 = j0 * l;
      const int lead = (int)(e0 & 3);                      // elements of quad g0 before e0
      const int tend = (int)min((int64_t)32, je - j0) * l;  // valid elements of this chunk
      const int nq = (32 * l + lead + 3) >> 2;
      for (int q = tid; q < nq; q += kTT) {
        const float4 z = normal_quad_f32(seed, sid, kPurposeSketch, (uint64_t)((e0 >> 2) + q));
        const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int t = 4 * q + u - lead;
          if (t >= 0 && t < 32 * l) put_b(Bh, Bl, boff[t], t < tend ? zz[u] : 0.0f);
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < WV; ++k) {
        const int t = tid + kTT * k;
        const int c = t >> 5, jj = t & 31;
        if (c < l) put_b(Bh, Bl, tc::sw128_offset((uint32_t)c, (uint32_t)jj), wr[k]);
      }
      if (kc + kNB < nk) {
        load(xr, kc + kNB);
        load_w(wr, kc + kNB);
      }
    }
    // hand the stage to the issuing warp (variants that used a CTA barrier with the
    // issue by thread 0, or an mbarrier with one arrival per thread, measured slower)
    tc::fence_proxy_async_smem();
    stage_barrier();
    return !abort_sh;
  };

  bool ok = true;
  if (issuer) {
    for (int kc = 0; kc < nk; ++kc) {
      stage_barrier();
      if (abort_sh) break;
      if (lane == 0) {
        const int s = kc & 1;
        uint8_t* Ah = sm + s * S::kBytes;
        uint8_t* Al = Ah + S::kA;
        uint8_t* Bh = Al + S::kA;
        uint8_t* Bl = Bh + S::kB;
        tc::tc_fence_after_sync();
        issue_3xtf32(tbase, tc::smem_u32(Ah), tc::smem_u32(Al), tc::smem_u32(Bh),
                     tc::smem_u32(Bl), IDESC, kc == 0);
        tc::mma_commit(&mbar[s]);
      }
      __syncwarp();
    }
  } else {
#pragma unroll
    for (int b = 0; b < kNB; ++b) {
      if (b < nk) {
        load(xbuf[b], b);
        if (SRC == 1) load_w(wbuf[b], b);
      }
    }
    for (int kc = 0; kc < nk && ok; kc += kNB) {
#pragma unroll
      for (int b = 0; b < kNB; ++b)
        if (ok && kc + b < nk) ok = step(xbuf[b], wbuf[b], kc + b);
    }
  }
  // the staging warps (whose phase bits track the stage barriers) wait for the last MMAs
  for (int kc = (nk >= 2 ? nk - 2 : 0); kc < nk && ok && !issuer; ++kc) {
    const int s = kc & 1;
    const uint32_t par = s ? par1 : par0;
    if (!tc::mbar_wait(&mbar[s], par, kWaitBudget)) ok = false;
    if (s) par1 ^= 1; else par0 ^= 1;
  }
  tc::tc_fence_after_sync();
  if (!ok && tid == 0) set_status(st, RCP_ETIMEOUT);

  // a wait that gave up may leave MMAs in flight: then tensor memory is not read
  // (the partials are zeroed) and the launch only records RCP_ETIMEOUT
  const bool ok_all = __syncthreads_and(ok) != 0;
  if (warp < 4) {  // warp w reads tensor-memory lanes 32 w .. 32 w + 31
    const int64_t r = i0 + warp * 32 + lane;
#pragma unroll
    for (int cg = 0; cg < NP / 32; ++cg) {
      float v[32];
      if (ok_all && nk > 0) {
        tc::tmem_ld32(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cg * 32), v);
      } else {
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = 0.0f;
      }
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        const int col = cg * 32 + k;
        if (col < l && r < I)
          part[((int64_t)blockIdx.y * l + col) * I + r] = v[k];
      }
    }
  }
  if (NORM) {
    double d = nrm;
    for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
    if (lane == 0) red[warp] = d;
  }
  tc::tc_fence_before_sync();
  __syncthreads();
  if (NORM && tid == 0) normpart[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] =
      ((red[0] + red[1]) + (red[2] + red[3])) + ((red[4] + red[5]) + (red[6] + red[7]));
  if (warp == 0) tc::tmem_dealloc(tbase, NCOLS);
}

// out = X_(1)^T Q for every j: TTM ? row-major J x l (the Kolda layout of T_2)
//                                     : l x J (the power-iteration W, transposed).
// Two tensor-memory accumulators: the epilogue of j-block b runs while the
// MMAs of block b + 1 are queued.
template <int NP, bool TTM>
__global__ void __launch_bounds__(kCTA, 2)
k_tc_cols(const float* __restrict__ X, int64_t I, int64_t J, int l, int64_t Ipad,
          const float* __restrict__ QTh, const float* __restrict__ QTl, float* __restrict__ out,
          DevState* st) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t mbar[3];  // two stages free + accumulator ready
  __shared__ uint32_t tbase_sh;
  __shared__ int abort_sh;
  using S = Stage<NP>;
  constexpr uint32_t NCOLS = 2 * NP;
  constexpr uint32_t IDESC = tc::idesc_tf32(128, NP);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int k = 0; k < 3; ++k) tc::mbar_init(&mbar[k], 1);
    abort_sh = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(&tbase_sh, NCOLS);
  tc::tc_fence_before_sync();
  __syncthreads();
  tc::tc_fence_after_sync();
  const uint32_t tbase = tbase_sh;

  const int nkc = (int)(Ipad / 32);
  const int64_t njb = (J + 127) / 128;
  const int64_t my_blocks = (njb > blockIdx.x) ? (njb - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const int64_t total = my_blocks * nkc;
  const int c16 = tid & 7, r0 = tid >> 3;  // 16-byte chunk along i; rows r0 + 32 p
  constexpr int QV = NP * 8 / kTT;  // float4 of Q^T hi (and lo) per thread and chunk
  constexpr int NB = kNB;
  float4 xbuf[NB][4];
  float4 qbuf[NB][2 * QV];
  uint32_t par0 = 0, par1 = 0, pacc = 0;
  auto load_q = [&](float4 (&qv)[2 * QV], int64_t g) {
    const int kc = (int)(g % nkc);
#pragma unroll
    for (int k = 0; k < QV; ++k) {
      const int t = tid + kTT * k;  // t = c * 8 + cc
      const int c = t >> 3, cc = t & 7;
      const int64_t src = (int64_t)c * Ipad + 32LL * kc + 4 * cc;
      qv[k] = __ldg((const float4*)(QTh + src));
      qv[QV + k] = __ldg((const float4*)(QTl + src));
    }
  };

  auto load = [&](float4 (&xv)[4], int64_t g) {
    const int64_t jblk = blockIdx.x + (g / nkc) * gridDim.x;
    const int kc = (int)(g % nkc);
    const int64_t i = 32LL * kc + 4 * c16;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int64_t j = jblk * 128 + r0 + 32 * p;
      xv[p] = (j < J && i < I) ? __ldg((const float4*)(X + j * I + i)) : make_float4(0, 0, 0, 0);
    }
  };
  auto epilogue = [&](int64_t blk_local) -> bool {
    bool good = tc::mbar_wait(&mbar[2], pacc, kWaitBudget);
    pacc ^= 1;
    tc::tc_fence_after_sync();
    const int64_t jblk = blockIdx.x + blk_local * gridDim.x;
    const int64_t j = jblk * 128 + warp * 32 + lane;
    const uint32_t acc = tbase + (uint32_t)((blk_local & 1) * NP);
#pragma unroll
    for (int cg = 0; cg < NP / 32 && warp < 4; ++cg) {  // warp w: tensor-memory lanes 32 w ..
      float v[32];
      tc::tmem_ld32(acc + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cg * 32), v);
      if (j < J && good) {
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          const int c = cg * 32 + k;
          if (c < l) {
            if (TTM) out[j * l + c] = v[k];
            else out[(int64_t)c * J + j] = v[k];
          }
        }
      }
    }
    tc::tc_fence_before_sync();
    return good;
  };
  auto step = [&](float4 (&xv)[4], float4 (&qv)[2 * QV], int64_t g) -> bool {
    const int s = (int)(g & 1);
    const int kc = (int)(g % nkc);
    const int64_t blk = g / nkc;
    uint8_t* Ah = sm + s * S::kBytes;
    uint8_t* Al = Ah + S::kA;
    uint8_t* Bh = Al + S::kA;
    uint8_t* Bl = Bh + S::kB;
    if (g >= 2) {
      const uint32_t par = s ? par1 : par0;
      if (!tc::mbar_wait(&mbar[s], par, kWaitBudget)) atomicExch(&abort_sh, 1);
      if (s) par1 ^= 1; else par0 ^= 1;
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const uint32_t r = (uint32_t)(r0 + 32 * p);
      const uint32_t off = r * 128 + ((((uint32_t)c16 ^ (r & 7u)) & 7u) << 4);
      float4 h, lo;
      h.x = tf32_hi(xv[p].x); lo.x = xv[p].x - h.x;
      h.y = tf32_hi(xv[p].y); lo.y = xv[p].y - h.y;
      h.z = tf32_hi(xv[p].z); lo.z = xv[p].z - h.z;
      h.w = tf32_hi(xv[p].w); lo.w = xv[p].w - h.w;
      *(float4*)(Ah + off) = h;
      *(float4*)(Al + off) = lo;
    }
#pragma unroll
    for (int k = 0; k < QV; ++k) {
      const int t = tid + kTT * k;
      const int c = t >> 3, cc = t & 7;
      const uint32_t off = c * 128 + ((((uint32_t)cc ^ ((uint32_t)c & 7u)) & 7u) << 4);
      *(float4*)(Bh + off) = qv[k];
      *(float4*)(Bl + off) = qv[QV + k];
    }
    if (g + NB < total) {
      load(xv, g + NB);
      load_q(qv, g + NB);
    }
    // hand the stage to the issuing warp; that barrier also orders the epilogue of
    // block blk - 2 (same accumulator, read by warps 0-3 before they staged chunk 0
    // of block blk) before the MMAs into it
    tc::fence_proxy_async_smem();
    stage_barrier();
    if (abort_sh) return false;
    bool good = true;
    if (kc == 0 && blk > 0) good = epilogue(blk - 1);
    return good;
  };

  const bool issuer = warp == kTT / 32;
  bool ok = true;
  if (issuer) {
    for (int64_t g = 0; g < total; ++g) {
      stage_barrier();
      if (abort_sh) break;
      if (lane == 0) {
        const int s = (int)(g & 1);
        const int kc = (int)(g % nkc);
        const int64_t blk = g / nkc;
        uint8_t* Ah = sm + s * S::kBytes;
        uint8_t* Al = Ah + S::kA;
        uint8_t* Bh = Al + S::kA;
        uint8_t* Bl = Bh + S::kB;
        tc::tc_fence_after_sync();
        issue_3xtf32(tbase + (uint32_t)((blk & 1) * NP), tc::smem_u32(Ah), tc::smem_u32(Al),
                     tc::smem_u32(Bh), tc::smem_u32(Bl), IDESC, kc == 0);
        tc::mma_commit(&mbar[s]);
        if (kc == nkc - 1) tc::mma_commit(&mbar[2]);
      }
      __syncwarp();
    }
  } else {
    if (total > 0) {
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        if (b < total) {
          load(xbuf[b], b);
          load_q(qbuf[b], b);
        }
      }
    }
    for (int64_t g = 0; g < total && ok; g += NB) {
#pragma unroll
      for (int b = 0; b < NB; ++b)
        if (ok && g + b < total) ok = step(xbuf[b], qbuf[b], g + b);
    }
    if (ok && total > 0) ok = epilogue(my_blocks - 1);
  }
  // the staging warps (whose phase bits track the stage barriers) wait for the last MMAs
  for (int64_t g = (total >= 2 ? total - 2 : 0); g < total && ok && !issuer; ++g) {
    const int s = (int)(g & 1);
    const uint32_t par = s ? par1 : par0;
    if (!tc::mbar_wait(&mbar[s], par, kWaitBudget)) ok = false;
    if (s) par1 ^= 1; else par0 ^= 1;
  }
  if (!ok && tid == 0) set_status(st, RCP_ETIMEOUT);
  tc::tc_fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, NCOLS);
}

// Column sweep with TMA-fed stages (the form used whenever the tensor maps
// can be built).  Per 32-row chunk kc of X's contiguous direction i and block
// of 128 columns j:
//   X producer (warp 0)  one thread: the 128 x 32 tile of X lands by TMA, in
//                        the 128-byte swizzled K-major layout, in a ring of RS
//                        stages that the converters free as soon as they have
//                        read it: HBM needs about 128 KB of loads in flight per
//                        SM, and a stage held through the MMAs' completion
//                        would leave too few in flight;
//   B producer (warp 10) one thread: the 2NP x 32 tile of [Q^T hi; Q^T lo] (from
//                        L2) into a ring of kTS stages freed by the MMAs;
//   converters (2-5)     thread = one row j of the A tile: its 32 values split
//                        into the TF32 truncation and the remainder, written to
//                        tensor memory (lane j), kTS stages of 64 columns;
//   issuer (warp 1)      one thread: A_hi [Q_hi | Q_lo] (N = 2 NP) and A_lo Q_hi
//                        (N = NP), A from tensor memory, into one accumulator,
//                        so columns [0, NP) collect hi*hi + lo*hi and
//                        [NP, 2 NP) hi*lo;
//   epilogue (6-9)       the sum of the two halves, written out; two
//                        accumulators, so block b's epilogue overlaps block
//                        b + 1's MMAs.
constexpr int kColsThreads = 352;
constexpr int kEpiPitchPad = 1;
constexpr int kTS = 4;  // tensor-memory A stages
constexpr int kGrp = 2; // chunks per hand-off to the MMA thread (kTS / kGrp hand-off slots)
constexpr int kSlots = kTS / kGrp;

__host__ __device__ constexpr uint32_t tmem_cols_pow2(uint32_t n) {
  return n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : n <= 256 ? 256 : 512;
}

template <int NP, int RS, int BS, bool TTM, bool WSPLIT = false>
__global__ void __launch_bounds__(kColsThreads, 1)
k_tc_cols_tma(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmQ,
              int64_t J, int l, int nkc, float* __restrict__ out, DevState* st) {
  constexpr uint32_t kA = kATile;
  constexpr uint32_t kB = 2 * NP * 128;
  constexpr uint32_t NACC = 2 * NP;          // tensor-memory columns of one accumulator
  constexpr uint32_t ACOL = 2 * NACC;        // first column of the A stages (64 columns each)
  constexpr uint32_t NCOLS = tmem_cols_pow2(ACOL + kTS * 64);
  constexpr uint32_t IDESC_W = tc::idesc_tf32(128, 2 * NP);
  constexpr uint32_t IDESC_N = tc::idesc_tf32(128, NP);
  constexpr int EP = NP + kEpiPitchPad;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* rawb = sm;                        // RS x 16 KB of X
  uint8_t* bring = sm + RS * kA;             // BS x kB of [Q_hi; Q_lo]
  float* ep = (float*)(bring + BS * kB);     // TTM epilogue rows (4 warps x 32 rows x EP)
  __shared__ uint64_t rfull[RS], rempty[RS], bfull[BS], bfree[BS], tconv[kSlots], tfree[kSlots],
      accf[2], acce[2];
  __shared__ uint32_t tbase_sh;
  __shared__ volatile int abort_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < RS; ++s) {
      tc::mbar_init(&rfull[s], 1);
      tc::mbar_init(&rempty[s], 4);
    }
    for (int s = 0; s < BS; ++s) {
      tc::mbar_init(&bfull[s], 1);
      tc::mbar_init(&bfree[s], 1);
    }
    for (int s = 0; s < kSlots; ++s) {
      tc::mbar_init(&tconv[s], 4);
      tc::mbar_init(&tfree[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&accf[b], 1);
      tc::mbar_init(&acce[b], 4);
    }
    abort_sh = 0;
    tc::fence_mbar_init();
    tc::tma_prefetch_desc(&tmX);
    tc::tma_prefetch_desc(&tmQ);
  }
  if (warp == 1) tc::tmem_alloc(&tbase_sh, NCOLS);
  tc::tc_fence_before_sync();
  __syncthreads();
  tc::tc_fence_after_sync();
  const uint32_t tbase = tbase_sh;

  const int64_t njb = (J + 127) / 128;
  const int64_t nblk = njb > blockIdx.x ? (njb - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const int64_t total = nblk * nkc;
  bool ok = true;
  auto fail = [&]() {
    ok = false;
    abort_sh = 1;
  };

  if (warp == 0) {
    // ---- producer of the X ring
    if (lane == 0) {
      int64_t issued = 0;
      for (int64_t g = 0; g < total && !abort_sh; ++g) {
        const int r = (int)(g % RS);
        if (g >= RS && !tc::mbar_wait(&rempty[r], (uint32_t)((g / RS - 1) & 1), kWaitBudget)) {
          fail();
          break;
        }
        const int64_t jblk = blockIdx.x + (g / nkc) * gridDim.x;
        tc::mbar_arrive_expect_tx(&rfull[r], kA);
        tc::tma_load_2d(rawb + r * kA, &tmX, 32 * (int)(g % nkc), (int32_t)(jblk * 128), &rfull[r]);
        issued = g + 1;
      }
      // every copy issued has landed before the CTA may leave (bounded)
      for (int64_t g = issued > RS ? issued - RS : 0; g < issued; ++g)
        if (!tc::mbar_wait(&rfull[g % RS], (uint32_t)((g / RS) & 1), kWaitBudget)) fail();
    }
  } else if (warp == 10) {
    // ---- producer of the B ring
    if (lane == 0) {
      int64_t issued = 0;
      for (int64_t g = 0; g < total && !abort_sh; ++g) {
        const int b = (int)(g % BS);
        if (g >= BS && !tc::mbar_wait(&bfree[b], (uint32_t)((g / BS - 1) & 1), kWaitBudget)) {
          fail();
          break;
        }
        tc::mbar_arrive_expect_tx(&bfull[b], kB);
        tc::tma_load_2d(bring + b * kB, &tmQ, 32 * (int)(g % nkc), 0, &bfull[b]);
        issued = g + 1;
      }
      for (int64_t g = issued > BS ? issued - BS : 0; g < issued; ++g)
        if (!tc::mbar_wait(&bfull[g % BS], (uint32_t)((g / BS) & 1), kWaitBudget)) fail();
    }
  } else if (warp == 1) {
    // ---- MMA issuer.  This thread's shared-memory accesses (barrier polls, flags)
    // wait behind its MMAs in flight, so the loop polls once per group of kGrp
    // chunks and keeps its indices in registers (no divisions).
    if (lane == 0) {
      int64_t issued = 0;
      int kc = 0, b = 0, acc = 0, slot = 0;
      int64_t bl = 0;
      uint32_t sph = 0;
      for (int64_t g0 = 0; g0 < total; g0 += kGrp) {
        // the group's chunks are converted and their B tiles have landed
        if (!tc::mbar_wait(&tconv[slot], sph, kWaitBudget)) {
          fail();
          break;
        }
        tc::tc_fence_after_sync();
        bool bad = false;
        for (int c = 0; c < kGrp && g0 + c < total; ++c) {
          if (kc == 0 && bl >= 2 &&
              !tc::mbar_wait(&acce[acc], (uint32_t)((bl / 2 - 1) & 1), kWaitBudget)) {
            bad = true;
            break;
          }
          const uint32_t d = tbase + (uint32_t)acc * NACC;
          const uint32_t ahi = tbase + ACOL + (uint32_t)(slot * kGrp + c) * 64;
          const uint32_t bq = tc::smem_u32(bring + b * kB);
#pragma unroll
          for (int k = 0; k < 4; ++k)
            tc::mma_tf32_tmem_a(d, ahi + 8u * k, tc::desc_kmajor_sw128(bq + 32u * k), IDESC_W,
                                (kc > 0 || k > 0) ? 1u : 0u);
#pragma unroll
          for (int k = 0; k < 4; ++k)
            tc::mma_tf32_tmem_a(d, ahi + 32u + 8u * k, tc::desc_kmajor_sw128(bq + 32u * k),
                                IDESC_N, 1u);
          tc::mma_commit(&bfree[b]);
          if (kc == nkc - 1) tc::mma_commit(&accf[acc]);
          issued = g0 + c + 1;
          if (++b == BS) b = 0;
          if (++kc == nkc) {
            kc = 0;
            ++bl;
            acc ^= 1;
          }
        }
        tc::mma_commit(&tfree[slot]);
        if (bad) {
          fail();
          break;
        }
        if (++slot == kSlots) {
          slot = 0;
          sph ^= 1u;
        }
      }
      // the tensor cores are done with every stage before the CTA may leave
      for (int64_t g = issued > BS ? issued - BS : 0; g < issued; ++g)
        if (!tc::mbar_wait(&bfree[g % BS], (uint32_t)((g / BS) & 1), kWaitBudget)) fail();
    }
  } else if (warp < 6) {
    // ---- converters: warp w owns tile rows (tensor-memory lanes) 32 (w % 4) .. + 31
    const int q = warp & 3;
    const uint32_t row = (uint32_t)(32 * q + lane);
    for (int64_t g = 0; g < total && !abort_sh; ++g) {
      const int r = (int)(g % RS), t = (int)(g % kTS);
      if (!tc::mbar_wait(&rfull[r], (uint32_t)((g / RS) & 1), kWaitBudget)) {
        fail();
        break;
      }
      const uint8_t* A = rawb + r * kA;
      float hv[32], lv[32];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float4 v = *(const float4*)(A + row * 128 + ((((uint32_t)c ^ (row & 7u)) & 7u) << 4));
        hv[4 * c] = tf32_hi(v.x);     lv[4 * c] = v.x - hv[4 * c];
        hv[4 * c + 1] = tf32_hi(v.y); lv[4 * c + 1] = v.y - hv[4 * c + 1];
        hv[4 * c + 2] = tf32_hi(v.z); lv[4 * c + 2] = v.z - hv[4 * c + 2];
        hv[4 * c + 3] = tf32_hi(v.w); lv[4 * c + 3] = v.w - hv[4 * c + 3];
      }
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&rempty[r]);  // the raw tile is in registers now
      // group gq = g / kGrp uses slot gq % kSlots (A stages slot kGrp .. + kGrp - 1);
      // its first chunk waits until the MMAs of the slot's previous group are done
      const int64_t gq = g / kGrp;
      const int slot = (int)(gq % kSlots), cg = (int)(g % kGrp);
      if (cg == 0 && gq >= kSlots &&
          !tc::mbar_wait(&tfree[slot], (uint32_t)((gq / kSlots - 1) & 1), kWaitBudget)) {
        fail();
        break;
      }
      tc::tc_fence_after_sync();
      const uint32_t ta = tbase + ((uint32_t)(32 * q) << 16) + ACOL + (uint32_t)t * 64;
      tc::tmem_st32(ta, hv);
      tc::tmem_st32(ta + 32u, lv);
      tc::tmem_st_wait();
      tc::tc_fence_before_sync();
      __syncwarp();
      if (lane == 0) {
        // the B tile of this chunk has landed too (the issuer waits on tconv only)
        if (!tc::mbar_wait(&bfull[g % BS], (uint32_t)((g / BS) & 1), kWaitBudget)) fail();
        if (cg == kGrp - 1 || g == total - 1) tc::mbar_arrive(&tconv[slot]);
      }
    }
  } else {
    // ---- epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31
    const int q = warp & 3;
    for (int64_t bl = 0; bl < nblk && !abort_sh; ++bl) {
      const int acc = (int)(bl & 1);
      if (!tc::mbar_wait(&accf[acc], (uint32_t)((bl / 2) & 1), kWaitBudget)) {
        fail();
        break;
      }
      tc::tc_fence_after_sync();
      const int64_t jblk = blockIdx.x + bl * gridDim.x;
      const int64_t j = jblk * 128 + 32 * q + lane;
      const uint32_t ta = tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)acc * NACC;
#pragma unroll
      for (int cg = 0; cg < NP / 32; ++cg) {
        float a[32], b[32];
        tc::tmem_ld32(ta + (uint32_t)(cg * 32), a);
        tc::tmem_ld32(ta + (uint32_t)(NP + cg * 32), b);
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          const int c = cg * 32 + k;
          const float v = a[k] + b[k];
          if (TTM) {
            ep[(32 * q + lane) * EP + c] = v;
          } else if (c < l && j < J) {
            if (WSPLIT) {  // [W_hi; W_lo], l x J each, for the TMA-fed row sweep
              const float hv = tf32_hi(v);
              out[(int64_t)c * J + j] = hv;
              out[((int64_t)l + c) * J + j] = v - hv;
            } else {
              out[(int64_t)c * J + j] = v;
            }
          }
        }
      }
      tc::tc_fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&acce[acc]);
      if (TTM) {
        // rows j0 .. j0 + 31 of the row-major J x l output are one contiguous run
        const int64_t j0 = jblk * 128 + 32 * q;
        const int64_t nrow = J - j0 < 32 ? J - j0 : 32;
        const int64_t n = nrow > 0 ? nrow * l : 0;
        float* o = out + j0 * l;
        for (int64_t e = lane; e < n; e += 32) {
          const int r = (int)(e / l), c = (int)(e - (int64_t)r * l);
          o[e] = ep[(32 * q + r) * EP + c];
        }
        __syncwarp();
      }
    }
  }
  if (!ok) set_status(st, RCP_ETIMEOUT);
  tc::tc_fence_before_sync();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tbase, NCOLS);
}

// Row sweep with TMA-fed stages for the power iteration's apply step,
// P = X_(1) W over this CTA's row block (rb rows of i, rb a multiple of 4, the
// blocks as equal as possible) and its range of 32-column chunks of j; W is
// stored by the column sweep as [W_hi; W_lo], l x J each.  (The sketch, whose
// cost is drawing Omega_1 per chunk, keeps the register-staged k_tc_rows: two
// CTAs of 8 warps per SM share the draw.  A TMA-fed form measured slower with
// the draw in its converters, and slower still with four generator warps.)
//   X producer (warp 0) one thread: the rb x 32 tile of X (i contiguous, no
//                       swizzle) lands by TMA in a ring of RS stages that the
//                       converters free once they have read it;
//   B producer (10)     one thread: the 2NP x 32 tile of [W_hi; W_lo]
//                       (128-byte swizzle) into a ring of kTS stages freed by
//                       the MMAs;
//   converters (2-9)    256 threads, thread = row r (tensor-memory lane) and
//                       one half of the chunk's 32 columns: the row's values
//                       split into TF32 truncation and remainder, written to
//                       tensor memory (rows >= rb as zeros);
//   issuer (warp 1)     one thread: A_hi [V_hi | V_lo] (N = 2 NP) and A_lo V_hi
//                       (N = NP), A from tensor memory, into one accumulator
//                       for the whole range;
//   epilogue            converter warps 2-5 (tensor-memory lanes 64 .. 127,
//                       0 .. 63): the two halves summed into the split's partial.
constexpr int kRowsThreads = 352;

template <int NP, int RS, int BS>
__global__ void __launch_bounds__(kRowsThreads, 1)
k_tc_rows_tma(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW,
              int64_t I, int64_t J, int l, int rb, int64_t cper, float* __restrict__ part,
              DevState* st) {
  constexpr uint32_t kB = 2 * NP * 128;
  constexpr uint32_t kXR = 16384;                      // X stage (rb x 32 floats, rb <= 128)
  constexpr uint32_t NACC = 2 * NP;
  constexpr uint32_t ACOL = NACC;                      // A stages: 64 columns each
  constexpr uint32_t NCOLS = tmem_cols_pow2(ACOL + kTS * 64);
  constexpr uint32_t IDESC_W = tc::idesc_tf32(128, 2 * NP);
  constexpr uint32_t IDESC_N = tc::idesc_tf32(128, NP);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* rawb = sm;
  uint8_t* bring = sm + RS * kXR;                      // BS B stages of [W_hi; W_lo]
  __shared__ uint64_t rfull[RS], rempty[RS], bfull[BS], bfree[BS], tconv[kSlots], tfree[kSlots], accf;
  __shared__ uint32_t tbase_sh;
  __shared__ volatile int abort_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int blk = blockIdx.x, split = blockIdx.y;
  const int64_t i0 = (int64_t)blk * rb;
  const int64_t nchunk = (J + 31) / 32;
  const int64_t c0 = (int64_t)split * cper;
  const int64_t c1 = c0 + cper < nchunk ? c0 + cper : nchunk;
  const int64_t total = c1 > c0 ? c1 - c0 : 0;

  if (tid == 0) {
    for (int s = 0; s < RS; ++s) {
      tc::mbar_init(&rfull[s], 1);
      tc::mbar_init(&rempty[s], 8);
    }
    for (int s = 0; s < BS; ++s) {
      tc::mbar_init(&bfull[s], 1);
      tc::mbar_init(&bfree[s], 1);
    }
    for (int s = 0; s < kSlots; ++s) {
      tc::mbar_init(&tconv[s], 8);
      tc::mbar_init(&tfree[s], 1);
    }
    tc::mbar_init(&accf, 1);
    abort_sh = 0;
    tc::fence_mbar_init();
    tc::tma_prefetch_desc(&tmX);
    tc::tma_prefetch_desc(&tmW);
  }
  if (warp == 1) tc::tmem_alloc(&tbase_sh, NCOLS);
  tc::tc_fence_before_sync();
  __syncthreads();
  tc::tc_fence_after_sync();
  const uint32_t tbase = tbase_sh;
  bool ok = true;
  auto fail = [&]() {
    ok = false;
    abort_sh = 1;
  };

  if (warp == 0) {
    if (lane == 0) {
      int64_t issued = 0;
      for (int64_t g = 0; g < total && !abort_sh; ++g) {
        const int r = (int)(g % RS);
        if (g >= RS && !tc::mbar_wait(&rempty[r], (uint32_t)((g / RS - 1) & 1), kWaitBudget)) {
          fail();
          break;
        }
        tc::mbar_arrive_expect_tx(&rfull[r], (uint32_t)(rb * 32 * 4));
        tc::tma_load_2d(rawb + r * kXR, &tmX, (int32_t)i0, (int32_t)(32 * (c0 + g)), &rfull[r]);
        issued = g + 1;
      }
      for (int64_t g = issued > RS ? issued - RS : 0; g < issued; ++g)
        if (!tc::mbar_wait(&rfull[g % RS], (uint32_t)((g / RS) & 1), kWaitBudget)) fail();
    }
  } else if (warp == 10) {
    if (lane == 0) {
      int64_t issued = 0;
      for (int64_t g = 0; g < total && !abort_sh; ++g) {
        const int b = (int)(g % BS);
        if (g >= BS && !tc::mbar_wait(&bfree[b], (uint32_t)((g / BS - 1) & 1), kWaitBudget)) {
          fail();
          break;
        }
        tc::mbar_arrive_expect_tx(&bfull[b], kB);
        tc::tma_load_3d(bring + b * kB, &tmW, (int32_t)(32 * (c0 + g)), 0, 0, &bfull[b]);
        issued = g + 1;
      }
      for (int64_t g = issued > BS ? issued - BS : 0; g < issued; ++g)
        if (!tc::mbar_wait(&bfull[g % BS], (uint32_t)((g / BS) & 1), kWaitBudget)) fail();
    }
  } else if (warp == 1) {
    // MMA issuer: one poll per group of kGrp chunks, indices in registers (see
    // the column sweep)
    if (lane == 0) {
      int64_t issued = 0;
      int b = 0, slot = 0;
      uint32_t sph = 0;
      for (int64_t g0 = 0; g0 < total; g0 += kGrp) {
        if (!tc::mbar_wait(&tconv[slot], sph, kWaitBudget)) {
          fail();
          break;
        }
        tc::tc_fence_after_sync();
        for (int c = 0; c < kGrp && g0 + c < total; ++c) {
          const int64_t g = g0 + c;
          const uint32_t ahi = tbase + ACOL + (uint32_t)(slot * kGrp + c) * 64;
          const uint32_t bq = tc::smem_u32(bring + (uint32_t)b * kB);
#pragma unroll
          for (int k = 0; k < 4; ++k)
            tc::mma_tf32_tmem_a(tbase, ahi + 8u * k, tc::desc_kmajor_sw128(bq + 32u * k), IDESC_W,
                                (g > 0 || k > 0) ? 1u : 0u);
#pragma unroll
          for (int k = 0; k < 4; ++k)
            tc::mma_tf32_tmem_a(tbase, ahi + 32u + 8u * k, tc::desc_kmajor_sw128(bq + 32u * k),
                                IDESC_N, 1u);
          tc::mma_commit(&bfree[b]);
          issued = g + 1;
          if (++b == BS) b = 0;
        }
        tc::mma_commit(&tfree[slot]);
        if (++slot == kSlots) {
          slot = 0;
          sph ^= 1u;
        }
      }
      if (issued > 0) tc::mma_commit(&accf);
      for (int64_t g = issued > BS ? issued - BS : 0; g < issued; ++g)
        if (!tc::mbar_wait(&bfree[g % BS], (uint32_t)((g / BS) & 1), kWaitBudget)) fail();
    }
  } else {
    // ---- converters (256 threads): row r = lane of the warp's quarter, columns 16 h .. + 15
    const int q = warp & 3, h = (warp - 2) >> 2;
    const int r = 32 * q + lane;
    const bool rv = r < rb;
    for (int64_t g = 0; g < total && !abort_sh; ++g) {
      const int rs = (int)(g % RS), t = (int)(g % kTS);
      if (!tc::mbar_wait(&rfull[rs], (uint32_t)((g / RS) & 1), kWaitBudget)) {
        fail();
        break;
      }
      const float* Xr = (const float*)(rawb + rs * kXR);
      float hv[16], lv[16];
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        const float x = rv ? Xr[(16 * h + jj) * rb + r] : 0.0f;
        hv[jj] = tf32_hi(x);
        lv[jj] = x - hv[jj];
      }
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&rempty[rs]);  // the X tile is in registers now
      const int64_t gq = g / kGrp;
      const int slot = (int)(gq % kSlots), cg = (int)(g % kGrp);
      if (cg == 0 && gq >= kSlots &&
          !tc::mbar_wait(&tfree[slot], (uint32_t)((gq / kSlots - 1) & 1), kWaitBudget)) {
        fail();
        break;
      }
      tc::tc_fence_after_sync();
      const uint32_t ta = tbase + ((uint32_t)(32 * q) << 16) + ACOL + (uint32_t)t * 64 + 16u * h;
      tc::tmem_st16(ta, hv);
      tc::tmem_st16(ta + 32u, lv);
      tc::tmem_st_wait();
      tc::tc_fence_before_sync();
      __syncwarp();
      if (lane == 0) {
        if (!tc::mbar_wait(&bfull[g % BS], (uint32_t)((g / BS) & 1), kWaitBudget)) fail();
        if (cg == kGrp - 1 || g == total - 1) tc::mbar_arrive(&tconv[slot]);
      }
    }
    // ---- epilogue: warps 2-5 read tensor-memory lanes 32 (w % 4) .. + 31
    if (warp < 6) {
      const bool got = total > 0 && !abort_sh && tc::mbar_wait(&accf, 0, kWaitBudget);
      if (total > 0 && !got) fail();
      tc::tc_fence_after_sync();
      const int64_t i = i0 + r;
      const bool w = rv && i < I;
#pragma unroll
      for (int cg = 0; cg < NP / 32; ++cg) {
        float a[32], b[32];
        if (got) {
          tc::tmem_ld32(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(cg * 32), a);
          tc::tmem_ld32(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(NP + cg * 32), b);
        } else {
#pragma unroll
          for (int k = 0; k < 32; ++k) a[k] = b[k] = 0.0f;
        }
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          const int c = cg * 32 + k;
          if (w && c < l) part[((int64_t)split * l + c) * I + i] = a[k] + b[k];
        }
      }
    }
  }
  if (!ok) set_status(st, RCP_ETIMEOUT);
  tc::tc_fence_before_sync();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tbase, NCOLS);
}

// QT = Q^T in FP32 split into TF32 hi + lo, padded with zeros to NP x Ipad.
__global__ void k_q_to_qt32(const double* __restrict__ Q, int64_t I, int l, int NP, int64_t Ipad,
                            float* __restrict__ QTh, float* __restrict__ QTl) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)NP * Ipad) return;
  const int c = (int)(e / Ipad);
  const int64_t i = e % Ipad;
  const float v = (c < l && i < I) ? (float)Q[i + I * c] : 0.0f;
  const float h = tf32_hi(v);
  QTh[e] = h;
  QTl[e] = v - h;
}

__global__ void k_reduce_f32(const float* __restrict__ part, int64_t nsplit, int64_t n,
                             double* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  double acc = 0.0;
  for (int64_t s = 0; s < nsplit; ++s) acc += (double)part[s * n + e];
  out[e] = acc;
}

template <int NP, int SRC, bool NORM>
cudaError_t rows_launch(const float* X, int64_t I, int64_t J, int l, uint64_t seed, uint32_t sid,
                        const float* WT, int nsplit, int64_t jchunk, float* part,
                        double* normpart, DevState* st, cudaStream_t s) {
  auto kern = k_tc_rows<NP, SRC, NORM>;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Stage<NP>::kSmem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((I + 127) / 128), (unsigned)nsplit);
  count_launches(1);
  kern<<<grid, kCTA, Stage<NP>::kSmem, s>>>(X, I, J, l, seed, sid, WT, jchunk, part, normpart, st);
  return cudaGetLastError();
}

template <int NP, bool TTM>
cudaError_t cols_launch(const float* X, int64_t I, int64_t J, int l, int64_t Ipad,
                        const float* QT, float* out, DevState* st, int grid, cudaStream_t s) {
  auto kern = k_tc_cols<NP, TTM>;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Stage<NP>::kSmem);
  if (e != cudaSuccess) return e;
  count_launches(1);
  kern<<<grid, kCTA, Stage<NP>::kSmem, s>>>(X, I, J, l, Ipad, QT, QT + (int64_t)NP * Ipad, out, st);
  return cudaGetLastError();
}

// cuTensorMapEncodeTiled from the driver, resolved once through the runtime
// (no link against the driver library).
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
    else
      cudaGetLastError();
  }
  return fn;
}

// FP32 tensor map of rank 2 or 3 (dims innermost first, strides in bytes of
// dims 1..), box `box`; out-of-range elements read as zero.
bool tmap_f32(CUtensorMap* m, const float* base, int rank, const cuuint64_t* dims,
              const cuuint64_t* strides, const cuuint32_t* box, bool swizzle128) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_tiled();
  if (!enc || ((uintptr_t)base & 15)) return false;
  for (int k = 0; k < rank - 1; ++k)
    if (strides[k] % 16) return false;
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, (void*)base, dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2D FP32 tensor map over a row-major d1 x d0 array (row pitch d0), box
// b1 x 32 with the 128-byte swizzle.
bool tmap_2d_f32(CUtensorMap* m, const float* base, uint64_t d0, uint64_t d1, uint32_t b1) {
  const cuuint64_t dims[2] = {d0, d1};
  const cuuint64_t strides[1] = {d0 * 4};
  const cuuint32_t box[2] = {32, b1};
  return tmap_f32(m, base, 2, dims, strides, box, true);
}

template <int NP, int RS, int BS, bool TTM, bool WSPLIT = false>
cudaError_t cols_tma_launch(const CUtensorMap& tmX, const CUtensorMap& tmQ, int64_t J, int l,
                            int nkc, float* out, DevState* st, int grid, cudaStream_t s) {
  auto kern = k_tc_cols_tma<NP, RS, BS, TTM, WSPLIT>;
  const int smem = RS * kATile + BS * 2 * NP * 128 +
                   (TTM ? 4 * 32 * (NP + kEpiPitchPad) * 4 : 0) + 1024;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  count_launches(1);
  kern<<<grid, kColsThreads, smem, s>>>(tmX, tmQ, J, l, nkc, out, st);
  return cudaGetLastError();
}

template <int NP, int RS, int BS>
cudaError_t rows_tma_launch(const CUtensorMap& tmX, const CUtensorMap& tmW, int64_t I, int64_t J,
                            int l, int rb, int nb, int ns, int64_t cper, float* part, DevState* st,
                            cudaStream_t s) {
  auto kern = k_tc_rows_tma<NP, RS, BS>;
  const int smem = RS * 16384 + BS * 2 * NP * 128 + 1024;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  count_launches(1);
  kern<<<dim3((unsigned)nb, (unsigned)ns), kRowsThreads, smem, s>>>(tmX, tmW, I, J, l, rb, cper, part,
                                                                   st);
  return cudaGetLastError();
}

}  // namespace

bool tc_mode1_supported(int64_t I, int l) { return l <= 64 && I % 4 == 0 && I <= 4096; }

int tc_np(int l) { return l <= 32 ? 32 : 64; }

int64_t tc_ipad(int64_t I) { return (I + 31) / 32 * 32; }

// Split of J for the row sweep: about two CTAs per SM, chunks of 32 columns.
void tc_rows_split(int64_t I, int64_t J, int nsm, int* nsplit, int64_t* jchunk) {
  const int64_t mgroups = (I + 127) / 128;
  int64_t want = (2LL * nsm + mgroups - 1) / mgroups;
  int64_t chunk = (J + want - 1) / want;
  chunk = (chunk + 31) / 32 * 32;
  if (chunk < 64) chunk = 64;
  *jchunk = chunk;
  *nsplit = (int)((J + chunk - 1) / chunk);
}

int tc_cols_grid(int64_t J, int nsm) {
  const int64_t njb = (J + 127) / 128;
  const int64_t cap = 2LL * nsm;
  return (int)(njb < cap ? njb : cap);
}
cudaError_t launch_tc_rows(const float* X, int64_t I, int64_t J, int l, uint64_t seed, uint32_t sid,
                           const float* WT, int nsplit, int64_t jchunk, float* part,
                           double* normpart, DevState* st, cudaStream_t s) {
  const bool norm = normpart != nullptr;
  if (tc_np(l) == 32) {
    if (WT) return rows_launch<32, 1, false>(X, I, J, l, 0, 0, WT, nsplit, jchunk, part, nullptr, st, s);
    if (norm) return rows_launch<32, 0, true>(X, I, J, l, seed, sid, nullptr, nsplit, jchunk, part, normpart, st, s);
    return rows_launch<32, 0, false>(X, I, J, l, seed, sid, nullptr, nsplit, jchunk, part, nullptr, st, s);
  }
  if (WT) return rows_launch<64, 1, false>(X, I, J, l, 0, 0, WT, nsplit, jchunk, part, nullptr, st, s);
  if (norm) return rows_launch<64, 0, true>(X, I, J, l, seed, sid, nullptr, nsplit, jchunk, part, normpart, st, s);
  return rows_launch<64, 0, false>(X, I, J, l, seed, sid, nullptr, nsplit, jchunk, part, nullptr, st, s);
}

// True when the TMA-fed sweeps can read X: the tensor-map encoder is there
// and X starts on a 16-byte boundary (I % 4 == 0 is tc_mode1_supported's).
bool tc_tma_ok(const float* X) { return encode_tiled() != nullptr && ((uintptr_t)X & 15) == 0; }

// Row blocks and j-splits of the TMA-fed row sweep: nb blocks of rb rows (a
// multiple of 4, as equal as possible), about one CTA per SM.
void tc_rows_tma_shape(int64_t I, int64_t J, int nsm, int* nb, int* rb, int* ns, int64_t* cper) {
  const int64_t b = (I + 127) / 128;
  int64_t r = (I + b - 1) / b;
  r = (r + 3) / 4 * 4;
  const int64_t nchunk = (J + 31) / 32;
  int64_t n = nsm / b;
  if (n < 1) n = 1;
  if (n > nchunk) n = nchunk;
  *nb = (int)b;
  *rb = (int)r;
  *cper = (nchunk + n - 1) / n;
  *ns = (int)((nchunk + *cper - 1) / *cper);
}

// TMA-fed row sweep of the power iteration (tc_tma_ok(X) must hold): P = X_(1) W
// with Wsplit the column sweep's [W_hi; W_lo] (2 l x J).  *nsplit receives the
// number of j-split partials per row written to part.
cudaError_t launch_tc_rows_tma(const float* X, int64_t I, int64_t J, int l, const float* Wsplit,
                               float* part, DevState* st, int nsm, cudaStream_t s, int* nsplit) {
  int nb = 0, rb = 0, ns = 0;
  int64_t cper = 0;
  tc_rows_tma_shape(I, J, nsm, &nb, &rb, &ns, &cper);
  *nsplit = ns;
  const int NP = tc_np(l);
  CUtensorMap tmX, tmW;
  {
    const cuuint64_t dims[2] = {(cuuint64_t)I, (cuuint64_t)J};
    const cuuint64_t strides[1] = {(cuuint64_t)I * 4};
    const cuuint32_t box[2] = {(cuuint32_t)rb, 32};
    if (!tmap_f32(&tmX, X, 2, dims, strides, box, false)) return cudaErrorInvalidValue;
  }
  {
    const cuuint64_t dims[3] = {(cuuint64_t)J, (cuuint64_t)l, 2};
    const cuuint64_t strides[2] = {(cuuint64_t)J * 4, (cuuint64_t)l * J * 4};
    const cuuint32_t box[3] = {32, (cuuint32_t)NP, 2};
    if (!tmap_f32(&tmW, Wsplit, 3, dims, strides, box, true)) return cudaErrorInvalidValue;
  }
  // X stages and B stages: about 128 KB of X in flight
  if (NP == 32) return rows_tma_launch<32, 8, 8>(tmX, tmW, I, J, l, rb, nb, ns, cper, part, st, s);
  return rows_tma_launch<64, 6, 6>(tmX, tmW, I, J, l, rb, nb, ns, cper, part, st, s);
}

// Column sweep; tma selects the TMA-fed kernel (tc_tma_ok(X) must hold), and
// wsplit (with !ttm) its [W_hi; W_lo] output for the TMA-fed row sweep.
cudaError_t launch_tc_cols(const float* X, int64_t I, int64_t J, int l, const float* QT, float* out,
                           bool ttm, DevState* st, int grid, cudaStream_t s, bool tma, bool wsplit) {
  const int64_t Ipad = tc_ipad(I);
  if (tma) {
    // the TMA-fed form: one CTA per SM, persistent over the 128-column blocks
    const int NP = tc_np(l);
    CUtensorMap tmX, tmQ;
    if (tmap_2d_f32(&tmX, X, (uint64_t)I, (uint64_t)J, 128) &&
        tmap_2d_f32(&tmQ, QT, (uint64_t)Ipad, (uint64_t)(2 * NP), (uint32_t)(2 * NP))) {
      int nsm = 0, dev = 0;
      if (cudaGetDevice(&dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return cudaGetLastError();
      const int64_t njb = (J + 127) / 128;
      const int g = (int)(njb < nsm ? njb : nsm);
      const int nkc = (int)(Ipad / 32);
      // raw stages: as many as fit beside the split stages (and the product's rows)
      // X stages and B stages: as many as fit (about 128 KB of X in flight)
      if (NP == 32) {
        if (ttm) return cols_tma_launch<32, 8, 8, true>(tmX, tmQ, J, l, nkc, out, st, g, s);
        if (wsplit) return cols_tma_launch<32, 8, 8, false, true>(tmX, tmQ, J, l, nkc, out, st, g, s);
        return cols_tma_launch<32, 8, 8, false>(tmX, tmQ, J, l, nkc, out, st, g, s);
      }
      if (ttm) return cols_tma_launch<64, 6, 6, true>(tmX, tmQ, J, l, nkc, out, st, g, s);
      if (wsplit) return cols_tma_launch<64, 6, 6, false, true>(tmX, tmQ, J, l, nkc, out, st, g, s);
      return cols_tma_launch<64, 6, 6, false>(tmX, tmQ, J, l, nkc, out, st, g, s);
    }
    return cudaErrorInvalidValue;
  }
  if (tc_np(l) == 32) {
    if (ttm) return cols_launch<32, true>(X, I, J, l, Ipad, QT, out, st, grid, s);
    return cols_launch<32, false>(X, I, J, l, Ipad, QT, out, st, grid, s);
  }
  if (ttm) return cols_launch<64, true>(X, I, J, l, Ipad, QT, out, st, grid, s);
  return cols_launch<64, false>(X, I, J, l, Ipad, QT, out, st, grid, s);
}

cudaError_t launch_q_to_qt32(const double* Q, int64_t I, int l, float* QT, cudaStream_t s) {
  const int NP = tc_np(l);
  const int64_t Ipad = tc_ipad(I);
  const int64_t n = (int64_t)NP * Ipad;
  count_launches(1);
  k_q_to_qt32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Q, I, l, NP, Ipad, QT, QT + n);
  return cudaGetLastError();
}

cudaError_t launch_reduce_f32(const float* part, int64_t nsplit, int64_t n, double* out,
                              cudaStream_t s) {
  count_launches(1);
  k_reduce_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(part, nsplit, n, out);
  return cudaGetLastError();
}

}  // namespace rcp

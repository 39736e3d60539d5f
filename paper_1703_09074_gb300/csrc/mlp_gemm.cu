// Dense layers of the warm-start network on the tcgen05 tensor cores.
//
// Every product of the network's forward and backward passes is written as
//   C[M x N] = A[M x K] * B[N x K]^T        (both operands K-contiguous, BF16)
// with FP32 accumulation in tensor memory.  The weight-gradient products use
// the transposed activations, which the epilogue kernels write next to the
// row-major ones, so one kernel shape serves all of them.
//
// Tile: 128 x 128 outputs per CTA, K consumed in steps of 64 (one 128-byte
// swizzled row per operand row), four shared-memory stages filled with
// 16-byte cp.async copies, MMAs issued by one thread (four K = 16
// instructions per stage) and tracked with one mbarrier per stage.  Long K
// (the 13824-wide input layer) is split over gridDim.z; each split writes its
// own FP32 partial slice, which the epilogue kernels sum in a fixed order.
// Every wait is bounded: a stalled pipeline sets the error word and the CTA
// leaves after freeing its tensor memory.
#include <cuda_bf16.h>

#include "rcp_internal.cuh"
#include "tc_ptx.cuh"

namespace rcp {

namespace {

constexpr int kGT = 128;            // threads per CTA
constexpr int kBM = 128, kBN = 128, kBK = 64;
constexpr int kStages = 4;
constexpr int kStageBytes = kBM * kBK * 2;   // one operand tile
constexpr long long kWaitBudget = 2000000000LL;  // clock cycles (about a second)

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__global__ void __launch_bounds__(kGT, 1)
k_gemm_bf16_tn(const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ B,
               float* __restrict__ C, int M, int N, int K, int kchunk, int* err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = smem;
  unsigned char* sB = smem + kStages * kStageBytes;
  __shared__ uint64_t bar[kStages];
  __shared__ uint32_t tbase;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
  const int kb = blockIdx.z * kchunk;
  const int nk = kchunk / kBK;

  if (warp == 0) tc::tmem_alloc(&tbase, 128);
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) tc::mbar_init(&bar[s], 1);
    tc::fence_mbar_init();
  }
  tc::tc_fence_before_sync();
  __syncthreads();
  tc::tc_fence_after_sync();
  const uint32_t tmem = tbase;

  // stage s <- K columns [kk, kk + 64) of rows m0.. of A and n0.. of B
  auto load_stage = [&](int kt, int s) {
    const int64_t kk = kb + (int64_t)kt * kBK;
#pragma unroll
    for (int c0 = 0; c0 < kBM * 8; c0 += kGT) {
      const int c = c0 + tid;
      const int row = c >> 3, ch = c & 7;
      const uint32_t off = row * 128u + ((((uint32_t)ch ^ (uint32_t)(row & 7)) & 7u) << 4);
      cp_async16(tc::smem_u32(sA + s * kStageBytes + off), A + (int64_t)(m0 + row) * K + kk + ch * 8);
      cp_async16(tc::smem_u32(sB + s * kStageBytes + off), B + (int64_t)(n0 + row) * K + kk + ch * 8);
    }
  };

#pragma unroll
  for (int s = 0; s < kStages - 1; ++s) {
    if (s < nk) load_stage(s, s);
    cp_async_commit();
  }
  constexpr uint32_t idesc = tc::idesc_bf16(kBM, kBN);
  bool ok = true;
  for (int kt = 0; kt < nk; ++kt) {
    const int s = kt % kStages;
    cp_async_wait<kStages - 2>();       // this thread's copies of stage kt have landed
    tc::fence_proxy_async_smem();       // ... and are visible to the tensor cores
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
    if (tid == 0) {
      tc::tc_fence_after_sync();
      const uint32_t a0 = tc::smem_u32(sA + s * kStageBytes);
      const uint32_t b0 = tc::smem_u32(sB + s * kStageBytes);
#pragma unroll
      for (int j = 0; j < kBK / 16; ++j)  // K = 16 per instruction: 32 bytes along the row
        tc::mma_bf16(tmem, tc::desc_kmajor_sw128(a0 + 32u * j), tc::desc_kmajor_sw128(b0 + 32u * j), idesc,
                     (kt | j) != 0 ? 1u : 0u);
      tc::mma_commit(&bar[s]);
    }
    // refill the stage read by the MMAs of step kt - 1 with K step kt + kStages - 1
    const int kn = kt + kStages - 1;
    if (kn < nk) {
      const int sp = kn % kStages;
      bool w = true;
      if (kt >= 1) w = tc::mbar_wait(&bar[sp], (uint32_t)(((kt - 1) / kStages) & 1), kWaitBudget);
      if (w) load_stage(kn, sp);
      ok = ok && w;
    }
    cp_async_commit();
  }
  // the last commit covers every MMA of this CTA
  bool fin = ok && tc::mbar_wait(&bar[(nk - 1) % kStages], (uint32_t)(((nk - 1) / kStages) & 1),
                                 kWaitBudget);
  fin = __syncthreads_and(fin);
  tc::tc_fence_after_sync();
  if (fin) {
    // warp w owns TMEM lanes (rows) 32 w .. 32 w + 31; thread <-> row
    const int row = m0 + warp * 32 + lane;
    float* crow = C + (int64_t)blockIdx.z * M * N + (int64_t)row * N + n0;
#pragma unroll 1
    for (int c = 0; c < kBN; c += 32) {
      float v[32];
      tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
#pragma unroll
      for (int k = 0; k < 32; k += 4)
        *(float4*)(crow + c + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
    }
  } else if (tid == 0) {
    atomicExch(err, (int)RCP_ETIMEOUT);
    // give in-flight MMAs a bounded chance to drain before the memory is freed
    if (nk > 0) tc::mbar_wait(&bar[(nk - 1) % kStages], (uint32_t)(((nk - 1) / kStages) & 1), kWaitBudget);
  }
  tc::tc_fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

}  // namespace

size_t gemm_bf16_smem() { return (size_t)2 * kStages * kStageBytes + 1024; }

cudaError_t prepare_gemm_bf16() {
  return cudaFuncSetAttribute(k_gemm_bf16_tn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)gemm_bf16_smem());
}

// C[z] = A[:, z-th K slice] * B[:, z-th K slice]^T for z < splits.  Requires
// M % 128 == 0, N % 128 == 0, K % (64 * splits) == 0 (checked by the caller).
cudaError_t launch_gemm_bf16(const void* A, const void* B, float* C, int M, int N, int K,
                             int splits, int* err, cudaStream_t s) {
  const dim3 grid(N / kBN, M / kBM, splits);
  count_launches(1);
  k_gemm_bf16_tn<<<grid, kGT, gemm_bf16_smem(), s>>>((const __nv_bfloat16*)A,
                                                     (const __nv_bfloat16*)B, C, M, N, K,
                                                     K / splits, err);
  return cudaGetLastError();
}

}  // namespace rcp

// Elementwise evaluation of the device arithmetic building blocks that the
// Gram solves, the column norms and the CholeskyQR factorisations rest on
// (double-word sum, product, reciprocal and square root; the FP64 reciprocal
// square root), exposed so that their error bounds can be checked against
// exact arithmetic on the host.
#include "dw_arith.cuh"
#include "rcp_internal.cuh"
#include "small_la.cuh"

namespace rcp {
namespace {

__global__ void k_arith(int op, const double* __restrict__ x, const double* __restrict__ y,
                        int64_t n, double* __restrict__ out_hi, double* __restrict__ out_lo) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  if (op == RCP_ARITH_RSQRT64) {
    out_hi[k] = rsqrt64(x[k]);
    out_lo[k] = 0.0;
    return;
  }
  const dwf a = dw_from_double(x[k]);
  dwf r;
  if (op == RCP_ARITH_DW_ADD) r = dw_add(a, dw_from_double(y[k]));
  else if (op == RCP_ARITH_DW_MUL) r = dw_mul(a, dw_from_double(y[k]));
  else if (op == RCP_ARITH_DW_RCP) r = dw_rcp(a);
  else r = dw_sqrt(a);
  out_hi[k] = (double)r.hi;
  out_lo[k] = (double)r.lo;
}

// kFmaChains independent FMA chains per thread, iters steps each; the sum is
// stored only in a case that cannot occur, so the chains stay live.
constexpr int kFmaChains = 8;
__device__ double g_fma_sink;
template <typename T>
__global__ void k_fma_chains(int iters, T seed) {
  T v[kFmaChains];
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) v[k] = seed + (T)(threadIdx.x + k) * (T)1e-6;
  const T m = (T)0.9999999, c = (T)1e-7;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) v[k] = fma(v[k], m, c);
  T s = 0;
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) s += v[k];
  if (s == (T)-12345.0) g_fma_sink = (double)s;
}

}  // namespace
}  // namespace rcp

extern "C" rcp_status rcp_measure_fma_rate(int32_t fp64, double* tflops, void* cuda_stream) {
  if (!tflops || (fp64 != 0 && fp64 != 1)) return RCP_EINVAL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return RCP_ECUDA;
  // 8 (FP64) or 16 (FP32) CTAs of 256 threads per SM; about 1 ms per launch
  const int threads = 256, blocks = nsm * (fp64 ? 8 : 16);
  const int iters = fp64 ? 1024 : 65536;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return RCP_ECUDA;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return RCP_ECUDA;
  }
  float ms = 0.0f;
  bool ok = true;
  for (int rep = 0; rep < 2 && ok; ++rep) {  // the first launch warms up; the second is timed
    ok = cudaEventRecord(a, s) == cudaSuccess;
    rcp::count_launches(1);
    if (fp64) rcp::k_fma_chains<double><<<blocks, threads, 0, s>>>(iters, 1.0);
    else rcp::k_fma_chains<float><<<blocks, threads, 0, s>>>(iters, 1.0f);
    ok = ok && cudaGetLastError() == cudaSuccess && cudaEventRecord(b, s) == cudaSuccess &&
         cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (!ok || ms <= 0.0f) return RCP_ECUDA;
  const double flops = 2.0 * rcp::kFmaChains * (double)iters * threads * (double)blocks;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return RCP_OK;
}

extern "C" rcp_status rcp_test_arith(int32_t op, const double* x_dev, const double* y_dev,
                                     int64_t n, double* out_hi_dev, double* out_lo_dev,
                                     void* cuda_stream) {
  if (op < RCP_ARITH_DW_ADD || op > RCP_ARITH_RSQRT64 || n < 0) return RCP_EINVAL;
  if (n == 0) return RCP_OK;
  const bool binary = op == RCP_ARITH_DW_ADD || op == RCP_ARITH_DW_MUL;
  if (!x_dev || !out_hi_dev || !out_lo_dev || (binary && !y_dev)) return RCP_EINVAL;
  const int threads = 256;
  const int64_t blocks = (n + threads - 1) / threads;
  if (blocks > 0x7fffffffLL) return RCP_EINVAL;
  rcp::count_launches(1);
  rcp::k_arith<<<(unsigned)blocks, threads, 0, (cudaStream_t)cuda_stream>>>(
      op, x_dev, y_dev, n, out_hi_dev, out_lo_dev);
  return cudaGetLastError() == cudaSuccess ? RCP_OK : RCP_ECUDA;
}

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

}  // namespace
}  // namespace rcp

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

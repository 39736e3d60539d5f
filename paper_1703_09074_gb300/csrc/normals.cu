// The counter-based Gaussian stream of the test matrices (Section 3.1), exposed
// for checking against an independent implementation of the same definition.
#include "rcp_internal.cuh"

namespace rcp {
namespace {

__global__ void k_normals(uint64_t seed, uint32_t stream, uint32_t purpose, int64_t first,
                          int64_t count, double* out, uint32_t* words, float* f32_out) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  const int64_t e = first + k;
  if (out) {
    const double2 z = normal_pair_f64(seed, stream, purpose, (uint64_t)(e >> 1));
    out[k] = (e & 1) ? z.y : z.x;
  }
  if (words) {
    const uint4 w = philox_words(seed, stream, purpose, (uint64_t)(e >> 1));
    words[4 * k + 0] = w.x;
    words[4 * k + 1] = w.y;
    words[4 * k + 2] = w.z;
    words[4 * k + 3] = w.w;
  }
  if (f32_out) {
    const float4 z = normal_quad_f32(seed, stream, purpose, (uint64_t)(e >> 2));
    const int slot = (int)(e & 3);
    f32_out[k] = slot == 0 ? z.x : slot == 1 ? z.y : slot == 2 ? z.z : z.w;
  }
}

}  // namespace
}  // namespace rcp

extern "C" rcp_status rcp_test_normals(uint64_t seed, uint32_t stream, uint32_t purpose,
                                       int64_t first, int64_t count, double* out_dev,
                                       uint32_t* words_dev, float* f32_out_dev, void* cuda_stream) {
  if (count < 0 || first < 0) return RCP_EINVAL;
  if (count == 0) return RCP_OK;
  const int threads = 256;
  const int64_t blocks = (count + threads - 1) / threads;
  if (blocks > 0x7fffffffLL) return RCP_EINVAL;
  rcp::count_launches(1);
  rcp::k_normals<<<(unsigned)blocks, threads, 0, (cudaStream_t)cuda_stream>>>(
      seed, stream, purpose, first, count, out_dev, words_dev, f32_out_dev);
  return cudaGetLastError() == cudaSuccess ? RCP_OK : RCP_ECUDA;
}

// Synthetic CP tensors generated on the device (training data for the warm
// start and benchmark inputs): X = sum_r lambda_r a_1r o ... o a_Nr + sigma z.
#include <math.h>

#include "rcp_internal.cuh"

namespace rcp {
namespace {

constexpr uint32_t kPurposeSynth = 3;

struct SynthArgs {
  int N, R;
  int64_t dims[kMaxN];
  const float* A[kMaxN];
  const float* lam;
  float sigma;
  uint64_t seed;
  int64_t total;
};

__global__ void __launch_bounds__(256) k_synth_cp(SynthArgs a, float* __restrict__ X) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < a.total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t idx[kMaxN];
    int64_t q = e;
    for (int n = 0; n < a.N; ++n) {
      const int64_t d = a.dims[n];
      const int64_t t = q / d;
      idx[n] = q - t * d;
      q = t;
    }
    float s = 0.0f;
    for (int r = 0; r < a.R; ++r) {
      float p = a.lam[r];
      for (int n = 0; n < a.N; ++n) p *= a.A[n][idx[n] + a.dims[n] * r];
      s += p;
    }
    if (a.sigma != 0.0f) {
      // Box-Muller on two 24-bit uniforms: u1 in (0, 1], u2 in [0, 1)
      const uint4 w = philox4x32_10(make_uint4((uint32_t)e, (uint32_t)(e >> 32), 0u, kPurposeSynth),
                                    make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32)));
      const float s24 = 5.9604644775390625e-08f;
      const float rr = sqrtf(-2.0f * logf((float)((w.x >> 8) + 1u) * s24));
      float sn, cs;
      sincospif(2.0f * (float)(w.y >> 8) * s24, &sn, &cs);
      s += a.sigma * rr * cs;
    }
    X[e] = s;
  }
}

}  // namespace
}  // namespace rcp

using namespace rcp;

extern "C" rcp_status rcp_synth_cp(int32_t ndim, const int64_t* dims, int32_t rank,
                                   const float* const* factors, const float* lambda_dev,
                                   float sigma, uint64_t seed, float* X_dev, void* stream) {
  if (ndim < 1 || ndim > kMaxN || !dims || rank < 1 || !factors || !lambda_dev || !X_dev ||
      !(sigma >= 0.0f))
    return RCP_EINVAL;
  SynthArgs a{};
  a.N = ndim;
  a.R = rank;
  a.total = 1;
  for (int n = 0; n < ndim; ++n) {
    if (dims[n] < 1 || !factors[n]) return RCP_EINVAL;
    a.dims[n] = dims[n];
    a.A[n] = factors[n];
    a.total *= dims[n];
  }
  a.lam = lambda_dev;
  a.sigma = sigma;
  a.seed = seed;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return RCP_ECUDA;
  const int64_t blocks = (a.total + 255) / 256;
  const int grid = (int)(blocks < 16LL * nsm ? blocks : 16LL * nsm);
  count_launches(1);
  k_synth_cp<<<grid, 256, 0, (cudaStream_t)stream>>>(a, X_dev);
  return cudaGetLastError() == cudaSuccess ? RCP_OK : RCP_ECUDA;
}

// The warm-start network: a 3-layer perceptron
//   x (24^3) -> relu(W1 x + b1) (512) -> relu(W2 h1 + b2) (512) -> W3 h2 + b3 (3 x 24 x 16)
// with BF16 weights (FP32 master copy), BF16 activations as GEMM operands and
// FP32 accumulation; forward, backward and Adam run in this file's kernels and
// in the tcgen05 GEMM of mlp_gemm.cu.  The network is an addition to the
// method (the paper starts ALS from eigenvectors or random factors, Section
// 3.2); what it computes is fixed by the forward/backward definitions below,
// which the FP64 CPU reference restates.
#include <cuda_bf16.h>

#include <cstring>
#include <new>
#include <vector>

#include "mlp_internal.cuh"

namespace rcp {

cudaError_t prepare_gemm_bf16();
cudaError_t launch_gemm_bf16(const void* A, const void* B, float* C, int M, int N, int K,
                             int splits, int* err, cudaStream_t s);

namespace {

// ---------------------------------------------------------------- epilogue
// out[m][n] = act(sum_s P[s][m][n] + bias[n]) for m < M, n < N, where act is
// identity, relu, or multiplication by [mask[m][n] > 0] (the relu derivative
// taken from the post-activation values).  Optional outputs: BF16 row-major,
// BF16 transposed (N x M), FP32 row-major, and column sums (the bias
// gradient), each summed in a fixed order.  One CTA per 32 columns.
__global__ void __launch_bounds__(256) k_epi(const float* __restrict__ P, int S, int M, int N,
                                             const float* __restrict__ bias,
                                             const __nv_bfloat16* __restrict__ mask, int relu,
                                             __nv_bfloat16* __restrict__ out,
                                             __nv_bfloat16* __restrict__ outT,
                                             float* __restrict__ outf, float* __restrict__ colsum) {
  __shared__ float tile[32][33];
  __shared__ float cs[8][32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int n = blockIdx.x * 32 + tx;
  const int64_t MN = (int64_t)M * N;
  float csum = 0.0f;
  for (int m0 = 0; m0 < M; m0 += 32) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int m = m0 + ty + 8 * k;
      float v = 0.0f;
      if (m < M && n < N) {
        const int64_t o = (int64_t)m * N + n;
        for (int s = 0; s < S; ++s) v += P[s * MN + o];
        if (bias) v += bias[n];
        if (relu) v = fmaxf(v, 0.0f);
        if (mask && !(__bfloat162float(mask[o]) > 0.0f)) v = 0.0f;
        if (out) out[o] = __float2bfloat16_rn(v);
        if (outf) outf[o] = v;
        csum += v;
      }
      tile[ty + 8 * k][tx] = v;
    }
    __syncthreads();
    if (outT) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int nn = blockIdx.x * 32 + ty + 8 * k;
        const int m = m0 + tx;
        if (nn < N && m < M) outT[(int64_t)nn * M + m] = __float2bfloat16_rn(tile[tx][ty + 8 * k]);
      }
    }
    __syncthreads();
  }
  if (colsum) {
    cs[ty][tx] = csum;
    __syncthreads();
    if (ty == 0 && n < N) {
      float s = 0.0f;
      for (int k = 0; k < 8; ++k) s += cs[k][tx];
      colsum[n] = s;
    }
  }
}

// dst[c][r] = src[r][c] for a rows x cols BF16 matrix.
__global__ void __launch_bounds__(256) k_transpose_bf16(const __nv_bfloat16* __restrict__ src,
                                                        __nv_bfloat16* __restrict__ dst, int rows,
                                                        int cols) {
  __shared__ __nv_bfloat16 t[32][34];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int r = r0 + ty + 8 * k, c = c0 + tx;
    if (r < rows && c < cols) t[ty + 8 * k][tx] = src[(int64_t)r * cols + c];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int c = c0 + ty + 8 * k, r = r0 + tx;
    if (r < rows && c < cols) dst[(int64_t)c * rows + r] = t[tx][ty + 8 * k];
  }
}

// Adam (Kingma & Ba 2015) on the FP32 master copy, then the BF16 working copy:
//   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
//   w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, __nv_bfloat16* __restrict__ wb, int64_t n,
                       float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    wb[i] = __float2bfloat16_rn(wi);
  }
}

// FP32 -> BF16 copy of the master parameters (after loading or initialising).
__global__ void k_to_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    wb[i] = __float2bfloat16_rn(w[i]);
}

// Input rows (FP32, count x 24^3) to BF16 rows (batch x 24^3, rows >= count
// zero) and, for training, the transposed BF16 copy used by the W1 gradient.
__global__ void __launch_bounds__(256) k_pack_rows(const float* __restrict__ X32, int count,
                                                   int batch, __nv_bfloat16* __restrict__ Xb,
                                                   __nv_bfloat16* __restrict__ XTb) {
  __shared__ float tile[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int r = r0 + ty + 8 * k, c = c0 + tx;
    float v = 0.0f;
    if (r < count) v = X32[(int64_t)r * kMlpIn + c];
    if (r < batch) Xb[(int64_t)r * kMlpIn + c] = __float2bfloat16_rn(v);
    tile[ty + 8 * k][tx] = v;
  }
  __syncthreads();
  if (XTb) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int c = c0 + ty + 8 * k, r = r0 + tx;
      if (r < batch) XTb[(int64_t)c * batch + r] = __float2bfloat16_rn(tile[tx][ty + 8 * k]);
    }
  }
}

inline int grid1(int64_t n, int nsm) {
  const int64_t b = (n + 255) / 256;
  return (int)(b < 8LL * nsm ? b : 8LL * nsm);
}

}  // namespace

// ---------------------------------------------------------------- host side
void mlp_param_offsets(int64_t off[7]) {
  off[0] = 0;                                             // W1: Hidden x In
  off[1] = off[0] + (int64_t)kMlpHidden * kMlpIn;         // b1
  off[2] = off[1] + kMlpHidden;                           // W2: Hidden x Hidden
  off[3] = off[2] + (int64_t)kMlpHidden * kMlpHidden;     // b2
  off[4] = off[3] + kMlpHidden;                           // W3: Out x Hidden
  off[5] = off[4] + (int64_t)kMlpOut * kMlpHidden;        // b3
  off[6] = off[5] + kMlpOut;                              // total
}

#define MLP_TRY(x)                                                   \
  do {                                                               \
    cudaError_t e_ = (x);                                            \
    if (e_ != cudaSuccess) {                                         \
      cudaGetLastError();                                            \
      return e_ == cudaErrorMemoryAllocation ? RCP_ENOMEM : RCP_ECUDA; \
    }                                                                \
  } while (0)

rcp_status mlp_forward_enqueue(rcp_mlp_s* p, const float* x, int count, bool train, cudaStream_t s) {
  const int Bt = p->batch;
  int64_t off[7];
  mlp_param_offsets(off);
  int* err = &p->dst->status;
  count_launches(1);
  k_pack_rows<<<dim3(kMlpIn / 32, Bt / 32), 256, 0, s>>>(x, count, Bt, p->Xb, train ? p->XTb : nullptr);
  MLP_TRY(cudaGetLastError());
  MLP_TRY(launch_gemm_bf16(p->Xb, p->Wb + off[0], p->P, Bt, kMlpHidden, kMlpIn, kMlpSplit1, err, s));
  count_launches(1);
  k_epi<<<kMlpHidden / 32, 256, 0, s>>>(p->P, kMlpSplit1, Bt, kMlpHidden, p->w + off[1], nullptr, 1,
                                        p->H1b, train ? p->H1Tb : nullptr, nullptr, nullptr);
  MLP_TRY(cudaGetLastError());
  MLP_TRY(launch_gemm_bf16(p->H1b, p->Wb + off[2], p->P, Bt, kMlpHidden, kMlpHidden, 1, err, s));
  count_launches(1);
  k_epi<<<kMlpHidden / 32, 256, 0, s>>>(p->P, 1, Bt, kMlpHidden, p->w + off[3], nullptr, 1, p->H2b,
                                        train ? p->H2Tb : nullptr, nullptr, nullptr);
  MLP_TRY(cudaGetLastError());
  MLP_TRY(launch_gemm_bf16(p->H2b, p->Wb + off[4], p->P, Bt, kMlpOut, kMlpHidden, 1, err, s));
  count_launches(1);
  k_epi<<<kMlpOut / 32, 256, 0, s>>>(p->P, 1, Bt, kMlpOut, p->w + off[5], nullptr, 0, nullptr,
                                     nullptr, p->Y, nullptr);
  MLP_TRY(cudaGetLastError());
  if (train) p->has_grad = true;
  return RCP_OK;
}

// Backward from dY (FP32, batch x Out) to every parameter gradient (p->g, flat).
rcp_status mlp_backward_enqueue(rcp_mlp_s* p, const float* dY, cudaStream_t s) {
  const int Bt = p->batch;
  int64_t off[7];
  mlp_param_offsets(off);
  int* err = &p->dst->status;
  count_launches(1);  // dY -> BF16 copies and the b3 gradient
  k_epi<<<kMlpOut / 32, 256, 0, s>>>(dY, 1, Bt, kMlpOut, nullptr, nullptr, 0, p->dYb, p->dYTb,
                                     nullptr, p->g + off[5]);
  MLP_TRY(cudaGetLastError());
  // dW3 = dY^T H2
  MLP_TRY(launch_gemm_bf16(p->dYTb, p->H2Tb, p->g + off[4], kMlpOut, kMlpHidden, Bt, 1, err, s));
  // dH2 = dY W3, masked by relu'(Z2)
  MLP_TRY(launch_gemm_bf16(p->dYb, p->WTb3, p->P, Bt, kMlpHidden, kMlpOut, 1, err, s));
  count_launches(1);
  k_epi<<<kMlpHidden / 32, 256, 0, s>>>(p->P, 1, Bt, kMlpHidden, nullptr, p->H2b, 0, p->dZ2b,
                                        p->dZ2Tb, nullptr, p->g + off[3]);
  MLP_TRY(cudaGetLastError());
  // dW2 = dZ2^T H1
  MLP_TRY(launch_gemm_bf16(p->dZ2Tb, p->H1Tb, p->g + off[2], kMlpHidden, kMlpHidden, Bt, 1, err, s));
  // dH1 = dZ2 W2, masked by relu'(Z1)
  MLP_TRY(launch_gemm_bf16(p->dZ2b, p->WTb2, p->P, Bt, kMlpHidden, kMlpHidden, 1, err, s));
  count_launches(1);
  k_epi<<<kMlpHidden / 32, 256, 0, s>>>(p->P, 1, Bt, kMlpHidden, nullptr, p->H1b, 0, nullptr,
                                        p->dZ1Tb, nullptr, p->g + off[1]);
  MLP_TRY(cudaGetLastError());
  // dW1 = dZ1^T X
  MLP_TRY(launch_gemm_bf16(p->dZ1Tb, p->XTb, p->g + off[0], kMlpHidden, kMlpIn, Bt, 1, err, s));
  return RCP_OK;
}

rcp_status mlp_transposes(rcp_mlp_s* p, cudaStream_t s) {
  int64_t off[7];
  mlp_param_offsets(off);
  count_launches(2);
  k_transpose_bf16<<<dim3(kMlpHidden / 32, kMlpHidden / 32), 256, 0, s>>>(p->Wb + off[2], p->WTb2,
                                                                          kMlpHidden, kMlpHidden);
  MLP_TRY(cudaGetLastError());
  k_transpose_bf16<<<dim3(kMlpHidden / 32, kMlpOut / 32), 256, 0, s>>>(p->Wb + off[4], p->WTb3,
                                                                       kMlpOut, kMlpHidden);
  MLP_TRY(cudaGetLastError());
  return RCP_OK;
}

rcp_status mlp_refresh_bf16(rcp_mlp_s* p, cudaStream_t s) {
  int64_t off[7];
  mlp_param_offsets(off);
  count_launches(1);
  k_to_bf16<<<grid1(off[6], p->nsm), 256, 0, s>>>(p->w, p->Wb, off[6]);
  MLP_TRY(cudaGetLastError());
  return mlp_transposes(p, s);
}

rcp_status mlp_adam_enqueue(rcp_mlp_s* p, float lr, float b1, float b2, float eps, cudaStream_t s) {
  int64_t off[7];
  mlp_param_offsets(off);
  p->t += 1;
  const double c1 = 1.0 - pow((double)b1, (double)p->t), c2 = 1.0 - pow((double)b2, (double)p->t);
  count_launches(1);
  k_adam<<<grid1(off[6], p->nsm), 256, 0, s>>>(p->w, p->m, p->v, p->g, p->Wb, off[6], lr, b1, b2,
                                               eps, (float)c1, (float)c2);
  MLP_TRY(cudaGetLastError());
  return mlp_transposes(p, s);
}

namespace {

// Seeded initial parameters: W1, W2 ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from
// the counter-based stream (purpose 2, counter = parameter index); W3 and the
// biases zero, so that the untrained network outputs Y = 0 (the eigenvector
// initialisation) and training starts from it.
__global__ void k_mlp_init(float* __restrict__ w, uint64_t seed, int64_t n, int64_t o1, int64_t o2,
                           int64_t o3, int64_t o4, int64_t o5) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float v = 0.0f;
    float fan = 0.0f;
    if (i < o1) fan = (float)kMlpIn;
    else if (i >= o2 && i < o3) fan = (float)kMlpHidden;
    (void)o4;
    (void)o5;
    if (fan > 0.0f) {
      const uint4 r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), 0u, 2u),
                                    make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
      const float u = ((float)(r.x >> 8) + 0.5f) * (1.0f / 16777216.0f);  // (0, 1)
      v = (2.0f * u - 1.0f) * rsqrtf(fan);
    }
    w[i] = v;
  }
}

}  // namespace
}  // namespace rcp

using namespace rcp;

namespace {

void free_mlp(rcp_mlp_t p) {
  if (!p) return;
  void* bufs[] = {p->w, p->m, p->v, p->g, p->Wb, p->WTb2, p->WTb3, p->x32, p->Xb, p->XTb,
                  p->H1b, p->H1Tb, p->H2b, p->H2Tb, p->dYb, p->dYTb, p->dZ2b, p->dZ2Tb,
                  p->dZ1Tb, p->P, p->Y, p->dY, p->loss, p->U, p->meta, p->dst};
  for (void* b : bufs) cudaFree(b);
  delete p;
}

}  // namespace

extern "C" {

int64_t rcp_mlp_param_count(void) {
  int64_t off[7];
  mlp_param_offsets(off);
  return off[6];
}

rcp_status rcp_mlp_create(int32_t batch, uint64_t seed, void* stream, rcp_mlp_t* out) {
  if (!out || batch < 128 || batch % 128 != 0 || batch > 65536) return RCP_EINVAL;
  rcp_mlp_t p = new (std::nothrow) rcp_mlp_s();
  if (!p) return RCP_ENOMEM;
  memset((void*)p, 0, sizeof(*p));
  p->stream = (cudaStream_t)stream;
  p->batch = batch;
  p->seed = seed;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      prepare_gemm_bf16() != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return RCP_ECUDA;
  }
  int64_t off[7];
  mlp_param_offsets(off);
  const int64_t np = off[6], Bt = batch;
  const size_t bf = sizeof(__nv_bfloat16);
  bool ok = cudaMalloc((void**)&p->w, np * 4) == cudaSuccess &&
            cudaMalloc((void**)&p->m, np * 4) == cudaSuccess &&
            cudaMalloc((void**)&p->v, np * 4) == cudaSuccess &&
            cudaMalloc((void**)&p->g, np * 4) == cudaSuccess &&
            cudaMalloc((void**)&p->Wb, np * bf) == cudaSuccess &&
            cudaMalloc((void**)&p->WTb2, (size_t)kMlpHidden * kMlpHidden * bf) == cudaSuccess &&
            cudaMalloc((void**)&p->WTb3, (size_t)kMlpHidden * kMlpOut * bf) == cudaSuccess &&
            cudaMalloc((void**)&p->x32, Bt * kMlpIn * 4) == cudaSuccess &&
            cudaMalloc((void**)&p->Xb, Bt * kMlpIn * bf) == cudaSuccess &&
            cudaMalloc((void**)&p->XTb, Bt * kMlpIn * bf) == cudaSuccess &&
            cudaMalloc((void**)&p->H1b, Bt * kMlpHidden * bf) == cudaSuccess &&
            cudaMalloc((void**)&p->H1Tb, Bt * kMlpHidden * bf) == cudaSuccess &&
            cudaMalloc((void**)&p->H2b, Bt * kMlpHidden * bf) == cudaSuccess &&
            cudaMalloc((void**)&p->H2Tb, Bt * kMlpHidden * bf) == cudaSuccess &&
            cudaMalloc((void**)&p->dYb, Bt * kMlpOut * bf) == cudaSuccess &&
            cudaMalloc((void**)&p->dYTb, Bt * kMlpOut * bf) == cudaSuccess &&
            cudaMalloc((void**)&p->dZ2b, Bt * kMlpHidden * bf) == cudaSuccess &&
            cudaMalloc((void**)&p->dZ2Tb, Bt * kMlpHidden * bf) == cudaSuccess &&
            cudaMalloc((void**)&p->dZ1Tb, Bt * kMlpHidden * bf) == cudaSuccess &&
            cudaMalloc((void**)&p->P, (size_t)kMlpSplit1 * Bt * kMlpHidden * 4) == cudaSuccess &&
            cudaMalloc((void**)&p->Y, Bt * kMlpOut * 4) == cudaSuccess &&
            cudaMalloc((void**)&p->dY, Bt * kMlpOut * 4) == cudaSuccess &&
            cudaMalloc((void**)&p->loss, Bt * 4) == cudaSuccess &&
            cudaMalloc((void**)&p->U, Bt * 3 * kWsL * kWsL * 4) == cudaSuccess &&
            cudaMalloc((void**)&p->meta, Bt * 4 * sizeof(int)) == cudaSuccess &&
            cudaMalloc((void**)&p->dst, sizeof(DevState)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_mlp(p);
    return RCP_ENOMEM;
  }
  cudaStream_t s = p->stream;
  ok = cudaMemsetAsync(p->m, 0, np * 4, s) == cudaSuccess &&
       cudaMemsetAsync(p->v, 0, np * 4, s) == cudaSuccess &&
       cudaMemsetAsync(p->g, 0, np * 4, s) == cudaSuccess &&
       cudaMemsetAsync(p->dY, 0, Bt * kMlpOut * 4, s) == cudaSuccess &&
       cudaMemsetAsync(p->dst, 0, sizeof(DevState), s) == cudaSuccess;
  count_launches(1);
  k_mlp_init<<<grid1(np, p->nsm), 256, 0, s>>>(p->w, seed, np, off[1], off[2], off[3], off[4], off[5]);
  if (!ok || cudaGetLastError() != cudaSuccess || mlp_refresh_bf16(p, s) != RCP_OK) {
    cudaGetLastError();
    free_mlp(p);
    return RCP_ECUDA;
  }
  *out = p;
  return RCP_OK;
}

rcp_status rcp_mlp_destroy(rcp_mlp_t p) {
  if (!p) return RCP_OK;
  cudaStreamSynchronize(p->stream);
  free_mlp(p);
  return RCP_OK;
}

rcp_status rcp_mlp_get_params(rcp_mlp_t p, float* params, float* adam_m, float* adam_v, int64_t* step) {
  if (!p) return RCP_EINVAL;
  const int64_t np = rcp_mlp_param_count();
  MLP_TRY(cudaStreamSynchronize(p->stream));
  if (params) MLP_TRY(cudaMemcpy(params, p->w, np * 4, cudaMemcpyDeviceToHost));
  if (adam_m) MLP_TRY(cudaMemcpy(adam_m, p->m, np * 4, cudaMemcpyDeviceToHost));
  if (adam_v) MLP_TRY(cudaMemcpy(adam_v, p->v, np * 4, cudaMemcpyDeviceToHost));
  if (step) *step = p->t;
  return RCP_OK;
}

rcp_status rcp_mlp_set_params(rcp_mlp_t p, const float* params, const float* adam_m,
                              const float* adam_v, int64_t step) {
  if (!p || step < 0) return RCP_EINVAL;
  const int64_t np = rcp_mlp_param_count();
  MLP_TRY(cudaStreamSynchronize(p->stream));
  if (params) MLP_TRY(cudaMemcpy(p->w, params, np * 4, cudaMemcpyHostToDevice));
  if (adam_m) MLP_TRY(cudaMemcpy(p->m, adam_m, np * 4, cudaMemcpyHostToDevice));
  if (adam_v) MLP_TRY(cudaMemcpy(p->v, adam_v, np * 4, cudaMemcpyHostToDevice));
  p->t = step;
  return mlp_refresh_bf16(p, p->stream);
}

rcp_status rcp_mlp_forward(rcp_mlp_t p, const float* x_dev, int32_t count, int32_t train, float* y_dev) {
  if (!p || !x_dev || count < 1 || count > p->batch) return RCP_EINVAL;
  rcp_status st = mlp_forward_enqueue(p, x_dev, count, train != 0, p->stream);
  if (st != RCP_OK) return st;
  if (y_dev)
    MLP_TRY(cudaMemcpyAsync(y_dev, p->Y, (size_t)count * kMlpOut * 4, cudaMemcpyDeviceToDevice,
                            p->stream));
  return RCP_OK;
}

rcp_status rcp_mlp_backward(rcp_mlp_t p, const float* dy_dev, float* grad_dev) {
  if (!p || !dy_dev) return RCP_EINVAL;
  if (!p->has_grad) return RCP_EORDER;
  rcp_status st = mlp_backward_enqueue(p, dy_dev, p->stream);
  if (st != RCP_OK) return st;
  if (grad_dev)
    MLP_TRY(cudaMemcpyAsync(grad_dev, p->g, rcp_mlp_param_count() * 4, cudaMemcpyDeviceToDevice,
                            p->stream));
  return RCP_OK;
}

rcp_status rcp_mlp_adam(rcp_mlp_t p, float lr, float beta1, float beta2, float eps) {
  if (!p || !(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) ||
      !(eps > 0.0f))
    return RCP_EINVAL;
  return mlp_adam_enqueue(p, lr, beta1, beta2, eps, p->stream);
}

rcp_status rcp_mlp_status(rcp_mlp_t p) {
  if (!p) return RCP_EINVAL;
  DevState h;
  MLP_TRY(cudaMemcpyAsync(&h, p->dst, sizeof(h), cudaMemcpyDeviceToHost, p->stream));
  MLP_TRY(cudaStreamSynchronize(p->stream));
  return (rcp_status)h.status;
}

rcp_status rcp_ws_canonicalize(const float* Bpad_dev, const int32_t* meta_dev, int32_t count,
                               float* x_dev, float* U_dev, void* stream) {
  if (!Bpad_dev || !meta_dev || !x_dev || !U_dev || count < 1) return RCP_EINVAL;
  MLP_TRY(prepare_ws());
  MLP_TRY(launch_ws_canon(Bpad_dev, meta_dev, count, x_dev, U_dev, (cudaStream_t)stream));
  return RCP_OK;
}

rcp_status rcp_ws_loss(const float* y_dev, const float* t_dev, const int32_t* meta_dev,
                       int32_t count, float scale, float* dy_dev, float* loss_dev, void* stream) {
  if (!y_dev || !t_dev || !meta_dev || !dy_dev || !loss_dev || count < 1) return RCP_EINVAL;
  MLP_TRY(launch_ws_loss(y_dev, t_dev, meta_dev, count, scale, dy_dev, loss_dev,
                         (cudaStream_t)stream));
  return RCP_OK;
}

rcp_status rcp_mlp_train_step(rcp_mlp_t p, const float* x_dev, const float* t_dev,
                              const int32_t* meta_dev, int32_t count, float lr, float* loss_dev) {
  if (!p || !x_dev || !t_dev || !meta_dev || count < 1 || count > p->batch || !(lr >= 0.0f))
    return RCP_EINVAL;
  cudaStream_t s = p->stream;
  rcp_status st = mlp_forward_enqueue(p, x_dev, count, true, s);
  if (st != RCP_OK) return st;
  // the loss writes dY rows < count only; rows >= count are cleared here, since an
  // earlier step with a larger count leaves its gradient in them and the forward
  // pass gives zero input rows nonzero (bias) activations that would carry it on
  if (count < p->batch)
    MLP_TRY(cudaMemsetAsync(p->dY + (int64_t)count * kMlpOut, 0,
                            (size_t)(p->batch - count) * kMlpOut * 4, s));
  MLP_TRY(launch_ws_loss(p->Y, t_dev, meta_dev, count, 1.0f / (float)count, p->dY, p->loss, s));
  st = mlp_backward_enqueue(p, p->dY, s);
  if (st != RCP_OK) return st;
  st = mlp_adam_enqueue(p, lr, 0.9f, 0.999f, 1e-8f, s);
  if (st != RCP_OK) return st;
  if (loss_dev)
    MLP_TRY(cudaMemcpyAsync(loss_dev, p->loss, (size_t)count * 4, cudaMemcpyDeviceToDevice, s));
  return RCP_OK;
}

}  // extern "C"

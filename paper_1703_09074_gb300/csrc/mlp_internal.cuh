// Internal declarations of the warm-start network and its data preparation.
#pragma once

#include <cuda_bf16.h>

#include "rcp_internal.cuh"

namespace rcp {

constexpr int kWsL = RCP_WS_LPAD;                   // padded mode size of B (24)
constexpr int kWsR = RCP_WS_RPAD;                   // padded rank (16)
constexpr int kMlpIn = kWsL * kWsL * kWsL;          // 13824
constexpr int kMlpHidden = 512;
constexpr int kMlpOut = 3 * kWsL * kWsR;            // 1152
constexpr int kMlpSplit1 = 27;                      // K splits of the input layer (27 x 512)

void mlp_param_offsets(int64_t off[7]);

}  // namespace rcp

struct rcp_mlp_s {
  cudaStream_t stream;
  int nsm;
  int batch;                 // rows per pass (multiple of 128)
  int64_t t;                 // Adam steps taken
  uint64_t seed;
  float *w, *m, *v, *g;      // master parameters, Adam moments, gradients (flat)
  __nv_bfloat16 *Wb;         // BF16 copy of the flat parameters (weights used as GEMM operands)
  __nv_bfloat16 *WTb2, *WTb3;  // transposed BF16 W2 (H x H) and W3 (H x Out)
  float* x32;                // batch x In FP32 input rows (internal inputs)
  __nv_bfloat16 *Xb, *XTb, *H1b, *H1Tb, *H2b, *H2Tb, *dYb, *dYTb, *dZ2b, *dZ2Tb, *dZ1Tb;
  float* P;                  // split partials
  float *Y, *dY;             // batch x Out
  float* loss;               // batch
  float* U;                  // batch x 3 x L x L canonical bases (internal inputs)
  int* meta;                 // batch x 4 (l1, l2, l3, R) (internal inputs)
  rcp::DevState* dst;        // status word
  bool has_grad;             // a training forward pass was enqueued
};

namespace rcp {
rcp_status mlp_forward_enqueue(rcp_mlp_s* p, const float* x, int count, bool train, cudaStream_t s);
rcp_status mlp_backward_enqueue(rcp_mlp_s* p, const float* dY, cudaStream_t s);
rcp_status mlp_adam_enqueue(rcp_mlp_s* p, float lr, float b1, float b2, float eps, cudaStream_t s);
rcp_status mlp_refresh_bf16(rcp_mlp_s* p, cudaStream_t s);
cudaError_t prepare_gemm_bf16();

// warm-start data path (warmstart.cu)
struct WsItem {
  const float* core;   // Kolda l1 x l2 x l3 (FP32), or nullptr when the tensor is not eligible
  int l[3];
  int R;
  double* At[3];       // ALS initial factors (column-major l_n x R), written by the init kernel
  int* user_init;      // the ALS argument word to set (1 = use At, 0 = random init)
  DevState* st;        // receives RCP_INFO_LEARNED_INIT
};
cudaError_t prepare_ws();
cudaError_t launch_ws_gather(const WsItem* items, int count, float* Bpad, int* meta, cudaStream_t s);
cudaError_t launch_ws_canon(const float* Bpad, const int* meta, int count, float* x, float* U,
                            cudaStream_t s);
cudaError_t launch_ws_loss(const float* Y, const float* T, const int* meta, int count, float scale,
                           float* dY, float* loss, cudaStream_t s);
cudaError_t launch_ws_init(const float* Y, const float* U, const int* meta, const WsItem* items,
                           int count, cudaStream_t s);
cudaError_t launch_ws_targets(const WsItem* items, const float* U, int count, float* T,
                              cudaStream_t s);
}  // namespace rcp

// The learned warm start on the single-tensor path (rcp_set_warm_start): the
// same data path as the batched form's, for the one compressed tensor of a
// plan -- gather B into the padded 24^3 layout, canonical basis and network
// input, one forward pass, initial factors A_n = U_n (E + Y_n) for n = 2, 3.
// A device word tells the stage-2 kernel whether the prediction was usable
// (every column finite and nonzero); otherwise it keeps the seeded start.
#include <new>

#include "mlp_internal.cuh"

struct rcp_plan_ws_s {
  rcp_mlp_s* net = nullptr;
  rcp::WsItem* item = nullptr;   // device, one item
  float* B = nullptr;            // 24^3 padded core
  float* x = nullptr;            // 24^3 network input
  float* U = nullptr;            // 3 x 24 x 24 canonical bases
  int* meta = nullptr;           // 4
  int* flag = nullptr;           // 1: the stage-2 solver starts from the predicted factors
};

namespace rcp {

void plan_ws_free(rcp_plan_s* p) {
  rcp_plan_ws_s* w = p->ws;
  if (!w) return;
  cudaFree(w->item);
  cudaFree(w->B);
  cudaFree(w->x);
  cudaFree(w->U);
  cudaFree(w->meta);
  cudaFree(w->flag);
  delete w;
  p->ws = nullptr;
}

// Enqueue the warm start on the plan's stream; *flag_dev receives the device
// word that says whether the stage-2 solver uses the predicted factors.
rcp_status plan_ws_enqueue(rcp_plan_s* p, const int** flag_dev) {
  rcp_plan_ws_s* w = p->ws;
  *flag_dev = nullptr;
  if (!w || !w->net) return RCP_OK;
  cudaStream_t s = p->stream;
  if (launch_ws_gather(w->item, 1, w->B, w->meta, s) != cudaSuccess) return RCP_ECUDA;
  if (launch_ws_canon(w->B, w->meta, 1, w->x, w->U, s) != cudaSuccess) return RCP_ECUDA;
  if (mlp_forward_enqueue(w->net, w->x, 1, false, s) != RCP_OK) return RCP_ECUDA;
  if (launch_ws_init(w->net->Y, w->U, w->meta, w->item, 1, s) != cudaSuccess) return RCP_ECUDA;
  *flag_dev = w->flag;
  return RCP_OK;
}

}  // namespace rcp

extern "C" rcp_status rcp_set_warm_start(rcp_plan_t p, rcp_mlp_t net) {
  using namespace rcp;
  if (!p || p->N < 2) return RCP_EINVAL;
  if (!net) {
    if (p->ws) p->ws->net = nullptr;
    return RCP_OK;
  }
  if (p->prec != RCP_PREC_MIXED || p->N != 3 || p->R > kWsR) return RCP_EINVAL;
  for (int n = 0; n < 3; ++n)
    if (p->l[n] > kWsL) return RCP_EINVAL;
  if (!p->ws) {
    rcp_plan_ws_s* w = new (std::nothrow) rcp_plan_ws_s();
    if (!w) return RCP_ENOMEM;
    p->ws = w;
    if (cudaMalloc((void**)&w->item, sizeof(WsItem)) != cudaSuccess ||
        cudaMalloc((void**)&w->B, (size_t)kMlpIn * 4) != cudaSuccess ||
        cudaMalloc((void**)&w->x, (size_t)kMlpIn * 4) != cudaSuccess ||
        cudaMalloc((void**)&w->U, (size_t)3 * kWsL * kWsL * 4) != cudaSuccess ||
        cudaMalloc((void**)&w->meta, 4 * sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&w->flag, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      plan_ws_free(p);
      return RCP_ENOMEM;
    }
    if (prepare_ws() != cudaSuccess) return RCP_ECUDA;
    WsItem it{};
    it.core = (const float*)p->bufT[(p->N - 1) % 2];   // B of the precision form (FP32)
    for (int n = 0; n < 3; ++n) {
      it.l[n] = p->l[n];
      it.At[n] = p->At[n];
    }
    it.R = p->R;
    it.user_init = w->flag;
    it.st = p->dstate;
    if (cudaMemcpy(w->item, &it, sizeof(it), cudaMemcpyHostToDevice) != cudaSuccess)
      return RCP_ECUDA;
  }
  p->ws->net = net;
  return RCP_OK;
}

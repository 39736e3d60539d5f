// Allocation-free mode-1 range finder for callers that cannot allocate device
// memory (no plan, no cudaMalloc): code running inside another library's
// allocator-free region, a host process whose device memory is owned and
// budgeted by a framework that forbids allocation after start-up, or a caller
// in a signal or teardown path.  The caller passes the input tensor and the
// output basis; the split partials and the QR scratch live in one file-scope
// device array that every GPU loading this library holds until process exit.
#include <mutex>

#include "rcp_internal.cuh"

namespace rcp {
cudaError_t launch_cholqr(double* Y, int64_t I, int l, double* Gp, double* Rinv, DevState* st,
                          cudaStream_t s, bool final_qr, bool no_shift = false);
}  // namespace rcp

namespace {

// Scratch layout (doubles): [ partials | sketch Y | packed Gram | R^{-1} | DevState ]
constexpr int64_t kScratchDoubles = 1 << 19;  // 4 MiB
constexpr int64_t kSmallDoubles = (int64_t)rcp::kMaxL * (rcp::kMaxL + 1) / 2 + rcp::kMaxL * rcp::kMaxL +
                                  (int64_t)(sizeof(rcp::DevState) + 7) / 8;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_addr[kMaxDevices];  // device address of g_noalloc_scratch, per device

__global__ void k_copy_status(const rcp::DevState* st, int32_t* out) { *out = st->status; }

// Resolve the scratch array's device address for the current device (once per device).
rcp_status scratch_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RCP_ECUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return RCP_ECUDA;
    }
    g_addr[dev] = (double*)p;
  }
  *out = g_addr[dev];
  return RCP_OK;
}

}  // namespace

extern "C" rcp_status rcp_sketch_mode1_static(const void* X_dev, int32_t in_dtype, int32_t ndim,
                                              const int64_t* dims, int32_t rank, int32_t oversample,
                                              uint64_t seed, double* Q_dev, int32_t* status_dev,
                                              void* stream) {
  using namespace rcp;
  if (!X_dev || !Q_dev || !dims) return RCP_EINVAL;
  if (in_dtype != RCP_DTYPE_F64 && in_dtype != RCP_DTYPE_F32) return RCP_EINVAL;
  if (ndim < 2 || ndim > kMaxN || rank < 1 || rank > RCP_MAX_RANK || oversample < 0)
    return RCP_EINVAL;
  int64_t J = 1, total = 1;
  for (int n = 0; n < ndim; ++n) {
    if (dims[n] < 1 || dims[n] > (1LL << 40)) return RCP_EINVAL;
    // the element count must not overflow (a wrapped J would size the sweep wrongly)
    if (!mul_elems(total, dims[n], &total)) return RCP_EINVAL;
    if (n > 0) J *= dims[n];
  }
  const int64_t I = dims[0];
  int64_t l = (int64_t)rank + oversample;
  if (l > I) l = I;
  if (l > J) l = J;
  if (l < rank || l > RCP_MAX_L) return RCP_EINVAL;
  // partials of at least one split plus the sketch itself must fit beside the small scratch
  const int64_t room = kScratchDoubles - kSmallDoubles - I * l;
  if (room < I * l) return RCP_EINVAL;

  double* base = nullptr;
  rcp_status st = scratch_for_current_device(&base);
  if (st != RCP_OK) return st;
  int nsm = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return RCP_ECUDA;

  const ModeView v{1, I, J, J};
  int64_t nsplit = sketch_splits(v, nsm);
  if (nsplit * I * l > room) nsplit = room / (I * l);
  double* part = base;
  double* Y = base + nsplit * I * l;
  double* Gp = Y + I * l;
  double* Rinv = Gp + (int64_t)kMaxL * (kMaxL + 1) / 2;
  DevState* dst = (DevState*)(Rinv + (int64_t)kMaxL * kMaxL);
  cudaStream_t s = (cudaStream_t)stream;

  // the status word must start at zero; the partials and Y are fully overwritten
  if (cudaMemsetAsync(dst, 0, sizeof(DevState), s) != cudaSuccess) return RCP_ECUDA;
  if (launch_sketch_f64(X_dev, in_dtype, v, (int)l, seed, 1u, nullptr, (int)nsplit, part, nullptr,
                        s) != cudaSuccess)
    return RCP_ECUDA;
  if (launch_reduce(part, nsplit, I * l, Y, nullptr, 0, s) != cudaSuccess) return RCP_ECUDA;
  if (launch_cholqr(Y, I, (int)l, Gp, Rinv, dst, s, true) != cudaSuccess) return RCP_ECUDA;
  if (cudaMemcpyAsync(Q_dev, Y, sizeof(double) * I * l, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return RCP_ECUDA;
  if (status_dev) {
    count_launches(1);
    k_copy_status<<<1, 1, 0, s>>>(dst, status_dev);
    if (cudaGetLastError() != cudaSuccess) return RCP_ECUDA;
  }
  return RCP_OK;
}

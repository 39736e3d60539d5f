// Host side of the C ABI declared in include/rcp.h: plan creation and workspace
// sizing, the order of Algorithm 1 and Algorithm 2, and the launch sequences.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "rcp_internal.cuh"

namespace rcp {
cudaError_t launch_gram(const double* Y, int64_t I, int l, double* Gp, cudaStream_t s);
cudaError_t launch_chol(const double* Gp, int l, double* Rinv, DevState* st, double shift_rows,
                        int round, int als_mode, cudaStream_t s, bool no_shift = false);
cudaError_t launch_cholqr(double* Y, int64_t I, int l, double* Gp, double* Rinv, DevState* st,
                          cudaStream_t s, bool final_qr, bool no_shift = false);
cudaError_t launch_sum_to(const double* part, int64_t n, double* dst, cudaStream_t s);
cudaError_t launch_lu_norm(double* Y, int64_t M, int l, int64_t L, uint8_t* used, double* cval,
                           int64_t* cidx, double* prow, DevState* st, int nsm, cudaStream_t s);
cudaError_t launch_sumsq(const double* x, int64_t n, double* part, int nblocks, double* dst,
                         cudaStream_t s);
}  // namespace rcp

using namespace rcp;

int64_t& rcp::launch_counter() {
  static thread_local int64_t count = 0;
  return count;
}

namespace {

// Records a pair of CUDA events on the plan's stream around the launches made
// in its scope when profiling is on.
struct Span {
  rcp_plan_t p;
  int idx = -1;
  Span(rcp_plan_t p_, int kind, int mode) : p(p_) {
    if (p->prof_on && p->prof_n < p->prof_cap) {
      idx = p->prof_n++;
      p->prof[idx].kind = kind;
      p->prof[idx].mode = mode;
      cudaEventRecord(p->prof[idx].a, p->stream);
    }
  }
  ~Span() {
    if (idx >= 0) cudaEventRecord(p->prof[idx].b, p->stream);
  }
};

#define RCP_TRY(call)                                  \
  do {                                                 \
    cudaError_t _e = (call);                           \
    if (_e != cudaSuccess) return RCP_ECUDA;           \
  } while (0)

bool valid_plan(rcp_plan_t p) { return p != nullptr && p->N >= 2; }

bool mode_skipped(const rcp_config* cfg, int n0) { return (cfg->skip_modes >> n0) & 1; }

// l_n of Algorithm 1 step 3 for 0-based mode n0 of the current shape (I_n, J_n):
// min(R + p_n, I_n, J_n), p_n the mode's own oversampling when the plan sets
// one (the remark after Algorithm 1); an uncompressed mode keeps l_n = I_n.
int64_t mode_width(const rcp_config* cfg, int n0, int64_t In, int64_t J) {
  if (mode_skipped(cfg, n0)) return In;
  const int64_t pn = (cfg->flags & RCP_FLAG_MODE_OVERSAMPLE) ? cfg->mode_oversample[n0]
                                                             : cfg->oversample;
  return std::min<int64_t>((int64_t)cfg->rank + pn, std::min(In, J));
}

template <typename T>
rcp_status dalloc(T** ptr, int64_t elems) {
  *ptr = nullptr;
  if (elems <= 0) elems = 1;
  if (cudaMalloc((void**)ptr, (size_t)elems * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return RCP_ENOMEM;
  }
  return RCP_OK;
}

void free_plan(rcp_plan_t p) {
  if (!p) return;
  cudaFree(p->bufT[0]);
  cudaFree(p->bufT[1]);
  for (int n = 0; n < kMaxN; ++n) {
    cudaFree(p->Q[n]);
    cudaFree(p->At[n]);
    cudaFree(p->Gm[n]);
    cudaFree(p->A_stage[n]);
  }
  cudaFree(p->Y);
  cudaFree(p->part);
  cudaFree(p->tmp);
  cudaFree(p->gpart);
  cudaFree(p->G);
  cudaFree(p->Rinv);
  cudaFree(p->RWinv);
  cudaFree(p->normpart);
  cudaFree(p->M);
  cudaFree(p->lam);
  cudaFree(p->Bcore_own);
  cudaFree(p->part32);
  cudaFree(p->QT32);
  cudaFree(p->dstate);
  cudaFree(p->bar);
  cudaFree(p->abort_flag);
  plan_ws_free(p);
  cudaFree(p->X_stage);
  cudaFree(p->lu_used);
  cudaFree(p->lu_cval);
  cudaFree(p->lu_cidx);
  cudaFree(p->lu_prow);
  cudaFree(p->lam_stage);
  cudaFree(p->als_S);
  if (p->prof) {
    for (int k = 0; k < p->prof_cap; ++k) {
      cudaEventDestroy(p->prof[k].a);
      cudaEventDestroy(p->prof[k].b);
    }
    delete[] p->prof;
  }
  delete p;
}

// Input of mode n (1-based): X for n = 1, else the buffer T_n was written to.
const void* mode_input(rcp_plan_t p, const void* X, int n, int* dtype) {
  if (n == 1) {
    *dtype = p->cfg.in_dtype;
    return X;
  }
  *dtype = RCP_DTYPE_F64;
  return p->bufT[(n - 2) % 2];
}

double* mode_output(rcp_plan_t p, int n) { return (double*)p->bufT[(n - 1) % 2]; }

rcp_status check_device(rcp_plan_t p) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return RCP_ECUDA;
  if (dev != p->device && cudaSetDevice(p->device) != cudaSuccess) return RCP_ECUDA;
  return RCP_OK;
}

}  // namespace

extern "C" {

const char* rcp_status_str(rcp_status s) {
  switch (s) {
    case RCP_OK: return "ok";
    case RCP_EINVAL: return "invalid argument";
    case RCP_ENOMEM: return "out of memory";
    case RCP_ECUDA: return "CUDA runtime error";
    case RCP_ESINGULAR: return "singular Gram matrix";
    case RCP_ENAN: return "non-finite value";
    case RCP_ETIMEOUT: return "device wait timed out";
    case RCP_EORDER: return "calls out of order";
    case RCP_ENOTCONV: return "ALS stopped at max_iters";
  }
  return "unknown status";
}

rcp_status rcp_plan(const rcp_config* cfg, void* stream, rcp_plan_t* out) {
  if (!cfg || !out) return RCP_EINVAL;
  const int N = cfg->ndim;
  if (N < 2 || N > kMaxN) return RCP_EINVAL;
  if (cfg->rank < 1 || cfg->rank > RCP_MAX_RANK) return RCP_EINVAL;
  if (cfg->oversample < 0 || cfg->power_iters < 0 || cfg->max_iters < 1) return RCP_EINVAL;
  if (!(cfg->tol >= 0.0)) return RCP_EINVAL;
  if (cfg->in_dtype != RCP_DTYPE_F64 && cfg->in_dtype != RCP_DTYPE_F32) return RCP_EINVAL;
  if (cfg->precision != RCP_PREC_F64 && cfg->precision != RCP_PREC_MIXED) return RCP_EINVAL;
  if (cfg->precision == RCP_PREC_MIXED && cfg->in_dtype != RCP_DTYPE_F32) return RCP_EINVAL;
  if (cfg->init != RCP_INIT_RANDN && cfg->init != RCP_INIT_EIG && cfg->init != RCP_INIT_LEARNED)
    return RCP_EINVAL;
  if (cfg->init == RCP_INIT_LEARNED && cfg->precision != RCP_PREC_MIXED) return RCP_EINVAL;
  if (cfg->solver != RCP_SOLVER_ALS && cfg->solver != RCP_SOLVER_BCD) return RCP_EINVAL;
  if (cfg->wait_budget < 0) return RCP_EINVAL;
  if (cfg->flags & ~(RCP_FLAG_HOST_STAGING | RCP_FLAG_NO_SHIFT | RCP_FLAG_MODE_OVERSAMPLE |
                     RCP_FLAG_LU_NORM | RCP_FLAG_INDEPENDENT))
    return RCP_EINVAL;
  if (cfg->skip_modes & ~((1 << N) - 1)) return RCP_EINVAL;
  if ((cfg->flags & RCP_FLAG_LU_NORM) && cfg->precision != RCP_PREC_F64) return RCP_EINVAL;
  {
    int64_t total = 1;
    for (int n = 0; n < N; ++n) {
      if (cfg->dims[n] < 1 || cfg->dims[n] > (1LL << 40)) return RCP_EINVAL;
      if (!mul_elems(total, cfg->dims[n], &total)) return RCP_EINVAL;  // no int64 overflow below
    }
  }
  {
    // every l_n = min(R + p, I_n, J_n) must lie in [R, RCP_MAX_L] (checked before any CUDA call)
    int64_t cur[kMaxN];
    for (int n = 0; n < N; ++n) cur[n] = cfg->dims[n];
    const bool indep = (cfg->flags & RCP_FLAG_INDEPENDENT) != 0;
    for (int n = 0; n < N; ++n) {
      int64_t J = 1;
      for (int m = 0; m < N; ++m)
        if (m != n) J *= indep ? cfg->dims[m] : cur[m];
      if ((cfg->flags & RCP_FLAG_MODE_OVERSAMPLE) && cfg->mode_oversample[n] < 0) return RCP_EINVAL;
      const int64_t l = mode_width(cfg, n, cur[n], J);
      if (l < cfg->rank || l > RCP_MAX_L) return RCP_EINVAL;
      cur[n] = l;
    }
  }

  rcp_plan_t p = new (std::nothrow) rcp_plan_s();
  if (!p) return RCP_ENOMEM;
  memset((void*)p, 0, sizeof(*p));
  p->cfg = *cfg;
  p->stream = (cudaStream_t)stream;
  p->N = N;
  p->R = cfg->rank;
  p->prec = cfg->precision;
  p->work_elem = cfg->precision == RCP_PREC_MIXED ? 4 : 8;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    delete p;
    return RCP_ECUDA;
  }
  if (cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) {
    delete p;
    return RCP_ECUDA;
  }

  // widths l_n = min(R + p, I_n, J_n) over the shrinking tensor (Algorithm 1 step 3)
  int64_t cur[kMaxN];
  for (int n = 0; n < N; ++n) cur[n] = p->dims[n] = cfg->dims[n];
  int64_t bufmax = 1, Imax = 1, part_max = 1, gpart_max = 1, norm_max = 1, red_max = 1;
  const bool indep = (cfg->flags & RCP_FLAG_INDEPENDENT) != 0;
  for (int n = 0; n < N; ++n) {
    int64_t J = 1, L = 1, Rt = 1;
    for (int m = 0; m < N; ++m)
      if (m != n) J *= cur[m];
    for (int m = 0; m < n; ++m) L *= cur[m];
    for (int m = n + 1; m < N; ++m) Rt *= cur[m];
    // mode n of X itself: the operand of the independent sketches
    ModeView xv{1, p->dims[n], 1, 1};
    for (int m = 0; m < n; ++m) xv.L *= p->dims[m];
    for (int m = n + 1; m < N; ++m) xv.Rt *= p->dims[m];
    xv.J = xv.L * xv.Rt;
    p->xview[n] = xv;
    const int64_t l = mode_width(cfg, n, cur[n], indep ? xv.J : J);
    if (l < cfg->rank || l > RCP_MAX_L) {
      delete p;
      return RCP_EINVAL;
    }
    p->l[n] = (int)l;
    p->view[n] = ModeView{L, cur[n], Rt, J};
    bufmax = std::max(bufmax, J * l);
    Imax = std::max(Imax, cur[n]);
    const int ns = sketch_splits(p->view[n], p->nsm);
    part_max = std::max(part_max, (int64_t)ns * cur[n] * l);
    red_max = std::max(red_max, cur[n] * l);
    const int ng = project_grid(p->view[n], p->nsm);
    gpart_max = std::max(gpart_max, (int64_t)ng * (l * (l + 1) / 2));
    norm_max = std::max(norm_max, (int64_t)ns * ((cur[n] + 255) / 256));
    if (indep) {  // the range finder's W and partials over X_(n)
      bufmax = std::max(bufmax, xv.J * l);
      const int nsx = sketch_splits(xv, p->nsm);
      part_max = std::max(part_max, (int64_t)nsx * xv.I * l);
      gpart_max = std::max(gpart_max, (int64_t)project_grid(xv, p->nsm) * (l * (l + 1) / 2));
      norm_max = std::max(norm_max, (int64_t)nsx * ((xv.I + 255) / 256));
    }
    cur[n] = l;
  }
  p->core_elems = 1;
  for (int n = 0; n < N; ++n) p->core_elems *= p->l[n];
  // ALS MTTKRP partials
  for (int n = 0; n < N; ++n) {
    ModeView v{1, p->l[n], 1, 0};
    for (int m = 0; m < n; ++m) v.L *= p->l[m];
    for (int m = n + 1; m < N; ++m) v.Rt *= p->l[m];
    v.J = v.L * v.Rt;
    part_max = std::max(part_max, (int64_t)sketch_splits(v, p->nsm) * p->l[n] * p->R);
  }
  {
    int lmx = 1;
    for (int n = 0; n < N; ++n) lmx = lmx > p->l[n] ? lmx : p->l[n];
    part_max = std::max(part_max, (int64_t)p->nsm * lmx * p->R);  // persistent ALS partials
    part_max = std::max(part_max, (int64_t)N * 32 * 32);  // one-cluster ALS: N x 32 x 32 float2
  }
  part_max = std::max(part_max, bcd_scratch_elems(p));  // rCP-BCD contraction buffers
  p->bufT_elems = bufmax;
  p->part_elems = part_max;
  p->tmp_elems = std::max<int64_t>(16 * std::max(red_max, (int64_t)kMaxL * (kMaxL + 1) / 2),
                                   (int64_t)kMaxN * RCP_MAX_RANK);
  p->tmp_elems = std::max<int64_t>(p->tmp_elems, (int64_t)kMaxN * kMaxL * kMaxL);  // eig-init Grams
  p->gpart_elems = gpart_max;
  p->normpart_elems = std::max<int64_t>(norm_max, 4096);

  rcp_status st = RCP_OK;
  auto A = [&](rcp_status s) {
    if (st == RCP_OK) st = s;
  };
  A(dalloc((double**)&p->bufT[0], bufmax));
  A(dalloc((double**)&p->bufT[1], bufmax));
  for (int n = 0; n < N; ++n) {
    A(dalloc(&p->Q[n], p->dims[n] * p->l[n]));
    A(dalloc(&p->At[n], (int64_t)p->l[n] * p->R));
    A(dalloc(&p->Gm[n], (int64_t)p->R * p->R));
  }
  A(dalloc(&p->Y, Imax * kMaxL));
  A(dalloc(&p->part, part_max));
  A(dalloc(&p->tmp, p->tmp_elems));
  A(dalloc(&p->gpart, gpart_max));
  A(dalloc(&p->G, kMaxL * (kMaxL + 1) / 2));
  A(dalloc(&p->Rinv, kMaxL * kMaxL));
  A(dalloc(&p->RWinv, kMaxL * kMaxL));
  A(dalloc(&p->normpart, p->normpart_elems));
  A(dalloc(&p->M, (int64_t)kMaxL * p->R));
  A(dalloc(&p->lam, p->R));
  A(dalloc(&p->dstate, 1));
  A(dalloc(&p->bar, 4));
  A(dalloc(&p->abort_flag, 4));
  if (p->prec == RCP_PREC_MIXED) {
    p->tc1 = !mode_skipped(cfg, 0) && tc_mode1_supported(p->dims[0], p->l[0]);
    int64_t p32 = 1;
    if (p->tc1) {
      // partials of either row sweep (register-staged or TMA-fed)
      int ns = 0, nb = 0, rb = 0, ns2 = 0;
      int64_t jc = 0, cper = 0;
      tc_rows_split(p->dims[0], p->view[0].J, p->nsm, &ns, &jc);
      tc_rows_tma_shape(p->dims[0], p->view[0].J, p->nsm, &nb, &rb, &ns2, &cper);
      p32 = (int64_t)std::max(ns, ns2) * p->dims[0] * p->l[0];
    }
    p->part32_elems = p32;
    A(dalloc(&p->part32, p32));
    A(dalloc(&p->QT32, (int64_t)2 * 64 * tc_ipad(Imax)));
    A(dalloc(&p->Bcore_own, p->core_elems));
    // the dimension-tree MTTKRP of the persistent ALS kernel (cores beyond the
    // one-cluster kernel): B contracted over mode 1 or 2, R <= 32 columns
    if (st == RCP_OK && N >= 3 && p->R <= 32 && !als_cluster_fits(p)) {
      int lmx = 1;
      for (int n = 0; n < N; ++n) lmx = lmx > p->l[n] ? lmx : p->l[n];
      if (lmx <= 64) {
        const int64_t rest = p->core_elems / (p->l[0] < p->l[1] ? p->l[0] : p->l[1]);
        A(dalloc(&p->als_S, rest * 32));
      }
    }
  }
  if (cfg->flags & RCP_FLAG_LU_NORM) {
    int64_t mrows = 1;
    for (int n = 0; n < N; ++n) {
      mrows = std::max(mrows, std::max(p->view[n].I, p->view[n].J));
      if (indep) mrows = std::max(mrows, p->xview[n].J);
    }
    A(dalloc((uint8_t**)&p->lu_used, mrows));
    A(dalloc(&p->lu_cval, 2 * (int64_t)p->nsm));
    A(dalloc((int64_t**)&p->lu_cidx, 2 * (int64_t)p->nsm));
    A(dalloc(&p->lu_prow, kMaxL + 1));
  }
  if (cfg->flags & RCP_FLAG_HOST_STAGING) {
    int64_t nx = 1;
    for (int n = 0; n < N; ++n) nx *= p->dims[n];
    const int64_t esz = cfg->in_dtype == RCP_DTYPE_F32 ? 4 : 8;
    A(dalloc((char**)&p->X_stage, nx * esz));
    for (int n = 0; n < N; ++n) A(dalloc(&p->A_stage[n], p->dims[n] * p->R));
    A(dalloc(&p->lam_stage, p->R));
  }
  if (st == RCP_OK && cudaMemsetAsync(p->dstate, 0, sizeof(DevState), p->stream) != cudaSuccess)
    st = RCP_ECUDA;
  if (st != RCP_OK) {
    free_plan(p);
    return st;
  }
  *out = p;
  return RCP_OK;
}

rcp_status rcp_plan_destroy(rcp_plan_t plan) {
  if (!plan) return RCP_OK;
  cudaStreamSynchronize(plan->stream);
  free_plan(plan);
  return RCP_OK;
}

int32_t rcp_width(rcp_plan_t plan, int32_t mode) {
  if (!valid_plan(plan) || mode < 1 || mode > plan->N) return -1;
  return plan->l[mode - 1];
}

}  // extern "C"

namespace {

// Algorithm 1 steps (5)-(12) for mode n on the FP64 path.
rcp_status sketch_f64(rcp_plan_t p, const void* X, int mode) {
  cudaStream_t s = p->stream;
  const bool ns = (p->cfg.flags & RCP_FLAG_NO_SHIFT) != 0;
  const int n0 = mode - 1;
  const bool indep = (p->cfg.flags & RCP_FLAG_INDEPENDENT) != 0;
  const ModeView v = indep ? p->xview[n0] : p->view[n0];
  const int l = p->l[n0];
  int dt = p->cfg.in_dtype;
  const void* T = indep ? X : mode_input(p, X, mode, &dt);
  double* W = mode_output(p, mode);  // scratch here; rcp_compress writes T_{n+1} there later
  const int nsplit = sketch_splits(v, p->nsm);
  const int64_t ny = v.I * l;
  // Y = T_(n) Omega_n (step 6); mode 1 also accumulates |X|^2
  double* normpart = (mode == 1) ? p->normpart : nullptr;
  {
    Span sp(p, RCP_KT_SKETCH, mode);
    RCP_TRY(launch_sketch_f64(T, dt, v, l, p->cfg.seed, (uint32_t)mode, nullptr, nsplit, p->part,
                              normpart, s));
  }
  RCP_TRY(launch_reduce(p->part, nsplit, ny, p->Y, p->tmp, p->tmp_elems, s));
  if (mode == 1) {
    const int64_t nn = (int64_t)nsplit * ((v.I + 255) / 256);
    RCP_TRY(launch_sum_to(p->normpart, nn, &p->dstate->norm_x2, s));
  }
  const int ng = project_grid(v, p->nsm);
  if ((p->cfg.flags & RCP_FLAG_LU_NORM) && p->cfg.power_iters > 0) {
    // steps 7-11 as printed: Q = lu(Y), Z = lu(T_(n)^T Q), Y = T_(n) Z; then
    // the QR of step 12 (CholeskyQR2)
    for (int it = 0; it < p->cfg.power_iters; ++it) {
      RCP_TRY(launch_lu_norm(p->Y, v.I, l, v.I, p->lu_used, p->lu_cval, p->lu_cidx, p->lu_prow,
                             p->dstate, p->nsm, s));
      {
        Span sp(p, RCP_KT_PROJECT, mode);
        RCP_TRY(launch_project_f64(T, dt, v, l, p->Y, W, p->gpart, ng, s));
      }
      RCP_TRY(launch_lu_norm(W, v.J, l, v.L, p->lu_used, p->lu_cval, p->lu_cidx, p->lu_prow,
                             p->dstate, p->nsm, s));
      {
        Span sp(p, RCP_KT_APPLY, mode);
        RCP_TRY(launch_sketch_f64(T, dt, v, l, 0, 0, W, nsplit, p->part, nullptr, s));
      }
      RCP_TRY(launch_reduce(p->part, nsplit, ny, p->Y, p->tmp, p->tmp_elems, s));
    }
    RCP_TRY(launch_cholqr(p->Y, v.I, l, p->G, p->Rinv, p->dstate, s, true, ns));
    return RCP_OK;
  }
  RCP_TRY(launch_cholqr(p->Y, v.I, l, p->G, p->Rinv, p->dstate, s, p->cfg.power_iters == 0, ns));
  // q normalised power iterations (steps 7-11)
  const int npairs = l * (l + 1) / 2;
  for (int it = 0; it < p->cfg.power_iters; ++it) {
    // W = T_(n)^T Q and its Gram (step 9)
    {
      Span sp(p, RCP_KT_PROJECT, mode);
      RCP_TRY(launch_project_f64(T, dt, v, l, p->Y, W, p->gpart, ng, s));
    }
    RCP_TRY(launch_reduce(p->gpart, ng, npairs, p->G, p->tmp, p->tmp_elems, s));
    RCP_TRY(launch_chol(p->G, l, p->RWinv, p->dstate, (double)v.J, -1, 0, s, ns));
    // Y = T_(n) W R_W^{-1} (step 10), then Q = qr(Y) (step 8 of the next iteration / step 12)
    {
      Span sp(p, RCP_KT_APPLY, mode);
      RCP_TRY(launch_sketch_f64(T, dt, v, l, 0, 0, W, nsplit, p->part, nullptr, s));
    }
    RCP_TRY(launch_reduce(p->part, nsplit, ny, p->Y, p->tmp, p->tmp_elems, s));
    RCP_TRY(launch_trmm(p->Y, v.I, l, p->RWinv, p->Y, p->dstate, 0, s));
    RCP_TRY(launch_cholqr(p->Y, v.I, l, p->G, p->Rinv, p->dstate, s,
                          it == p->cfg.power_iters - 1, ns));
  }
  return RCP_OK;
}

// Mixed-precision form: mode 1 on the tensor cores (TF32 operands, FP32
// accumulation), later modes on FP32 CUDA cores; every QR in FP64.  The
// power-iteration W is not normalised: Y = T_(n) W differs from T_(n) Z by an
// upper-triangular right factor, which the QR of Y removes.
rcp_status sketch_mixed(rcp_plan_t p, const void* X, int mode) {
  cudaStream_t s = p->stream;
  const bool ns = (p->cfg.flags & RCP_FLAG_NO_SHIFT) != 0;
  const int n0 = mode - 1;
  const bool indep = (p->cfg.flags & RCP_FLAG_INDEPENDENT) != 0;
  const ModeView v = indep ? p->xview[n0] : p->view[n0];
  const int l = p->l[n0];
  const float* T = (const float*)(mode == 1 || indep ? X : p->bufT[(mode - 2) % 2]);
  float* W = (float*)mode_output(p, mode);
  const int64_t ny = v.I * l;
  if (mode == 1 && p->tc1) {
    // TMA-fed sweeps when X allows tensor maps (and the rows of the split W,
    // J floats each, start on 16-byte boundaries), else the register-staged ones
    const bool tma = tc_tma_ok(T) && v.J % 4 == 0;
    int nsplit = 0;
    int64_t jchunk = 0;
    tc_rows_split(v.I, v.J, p->nsm, &nsplit, &jchunk);
    const int cgrid = tc_cols_grid(v.J, p->nsm);
    {
      Span sp(p, RCP_KT_SKETCH, mode);
      RCP_TRY(launch_tc_rows(T, v.I, v.J, l, p->cfg.seed, (uint32_t)mode, nullptr, nsplit, jchunk,
                             p->part32, p->normpart, p->dstate, s));
    }
    RCP_TRY(launch_reduce_f32(p->part32, nsplit, ny, p->Y, s));
    const int64_t nn = (int64_t)nsplit * ((v.I + 127) / 128);  // one partial per row-sweep CTA
    RCP_TRY(launch_sum_to(p->normpart, nn, &p->dstate->norm_x2, s));
    RCP_TRY(launch_cholqr(p->Y, v.I, l, p->G, p->Rinv, p->dstate, s, p->cfg.power_iters == 0, ns));
    for (int it = 0; it < p->cfg.power_iters; ++it) {
      RCP_TRY(launch_q_to_qt32(p->Y, v.I, l, p->QT32, s));
      {
        Span sp(p, RCP_KT_PROJECT, mode);
        RCP_TRY(launch_tc_cols(T, v.I, v.J, l, p->QT32, W, false, p->dstate, cgrid, s, tma, tma));
      }
      {
        Span sp(p, RCP_KT_APPLY, mode);
        if (tma) {
          RCP_TRY(launch_tc_rows_tma(T, v.I, v.J, l, W, p->part32, p->dstate, p->nsm, s, &nsplit));
        } else {
          RCP_TRY(launch_tc_rows(T, v.I, v.J, l, 0, 0, W, nsplit, jchunk, p->part32, nullptr,
                                 p->dstate, s));
        }
      }
      RCP_TRY(launch_reduce_f32(p->part32, nsplit, ny, p->Y, s));
      RCP_TRY(launch_cholqr(p->Y, v.I, l, p->G, p->Rinv, p->dstate, s,
                          it == p->cfg.power_iters - 1, ns));
    }
    return RCP_OK;
  }
  const int nsplit = sketch_splits(v, p->nsm);
  double* normpart = (mode == 1) ? p->normpart : nullptr;
  {
    Span sp(p, RCP_KT_SKETCH, mode);
    RCP_TRY(launch_sketch_f32(T, v, l, p->cfg.seed, (uint32_t)mode, nullptr, nsplit, p->part,
                              normpart, s));
  }
  RCP_TRY(launch_reduce(p->part, nsplit, ny, p->Y, p->tmp, p->tmp_elems, s));
  if (mode == 1) {
    const int64_t nn = (int64_t)nsplit * ((v.I + 255) / 256);
    RCP_TRY(launch_sum_to(p->normpart, nn, &p->dstate->norm_x2, s));
  }
  RCP_TRY(launch_cholqr(p->Y, v.I, l, p->G, p->Rinv, p->dstate, s, p->cfg.power_iters == 0, ns));
  const int ng = project_grid(v, p->nsm);
  for (int it = 0; it < p->cfg.power_iters; ++it) {
    {
      Span sp(p, RCP_KT_PROJECT, mode);
      RCP_TRY(launch_project_f32(T, v, l, p->Y, W, ng, s));
    }
    {
      Span sp(p, RCP_KT_APPLY, mode);
      RCP_TRY(launch_sketch_f32(T, v, l, 0, 0, W, nsplit, p->part, nullptr, s));
    }
    RCP_TRY(launch_reduce(p->part, nsplit, ny, p->Y, p->tmp, p->tmp_elems, s));
    RCP_TRY(launch_cholqr(p->Y, v.I, l, p->G, p->Rinv, p->dstate, s,
                          it == p->cfg.power_iters - 1, ns));
  }
  return RCP_OK;
}

}  // namespace

extern "C" {

rcp_status rcp_sketch(rcp_plan_t p, const void* X, int32_t mode, double* Q_out) {
  if (!valid_plan(p) || mode < 1 || mode > p->N) return RCP_EINVAL;
  if ((mode == 1 || (p->cfg.flags & RCP_FLAG_INDEPENDENT)) && !X) return RCP_EINVAL;
  if (mode == 1) {
    p->sketched = p->compressed = 0;  // a new decomposition starts at mode 1
  } else if (p->compressed != mode - 1) {
    return RCP_EORDER;
  }
  if (check_device(p) != RCP_OK) return RCP_ECUDA;
  cudaStream_t s = p->stream;
  const int n0 = mode - 1;
  const int64_t ny = p->view[n0].I * p->l[n0];
  if (mode == 1) {
    RCP_TRY(cudaMemsetAsync(p->dstate, 0, sizeof(DevState), s));
    p->als_done = false;
  }
  if (mode_skipped(&p->cfg, n0)) {
    // an uncompressed mode (the remark after Algorithm 1): Q_n = I, and |X|^2,
    // which the mode-1 sketch otherwise accumulates, from its own pass
    RCP_TRY(launch_identity(p->Y, p->view[n0].I, s));
    if (mode == 1) {
      const int64_t nx = p->view[0].I * p->view[0].J;
      RCP_TRY(launch_sumsq_any(X, p->cfg.in_dtype, nx, p->normpart, 64, &p->dstate->norm_x2, s));
    }
  } else {
    const rcp_status st =
        p->prec == RCP_PREC_MIXED ? sketch_mixed(p, X, mode) : sketch_f64(p, X, mode);
    if (st != RCP_OK) return st;
  }
  RCP_TRY(cudaMemcpyAsync(p->Q[n0], p->Y, sizeof(double) * ny, cudaMemcpyDeviceToDevice, s));
  if (Q_out)
    RCP_TRY(cudaMemcpyAsync(Q_out, p->Y, sizeof(double) * ny, cudaMemcpyDeviceToDevice, s));
  p->sketched = mode;
  return RCP_OK;
}

rcp_status rcp_compress(rcp_plan_t p, const void* X, int32_t mode) {
  if (!valid_plan(p) || mode < 1 || mode > p->N) return RCP_EINVAL;
  if (mode == 1 && !X) return RCP_EINVAL;
  if (p->sketched != mode || p->compressed != mode - 1) return RCP_EORDER;
  if (check_device(p) != RCP_OK) return RCP_ECUDA;
  const int n0 = mode - 1;
  const ModeView& v = p->view[n0];
  if (mode_skipped(&p->cfg, n0)) {
    // T_{n+1} = T_n: the working tensor moves to the next buffer unchanged
    int dt = 0;
    const void* T = p->prec == RCP_PREC_MIXED ? (mode == 1 ? X : p->bufT[(mode - 2) % 2])
                                              : mode_input(p, X, mode, &dt);
    const int64_t ne = v.I * v.J;
    void* out = mode_output(p, mode);
    if (p->prec != RCP_PREC_MIXED && dt == RCP_DTYPE_F32) {
      RCP_TRY(launch_to_f64(T, RCP_DTYPE_F32, ne, (double*)out, p->stream));
    } else {
      RCP_TRY(cudaMemcpyAsync(out, T, (size_t)ne * p->work_elem, cudaMemcpyDeviceToDevice,
                              p->stream));
    }
  } else if (p->prec == RCP_PREC_MIXED) {
    const float* T = (const float*)(mode == 1 ? X : p->bufT[(mode - 2) % 2]);
    float* out = (float*)mode_output(p, mode);
    Span sp(p, RCP_KT_TTM, mode);
    if (mode == 1 && p->tc1) {
      RCP_TRY(launch_q_to_qt32(p->Q[0], v.I, p->l[0], p->QT32, p->stream));
      RCP_TRY(launch_tc_cols(T, v.I, v.J, p->l[0], p->QT32, out, true, p->dstate,
                             tc_cols_grid(v.J, p->nsm), p->stream, tc_tma_ok(T), false));
    } else {
      RCP_TRY(launch_project_f32(T, v, p->l[n0], p->Q[n0], out, project_grid(v, p->nsm), p->stream));
    }
  } else {
    int dt = 0;
    const void* T = mode_input(p, X, mode, &dt);
    Span sp(p, RCP_KT_TTM, mode);
    RCP_TRY(launch_project_f64(T, dt, v, p->l[n0], p->Q[n0], mode_output(p, mode), nullptr,
                               project_grid(v, p->nsm), p->stream));
  }
  p->compressed = mode;
  if (mode == p->N) {
    if (p->prec == RCP_PREC_MIXED) {
      RCP_TRY(launch_to_f64(mode_output(p, mode), RCP_DTYPE_F32, p->core_elems, p->Bcore_own,
                            p->stream));
      p->Bcore64 = p->Bcore_own;
    } else {
      p->Bcore64 = mode_output(p, mode);
    }
  }
  return RCP_OK;
}

rcp_status rcp_als_init(rcp_plan_t p, const double* const* At_dev) {
  if (!valid_plan(p) || !At_dev) return RCP_EINVAL;
  for (int n = 1; n < p->N; ++n)
    if (!At_dev[n]) return RCP_EINVAL;
  if (check_device(p) != RCP_OK) return RCP_ECUDA;
  for (int n = 1; n < p->N; ++n)
    RCP_TRY(cudaMemcpyAsync(p->At[n], At_dev[n], sizeof(double) * p->l[n] * p->R,
                            cudaMemcpyDeviceToDevice, p->stream));
  p->user_init = true;
  return RCP_OK;
}

static rcp_status read_state(rcp_plan_t p, DevState* h) {
  if (cudaMemcpyAsync(h, p->dstate, sizeof(DevState), cudaMemcpyDeviceToHost, p->stream) !=
      cudaSuccess)
    return RCP_ECUDA;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return RCP_ECUDA;
  return RCP_OK;
}

rcp_status rcp_als(rcp_plan_t p, double* lambda_host, double* fit_host, int32_t* iters_host) {
  if (!valid_plan(p)) return RCP_EINVAL;
  if (p->compressed != p->N) return RCP_EORDER;
  if (check_device(p) != RCP_OK) return RCP_ECUDA;
  cudaStream_t s = p->stream;
  {
    Span sp(p, RCP_KT_ALS, 0);
    const bool f32 = p->prec == RCP_PREC_MIXED;
    const int* init_dev = nullptr;  // device word chosen by the learned warm start
    if (p->cfg.init == RCP_INIT_EIG && !p->user_init) {
      // Algorithm 2 step 2: eigenvectors of B_(n) B_(n)^T as the initial factors
      RCP_TRY(launch_eig_init(p, p->Bcore64, p->tmp, s));
      p->user_init = true;
    } else if (p->cfg.init == RCP_INIT_LEARNED && !p->user_init) {
      // the warm-start network's factors, or the seeded start where it has none
      const rcp_status ws = plan_ws_enqueue(p, &init_dev);
      if (ws != RCP_OK) return ws;
    }
    if (p->cfg.solver == RCP_SOLVER_BCD) {
      // Algorithm 3: successive rank-one deflation (one CTA, every component in one launch)
      const void* B = f32 ? (const void*)mode_output(p, p->N) : (const void*)p->Bcore64;
      RCP_TRY(launch_bcd(p, B, f32, p->part, init_dev, s));
    } else if (f32 && als_cluster_fits(p)) {
      // small core: one thread-block cluster runs every sweep
      RCP_TRY(launch_als_cluster(p, (const float*)mode_output(p, p->N), init_dev, s));
    } else if (als_persistent_fits(p, f32)) {
      // one cooperative kernel runs every sweep (FP32 MTTKRP in the mixed form)
      RCP_TRY(cudaMemsetAsync(p->bar, 0, 4 * sizeof(unsigned), s));
      RCP_TRY(cudaMemsetAsync(p->abort_flag, 0, 4 * sizeof(int), s));
      const void* B = f32 ? (const void*)mode_output(p, p->N) : (const void*)p->Bcore64;
      RCP_TRY(launch_als_persistent(p, B, f32, init_dev, s));
    } else {
      RCP_TRY(launch_sumsq(p->Bcore64, p->core_elems, p->normpart, 64, &p->dstate->norm_b2, s));
      RCP_TRY(launch_als_init(p, s));
      for (int it = 0; it < p->cfg.max_iters; ++it)
        for (int n0 = 0; n0 < p->N; ++n0) RCP_TRY(launch_als_sweep(p, n0, s));
    }
    p->user_init = false;
  }
  p->als_done = true;
  if (lambda_host || fit_host || iters_host) {
    if (lambda_host)
      RCP_TRY(cudaMemcpyAsync(lambda_host, p->lam, sizeof(double) * p->R, cudaMemcpyDeviceToHost, s));
    DevState h;
    if (read_state(p, &h) != RCP_OK) return RCP_ECUDA;
    if (fit_host) *fit_host = h.fit;
    if (iters_host) *iters_host = h.als_iters;
    if (h.status) return (rcp_status)h.status;
    if (h.als_done == 2 && p->cfg.tol > 0.0) return RCP_ENOTCONV;
  }
  return RCP_OK;
}

rcp_status rcp_project(rcp_plan_t p, double* const* A_dev, double* lambda_dev) {
  if (!valid_plan(p) || !A_dev || !lambda_dev) return RCP_EINVAL;
  for (int n = 0; n < p->N; ++n)
    if (!A_dev[n]) return RCP_EINVAL;
  if (!p->als_done) return RCP_EORDER;
  if (check_device(p) != RCP_OK) return RCP_ECUDA;
  RCP_TRY(launch_backproject(p, A_dev, lambda_dev, p->stream));
  return RCP_OK;
}

rcp_status rcp_decompose(rcp_plan_t p, const void* X, double* const* A_dev, double* lambda_dev) {
  if (!valid_plan(p) || !X || !A_dev || !lambda_dev) return RCP_EINVAL;
  for (int n = 0; n < p->N; ++n)
    if (!A_dev[n]) return RCP_EINVAL;
  p->sketched = p->compressed = 0;
  p->als_done = false;
  for (int mode = 1; mode <= p->N; ++mode) {
    rcp_status st = rcp_sketch(p, X, mode, nullptr);
    if (st != RCP_OK) return st;
    st = rcp_compress(p, X, mode);
    if (st != RCP_OK) return st;
  }
  rcp_status st = rcp_als(p, nullptr, nullptr, nullptr);
  if (st != RCP_OK) return st;
  return rcp_project(p, A_dev, lambda_dev);
}

rcp_status rcp_result_get(rcp_plan_t p, rcp_result* out) {
  if (!valid_plan(p)) return RCP_EINVAL;
  if (check_device(p) != RCP_OK) return RCP_ECUDA;
  DevState h;
  if (read_state(p, &h) != RCP_OK) return RCP_ECUDA;
  if (out) {
    memset(out, 0, sizeof(*out));
    out->fit = h.fit;
    out->iters = h.als_iters;
    out->info = h.info;
    out->norm_x2 = h.norm_x2;
    out->norm_b2 = h.norm_b2;
    const double r2 = h.norm_x2 - h.fit * h.norm_b2;
    out->rel_err = h.norm_x2 > 0.0 ? sqrt(std::max(r2, 0.0) / h.norm_x2) : 0.0;
    out->device_status = h.status;
    for (int n = 0; n < p->N; ++n) out->widths[n] = p->l[n];
  }
  return (rcp_status)h.status;
}

rcp_status rcp_decompose_host(rcp_plan_t p, const void* X_host, double* const* A_host,
                              double* lambda_host, rcp_result* res) {
  if (!valid_plan(p) || !X_host || !A_host || !lambda_host) return RCP_EINVAL;
  if (!(p->cfg.flags & RCP_FLAG_HOST_STAGING) || !p->X_stage) return RCP_EINVAL;
  for (int n = 0; n < p->N; ++n)
    if (!A_host[n]) return RCP_EINVAL;
  if (check_device(p) != RCP_OK) return RCP_ECUDA;
  cudaStream_t s = p->stream;
  int64_t nx = 1;
  for (int n = 0; n < p->N; ++n) nx *= p->dims[n];
  const size_t bytes = (size_t)nx * (p->cfg.in_dtype == RCP_DTYPE_F32 ? 4 : 8);
  RCP_TRY(cudaMemcpyAsync(p->X_stage, X_host, bytes, cudaMemcpyHostToDevice, s));
  rcp_status st = rcp_decompose(p, p->X_stage, p->A_stage, p->lam_stage);
  if (st != RCP_OK) return st;
  for (int n = 0; n < p->N; ++n)
    RCP_TRY(cudaMemcpyAsync(A_host[n], p->A_stage[n], sizeof(double) * p->dims[n] * p->R,
                            cudaMemcpyDeviceToHost, s));
  RCP_TRY(cudaMemcpyAsync(lambda_host, p->lam_stage, sizeof(double) * p->R, cudaMemcpyDeviceToHost, s));
  return rcp_result_get(p, res);
}

rcp_status rcp_get_core(rcp_plan_t p, double* B_dev) {
  if (!valid_plan(p) || !B_dev) return RCP_EINVAL;
  if (p->compressed != p->N) return RCP_EORDER;
  if (check_device(p) != RCP_OK) return RCP_ECUDA;
  RCP_TRY(cudaMemcpyAsync(B_dev, p->Bcore64, sizeof(double) * p->core_elems,
                          cudaMemcpyDeviceToDevice, p->stream));
  return RCP_OK;
}

rcp_status rcp_get_compressed_factors(rcp_plan_t p, double* const* At_dev, double* lambda_dev) {
  if (!valid_plan(p) || !At_dev) return RCP_EINVAL;
  if (!p->als_done) return RCP_EORDER;
  if (check_device(p) != RCP_OK) return RCP_ECUDA;
  for (int n = 0; n < p->N; ++n)
    if (At_dev[n])
      RCP_TRY(cudaMemcpyAsync(At_dev[n], p->At[n], sizeof(double) * p->l[n] * p->R,
                              cudaMemcpyDeviceToDevice, p->stream));
  if (lambda_dev)
    RCP_TRY(cudaMemcpyAsync(lambda_dev, p->lam, sizeof(double) * p->R, cudaMemcpyDeviceToDevice,
                            p->stream));
  return RCP_OK;
}

rcp_status rcp_profile_enable(rcp_plan_t p, int32_t enable) {
  if (!valid_plan(p)) return RCP_EINVAL;
  if (check_device(p) != RCP_OK) return RCP_ECUDA;
  if (enable && !p->prof) {
    const int cap = 8192;
    p->prof = new (std::nothrow) rcp_plan_s::ProfRec[cap];
    if (!p->prof) return RCP_ENOMEM;
    for (int k = 0; k < cap; ++k) {
      if (cudaEventCreate(&p->prof[k].a) != cudaSuccess ||
          cudaEventCreate(&p->prof[k].b) != cudaSuccess)
        return RCP_ECUDA;
      p->prof_cap = k + 1;
    }
  }
  if (enable) {
    p->prof_n = 0;
    p->launch_base = launch_counter();
  }
  p->prof_on = enable != 0;
  return RCP_OK;
}

rcp_status rcp_profile_read(rcp_plan_t p, int32_t kind, int32_t mode, int64_t* launches,
                            double* total_ms) {
  if (!valid_plan(p) || kind < 0 || kind >= RCP_KT_COUNT) return RCP_EINVAL;
  if (check_device(p) != RCP_OK) return RCP_ECUDA;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return RCP_ECUDA;
  if (kind == RCP_KT_ALL) {
    if (launches) *launches = launch_counter() - p->launch_base;
    if (total_ms) *total_ms = 0.0;
    return RCP_OK;
  }
  int64_t cnt = 0;
  double ms = 0.0;
  for (int k = 0; k < p->prof_n; ++k) {
    const auto& r = p->prof[k];
    if (r.kind != kind || (mode != 0 && r.mode != mode)) continue;
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return RCP_ECUDA;
    ms += t;
    ++cnt;
  }
  if (launches) *launches = cnt;
  if (total_ms) *total_ms = ms;
  return RCP_OK;
}

rcp_status rcp_last_error(rcp_plan_t p, int32_t* device_status) {
  if (!valid_plan(p)) return RCP_EINVAL;
  if (check_device(p) != RCP_OK) return RCP_ECUDA;
  DevState h;
  if (read_state(p, &h) != RCP_OK) return RCP_ECUDA;
  if (device_status) *device_status = h.status;
  return (rcp_status)h.status;
}

}  // extern "C"

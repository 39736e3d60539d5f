// Internal declarations of the GB300 randomized-CP library.
//
// Notation follows the paper (arXiv 1703.09074, Section 3): T_n is the tensor
// entering mode n of Algorithm 1 (T_1 = X, T_{n+1} = T_n x_n Q_n^T).  In the
// Kolda layout T_n is viewed as a 3-index array (L_n, I_n, Rt_n) where
// L_n = l_1 ... l_{n-1} (already-compressed modes, fastest), I_n is the current
// mode and Rt_n = I_{n+1} ... I_N.  Column j of the unfolding T_(n) is
// j = a + L_n b, and element (a, i, b) sits at a + L_n (i + I_n b).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rcp.h"

namespace rcp {

constexpr int kMaxN = RCP_MAX_NDIM;
constexpr int kMaxL = RCP_MAX_L;

// 3-index view of the working tensor of one mode.
struct ModeView {
  int64_t L, I, Rt, J;  // J = L * Rt
};

// Dims of every mode of the tensor that ALS sees, for Khatri-Rao row indexing.
struct KrDims {
  int N;
  int n;             // 0-based mode being updated
  int dims[kMaxN];   // l_1..l_N
  const double* A[kMaxN];  // factor matrices, l_m x R column-major
};

// Device-side scalars of one plan.
struct DevState {
  int status;          // rcp_status recorded on the device
  int info;            // RCP_INFO_* bits
  int extra_round;     // set when a QR needed the shifted fallback (one more CholQR round)
  int als_done;        // ALS converged or hit the cap
  int als_iters;       // sweeps run
  int chol32_fail;     // the FP32 Cholesky of a CholeskyQR round fell back to FP64
  double norm_x2;
  double norm_b2;
  double fit;
  double fit_prev;
  double ip;           // <Bhat, B> of the last sweep
};

struct Workspace;

}  // namespace rcp

struct rcp_plan_ws_s;

struct rcp_plan_s {
  rcp_config cfg;
  cudaStream_t stream;
  int device;
  int N;
  int R;
  int prec;            // rcp_precision
  int64_t dims[rcp::kMaxN];
  int l[rcp::kMaxN];
  rcp::ModeView view[rcp::kMaxN];
  rcp::ModeView xview[rcp::kMaxN];   // mode n of the input X itself (independent sketches)
  int64_t core_elems;  // l_1 ... l_N
  int nsm;

  // working tensors: T_{n+1} / W alternate between two buffers
  void* bufT[2];
  int64_t bufT_elems;
  int work_elem;       // 8 (FP64 path) or 4 (mixed path)

  double* Q[rcp::kMaxN];     // Q_n, I_n x l_n
  double* Y;                 // current sketch, I_max x kMaxL
  double* Y2;                // second buffer for the QR rounds
  double* part;              // split partials
  int64_t part_elems;
  double* tmp;               // second-level reduction buffer
  int64_t tmp_elems;
  double* gpart;             // Gram partials of W
  int64_t gpart_elems;
  double* G;                 // l x l Gram
  double* Rinv;              // l x l inverse Cholesky factor
  double* RWinv;             // l x l inverse Cholesky factor of W's Gram
  double* normpart;          // |X|^2 partials
  int64_t normpart_elems;

  // ALS
  double* At[rcp::kMaxN];    // Atilde_n, l_n x R
  double* Gm[rcp::kMaxN];    // Gram of Atilde_n, R x R
  double* M;                 // MTTKRP result l_max x R
  double* lam;               // R
  double* Bcore64;           // FP64 copy of B for the FP64 ALS (points into bufT when FP64)
  double* Bcore_own;         // owned FP64 copy (mixed path)
  rcp::DevState* dstate;
  bool user_init;

  // state machine of Algorithm 1 / 2
  int sketched;    // last mode sketched (0 = none)
  int compressed;  // last mode compressed (0 = none)
  bool als_done;

  // persistent ALS: grid barrier words and abort flag
  unsigned* bar;
  int* abort_flag;

  // mixed-precision form
  bool tc1;                  // mode 1 runs on the tensor cores
  float* part32;             // FP32 split partials of the tensor-core row sweep
  int64_t part32_elems;
  float* QT32;               // Q^T in FP32, padded to NP x Ipad

  // pivoted-LU normalisation (RCP_FLAG_LU_NORM): row flags, per-CTA candidates, pivot row
  uint8_t* lu_used;
  double* lu_cval;
  int64_t* lu_cidx;
  double* lu_prow;

  // learned warm start of the single-tensor path (rcp_set_warm_start)
  rcp_plan_ws_s* ws;
  float* als_S;   // contracted core of the dimension-tree MTTKRP (mixed form, large cores)

  // host staging (rcp_decompose_host)
  void* X_stage;
  double* A_stage[rcp::kMaxN];
  double* lam_stage;

  // profiling: CUDA events around sweep launches, and the launch count
  struct ProfRec {
    int kind, mode;
    cudaEvent_t a, b;
  };
  ProfRec* prof;
  int prof_cap, prof_n;
  bool prof_on;
  int64_t launch_base;
};

namespace rcp {

// ---------------------------------------------------------------- Philox4x32-10
// Salmon et al., SC'11: ten rounds of two 32x32->64 multiplies, Weyl key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ uint4 philox_words(uint64_t seed, uint32_t stream, uint32_t purpose,
                                              uint64_t g) {
  return philox4x32_10(make_uint4((uint32_t)g, (uint32_t)(g >> 32), stream, purpose),
                       make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// FP64 Box-Muller pair for counter g: u1 in (0, 1] from words (x, y), u2 in [0, 1) from (z, w).
__device__ __forceinline__ double2 normal_pair_f64(uint64_t seed, uint32_t stream,
                                                   uint32_t purpose, uint64_t g) {
  const uint4 x = philox_words(seed, stream, purpose, g);
  const double inv53 = 1.0 / 9007199254740992.0;
  const double ua = ((double)(x.x >> 5) * 67108864.0 + (double)(x.y >> 6)) * inv53;
  const double u2 = ((double)(x.z >> 5) * 67108864.0 + (double)(x.w >> 6)) * inv53;
  const double r = sqrt(-2.0 * log(1.0 - ua));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  return make_double2(r * c, r * s);
}

// Reduced-precision stream: four FP32 normals per counter (two Box-Muller pairs
// from 24-bit uniforms u1 = (w >> 8) + 1, u2 = w >> 8, scaled by 2^-24).
__device__ __forceinline__ float4 normal_quad_f32(uint64_t seed, uint32_t stream,
                                                  uint32_t purpose, uint64_t g) {
  const uint4 x = philox_words(seed, stream, purpose, g);
  const float s24 = 5.9604644775390625e-08f;
  const float ra = sqrtf(-2.0f * logf((float)((x.x >> 8) + 1u) * s24));
  const float rb = sqrtf(-2.0f * logf((float)((x.z >> 8) + 1u) * s24));
  float sa, ca, sb, cb;
  sincospif(2.0f * (float)(x.y >> 8) * s24, &sa, &ca);
  sincospif(2.0f * (float)(x.w >> 8) * s24, &sb, &cb);
  return make_float4(ra * ca, ra * sa, rb * cb, rb * sb);
}

// Kernels launched by this library on the calling host thread (profiling only).
int64_t& launch_counter();
inline void count_launches(int k) { launch_counter() += k; }

// Largest element count of an input tensor (product of its dims) accepted by the
// entry points: 2^48, far beyond any device memory, so that every product of
// dims formed from accepted sizes stays inside int64.
constexpr int64_t kMaxElems = 1LL << 48;

// *out = a * b when the product is at most kMaxElems (a, b >= 1); false otherwise.
inline bool mul_elems(int64_t a, int64_t b, int64_t* out) {
  int64_t r = 0;
  if (__builtin_mul_overflow(a, b, &r) || r > kMaxElems) return false;
  *out = r;
  return true;
}

constexpr uint32_t kPurposeSketch = 0;
constexpr uint32_t kPurposeAlsInit = 1;

__device__ __forceinline__ void set_status(DevState* st, int code) {
  atomicCAS(&st->status, 0, code);
}

// Arguments of one CP-ALS problem for the persistent ALS kernel (als_persistent.cu).
struct PersArgs {
  int N, R, G;
  int GA;                // CTAs that compute MTTKRP partials (GA <= G)
  int dims[kMaxN];       // l_1..l_N
  const void* B;         // TM, Kolda layout
  double* At[kMaxN];     // out: normalised factors (column-major l_n x R); in: user init
  double* lam;           // out: lambda
  double* part;          // G x (l_max x R) MTTKRP partials
  double* rows;          // l_max x R new factor rows (unnormalised)
  double* ipp;           // l_max partial inner products
  double* nbp;           // G partial |B|^2
  unsigned* bar;         // grid barrier: count, generation
  int* abort_flag;
  DevState* st;
  uint64_t seed;
  double tol;
  int max_iters;
  int user_init;
  int direct64;          // solve with the FP64 Cholesky factor only (no FP32 factor + refinement)
  long long budget;      // clock cycles per grid-barrier wait (0: the default)
  const int* user_init_dev;  // when set, a device word that replaces user_init
  float* S;              // mixed form, N >= 3, R <= 32: the contracted core of the
                         // dimension-tree MTTKRP (core / l_c x 32 floats), else null
};

// ---------------------------------------------------------------- batched form
struct BItem {
  int b;   // tensor index
  int bx;  // block coordinates within that tensor's grid
  int by;
};

struct BRowSweep {  // P = T_(n) V for one tensor (V = Omega_n or W)
  const float* T;
  ModeView v;
  int64_t rows_per_cta;
  int l;
  uint64_t seed;
  uint32_t sid;
  const float* W;
  int64_t jchunk;
  double* part;
  double* normpart;
  int gx;
};

struct BColSweep {  // W = T_(n)^T Q for one tensor, W in the Kolda layout of T_{n+1}
  const float* T;
  ModeView v;
  int l;
  const double* Q;
  float* W;
};
// Columns per block of the batched column sweep (its CTA width).  A column work
// item (b, bx, nb) covers tensor b's blocks bx, bx + nb, bx + 2 nb, ...
constexpr int kBColBlock = 256;

// ---------------------------------------------------------------- launchers
// Sweeps over the working tensor (sweeps_f64.cu).
cudaError_t launch_sketch_f64(const void* T, int in_dtype, ModeView v, int l, uint64_t seed,
                              uint32_t stream_id, const double* W, int nsplit, double* part,
                              double* normpart, cudaStream_t s);
cudaError_t launch_project_f64(const void* T, int in_dtype, ModeView v, int l, const double* Q,
                               double* W, double* gpart, int nblocks, cudaStream_t s);
cudaError_t launch_sketch_f32(const float* T, ModeView v, int l, uint64_t seed, uint32_t stream_id,
                              const float* W, int nsplit, double* part, double* normpart,
                              cudaStream_t s);
cudaError_t launch_project_f32(const float* T, ModeView v, int l, const double* Q, float* W,
                               int nblocks, cudaStream_t s);
cudaError_t launch_mttkrp_f64(const double* B, ModeView v, int R, const KrDims& kr, int nsplit,
                              double* part, cudaStream_t s);
int project_grid(const ModeView& v, int nsm);
cudaError_t launch_b_row_sweep(const BRowSweep* P, const BItem* items, int nitems, unsigned* counter,
                               int lmax, bool use_w, int depth, const float* const* xptrs,
                               int grid, cudaStream_t s);
cudaError_t launch_b_col_sweep(const BColSweep* P, const BItem* items, int nitems, unsigned* counter,
                               int lmax, bool mode1, const float* const* xptrs, int grid,
                               cudaStream_t s);
int sweep_rows_per_cta(int64_t I);
int sweep_row_blocks(int64_t I);
int sketch_splits(const ModeView& v, int nsm);

// Tensor-core mode-1 sweeps of the mixed-precision form (tc_sweeps.cu).
bool tc_mode1_supported(int64_t I, int l);
int tc_np(int l);
int64_t tc_ipad(int64_t I);
void tc_rows_split(int64_t I, int64_t J, int nsm, int* nsplit, int64_t* jchunk);
int tc_cols_grid(int64_t J, int nsm);
cudaError_t launch_tc_rows(const float* X, int64_t I, int64_t J, int l, uint64_t seed, uint32_t sid,
                           const float* WT, int nsplit, int64_t jchunk, float* part,
                           double* normpart, DevState* st, cudaStream_t s);
cudaError_t launch_tc_cols(const float* X, int64_t I, int64_t J, int l, const float* QT, float* out,
                           bool ttm, DevState* st, int grid, cudaStream_t s, bool tma, bool wsplit);
bool tc_tma_ok(const float* X);
void tc_rows_tma_shape(int64_t I, int64_t J, int nsm, int* nb, int* rb, int* ns, int64_t* cper);
cudaError_t launch_tc_rows_tma(const float* X, int64_t I, int64_t J, int l, const float* Wsplit,
                               float* part, DevState* st, int nsm, cudaStream_t s, int* nsplit);
cudaError_t launch_q_to_qt32(const double* Q, int64_t I, int l, float* QT, cudaStream_t s);
cudaError_t launch_reduce_f32(const float* part, int64_t nsplit, int64_t n, double* out,
                              cudaStream_t s);

// Small dense FP64 linear algebra (dense_f64.cu).
cudaError_t launch_reduce(const double* part, int64_t nsplit, int64_t n, double* out, double* tmp,
                          int64_t tmp_elems, cudaStream_t s);
cudaError_t launch_cholqr_round(const double* Yin, int64_t I, int l, double* G, double* Rinv,
                                double* Qout, DevState* st, int round, cudaStream_t s);
cudaError_t launch_gram_chol(const double* G, int l, double* Rinv, DevState* st, int allow_shift,
                             double shift_scale_rows, cudaStream_t s);
cudaError_t launch_trmm(const double* Y, int64_t I, int l, const double* Rinv, double* out,
                        const DevState* st, int only_if_extra, cudaStream_t s);
cudaError_t launch_norm_reduce(const double* part, int64_t n, double* dst, cudaStream_t s);

// ALS and recovery (als_f64.cu).
cudaError_t launch_als_init(rcp_plan_s* p, cudaStream_t s);
cudaError_t launch_als_sweep(rcp_plan_s* p, int mode0, cudaStream_t s);
cudaError_t launch_backproject(rcp_plan_s* p, double* const* A_dev, double* lambda_dev,
                               cudaStream_t s);
bool als_persistent_fits(const rcp_plan_s* p, bool f32);
bool als_cluster_fits(const rcp_plan_s* p);
cudaError_t launch_eig_init(rcp_plan_s* p, const double* B, double* gram, cudaStream_t s);
size_t cluster_batched_args(int N, int R, const int* l, int rmax, const float* B,
                            double* const* At, double* lam, float2* facdw, DevState* st,
                            uint64_t seed, double tol, int max_iters, const int* user_init_dev,
                            void* out);
size_t cluster_args_bytes();
cudaError_t prepare_als_cluster_batched(int rmax, size_t smem);
cudaError_t launch_als_cluster_batched(const void* dev_args, int count, int rmax, size_t smem,
                                       cudaStream_t s);
void plan_ws_free(rcp_plan_s* p);
rcp_status plan_ws_enqueue(rcp_plan_s* p, const int** flag_dev);
int64_t bcd_scratch_elems(const rcp_plan_s* p);
cudaError_t launch_bcd(rcp_plan_s* p, const void* B, bool f32, double* scratch,
                       const int* user_init_dev, cudaStream_t s);
cudaError_t launch_als_cluster(rcp_plan_s* p, const float* B, const int* user_init_dev,
                               cudaStream_t s);
cudaError_t launch_als_persistent(rcp_plan_s* p, const void* B, bool f32, const int* user_init_dev,
                                  cudaStream_t s);
cudaError_t launch_to_f64(const void* src, int src_dtype, int64_t n, double* dst, cudaStream_t s);
cudaError_t launch_sumsq_any(const void* x, int dtype, int64_t n, double* part, int nblocks,
                             double* dst, cudaStream_t s);
cudaError_t launch_identity(double* Q, int64_t I, cudaStream_t s);
cudaError_t launch_sumsq(const double* x, int64_t n, double* dst, cudaStream_t s);

}  // namespace rcp

// Internal declarations shared by the CUDA translation units of the hypercube
// queue solver.  Not part of the public ABI (see include/hq.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/hq.h"

#define HQ_MAXN 29
// Largest N for which the solver keeps the double-float table and iterates and the
// batched kernel's per-state lists (at N = 29 they would not fit beside the FP64 and FP32
// tables in the GPU's memory): above it the double-float precisions and batching are
// unavailable.
#define HQ_DF_MAXN 28
#define HQ_LO_BITS 10          // low-part width of the split rank tables
#define HQ_THREADS 256         // threads per CTA of the streaming kernels

// Work items of the sweep.  A rank block (hi, w) of layer n is the set of its states whose
// high part (bits >= L) is hi and whose low part has w busy units; it holds C(L, w)
// states at the consecutive ranks RH[hi][w] + RL[lo].  The low-part neighbours of its
// states are the whole blocks (hi, w-1) of layer n-1 and (hi, w+1) of layer n+1 (at most
// C(10, 5) = 252 states each); a high-part neighbour across unit L+j sits at rank
// RH[hi ^ 2^j][w] + RL[lo] of layer n -/+ 1, so consecutive states of a block have their
// high-part neighbours at consecutive ranks.  An item is a run of at most 32 consecutive
// states of one block, processed by one warp: uint4 {rank0, hi | w << 20 | (count-1) << 24,
// rank of block (hi, w-1) in layer n-1, rank of block (hi, w+1) in layer n+1}.
#define HQ_ITEM_HI_BITS 20
// Items of the direct sweep (hq_persist.cu): runs of at most HQ_SW_ITEM consecutive states
// of one rank block, 8 bytes: x = hi | w << 20 | (count-1) << 24, y = rank of the item's
// first state in layer n | n << 27 (ranks below 2^27: C(29, 14) = 7.8e7).  The sweep takes
// its high-part neighbour bases, its own block base and its low-part neighbour blocks
// from RH once per rank block.
#define HQ_SW_HI_BITS 20
#define HQ_SW_ITEM 32
#define HQ_MLP_UNIT_FEATURES 8  // per-unit features of an instance
#define HQ_MLP_FEATURES 9       // inputs of the warm-start network: unit features + n / N
#define HQ_MAX_BLOCK 252   // C(HQ_LO_BITS, HQ_LO_BITS / 2)
// Pull-form table layout: state-major.  The n entries of a state of layer n (busy slot s =
// s-th busy unit, increasing) are one record of HQ_TW(n) entries (n rounded up to 4, zero
// padded), so a record starts 16-byte aligned and loads as whole vectors; layer n's
// records start at toff[n], rank k's at toff[n] + k HQ_TW(n).
#define HQ_TW(n) (((n) + 3) & ~3)

// ---------------------------------------------------------------------------
// error plumbing (host)
// ---------------------------------------------------------------------------
void hq_set_error(const std::string& msg);
int hq_cuda_fail(cudaError_t e, const char* what, const char* file, int line);
void hq_count_launch(int64_t k = 1);

#define HQ_CUDA(call)                                                   \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess) return hq_cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define HQ_LAUNCHED()                                                   \
  do {                                                                  \
    cudaError_t e_ = cudaGetLastError();                                \
    if (e_ != cudaSuccess) return hq_cuda_fail(e_, "kernel launch", __FILE__, __LINE__); \
    hq_count_launch();                                                  \
  } while (0)

// ---------------------------------------------------------------------------
// double-float ("DF64") arithmetic: a value is hi + lo with two floats.
// All steps use round-to-nearest intrinsics so that the compiler cannot fuse
// them into FMAs (the error-free transforms rely on each rounding).
// TwoSum (Knuth) and TwoProduct via FMA are the classical error-free
// transforms of Dekker (1971) and Knuth (TAOCP vol. 2).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 df_fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return make_float2(s, e);
}
__device__ __forceinline__ float2 df_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return make_float2(s, e);
}
__device__ __forceinline__ float2 df_norm(float2 a) { return df_fast_two_sum(a.x, a.y); }
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  float2 s = df_two_sum(a.x, b.x);
  float e = __fadd_rn(s.y, __fadd_rn(a.y, b.y));
  return df_fast_two_sum(s.x, e);
}
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 df_sub(float2 a, float2 b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  float p = __fmul_rn(a.x, b.x);
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  return df_fast_two_sum(p, e);
}
// acc += a * b with acc kept as an unnormalised pair (value = acc.x + acc.y)
__device__ __forceinline__ void df_fma_acc(float2& acc, float2 a, float2 b) {
  float p = __fmul_rn(a.x, b.x);
  float pe = fmaf(a.x, b.x, -p);
  pe = fmaf(a.x, b.y, pe);
  pe = fmaf(a.y, b.x, pe);
  float s = __fadd_rn(acc.x, p);
  float bb = __fsub_rn(s, acc.x);
  float err = __fadd_rn(__fsub_rn(acc.x, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  acc.x = s;
  acc.y = __fadd_rn(acc.y, __fadd_rn(err, pe));
}
__device__ __forceinline__ float2 df_from_double(double x) {
  float h = __double2float_rn(x);
  float l = __double2float_rn(x - (double)h);
  return make_float2(h, l);
}
__device__ __forceinline__ double df_to_double(float2 a) { return (double)a.x + (double)a.y; }

// ---------------------------------------------------------------------------
// arithmetic policies of the sweep: storage type V::T, accumulator V::A
// ---------------------------------------------------------------------------
struct PolF64 {
  typedef double T;
  static constexpr int kind = HQ_PREC_FP64;
  __device__ static T zero() { return 0.0; }
  __device__ static void fma_acc(T& acc, T a, T b) { acc = fma(a, b, acc); }
  __device__ static T mul(T a, T b) { return a * b; }
  __device__ static T add(T a, T b) { return a + b; }
  __device__ static T sub(T a, T b) { return a - b; }
  __device__ static T norm(T a) { return a; }
  __device__ static T from_d(double x) { return x; }
  __device__ static double to_d(T a) { return a; }
  __device__ static float absdiff(T a, T b) { return (float)fabs(a - b); }
  __device__ static T shfl_xor(T a, int m) { return __shfl_xor_sync(0xffffffffu, a, m); }
};
struct PolDF {
  typedef float2 T;
  static constexpr int kind = HQ_PREC_DF64;
  __device__ static T zero() { return make_float2(0.f, 0.f); }
  __device__ static void fma_acc(T& acc, T a, T b) { df_fma_acc(acc, a, b); }
  __device__ static T mul(T a, T b) { return df_mul(a, b); }
  __device__ static T add(T a, T b) { return df_add(a, b); }
  __device__ static T sub(T a, T b) { return df_sub(a, b); }
  __device__ static T norm(T a) { return df_norm(a); }
  __device__ static T from_d(double x) { return df_from_double(x); }
  __device__ static double to_d(T a) { return df_to_double(a); }
  // |a - b| for nearby values: the hi difference is exact (Sterbenz), lo adds the rest
  __device__ static float absdiff(T a, T b) {
    return fabsf(__fadd_rn(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y)));
  }
  __device__ static T shfl_xor(T a, int m) {
    return make_float2(__shfl_xor_sync(0xffffffffu, a.x, m), __shfl_xor_sync(0xffffffffu, a.y, m));
  }
};
struct PolF32 {
  typedef float T;
  static constexpr int kind = HQ_PREC_FP32;
  __device__ static T zero() { return 0.f; }
  __device__ static void fma_acc(T& acc, T a, T b) { acc = fmaf(a, b, acc); }
  __device__ static T mul(T a, T b) { return a * b; }
  __device__ static T add(T a, T b) { return a + b; }
  __device__ static T sub(T a, T b) { return a - b; }
  __device__ static T norm(T a) { return a; }
  __device__ static T from_d(double x) { return (float)x; }
  __device__ static double to_d(T a) { return (double)a; }
  __device__ static float absdiff(T a, T b) { return fabsf(a - b); }
  __device__ static T shfl_xor(T a, int m) { return __shfl_xor_sync(0xffffffffu, a, m); }
};

// ---------------------------------------------------------------------------
// device-resident scalars of the iteration (all FP64)
// ---------------------------------------------------------------------------
struct DevScalars {
  double lam_n[HQ_MAXN + 1];   // lambda^k(n)   (Eq. 13)
  double mu_n[HQ_MAXN + 1];    // mu^k(n)       (Eq. 14, closed-form inner limit)
  double c1[HQ_MAXN + 1];      // alpha mu* of the last update of layer n
  double c2[HQ_MAXN + 1];      // beta of the last update of layer n
  double step_layer[HQ_MAXN + 1];
  double sum_layer[HQ_MAXN + 1];
  double step;                 // max_n step_layer[n] of the last sweep
  double step_prev;
  int sweeps;                  // sweeps done on the device
  int flags;                   // bit 0: non-finite value seen
  unsigned ticket[4];          // last-block tickets
  unsigned bar_count;          // grid barrier of the persistent sweep kernel: arrivals
  double red[16];              // results of whole-vector reductions
  double lsum[HQ_MAXN + 1];    // sum_m p_n(B_m) per layer (whole-vector pass)
  double lmu[HQ_MAXN + 1];     // sum_m mu_m p_n(B_m) per layer
  long long lsum_q[HQ_MAXN + 1];  // the same two sums in 64-bit fixed point (exact adds)
  long long lmu_q[HQ_MAXN + 1];
  double res_num[HQ_MAXN + 1]; // max_m |out_m - in_m| per layer (residual)
  double res_den[HQ_MAXN + 1]; // max_m out_m per layer
  double fac[HQ_MAXN + 1];     // P{B} = fac[w(B)] * p_w(B) after the birth-death step
  double lam;                  // lambda = sum_j lambda_j of the loaded instance
  // refinement (correction sweeps against an FP64 base p0): the base's layer scalars
  // c1^0(n), c2^0(n) and its per-layer sums {sum mu A0, sum mu B0, sum A0, sum B0}
  double ir_c1[HQ_MAXN + 1];
  double ir_c2[HQ_MAXN + 1];
  double ir_sum[4][HQ_MAXN + 1];  // the base's layer sums, in the order of ls
  // the direct sweep's layer sums of the current iterate (FP64): ls[0][n] = sum p,
  // ls[1][n] = sum mu_m p, ls[2][n] = sum w''(m) p, ls[3][n] = sum v''(m) p, with the
  // per-state weights w'' (upward) and v'' (downward) of hq_build_weights; correction
  // sweeps: the full sums of p0 + e (ir_sum holds the base's)
  double ls[4][HQ_MAXN + 1];
  unsigned long long t_start;  // %globaltimer at the start of the last sweep launch (ns)
  unsigned long long t_phase[64];  // %globaltimer at the release of phase g of that launch
};

// rank of a state from the split tables (see hq_layout.cu)
__device__ __forceinline__ uint32_t hq_rank_split(const uint32_t* s_RL, const uint32_t* RH, int L,
                                                  uint32_t x) {
  uint32_t lo = x & ((1u << L) - 1u);
  return s_RL[lo] + __ldg(RH + (size_t)(x >> L) * (L + 1) + __popc(lo));
}

// typed streaming / read-only loads
__device__ __forceinline__ double ld_stream(const double* p) { return __ldcs(p); }
__device__ __forceinline__ float2 ld_stream(const float2* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float* p) { return __ldcs(p); }
__device__ __forceinline__ double ld_ro(const double* p) { return __ldg(p); }
__device__ __forceinline__ float2 ld_ro(const float2* p) { return __ldg(p); }
__device__ __forceinline__ float ld_ro(const float* p) { return __ldg(p); }

// per-precision vectors
struct PrecBufs {
  void* T = nullptr;   // pull-form table in this precision, toff layout
  void* r = nullptr;   // 1/(lambda + mu_m), layer-ranked
  void* p = nullptr;   // conditional p, layer-ranked
  void* nu = nullptr;  // nu_i in this precision (N)
};

struct hq_solver {
  int N = 0, J = 0, mode = 0, C = 0;
  int dev = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int64_t S = 0;
  int64_t off[HQ_MAXN + 2];    // layer n states start at off[n] (padded to 32 entries)
  int64_t toff[HQ_MAXN + 2];   // table entries of layer n start at toff[n]
  int64_t lsize[HQ_MAXN + 1];  // C(N, n)
  int64_t lpad[HQ_MAXN + 1];   // C(N, n) rounded up to 32: layer stride
  int64_t tw[HQ_MAXN + 1];     // table record width of layer n, HQ_TW(n)
  int64_t Sp = 0;              // padded length of the layer-ranked vectors
  int64_t tentries = 0;        // padded table length
  int64_t ab_half_bytes = 0;   // one half of the (A, B) double buffer
  int L = 0, H = 0;            // split rank tables: low L bits, high H bits
  int64_t max_layer = 0;
  int64_t dev_bytes = 0;
  double lam = 0, nu_sum = 0;
  bool loaded = false, solved = false;
  int cur_prec = -1;           // precision holding the current iterate
  double omega = 1.0;          // over-relaxation of the finalised layers (1: Algorithm 1)
  // every change of the iterate bumps it_version; res_version is the version whose FP64
  // residual, layer law and summary the last residual pass computed
  uint64_t it_version = 1, res_version = 0;

  // N-dependent layout
  uint32_t* masks = nullptr;   // S, layer-ranked state masks
  uint32_t* RL = nullptr;      // 2^L
  uint32_t* RH = nullptr;      // 2^H x (L+1)
  uint32_t* lidx = nullptr;    // 3 x Sp: low-part neighbour positions (4 bytes a word)
  uint4* items = nullptr;      // work items of the batched sweep, layer by layer
  int ifirst[HQ_MAXN + 2];     // items of layer n: [ifirst[n], ifirst[n+1])
  // direct sweep: items of each sweep order, phase by phase ([order][pfirst[ph], pfirst[ph+1]))
  uint2* sitems[2] = {nullptr, nullptr};
  int* sblocks[2] = {nullptr, nullptr};  // first item of each rank block (and the end)
  int* sperm[2] = {nullptr, nullptr};    // per phase, its blocks by decreasing cost
  int spbfirst[2][HQ_MAXN + 2];  // rank blocks of phase ph: [spbfirst[ph], spbfirst[ph+1])
  int snph[2] = {0, 0};        // phases per sweep of each order
  int order = HQ_ORDER_ASCENDING;  // sweep order of the solve in progress
  unsigned spin_limit = 0;     // bounded waits of the sweep kernel (0: the default)
  int dbg_skip_cta = -1;       // fault injection: this CTA skips one barrier arrival
  cudaEvent_t kev[2] = {nullptr, nullptr};  // brackets of each sweep launch in hq_solve
  bool df_ready = false;       // the double-float table matches the current instance
  void* wv64 = nullptr;        // per-state weights (w'', v'') in FP64 (double2, layer-ranked)
  void* wv32 = nullptr;        // the same in FP32 (float2)
  double* mutab = nullptr;     // mu of a low part (2^L entries), then of a high part (2^H)
  // instance
  double* lam_j = nullptr;     // J
  double* nu = nullptr;        // N
  int32_t* pref = nullptr;     // J x N
  uint32_t* pre = nullptr;     // J x N: units ranked before u by node j
  double* zeta = nullptr;      // N x 2^(N-1) scratch of the subset-sum transforms
  PrecBufs b64, bdf, b32;
  void* ab = nullptr;          // (A, B) pairs of two consecutive layers (double buffer)
  double* partials = nullptr;  // block partials of the reductions
  int64_t partials_len = 0;
  DevScalars* sc = nullptr;
  DevScalars* hsc = nullptr;   // pinned host mirror
  int* dflag = nullptr;        // device validation flag
  // results
  double* P = nullptr;         // S, y-order
  double* pn = nullptr;        // N + C + 1
  double* rho = nullptr;       // N
  double* R = nullptr;         // J x N
  double* W = nullptr;         // N x J
  double* summary = nullptr;   // 8
  double* pcond = nullptr;     // S, y-order conditional (normalised)
  double ms_table = 0;
  // learned warm start: attached model (borrowed) and scratch
  hq_mlp* mlp = nullptr;
  // refinement: the FP64 base p0 (layer-ranked, Sp) and 6 x Sp FP32 per-state base terms
  // {rho0, A0, B0, G_rho, G_A, G_B}; the iterate of the correction sweeps is e = p - p0,
  // held in b32.p; ir_part: 4 FP64 partial sums per work item of the base pass
  double* ir_base = nullptr;
  float* ir = nullptr;         // 3 x Sp FP32 base terms {rho0, A0, B0} of the correction sweeps
  double* ir_part = nullptr;
  float* wfeat = nullptr;      // N (N-1) rows x HQ_MLP_FEATURES: (layer n, unit i) pairs
  float* wy = nullptr;         // N (N-1) predictions (logit q_i(n))
  double* wlx = nullptr;       // log x_i(n) [HQ_MAXN^2], log e_n [HQ_MAXN + 1]
};

// ---------------------------------------------------------------------------
// kernels / launchers implemented across translation units
// ---------------------------------------------------------------------------
double hq_binom(int n, int k);

// layout (hq_layout.cu)
int hq_build_layout(hq_solver* h);
int hq_validate_device(hq_solver* h);
int hq_build_rates(hq_solver* h);  // r_m in all precisions

// learned warm start (hq_mlp.cu)
int hq_mlp_predict_dev(hq_mlp* m, const float* X, int B, float* y_dev, cudaStream_t s);
int hq_mlp_features_dev(hq_solver* h, float* X);
int hq_mlp_warm_start(hq_solver* h, hq_mlp* m, double* P, double* rho);
int hq_product_warm_start(hq_solver* h, double* P);  // the analytic control (HQ_WARM_PRODUCT)

// refinement (hq_refine.cu): correction sweeps run as sweep precision HQ_PREC_IRC on
// the FP32 buffers; hq_ir_begin sets up a base from the iterate held in precision
// `from` (from == HQ_PREC_IRC: re-base on p0 + e), hq_ir_assemble writes p0 + e to b64.p
#define HQ_PREC_IRC 16
int hq_ir_begin(hq_solver* h, int from);
int hq_ir_assemble(hq_solver* h);
int hq_base_pass(hq_solver* h);  // base scalars c^0 and the FP32 base terms (hq_persist.cu)
int hq_residual_fused(hq_solver* h);  // residual maxima of layers 1..N-1 into res_num/res_den[1]

// work items and low-part positions of the sweep (hq_items.cu)
int hq_item_list(int N, std::vector<uint4>& items, int* ifirst);  // host list, layer by layer
// direct-sweep items of one order, phase by phase, and their rank blocks: block b holds
// items [blocks[b], blocks[b + 1]); phase ph holds blocks [pbfirst[ph], pbfirst[ph + 1])
int hq_sweep_item_list(int N, int order, std::vector<uint2>& items, std::vector<int>& blocks, int* pbfirst,
                       int* nphases);
int hq_build_items(hq_solver* h);     // at hq_create, after the layout
int hq_build_weights(hq_solver* h);   // at hq_load, after the table and r (hq_persist.cu)
int hq_iter_sums(hq_solver* h, int prec, const void* p, double* dst);  // 4 layer sums -> dst[4][N+1] (device)
// the double-float copy of the table, made on the first use of a double-float precision
// after each hq_load (the FP32 copy is written with the FP64 table)
int hq_ensure_df(hq_solver* h);

// table (hq_table.cu)
int hq_build_table(hq_solver* h);
int hq_zeta_subset(hq_solver* h, long long* buf, int bits, int count, bool superset);  // 64-bit fixed point

// sweep (hq_sweep.cu)
int hq_init_iterate(hq_solver* h, int prec, const double* warm_y, int warm_mem);
// sums = false: leave the sweep's layer sums alone (a converted copy for the residual)
int hq_convert_iterate(hq_solver* h, int from, int to, bool sums = true);
int hq_run_sweeps(hq_solver* h, int prec, int nsweeps, cudaEvent_t ev0, cudaEvent_t ev1);
PrecBufs& hq_bufs(hq_solver* h, int prec);

// results (hq_post.cu)
int hq_layer_sums(hq_solver* h, int prec);
int hq_finalize(hq_solver* h, int prec, bool full_outputs, double* residual_out);
int hq_compute_residual(hq_solver* h, double* residual_out);

// C ABI of the solver (include/hq.h): handle lifecycle, instance loading, the
// outer loop of Algorithm 1 with its convergence checks, and result getters.
#include <math.h>
#include <string.h>

#include <chrono>
#include <string>

#include "hq_internal.cuh"

static thread_local std::string g_last_error;
static thread_local int64_t g_launches = 0;

void hq_set_error(const std::string& msg) { g_last_error = msg; }

int hq_cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e) + " (" + file + ":" +
                 std::to_string(line) + ")";
  return e == cudaErrorMemoryAllocation ? HQ_ENOMEM : HQ_ECUDA;
}

void hq_count_launch(int64_t k) { g_launches += k; }

extern "C" int64_t hq_launch_count(int reset) {
  int64_t v = g_launches;
  if (reset) g_launches = 0;
  return v;
}

extern "C" const char* hq_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* hq_strerror(int code) {
  switch (code) {
    case HQ_OK: return "ok";
    case HQ_EINVAL: return "invalid argument or instance";
    case HQ_ENOMEM: return "device memory allocation failed";
    case HQ_EUNSTABLE: return "infinite queue is unstable (lambda >= sum nu)";
    case HQ_ENOTCONVERGED: return "tolerance not reached within max_sweeps";
    case HQ_EDIVERGED: return "iteration produced a non-finite or diverging iterate";
    case HQ_ETIMEOUT: return "a bounded device wait timed out";
    case HQ_ECUDA: return "CUDA runtime error";
    case HQ_ESTATE: return "call out of order";
    default: return "unknown status";
  }
}

extern "C" void hq_default_opts(hq_opts* o) {
  memset(o, 0, sizeof(*o));
  o->tol = 1e-10;
  o->tol_kind = HQ_TOL_RESIDUAL;
  o->max_sweeps = 100000;
  o->precision = HQ_PREC_FP32_DF64;
  o->check_every = 8;
  o->warm_start = HQ_WARM_NONE;
  o->warm_mem = HQ_HOST;
  o->warm_p = nullptr;
  o->fp32_stall = 0.9;
  o->omega = 1.0;
}

static void free_all(hq_solver* h) {
  void* ptrs[] = {h->masks, h->RL, h->RH, h->lam_j, h->nu, h->pref, h->pre, h->zeta,
                  h->lidx, h->items, h->wfeat, h->wy, h->wlx,
                  h->b64.T, h->b64.r, h->b64.p, h->b64.nu, h->bdf.T, h->bdf.r, h->bdf.p, h->bdf.nu,
                  h->b32.T, h->b32.r, h->b32.p, h->b32.nu, h->ab, h->partials, h->sc, h->dflag,
                  h->P, h->pn, h->rho, h->R, h->W, h->summary, h->pcond, h->ir_base, h->ir, h->ir_part,
                  h->wv64, h->wv32, h->mutab, h->sitems[0], h->sitems[1], h->sblocks[0], h->sblocks[1],
                  h->sperm[0], h->sperm[1]};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->hsc) cudaFreeHost(h->hsc);
  for (cudaEvent_t& e : h->kev)
    if (e) cudaEventDestroy(e), e = nullptr;
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

template <class T>
static int dalloc(hq_solver* h, T** p, int64_t bytes) {
  if (bytes <= 0) bytes = 16;
  cudaError_t e = cudaMalloc((void**)p, (size_t)bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    hq_set_error("cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                 cudaGetErrorString(e));
    return HQ_ENOMEM;
  }
  h->dev_bytes += bytes;
  return HQ_OK;
}

#define HQ_TRY(x)            \
  do {                       \
    int rc_ = (x);           \
    if (rc_ != HQ_OK) {      \
      free_all(h);           \
      delete h;              \
      return rc_;            \
    }                        \
  } while (0)

extern "C" int hq_create(int N, int J, int mode, int capacity_C, void* stream, hq_solver** out) {
  if (!out) { hq_set_error("out is NULL"); return HQ_EINVAL; }
  *out = nullptr;
  if (N < 1 || N > HQ_MAXN) { hq_set_error("N must be in 1..29"); return HQ_EINVAL; }
  if (J < 1) { hq_set_error("J must be >= 1"); return HQ_EINVAL; }
  if (mode < HQ_LOSS || mode > HQ_INFINITE) { hq_set_error("mode must be 0, 1 or 2"); return HQ_EINVAL; }
  if (mode == HQ_FINITE && (capacity_C < 1 || capacity_C > (1 << 20))) {
    hq_set_error("finite buffer needs 1 <= C <= 2^20");
    return HQ_EINVAL;
  }
  hq_solver* h = new hq_solver();
  h->N = N;
  h->J = J;
  h->mode = mode;
  h->C = mode == HQ_FINITE ? capacity_C : 0;
  cudaGetDevice(&h->dev);
  h->stream = (cudaStream_t)stream;
  if (!h->stream) {
    // keep the solver's work off the legacy default stream: use a stream of our own
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete h;
      hq_set_error("cudaStreamCreateWithFlags failed");
      return HQ_ECUDA;
    }
    h->own_stream = true;
  }
  h->S = (int64_t)1 << N;
  h->off[0] = 0;
  h->toff[0] = 0;
  h->max_layer = 0;
  for (int n = 0; n <= N; n++) {
    // every layer (and every table row) starts on a 32-entry boundary, so bulk copies
    // of whole tiles start 16-byte aligned and may read up to 31 entries of padding
    h->lsize[n] = (int64_t)hq_binom(N, n);
    h->lpad[n] = (h->lsize[n] + 31) & ~(int64_t)31;
    h->off[n + 1] = h->off[n] + h->lpad[n];
    h->tw[n] = HQ_TW(n);
    h->toff[n + 1] = h->toff[n] + h->tw[n] * h->lpad[n];
    if (h->lpad[n] > h->max_layer) h->max_layer = h->lpad[n];
  }
  for (int n = N + 2; n < HQ_MAXN + 2; n++) {
    h->off[n] = h->off[N + 1];
    h->toff[n] = h->toff[N + 1];
  }
  h->tentries = h->toff[N + 1];
  h->Sp = h->off[N + 1];
  h->L = N < HQ_LO_BITS ? N : HQ_LO_BITS;
  h->H = N - h->L;
  const int64_t S = h->S, SP = h->Sp, TE = h->tentries, half = S / 2 > 0 ? S / 2 : 1;
  HQ_TRY(dalloc(h, &h->masks, SP * 4));
  HQ_TRY(dalloc(h, &h->RL, (int64_t)4 << h->L));
  HQ_TRY(dalloc(h, &h->RH, ((int64_t)4 << h->H) * (h->L + 1)));
  HQ_TRY(dalloc(h, &h->lam_j, (int64_t)J * 8));
  HQ_TRY(dalloc(h, &h->nu, (int64_t)N * 8));
  HQ_TRY(dalloc(h, &h->pref, (int64_t)J * N * 4));
  HQ_TRY(dalloc(h, &h->pre, (int64_t)J * N * 4));
  HQ_TRY(dalloc(h, &h->zeta, half * N * 8));
  HQ_TRY(dalloc(h, (double**)&h->b64.T, TE * 8));
  const bool df = N <= HQ_DF_MAXN;  // double-float table, iterates and batch lists
  if (df) HQ_TRY(dalloc(h, (float2**)&h->bdf.T, TE * 8));
  HQ_TRY(dalloc(h, (float**)&h->b32.T, TE * 4));
  if (df) HQ_TRY(dalloc(h, &h->lidx, SP * 12));
  HQ_TRY(dalloc(h, &h->wfeat, (int64_t)HQ_MAXN * HQ_MAXN * HQ_MLP_FEATURES * 4));
  HQ_TRY(dalloc(h, &h->wy, (int64_t)HQ_MAXN * HQ_MAXN * 4));
  HQ_TRY(dalloc(h, &h->wlx, ((int64_t)HQ_MAXN * HQ_MAXN + HQ_MAXN + 1) * 8));
  HQ_TRY(dalloc(h, (double**)&h->b64.r, SP * 8));
  if (df) HQ_TRY(dalloc(h, (float2**)&h->bdf.r, SP * 8));
  HQ_TRY(dalloc(h, (float**)&h->b32.r, SP * 4));
  HQ_TRY(dalloc(h, (double**)&h->b64.p, SP * 8));
  if (df) HQ_TRY(dalloc(h, (float2**)&h->bdf.p, SP * 8));
  HQ_TRY(dalloc(h, (float**)&h->b32.p, SP * 4));
  HQ_TRY(dalloc(h, &h->ir_base, SP * 8));
  HQ_TRY(dalloc(h, &h->ir, SP * 12));
  HQ_TRY(dalloc(h, (double2**)&h->wv64, SP * 16));
  HQ_TRY(dalloc(h, (float2**)&h->wv32, SP * 8));
  HQ_TRY(dalloc(h, &h->mutab, (((int64_t)1 << h->L) + ((int64_t)1 << h->H)) * 8));
  HQ_TRY(dalloc(h, (double**)&h->b64.nu, (int64_t)HQ_MAXN * 8));
  HQ_TRY(dalloc(h, (float2**)&h->bdf.nu, (int64_t)HQ_MAXN * 8));
  HQ_TRY(dalloc(h, (float**)&h->b32.nu, (int64_t)HQ_MAXN * 4));
  // the staging copies of the sweep read up to 15 bytes past a layer's last pair
  h->ab_half_bytes = h->max_layer * 16 + 256;
  HQ_TRY(dalloc(h, (double**)&h->ab, 2 * h->ab_half_bytes));
  // block partials of the reductions: the sweep kernel's [2][words][grid], the layer
  // sums' [warps][N+1][4] and the residual's per-block pairs
  int64_t blocks = (h->max_layer + HQ_THREADS - 1) / HQ_THREADS;
  h->partials_len = blocks * 2 > ((int64_t)1 << 20) ? blocks * 2 : ((int64_t)1 << 20);
  HQ_TRY(dalloc(h, &h->partials, h->partials_len * 8));
  HQ_TRY(dalloc(h, &h->sc, (int64_t)sizeof(DevScalars)));
  HQ_TRY(dalloc(h, &h->dflag, 16));
  HQ_TRY(dalloc(h, &h->P, S * 8));
  HQ_TRY(dalloc(h, &h->pcond, S * 8));
  HQ_TRY(dalloc(h, &h->pn, (int64_t)(N + h->C + 1) * 8));
  HQ_TRY(dalloc(h, &h->rho, (int64_t)N * 8));
  HQ_TRY(dalloc(h, &h->R, (int64_t)J * N * 8));
  HQ_TRY(dalloc(h, &h->W, (int64_t)J * N * 8));
  HQ_TRY(dalloc(h, &h->summary, 16 * 8));
  if (cudaMallocHost((void**)&h->hsc, sizeof(DevScalars)) != cudaSuccess) {
    cudaGetLastError();
    free_all(h);
    delete h;
    hq_set_error("cudaMallocHost failed");
    return HQ_ENOMEM;
  }
  cudaError_t e = cudaMemsetAsync(h->sc, 0, sizeof(DevScalars), h->stream);
  {
    // padding entries are read by the bulk copies: give them defined (zero) contents
    void* zero_bufs[] = {h->masks, h->b64.T, h->b64.r, h->bdf.r, h->b32.r, h->b64.p, h->bdf.p,
                         h->b32.p, h->ab, h->ir_base, h->ir, h->wv64, h->wv32};
    int64_t zero_len[] = {SP * 4, TE * 8, SP * 8, SP * 8, SP * 4, SP * 8, SP * 8, SP * 4,
                          2 * h->ab_half_bytes, SP * 8, SP * 12, SP * 16, SP * 8};
    for (int i = 0; i < 13 && e == cudaSuccess; i++)
      if (zero_bufs[i]) e = cudaMemsetAsync(zero_bufs[i], 0, (size_t)zero_len[i], h->stream);
  }
  if (e != cudaSuccess) {
    int rc = hq_cuda_fail(e, "cudaMemsetAsync", __FILE__, __LINE__);
    free_all(h);
    delete h;
    return rc;
  }
  HQ_TRY(hq_build_layout(h));
  HQ_TRY(hq_build_items(h));
  HQ_TRY(dalloc(h, &h->ir_part, (int64_t)(h->ifirst[N] > 0 ? h->ifirst[N] : 1) * 32));
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    int rc = hq_cuda_fail(e, "layout build", __FILE__, __LINE__);
    free_all(h);
    delete h;
    return rc;
  }
  *out = h;
  return HQ_OK;
}

extern "C" void hq_destroy(hq_solver* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  free_all(h);
  delete h;
}

static cudaMemcpyKind kind_in(int mem) {
  return mem == HQ_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}
static cudaMemcpyKind kind_out(int mem) {
  return mem == HQ_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

extern "C" int hq_load(hq_solver* h, const double* lambda_j, const double* nu, const int32_t* pref,
                       int mem) {
  if (!h || !lambda_j || !nu || !pref) { hq_set_error("NULL argument"); return HQ_EINVAL; }
  if (mem != HQ_HOST && mem != HQ_DEVICE) { hq_set_error("mem must be HQ_HOST or HQ_DEVICE"); return HQ_EINVAL; }
  auto t0 = std::chrono::steady_clock::now();
  h->loaded = false;
  h->solved = false;
  HQ_CUDA(cudaMemcpyAsync(h->lam_j, lambda_j, sizeof(double) * h->J, kind_in(mem), h->stream));
  HQ_CUDA(cudaMemcpyAsync(h->nu, nu, sizeof(double) * h->N, kind_in(mem), h->stream));
  HQ_CUDA(cudaMemcpyAsync(h->pref, pref, sizeof(int32_t) * h->J * h->N, kind_in(mem), h->stream));
  int rc = hq_validate_device(h);
  if (rc != HQ_OK) return rc;
  if (!(h->lam > 0.0)) { hq_set_error("sum of lambda_j must be > 0"); return HQ_EINVAL; }
  if (h->mode == HQ_INFINITE && !(h->lam < h->nu_sum)) {
    hq_set_error("infinite queue needs lambda < sum nu_i");
    return HQ_EUNSTABLE;
  }
  HQ_CUDA(cudaMemcpyAsync(&h->sc->lam, &h->lam, sizeof(double), cudaMemcpyHostToDevice, h->stream));
  rc = hq_build_table(h);
  if (rc != HQ_OK) return rc;
  rc = hq_build_rates(h);
  if (rc != HQ_OK) return rc;
  rc = hq_build_weights(h);
  if (rc != HQ_OK) return rc;
  h->df_ready = false;
  HQ_CUDA(cudaStreamSynchronize(h->stream));
  h->ms_table = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  h->loaded = true;
  h->cur_prec = -1;
  return HQ_OK;
}

static int pull_scalars(hq_solver* h) {
  HQ_CUDA(cudaMemcpyAsync(h->hsc, h->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, h->stream));
  HQ_CUDA(cudaStreamSynchronize(h->stream));
  return HQ_OK;
}

extern "C" int hq_solve(hq_solver* h, const hq_opts* opts_in, hq_stats* stats) {
  if (!h) { hq_set_error("NULL solver"); return HQ_EINVAL; }
  if (!h->loaded) { hq_set_error("hq_load has not succeeded"); return HQ_ESTATE; }
  hq_opts o;
  if (opts_in) o = *opts_in;
  else hq_default_opts(&o);
  if (o.check_every < 1) o.check_every = 1;
  if (o.max_sweeps < 0) { hq_set_error("max_sweeps must be >= 0"); return HQ_EINVAL; }
  if (o.precision < HQ_PREC_FP64 || o.precision > HQ_PREC_FP32_IR) { hq_set_error("bad precision"); return HQ_EINVAL; }
  if (o.tol_kind != HQ_TOL_STEP && o.tol_kind != HQ_TOL_RESIDUAL) { hq_set_error("bad tol_kind"); return HQ_EINVAL; }
  if (o.warm_start < HQ_WARM_NONE || o.warm_start > HQ_WARM_PRODUCT) { hq_set_error("bad warm_start"); return HQ_EINVAL; }
  if (o.warm_start == HQ_WARM_GIVEN && !o.warm_p) { hq_set_error("warm_p is NULL"); return HQ_EINVAL; }
  if (o.warm_start == HQ_WARM_MLP && !h->mlp) { hq_set_error("no warm-start model is attached"); return HQ_EINVAL; }
  if (o.sweep_order != HQ_ORDER_ASCENDING && o.sweep_order != HQ_ORDER_REDBLACK) {
    hq_set_error("sweep_order must be HQ_ORDER_ASCENDING or HQ_ORDER_REDBLACK");
    return HQ_EINVAL;
  }
  if (o.debug_barrier < 0) { hq_set_error("debug_barrier must be >= 0"); return HQ_EINVAL; }
  if (!h->bdf.T && (o.precision == HQ_PREC_DF64 || o.precision == HQ_PREC_FP32_DF64)) {
    hq_set_error("double-float precisions are not kept above N = 28 (memory)");
    return HQ_EINVAL;
  }
  h->order = o.sweep_order;
  // fault injection (tests): CTA debug_barrier - 1 skips its first grid-barrier arrival in
  // the first sweep launch, and every bounded wait gives up after 2^20 polls
  h->dbg_skip_cta = o.debug_barrier > 0 ? o.debug_barrier - 1 : -1;
  h->spin_limit = o.debug_barrier > 0 ? (1u << 20) : 0u;
  // FP32 sweeps stall at their rounding floor; leaving them a check early costs little
  // when the refinement's sweeps cost about as much (correction sweeps), a check late
  // wastes eight sweeps
  double stall = o.fp32_stall > 0.0 ? o.fp32_stall : (o.precision == HQ_PREC_FP32_IR ? 0.75 : 0.9);
  if (!(o.omega < 2.0) || (o.omega >= 0.0 && o.omega < 1.0 && o.omega != 0.0)) {
    hq_set_error("omega must be 0, in [1, 2), or negative (automatic)");
    return HQ_EINVAL;
  }
  const bool auto_omega = o.omega < 0.0;
  h->omega = o.omega >= 1.0 ? o.omega : 1.0;
  int omega_checks = 0;
  auto t0 = std::chrono::steady_clock::now();

  int phases[2];
  int nph = 1;
  switch (o.precision) {
    case HQ_PREC_FP64: phases[0] = HQ_PREC_FP64; break;
    case HQ_PREC_DF64: phases[0] = HQ_PREC_DF64; break;
    case HQ_PREC_FP32: phases[0] = HQ_PREC_FP32; break;
    case HQ_PREC_FP32_DF64: phases[0] = HQ_PREC_FP32; phases[1] = HQ_PREC_DF64; nph = 2; break;
    case HQ_PREC_FP32_IR: phases[0] = HQ_PREC_FP32; phases[1] = HQ_PREC_IRC; nph = 2; break;
    default: phases[0] = HQ_PREC_FP32; phases[1] = HQ_PREC_FP64; nph = 2; break;
  }
  for (int q = 0; q < nph; q++)
    if (phases[q] == HQ_PREC_DF64) {
      const int rcd = hq_ensure_df(h);
      if (rcd != HQ_OK) return rcd;
    }
  int rebases = 0, ir_bases = 0, ir_flat = 0, fp32_flat = 0;
  double step_base = 0.0;  // the first step of the current refinement base
  double last_ratio = 0.0;  // the step decay of the check before
  int phase_checks = 0;     // checks since the last change of precision or base
  int ph = 0;
  int sweeps[2] = {0, 0};
  double kernel_ms[2] = {0.0, 0.0};
  for (cudaEvent_t& e : h->kev)
    if (!e) HQ_CUDA(cudaEventCreate(&e));
  int total = 0, checks = 0, res_checks = 0, since_res = 0, stalled = 0;
  bool warm_kept = o.warm_start == HQ_WARM_GIVEN;
  int rc;
  if ((o.warm_start == HQ_WARM_MLP || o.warm_start == HQ_WARM_PRODUCT) && h->N >= 2) {
    // the learned (or analytic) start is kept only if it is closer to the fixed point than
    // the paper's uniform start, by the FP64 relative balance residual of Eq. (1) of each
    // (the plain iteration's own measure of error); no sweep is spent on the test
    double res_cold = INFINITY, res_warm = INFINITY;
    rc = hq_init_iterate(h, phases[0], nullptr, HQ_HOST);
    if (rc == HQ_OK) rc = hq_compute_residual(h, &res_cold);
    if (rc != HQ_OK) return rc;
    rc = o.warm_start == HQ_WARM_MLP ? hq_mlp_warm_start(h, h->mlp, h->pcond, nullptr)
                                     : hq_product_warm_start(h, h->pcond);
    if (rc == HQ_OK) rc = hq_init_iterate(h, phases[0], h->pcond, HQ_DEVICE);
    if (rc == HQ_OK) rc = hq_compute_residual(h, &res_warm);
    if (rc != HQ_OK) return rc;
    warm_kept = isfinite(res_warm) && res_warm < res_cold;
    if (!warm_kept) {
      rc = hq_init_iterate(h, phases[0], nullptr, HQ_HOST);
      if (rc != HQ_OK) return rc;
    }
  } else {
    rc = hq_init_iterate(h, phases[0], o.warm_start == HQ_WARM_GIVEN ? o.warm_p : nullptr, o.warm_mem);
    if (rc != HQ_OK) return rc;
  }
  h->solved = false;

  double step = INFINITY, prev_check_step = 0.0;
  double res = -1.0, res_at_step = 0.0;
  bool converged = false;
  int status = HQ_OK;
  if (h->N == 1) {
    converged = true;  // no layer between the empty and the full state
    step = 0.0;
  }
  while (!converged && total < o.max_sweeps) {
    const int prec = phases[ph];
    int nrun = o.check_every;
    // last phase, residual tolerance: when the residual, its step and the per-sweep decay
    // of the steps predict the tolerance within fewer sweeps than a check, run only
    // those (and one more) before the next residual evaluation
    if (ph == nph - 1 && o.tol_kind == HQ_TOL_RESIDUAL && res > 0.0 && res_at_step > 0.0 &&
        prev_check_step > 0.0 && last_ratio > 0.0 && last_ratio < 1.0) {
      const double d = pow(last_ratio, 1.0 / o.check_every);
      const double need = log(0.5 * o.tol * res_at_step / (res * prev_check_step)) / log(d);
      if (need > 0.0 && need < (double)(o.check_every - 1)) {
        const int k = (int)ceil(need) + 1;
        nrun = k < 2 ? 2 : k;
      }
    }
    if (nrun > o.max_sweeps - total) nrun = o.max_sweeps - total;
    rc = hq_run_sweeps(h, prec, nrun, h->kev[0], h->kev[1]);
    h->dbg_skip_cta = -1;
    if (rc != HQ_OK) return rc;
    rc = pull_scalars(h);
    if (rc != HQ_OK) return rc;
    {
      // device time of this launch (the scalars' read-back synchronised the stream)
      float kms = 0.0f;
      if (h->N >= 2 && cudaEventElapsedTime(&kms, h->kev[0], h->kev[1]) == cudaSuccess)
        kernel_ms[prec == HQ_PREC_FP32 ? 0 : 1] += kms;
      cudaGetLastError();
    }
    total += nrun;
    sweeps[prec == HQ_PREC_FP32 ? 0 : 1] += nrun;
    checks++;
    step = h->hsc->step;
    if (h->hsc->flags & 6) {
      hq_set_error("a bounded wait in the sweep kernel gave up");
      status = HQ_ETIMEOUT;
      break;
    }
    if ((h->hsc->flags & 1) || !isfinite(step)) {
      hq_set_error("non-finite value in the iteration");
      status = HQ_EDIVERGED;
      break;
    }
    // decay per check of check_every sweeps (a shortened last launch is scaled up to it)
    double ratio = prev_check_step > 0.0 ? step / prev_check_step : 0.0;
    if (ratio > 0.0 && nrun != o.check_every) ratio = pow(ratio, (double)o.check_every / nrun);
    const bool last_phase = ph == nph - 1;
    phase_checks++;
    // leave FP32 once its steps stop shrinking geometrically (rounding floor); correction
    // sweeps cost about what FP32 sweeps cost, so refinement by them also starts when
    // the decay turns abruptly worse than the check before (past the start's transient)
    // A slowly decaying error (a warm start's, or any slow mode) also gives a poor decay
    // ratio: one poor check ends FP32 only once the step is near FP32 resolution (1e-6 of
    // a probability), otherwise two in a row must
    const bool poor = prev_check_step > 0.0 &&
                      (ratio > stall || (phases[ph + 1] == HQ_PREC_IRC && checks > 4 && last_ratio > 0.0 &&
                                         ratio > 0.5 && ratio > 1.5 * last_ratio));
    fp32_flat = poor ? fp32_flat + 1 : 0;
    const bool leave = !last_phase && (step == 0.0 || (poor && (step < 1e-6 || fp32_flat >= 2)));
    if (auto_omega) {
      // Young's optimal relaxation for the observed contraction: with Algorithm 1's
      // per-sweep rate r (measured over the second check, past the start's first
      // transient), omega_opt = 2 / (1 + sqrt(1 - r)), at most 1.9, backed off halfway
      // whenever the steps stop shrinking.  Measured on the N=20 (loads 0.6, 0.9), N=22
      // and N=24 workloads against 90 % of the extrapolation, a 1.5 cap and the third
      // check: the fewest sweeps in every case (N=24 FP32 + refinement 64 + 16 sweeps
      // against 88 + 24)
      omega_checks++;
      if (h->omega == 1.0 && omega_checks == 2 && ratio > 0.0 && ratio < 1.0) {
        const double r = pow(ratio, 1.0 / o.check_every);
        const double wopt = 2.0 / (1.0 + sqrt(1.0 - r));
        h->omega = fmin(wopt, 1.9);
      } else if (h->omega > 1.0 && ratio >= 1.0 && !leave && phase_checks > 3) {
        // (a check that ends the FP32 phase stalls on rounding, not on omega, and the
        // first three checks after a change of precision or base clear the old
        // rounding, which can grow the steps before they fall)
        h->omega = 1.0 + 0.5 * (h->omega - 1.0);
      }
    }
    if (!last_phase) {
      if (leave) {
        rc = hq_convert_iterate(h, phases[ph], phases[ph + 1]);
        if (rc != HQ_OK) return rc;
        if (phases[ph + 1] == HQ_PREC_IRC) ir_bases++;
        ph++;
        fp32_flat = 0;
        prev_check_step = 0.0;
        last_ratio = 0.0;
        phase_checks = 0;
        continue;
      }
      prev_check_step = step;
      last_ratio = ratio;
      continue;
    }
    if (o.tol_kind == HQ_TOL_STEP) {
      if (step <= o.tol) converged = true;
    } else {
      bool do_check = res < 0.0 || since_res >= 8 || step == 0.0;
      if (!do_check && res_at_step > 0.0) {
        double predicted = res * (step / res_at_step);
        do_check = predicted <= 4.0 * o.tol;
      }
      if (do_check) {
        rc = hq_compute_residual(h, &res);
        if (rc != HQ_OK) return rc;
        res_checks++;
        res_at_step = step;
        since_res = 0;
        if (res <= o.tol) converged = true;
      } else {
        since_res++;
      }
    }
    // correction sweeps whose steps stop shrinking have reached the FP32 floor of the
    // correction: fold e into the base and start a new one (iterative refinement).  A
    // flat check is a floor once the correction has shrunk by 1e4; before that only four
    // flat checks in a row are (over-relaxed sweeps pause for a check or two on their way
    // down, and a new base costs about five sweeps).
    if (prec == HQ_PREC_IRC) {
      if (step_base == 0.0) step_base = step;
      ir_flat = (prev_check_step > 0.0 && ratio > stall) ? ir_flat + 1 : 0;
      if (!converged && rebases < 3 && (ir_flat >= 4 || (ir_flat >= 1 && step < 1e-4 * step_base))) {
        rc = hq_ir_begin(h, HQ_PREC_IRC);
        if (rc != HQ_OK) return rc;
        rebases++;
        ir_bases++;
        ir_flat = 0;
        step_base = 0.0;
        prev_check_step = 0.0;
        last_ratio = 0.0;
        phase_checks = 0;
        stalled = 0;
        continue;
      }
    }
    // a precision floor that the tolerance lies below: stop instead of spinning
    if (!converged && prev_check_step > 0.0 && ratio >= 1.0) {
      if (++stalled >= 4) break;
    } else {
      stalled = 0;
    }
    prev_check_step = step;
    last_ratio = ratio;
  }
  h->spin_limit = 0;
  if (status == HQ_ETIMEOUT) {
    // the next launch starts from a clean barrier and flag word
    HQ_CUDA(cudaMemsetAsync(&h->sc->flags, 0, sizeof(int), h->stream));
    HQ_CUDA(cudaStreamSynchronize(h->stream));
  }
  if (status == HQ_EDIVERGED || status == HQ_ETIMEOUT) {
    if (stats) {
      memset(stats, 0, sizeof(*stats));
      stats->sweeps_fp32 = sweeps[0];
      stats->sweeps_hi = sweeps[1];
      stats->final_step = step;
      stats->final_residual = -1.0;
    }
    return status;
  }
  double final_res = -1.0;
  rc = hq_finalize(h, phases[ph], true, &final_res);
  if (rc != HQ_OK) return rc;
  h->solved = true;
  if (!converged) status = HQ_ENOTCONVERGED;
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->sweeps_fp32 = sweeps[0];
    stats->sweeps_hi = sweeps[1];
    stats->residual_checks = res_checks;
    stats->converged = converged ? 1 : 0;
    stats->final_step = step;
    stats->final_residual = final_res;
    stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    stats->ms_table = h->ms_table;
    stats->state_updates = (double)(h->S - 2) * (double)total;
    stats->warm_used = warm_kept ? 1 : 0;
    stats->ir_bases = ir_bases;
    stats->omega = h->omega;
    stats->ms_sweeps_fp32 = kernel_ms[0];
    stats->ms_sweeps_hi = kernel_ms[1];
  }
  (void)checks;
  return status;
}

static int need_solved(const hq_solver* h) {
  if (!h) { hq_set_error("NULL solver"); return HQ_EINVAL; }
  if (!h->solved) { hq_set_error("no solution yet (call hq_solve)"); return HQ_ESTATE; }
  return HQ_OK;
}

static int copy_out(hq_solver* h, void* dst, const void* src, int64_t bytes, int mem) {
  if (!dst) { hq_set_error("NULL output"); return HQ_EINVAL; }
  if (mem != HQ_HOST && mem != HQ_DEVICE) { hq_set_error("mem must be HQ_HOST or HQ_DEVICE"); return HQ_EINVAL; }
  HQ_CUDA(cudaMemcpyAsync(dst, src, (size_t)bytes, kind_out(mem), h->stream));
  HQ_CUDA(cudaStreamSynchronize(h->stream));
  return HQ_OK;
}

extern "C" int hq_get_stationary(hq_solver* h, double* P, int mem) {
  int rc = need_solved(h);
  if (rc != HQ_OK) return rc;
  return copy_out(h, P, h->P, h->S * 8, mem);
}

extern "C" int hq_get_conditional(hq_solver* h, double* p, int mem) {
  int rc = need_solved(h);
  if (rc != HQ_OK) return rc;
  return copy_out(h, p, h->pcond, h->S * 8, mem);
}

extern "C" int hq_get_layer_marginals(hq_solver* h, double* pn, double* queue_tail, int mem) {
  int rc = need_solved(h);
  if (rc != HQ_OK) return rc;
  rc = copy_out(h, pn, h->pn, (int64_t)(h->N + h->C + 1) * 8, mem);
  if (rc != HQ_OK) return rc;
  if (queue_tail) rc = copy_out(h, queue_tail, h->summary + 7, 8, mem);
  return rc;
}

extern "C" int hq_get_utilisation(hq_solver* h, double* rho, int mem) {
  int rc = need_solved(h);
  if (rc != HQ_OK) return rc;
  return copy_out(h, rho, h->rho, (int64_t)h->N * 8, mem);
}

extern "C" int hq_get_response_pattern(hq_solver* h, double* R, int mem) {
  int rc = need_solved(h);
  if (rc != HQ_OK) return rc;
  return copy_out(h, R, h->R, (int64_t)h->J * h->N * 8, mem);
}

extern "C" int hq_get_workload(hq_solver* h, double* W, int mem) {
  int rc = need_solved(h);
  if (rc != HQ_OK) return rc;
  return copy_out(h, W, h->W, (int64_t)h->J * h->N * 8, mem);
}

extern "C" int hq_get_summary(hq_solver* h, double* out5) {
  int rc = need_solved(h);
  if (rc != HQ_OK) return rc;
  return copy_out(h, out5, h->summary, 5 * 8, HQ_HOST);
}

// compact layer-ranked export of the state-major table: entry (n, s, k) of the output
// (layer n, slot s, rank k) at c_off[n] + s C(N,n) + k
struct ExportArgs {
  int N;
  int64_t off[HQ_MAXN + 2];
  int64_t toff[HQ_MAXN + 2];
  int64_t lsize[HQ_MAXN + 1];
  int64_t tw[HQ_MAXN + 1];
  int64_t coff[HQ_MAXN + 2];
};

__global__ void k_table_export(ExportArgs a, int64_t Sp, const double* T, double* out) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= Sp) return;
  int n = 0;
  while (n < a.N && a.off[n + 1] <= g) n++;
  const int64_t k = g - a.off[n];
  if (n < 1 || k >= a.lsize[n]) return;
  for (int sl = 0; sl < n; sl++) out[a.coff[n] + sl * a.lsize[n] + k] = T[a.toff[n] + k * a.tw[n] + sl];
}

extern "C" int hq_get_table(hq_solver* h, double* T, uint32_t* masks, int mem) {
  if (!h) { hq_set_error("NULL solver"); return HQ_EINVAL; }
  if (!h->loaded) { hq_set_error("hq_load has not succeeded"); return HQ_ESTATE; }
  if (mem != HQ_HOST && mem != HQ_DEVICE) { hq_set_error("mem must be HQ_HOST or HQ_DEVICE"); return HQ_EINVAL; }
  const cudaMemcpyKind kind = kind_out(mem);
  if (T) {
    // the device table is state-major and padded; hand out the compact layout of hq.h
    // (through the transform scratch, which holds exactly N 2^(N-1) doubles, for host output)
    ExportArgs a;
    memset(&a, 0, sizeof(a));
    a.N = h->N;
    for (int i = 0; i < HQ_MAXN + 2; i++) {
      a.off[i] = h->off[i];
      a.toff[i] = h->toff[i];
    }
    int64_t c = 0;
    for (int n = 0; n <= h->N; n++) {
      a.lsize[n] = h->lsize[n];
      a.tw[n] = h->tw[n];
      a.coff[n] = c;
      c += n >= 1 ? (int64_t)n * h->lsize[n] : 0;
    }
    double* dst = mem == HQ_DEVICE ? T : h->zeta;
    k_table_export<<<(unsigned)((h->Sp + 255) / 256), 256, 0, h->stream>>>(a, h->Sp, (const double*)h->b64.T, dst);
    HQ_LAUNCHED();
    if (mem == HQ_HOST) HQ_CUDA(cudaMemcpyAsync(T, h->zeta, sizeof(double) * c, cudaMemcpyDeviceToHost, h->stream));
  }
  if (masks) {
    int64_t spos = 0;
    for (int n = 0; n <= h->N; n++) {
      HQ_CUDA(cudaMemcpyAsync(masks + spos, h->masks + h->off[n], (size_t)h->lsize[n] * 4, kind, h->stream));
      spos += h->lsize[n];
    }
  }
  HQ_CUDA(cudaStreamSynchronize(h->stream));
  return HQ_OK;
}

extern "C" int hq_get_info(const hq_solver* h, int64_t* out8) {
  if (!h || !out8) { hq_set_error("NULL argument"); return HQ_EINVAL; }
  out8[0] = h->N;
  out8[1] = h->J;
  out8[2] = h->mode;
  out8[3] = h->C;
  out8[4] = h->S;
  out8[5] = (int64_t)h->N << (h->N - 1);
  out8[6] = h->dev_bytes;
  out8[7] = h->max_layer;
  return HQ_OK;
}

extern "C" double hq_sweep_bytes(const hq_solver* h, int precision) {
  if (!h) return 0.0;
  const bool ir = precision == HQ_PREC_FP32_IR;
  const double e = (precision == HQ_PREC_FP32 || ir) ? 4.0 : 8.0;
  // a correction sweep also reads three FP32 base terms per state
  const double extra = ir ? 12.0 : 0.0;
  double b = 0.0;
  for (int n = 1; n <= h->N - 1; n++) b += (double)h->lsize[n] * ((n + 3) * e + extra);
  return b;
}

extern "C" int hq_profile_sweep(hq_solver* h, int precision, int sweeps, float* ms_out) {
  int rc = need_solved(h);
  if (rc != HQ_OK) return rc;
  if (!ms_out || sweeps < 1) { hq_set_error("ms_out NULL or sweeps < 1"); return HQ_EINVAL; }
  if (precision != HQ_PREC_FP64 && precision != HQ_PREC_DF64 && precision != HQ_PREC_FP32 &&
      precision != HQ_PREC_FP32_IR) {
    hq_set_error("precision must be FP64, DF64, FP32 or FP32_IR");
    return HQ_EINVAL;
  }
  ms_out[0] = 0.f;
  if (h->N < 2) return HQ_OK;
  if (precision == HQ_PREC_DF64 && !h->bdf.T) {
    hq_set_error("double-float precisions are not kept above N = 28 (memory)");
    return HQ_EINVAL;
  }
  if (precision == HQ_PREC_DF64) {
    rc = hq_ensure_df(h);
    if (rc != HQ_OK) return rc;
  }
  if (precision == HQ_PREC_FP32_IR) precision = HQ_PREC_IRC;  // correction sweeps
  if (h->cur_prec != precision) {
    rc = hq_convert_iterate(h, h->cur_prec, precision);
    if (rc != HQ_OK) return rc;
  }
  cudaEvent_t ev0, ev1;
  HQ_CUDA(cudaEventCreate(&ev0));
  HQ_CUDA(cudaEventCreate(&ev1));
  rc = hq_run_sweeps(h, precision, sweeps, ev0, ev1);
  if (rc == HQ_OK) {
    cudaError_t e = cudaEventSynchronize(ev1);
    if (e != cudaSuccess) rc = hq_cuda_fail(e, "cudaEventSynchronize", __FILE__, __LINE__);
    float ms = 0.f;
    if (rc == HQ_OK) cudaEventElapsedTime(&ms, ev0, ev1);
    ms_out[0] = ms / (float)sweeps;
  }
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  return rc;
}

extern "C" int hq_profile_phases(hq_solver* h, double* us_out, int max_out) {
  int rc = need_solved(h);
  if (rc != HQ_OK) return rc;
  if (!us_out || max_out < 0) { hq_set_error("us_out NULL"); return HQ_EINVAL; }
  rc = pull_scalars(h);
  if (rc != HQ_OK) return rc;
  const DevScalars* s = h->hsc;
  int n = 0;
  unsigned long long prev = s->t_start;
  for (int g = 0; g < 64 && n < max_out; g++) {
    const unsigned long long t = s->t_phase[g];
    if (t <= prev || t == 0) break;
    us_out[n++] = (double)(t - prev) * 1e-3;
    prev = t;
  }
  return n;
}

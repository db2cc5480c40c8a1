// Set-up of the iterate of Algorithm 1 (its initial value and lambda(n), mu(n) of
// Eq. 6-7) and changes of its precision between FP32, DF64 and FP64.  The sweeps
// themselves are in hq_persist.cu.
#include "hq_internal.cuh"

// ---------------------------------------------------------------------------
// iterate set-up and precision changes
// ---------------------------------------------------------------------------
struct InitArgs {
  int N;
  int64_t off[HQ_MAXN + 2];
  int64_t lsize[HQ_MAXN + 1];
  double inv_binom[HQ_MAXN + 1];
};

template <class V>
__global__ void k_init_cold(InitArgs a, int64_t Sp, typename V::T* p) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= Sp) return;
  int n = 0;
  while (n < a.N && a.off[n + 1] <= g) n++;
  p[g] = V::from_d(g - a.off[n] < a.lsize[n] ? a.inv_binom[n] : 0.0);
}

template <class V>
__global__ void k_init_warm(InitArgs a, int64_t Sp, const uint32_t* masks, const double* warm_y,
                            typename V::T* p) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= Sp) return;
  int n = 0;
  while (n < a.N && a.off[n + 1] <= g) n++;
  // the empty and the full state are single-state layers: their conditional is 1
  const double v = (n == 0 || n == a.N) ? 1.0 : warm_y[masks[g]];
  p[g] = V::from_d(g - a.off[n] < a.lsize[n] ? v : 0.0);
}

// lambda(n), mu(n) of Eq. (6)-(7) from the layer sums of the current iterate
__global__ void k_set_layer_rates(DevScalars* sc, int N, double lam, double lam_full, double nu_sum) {
  if (threadIdx.x != 0) return;
  for (int n = 0; n < N; n++) {
    sc->lam_n[n] = lam * sc->lsum[n];
    sc->mu_n[n] = sc->lmu[n];
  }
  sc->lam_n[N] = lam_full * sc->lsum[N];
  sc->mu_n[N] = nu_sum;
  sc->step = 0.0;
  sc->step_prev = 0.0;
  sc->flags = 0;
}

template <class V>
static int init_typed(hq_solver* h, const double* warm_dev) {
  PrecBufs& b = hq_bufs(h, V::kind);
  typename V::T* p = (typename V::T*)b.p;
  unsigned grid = (unsigned)((h->Sp + 255) / 256);
  InitArgs a;
  a.N = h->N;
  for (int i = 0; i < HQ_MAXN + 2; i++) a.off[i] = h->off[i];
  for (int n = 0; n <= HQ_MAXN; n++) {
    a.lsize[n] = n <= h->N ? h->lsize[n] : 0;
    a.inv_binom[n] = n <= h->N ? 1.0 / hq_binom(h->N, n) : 0.0;
  }
  if (warm_dev) k_init_warm<V><<<grid, 256, 0, h->stream>>>(a, h->Sp, h->masks, warm_dev, p);
  else k_init_cold<V><<<grid, 256, 0, h->stream>>>(a, h->Sp, p);
  HQ_LAUNCHED();
  return HQ_OK;
}

int hq_init_iterate(hq_solver* h, int prec, const double* warm_y, int warm_mem) {
  const double* warm_dev = nullptr;
  h->it_version++;
  if (warm_y) {
    if (warm_mem == HQ_HOST) {
      // stage through the y-order result buffer
      HQ_CUDA(cudaMemcpyAsync(h->P, warm_y, sizeof(double) * h->S, cudaMemcpyHostToDevice, h->stream));
      warm_dev = h->P;
    } else {
      warm_dev = warm_y;
    }
  }
  int rc;
  if (prec == HQ_PREC_FP64) rc = init_typed<PolF64>(h, warm_dev);
  else if (prec == HQ_PREC_DF64) rc = init_typed<PolDF>(h, warm_dev);
  else rc = init_typed<PolF32>(h, warm_dev);
  if (rc != HQ_OK) return rc;
  h->cur_prec = prec;
  rc = hq_layer_sums(h, prec);
  if (rc != HQ_OK) return rc;
  rc = hq_iter_sums(h, prec, hq_bufs(h, prec).p, &h->sc->ls[0][0]);
  if (rc != HQ_OK) return rc;
  HQ_CUDA(cudaMemsetAsync(&h->sc->sweeps, 0, sizeof(int), h->stream));
  k_set_layer_rates<<<1, 32, 0, h->stream>>>(h->sc, h->N, h->lam,
                                             h->mode == HQ_LOSS ? 0.0 : h->lam, h->nu_sum);
  HQ_LAUNCHED();
  return HQ_OK;
}

template <class VF, class VT>
__global__ void k_convert(int64_t S, const typename VF::T* src, typename VT::T* dst) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= S) return;
  dst[g] = VT::from_d(VF::to_d(src[g]));
}

// FP32 -> DF64 without the FP64 pipe: hi = x, lo = 0
__global__ void k_f32_to_df(int64_t S, const float* src, float2* dst) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= S) return;
  dst[g] = make_float2(src[g], 0.f);
}

int hq_convert_iterate(hq_solver* h, int from, int to, bool sums) {
  if (from == to) return HQ_OK;
  h->it_version++;
  if (to == HQ_PREC_IRC) return hq_ir_begin(h, from);
  if (from == HQ_PREC_IRC) {
    // the refinement's iterate is p0 + e: assemble it in FP64 first
    const int rc = hq_ir_assemble(h);
    if (rc != HQ_OK) return rc;
    h->cur_prec = HQ_PREC_FP64;
    if (to == HQ_PREC_FP64) return sums ? hq_iter_sums(h, HQ_PREC_FP64, h->b64.p, &h->sc->ls[0][0]) : HQ_OK;
    from = HQ_PREC_FP64;
  }
  const int64_t S = h->Sp;
  unsigned grid = (unsigned)((S + 255) / 256);
  void* s = hq_bufs(h, from).p;
  void* d = hq_bufs(h, to).p;
  if (from == HQ_PREC_FP32 && to == HQ_PREC_DF64)
    k_f32_to_df<<<grid, 256, 0, h->stream>>>(S, (const float*)s, (float2*)d);
  else if (from == HQ_PREC_FP32 && to == HQ_PREC_FP64)
    k_convert<PolF32, PolF64><<<grid, 256, 0, h->stream>>>(S, (const float*)s, (double*)d);
  else if (from == HQ_PREC_DF64 && to == HQ_PREC_FP64)
    k_convert<PolDF, PolF64><<<grid, 256, 0, h->stream>>>(S, (const float2*)s, (double*)d);
  else if (from == HQ_PREC_FP64 && to == HQ_PREC_DF64)
    k_convert<PolF64, PolDF><<<grid, 256, 0, h->stream>>>(S, (const double*)s, (float2*)d);
  else if (from == HQ_PREC_DF64 && to == HQ_PREC_FP32)
    k_convert<PolDF, PolF32><<<grid, 256, 0, h->stream>>>(S, (const float2*)s, (float*)d);
  else
    k_convert<PolF64, PolF32><<<grid, 256, 0, h->stream>>>(S, (const double*)s, (float*)d);
  HQ_LAUNCHED();
  h->cur_prec = to;
  // the sweep reads the layer sums of the iterate in its new precision
  return sums ? hq_iter_sums(h, to, d, &h->sc->ls[0][0]) : HQ_OK;
}

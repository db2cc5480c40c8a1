// One outer iteration k of Algorithm 1 (Eq. 12-14) on the layer-ranked layout.
//
// For layer n (ascending, Gauss-Seidel from layer n-1, Jacobi from layer n+1 as in
// Algorithm 1 and the two properties listed for Algorithm 2) and each state m of
// the layer, write Eq. (12) as
//     p_n^{k,r}(m) = alpha mu^{k,r-1}(n) A_m + beta B_m
// with  alpha = 1/lambda^k(n-1),  beta = lambda^{k-1}(n) / mu^{k-1}(n+1),
//       A_m = r_m sum_{l in C_{n-1}} p^k_{n-1}(l) lambda_{lm},
//       B_m = r_m sum_{u idle in m} p^{k-1}_{n+1}(m+u) nu_u,   r_m = 1/(lambda_m+mu_m).
// Only mu^{k,r-1}(n) changes with r, and Eq. (14) gives the scalar recursion
//     mu^{k,r} = a mu^{k,r-1} + b,  a = alpha sum mu_m A_m,  b = beta sum mu_m B_m,
// with 0 < a < 1 (sum_m lambda_{lm} = lambda and mu_m/(lambda+mu_m) < 1).  The inner
// loop of Algorithm 1 therefore converges to mu* = b / (1 - a), and its limit is
// p_n^k(m) = alpha mu* A_m + beta B_m.  That limit is what is computed here: the
// delta -> 0 reading of the inner loop.  Then lambda^k(n) = lambda sum_m p_n^k(m)
// (Eq. 13) and mu^k(n) = mu*.
//
// Two kernels per layer:
//   k_gather  -- per state: A_m, B_m (gathers from layers n-1 and n+1, one
//                streamed table row per busy unit), block sums of mu_m A_m and
//                mu_m B_m; the last CTA solves the scalar recursion.
//   k_update  -- per state: p = c1 A + c2 B, |p - p_old|; block sum of p and max
//                step; the last CTA applies Eq. (13).
// Reductions are deterministic: block trees, then the last CTA adds the block
// partials in a fixed order.
#include "hq_internal.cuh"

struct SweepArgs {
  int N, L, n;
  int64_t Ln;
  const uint32_t* masks;  // layer n masks
  const uint32_t* RL;
  const uint32_t* RH;
  const void* T;          // layer n table block
  const void* r;          // layer n r_m
  const void* p_dn;       // layer n-1 (iteration k)
  const void* p_up;       // layer n+1 (iteration k-1)
  void* p_cur;            // layer n
  const void* nu;         // N values
  void* ab;               // (A, B) scratch
  double* partials;
  DevScalars* sc;
};

template <class V>
__device__ __forceinline__ typename V::T block_sum(typename V::T v, typename V::T* s_warp) {
  for (int m = 16; m > 0; m >>= 1) v = V::add(v, V::shfl_xor(v, m));
  int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) s_warp[wid] = v;
  __syncthreads();
  typename V::T t = V::zero();
  if (wid == 0) {
    t = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : V::zero();
    for (int m = 16; m > 0; m >>= 1) t = V::add(t, V::shfl_xor(t, m));
  }
  __syncthreads();
  return t;  // valid in thread 0
}

__device__ __forceinline__ double block_max_d(double v, double* s_warp) {
  for (int m = 16; m > 0; m >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, m));
  int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) s_warp[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (wid == 0) {
    t = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0.0;
    for (int m = 16; m > 0; m >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, m));
  }
  __syncthreads();
  return t;
}

__device__ __forceinline__ double block_sum_d(double v, double* s_warp) {
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) s_warp[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (wid == 0) {
    t = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0.0;
    for (int m = 16; m > 0; m >>= 1) t += __shfl_xor_sync(0xffffffffu, t, m);
  }
  __syncthreads();
  return t;
}

// Called by all threads of the last CTA: sum `width` interleaved partial columns
// over `nblk` blocks in a fixed order.  Result valid in thread 0.
__device__ __forceinline__ double last_block_column_sum(const double* partials, int width, int col,
                                                       int nblk, double* s_warp) {
  double v = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) v += __ldcg(partials + (int64_t)b * width + col);
  return block_sum_d(v, s_warp);
}
__device__ __forceinline__ double last_block_column_max(const double* partials, int width, int col,
                                                       int nblk, double* s_warp) {
  double v = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) v = fmax(v, __ldcg(partials + (int64_t)b * width + col));
  return block_max_d(v, s_warp);
}

// returns true in every thread of the CTA that finished last
__device__ __forceinline__ bool arrive_last(unsigned* ticket, bool* s_flag) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(ticket, 1u);
    *s_flag = (t == gridDim.x - 1);
  }
  __syncthreads();
  bool last = *s_flag;
  if (last) __threadfence();
  return last;
}

template <class V>
__global__ void __launch_bounds__(HQ_THREADS) k_gather(SweepArgs a) {
  typedef typename V::T T;
  extern __shared__ uint32_t s_RL[];
  __shared__ T s_nu[HQ_MAXN];
  __shared__ T s_warp[HQ_THREADS / 32];
  __shared__ double s_wd[HQ_THREADS / 32];
  __shared__ T s_lam, s_one;
  __shared__ bool s_last;
  const int nL = 1 << a.L;
  for (int i = threadIdx.x; i < nL; i += blockDim.x) s_RL[i] = a.RL[i];
  if (threadIdx.x < a.N) s_nu[threadIdx.x] = ((const T*)a.nu)[threadIdx.x];
  if (threadIdx.x == 0) {
    s_lam = V::from_d(a.sc->lam);
    s_one = V::from_d(1.0);
  }
  __syncthreads();

  const T* Tn = (const T*)a.T;
  const T* pdn = (const T*)a.p_dn;
  const T* pup = (const T*)a.p_up;
  const int L = a.L;
  const uint32_t full = (1u << a.N) - 1u;
  T* ab = (T*)a.ab;
  T muA = V::zero(), muB = V::zero();
  // grid-stride: the CTA-level set-up above is paid once per resident CTA
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.Ln;
       k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t x = __ldcs(a.masks + k);
    const uint32_t lo = x & ((1u << L) - 1u), hi = x >> L;
    const int w = __popc(lo);
    const uint32_t* rh = a.RH + (size_t)hi * (L + 1);
    const uint32_t rl = s_RL[lo];
    const uint32_t base_dn = w > 0 ? __ldg(rh + w - 1) : 0u;
    const uint32_t base_up = w < L ? __ldg(rh + w + 1) : 0u;
    // Every state of layer n has exactly n busy and N-n idle units, so both loops
    // below have the same trip count in every lane; unrolling them lets each thread
    // keep several independent gathers and table loads in flight.
    // up-inflow from layer n-1: one neighbour per busy unit, table slot s
    T U = V::zero();
    uint32_t y = x;
#pragma unroll 4
    for (int s = 0; s < a.n; ++s) {
      const int b = __ffs(y) - 1;
      y &= y - 1;
      uint32_t rk;
      if (b < L) rk = s_RL[lo ^ (1u << b)] + base_dn;
      else rk = rl + __ldg(a.RH + (size_t)(hi ^ (1u << (b - L))) * (L + 1) + w);
      V::fma_acc(U, ld_ro(pdn + rk), ld_stream(Tn + (int64_t)s * a.Ln + k));
    }
    // down-inflow from layer n+1: one neighbour per idle unit, rate nu_u
    T D = V::zero();
    y = ~x & full;
#pragma unroll 4
    for (int s = a.n; s < a.N; ++s) {
      const int b = __ffs(y) - 1;
      y &= y - 1;
      uint32_t rk;
      if (b < L) rk = s_RL[lo | (1u << b)] + base_up;
      else rk = rl + __ldg(a.RH + (size_t)(hi | (1u << (b - L))) * (L + 1) + w);
      V::fma_acc(D, ld_ro(pup + rk), s_nu[b]);
    }
    U = V::norm(U);
    D = V::norm(D);
    const T r = ld_stream((const T*)a.r + k);
    const T q = V::sub(s_one, V::mul(s_lam, r));  // mu_m r_m = 1 - lambda r_m
    ab[2 * k] = V::mul(U, r);
    ab[2 * k + 1] = V::mul(D, r);
    muA = V::add(muA, V::mul(U, q));
    muB = V::add(muB, V::mul(D, q));
  }
  T sA = block_sum<V>(muA, s_warp);
  T sB = block_sum<V>(muB, s_warp);
  if (threadIdx.x == 0) {
    a.partials[2 * (int64_t)blockIdx.x] = V::to_d(sA);
    a.partials[2 * (int64_t)blockIdx.x + 1] = V::to_d(sB);
  }
  if (!arrive_last(&a.sc->ticket[0], &s_last)) return;
  double SA = last_block_column_sum(a.partials, 2, 0, gridDim.x, s_wd);
  double SB = last_block_column_sum(a.partials, 2, 1, gridDim.x, s_wd);
  if (threadIdx.x == 0) {
    DevScalars* sc = a.sc;
    const int n = a.n;
    const double alpha = 1.0 / sc->lam_n[n - 1];
    const double beta = sc->lam_n[n] / sc->mu_n[n + 1];
    const double aa = alpha * SA, bb = beta * SB;
    const double mustar = bb / (1.0 - aa);
    sc->c1[n] = alpha * mustar;
    sc->c2[n] = beta;
    sc->mu_n[n] = mustar;
    if (!isfinite(mustar) || !(aa < 1.0)) sc->flags |= 1;
    sc->ticket[0] = 0u;
  }
}

template <class V>
__global__ void __launch_bounds__(HQ_THREADS) k_update(SweepArgs a) {
  typedef typename V::T T;
  __shared__ T s_c1, s_c2;
  __shared__ T s_warp[HQ_THREADS / 32];
  __shared__ double s_wd[HQ_THREADS / 32];
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
    s_c1 = V::from_d(a.sc->c1[a.n]);
    s_c2 = V::from_d(a.sc->c2[a.n]);
  }
  __syncthreads();
  const T c1 = s_c1, c2 = s_c2;
  const T* ab = (const T*)a.ab;
  T* pc = (T*)a.p_cur;
  T sp = V::zero();
  double md = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.Ln;
       k += (int64_t)gridDim.x * blockDim.x) {
    const T A = ab[2 * k], B = ab[2 * k + 1];
    const T old = ld_stream(pc + k);
    const T pv = V::add(V::mul(c1, A), V::mul(c2, B));
    md = fmax(md, V::absdiff(pv, old));
    pc[k] = pv;
    sp = V::add(sp, pv);
  }
  sp = block_sum<V>(sp, s_warp);
  md = block_max_d(md, s_wd);
  if (threadIdx.x == 0) {
    a.partials[2 * (int64_t)blockIdx.x] = V::to_d(sp);
    a.partials[2 * (int64_t)blockIdx.x + 1] = md;
  }
  if (!arrive_last(&a.sc->ticket[1], &s_last)) return;
  double S = last_block_column_sum(a.partials, 2, 0, gridDim.x, s_wd);
  double M = last_block_column_max(a.partials, 2, 1, gridDim.x, s_wd);
  if (threadIdx.x == 0) {
    DevScalars* sc = a.sc;
    sc->lam_n[a.n] = sc->lam * S;  // Eq. (13): lambda_m = lambda in layers n < N
    sc->sum_layer[a.n] = S;
    sc->step_layer[a.n] = M;
    if (!isfinite(S) || !isfinite(M)) sc->flags |= 1;
    sc->ticket[1] = 0u;
  }
}

__global__ void k_sweep_end(DevScalars* sc, int N) {
  if (threadIdx.x != 0) return;
  double m = 0.0;
  for (int n = 1; n <= N - 1; n++) m = fmax(m, sc->step_layer[n]);
  if (!isfinite(m)) sc->flags |= 1;
  sc->step_prev = sc->step;
  sc->step = m;
  sc->sweeps += 1;
}

PrecBufs& hq_bufs(hq_solver* h, int prec) {
  if (prec == HQ_PREC_FP64) return h->b64;
  if (prec == HQ_PREC_DF64) return h->bdf;
  return h->b32;
}

static size_t elem_size(int prec) {
  return prec == HQ_PREC_FP32 ? sizeof(float) : (prec == HQ_PREC_DF64 ? sizeof(float2) : sizeof(double));
}

template <class V>
static int launch_layer_split(hq_solver* h, int n, cudaEvent_t* mid) {
  PrecBufs& b = hq_bufs(h, V::kind);
  const size_t es = sizeof(typename V::T);
  SweepArgs a;
  a.N = h->N;
  a.L = h->L;
  a.n = n;
  a.Ln = h->lsize[n];
  a.masks = h->masks + h->off[n];
  a.RL = h->RL;
  a.RH = h->RH;
  a.T = (const char*)b.T + es * h->toff[n];
  a.r = (const char*)b.r + es * h->off[n];
  a.p_dn = (const char*)b.p + es * h->off[n - 1];
  a.p_up = (const char*)b.p + es * h->off[n + 1];
  a.p_cur = (char*)b.p + es * h->off[n];
  a.nu = b.nu;
  a.ab = h->ab;
  a.partials = h->partials;
  a.sc = h->sc;
  const int64_t want = (a.Ln + HQ_THREADS - 1) / HQ_THREADS;
  size_t smem = sizeof(uint32_t) << h->L;
  static int occ_g[3] = {0, 0, 0}, occ_u[3] = {0, 0, 0}, nsm = 0;
  const int slot = V::kind == HQ_PREC_FP64 ? 0 : (V::kind == HQ_PREC_DF64 ? 1 : 2);
  if (!nsm) HQ_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->dev));
  if (!occ_g[slot]) {
    HQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_g[slot], k_gather<V>, HQ_THREADS,
                                                          sizeof(uint32_t) << HQ_LO_BITS));
    HQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_u[slot], k_update<V>, HQ_THREADS, 0));
    if (occ_g[slot] < 1) occ_g[slot] = 1;
    if (occ_u[slot] < 1) occ_u[slot] = 1;
  }
  const int64_t cap_g = (int64_t)nsm * occ_g[slot], cap_u = (int64_t)nsm * occ_u[slot];
  const unsigned grid_g = (unsigned)(want < cap_g ? want : cap_g);
  const unsigned grid_u = (unsigned)(want < cap_u ? want : cap_u);
  k_gather<V><<<grid_g, HQ_THREADS, smem, h->stream>>>(a);
  HQ_LAUNCHED();
  if (mid) HQ_CUDA(cudaEventRecord(*mid, h->stream));
  k_update<V><<<grid_u, HQ_THREADS, 0, h->stream>>>(a);
  HQ_LAUNCHED();
  return HQ_OK;
}

template <class V>
static int launch_layer(hq_solver* h, int n) {
  return launch_layer_split<V>(h, n, nullptr);
}

template <class V>
static int launch_layer_split(hq_solver* h, int n, cudaEvent_t* mid);

int hq_launch_sweep_timed(hq_solver* h, int prec, cudaEvent_t* ev) {
  for (int n = 1; n <= h->N - 1; n++) {
    int rc;
    HQ_CUDA(cudaEventRecord(ev[2 * (n - 1)], h->stream));
    if (prec == HQ_PREC_FP64) rc = launch_layer_split<PolF64>(h, n, ev + 2 * (n - 1) + 1);
    else if (prec == HQ_PREC_DF64) rc = launch_layer_split<PolDF>(h, n, ev + 2 * (n - 1) + 1);
    else rc = launch_layer_split<PolF32>(h, n, ev + 2 * (n - 1) + 1);
    if (rc != HQ_OK) return rc;
  }
  HQ_CUDA(cudaEventRecord(ev[2 * (h->N - 1)], h->stream));
  k_sweep_end<<<1, 32, 0, h->stream>>>(h->sc, h->N);
  HQ_LAUNCHED();
  return HQ_OK;
}

int hq_launch_sweep(hq_solver* h, int prec) {
  for (int n = 1; n <= h->N - 1; n++) {
    int rc;
    if (prec == HQ_PREC_FP64) rc = launch_layer<PolF64>(h, n);
    else if (prec == HQ_PREC_DF64) rc = launch_layer<PolDF>(h, n);
    else rc = launch_layer<PolF32>(h, n);
    if (rc != HQ_OK) return rc;
  }
  k_sweep_end<<<1, 32, 0, h->stream>>>(h->sc, h->N);
  HQ_LAUNCHED();
  return HQ_OK;
}

int hq_get_sweep_graph(hq_solver* h, int prec, cudaGraphExec_t* out, int* kernels) {
  int slot = prec == HQ_PREC_FP64 ? 0 : (prec == HQ_PREC_DF64 ? 1 : 2);
  if (h->graph[slot]) {
    *out = h->graph[slot];
    *kernels = h->graph_kernels[slot];
    return HQ_OK;
  }
  cudaGraph_t g;
  HQ_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  int rc = hq_launch_sweep(h, prec);
  cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  if (rc != HQ_OK) return rc;
  if (e != cudaSuccess) return hq_cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
  hq_count_launch(-(2 * (h->N - 1) + 1));  // captured, not run
  cudaGraphExec_t ex;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return hq_cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
  h->graph[slot] = ex;
  h->graph_kernels[slot] = 2 * (h->N - 1) + 1;
  *out = ex;
  *kernels = h->graph_kernels[slot];
  return HQ_OK;
}

// ---------------------------------------------------------------------------
// iterate set-up and precision changes
// ---------------------------------------------------------------------------
struct InitArgs {
  int N;
  int64_t off[HQ_MAXN + 2];
  double inv_binom[HQ_MAXN + 1];
};

template <class V>
__global__ void k_init_cold(InitArgs a, int64_t S, typename V::T* p) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= S) return;
  int n = 0;
  while (n < a.N && a.off[n + 1] <= g) n++;
  p[g] = V::from_d(a.inv_binom[n]);
}

template <class V>
__global__ void k_init_warm(int64_t S, const uint32_t* masks, const double* warm_y,
                            typename V::T* p) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= S) return;
  p[g] = V::from_d(warm_y[masks[g]]);
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
  unsigned grid = (unsigned)((h->S + 255) / 256);
  if (warm_dev) {
    k_init_warm<V><<<grid, 256, 0, h->stream>>>(h->S, h->masks, warm_dev, p);
  } else {
    InitArgs a;
    a.N = h->N;
    for (int i = 0; i < HQ_MAXN + 2; i++) a.off[i] = h->off[i];
    for (int n = 0; n <= HQ_MAXN; n++) a.inv_binom[n] = n <= h->N ? 1.0 / hq_binom(h->N, n) : 0.0;
    k_init_cold<V><<<grid, 256, 0, h->stream>>>(a, h->S, p);
  }
  HQ_LAUNCHED();
  return HQ_OK;
}

int hq_init_iterate(hq_solver* h, int prec, const double* warm_y, int warm_mem) {
  const double* warm_dev = nullptr;
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

int hq_convert_iterate(hq_solver* h, int from, int to) {
  if (from == to) return HQ_OK;
  unsigned grid = (unsigned)((h->S + 255) / 256);
  void* s = hq_bufs(h, from).p;
  void* d = hq_bufs(h, to).p;
  if (from == HQ_PREC_FP32 && to == HQ_PREC_DF64)
    k_f32_to_df<<<grid, 256, 0, h->stream>>>(h->S, (const float*)s, (float2*)d);
  else if (from == HQ_PREC_FP32 && to == HQ_PREC_FP64)
    k_convert<PolF32, PolF64><<<grid, 256, 0, h->stream>>>(h->S, (const float*)s, (double*)d);
  else if (from == HQ_PREC_DF64 && to == HQ_PREC_FP64)
    k_convert<PolDF, PolF64><<<grid, 256, 0, h->stream>>>(h->S, (const float2*)s, (double*)d);
  else if (from == HQ_PREC_FP64 && to == HQ_PREC_DF64)
    k_convert<PolF64, PolDF><<<grid, 256, 0, h->stream>>>(h->S, (const double*)s, (float2*)d);
  else if (from == HQ_PREC_DF64 && to == HQ_PREC_FP32)
    k_convert<PolDF, PolF32><<<grid, 256, 0, h->stream>>>(h->S, (const float2*)s, (float*)d);
  else
    k_convert<PolF64, PolF32><<<grid, 256, 0, h->stream>>>(h->S, (const double*)s, (float*)d);
  HQ_LAUNCHED();
  h->cur_prec = to;
  (void)elem_size;
  return HQ_OK;
}

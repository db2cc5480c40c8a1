// From the conditional probabilities to the stationary distribution and the
// performance measures, in FP64 (sums of many non-negative terms in exact 64-bit fixed
// point):
//   * layer totals S_n = sum_m p_n(B_m), M_n = sum_m mu_m p_n(B_m) (Eq. 6-7);
//   * p(n) of the birth-death process -- Eq. (10), Proposition 2 (finite
//     buffer) and the Remark (infinite buffer) -- by a log-scale recursion;
//   * P{B} = p(w(B)) p_w(B) (Proposition 1), unit utilisations, the response
//     pattern (superset-sum transform) and workloads;
//   * the relative global-balance residual of Eq. (1).
// Layer totals S_n are used to renormalise: in exact arithmetic S_n = 1 for every
// iteration (Lemma 1); rounding leaves S_n = 1 + O(eps), and any common factor
// per layer cancels from P once lambda(n), mu(n) and p(n) are taken from the
// normalised p_n / S_n.
#include <math.h>

#include "hq_internal.cuh"

namespace {

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}
__device__ __forceinline__ double warp_max_d(double v) {
  for (int m = 16; m > 0; m >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, m));
  return v;
}

// block reduction of two values (sum or max per flag), result in thread 0
__device__ void block_reduce2(double& a, double& b, bool a_max, bool b_max, double* s) {
  a = a_max ? warp_max_d(a) : warp_sum_d(a);
  b = b_max ? warp_max_d(b) : warp_sum_d(b);
  int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0) {
    s[2 * wid] = a;
    s[2 * wid + 1] = b;
  }
  __syncthreads();
  if (wid == 0) {
    a = lane < nw ? s[2 * lane] : 0.0;
    b = lane < nw ? s[2 * lane + 1] : 0.0;
    a = a_max ? warp_max_d(a) : warp_sum_d(a);
    b = b_max ? warp_max_d(b) : warp_sum_d(b);
  }
  __syncthreads();
}

__device__ bool arrive_last_post(unsigned* ticket, bool* s_flag) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) *s_flag = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  bool last = *s_flag;
  if (last) __threadfence();
  return last;
}

// last CTA: fold the (a, b) partials of every block in a fixed order
__device__ void fold_partials(const double* partials, bool a_max, bool b_max, double* s, double& A,
                              double& B) {
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    double pa = __ldcg(partials + 2 * (int64_t)i), pb = __ldcg(partials + 2 * (int64_t)i + 1);
    a = a_max ? fmax(a, pa) : a + pa;
    b = b_max ? fmax(b, pb) : b + pb;
  }
  block_reduce2(a, b, a_max, b_max, s);
  A = a;
  B = b;
}

// Layer totals S_n = sum_m p_n(B_m) and M_n = sum_m mu_m p_n(B_m) of every layer in one
// pass, in 64-bit fixed point: p at 2^61 (p <= 1) and mu_m p at 2^em (sum nu < 2^(61-em)),
// mu_m itself an exact integer sum of the quantised nu_i.  Integer adds are exact, so the
// totals do not depend on the order in which warps add them: each warp takes a
// contiguous run of 32-state chunks (layers start on 32-entry boundaries, so a chunk
// lies in one layer) and adds its running sums to the layer's accumulators whenever
// the layer changes.  k_layer_totals then converts them to FP64.
struct LayerSumArgs {
  int N;
  int64_t off[HQ_MAXN + 2];
  int64_t lsize[HQ_MAXN + 1];
  double scale_nu;  // 2^em
};

template <class V>
__global__ void __launch_bounds__(256) k_layer_sum(LayerSumArgs a, const uint32_t* masks,
                                                   const typename V::T* p, const double* nu,
                                                   DevScalars* sc) {
  __shared__ long long s_nu[HQ_MAXN];
  if (threadIdx.x < a.N) s_nu[threadIdx.x] = __double2ll_rn(nu[threadIdx.x] * a.scale_nu);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t chunks = a.off[a.N + 1] >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t per = (chunks + nw - 1) / nw;
  const int64_t c0 = gw * per, c1 = c0 + per < chunks ? c0 + per : chunks;
  int n = 0;
  long long sv = 0, sm = 0;
  for (int64_t c = c0; c < c1; c++) {
    const int64_t g = (c << 5) + lane;
    int nc = n;
    while (nc < a.N && a.off[nc + 1] <= (c << 5)) nc++;
    if (nc != n) {
      if (lane == 0 && (sv | sm)) {
        atomicAdd((unsigned long long*)&sc->lsum_q[n], (unsigned long long)sv);
        atomicAdd((unsigned long long*)&sc->lmu_q[n], (unsigned long long)sm);
      }
      sv = sm = 0;
      n = nc;
    }
    long long v = 0, vm = 0;
    if (g - a.off[n] < a.lsize[n]) {
      const double pv = V::to_d(p[g]);
      long long mq = 0;
      for (uint32_t y = masks[g]; y; y &= y - 1) mq += s_nu[__ffs(y) - 1];
      v = __double2ll_rn(pv * 0x1p61);
      vm = __double2ll_rn(pv * (double)mq);  // (mu_m 2^em) p
    }
    for (int m = 16; m > 0; m >>= 1) {
      v += __shfl_xor_sync(0xffffffffu, v, m);
      vm += __shfl_xor_sync(0xffffffffu, vm, m);
    }
    sv += v;
    sm += vm;
  }
  if (lane == 0 && (sv | sm) && c0 < c1) {
    atomicAdd((unsigned long long*)&sc->lsum_q[n], (unsigned long long)sv);
    atomicAdd((unsigned long long*)&sc->lmu_q[n], (unsigned long long)sm);
  }
}

__global__ void k_layer_totals(int N, double inv_scale_nu, DevScalars* sc) {
  for (int n = threadIdx.x; n <= N; n += blockDim.x) {
    sc->lsum[n] = (double)sc->lsum_q[n] * 0x1p-61;
    sc->lmu[n] = (double)sc->lmu_q[n] * inv_scale_nu;
  }
}

// Birth-death step on the normalised layers: lambda(n) = lambda for n < N,
// lambda(N) = 0 (loss) or lambda (queued), mu(n) = M_n / S_n; log G(n) =
// sum_{s<=n} [log lambda(s-1) - log mu(s)].  Finite buffer: lambda(n) = lambda,
// mu(n) = sum nu for n > N (Proposition 2).  Infinite: geometric tail with ratio
// lambda / sum nu (Remark).  Writes pn[0..top], fac[n] = p(n)/S_n and the queue
// quantities into summary[1,2,5,6,7].
__global__ void k_birth_death(DevScalars* sc, int N, int mode, int C, double lam, double nu_sum,
                              double* pn, double* summary) {
  if (threadIdx.x != 0) return;
  const int top = mode == HQ_FINITE ? N + C : N;
  // log G(n) in pn[] first
  pn[0] = 0.0;
  double lmax = 0.0;
  for (int n = 1; n <= top; n++) {
    double ln1, mn;
    if (n <= N) {
      ln1 = (n - 1 < N) ? lam : (mode == HQ_LOSS ? 0.0 : lam);
      mn = sc->lmu[n] / sc->lsum[n];
    } else {
      ln1 = lam;
      mn = nu_sum;
    }
    pn[n] = pn[n - 1] + log(ln1) - log(mn);
    lmax = fmax(lmax, pn[n]);
  }
  double rq = lam / nu_sum;
  double Z = 0.0;
  for (int n = 0; n <= top; n++) Z += exp(pn[n] - lmax);
  double tail = 0.0;
  if (mode == HQ_INFINITE) {
    tail = exp(pn[N] - lmax) * rq / (1.0 - rq);
    Z += tail;
  }
  for (int n = 0; n <= top; n++) pn[n] = exp(pn[n] - lmax) / Z;
  tail /= Z;
  for (int n = 0; n <= N; n++) sc->fac[n] = pn[n] / sc->lsum[n];
  double q_busy = 0.0, q_wait = 0.0, pq1 = 0.0, p_block = 0.0;
  if (mode == HQ_LOSS) {
    p_block = pn[N];
  } else if (mode == HQ_FINITE) {
    for (int c = 1; c <= C; c++) q_busy += pn[N + c];
    for (int c = 0; c < C; c++) q_wait += pn[N + c];
    pq1 = pn[N + 1];
    p_block = pn[N + C];
  } else {
    q_busy = tail;
    q_wait = pn[N] + tail;
    pq1 = pn[N] * rq;
  }
  summary[1] = p_block;
  summary[2] = q_wait;
  summary[5] = q_busy;
  summary[6] = pq1;
  summary[7] = tail;
}

struct ResArgs {
  int N, L, n, mode;
  int64_t Ln;
  int64_t tw;              // table record width of layer n
  const uint32_t* masks;   // layer n
  const uint32_t* RL;
  const uint32_t* RH;
  const double* T;         // layer n block of the FP64 table
  const double* p_dn;      // layer n-1 (or null)
  const double* p_cur;     // layer n
  const double* p_up;      // layer n+1 (or null)
  const double* nu;
  double lam_m;            // lambda_m of this layer's states
  double pq1_nusum;        // queued inflow into the all-busy state
  double* partials;
  DevScalars* sc;
};

// Eq. (1) at every state of layer n: out = P{m}(lambda_m + mu_m),
// in = sum_{busy u} P{m-u} lambda_{(m-u) m} + sum_{idle u} P{m+u} nu_u.
__global__ void __launch_bounds__(256) k_residual(ResArgs a) {
  extern __shared__ uint32_t s_RL[];
  __shared__ double snu[HQ_MAXN];
  __shared__ double s[64];
  __shared__ bool s_last;
  for (int i = threadIdx.x; i < (1 << a.L); i += blockDim.x) s_RL[i] = a.RL[i];
  if (threadIdx.x < a.N) snu[threadIdx.x] = a.nu[threadIdx.x];
  __syncthreads();
  const int n = a.n;
  const double f_dn = n > 0 ? a.sc->fac[n - 1] : 0.0;
  const double f_cur = a.sc->fac[n];
  const double f_up = n < a.N ? a.sc->fac[n + 1] : 0.0;
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double d = 0.0, o = 0.0;
  if (k < a.Ln) {
    const int L = a.L;
    uint32_t x = a.masks[k];
    uint32_t lo = x & ((1u << L) - 1u), hi = x >> L;
    int w = __popc(lo);
    const uint32_t* rh = a.RH + (size_t)hi * (L + 1);
    uint32_t rl = s_RL[lo];
    double mu = 0.0, up = 0.0, dn = 0.0;
    int s_ = 0;
    for (uint32_t y = x; y; y &= y - 1, ++s_) {
      int b = __ffs(y) - 1;
      mu += snu[b];
      uint32_t rk = (b < L) ? s_RL[lo ^ (1u << b)] + __ldg(rh + w - 1)
                            : rl + __ldg(a.RH + (size_t)(hi ^ (1u << (b - L))) * (L + 1) + w);
      up = fma(__ldg(a.p_dn + rk), __ldcs(a.T + k * a.tw + s_), up);
    }
    if (n < a.N) {
      uint32_t full = (1u << a.N) - 1u;
      for (uint32_t y = ~x & full; y; y &= y - 1) {
        int b = __ffs(y) - 1;
        uint32_t rk = (b < L) ? s_RL[lo | (1u << b)] + __ldg(rh + w + 1)
                              : rl + __ldg(a.RH + (size_t)(hi | (1u << (b - L))) * (L + 1) + w);
        dn = fma(__ldg(a.p_up + rk), snu[b], dn);
      }
    }
    double P = f_cur * a.p_cur[k];
    o = P * (a.lam_m + mu);
    double in = f_dn * up + f_up * dn + (n == a.N ? a.pq1_nusum : 0.0);
    d = fabs(o - in);
  }
  block_reduce2(d, o, true, true, s);
  if (threadIdx.x == 0) {
    a.partials[2 * (int64_t)blockIdx.x] = d;
    a.partials[2 * (int64_t)blockIdx.x + 1] = o;
  }
  if (!arrive_last_post(&a.sc->ticket[3], &s_last)) return;
  double A, B;
  fold_partials(a.partials, true, true, s, A, B);
  if (threadIdx.x == 0) {
    a.sc->res_num[n] = A;
    a.sc->res_den[n] = B;
    a.sc->ticket[3] = 0u;
  }
}

__global__ void k_residual_final(DevScalars* sc, int N, double* summary) {
  if (threadIdx.x != 0) return;
  double num = 0.0, den = 0.0;
  for (int n = 0; n <= N; n++) {
    num = fmax(num, sc->res_num[n]);
    den = fmax(den, sc->res_den[n]);
  }
  double r = num / den;
  sc->red[0] = r;
  summary[3] = r;
}

struct ScatterArgs {
  int N;
  int64_t off[HQ_MAXN + 2];  // padded layer starts
  int64_t lsize[HQ_MAXN + 1];
};

// P{B} in y-order and the normalised conditional p_n(B) in y-order
__global__ void k_scatter(ScatterArgs a, int64_t S, const uint32_t* masks, const double* p,
                          const DevScalars* sc, double* P, double* pcond) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= S) return;
  int n = 0;
  while (n < a.N && a.off[n + 1] <= g) n++;
  if (g - a.off[n] >= a.lsize[n]) return;  // padding
  uint32_t x = masks[g];
  double v = p[g];
  P[x] = sc->fac[n] * v;
  pcond[x] = v / sc->lsum[n];
}

// rho_i = sum_{B containing i} P{B}: warp w covers 32 consecutive y; bits 0..4 of
// y vary across the lanes (masked warp sums), higher bits are common to the warp.  The
// sums are in 64-bit fixed point (P at 2^61; every partial sum is at most 1), so they
// are exact integer adds rather than FP64 work.
__device__ __forceinline__ long long warp_sum_q(long long v) {
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

__global__ void k_rho_partial(int N, int64_t S, const double* P, long long* partials) {
  __shared__ long long s[HQ_THREADS / 32][HQ_MAXN];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long acc[HQ_MAXN];
#pragma unroll
  for (int i = 0; i < HQ_MAXN; i++) acc[i] = 0;
  const int64_t nwarps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid;
  for (int64_t base = gw * 32; base < S; base += nwarps_total * 32) {
    int64_t y = base + lane;
    const long long v = y < S ? __double2ll_rn(P[y] * 0x1p61) : 0;
    const long long tot = warp_sum_q(v);
#pragma unroll
    for (int i = 0; i < 5; i++) {
      const long long t = warp_sum_q(((y >> i) & 1) ? v : 0);
      if (i < N) acc[i] += t;
    }
#pragma unroll
    for (int i = 5; i < HQ_MAXN; i++)
      if (i < N && ((base >> i) & 1)) acc[i] += tot;
  }
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < HQ_MAXN; i++) s[wid][i] = acc[i];
  }
  __syncthreads();
  if (threadIdx.x < N) {
    long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += s[w][threadIdx.x];
    partials[(int64_t)blockIdx.x * HQ_MAXN + threadIdx.x] = t;
  }
}

__global__ void k_rho_final(int N, int nblk, const long long* partials, const double* summary,
                            double* rho) {
  int i = threadIdx.x;
  if (i >= N) return;
  long long t = 0;
  for (int b = 0; b < nblk; b++) t += partials[(int64_t)b * HQ_MAXN + i];
  rho[i] = (double)t * 0x1p-61 + summary[5];  // queued states: every unit busy
}

// F[B] = P{B} in 64-bit fixed point P 2^61, y-order (P <= 1 and every superset sum of P
// is <= 1, so the sums are exact integer adds; the quantum 2^-62 is far below the
// outputs' accuracy)
__global__ void k_fill_fixed(int64_t S, const double* P, long long* F) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < S) F[g] = __double2ll_rn(P[g] * 0x1p61);
}

// R[j*N+i] = sum of P over the states with every unit node j prefers to i busy and unit
// i idle = F[pre] - F[pre + i] with F the superset sums of P (exact integers), plus
// waiting calls served by i
__global__ void k_response(int N, int J, int mode, const uint32_t* pre, const long long* F,
                           const double* nu, double nu_sum, const double* summary, double* R) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (int64_t)J * N) return;
  int i = (int)(g % N);
  const uint32_t m = pre[g];
  double v = (double)(F[m] - F[m | (1u << i)]) * 0x1p-61;
  if (mode != HQ_LOSS) v += summary[2] * nu[i] / nu_sum;
  R[g] = v;
}

__global__ void k_workload(int N, int J, const double* lam_j, const double* nu, const double* R,
                           double* W) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (int64_t)J * N) return;
  int i = (int)(g / J), j = (int)(g % J);
  W[g] = lam_j[j] * R[(int64_t)j * N + i] / nu[i];
}

__global__ void k_summary(int N, const double* nu, const double* rho, const double* pn,
                          double* summary) {
  if (threadIdx.x != 0) return;
  double thr = 0.0;
  for (int i = 0; i < N; i++) thr += nu[i] * rho[i];
  double busy = 0.0;
  for (int n = 0; n <= N; n++) busy += n * pn[n];
  summary[0] = thr;
  summary[4] = busy + N * summary[5];
}

}  // namespace

template <class V>
static int layer_sums_typed(hq_solver* h) {
  const typename V::T* p = (const typename V::T*)hq_bufs(h, V::kind).p;
  LayerSumArgs a;
  a.N = h->N;
  for (int i = 0; i < HQ_MAXN + 2; i++) a.off[i] = h->off[i];
  for (int i = 0; i <= HQ_MAXN; i++) a.lsize[i] = i <= h->N ? h->lsize[i] : 0;
  int ex = 0;
  frexp(h->nu_sum > 0.0 ? h->nu_sum : 1.0, &ex);  // sum nu < 2^ex: mu_m p < 2^61 at 2^(61-ex)
  a.scale_nu = ldexp(1.0, 61 - ex);
  HQ_CUDA(cudaMemsetAsync(h->sc->lsum_q, 0, sizeof(long long) * 2 * (HQ_MAXN + 1), h->stream));
  const int64_t chunks = h->Sp >> 5;
  const int64_t want = (chunks + 7) / 8;  // 8 warps per CTA
  const unsigned grid = (unsigned)(want < 152 * 8 ? (want > 0 ? want : 1) : 152 * 8);
  k_layer_sum<V><<<grid, 256, 0, h->stream>>>(a, h->masks, p, h->nu, h->sc);
  HQ_LAUNCHED();
  k_layer_totals<<<1, 32, 0, h->stream>>>(h->N, 1.0 / a.scale_nu, h->sc);
  HQ_LAUNCHED();
  return HQ_OK;
}

int hq_layer_sums(hq_solver* h, int prec) {
  if (prec == HQ_PREC_FP64) return layer_sums_typed<PolF64>(h);
  if (prec == HQ_PREC_DF64) return layer_sums_typed<PolDF>(h);
  return layer_sums_typed<PolF32>(h);
}

// p64 <- current iterate; layer totals; birth-death; residual of Eq. (1)
static int prepare_fp64(hq_solver* h) {
  if (h->cur_prec != HQ_PREC_FP64) {
    int saved = h->cur_prec;
    int rc = hq_convert_iterate(h, saved, HQ_PREC_FP64, false);
    if (rc != HQ_OK) return rc;
    h->cur_prec = saved;  // the iterate still lives in its own precision
  }
  int rc = hq_layer_sums(h, HQ_PREC_FP64);
  if (rc != HQ_OK) return rc;
  k_birth_death<<<1, 32, 0, h->stream>>>(h->sc, h->N, h->mode, h->C, h->lam, h->nu_sum, h->pn,
                                         h->summary);
  HQ_LAUNCHED();
  return HQ_OK;
}

static int residual_pass(hq_solver* h) {
  const double* p = (const double*)h->b64.p;
  const double* T = (const double*)h->b64.T;
  double pq1_nusum = 0.0;
  if (h->mode != HQ_LOSS) {
    // pq1 lives in summary[6] on the device; fold it in through a tiny copy
    // into the per-launch argument is not possible, so read it back once
    double v = 0.0;
    HQ_CUDA(cudaMemcpyAsync(&v, h->summary + 6, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    HQ_CUDA(cudaStreamSynchronize(h->stream));
    pq1_nusum = v * h->nu_sum;
  }
  // layers 1..N-1 in one pass with the sweep's gather (fused kernel, hq_persist.cu); it
  // zeroes every layer's maxima first.  Layers 0 and N (one state each) by k_residual.
  int rc = hq_residual_fused(h);
  if (rc != HQ_OK) return rc;
  for (int n = 0; n <= h->N; n++) {
    if (h->N >= 2 && n > 0 && n < h->N) continue;
    ResArgs a;
    a.N = h->N;
    a.L = h->L;
    a.n = n;
    a.mode = h->mode;
    a.Ln = h->lsize[n];
    a.tw = h->tw[n];
    a.masks = h->masks + h->off[n];
    a.RL = h->RL;
    a.RH = h->RH;
    a.T = n >= 1 ? T + h->toff[n] : T;
    a.p_dn = n >= 1 ? p + h->off[n - 1] : p;
    a.p_cur = p + h->off[n];
    a.p_up = n < h->N ? p + h->off[n + 1] : p;
    a.nu = h->nu;
    a.lam_m = (n == h->N && h->mode == HQ_LOSS) ? 0.0 : h->lam;
    a.pq1_nusum = pq1_nusum;
    a.partials = h->partials;
    a.sc = h->sc;
    k_residual<<<(unsigned)((a.Ln + 255) / 256), 256, sizeof(uint32_t) << h->L, h->stream>>>(a);
    HQ_LAUNCHED();
  }
  k_residual_final<<<1, 32, 0, h->stream>>>(h->sc, h->N, h->summary);
  HQ_LAUNCHED();
  return HQ_OK;
}

int hq_compute_residual(hq_solver* h, double* residual_out) {
  int rc = prepare_fp64(h);
  if (rc != HQ_OK) return rc;
  rc = residual_pass(h);
  if (rc != HQ_OK) return rc;
  h->res_version = h->it_version;
  double r = 0.0;
  HQ_CUDA(cudaMemcpyAsync(&r, h->summary + 3, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  HQ_CUDA(cudaStreamSynchronize(h->stream));
  *residual_out = r;
  return HQ_OK;
}

int hq_finalize(hq_solver* h, int prec, bool full_outputs, double* residual_out) {
  (void)prec;
  int rc = HQ_OK;
  // a residual check of this very iterate already left the FP64 iterate, the layer law
  // and the residual in place
  if (h->res_version != h->it_version) {
    rc = prepare_fp64(h);
    if (rc != HQ_OK) return rc;
    rc = residual_pass(h);
    if (rc != HQ_OK) return rc;
    h->res_version = h->it_version;
  }
  if (full_outputs) {
    ScatterArgs sa;
    sa.N = h->N;
    for (int i = 0; i < HQ_MAXN + 2; i++) sa.off[i] = h->off[i];
    for (int i = 0; i <= HQ_MAXN; i++) sa.lsize[i] = i <= h->N ? h->lsize[i] : 0;
    unsigned grid = (unsigned)((h->Sp + 255) / 256);
    k_scatter<<<grid, 256, 0, h->stream>>>(sa, h->Sp, h->masks, (const double*)h->b64.p, h->sc, h->P,
                                           h->pcond);
    HQ_LAUNCHED();
    int64_t want = (h->S + 255) / 256;
    int nblk = (int)(want < 152 * 8 ? want : 152 * 8);
    k_rho_partial<<<nblk, 256, 0, h->stream>>>(h->N, h->S, h->P, (long long*)h->partials);
    HQ_LAUNCHED();
    k_rho_final<<<1, 32, 0, h->stream>>>(h->N, nblk, (const long long*)h->partials, h->summary, h->rho);
    HQ_LAUNCHED();
    // one superset-sum transform of P over all N bits (in the transform scratch, which
    // holds N 2^(N-1) >= 2^N values): every response probability is a difference of two
    // of its entries
    k_fill_fixed<<<(unsigned)((h->S + 255) / 256), 256, 0, h->stream>>>(h->S, h->P, (long long*)h->zeta);
    HQ_LAUNCHED();
    rc = hq_zeta_subset(h, (long long*)h->zeta, h->N, 1, true);
    if (rc != HQ_OK) return rc;
    int64_t jn = (int64_t)h->J * h->N;
    k_response<<<(unsigned)((jn + 255) / 256), 256, 0, h->stream>>>(
        h->N, h->J, h->mode, h->pre, (const long long*)h->zeta, h->nu, h->nu_sum, h->summary, h->R);
    HQ_LAUNCHED();
    k_workload<<<(unsigned)((jn + 255) / 256), 256, 0, h->stream>>>(h->N, h->J, h->lam_j, h->nu,
                                                                  h->R, h->W);
    HQ_LAUNCHED();
    k_summary<<<1, 32, 0, h->stream>>>(h->N, h->nu, h->rho, h->pn, h->summary);
    HQ_LAUNCHED();
  }
  double r = 0.0;
  HQ_CUDA(cudaMemcpyAsync(&r, h->summary + 3, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  HQ_CUDA(cudaStreamSynchronize(h->stream));
  if (residual_out) *residual_out = r;
  return HQ_OK;
}

// Layer-ranked state layout of the hypercube (layers C_n of Section 2.2).
//
// The 2^N states are grouped by the number of busy units n; inside layer n the
// C(N,n) states are ordered colexicographically, which for n-subsets is the
// increasing order of their bitmask.  A state's rank inside its layer is
// rank(x) = sum_t C(c_t, t+1) over its busy units c_0 < c_1 < ... (the
// combinatorial number system).  Ranks are evaluated through a split table:
// with x = (hi, lo), lo the low L bits and w = popc(lo),
//     rank(x) = RL[lo] + RH[hi][w],
// RL[lo] = sum over lo's busy units, RH[hi][w] = sum_k C(L + pos_k, w + k + 1)
// over hi's busy units pos_k.  A one-bit neighbour of x therefore costs two
// table reads, and states that share hi (contiguous in colex order) find their
// hi-flip neighbours at contiguous ranks.
#include <math.h>

#include <vector>

#include "hq_internal.cuh"

double hq_binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; i++) r = r * (double)(n - k + i) / (double)i;
  return floor(r + 0.5);
}

struct BinomTable {
  uint32_t c[33][33];
};

static BinomTable make_binom_table() {
  BinomTable t;
  for (int n = 0; n <= 32; n++)
    for (int k = 0; k <= 32; k++) t.c[n][k] = k > n ? 0u : (uint32_t)hq_binom(n, k);
  return t;
}

struct LayoutArgs {
  int N;
  int64_t off[HQ_MAXN + 2];    // padded layer starts
  int64_t lsize[HQ_MAXN + 1];
};

// colex unrank: state mask of global layer-ranked index g (padding slots get 0)
__global__ void k_masks(LayoutArgs a, BinomTable bt, uint32_t* masks, int64_t S) {
  __shared__ uint32_t sb[33][33];
  for (int i = threadIdx.x; i < 33 * 33; i += blockDim.x) sb[i / 33][i % 33] = bt.c[i / 33][i % 33];
  __syncthreads();
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= S) return;
  int n = 0;
  while (n < a.N && a.off[n + 1] <= g) n++;
  if (g - a.off[n] >= a.lsize[n]) {
    masks[g] = 0u;
    return;
  }
  uint32_t k = (uint32_t)(g - a.off[n]);
  uint32_t x = 0;
  int c = a.N - 1;
  for (int t = n; t >= 1; t--) {
    while (sb[c][t] > k) c--;
    x |= 1u << c;
    k -= sb[c][t];
    c--;
  }
  masks[g] = x;
}

__global__ void k_rank_lo(int L, BinomTable bt, uint32_t* RL) {
  uint32_t lo = blockIdx.x * blockDim.x + threadIdx.x;
  if (lo >= (1u << L)) return;
  uint32_t r = 0;
  int t = 0;
  for (int b = 0; b < L; b++)
    if ((lo >> b) & 1u) {
      r += bt.c[b][t + 1];
      t++;
    }
  RL[lo] = r;
}

__global__ void k_rank_hi(int L, int H, BinomTable bt, uint32_t* RH) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t total = ((int64_t)1 << H) * (L + 1);
  if (i >= total) return;
  uint32_t hi = (uint32_t)(i / (L + 1));
  int w = (int)(i % (L + 1));
  uint32_t r = 0;
  int k = 0;
  for (int b = 0; b < H; b++)
    if ((hi >> b) & 1u) {
      int pos = L + b;
      int idx = w + k + 1;
      r += idx <= 32 ? bt.c[pos][idx] : 0u;
      k++;
    }
  RH[i] = r;
}

int hq_build_layout(hq_solver* h) {
  const int N = h->N;
  BinomTable bt = make_binom_table();
  LayoutArgs a;
  a.N = N;
  for (int i = 0; i < HQ_MAXN + 2; i++) a.off[i] = h->off[i];
  for (int i = 0; i <= HQ_MAXN; i++) a.lsize[i] = i <= N ? h->lsize[i] : 0;
  int64_t S = h->Sp;
  k_masks<<<(unsigned)((S + 255) / 256), 256, 0, h->stream>>>(a, bt, h->masks, S);
  HQ_LAUNCHED();
  k_rank_lo<<<(unsigned)(((1u << h->L) + 255) / 256), 256, 0, h->stream>>>(h->L, bt, h->RL);
  HQ_LAUNCHED();
  int64_t tot = ((int64_t)1 << h->H) * (h->L + 1);
  k_rank_hi<<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>(h->L, h->H, bt, h->RH);
  HQ_LAUNCHED();
  return HQ_OK;
}

// ---------------------------------------------------------------------------
// instance validation on the device (inputs that already live in HBM) and the
// region-wide totals lambda = sum_j lambda_j, sum_i nu_i in a fixed order.
// flag bits: 1 bad lambda_j, 2 bad nu_i, 4 preference row not a permutation
// ---------------------------------------------------------------------------
__global__ void k_validate(int N, int J, const double* lam_j, const double* nu,
                           const int32_t* pref, int* flag, double* totals) {
  __shared__ double s[1024];
  int bad = 0;
  double acc = 0.0;
  for (int j = threadIdx.x; j < J; j += blockDim.x) {
    double v = lam_j[j];
    if (!(v >= 0.0) || isinf(v)) bad |= 1;
    acc += v;
    uint32_t seen = 0;
    for (int hh = 0; hh < N; hh++) {
      int u = pref[(int64_t)j * N + hh];
      if (u < 0 || u >= N || ((seen >> u) & 1u)) bad |= 4;
      else seen |= 1u << u;
    }
  }
  if (threadIdx.x < N) {
    double v = nu[threadIdx.x];
    if (!(v > 0.0) || isinf(v)) bad |= 2;
  }
  if (bad) atomicOr(flag, bad);
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    totals[0] = s[0];
    double t = 0.0;
    for (int i = 0; i < N; i++) t += nu[i];
    totals[1] = t;
  }
}

int hq_validate_device(hq_solver* h) {
  HQ_CUDA(cudaMemsetAsync(h->dflag, 0, sizeof(int), h->stream));
  k_validate<<<1, 1024, 0, h->stream>>>(h->N, h->J, h->lam_j, h->nu, h->pref, h->dflag,
                                        h->summary);
  HQ_LAUNCHED();
  int flag = 0;
  double tot[2];
  HQ_CUDA(cudaMemcpyAsync(&flag, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  HQ_CUDA(cudaMemcpyAsync(tot, h->summary, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  HQ_CUDA(cudaStreamSynchronize(h->stream));
  if (flag & 1) { hq_set_error("lambda_j must be finite and >= 0"); return HQ_EINVAL; }
  if (flag & 2) { hq_set_error("nu_i must be finite and > 0"); return HQ_EINVAL; }
  if (flag & 4) { hq_set_error("each preference row must be a permutation of 0..N-1"); return HQ_EINVAL; }
  h->lam = tot[0];
  h->nu_sum = tot[1];
  return HQ_OK;
}

// ---------------------------------------------------------------------------
// r_m = 1 / (lambda_m + mu_m), layer-ranked, in the three precisions.
// lambda_m = lambda except the all-busy state of the loss system (0).
// ---------------------------------------------------------------------------
__global__ void k_rates(LayoutArgs la, int64_t S, const uint32_t* masks, const double* nu, double lam,
                        double lam_full, double* r64, float2* rdf, float* r32) {
  const int N = la.N;
  __shared__ double snu[HQ_MAXN];
  if (threadIdx.x < N) snu[threadIdx.x] = nu[threadIdx.x];
  __syncthreads();
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= S) return;
  int n = 0;
  while (n < N && la.off[n + 1] <= g) n++;
  if (g - la.off[n] >= la.lsize[n]) return;  // padding keeps its zeros
  uint32_t x = masks[g];
  double mu = 0.0;
  for (uint32_t y = x; y; y &= y - 1) mu += snu[__ffs(y) - 1];
  double lm = (n == N) ? lam_full : lam;
  double r = 1.0 / (lm + mu);
  r64[g] = r;
  if (rdf) rdf[g] = df_from_double(r);
  r32[g] = (float)r;
}

__global__ void k_nu_prec(int N, const double* nu, float2* nudf, float* nu32) {
  int i = threadIdx.x;
  if (i < N) {
    nudf[i] = df_from_double(nu[i]);
    nu32[i] = (float)nu[i];
  }
}

int hq_build_rates(hq_solver* h) {
  double lam_full = h->mode == HQ_LOSS ? 0.0 : h->lam;
  LayoutArgs la;
  la.N = h->N;
  for (int i = 0; i < HQ_MAXN + 2; i++) la.off[i] = h->off[i];
  for (int i = 0; i <= HQ_MAXN; i++) la.lsize[i] = i <= h->N ? h->lsize[i] : 0;
  k_rates<<<(unsigned)((h->Sp + 255) / 256), 256, 0, h->stream>>>(
      la, h->Sp, h->masks, h->nu, h->lam, lam_full, (double*)h->b64.r, (float2*)h->bdf.r,
      (float*)h->b32.r);
  HQ_LAUNCHED();
  HQ_CUDA(cudaMemcpyAsync(h->b64.nu, h->nu, sizeof(double) * h->N, cudaMemcpyDeviceToDevice,
                          h->stream));
  k_nu_prec<<<1, 32, 0, h->stream>>>(h->N, h->nu, (float2*)h->bdf.nu, (float*)h->b32.nu);
  HQ_LAUNCHED();
  return HQ_OK;
}

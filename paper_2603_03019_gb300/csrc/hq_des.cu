// Discrete-event simulation of the loss system with general service times, the check of
// Section 5.5 ("Results for General Service Time Distributions"): the stationary
// solution of the exponential model is exact for the loss system under any service
// distribution with the same means (insensitivity), so utilisations and the mean
// response time from a simulation with log-normal, gamma or uniform service times must
// agree with it.  One GPU thread simulates one replication from an empty system; the
// replications are independent, so they are the data-parallel axis.
//
// Model, per replication: Poisson arrivals of rate lambda = sum_j lambda_j; node j with
// probability lambda_j / lambda (binary search of the cumulative rates); the first idle
// unit of node j's preference list serves the call (Section 2.1's dispatch rule); a call
// that finds every unit busy is lost.  Unit i's service time has mean m = 1/nu_i and
// shape `kind`: 0 exponential, 1 log-normal with the exponential's variance, 2 gamma
// of shape 5 (scale m/5, a sum of five exponentials), 3 gamma of shape 1/2 (m Z^2, Z
// standard normal), 4 uniform on [0, 2m]; normals by the Box-Muller transform.
//
// Random numbers come from one counter-based generator so that each replication's
// stream does not depend on scheduling: x = F(key_r + (c + 1) gamma) with F the
// splitmix64 finaliser (Steele, Lea & Flood, OOPSLA 2014), gamma = 0x9e3779b97f4a7c15,
// key_r = F(seed + (r + 1) gamma), u = ((x >> 11) + 1) 2^-53 in (0, 1]; draw c = 8 a + k
// of arrival a: k = 0 inter-arrival time, 1 node, 2..6 service time.  Every FP64 step
// is written with explicit round-to-nearest operations (no contraction into FMA), so the
// trajectory depends only on the math functions' last-bit rounding.
#include "hq_internal.cuh"

namespace {

constexpr int kDesMaxN = 32;
constexpr int kDesThreads = 64;
constexpr uint64_t kGamma = 0x9e3779b97f4a7c15ULL;

__device__ __forceinline__ uint64_t des_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double des_u(uint64_t key, uint64_t c) {
  const uint64_t x = des_mix(key + (c + 1) * kGamma);
  return __dmul_rn((double)((x >> 11) + 1), 0x1.0p-53);
}

__device__ __forceinline__ double des_normal(double u1, double u2) {
  const double two_pi = 6.283185307179586476925286766559;
  return __dmul_rn(sqrt(__dmul_rn(-2.0, log(u1))), cos(__dmul_rn(two_pi, u2)));
}

__device__ double des_service(int kind, double m, uint64_t key, uint64_t c0) {
  const double u2 = des_u(key, c0), u3 = des_u(key, c0 + 1);
  switch (kind) {
    case 0:
      return __dmul_rn(-m, log(u2));
    case 1: {
      const double s2 = log(2.0);
      const double mu = __dsub_rn(log(m), __dmul_rn(0.5, s2));
      return exp(__dadd_rn(mu, __dmul_rn(sqrt(s2), des_normal(u2, u3))));
    }
    case 2: {
      double prod = __dmul_rn(u2, u3);
      prod = __dmul_rn(prod, des_u(key, c0 + 2));
      prod = __dmul_rn(prod, des_u(key, c0 + 3));
      prod = __dmul_rn(prod, des_u(key, c0 + 4));
      return __dmul_rn(-__ddiv_rn(m, 5.0), log(prod));
    }
    case 3: {
      const double z = des_normal(u2, u3);
      return __dmul_rn(m, __dmul_rn(z, z));
    }
    default:
      return __dmul_rn(__dmul_rn(2.0, m), u2);
  }
}

// cumulative node rates, summed in node order by one thread (the oracle's order)
__global__ void k_des_cdf(int J, const double* lam_j, double* cdf) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double acc = 0.0;
  for (int j = 0; j < J; j++) {
    acc = __dadd_rn(acc, lam_j[j]);
    cdf[j] = acc;
  }
}

struct DesArgs {
  int N, J, kind;
  int64_t reps, arrivals, warmup;
  uint64_t seed;
  const double* cdf;
  const double* nu;
  const int32_t* pref;
  const double* travel;
  double* busy;     // reps x N
  int64_t* served;  // reps x N
  int64_t* lost;    // reps
  double* window;   // reps
  double* resp;     // reps
};

__global__ void __launch_bounds__(kDesThreads) k_des_loss(DesArgs a) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= a.reps) return;
  const int N = a.N, J = a.J;
  const double lam = __ldg(a.cdf + J - 1);
  const uint64_t key = des_mix(a.seed + (uint64_t)(r + 1) * kGamma);
  double fr[kDesMaxN], busy[kDesMaxN];
  int64_t served[kDesMaxN];
  for (int i = 0; i < N; i++) {
    fr[i] = 0.0;
    busy[i] = 0.0;
    served[i] = 0;
  }
  int64_t lost = 0;
  double resp = 0.0, t = 0.0, t0 = 0.0;
  for (int64_t k = 0; k < a.arrivals; k++) {
    const uint64_t c = 8 * (uint64_t)k;
    t = __dadd_rn(t, __ddiv_rn(-log(des_u(key, c)), lam));
    const bool in_window = k >= a.warmup;
    if (k == a.warmup) {
      t0 = t;
      for (int i = 0; i < N; i++)
        if (fr[i] > t0) busy[i] = __dsub_rn(fr[i], t0);
    }
    const double target = __dmul_rn(des_u(key, c + 1), lam);
    int lo = 0, hi = J - 1;
    while (lo < hi) {
      const int mid = (lo + hi) / 2;
      if (__ldg(a.cdf + mid) >= target) hi = mid;
      else lo = mid + 1;
    }
    const int j = lo;
    int unit = -1;
    for (int h = 0; h < N; h++) {
      const int i = __ldg(a.pref + (int64_t)j * N + h);
      if (fr[i] <= t) {
        unit = i;
        break;
      }
    }
    if (unit < 0) {
      if (in_window) lost++;
      continue;
    }
    const double s = des_service(a.kind, __ddiv_rn(1.0, __ldg(a.nu + unit)), key, c + 2);
    fr[unit] = __dadd_rn(t, s);
    if (in_window) {
      busy[unit] = __dadd_rn(busy[unit], s);
      served[unit]++;
      resp = __dadd_rn(resp, __ldg(a.travel + (int64_t)j * N + unit));
    }
  }
  for (int i = 0; i < N; i++) {
    if (fr[i] > t) busy[i] = __dsub_rn(busy[i], __dsub_rn(fr[i], t));
    a.busy[r * N + i] = busy[i];
    a.served[r * N + i] = served[i];
  }
  a.lost[r] = lost;
  a.window[r] = __dsub_rn(t, t0);
  a.resp[r] = resp;
}

__global__ void k_des_check(int N, int J, const double* lam_j, const double* nu, const int32_t* pref, int* flag) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < N) {
    const double v = nu[j];
    if (!(v > 0.0) || isinf(v)) atomicOr(flag, 2);
  }
  if (j >= J) return;
  const double l = lam_j[j];
  if (!(l >= 0.0) || isinf(l)) atomicOr(flag, 2);
  uint64_t seen = 0;
  for (int h = 0; h < N; h++) {
    const int u = pref[(int64_t)j * N + h];
    if (u < 0 || u >= N || ((seen >> u) & 1ull)) {
      atomicOr(flag, 1);
      return;
    }
    seen |= 1ull << u;
  }
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

}  // namespace

extern "C" int hq_des_simulate(int N, int J, const double* lambda_j, const double* nu, const int32_t* pref,
                               const double* travel, int service_kind, int64_t reps, int64_t arrivals,
                               int64_t warmup, uint64_t seed, double* busy, int64_t* served, int64_t* lost,
                               double* window, double* resp, int mem, void* stream) {
  if (N < 1 || N > kDesMaxN || J < 1) {
    hq_set_error("hq_des_simulate: N must be in 1..32 and J >= 1");
    return HQ_EINVAL;
  }
  if (service_kind < 0 || service_kind > 4 || reps < 1 || reps > ((int64_t)1 << 31) || arrivals < 2 ||
      warmup < 0 || warmup >= arrivals - 1) {
    hq_set_error("hq_des_simulate: service_kind in 0..4, reps >= 1, arrivals >= 2, 0 <= warmup < arrivals - 1");
    return HQ_EINVAL;
  }
  if (!lambda_j || !nu || !pref || !travel || !busy || !served || !lost || !window || !resp) {
    hq_set_error("hq_des_simulate: NULL pointer");
    return HQ_EINVAL;
  }
  if (mem != HQ_HOST && mem != HQ_DEVICE) {
    hq_set_error("hq_des_simulate: mem must be HQ_HOST or HQ_DEVICE");
    return HQ_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nJ = (size_t)J, nN = (size_t)N, nJN = nJ * nN, nR = (size_t)reps;
  // device copies of host inputs, device outputs for host callers, the cumulative rates
  DevBuf b_in, b_out, b_cdf;
  const double *d_lam = lambda_j, *d_nu = nu, *d_travel = travel;
  const int32_t* d_pref = pref;
  double *d_busy = busy, *d_window = window, *d_resp = resp;
  int64_t *d_served = served, *d_lost = lost;
  const size_t in_bytes = 8 * nJ + 8 * nN + 4 * nJN + 8 * nJN + 16;
  const size_t out_bytes = 8 * nR * nN + 8 * nR * nN + 8 * nR * 3 + 64;
  HQ_CUDA(cudaMalloc(&b_cdf.p, 8 * nJ + 16));
  if (mem == HQ_HOST) {
    HQ_CUDA(cudaMalloc(&b_in.p, in_bytes));
    HQ_CUDA(cudaMalloc(&b_out.p, out_bytes));
    char* q = (char*)b_in.p;
    double* lam_d = (double*)q;
    q += 8 * nJ;
    double* nu_d = (double*)q;
    q += 8 * nN;
    double* tr_d = (double*)q;
    q += 8 * nJN;
    int32_t* pr_d = (int32_t*)q;
    HQ_CUDA(cudaMemcpyAsync(lam_d, lambda_j, 8 * nJ, cudaMemcpyHostToDevice, st));
    HQ_CUDA(cudaMemcpyAsync(nu_d, nu, 8 * nN, cudaMemcpyHostToDevice, st));
    HQ_CUDA(cudaMemcpyAsync(tr_d, travel, 8 * nJN, cudaMemcpyHostToDevice, st));
    HQ_CUDA(cudaMemcpyAsync(pr_d, pref, 4 * nJN, cudaMemcpyHostToDevice, st));
    d_lam = lam_d;
    d_nu = nu_d;
    d_travel = tr_d;
    d_pref = pr_d;
    char* o = (char*)b_out.p;
    d_busy = (double*)o;
    o += 8 * nR * nN;
    d_served = (int64_t*)o;
    o += 8 * nR * nN;
    d_lost = (int64_t*)o;
    o += 8 * nR;
    d_window = (double*)o;
    o += 8 * nR;
    d_resp = (double*)o;
  }
  int* d_flag = (int*)((double*)b_cdf.p + nJ);
  HQ_CUDA(cudaMemsetAsync(d_flag, 0, sizeof(int), st));
  const int chk = J > N ? J : N;
  k_des_check<<<(chk + 127) / 128, 128, 0, st>>>(N, J, d_lam, d_nu, d_pref, d_flag);
  HQ_LAUNCHED();
  int host_flag = 0;
  HQ_CUDA(cudaMemcpyAsync(&host_flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  HQ_CUDA(cudaStreamSynchronize(st));
  if (host_flag & 1) {
    hq_set_error("hq_des_simulate: a preference row is not a permutation of 0..N-1");
    return HQ_EINVAL;
  }
  if (host_flag & 2) {
    hq_set_error("hq_des_simulate: lambda_j must be finite and >= 0, nu finite and > 0");
    return HQ_EINVAL;
  }
  k_des_cdf<<<1, 32, 0, st>>>(J, d_lam, (double*)b_cdf.p);
  HQ_LAUNCHED();
  DesArgs a;
  a.N = N;
  a.J = J;
  a.kind = service_kind;
  a.reps = reps;
  a.arrivals = arrivals;
  a.warmup = warmup;
  a.seed = seed;
  a.cdf = (const double*)b_cdf.p;
  a.nu = d_nu;
  a.pref = d_pref;
  a.travel = d_travel;
  a.busy = d_busy;
  a.served = d_served;
  a.lost = d_lost;
  a.window = d_window;
  a.resp = d_resp;
  k_des_loss<<<(unsigned)((reps + kDesThreads - 1) / kDesThreads), kDesThreads, 0, st>>>(a);
  HQ_LAUNCHED();
  if (mem == HQ_HOST) {
    HQ_CUDA(cudaMemcpyAsync(busy, d_busy, 8 * nR * nN, cudaMemcpyDeviceToHost, st));
    HQ_CUDA(cudaMemcpyAsync(served, d_served, 8 * nR * nN, cudaMemcpyDeviceToHost, st));
    HQ_CUDA(cudaMemcpyAsync(lost, d_lost, 8 * nR, cudaMemcpyDeviceToHost, st));
    HQ_CUDA(cudaMemcpyAsync(window, d_window, 8 * nR, cudaMemcpyDeviceToHost, st));
    HQ_CUDA(cudaMemcpyAsync(resp, d_resp, 8 * nR, cudaMemcpyDeviceToHost, st));
  }
  HQ_CUDA(cudaStreamSynchronize(st));
  return HQ_OK;
}

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
// key_r = F(seed + (r + 1) gamma); draw c = 8 a + k of arrival a: k = 0 inter-arrival
// time, 1 node, 2..6 service time.  The node's uniform is ((x >> 11) + 1) 2^-53 in
// (0, 1]; the variates' are ((x >> 40) + 1) 2^-24, exact in FP32.
//
// The variates are FP32 (their relative rounding, about 1e-7, is far below any
// statistical effect), built with a logarithm, an exponential and a cosine written here
// from their series, every step one explicit round-to-nearest operation; the clock and
// the sums are FP64.  On this GPU the FP32 pipe is many times faster than the FP64 one,
// and the same steps in the CPU oracle give every replication the same trajectory.
//
// What remains FP64 in the loop is kept off the FP64 pipe where an exact integer form
// exists: the node search compares the node's 53-bit draw with per-node integer
// thresholds (K_j = the largest k with RN(k 2^-53 lambda) <= cdf_j, so "cdf_j >= the
// target" is "K_j >= k"), starting from a guide table (Chen and Asau's method: the
// first node of each of 1024 equal ranges of k); FP32 values widen to FP64 by moving
// their bits; the free-unit scan compares the bit patterns of non-negative
// finite doubles, which order as integers; the unit's mean 1/nu_i and its derived
// constants are a per-unit table.  The part of a service time that does not depend on
// the unit is drawn at the top of the loop with the next inter-arrival time and node
// (three independent chains the scheduler interleaves) and finished once the unit is
// known; a lost call's draw is wasted.  Each replication's trajectory is unchanged.
#include "hq_internal.cuh"

namespace {

constexpr int kDesMaxN = 32;
constexpr int kDesThreads = 64;
constexpr int kGuideBits = 10;  // the guide table: 2^10 ranges of the 53-bit node draw
constexpr uint64_t kGamma = 0x9e3779b97f4a7c15ULL;

__device__ __forceinline__ uint64_t des_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

// the node's uniform is k 2^-53 with k = (x >> 11) + 1 in 1..2^53; the search uses k itself
__device__ __forceinline__ uint64_t des_k53(uint64_t key, uint64_t c) {
  const uint64_t x = des_mix(key + (c + 1) * kGamma);
  return (x >> 11) + 1;
}

__device__ __forceinline__ float des_u24(uint64_t key, uint64_t c) {
  const uint64_t x = des_mix(key + (c + 1) * kGamma);
  return __fmul_rn((float)((x >> 40) + 1), 0x1.0p-24f);
}

// the FP64 value of an FP32 x (exact), by moving its bits: sign, exponent rebased from
// 127 to 1023, fraction shifted to the top; a subnormal x is normalised first
__device__ __forceinline__ double des_widen(float x) {
  const uint32_t b = __float_as_uint(x);
  const uint64_t sign = (uint64_t)(b >> 31) << 63;
  int e = (int)((b >> 23) & 0xffu);
  uint32_t m = b & 0x7fffffu;
  if (e == 0) {
    if (m == 0) return __longlong_as_double((long long)sign);
    const int sh = __clz(m) - 8;
    m = (m << sh) & 0x7fffffu;
    e = 1 - sh;
  }
  return __longlong_as_double((long long)(sign | ((uint64_t)(e + 896) << 52) | ((uint64_t)m << 29)));
}

// a * b + c with two roundings (never contracted into one FMA)
__device__ __forceinline__ float mad2(float a, float b, float c) { return __fadd_rn(__fmul_rn(a, b), c); }

// ln x for a positive normal x: x = m 2^e, m in [sqrt(1/2), sqrt(2)), ln m = 2 atanh(s)
// = 2 (s + s^3/3 + s^5/5 + s^7/7 + s^9/9), s = (m - 1)/(m + 1); e ln 2 by Cody and Waite's
// split (a 16-bit high part, so its product with e is exact)
__device__ float des_ln(float x) {
  const uint32_t b = __float_as_uint(x);
  int e = (int)((b >> 23) & 0xffu) - 127;
  float m = __uint_as_float((b & 0x7fffffu) | 0x3f800000u);
  if (m > 0x1.6a09e6p+0f) {
    m = __fmul_rn(m, 0.5f);
    e += 1;
  }
  const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
  const float z = __fmul_rn(s, s);
  float q = 0x1.c71c72p-4f;
  q = mad2(q, z, 0x1.24924ap-3f);
  q = mad2(q, z, 0x1.99999ap-3f);
  q = mad2(q, z, 0x1.555556p-2f);
  q = mad2(q, z, 1.0f);
  const float lnm = __fmul_rn(__fadd_rn(s, s), q);
  const float ef = (float)e;
  const float lo = mad2(ef, 0x1.7f7d1cp-20f, lnm);
  return mad2(ef, 0x1.62e4p-1f, lo);
}

// e^y: y = k ln 2 + r, |r| <= ln2 / 2, e^r from its Taylor series to r^8 / 8!
__device__ float des_exp(float y) {
  const float k = floorf(mad2(y, 0x1.715476p+0f, 0.5f));
  float r = __fsub_rn(y, __fmul_rn(k, 0x1.62e4p-1f));
  r = __fsub_rn(r, __fmul_rn(k, 0x1.7f7d1cp-20f));
  float p = 0x1.a01a02p-16f;
  p = mad2(p, r, 0x1.a01a02p-13f);
  p = mad2(p, r, 0x1.6c16c2p-10f);
  p = mad2(p, r, 0x1.111112p-7f);
  p = mad2(p, r, 0x1.555556p-5f);
  p = mad2(p, r, 0x1.555556p-3f);
  p = mad2(p, r, 0.5f);
  p = mad2(p, r, 1.0f);
  p = mad2(p, r, 1.0f);
  return __fmul_rn(p, __uint_as_float((uint32_t)((int)k + 127) << 23));
}

// cos(2 pi u), u in [0, 1]: symmetries to w in [0, 1/4]; the Taylor series of cos (angle
// <= pi/4, to a^10 / 10!) or of the sine of the complement (to b^9 / 9!)
__device__ float des_cos2pi(float u) {
  float v = u;
  if (v > 0.5f) v = __fsub_rn(1.0f, v);
  float sign = 1.0f;
  if (v > 0.25f) {
    v = __fsub_rn(0.5f, v);
    sign = -1.0f;
  }
  float c;
  if (v <= 0.125f) {
    const float a = __fmul_rn(0x1.921fb6p+2f, v);
    const float a2 = __fmul_rn(a, a);
    float p = -0x1.27e4fcp-22f;
    p = mad2(p, a2, 0x1.a01a02p-16f);
    p = __fsub_rn(__fmul_rn(p, a2), 0x1.6c16c2p-10f);
    p = mad2(p, a2, 0x1.555556p-5f);
    p = __fsub_rn(__fmul_rn(p, a2), 0.5f);
    c = mad2(p, a2, 1.0f);
  } else {
    const float bb = __fmul_rn(0x1.921fb6p+2f, __fsub_rn(0.25f, v));
    const float b2 = __fmul_rn(bb, bb);
    float p = 0x1.71de3ap-19f;
    p = __fsub_rn(__fmul_rn(p, b2), 0x1.a01a02p-13f);
    p = mad2(p, b2, 0x1.111112p-7f);
    p = __fsub_rn(__fmul_rn(p, b2), 0x1.555556p-3f);
    p = mad2(p, b2, 1.0f);
    c = __fmul_rn(bb, p);
  }
  return __fmul_rn(sign, c);
}

__device__ __forceinline__ float des_normal(float u1, float u2) {
  return __fmul_rn(__fsqrt_rn(__fmul_rn(-2.0f, des_ln(u1))), des_cos2pi(u2));
}

// The log-normal's variance parameter: ln 2, the exponential's variance for a unit mean
constexpr float kLnS2 = 0x1.62e43p-1f;

// The unit-independent part g of a service time from draws c0.. (Section 5.5's shapes):
// exponential ln u; log-normal a standard normal; gamma of shape 5 ln of the product of
// five uniforms; gamma of shape 1/2 Z^2; uniform u.
template <int kKind>
__device__ __forceinline__ float des_shape(uint64_t key, uint64_t c0) {
  const float u2 = des_u24(key, c0);
  if (kKind == 0) return des_ln(u2);
  if (kKind == 4) return u2;
  const float u3 = des_u24(key, c0 + 1);
  if (kKind == 1) return des_normal(u2, u3);
  if (kKind == 3) {
    const float z = des_normal(u2, u3);
    return __fmul_rn(z, z);
  }
  float prod = __fmul_rn(u2, u3);
  prod = __fmul_rn(prod, des_u24(key, c0 + 2));
  prod = __fmul_rn(prod, des_u24(key, c0 + 3));
  prod = __fmul_rn(prod, des_u24(key, c0 + 4));
  return des_ln(prod);
}

// The per-unit constant pu of a service time of mean m: m for the exponential and the
// gamma of shape 1/2, ln m - s^2/2 for the log-normal, m/5 for the gamma of shape 5, 2m
// for the uniform.
__device__ __forceinline__ float des_unit_const(int kind, float m) {
  switch (kind) {
    case 1:
      return __fsub_rn(des_ln(m), __fmul_rn(0.5f, kLnS2));
    case 2:
      return __fdiv_rn(m, 5.0f);
    case 4:
      return __fmul_rn(2.0f, m);
    default:
      return m;
  }
}

// the service time from its per-unit constant and its shape part
template <int kKind>
__device__ __forceinline__ float des_finish(float pu, float g) {
  if (kKind == 0 || kKind == 2) return __fmul_rn(-pu, g);
  if (kKind == 1) return des_exp(__fadd_rn(pu, __fmul_rn(__fsqrt_rn(kLnS2), g)));
  return __fmul_rn(pu, g);
}

// cumulative node rates, summed in node order by one thread (the oracle's order); bit 2
// of the flag if the total rate is outside [2^-60, 2^60]
__global__ void k_des_cdf(int J, const double* lam_j, double* cdf, int* flag) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double acc = 0.0;
  for (int j = 0; j < J; j++) {
    acc = __dadd_rn(acc, lam_j[j]);
    cdf[j] = acc;
  }
  if (!(acc >= 0x1.0p-60 && acc <= 0x1.0p+60)) atomicOr(flag, 4);
}

// Per node the integer threshold K_j = max{k in 0..2^53 : RN(RN(k 2^-53) lambda) <= cdf_j}
// (a binary search: the product is non-decreasing in k); per unit the service constant.
__global__ void k_des_prep(int N, int J, int kind, const double* cdf, const double* nu, uint64_t* kth,
                           float* pu) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < N) pu[j] = des_unit_const(kind, __double2float_rn(__ddiv_rn(1.0, nu[j])));
  if (j >= J) return;
  const double lam = cdf[J - 1], cj = cdf[j];
  uint64_t lo = 0, hi = 1ull << 53;
  while (lo < hi) {
    const uint64_t mid = hi - ((hi - lo) >> 1);
    if (__dmul_rn(__dmul_rn((double)mid, 0x1.0p-53), lam) <= cj) lo = mid;
    else hi = mid - 1;
  }
  kth[j] = lo;
}

// guide[b] = the first node j with K_j >= b 2^(53 - kGuideBits) + 1, the smallest draw of
// range b (K_{J-1} = 2^53, so it exists)
__global__ void k_des_guide(int J, const uint64_t* kth, int32_t* guide) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= (1 << kGuideBits)) return;
  const uint64_t kmin = ((uint64_t)b << (53 - kGuideBits)) + 1;
  int lo = 0, hi = J - 1;
  while (lo < hi) {
    const int mid = (lo + hi) / 2;
    if (kth[mid] >= kmin) hi = mid;
    else lo = mid + 1;
  }
  guide[b] = lo;
}

struct DesArgs {
  int N, J, kind;
  int64_t reps, arrivals, warmup;
  uint64_t seed;
  const double* cdf;
  const uint64_t* kth;  // J node thresholds
  const int32_t* guide; // 2^kGuideBits starting nodes
  const float* pu;      // N per-unit service constants
  const int32_t* pref;
  const double* travel;
  double* busy;     // reps x N
  int64_t* served;  // reps x N
  int64_t* lost;    // reps
  double* window;   // reps
  double* resp;     // reps
};

template <int kKind>
__global__ void __launch_bounds__(kDesThreads) k_des_loss(DesArgs a) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= a.reps) return;
  const int N = a.N, J = a.J;
  const float lamf = __double2float_rn(__ldg(a.cdf + J - 1));
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
    // three independent chains: inter-arrival time, node draw, the service time's shape
    const float dt = __fdiv_rn(-des_ln(des_u24(key, c)), lamf);
    const uint64_t kn = des_k53(key, c + 1);
    const float g = des_shape<kKind>(key, c + 2);
    t = __dadd_rn(t, des_widen(dt));
    const bool in_window = k >= a.warmup;
    if (k == a.warmup) {
      t0 = t;
      for (int i = 0; i < N; i++)
        if (fr[i] > t0) busy[i] = __dsub_rn(fr[i], t0);
    }
    // the first node with K_j >= kn, from its range's first candidate (K_{J-1} = 2^53)
    int j = __ldg(a.guide + ((kn - 1) >> (53 - kGuideBits)));
    while (j < J - 1 && __ldg(a.kth + j) < kn) j++;
    // fr and t are finite and >= +0, so their bit patterns order as integers
    const long long tb = __double_as_longlong(t);
    int unit = -1;
    for (int h = 0; h < N; h++) {
      const int i = __ldg(a.pref + (int64_t)j * N + h);
      if (__double_as_longlong(fr[i]) <= tb) {
        unit = i;
        break;
      }
    }
    if (unit < 0) {
      if (in_window) lost++;
      continue;
    }
    const double s = des_widen(des_finish<kKind>(__ldg(a.pu + unit), g));
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
    if (!(v >= 0x1.0p-60 && v <= 0x1.0p+60)) atomicOr(flag, 2);
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
  // cumulative rates (J), node thresholds (J), unit constants (32 floats), guide table,
  // the flag
  HQ_CUDA(cudaMalloc(&b_cdf.p, 16 * nJ + 4 * kDesMaxN + 4 * (1 << kGuideBits) + 16));
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
  double* d_cdf = (double*)b_cdf.p;
  uint64_t* d_kth = (uint64_t*)(d_cdf + nJ);
  float* d_pu = (float*)(d_kth + nJ);
  int32_t* d_guide = (int32_t*)(d_pu + kDesMaxN);
  int* d_flag = (int*)(d_guide + (1 << kGuideBits));
  HQ_CUDA(cudaMemsetAsync(d_flag, 0, sizeof(int), st));
  const int chk = J > N ? J : N;
  k_des_check<<<(chk + 127) / 128, 128, 0, st>>>(N, J, d_lam, d_nu, d_pref, d_flag);
  HQ_LAUNCHED();
  k_des_cdf<<<1, 32, 0, st>>>(J, d_lam, d_cdf, d_flag);
  HQ_LAUNCHED();
  int host_flag = 0;
  HQ_CUDA(cudaMemcpyAsync(&host_flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  HQ_CUDA(cudaStreamSynchronize(st));
  if (host_flag & 1) {
    hq_set_error("hq_des_simulate: a preference row is not a permutation of 0..N-1");
    return HQ_EINVAL;
  }
  if (host_flag & 6) {
    hq_set_error("hq_des_simulate: lambda_j must be finite and >= 0 with a total in [2^-60, 2^60], "
                 "nu in [2^-60, 2^60]");
    return HQ_EINVAL;
  }
  k_des_prep<<<(chk + 127) / 128, 128, 0, st>>>(N, J, service_kind, d_cdf, d_nu, d_kth, d_pu);
  HQ_LAUNCHED();
  k_des_guide<<<(1 << kGuideBits) / 128, 128, 0, st>>>(J, d_kth, d_guide);
  HQ_LAUNCHED();
  DesArgs a;
  a.N = N;
  a.J = J;
  a.kind = service_kind;
  a.reps = reps;
  a.arrivals = arrivals;
  a.warmup = warmup;
  a.seed = seed;
  a.cdf = d_cdf;
  a.kth = d_kth;
  a.pu = d_pu;
  a.guide = d_guide;
  a.pref = d_pref;
  a.travel = d_travel;
  a.busy = d_busy;
  a.served = d_served;
  a.lost = d_lost;
  a.window = d_window;
  a.resp = d_resp;
  const unsigned grid = (unsigned)((reps + kDesThreads - 1) / kDesThreads);
  switch (service_kind) {
    case 0:
      k_des_loss<0><<<grid, kDesThreads, 0, st>>>(a);
      break;
    case 1:
      k_des_loss<1><<<grid, kDesThreads, 0, st>>>(a);
      break;
    case 2:
      k_des_loss<2><<<grid, kDesThreads, 0, st>>>(a);
      break;
    case 3:
      k_des_loss<3><<<grid, kDesThreads, 0, st>>>(a);
      break;
    default:
      k_des_loss<4><<<grid, kDesThreads, 0, st>>>(a);
  }
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

// Allocation-free build of the upward-rate table, for callers that must not
// allocate device memory themselves: code that runs under an external memory
// manager (a framework's caching pool or a fixed device-memory budget that
// every buffer must come from), or latency-sensitive loops where a cudaMalloc,
// which can synchronise the whole device, is not acceptable.
//
// The caller passes the instance (device memory) and the output table (device
// memory).  The arithmetic is the regular load's: every lambda_j is quantised to 64-bit
// fixed point at the same power-of-two scale and summed by integer adds, so the table is
// bitwise the one hq_load builds.  The working memory of the transform -- the per-unit
// subset-sum buffers, the preference-prefix masks, an error word and the scale -- lives in one
// file-scope device array of fixed size, so this file never calls cudaMalloc,
// cudaFree or any allocating library routine.  Limits: N <= 16 units,
// J <= 4096 nodes (4.25 MiB of static device memory, held by every device that
// loads the library until the process exits).
//
// Every call shares that one array and leaves its contents behind; each call
// clears what must start at zero.  Two calls that overlap on the GPU (for
// example on two streams without ordering between them) race on the array and
// give wrong results: order them on one stream or synchronise between them.
#include <mutex>

#include "hq_internal.cuh"

#define HQ_STATIC_MAX_N 16
#define HQ_STATIC_MAX_J 4096
// layout of the array (units of 8 bytes):
//   [0, 16 * 2^15)                     subset-sum buffers, unit u at u * 2^(N-1)
//   next HQ_STATIC_MAX_J * 16 / 2      prefix masks (uint32, J x N)
//   next 32                            error word, the fixed-point scale and its inverse
#define HQ_STATIC_ZETA_WORDS ((size_t)HQ_STATIC_MAX_N << (HQ_STATIC_MAX_N - 1))
#define HQ_STATIC_PRE_WORDS ((size_t)HQ_STATIC_MAX_J * HQ_STATIC_MAX_N / 2)
#define HQ_STATIC_WORDS (HQ_STATIC_ZETA_WORDS + HQ_STATIC_PRE_WORDS + 32)

static __device__ __align__(256) double g_hq_static_scratch[HQ_STATIC_WORDS];

namespace {

std::mutex g_setup_mutex;
double* g_scratch_addr[256] = {nullptr};  // device address of the array, per device

__device__ __forceinline__ uint32_t st_squeeze(uint32_t x, int u) {
  return (x & ((1u << u) - 1u)) | ((x >> (u + 1)) << u);
}

// prefix masks: pre[j*N + u] = units node j ranks before u; bad rows raise flag
__global__ void k_st_prefix(int N, int J, const int32_t* pref, uint32_t* pre, int* flag) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= J) return;
  for (int u = 0; u < N; u++) pre[(int64_t)j * N + u] = 0u;
  uint32_t acc = 0, seen = 0;
  for (int h = 0; h < N; h++) {
    int u = pref[(int64_t)j * N + h];
    if (u < 0 || u >= N || ((seen >> u) & 1u)) {
      atomicOr(flag, 1);
      continue;
    }
    seen |= 1u << u;
    pre[(int64_t)j * N + u] = acc;
    acc |= 1u << u;
  }
}

__global__ void k_st_check_rates(int J, const double* lam_j, int* flag) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= J) return;
  double v = lam_j[j];
  if (!(v >= 0.0) || isinf(v)) atomicOr(flag, 2);
}

// lambda = sum_j lambda_j in the order the regular load uses (1024 threads, strided
// partials, then a halving tree), and from it the same power-of-two fixed-point scale
// 2^(61 - e), lambda < 2^e, so that both builds quantise every rate identically
__global__ void k_st_scale(int J, const double* lam_j, double* scale2) {
  __shared__ double s[1024];
  double acc = 0.0;
  for (int j = threadIdx.x; j < J; j += blockDim.x) acc += lam_j[j];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int ex = 0;
    frexp(s[0] > 0.0 ? s[0] : 1.0, &ex);
    scale2[0] = ldexp(1.0, 61 - ex);
    scale2[1] = ldexp(1.0, ex - 61);
  }
}

// per-unit histograms in 64-bit fixed point: exact integer adds, order-free
__global__ void k_st_hist(int N, int J, const uint32_t* pre, const double* lam_j, const double* scale2,
                          long long* zeta) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (int64_t)J * N) return;
  const int j = (int)(g / N), u = (int)(g % N);
  const uint32_t key = st_squeeze(pre[g], u);
  const long long q = __double2ll_rn(lam_j[j] * scale2[0]);
  if (q) atomicAdd((unsigned long long*)(zeta + ((int64_t)u << (N - 1)) + key), (unsigned long long)q);
}

// one bit of the subset-sum transform over all N buffers (integer adds)
__global__ void k_st_zeta_bit(int N, int b, long long* zeta) {
  const int64_t half = (int64_t)1 << (N - 1);
  const int64_t pairs = (half >> 1) * N;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < pairs;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = q / (half >> 1), r = q % (half >> 1);
    const int64_t lo = ((r >> b) << (b + 1)) | (r & ((1ll << b) - 1));
    long long* F = zeta + u * half;
    F[lo | (1ll << b)] += F[lo];
  }
}

// pull-form emit with an on-the-fly colex unrank (no mask buffer)
__global__ void k_st_emit(int N, const long long* zeta, const double* scale2, double* T) {
  __shared__ uint32_t bc[HQ_STATIC_MAX_N + 1][HQ_STATIC_MAX_N + 2];
  for (int i = threadIdx.x; i < (HQ_STATIC_MAX_N + 1) * (HQ_STATIC_MAX_N + 2); i += blockDim.x) {
    int a = i / (HQ_STATIC_MAX_N + 2), k = i % (HQ_STATIC_MAX_N + 2);
    uint32_t c = 0;
    if (k <= a) {
      c = 1;
      for (int t = 1; t <= k; t++) c = c * (uint32_t)(a - k + t) / (uint32_t)t;
    }
    bc[a][k] = c;
  }
  __syncthreads();
  const int64_t S = (int64_t)1 << N;
  const int64_t half = S >> 1;
  for (int64_t g = 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < S;
       g += (int64_t)gridDim.x * blockDim.x) {
    // layer n of global index g, its offsets in the state and table layouts
    int n = 1;
    int64_t off = 1, toff = 0;
    while (off + bc[N][n] <= g) {
      off += bc[N][n];
      toff += (int64_t)n * bc[N][n];
      n++;
    }
    const int64_t Ln = bc[N][n];
    uint32_t k = (uint32_t)(g - off);
    uint32_t x = 0;
    int c = N - 1;
    for (int t = n; t >= 1; t--) {
      while (bc[c][t] > k) c--;
      x |= 1u << c;
      k -= bc[c][t];
      c--;
    }
    const int64_t rank = g - off;
    int s = 0;
    for (uint32_t y = x; y; y &= y - 1, s++) {
      const int u = __ffs(y) - 1;
      T[toff + (int64_t)s * Ln + rank] = (double)zeta[(int64_t)u * half + st_squeeze(x, u)] * scale2[1];
    }
  }
}

// device address of the array on the current device; first call per device only
int static_scratch(double** out) {
  int dev = 0;
  HQ_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) {
    hq_set_error("device ordinal out of range");
    return HQ_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_hq_static_scratch);
    if (e != cudaSuccess || !p) return hq_cuda_fail(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
    g_scratch_addr[dev] = (double*)p;
  }
  *out = g_scratch_addr[dev];
  return HQ_OK;
}

}  // namespace

extern "C" int hq_dispatch_table_static(int N, int J, const double* lambda_j, const int32_t* pref,
                                        double* T, void* stream) {
  if (N < 1 || N > HQ_STATIC_MAX_N) {
    hq_set_error("hq_dispatch_table_static: N must be in 1..16 (size of its static scratch)");
    return HQ_EINVAL;
  }
  if (J < 1 || J > HQ_STATIC_MAX_J) {
    hq_set_error("hq_dispatch_table_static: J must be in 1..4096 (size of its static scratch)");
    return HQ_EINVAL;
  }
  if (!lambda_j || !pref || !T) {
    hq_set_error("hq_dispatch_table_static: NULL pointer");
    return HQ_EINVAL;
  }
  double* base = nullptr;
  int rc = static_scratch(&base);
  if (rc != HQ_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  long long* zeta = (long long*)base;
  uint32_t* pre = (uint32_t*)(base + HQ_STATIC_ZETA_WORDS);
  int* flag = (int*)(base + HQ_STATIC_ZETA_WORDS + HQ_STATIC_PRE_WORDS);
  double* scale2 = base + HQ_STATIC_ZETA_WORDS + HQ_STATIC_PRE_WORDS + 2;
  const int64_t half = (int64_t)1 << (N - 1);
  // what must start at zero: the error word and the N subset-sum buffers
  HQ_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
  HQ_CUDA(cudaMemsetAsync(zeta, 0, sizeof(long long) * half * N, st));
  k_st_prefix<<<(J + 127) / 128, 128, 0, st>>>(N, J, pref, pre, flag);
  HQ_LAUNCHED();
  k_st_check_rates<<<(J + 127) / 128, 128, 0, st>>>(J, lambda_j, flag);
  HQ_LAUNCHED();
  k_st_scale<<<1, 1024, 0, st>>>(J, lambda_j, scale2);
  HQ_LAUNCHED();
  k_st_hist<<<(unsigned)(((int64_t)J * N + 255) / 256), 256, 0, st>>>(N, J, pre, lambda_j, scale2, zeta);
  HQ_LAUNCHED();
  for (int b = 0; b + 1 < N; b++) {
    int64_t pairs = (half >> 1) * N;
    unsigned grid = (unsigned)((pairs + 255) / 256 < 2048 ? (pairs + 255) / 256 : 2048);
    k_st_zeta_bit<<<grid, 256, 0, st>>>(N, b, zeta);
    HQ_LAUNCHED();
  }
  const int64_t states = ((int64_t)1 << N) - 1;
  unsigned grid = (unsigned)((states + 255) / 256 < 2048 ? (states + 255) / 256 : 2048);
  k_st_emit<<<grid, 256, 0, st>>>(N, zeta, scale2, T);
  HQ_LAUNCHED();
  int host_flag = 0;
  HQ_CUDA(cudaMemcpyAsync(&host_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  HQ_CUDA(cudaStreamSynchronize(st));
  if (host_flag & 1) {
    hq_set_error("hq_dispatch_table_static: a preference row is not a permutation of 0..N-1");
    return HQ_EINVAL;
  }
  if (host_flag & 2) {
    hq_set_error("hq_dispatch_table_static: lambda_j must be finite and >= 0");
    return HQ_EINVAL;
  }
  return HQ_OK;
}

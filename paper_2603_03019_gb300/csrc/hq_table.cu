// Upward transition rates of Eq. (3), built once per instance into a pull-form,
// layer-ranked table.
//
// For a target state m with unit u busy, the rate of the upward move
// (m - u) -> m is
//     lambda_u(m - u) = sum_j lambda_j [all units node j ranks before u are busy in m]
// (u is then node j's first idle unit in m - u: the reading of Eq. (3) stated in
// the sentence that follows it, and the prefix walk of Algorithm 3).  With
// pre_j(u) the set of units node j prefers to u and
//     g_u(S) = sum_{j : pre_j(u) = S} lambda_j     (S a subset of the other N-1 units),
// the rate is the subset sum F_u(X) = sum_{S subset of X} g_u(S) at X = m - u.  So the
// whole table is N histograms plus N subset-sum (zeta) transforms over N-1 bits:
// O(N^2 2^N) work independent of J, instead of one first-idle search per
// (state, node) pair.  The sums are exact: each lambda_j is quantised once to 64-bit
// fixed point (a power-of-two scale that keeps lambda = sum_j lambda_j below 2^61,
// so the quantum is ~2^-62 lambda) and every sum after that is an integer add, which
// also keeps the transform off GB300's slow FP64 pipe.  The emit converts to FP64 in
// the pull layout (FP32 and double-float copies follow from it)
//     T[toff(n) + k HQ_TW(n) + s] = F_{c_s}(m_k - c_s),
// m_k the rank-k state of layer n and c_s its s-th busy unit, so the sweep reads
// slot s of consecutive states contiguously.
#include "hq_internal.cuh"

// remove bit u from x (x has bit u clear or it is ignored)
__device__ __forceinline__ uint32_t squeeze_bit(uint32_t x, int u) {
  uint32_t low = x & ((1u << u) - 1u);
  return low | ((x >> (u + 1)) << u);
}

// pre[j*N + u] = units node j ranks before unit u
__global__ void k_prefix_masks(int N, int J, const int32_t* pref, uint32_t* pre) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= J) return;
  uint32_t acc = 0;
  for (int h = 0; h < N; h++) {
    int u = pref[(int64_t)j * N + h];
    pre[(int64_t)j * N + u] = acc;
    acc |= 1u << u;
  }
}

// g_u histograms: one thread per (node j, unit u) adds round(lambda_j scale) (scale a
// power of two) to F_u[pre_j(u) without bit u].  The adds are integer atomics, so the
// sums are exact and do not depend on their order: O(J N) work, deterministic.
__global__ void k_histogram(int N, int J, const uint32_t* pre, const double* lam_j, double scale,
                            long long* zeta) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (int64_t)J * N) return;
  const int j = (int)(g / N), u = (int)(g % N);
  const int64_t half = (int64_t)1 << (N - 1);
  const uint32_t key = squeeze_bit(__ldg(pre + g), u);
  const long long q = __double2ll_rn(__ldg(lam_j + j) * scale);
  if (q) atomicAdd((unsigned long long*)(zeta + (int64_t)u * half + key), (unsigned long long)q);
}

// ---------------------------------------------------------------------------
// subset-sum (zeta) transform F(X) = sum_{S subset X} f(S), or the superset
// version F(X) = sum_{S superset X} f(S), over `bits` bits for `count` arrays
// laid end to end, of 64-bit fixed-point values (exact integer adds).  Pass 1
// handles the low bits inside a shared-memory tile of contiguous elements; later
// passes handle groups of high bits with tiles made of 2^g strided rows of kCols
// contiguous elements.
// ---------------------------------------------------------------------------
constexpr int kLowLog = 12;            // first pass: tiles of 4096 contiguous elements (32 KB)
constexpr int kLowThreads = 256;
constexpr int kTileLog = 14;           // later passes: tiles of 16384 elements (128 KB)
constexpr int kMinColsLog = 3;         // rows of at least 8 contiguous elements (64 B)
constexpr int kHighThreads = 1024;

__global__ void k_zeta_low(long long* buf, int bits, int tile_log, int64_t ntiles, bool superset) {
  extern __shared__ long long t[];
  int64_t tile = blockIdx.x;
  if (tile >= ntiles) return;
  int64_t tsize = (int64_t)1 << tile_log;
  long long* base = buf + tile * tsize;
  for (int64_t i = threadIdx.x; i < tsize; i += blockDim.x) t[i] = base[i];
  __syncthreads();
  int nb = bits < tile_log ? bits : tile_log;
  for (int b = 0; b < nb; b++) {
    int64_t bit = (int64_t)1 << b;
    for (int64_t q = threadIdx.x; q < tsize / 2; q += blockDim.x) {
      int64_t lo = ((q >> b) << (b + 1)) | (q & (bit - 1));
      int64_t hi = lo | bit;
      if (superset) t[lo] += t[hi];
      else t[hi] += t[lo];
    }
    __syncthreads();
  }
  for (int64_t i = threadIdx.x; i < tsize; i += blockDim.x) base[i] = t[i];
}

// bits [b0, b0+g) of each array; tile = 2^g rows (stride 2^b0) x 2^cols_log columns
__global__ void k_zeta_high(long long* buf, int bits, int b0, int g, int cols_log, int64_t per_array,
                            int64_t tiles_per_array, int count, bool superset) {
  extern __shared__ long long t[];
  int64_t tid = blockIdx.x;
  int a = (int)(tid / tiles_per_array);
  if (a >= count) return;
  int64_t tix = tid % tiles_per_array;
  // tix enumerates (column block within 2^b0, position above b0+g)
  int64_t colblocks = ((int64_t)1 << b0) >> cols_log;
  int64_t cb = tix % colblocks;
  int64_t above = tix / colblocks;
  long long* arr = buf + (int64_t)a * per_array;
  int64_t start = (above << (b0 + g)) + (cb << cols_log);
  int rows = 1 << g, cols = 1 << cols_log;
  int64_t stride = (int64_t)1 << b0;
  for (int i = threadIdx.x; i < rows * cols; i += blockDim.x) {
    int r = i >> cols_log, c = i & (cols - 1);
    t[i] = arr[start + r * stride + c];
  }
  __syncthreads();
  for (int b = 0; b < g; b++) {
    int bit = 1 << b;
    for (int q = threadIdx.x; q < (rows / 2) * cols; q += blockDim.x) {
      int rq = q >> cols_log, c = q & (cols - 1);
      int rlo = ((rq >> b) << (b + 1)) | (rq & (bit - 1));
      int rhi = rlo | bit;
      int ilo = (rlo << cols_log) | c, ihi = (rhi << cols_log) | c;
      if (superset) t[ilo] += t[ihi];
      else t[ihi] += t[ilo];
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < rows * cols; i += blockDim.x) {
    int r = i >> cols_log, c = i & (cols - 1);
    arr[start + r * stride + c] = t[i];
  }
  (void)bits;
}

// Pass 1 takes the low 12 bits; every later pass takes as many of the remaining bits as
// fit a full 16384-element tile with rows of at least 8 contiguous elements, and widens
// the rows when fewer bits remain (N=24: 12 + 11 bits in two passes; N=28: 12 + 11 + 4
// with 1024-element rows), so no pass degenerates into many tiny tiles.
int hq_zeta_subset(hq_solver* h, long long* buf, int bits, int count, bool superset) {
  if (bits <= 0) return HQ_OK;
  int64_t per = (int64_t)1 << bits;
  int tl = bits < kLowLog ? bits : kLowLog;
  int64_t ntiles = (per >> tl) * count;
  size_t smem = sizeof(long long) << tl;
  const int smax = (int)(sizeof(long long) << kTileLog);
  HQ_CUDA(cudaFuncSetAttribute(k_zeta_low, cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
  HQ_CUDA(cudaFuncSetAttribute(k_zeta_high, cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
  k_zeta_low<<<(unsigned)ntiles, kLowThreads, smem, h->stream>>>(buf, bits, tl, ntiles, superset);
  HQ_LAUNCHED();
  int b0 = tl;
  while (b0 < bits) {
    int g = bits - b0;
    if (g > kTileLog - kMinColsLog) g = kTileLog - kMinColsLog;
    int cols_log = kTileLog - g;
    if (cols_log > b0) cols_log = b0;
    int64_t colblocks = ((int64_t)1 << b0) >> cols_log;
    int64_t above = per >> (b0 + g);
    int64_t tpa = colblocks * above;
    size_t sm = sizeof(long long) << (g + cols_log);
    k_zeta_high<<<(unsigned)(tpa * count), kHighThreads, sm, h->stream>>>(buf, bits, b0, g, cols_log, per,
                                                                tpa, count, superset);
    HQ_LAUNCHED();
    b0 += g;
  }
  return HQ_OK;
}

struct EmitArgs {
  int N;
  int64_t off[HQ_MAXN + 2];   // padded layer starts
  int64_t toff[HQ_MAXN + 2];  // padded table layer starts
  int64_t lsize[HQ_MAXN + 1];
  int64_t tw[HQ_MAXN + 1];    // record width (state-major layout, HQ_TW)
};

// one thread per state of layers 1..N: slot s <- F_{c_s}(m - c_s) / scale, in FP64 and
// its FP32 copy
__global__ void k_emit(EmitArgs a, int64_t S, const uint32_t* masks, const long long* zeta, double inv_scale,
                       double* T64, float* T32) {
  int64_t g = a.off[1] + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= S) return;
  int n = 1;
  while (n < a.N && a.off[n + 1] <= g) n++;
  int64_t k = g - a.off[n];
  if (k >= a.lsize[n]) return;  // padding
  const int64_t rec = a.toff[n] + k * a.tw[n];
  int64_t half = (int64_t)1 << (a.N - 1);
  uint32_t x = masks[g];
  int s = 0;
  for (uint32_t y = x; y; y &= y - 1, s++) {
    int u = __ffs(y) - 1;
    const double v = (double)__ldg(zeta + (int64_t)u * half + squeeze_bit(x, u)) * inv_scale;
    T64[rec + s] = v;
    T32[rec + s] = (float)v;
  }
}

int hq_build_table(hq_solver* h) {
  const int N = h->N, J = h->J;
  int64_t half = (int64_t)1 << (N - 1);
  k_prefix_masks<<<(J + 255) / 256, 256, 0, h->stream>>>(N, J, h->pref, h->pre);
  HQ_LAUNCHED();
  // the fixed-point scale 2^e keeps every sum (at most lambda) below 2^61
  int ex = 0;
  frexp(h->lam > 0.0 ? h->lam : 1.0, &ex);  // lambda < 2^ex
  const int e = 61 - ex;
  const double scale = ldexp(1.0, e);  // exact powers of two: the scaling is exact
  long long* z = (long long*)h->zeta;
  HQ_CUDA(cudaMemsetAsync(z, 0, sizeof(long long) * half * N, h->stream));
  k_histogram<<<(unsigned)(((int64_t)J * N + 255) / 256), 256, 0, h->stream>>>(N, J, h->pre, h->lam_j, scale, z);
  HQ_LAUNCHED();
  int rc = hq_zeta_subset(h, z, N - 1, N, false);
  if (rc != HQ_OK) return rc;
  EmitArgs a;
  a.N = N;
  for (int i = 0; i < HQ_MAXN + 2; i++) {
    a.off[i] = h->off[i];
    a.toff[i] = h->toff[i];
  }
  for (int i = 0; i <= HQ_MAXN; i++) {
    a.lsize[i] = i <= N ? h->lsize[i] : 0;
    a.tw[i] = i <= N ? h->tw[i] : 0;
  }
  int64_t cnt = h->Sp - h->off[1];
  k_emit<<<(unsigned)((cnt + 255) / 256), 256, 0, h->stream>>>(
      a, h->Sp, h->masks, z, 1.0 / scale, (double*)h->b64.T, (float*)h->b32.T);
  HQ_LAUNCHED();
  return HQ_OK;
}

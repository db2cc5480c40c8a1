// Learned warm start (not in the paper): a small MLP that predicts, for every layer n
// and unit i, q_i(n) = P(unit i busy | n units busy) from features of the instance,
// trained on solves of the method itself; the prediction seeds Algorithm 1 with the
// layer-wise product form
//     p_n(B) = prod_{i in B} x_i(n) / e_n(x(n)),   x_i(n) = q_i(n) / (1 - q_i(n)),
// e_n the elementary symmetric polynomial of degree n (the per-layer normaliser), in
// place of the paper's uniform start 1 / C(N, n).
//
// Network (weights shared across units and layers, so one model serves every N; input
// F = 9: the unit's 8 features and n / N):
//   z1 = x W1 + b1,  a1 = relu(z1)   (F -> Hd, FP32 arithmetic: K = F is tiny)
//   z2 = a1 W2 + b2, a2 = relu(z2)   (Hd -> Hd, BF16 operands, FP32 accumulate, mma)
//   y  = a2 W3 + b3                  (Hd -> 1, FP32)
// y estimates logit(q_i(n)).  Activations a1, a2 are stored in BF16 (the rounding points
// the CPU reference of the gradient check reproduces); master weights are FP32 with
// BF16 copies for the tensor-core product.  Loss: mean squared error of y against
// logit(q) over the batch; optimiser: Adam.
//
// The Hd x Hd products run on the tensor cores with warp-level mma.sync BF16 tiles
// (m16n8k16): they are a few hundred MFLOP per training step, far from mattering next to
// the solver, so the simpler warp-level instruction is used instead of tcgen05.
#include <math.h>
#include <string.h>

#include <vector>

#include "hq_internal.cuh"

namespace {

constexpr int kF = HQ_MLP_FEATURES;

__device__ __forceinline__ uint16_t f2bf(float f) {
  // round to nearest even (NaN inputs do not occur: all values are finite)
  uint32_t u = __float_as_uint(f);
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
__device__ __forceinline__ float bf2f(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

// ---- tiled BF16 GEMM on mma.sync: C[M x N] (FP32) = op(A)[M x K] op(B)[K x N] ---------
// A: if TA, stored K x M row-major (element (m, k) at A[k * lda + m]), else M x K.
// B: if TB, stored N x K row-major (element (k, n) at B[n * ldb + k]), else K x N.
// CTA tile 64 x 64, K step 32, 4 warps of 32 x 32; out-of-range elements read as 0.
constexpr int kTM = 64, kTN = 64, kTK = 32;

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(128) k_gemm_bf16(int M, int N, int K, const uint16_t* A, int lda,
                                                   const uint16_t* B, int ldb, float* C, int ldc) {
  __shared__ uint16_t As[kTM][kTK + 8];  // (m, k)
  __shared__ uint16_t Bs[kTK][kTN + 8];  // (k, n)
  const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int g = lane >> 2, t = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
      for (int q = 0; q < 4; q++) acc[i][j][q] = 0.f;
  for (int k0 = 0; k0 < K; k0 += kTK) {
    for (int e = tid; e < kTM * kTK; e += 128) {
      const int mm = e / kTK, kk = e % kTK;
      const int gm = m0 + mm, gk = k0 + kk;
      uint16_t v = 0;
      if (gm < M && gk < K) v = TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
      As[mm][kk] = v;
    }
    for (int e = tid; e < kTK * kTN; e += 128) {
      const int kk = e / kTN, nn = e % kTN;
      const int gk = k0 + kk, gn = n0 + nn;
      uint16_t v = 0;
      if (gk < K && gn < N) v = TB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < kTK; ks += 16) {
      uint32_t af[2][4], bfr[4][2];
#pragma unroll
      for (int i = 0; i < 2; i++) {
        const int r = wm + i * 16 + g, c = ks + t * 2;
        af[i][0] = (uint32_t)As[r][c] | ((uint32_t)As[r][c + 1] << 16);
        af[i][1] = (uint32_t)As[r + 8][c] | ((uint32_t)As[r + 8][c + 1] << 16);
        af[i][2] = (uint32_t)As[r][c + 8] | ((uint32_t)As[r][c + 9] << 16);
        af[i][3] = (uint32_t)As[r + 8][c + 8] | ((uint32_t)As[r + 8][c + 9] << 16);
      }
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const int cn = wn + j * 8 + g, r = ks + t * 2;
        bfr[j][0] = (uint32_t)Bs[r][cn] | ((uint32_t)Bs[r + 1][cn] << 16);
        bfr[j][1] = (uint32_t)Bs[r + 8][cn] | ((uint32_t)Bs[r + 9][cn] << 16);
      }
#pragma unroll
      for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) mma_bf16(acc[i][j], af[i], bfr[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int r = m0 + wm + i * 16 + g, c = n0 + wn + j * 8 + t * 2;
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const int rr = r + (q >= 2 ? 8 : 0), cc = c + (q & 1);
        if (rr < M && cc < N) C[(size_t)rr * ldc + cc] = acc[i][j][q];
      }
    }
}

// ---- elementwise / small kernels -----------------------------------------------------------
// a1 = relu(x W1 + b1) in BF16 (K = F)
__global__ void k_layer1(int B, int Hd, const float* X, const float* W1, const float* b1, uint16_t* a1) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * Hd) return;
  const int r = (int)(i / Hd), j = (int)(i % Hd);
  float z = b1[j];
#pragma unroll
  for (int f = 0; f < kF; f++) z = fmaf(X[(size_t)r * kF + f], W1[(size_t)f * Hd + j], z);
  a1[i] = f2bf(fmaxf(z, 0.f));
}
// a2 = relu(z2 + b2) in BF16
__global__ void k_bias_relu(int64_t n, int Hd, const float* z, const float* b, uint16_t* a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  a[i] = f2bf(fmaxf(z[i] + b[i % Hd], 0.f));
}
// y = a2 W3 + b3: one warp per row
__global__ void k_layer3(int B, int Hd, const uint16_t* a2, const float* W3, const float* b3, float* y) {
  const int r = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (r >= B) return;
  float s = 0.f;
  for (int j = lane; j < Hd; j += 32) s = fmaf(bf2f(a2[(size_t)r * Hd + j]), W3[j], s);
  for (int m = 16; m > 0; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
  if (lane == 0) y[r] = s + b3[0];
}
// dy = 2 (y - t) / B; per-block loss partials (deterministic two-stage sum)
__global__ void k_loss(int B, const float* y, const float* t, float* dy, float* part) {
  __shared__ float s[256];
  float l = 0.f;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < B; r += gridDim.x * blockDim.x) {
    const float e = y[r] - t[r];
    dy[r] = 2.f * e / (float)B;
    l += e * e;
  }
  s[threadIdx.x] = l;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}
// dz2 = (dy W3^T) * [a2 > 0], BF16; one thread per element
__global__ void k_dz2(int B, int Hd, const float* dy, const float* W3, const uint16_t* a2, uint16_t* dz2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * Hd) return;
  const int r = (int)(i / Hd), j = (int)(i % Hd);
  dz2[i] = bf2f(a2[i]) > 0.f ? f2bf(dy[r] * W3[j]) : (uint16_t)0;
}
// dz1 = da1 * [a1 > 0], FP32 (it feeds the FP32 layer-1 gradient)
__global__ void k_dz1(int64_t n, const float* da1, const uint16_t* a1, float* dz1) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  dz1[i] = bf2f(a1[i]) > 0.f ? da1[i] : 0.f;
}
// column sums over the batch, deterministic: block c sums column c in a fixed order.
// kind 0: out[c] = sum_r v[r * ld + c] (FP32 v); kind 1: BF16 v; kind 2: weighted
// sum_r bf(a[r * ld + c]) * w[r]
__global__ void k_colsum(int B, int cols, int ld, int kind, const void* v, const float* w, float* out) {
  __shared__ float s[256];
  const int c = blockIdx.x;
  float acc = 0.f;
  for (int r = threadIdx.x; r < B; r += blockDim.x) {
    float x;
    if (kind == 0) x = ((const float*)v)[(size_t)r * ld + c];
    else if (kind == 1) x = bf2f(((const uint16_t*)v)[(size_t)r * ld + c]);
    else x = bf2f(((const uint16_t*)v)[(size_t)r * ld + c]) * w[r];
    acc += x;
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = s[0];
  (void)cols;
}
// dW1[f][j] = sum_r x[r][f] dz1[r][j]: block per (f, j-tile)
__global__ void k_dw1(int B, int Hd, const float* X, const float* dz1, float* dW1) {
  const int f = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= Hd) return;
  float acc = 0.f;
  for (int r = 0; r < B; r++) acc = fmaf(X[(size_t)r * kF + f], dz1[(size_t)r * Hd + j], acc);
  dW1[(size_t)f * Hd + j] = acc;
}
__global__ void k_adam(int64_t n, float* w, const float* g, float* m1, float* m2, float lr, float b1,
                       float b2, float c1, float c2, float eps) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float a = b1 * m1[i] + (1.f - b1) * gi;
  const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
  m1[i] = a;
  m2[i] = b;
  w[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}
__global__ void k_to_bf16(int64_t n, const float* w, uint16_t* o) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) o[i] = f2bf(w[i]);
}

unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ---- model ---------------------------------------------------------------------------------
struct hq_mlp {
  int Hd = 0, F = kF, cap = 0;  // hidden width, features, batch capacity
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int64_t np = 0;  // parameters
  // flat FP32 master parameters: W1 [F x Hd], b1 [Hd], W2 [Hd x Hd], b2 [Hd], W3 [Hd], b3 [1]
  float* w = nullptr;
  float* g = nullptr;
  float* m1 = nullptr;
  float* m2 = nullptr;
  uint16_t* w2bf = nullptr;  // BF16 copy of W2
  int64_t t = 0;             // Adam steps
  // batch scratch
  uint16_t *a1 = nullptr, *a2 = nullptr, *dz2 = nullptr;
  float *z2 = nullptr, *y = nullptr, *dy = nullptr, *da1 = nullptr, *dz1 = nullptr, *part = nullptr;
  float* hpart = nullptr;  // pinned
  int64_t o_W1 = 0, o_b1 = 0, o_W2 = 0, o_b2 = 0, o_W3 = 0, o_b3 = 0;
};

namespace {

void mlp_free_batch(hq_mlp* m) {
  void* p[] = {m->a1, m->a2, m->dz2, m->z2, m->y, m->dy, m->da1, m->dz1, m->part};
  for (void* q : p)
    if (q) cudaFree(q);
  m->a1 = m->a2 = m->dz2 = nullptr;
  m->z2 = m->y = m->dy = m->da1 = m->dz1 = m->part = nullptr;
  m->cap = 0;
}

int mlp_reserve(hq_mlp* m, int B) {
  if (B <= m->cap) return HQ_OK;
  mlp_free_batch(m);
  const size_t bh = (size_t)B * m->Hd;
  cudaError_t e = cudaSuccess;
  e = e == cudaSuccess ? cudaMalloc((void**)&m->a1, bh * 2) : e;
  e = e == cudaSuccess ? cudaMalloc((void**)&m->a2, bh * 2) : e;
  e = e == cudaSuccess ? cudaMalloc((void**)&m->dz2, bh * 2) : e;
  e = e == cudaSuccess ? cudaMalloc((void**)&m->z2, bh * 4) : e;
  e = e == cudaSuccess ? cudaMalloc((void**)&m->da1, bh * 4) : e;
  e = e == cudaSuccess ? cudaMalloc((void**)&m->dz1, bh * 4) : e;
  e = e == cudaSuccess ? cudaMalloc((void**)&m->y, (size_t)B * 4) : e;
  e = e == cudaSuccess ? cudaMalloc((void**)&m->dy, (size_t)B * 4) : e;
  e = e == cudaSuccess ? cudaMalloc((void**)&m->part, 1024 * 4) : e;
  if (e != cudaSuccess) {
    cudaGetLastError();
    mlp_free_batch(m);
    hq_set_error("cudaMalloc of the MLP batch scratch failed");
    return HQ_ENOMEM;
  }
  m->cap = B;
  return HQ_OK;
}

int gemm(cudaStream_t s, bool TA, bool TB, int M, int N, int K, const uint16_t* A, int lda, const uint16_t* B,
         int ldb, float* C, int ldc) {
  dim3 grid((N + kTN - 1) / kTN, (M + kTM - 1) / kTM);
  if (!TA && !TB) k_gemm_bf16<false, false><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc);
  else if (TA && !TB) k_gemm_bf16<true, false><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc);
  else if (!TA && TB) k_gemm_bf16<false, true><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc);
  else k_gemm_bf16<true, true><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc);
  HQ_LAUNCHED();
  return HQ_OK;
}

// forward pass of B rows of X (device, B x F) into m->y
int forward(hq_mlp* m, const float* X, int B) {
  const int Hd = m->Hd;
  const int64_t bh = (int64_t)B * Hd;
  k_layer1<<<nblk(bh), 256, 0, m->stream>>>(B, Hd, X, m->w + m->o_W1, m->w + m->o_b1, m->a1);
  HQ_LAUNCHED();
  int rc = gemm(m->stream, false, false, B, Hd, Hd, m->a1, Hd, m->w2bf, Hd, m->z2, Hd);
  if (rc != HQ_OK) return rc;
  k_bias_relu<<<nblk(bh), 256, 0, m->stream>>>(bh, Hd, m->z2, m->w + m->o_b2, m->a2);
  HQ_LAUNCHED();
  k_layer3<<<nblk((int64_t)B * 32), 256, 0, m->stream>>>(B, Hd, m->a2, m->w + m->o_W3, m->w + m->o_b3, m->y);
  HQ_LAUNCHED();
  return HQ_OK;
}

// loss and gradient of the mean squared error into m->g; loss to *loss (host)
int backward(hq_mlp* m, const float* X, const float* target, int B, float* loss) {
  const int Hd = m->Hd;
  const int64_t bh = (int64_t)B * Hd;
  const int nb = 120;
  k_loss<<<nb, 256, 0, m->stream>>>(B, m->y, target, m->dy, m->part);
  HQ_LAUNCHED();
  float* g = m->g;
  // layer 3: dW3 = a2^T dy, db3 = sum dy
  k_colsum<<<Hd, 256, 0, m->stream>>>(B, Hd, Hd, 2, m->a2, m->dy, g + m->o_W3);
  HQ_LAUNCHED();
  k_colsum<<<1, 256, 0, m->stream>>>(B, 1, 1, 0, m->dy, nullptr, g + m->o_b3);
  HQ_LAUNCHED();
  // layer 2: dz2 = (dy W3^T) [a2 > 0]; dW2 = a1^T dz2; db2 = colsum dz2
  k_dz2<<<nblk(bh), 256, 0, m->stream>>>(B, Hd, m->dy, m->w + m->o_W3, m->a2, m->dz2);
  HQ_LAUNCHED();
  int rc = gemm(m->stream, true, false, Hd, Hd, B, m->a1, Hd, m->dz2, Hd, g + m->o_W2, Hd);
  if (rc != HQ_OK) return rc;
  k_colsum<<<Hd, 256, 0, m->stream>>>(B, Hd, Hd, 1, m->dz2, nullptr, g + m->o_b2);
  HQ_LAUNCHED();
  // layer 1: da1 = dz2 W2^T; dz1 = da1 [a1 > 0]; dW1 = x^T dz1; db1 = colsum dz1
  rc = gemm(m->stream, false, true, B, Hd, Hd, m->dz2, Hd, m->w2bf, Hd, m->da1, Hd);
  if (rc != HQ_OK) return rc;
  k_dz1<<<nblk(bh), 256, 0, m->stream>>>(bh, m->da1, m->a1, m->dz1);
  HQ_LAUNCHED();
  k_dw1<<<dim3(nblk(Hd), kF), 256, 0, m->stream>>>(B, Hd, X, m->dz1, g + m->o_W1);
  HQ_LAUNCHED();
  k_colsum<<<Hd, 256, 0, m->stream>>>(B, Hd, Hd, 0, m->dz1, nullptr, g + m->o_b1);
  HQ_LAUNCHED();
  if (loss) {
    HQ_CUDA(cudaMemcpyAsync(m->hpart, m->part, nb * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    HQ_CUDA(cudaStreamSynchronize(m->stream));
    double s = 0.0;
    for (int i = 0; i < nb; i++) s += m->hpart[i];
    *loss = (float)(s / B);
  }
  return HQ_OK;
}

int refresh_bf16(hq_mlp* m) {
  const int64_t n = (int64_t)m->Hd * m->Hd;
  k_to_bf16<<<nblk(n), 256, 0, m->stream>>>(n, m->w + m->o_W2, m->w2bf);
  HQ_LAUNCHED();
  return HQ_OK;
}

// splitmix64 (a published counter-based generator) for the seeded initial weights
uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" int hq_mlp_create(int hidden, uint64_t seed, void* stream, hq_mlp** out) {
  if (!out) { hq_set_error("out is NULL"); return HQ_EINVAL; }
  *out = nullptr;
  if (hidden < 16 || hidden > 4096 || hidden % 16) { hq_set_error("hidden must be a multiple of 16 in 16..4096"); return HQ_EINVAL; }
  hq_mlp* m = new hq_mlp();
  m->Hd = hidden;
  const int Hd = hidden;
  m->o_W1 = 0;
  m->o_b1 = m->o_W1 + (int64_t)kF * Hd;
  m->o_W2 = m->o_b1 + Hd;
  m->o_b2 = m->o_W2 + (int64_t)Hd * Hd;
  m->o_W3 = m->o_b2 + Hd;
  m->o_b3 = m->o_W3 + Hd;
  m->np = m->o_b3 + 1;
  m->stream = (cudaStream_t)stream;
  if (!m->stream) {
    if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete m;
      hq_set_error("cudaStreamCreateWithFlags failed");
      return HQ_ECUDA;
    }
    m->own_stream = true;
  }
  const size_t nb = (size_t)m->np * 4;
  cudaError_t e = cudaMalloc((void**)&m->w, nb);
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->g, nb);
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->m1, nb);
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->m2, nb);
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->w2bf, (size_t)Hd * Hd * 2);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&m->hpart, 1024 * 4);
  if (e != cudaSuccess) {
    cudaGetLastError();
    hq_mlp_destroy(m);
    hq_set_error("allocation of the MLP failed");
    return HQ_ENOMEM;
  }
  // He-uniform initial weights (seeded, host), zero biases
  std::vector<float> h((size_t)m->np, 0.f);
  uint64_t s = seed;
  auto fill = [&](int64_t off, int64_t n, int fan_in) {
    const double lim = sqrt(6.0 / fan_in);
    for (int64_t i = 0; i < n; i++) {
      const double u = (double)(splitmix(s) >> 11) * (1.0 / 9007199254740992.0);
      h[off + i] = (float)((2.0 * u - 1.0) * lim);
    }
  };
  fill(m->o_W1, (int64_t)kF * Hd, kF);
  fill(m->o_W2, (int64_t)Hd * Hd, Hd);
  fill(m->o_W3, Hd, Hd);
  HQ_CUDA(cudaMemcpy(m->w, h.data(), nb, cudaMemcpyHostToDevice));
  HQ_CUDA(cudaMemset(m->m1, 0, nb));
  HQ_CUDA(cudaMemset(m->m2, 0, nb));
  HQ_CUDA(cudaMemset(m->g, 0, nb));
  int rc = refresh_bf16(m);
  if (rc == HQ_OK) HQ_CUDA(cudaStreamSynchronize(m->stream));
  if (rc != HQ_OK) {
    hq_mlp_destroy(m);
    return rc;
  }
  *out = m;
  return HQ_OK;
}

extern "C" void hq_mlp_destroy(hq_mlp* m) {
  if (!m) return;
  if (m->stream) cudaStreamSynchronize(m->stream);
  mlp_free_batch(m);
  void* p[] = {m->w, m->g, m->m1, m->m2, m->w2bf};
  for (void* q : p)
    if (q) cudaFree(q);
  if (m->hpart) cudaFreeHost(m->hpart);
  if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
  delete m;
}

extern "C" int64_t hq_mlp_num_params(const hq_mlp* m) { return m ? m->np : 0; }

extern "C" int hq_mlp_set_weights(hq_mlp* m, const float* w, int64_t n, int mem) {
  if (!m || !w) { hq_set_error("NULL argument"); return HQ_EINVAL; }
  if (n != m->np) { hq_set_error("parameter count mismatch"); return HQ_EINVAL; }
  HQ_CUDA(cudaMemcpyAsync(m->w, w, (size_t)n * 4, mem == HQ_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          m->stream));
  HQ_CUDA(cudaMemsetAsync(m->m1, 0, (size_t)n * 4, m->stream));
  HQ_CUDA(cudaMemsetAsync(m->m2, 0, (size_t)n * 4, m->stream));
  m->t = 0;
  int rc = refresh_bf16(m);
  if (rc != HQ_OK) return rc;
  HQ_CUDA(cudaStreamSynchronize(m->stream));
  return HQ_OK;
}

extern "C" int hq_mlp_get_weights(hq_mlp* m, float* w, int64_t n, int mem) {
  if (!m || !w) { hq_set_error("NULL argument"); return HQ_EINVAL; }
  if (n != m->np) { hq_set_error("parameter count mismatch"); return HQ_EINVAL; }
  HQ_CUDA(cudaMemcpyAsync(w, m->w, (size_t)n * 4, mem == HQ_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          m->stream));
  HQ_CUDA(cudaStreamSynchronize(m->stream));
  return HQ_OK;
}

extern "C" int hq_mlp_forward(hq_mlp* m, const float* X, int B, float* y) {
  if (!m || !X || !y || B < 1) { hq_set_error("bad argument"); return HQ_EINVAL; }
  int rc = mlp_reserve(m, B);
  if (rc != HQ_OK) return rc;
  rc = forward(m, X, B);
  if (rc != HQ_OK) return rc;
  HQ_CUDA(cudaMemcpyAsync(y, m->y, (size_t)B * 4, cudaMemcpyDeviceToDevice, m->stream));
  HQ_CUDA(cudaStreamSynchronize(m->stream));
  return HQ_OK;
}

extern "C" int hq_mlp_gradients(hq_mlp* m, const float* X, const float* target, int B, float* grad, float* loss) {
  if (!m || !X || !target || B < 1) { hq_set_error("bad argument"); return HQ_EINVAL; }
  int rc = mlp_reserve(m, B);
  if (rc == HQ_OK) rc = forward(m, X, B);
  if (rc == HQ_OK) rc = backward(m, X, target, B, loss);
  if (rc != HQ_OK) return rc;
  if (grad) HQ_CUDA(cudaMemcpyAsync(grad, m->g, (size_t)m->np * 4, cudaMemcpyDeviceToDevice, m->stream));
  HQ_CUDA(cudaStreamSynchronize(m->stream));
  return HQ_OK;
}

extern "C" int hq_mlp_train_step(hq_mlp* m, const float* X, const float* target, int B, float lr, float* loss) {
  if (!m || !X || !target || B < 1 || !(lr > 0.f)) { hq_set_error("bad argument"); return HQ_EINVAL; }
  int rc = mlp_reserve(m, B);
  if (rc == HQ_OK) rc = forward(m, X, B);
  if (rc == HQ_OK) rc = backward(m, X, target, B, loss);
  if (rc != HQ_OK) return rc;
  m->t++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)m->t), c2 = 1.f - powf(b2, (float)m->t);
  k_adam<<<nblk(m->np), 256, 0, m->stream>>>(m->np, m->w, m->g, m->m1, m->m2, lr, b1, b2, c1, c2, 1e-8f);
  HQ_LAUNCHED();
  rc = refresh_bf16(m);
  if (rc != HQ_OK) return rc;
  if (!loss) HQ_CUDA(cudaStreamSynchronize(m->stream));
  return HQ_OK;
}

int hq_mlp_predict_dev(hq_mlp* m, const float* X, int B, float* y_dev, cudaStream_t s) {
  // run on the model's stream, ordered after `s` and before later work on `s`
  cudaEvent_t e;
  HQ_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  HQ_CUDA(cudaEventRecord(e, s));
  HQ_CUDA(cudaStreamWaitEvent(m->stream, e, 0));
  int rc = mlp_reserve(m, B);
  if (rc == HQ_OK) rc = forward(m, X, B);
  if (rc == HQ_OK) HQ_CUDA(cudaMemcpyAsync(y_dev, m->y, (size_t)B * 4, cudaMemcpyDeviceToDevice, m->stream));
  if (rc == HQ_OK) {
    HQ_CUDA(cudaEventRecord(e, m->stream));
    HQ_CUDA(cudaStreamWaitEvent(s, e, 0));
  }
  cudaEventDestroy(e);
  return rc;
}

// ---- features of an instance and the product-form start ----------------------------------
namespace {

// Rows (layer n = 1..N-1, unit i), row r = (n-1) N + i: the unit's features -- nu_i
// relative to the mean, the demand shares of the nodes that rank i first, second and
// third, the first-choice offered load lambda s1_i / nu_i, the overall load lambda /
// sum nu, log(nu_i / mean nu), N / 16 -- and the layer fraction n / N.
__global__ void k_features(int N, int J, const double* lam_j, const int32_t* pref, const double* nu, double lam,
                           double nu_sum, float* X) {
  const int i = threadIdx.x;
  if (i >= N) return;
  double s[3] = {0.0, 0.0, 0.0};
  for (int j = 0; j < J; j++)
    for (int h = 0; h < 3 && h < N; h++)
      if (pref[(int64_t)j * N + h] == i) s[h] += lam_j[j];
  const double mean_nu = nu_sum / N;
  float u[HQ_MLP_UNIT_FEATURES];
  u[0] = (float)(nu[i] / mean_nu);
  u[1] = (float)(s[0] / lam);
  u[2] = (float)(s[1] / lam);
  u[3] = (float)(s[2] / lam);
  u[4] = (float)(s[0] / nu[i]);
  u[5] = (float)(lam / nu_sum);
  u[6] = (float)log(nu[i] / mean_nu);
  u[7] = (float)N / 16.f;
  for (int n = 1; n <= N - 1; n++) {
    float* x = X + ((size_t)(n - 1) * N + i) * HQ_MLP_FEATURES;
    for (int f = 0; f < HQ_MLP_UNIT_FEATURES; f++) x[f] = u[f];
    x[HQ_MLP_UNIT_FEATURES] = (float)n / (float)N;
  }
}

// Per layer n = 1..N-1 (one thread each): log x_i(n) = logit(q_i(n)) with q = sigmoid(y)
// clamped to [1e-4, 1 - 1e-4], and log e_n(x(n)) by the recursion e_k <- e_k + x_i e_{k-1}
// over the units, in log space.
__global__ void k_product_norm(int N, const float* y, double* lx, double* le) {
  const int n = threadIdx.x + 1;
  if (n > N - 1) {
    if (threadIdx.x == 0) le[0] = 0.0;
    if (n == N) le[N] = 0.0;
    return;
  }
  double e[HQ_MAXN + 1];
  e[0] = 0.0;
  for (int k = 1; k <= n; k++) e[k] = -INFINITY;
  for (int i = 0; i < N; i++) {
    double q = 1.0 / (1.0 + exp(-(double)y[(n - 1) * N + i]));
    q = fmin(fmax(q, 1e-4), 1.0 - 1e-4);
    const double l = log(q / (1.0 - q));
    lx[(size_t)(n - 1) * N + i] = l;
    const int top = i + 1 < n ? i + 1 : n;
    for (int k = top; k >= 1; k--) {
      const double a = e[k], b = e[k - 1] + l;
      const double mx = fmax(a, b);
      e[k] = mx == -INFINITY ? -INFINITY : mx + log(exp(a - mx) + exp(b - mx));
    }
  }
  le[n] = e[n];
  if (n == 1) le[0] = 0.0;
}

// p_n(B) = prod_{i in B} x_i(n) / e_n(x(n)), y-order; the empty and the full state: 1
__global__ void k_product_fill(int N, int64_t S, const double* lx, const double* le, double* P) {
  __shared__ double slx[HQ_MAXN * HQ_MAXN], sle[HQ_MAXN + 1];
  for (int k = threadIdx.x; k < N * (N - 1); k += blockDim.x) slx[k] = lx[k];
  if (threadIdx.x <= N) sle[threadIdx.x] = le[threadIdx.x];
  __syncthreads();
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= S) return;
  const int n = __popc((uint32_t)b);
  if (n == 0 || n == N) {
    P[b] = 1.0;
    return;
  }
  const double* l = slx + (size_t)(n - 1) * N;
  double s = 0.0;
  for (uint32_t y = (uint32_t)b; y; y &= y - 1) s += l[__ffs(y) - 1];
  P[b] = exp(s - sle[n]);
}

}  // namespace

// the analytic control: logit(rho0_i) for every layer, rho0_i = lambda1_i / nu_i clipped
// to [0.02, 0.98], lambda1_i the demand of the nodes ranking unit i first (summed in
// node order)
__global__ void k_analytic_logits(int N, int J, const double* lam_j, const int32_t* pref, const double* nu,
                                  float* y) {
  if (threadIdx.x != 0) return;
  double l1[HQ_MAXN];
  for (int i = 0; i < N; i++) l1[i] = 0.0;
  for (int j = 0; j < J; j++) l1[pref[(int64_t)j * N]] += lam_j[j];
  for (int i = 0; i < N; i++) {
    const double r = fmin(fmax(l1[i] / nu[i], 0.02), 0.98);
    const float l = (float)log(r / (1.0 - r));
    for (int n = 1; n <= N - 1; n++) y[(size_t)(n - 1) * N + i] = l;
  }
}

int hq_product_warm_start(hq_solver* h, double* P) {
  if (!h->wy || h->N < 2) {
    hq_set_error("solver scratch for the warm start is missing");
    return HQ_ESTATE;
  }
  k_analytic_logits<<<1, 32, 0, h->stream>>>(h->N, h->J, h->lam_j, h->pref, h->nu, h->wy);
  HQ_LAUNCHED();
  double* le = h->wlx + (size_t)HQ_MAXN * HQ_MAXN;
  k_product_norm<<<1, 32, 0, h->stream>>>(h->N, h->wy, h->wlx, le);
  HQ_LAUNCHED();
  k_product_fill<<<(unsigned)((h->S + 255) / 256), 256, 0, h->stream>>>(h->N, h->S, h->wlx, le, P);
  HQ_LAUNCHED();
  return HQ_OK;
}

int hq_mlp_features_dev(hq_solver* h, float* X) {
  k_features<<<1, 32, 0, h->stream>>>(h->N, h->J, h->lam_j, h->pref, h->nu, h->lam, h->nu_sum, X);
  HQ_LAUNCHED();
  return HQ_OK;
}

// prediction of a model for the loaded instance: y (logit q_i(n)) in h->wy; the
// layer-wise product-form start in y-order into P (S doubles, device) if not NULL
int hq_mlp_warm_start(hq_solver* h, hq_mlp* m, double* P, double* unused) {
  (void)unused;
  if (!h->wfeat || h->N < 2) {
    hq_set_error("solver scratch for the warm start is missing");
    return HQ_ESTATE;
  }
  const int R = h->N * (h->N - 1);
  int rc = hq_mlp_features_dev(h, h->wfeat);
  if (rc != HQ_OK) return rc;
  rc = hq_mlp_predict_dev(m, h->wfeat, R, h->wy, h->stream);
  if (rc != HQ_OK) return rc;
  double* le = h->wlx + (size_t)HQ_MAXN * HQ_MAXN;
  k_product_norm<<<1, 32, 0, h->stream>>>(h->N, h->wy, h->wlx, le);
  HQ_LAUNCHED();
  if (P) {
    k_product_fill<<<(unsigned)((h->S + 255) / 256), 256, 0, h->stream>>>(h->N, h->S, h->wlx, le, P);
    HQ_LAUNCHED();
  }
  return HQ_OK;
}

extern "C" int hq_mlp_features(hq_solver* h, float* X, int mem) {
  if (!h || !X) { hq_set_error("NULL argument"); return HQ_EINVAL; }
  if (!h->loaded) { hq_set_error("hq_load has not succeeded"); return HQ_ESTATE; }
  if (h->N < 2) { hq_set_error("N must be >= 2"); return HQ_EINVAL; }
  int rc = hq_mlp_features_dev(h, h->wfeat);
  if (rc != HQ_OK) return rc;
  HQ_CUDA(cudaMemcpyAsync(X, h->wfeat, sizeof(float) * h->N * (h->N - 1) * HQ_MLP_FEATURES,
                          mem == HQ_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
  HQ_CUDA(cudaStreamSynchronize(h->stream));
  return HQ_OK;
}

extern "C" int hq_attach_mlp(hq_solver* h, hq_mlp* m) {
  if (!h) { hq_set_error("NULL solver"); return HQ_EINVAL; }
  h->mlp = m;
  return HQ_OK;
}

extern "C" int hq_mlp_predict(hq_solver* h, hq_mlp* m, double* q, double* pn, double* rho, int mem) {
  if (!h || !m || !q) { hq_set_error("NULL argument"); return HQ_EINVAL; }
  if (!h->loaded) { hq_set_error("hq_load has not succeeded"); return HQ_ESTATE; }
  if (h->N < 2) { hq_set_error("N must be >= 2"); return HQ_EINVAL; }
  int rc = hq_mlp_warm_start(h, m, nullptr, nullptr);
  if (rc != HQ_OK) return rc;
  const int N = h->N, R = N * (N - 1);
  std::vector<float> y((size_t)R);
  std::vector<double> nu((size_t)N);
  HQ_CUDA(cudaMemcpyAsync(y.data(), h->wy, sizeof(float) * R, cudaMemcpyDeviceToHost, h->stream));
  HQ_CUDA(cudaMemcpyAsync(nu.data(), h->nu, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream));
  HQ_CUDA(cudaStreamSynchronize(h->stream));
  // q_i(n): 0 for n = 0, 1 for n = N
  std::vector<double> qq((size_t)(N + 1) * N, 0.0);
  for (int i = 0; i < N; i++) qq[(size_t)N * N + i] = 1.0;
  for (int n = 1; n <= N - 1; n++)
    for (int i = 0; i < N; i++) qq[(size_t)n * N + i] = 1.0 / (1.0 + exp(-(double)y[(size_t)(n - 1) * N + i]));
  // layer law of the loss system with lambda(n) = lambda and mu(n) = sum_i nu_i q_i(n)
  // (Eq. 10 with the predicted conditionals), then rho_i = sum_n P(n) q_i(n)
  std::vector<double> lp((size_t)N + 1, 0.0), p((size_t)N + 1), r((size_t)N, 0.0);
  for (int n = 1; n <= N; n++) {
    double mu = 0.0;
    for (int i = 0; i < N; i++) mu += nu[i] * qq[(size_t)n * N + i];
    lp[n] = lp[n - 1] + log(h->lam) - log(mu);
  }
  double mx = -INFINITY, z = 0.0;
  for (int n = 0; n <= N; n++) mx = fmax(mx, lp[n]);
  for (int n = 0; n <= N; n++) z += exp(lp[n] - mx);
  for (int n = 0; n <= N; n++) p[n] = exp(lp[n] - mx) / z;
  for (int n = 0; n <= N; n++)
    for (int i = 0; i < N; i++) r[i] += p[n] * qq[(size_t)n * N + i];
  const cudaMemcpyKind k = mem == HQ_DEVICE ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
  HQ_CUDA(cudaMemcpy(q, qq.data(), sizeof(double) * qq.size(), k));
  if (pn) HQ_CUDA(cudaMemcpy(pn, p.data(), sizeof(double) * (N + 1), k));
  if (rho) HQ_CUDA(cudaMemcpy(rho, r.data(), sizeof(double) * N, k));
  return HQ_OK;
}

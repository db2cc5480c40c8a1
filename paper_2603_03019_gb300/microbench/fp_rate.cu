// Issue-rate microbenchmark of the chip's FP64 and FP32 fused multiply-add: every thread
// runs kChains independent dependent chains a <- a * b + c for `iters` steps, on a grid of
// blocksPerSm x SM-count CTAs of 256 threads, timed with CUDA events around each launch
// (after one warm-up launch).  Prints one JSON line per type:
//   {"type": "f64", "fma_per_s": ..., "flop_per_s": ..., "ms": ..., "fma": ...}
// The FP64 figure bounds kernels whose FP64 work, not memory, sets their time: the
// stationary-distribution sweep in FP64 is such a kernel on this chip.
#include <cstdio>
#include <cstdlib>

#include <cuda_runtime.h>

constexpr int kChains = 8;

template <class T>
__global__ void __launch_bounds__(256) k_fma(int iters, T b, T c, T* out) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = a[k] * b + c;
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; k++) s += a[k];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
static int run(const char* name, int iters, int reps, int blocks_per_sm) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = nsm * blocks_per_sm, threads = 256;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * (size_t)grid * threads) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // b slightly below 1 and c small keep every chain finite and normal
  const T b = (T)0.999999, c = (T)1e-6;
  k_fma<T><<<grid, threads>>>(iters, b, c, out);
  if (cudaDeviceSynchronize() != cudaSuccess) return 2;
  float best = 1e30f, total = 0.f;
  for (int r = 0; r < reps; r++) {
    cudaEventRecord(e0);
    k_fma<T><<<grid, threads>>>(iters, b, c, out);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    total += ms;
    if (ms < best) best = ms;
  }
  if (cudaGetLastError() != cudaSuccess) return 3;
  const double fma = (double)grid * threads * kChains * (double)iters;
  printf("{\"type\": \"%s\", \"fma\": %.0f, \"ms_best\": %.4f, \"ms_mean\": %.4f, \"fma_per_s\": %.6e, "
         "\"flop_per_s\": %.6e, \"grid\": %d, \"threads\": %d, \"chains\": %d}\n",
         name, fma, best, total / reps, fma / (best * 1e-3), 2.0 * fma / (best * 1e-3), grid, threads, kChains);
  cudaFree(out);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return 0;
}

int main(int argc, char** argv) {
  const int iters64 = argc > 1 ? atoi(argv[1]) : 20000;
  const int reps = argc > 2 ? atoi(argv[2]) : 20;
  const int bps = argc > 3 ? atoi(argv[3]) : 4;
  if (iters64 < 1 || reps < 1 || bps < 1 || bps > 8) return 4;
  int rc = run<double>("f64", iters64, reps, bps);
  if (rc) return rc;
  return run<float>("f32", iters64 * 16, reps, bps);
}

// Outer iterations k of Algorithm 1 (Eq. 12-14) on the layer-ranked layout, as one
// persistent kernel per batch of sweeps.
//
// For layer n (ascending: Gauss-Seidel from layer n-1, Jacobi from layer n+1, as in
// Algorithm 1 and the two properties stated for Algorithm 2) and each state m, Eq. (12)
// reads
//     p_n^{k,r}(m) = alpha mu^{k,r-1}(n) A_m + beta B_m
// with  alpha = 1/lambda^k(n-1),  beta = lambda^{k-1}(n) / mu^{k-1}(n+1),
//       A_m = r_m sum_{l in C_{n-1}} p^k_{n-1}(l) lambda_{lm},
//       B_m = r_m sum_{u idle in m} p^{k-1}_{n+1}(m+u) nu_u,   r_m = 1/(lambda_m+mu_m).
// Only mu^{k,r-1}(n) depends on r; with Eq. (14) it obeys mu^{k,r} = a mu^{k,r-1} + b,
// a = alpha sum_m mu_m A_m in (0,1), b = beta sum_m mu_m B_m, so the inner loop of
// Algorithm 1 converges to mu* = b/(1-a) and p_n^k(m) = c1 A_m + c2 B_m with
// c1 = alpha mu*, c2 = beta (the delta -> 0 reading of the inner loop).  Then
// lambda^k(n) = lambda sum_m p_n^k(m) = lambda (c1 sum A + c2 sum B) (Eq. 13), mu^k(n) = mu*.
//
// Schedule.  Phase n of a sweep gathers layer n into (A, B) pairs; c1, c2 of layer n
// are only known once every CTA has added its share of sum mu_m A_m and sum mu_m B_m.
// So layer n-1 stays as (A, B) pairs until phase n: the gathers of layer n combine
// p_{n-1} = c1 A + c2 B on the fly (accumulating sum T A and sum T B separately), and
// phase n also writes the final p_{n-1} and its step |p^k - p^{k-1}|.  One grid
// barrier per layer; layer N-1 of sweep k is finalised in phase 1 of sweep k+1 (which
// does not read it), and a closing phase finalises the last sweep.  The CTA that
// arrives last at a barrier folds every CTA's partial sums in a fixed order, solves
// the layer's scalar recursion and publishes c1, c2, lambda(n), mu(n) and the step
// before it releases the others: the result is deterministic.
//
// Streaming.  Warp 0 copies the table rows, r_m and state masks of a tile of
// consecutive states to shared memory with bulk asynchronous copies (cp.async.bulk,
// completion on an mbarrier), up to kStages tiles ahead, across grid barriers too
// (the table never changes); warps 1..7 consume the tiles and free each stage through
// a second mbarrier.  Neighbour values are gathered through L2.  Each thread loads the
// rank bases of its state's high-part neighbours once, in parallel, into its own
// shared-memory slot, so no gather waits on a dependent table load.
//
// Every wait is bounded: a grid barrier or mbarrier that does not complete within its
// iteration limit sets an error bit in DevScalars::flags and the kernel runs to its
// end with in-bounds indices; the host reports HQ_ETIMEOUT.
#include <stdlib.h>
#include <string.h>

#include "hq_internal.cuh"

namespace {

constexpr int kThreads = HQ_THREADS;        // 256: warp 0 issues the bulk copies,
constexpr int kConsumers = kThreads - 32;  // warps 1..7 consume the staged tiles
constexpr int kStages = 2;
static_assert(HQ_MAX_TILE == 2 * kConsumers, "tile records hold two states per consumer thread");
constexpr int kMaxHi = HQ_MAXN - HQ_LO_BITS;  // high-part bits of a state mask
constexpr int kPW = 6;                        // partial words per CTA per phase
constexpr unsigned kSpinLimit = 1u << 24;

// stage size per precision: four CTAs per SM with the rank-base slots
template <class V> struct StageBytes { static constexpr int v = HQ_STAGE_WIDE; };
template <> struct StageBytes<PolF32> { static constexpr int v = HQ_STAGE_F32; };
// gathers in flight per thread (chunk length), within the 64-register budget
template <class V> struct Chunk { static constexpr int v = 4; };
template <> struct Chunk<PolF32> { static constexpr int v = 8; };

// ---- PTX helpers ------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// L2 policies: the table streams through once per sweep (evict first); the
// neighbour layers are gathered many times (evict last)
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// 1-D bulk copy global -> shared, completion counted on `bar`
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar,
                                         uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, "
      "[%3], %4;" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// polling load: coherent at gpu scope without the acquire's L1 invalidation, so
// spinning CTAs do not evict the cached rank tables of CTAs still working on the SM
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// ---- loads of values that other CTAs wrote in this launch: from L2 (.cg), kept there -----
__device__ __forceinline__ float ld_l2(const float* p, uint64_t pol) {
  float v;
  asm volatile("ld.global.cg.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ float2 ld_l2(const float2* p, uint64_t pol) {
  float2 v;
  asm volatile("ld.global.cg.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
               : "=f"(v.x), "=f"(v.y)
               : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ float4 ld_l2(const float4* p, uint64_t pol) {
  float4 v;
  asm volatile("ld.global.cg.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double ld_l2(const double* p, uint64_t pol) {
  double v;
  asm volatile("ld.global.cg.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double2 ld_l2(const double2* p, uint64_t pol) {
  double2 v;
  asm volatile("ld.global.cg.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
               : "=d"(v.x), "=d"(v.y)
               : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double ld_l2(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float2 ld_l2(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ float ld_l2(const float* p) { return __ldcg(p); }

// (A, B) pair storage per precision
template <class V> struct Pair;
template <> struct Pair<PolF64> {
  typedef double2 P;
  __device__ static P pack(double a, double b) { return make_double2(a, b); }
  __device__ static double A(P p) { return p.x; }
  __device__ static double B(P p) { return p.y; }
  __device__ static P ld(const P* q) { return __ldcg(q); }
  __device__ static P ld(const P* q, uint64_t pol) { return __ldca(q); }
};
template <> struct Pair<PolDF> {
  typedef float4 P;
  __device__ static P pack(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }
  __device__ static float2 A(P p) { return make_float2(p.x, p.y); }
  __device__ static float2 B(P p) { return make_float2(p.z, p.w); }
  __device__ static P ld(const P* q) { return __ldcg(q); }
  __device__ static P ld(const P* q, uint64_t pol) { return __ldca(q); }
};
template <> struct Pair<PolF32> {
  typedef float2 P;
  __device__ static P pack(float a, float b) { return make_float2(a, b); }
  __device__ static float A(P p) { return p.x; }
  __device__ static float B(P p) { return p.y; }
  __device__ static P ld(const P* q) { return __ldcg(q); }
  __device__ static P ld(const P* q, uint64_t pol) { return __ldca(q); }
};

template <class V>
__device__ __forceinline__ typename V::T warp_sum(typename V::T v) {
  for (int m = 16; m > 0; m >>= 1) v = V::add(v, V::shfl_xor(v, m));
  return v;
}

struct PersistArgs {
  int N, L, H, nsweeps;
  double lam;
  int64_t off[HQ_MAXN + 2];   // padded per-state offsets of the layers
  int64_t toff[HQ_MAXN + 2];  // padded table offsets of the layers
  int64_t lsize[HQ_MAXN + 1];
  int64_t lpad[HQ_MAXN + 1];  // table row stride of layer n
  int tk[HQ_MAXN + 1];        // states per tile in layer n
  int ntiles[HQ_MAXN + 1];
  int64_t rbytes[HQ_MAXN + 1];  // bytes of a tile record of layer n
  int64_t roff[HQ_MAXN + 2];    // first record of layer n
  const unsigned char* rec;     // tile records: masks, r_m, table rows
  const uint32_t* RL;
  const uint32_t* RH;
  void* p;
  const void* nu;
  void* ab0;
  void* ab1;
  double* partials;  // [2][gridDim][kPW]
  DevScalars* sc;
};

// work-item cursor of the bulk-copy producer: sweep k, layer n, tile t
struct Cursor {
  int k, n, t;
};

__device__ __forceinline__ bool cursor_fix(const PersistArgs& a, Cursor& c) {
  while (c.t >= a.ntiles[c.n]) {
    c.n++;
    c.t = blockIdx.x;
    if (c.n > a.N - 1) {
      c.n = 1;
      c.k++;
    }
    if (c.k >= a.nsweeps) return false;
  }
  return true;
}

// one bulk copy per tile: the tile's record is the exact image of the stage
template <class V>
__device__ void issue_tile(const PersistArgs& a, const Cursor& c, unsigned char* stage, uint64_t* bar) {
  const int n = c.n;
  const unsigned bytes = (unsigned)a.rbytes[n];
  mbar_expect_tx(bar, bytes);
  bulk_g2s(stage, a.rec + a.roff[n] + (int64_t)c.t * a.rbytes[n], bytes, bar, policy_evict_first());
}

template <class V>
__global__ void __launch_bounds__(kThreads, 4) k_persist(PersistArgs a) {
  typedef typename V::T T;
  typedef Pair<V> PR;
  typedef typename PR::P P2;
  constexpr int kStageBytes = StageBytes<V>::v;
  constexpr int CH = Chunk<V>::v;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* stages = smem;
  uint32_t* s_hb = (uint32_t*)(smem + kStages * kStageBytes);  // [H][kConsumers]
  __shared__ __align__(8) uint64_t full_bar[kStages];   // tile landed (transaction count)
  __shared__ __align__(8) uint64_t empty_bar[kStages];  // every consumer warp is done with it
  __shared__ double s_lam[HQ_MAXN + 1], s_mu[HQ_MAXN + 1];
  __shared__ T s_nu[HQ_MAXN];
  __shared__ double s_red[kPW][kThreads / 32];
  __shared__ double s_fold[kPW];
  __shared__ T s_lamT, s_one;
  __shared__ T s_c1, s_c2;
  __shared__ double s_step[2];
  __shared__ int s_last;
  __shared__ unsigned s_gen;

  DevScalars* sc = a.sc;
  const int N = a.N, L = a.L, H = a.H;
  const unsigned G = gridDim.x;
  const uint32_t* RL = a.RL;
  if (threadIdx.x < N) s_nu[threadIdx.x] = ((const T*)a.nu)[threadIdx.x];
  if (threadIdx.x <= N) {
    s_lam[threadIdx.x] = sc->lam_n[threadIdx.x];
    s_mu[threadIdx.x] = sc->mu_n[threadIdx.x];
  }
  if (threadIdx.x == 0) {
    s_lamT = V::from_d(a.lam);
    s_one = V::from_d(1.0);
    s_c1 = V::zero();
    s_c2 = V::zero();
    s_step[0] = s_step[1] = 0.0;
    if (blockIdx.x == 0) sc->t_start = globaltimer_ns();
    for (int i = 0; i < kStages; i++) {
      mbar_init(&full_bar[i], 1);
      mbar_init(&empty_bar[i], kConsumers / 32);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // Tiles of this CTA are numbered in the order they are consumed (sweep, layer,
  // tile); tile i uses stage i % kStages.  Thread 0 (warp 0) is the producer;
  // warps 1..7 consume.  `phase_end` = number of tiles consumed by the end of the
  // current phase, the same in every thread.
  Cursor pc{0, 1, (int)blockIdx.x};
  bool p_more = cursor_fix(a, pc);
  long issued = 0, consumed = 0, phase_end = 0;
  const bool producer = threadIdx.x == 0;
  const bool consumer = threadIdx.x >= 32;
  const int ctid = (int)threadIdx.x - 32;
  // Issue tiles while a stage is free.  A stage is waited for only if the tile that
  // occupies it is consumed in this phase: the consumers cannot free stages of a
  // later phase before the grid barrier, so waiting for one would never end.
  auto produce = [&]() {
    while (p_more) {
      if (issued >= kStages) {
        const long occ = issued - kStages;
        if (occ >= phase_end) break;
        unsigned it = 0;
        while (!mbar_try_wait(&empty_bar[issued % kStages], (unsigned)((occ / kStages) & 1))) {
          if (++it > kSpinLimit) {
            atomicOr(&sc->flags, 4);
            break;
          }
        }
      }
      issue_tile<V>(a, pc, stages + (issued % kStages) * kStageBytes, &full_bar[issued % kStages]);
      issued++;
      pc.t += G;
      p_more = cursor_fix(a, pc);
    }
  };

  const T* pv = (const T*)a.p;
  const uint64_t keep = policy_evict_last();  // L2 policy of the gathered neighbour values
  T* pw = (T*)a.p;
  const int64_t nthreads = (int64_t)G * blockDim.x;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int gphase = 0;  // phase counter within this launch

  // finalise layer lf from the (A, B) buffer `abf`: p = c1 A + c2 B, |p - p_old|
  auto finalize = [&](int lf, const P2* abf, double& md) {
    const T c1 = s_c1, c2 = s_c2;
    T* pl = pw + a.off[lf];
    const int64_t Lf = a.lsize[lf];
#pragma unroll 4
    for (int64_t k = gtid; k < Lf; k += nthreads) {
      const P2 q = PR::ld(abf + k);
      const T old = ld_l2(pl + k);
      const T v = V::add(V::mul(c1, PR::A(q)), V::mul(c2, PR::B(q)));
      md = fmax(md, V::absdiff(v, old));
      pl[k] = v;
    }
  };

  // Write this CTA's partials, then the grid barrier.  The last CTA to arrive folds
  // all partials in CTA order, solves the scalar recursion of layer lg (if lg > 0)
  // and publishes the result before it releases the others.  ks: sweep of the layer
  // finalised in this phase (its step goes into s_step).
  auto sync_phase = [&](T sA, T sB, T sa, T sb, double md, int lg, int ks) {
    const int buf = gphase & 1;
    {
      T w4[4] = {sA, sB, sa, sb};
      const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
      for (int i = 0; i < 4; i++) {
        const T v = warp_sum<V>(w4[i]);
        if (lane == 0) s_red[i][wid] = V::to_d(v);
      }
      for (int m = 16; m > 0; m >>= 1) md = fmax(md, __shfl_xor_sync(0xffffffffu, md, m));
      if (lane == 0) s_red[4][wid] = md;
      __syncthreads();
      if (threadIdx.x < 5) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); q++)
          t = (threadIdx.x == 4) ? fmax(t, s_red[threadIdx.x][q]) : t + s_red[threadIdx.x][q];
        a.partials[((size_t)buf * G + blockIdx.x) * kPW + threadIdx.x] = t;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      s_gen = ld_relaxed_u32(&sc->bar_gen);
      __threadfence();
      s_last = atomicAdd(&sc->bar_count, 1u) == G - 1;
    }
    __syncthreads();
    if (s_last) {
      // fold every CTA's partials in CTA order
      const double* part = a.partials + (size_t)buf * G * kPW;
      double v[kPW];
#pragma unroll
      for (int w = 0; w < kPW; w++) v[w] = 0.0;
      for (unsigned b = threadIdx.x; b < G; b += blockDim.x) {
#pragma unroll
        for (int w = 0; w < 5; w++) {
          const double x = __ldcg(part + (size_t)b * kPW + w);
          v[w] = (w == 4) ? fmax(v[w], x) : v[w] + x;
        }
      }
#pragma unroll
      for (int w = 0; w < 5; w++)
        for (int m = 16; m > 0; m >>= 1) {
          const double o = __shfl_xor_sync(0xffffffffu, v[w], m);
          v[w] = (w == 4) ? fmax(v[w], o) : v[w] + o;
        }
      const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
      if (lane == 0) {
#pragma unroll
        for (int w = 0; w < 5; w++) s_red[w][wid] = v[w];
      }
      __syncthreads();
      if (threadIdx.x < 5) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); q++)
          t = (threadIdx.x == 4) ? fmax(t, s_red[threadIdx.x][q]) : t + s_red[threadIdx.x][q];
        s_fold[threadIdx.x] = t;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double* pub = sc->pub[buf];
        if (lg > 0) {
          // closed-form limit of the inner loop (Eq. 12 and 14), then Eq. (13)
          const double alpha = 1.0 / s_lam[lg - 1];
          const double beta = s_lam[lg] / s_mu[lg + 1];
          const double aa = alpha * s_fold[0], bb = beta * s_fold[1];
          const double mustar = bb / (1.0 - aa);
          const double c1 = alpha * mustar;
          pub[0] = c1;
          pub[1] = beta;
          pub[2] = a.lam * (c1 * s_fold[2] + beta * s_fold[3]);
          pub[3] = mustar;
          if (!isfinite(mustar) || !(aa < 1.0)) atomicOr(&sc->flags, 1);
        }
        pub[4] = s_fold[4];
        if (gphase < 64) sc->t_phase[gphase] = globaltimer_ns();
        __threadfence();
        atomicExch(&sc->bar_count, 0u);
        __threadfence();
        atomicAdd(&sc->bar_gen, 1u);
      }
    } else if (threadIdx.x == 0) {
      unsigned it = 0;
      while (ld_relaxed_u32(&sc->bar_gen) == s_gen) {
        if (*(volatile int*)&sc->flags & 6) break;  // an earlier wait gave up: do not wait again
        if (++it > kSpinLimit) {
          atomicOr(&sc->flags, 2);
          break;
        }
      }
      __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const double* pub = sc->pub[buf];
      if (lg > 0) {
        s_c1 = V::from_d(__ldcg(pub + 0));
        s_c2 = V::from_d(__ldcg(pub + 1));
        s_lam[lg] = __ldcg(pub + 2);
        s_mu[lg] = __ldcg(pub + 3);
      }
      s_step[ks & 1] = fmax(s_step[ks & 1], __ldcg(pub + 4));
    }
    __syncthreads();
    gphase++;
  };

  for (int k = 0; k < a.nsweeps; k++) {
    for (int n = 1; n <= N - 1; n++) {
      if (threadIdx.x == 0 && n == 1) s_step[k & 1] = 0.0;  // sweep k starts
      // the layer this phase finalises: gathered in the previous phase
      const int fin_layer = gphase == 0 ? -1 : (n == 1 ? N - 1 : n - 1);
      // -- gather layer n -------------------------------------------------------------------
      const P2* ab_prev = (const P2*)(((gphase + 1) & 1) ? a.ab1 : a.ab0);
      P2* ab_cur = (P2*)((gphase & 1) ? a.ab1 : a.ab0);
      const T* p_up = pv + a.off[n + 1];
      const int tk = a.tk[n];
      const int64_t Ln = a.lsize[n];
      const T c1 = s_c1, c2 = s_c2;
      const int nb = n == 1 ? 0 : n;  // busy neighbours read from the (A, B) pairs
      const int ni = N - n;           // idle neighbours
      T sA = V::zero(), sB = V::zero(), sa = V::zero(), sb = V::zero();
      const long my_tiles =
          a.ntiles[n] > (int)blockIdx.x ? (long)((a.ntiles[n] - 1 - (int)blockIdx.x) / (int)G) + 1 : 0;
      phase_end = consumed + my_tiles;
      if (producer) produce();
      for (int t = blockIdx.x; consumer && t < a.ntiles[n]; t += G) {
        const long item = consumed++;
        const int st = (int)(item % kStages);
        unsigned char* stage = stages + st * kStageBytes;
        {
          unsigned it = 0;
          while (!mbar_try_wait(&full_bar[st], (unsigned)((item / kStages) & 1))) {
            if (++it > kSpinLimit) {
              atomicOr(&sc->flags, 4);
              break;
            }
          }
        }
        const int64_t k0 = (int64_t)t * tk;
        const int cnt = (int)min((int64_t)tk, Ln - k0);
        for (int i = ctid; i < cnt; i += kConsumers) {
          const uint32_t x = ((const uint32_t*)stage)[i];
          const T rv = ((const T*)(stage + tk * 4))[i];
          const T* trow = (const T*)(stage + tk * 4 + tk * (int)sizeof(T));
          const uint32_t lo = x & ((1u << L) - 1u), hi = x >> L;
          const int w = __popc(lo);
          const uint32_t* rh = a.RH + (size_t)hi * (L + 1);
          const uint32_t rl = __ldg(RL + lo);
          const uint32_t base_dn = w > 0 ? __ldg(rh + w - 1) : 0u;
          const uint32_t base_up = w < L ? __ldg(rh + w + 1) : 0u;
          // rank bases of the neighbours that differ in a high-part unit j: all loads
          // issued together, kept in this thread's shared-memory slot
#pragma unroll
          for (int j = 0; j < kMaxHi; j++)
            if (j < H) s_hb[j * kConsumers + ctid] = __ldg(a.RH + (size_t)(hi ^ (1u << j)) * (L + 1) + w);
          // Neighbours in chunks of CH: all ranks of a chunk, then all its gathers, then
          // the accumulation, so CH gathers are in flight before the first is used.
          // The chunk bounds depend only on n: no divergence.
          T UA = V::zero(), UB = V::zero(), D = V::zero();
          // busy neighbours: layer n-1, table slot s
          uint32_t yb = x;
          for (int s0 = 0; s0 < nb; s0 += CH) {
            P2 q[CH];
#pragma unroll
            for (int j = 0; j < CH; j++) {
              if (s0 + j < nb) {
                const int b = __ffs(yb) - 1;
                yb &= yb - 1;
                const uint32_t rk = b < L ? __ldg(RL + (lo ^ (1u << b))) + base_dn
                                          : rl + s_hb[(b - L) * kConsumers + ctid];
                q[j] = PR::ld(ab_prev + rk, keep);
              }
            }
#pragma unroll
            for (int j = 0; j < CH; j++) {
              if (s0 + j < nb) {
                const T tv = trow[(s0 + j) * tk + i];
                V::fma_acc(UA, PR::A(q[j]), tv);
                V::fma_acc(UB, PR::B(q[j]), tv);
              }
            }
          }
          // idle neighbours: layer n+1, rate nu_u
          uint32_t yi = ~x & ((1u << N) - 1u);
          for (int s0 = 0; s0 < ni; s0 += CH) {
            T pvv[CH];
            uint32_t ysave = yi;
#pragma unroll
            for (int j = 0; j < CH; j++) {
              if (s0 + j < ni) {
                const int b = __ffs(yi) - 1;
                yi &= yi - 1;
                const uint32_t rk = b < L ? __ldg(RL + (lo | (1u << b))) + base_up
                                          : rl + s_hb[(b - L) * kConsumers + ctid];
                pvv[j] = __ldca(p_up + rk);
              }
            }
#pragma unroll
            for (int j = 0; j < CH; j++) {
              if (s0 + j < ni) {
                const int b = __ffs(ysave) - 1;
                ysave &= ysave - 1;
                V::fma_acc(D, pvv[j], s_nu[b]);
              }
            }
          }
          // up-inflow: layer 0 is the empty state with p_0 = 1
          const T U = n == 1 ? trow[i] : V::add(V::mul(c1, V::norm(UA)), V::mul(c2, V::norm(UB)));
          D = V::norm(D);
          const T q = V::sub(s_one, V::mul(s_lamT, rv));  // mu_m r_m = 1 - lambda r_m
          const T A = V::mul(U, rv), B = V::mul(D, rv);
          ab_cur[k0 + i] = PR::pack(A, B);
          sA = V::add(sA, V::mul(U, q));
          sB = V::add(sB, V::mul(D, q));
          sa = V::add(sa, A);
          sb = V::add(sb, B);
        }
        __syncwarp();
        if ((threadIdx.x & 31) == 0) mbar_arrive(&empty_bar[st]);  // this warp is done
      }
      if (!consumer) consumed = phase_end;
      // -- finalise the layer gathered in the previous phase ------------------------------
      double md = 0.0;
      if (fin_layer > 0) finalize(fin_layer, ab_prev, md);
      sync_phase(sA, sB, sa, sb, md, n, n >= 2 ? k : k - 1);
    }
  }
  // closing phase: final values of layer N-1 of the last sweep
  if (gphase > 0) {
    const int kl = a.nsweeps - 1;
    double md = 0.0;
    finalize(N - 1, (const P2*)(((gphase + 1) & 1) ? a.ab1 : a.ab0), md);
    sync_phase(V::zero(), V::zero(), V::zero(), V::zero(), md, -1, kl);
    if (threadIdx.x == 0 && blockIdx.x == 0) {
      for (int i = 0; i <= N; i++) {
        sc->lam_n[i] = s_lam[i];
        sc->mu_n[i] = s_mu[i];
      }
      sc->step_prev = a.nsweeps > 1 ? s_step[(kl - 1) & 1] : sc->step;
      sc->step = s_step[kl & 1];
      sc->sweeps += a.nsweeps;
      if (!isfinite(sc->step)) atomicOr(&sc->flags, 1);
    }
  }
}

int g_occ[3] = {0, 0, 0};
int g_nsm = 0;

template <class V>
int launch_persist(hq_solver* h, int nsweeps, cudaEvent_t ev0, cudaEvent_t ev1) {
  typedef typename V::T T;
  constexpr int kStageBytes = StageBytes<V>::v;
  const int slot = V::kind == HQ_PREC_FP64 ? 0 : (V::kind == HQ_PREC_DF64 ? 1 : 2);
  const size_t smem_max = (size_t)kStages * kStageBytes + (size_t)kMaxHi * kConsumers * 4;
  const size_t smem = (size_t)kStages * kStageBytes + (size_t)h->H * kConsumers * 4;
  if (!g_nsm) HQ_CUDA(cudaDeviceGetAttribute(&g_nsm, cudaDevAttrMultiProcessorCount, h->dev));
  if (!g_occ[slot]) {
    HQ_CUDA(cudaFuncSetAttribute(k_persist<V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_max));
  }
  int occ = 0;
  HQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_persist<V>, kThreads, smem));
  if (occ < 1) {
    hq_set_error("persistent sweep kernel does not fit on an SM");
    return HQ_ECUDA;
  }
  g_occ[slot] = occ;
  const int G = g_nsm * occ;
  if ((int64_t)G * kPW * 2 > h->partials_len) {
    hq_set_error("partials buffer too small for the persistent grid");
    return HQ_ECUDA;
  }
  PersistArgs a;
  memset(&a, 0, sizeof(a));
  a.N = h->N;
  a.L = h->L;
  a.H = h->H;
  a.nsweeps = nsweeps;
  a.lam = h->lam;
  for (int i = 0; i < HQ_MAXN + 2; i++) {
    a.off[i] = h->off[i];
    a.toff[i] = h->toff[i];
  }
  PrecBufs& b = hq_bufs(h, V::kind);
  if (b.rl.esize != (int)sizeof(T)) {
    hq_set_error("tile records do not match the sweep precision");
    return HQ_ECUDA;
  }
  for (int n = 0; n <= HQ_MAXN; n++) {
    a.lsize[n] = n <= h->N ? h->lsize[n] : 0;
    a.lpad[n] = n <= h->N ? h->lpad[n] : 0;
    a.tk[n] = b.rl.tk[n];
    a.ntiles[n] = b.rl.ntiles[n];
    a.rbytes[n] = b.rl.rbytes[n];
    if (b.rl.rbytes[n] > kStageBytes) {
      hq_set_error("a tile record is larger than a shared-memory stage");
      return HQ_ECUDA;
    }
  }
  for (int n = 0; n < HQ_MAXN + 2; n++) a.roff[n] = b.rl.roff[n];
  a.rec = (const unsigned char*)b.rec;
  a.RL = h->RL;
  a.RH = h->RH;
  a.p = b.p;
  a.nu = b.nu;
  a.ab0 = h->ab;
  a.ab1 = (char*)h->ab + h->ab_half_bytes;
  a.partials = h->partials;
  a.sc = h->sc;
  void* args[] = {&a};
  // a barrier left half-entered by an aborted launch must not leak into this one
  HQ_CUDA(cudaMemsetAsync(&h->sc->bar_count, 0, sizeof(unsigned), h->stream));
  if (ev0) HQ_CUDA(cudaEventRecord(ev0, h->stream));
  HQ_CUDA(cudaLaunchCooperativeKernel((const void*)k_persist<V>, dim3(G), dim3(kThreads), args, smem,
                                      h->stream));
  HQ_LAUNCHED();
  if (ev1) HQ_CUDA(cudaEventRecord(ev1, h->stream));
  return HQ_OK;
}

}  // namespace

PrecBufs& hq_bufs(hq_solver* h, int prec) {
  if (prec == HQ_PREC_FP64) return h->b64;
  if (prec == HQ_PREC_DF64) return h->bdf;
  return h->b32;
}

int hq_run_sweeps(hq_solver* h, int prec, int nsweeps, cudaEvent_t ev0, cudaEvent_t ev1) {
  if (h->N < 2 || nsweeps < 1) return HQ_OK;
  if (prec == HQ_PREC_FP64) return launch_persist<PolF64>(h, nsweeps, ev0, ev1);
  if (prec == HQ_PREC_DF64) return launch_persist<PolDF>(h, nsweeps, ev0, ev1);
  return launch_persist<PolF32>(h, nsweeps, ev0, ev1);
}

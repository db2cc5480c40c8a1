// Batched solves: Algorithm 1 (Eq. 12-14) on many instances of uneven N at once, one
// persistent cooperative launch per convergence check.
//
// A batch wraps K loaded solvers (their tables, rates, iterates and outputs stay theirs).
// Phase n of a sweep (n = 1..Nmax, Nmax the largest N of the batch) does, for every
// still-active instance c:
//   * finalise layer n-1 (if 2 <= n <= N_c): p = c1 A + c2 B with the c1, c2 published for
//     that layer at the previous phase, and the step max |p - p_old| folded into the
//     instance's step by an atomic max on its FP32 bit pattern (order-free, so exact);
//   * gather layer n (if n <= N_c - 1) into (A, B) pairs, item by item exactly as the
//     one-instance kernel does (hq_sweep_dev.cuh), each item writing its four partial sums
//     to its own slot;
// then a grid barrier, a fold of every instance's item partials in item order (CTA b
// takes the instances b, b + G, ...) that solves the instance's scalar recursion of
// layer n (closed-form inner limit, Eq. 13) in FP64, and a second grid barrier.  The
// instances' layer orders stay independent; only the barriers are shared.
//
// The host repeats [reset the step buffers, launch check_every sweeps, read the steps
// back] until every instance's step is below the tolerance; that sequence is captured
// once as a CUDA graph and replayed.  Mixed precision runs FP32 sweeps until the FP32
// steps stop shrinking, then converts every instance to DF64 (or FP64).  The kernel
// variant (CTA size and CTAs per SM) is chosen by hq_batch_tune from timed sweeps.
//
// Every wait is bounded (the two grid barriers); a timeout sets a flag and the host
// reports HQ_ETIMEOUT.
#include <math.h>
#include <string.h>

#include <chrono>
#include <vector>

#include "hq_sweep_dev.cuh"

namespace {

using namespace hqdev;

constexpr unsigned kSpinLimit = 1u << 24;
// the kernel variants the tuner chooses among: threads per CTA and CTAs per SM (at most;
// fewer where shared memory does not allow them), all at 64 registers per thread
constexpr int kVariants = 4;
constexpr int kVarThreads[kVariants] = {512, 1024, 512, 256};
constexpr int kVarCtas[kVariants] = {2, 1, 1, 4};

// per-instance view for the device (one array entry per instance)
struct BCfg {
  int N, L, H, pad;
  double lam;
  int64_t Sp;
  int64_t off[HQ_MAXN + 2];
  int64_t toff[HQ_MAXN + 2];
  int64_t lsize[HQ_MAXN + 1];
  int64_t lpad[HQ_MAXN + 1];
  int64_t tw[HQ_MAXN + 1];
  const uint32_t* masks;
  const uint32_t* lidx;
  const uint32_t* RH;
  const void* T[3];  // by precision slot: FP64, DF64, FP32
  const void* r[3];
  void* p[3];
  const void* nu[3];
  void* ab0;
  void* ab1;
  DevScalars* sc;
};

template <class V> struct PSlot { static constexpr int v = 2; };
template <> struct PSlot<PolF64> { static constexpr int v = 0; };
template <> struct PSlot<PolDF> { static constexpr int v = 1; };

struct BatchArgs {
  int K, Nmax, nsweeps;
  int ifirst[HQ_MAXN + 2];  // gather items of phase n
  int ffirst[HQ_MAXN + 2];  // finalise chunks of phase n
  int cfirst[HQ_MAXN + 2];  // fold entries of phase n
  const BCfg* cfg;
  const int* active;        // K flags
  const double* omega;      // K over-relaxations of the finalised layers (1: none)
  const uint4* items;       // the instances' items, phase by phase
  const int* icfg;          // instance of each item
  const uint4* fchunks;     // {instance, layer, first rank, count} of the finalise chunks
  const uint4* folds;       // {instance, first item, end item, 0}
  double* ipart;            // 4 partial sums per item
  unsigned* step_bits;      // [2][K] FP32 bit patterns of the per-sweep step maxima
  unsigned* bar;            // [0] arrivals, [1] (unused), [2] flags
  unsigned spin_limit;      // polls before a wait gives up (0: the default)
  int dbg_skip_cta;         // fault injection: this CTA skips its first barrier arrival (-1: none)
};

template <class V, int kThreads>
__global__ void __launch_bounds__(kThreads, 1024 / kThreads) k_batch(BatchArgs a) {
  typedef typename V::T T;
  typedef Pair<V> PR;
  typedef typename PR::P P2;
  constexpr int PS = PSlot<V>::v;
  constexpr int kWarps = kThreads / 32;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint32_t s_RL[1 << HQ_LO_BITS];
  __shared__ int s_bin[HQ_LO_BITS + 1][HQ_LO_BITS + 2];  // s_bin[L][i] = C(L, i - 1)
  __shared__ double s_red[4][kWarps];
  __shared__ uint32_t s_hl[kWarps][32];  // per warp: the item's high-part neighbour bases
  __shared__ T s_hnu[kWarps][32];        // and its idle high-part units' rates

  const unsigned G = gridDim.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned char* slot_d = smem + (size_t)wid * Slot<V>::kBytes;
  unsigned char* slot_u = slot_d + Slot<V>::kD;
  // RL[lo] (the colex rank of lo among the masks of its popcount) does not depend on the
  // width L, so one table of 2^HQ_LO_BITS entries serves every instance
  for (int i = threadIdx.x; i < (1 << HQ_LO_BITS); i += blockDim.x) {
    uint32_t r = 0;
    int t = 0;
    for (int b = 0; b < HQ_LO_BITS; b++)
      if ((i >> b) & 1) {
        t++;
        // C(b, t) by the multiplicative formula (b < 10: exact in double)
        double c = 1.0;
        for (int q = 1; q <= t; q++) c = c * (double)(b - t + q) / (double)q;
        r += (uint32_t)(c + 0.5);
      }
    s_RL[i] = r;
  }
  for (int i = threadIdx.x; i < (HQ_LO_BITS + 1) * (HQ_LO_BITS + 2); i += blockDim.x) {
    const int L = i / (HQ_LO_BITS + 2), k = i % (HQ_LO_BITS + 2) - 1;
    int c = 0;
    if (k >= 0 && k <= L) {
      double v = 1.0;
      for (int q = 1; q <= k; q++) v = v * (double)(L - k + q) / (double)q;
      c = (int)(v + 0.5);
    }
    s_bin[L][i % (HQ_LO_BITS + 2)] = c;
  }
  __syncthreads();

  const int gwarp = (int)blockIdx.x * kWarps + wid;
  const int nwarps = (int)G * kWarps;
  const int64_t nthreads = (int64_t)G * blockDim.x;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int gbar = 0;  // grid barriers passed in this launch

  // grid barrier: released arrivals on a counter (zeroed before the launch); every CTA
  // waits until the count of barrier g reaches G (g + 1)
  auto grid_barrier = [&]() {
    __syncthreads();
    if (threadIdx.x == 0) {
      if (!(a.dbg_skip_cta == (int)blockIdx.x && gbar == 0)) red_add_release(&a.bar[0], 1u);
      const unsigned target = G * (unsigned)(gbar + 1);
      const unsigned limit = a.spin_limit ? a.spin_limit : kSpinLimit;
      unsigned it = 0;
      while ((int)(ld_relaxed_u32(&a.bar[0]) - target) < 0) {
        if (*(volatile unsigned*)&a.bar[2] & 2u) break;
        if (++it > limit) {
          atomicOr(&a.bar[2], 2u);
          break;
        }
      }
      fence_acq_rel_gpu();
    }
    __syncthreads();
    gbar++;
  };

  for (int k = 0; k < a.nsweeps; k++) {
    unsigned* sbits = a.step_bits + (size_t)(k & 1) * a.K;
    for (int n = 1; n <= a.Nmax; n++) {
      const int par = (n - 1 + k * a.Nmax) & 1;  // (A, B) buffer of layer n: parity of its phase
      if (n == 1)
        for (int64_t c = gtid; c < a.K; c += nthreads) sbits[c] = 0u;
      // -- finalise layer n-1 of every active instance --------------------------------------
      for (int ch = a.ffirst[n] + gwarp; ch < a.ffirst[n + 1]; ch += nwarps) {
        const uint4 f = __ldg(a.fchunks + ch);
        const int c = (int)f.x;
        if (!a.active[c]) continue;
        const BCfg& C = a.cfg[c];
        const int lf = (int)f.y;
        const T c1 = V::from_d(__ldcg(&C.sc->c1[lf])), c2 = V::from_d(__ldcg(&C.sc->c2[lf]));
        const double omd = a.omega[c];
        const T om = V::from_d(omd);
        const P2* abf = (const P2*)((par ^ 1) ? C.ab1 : C.ab0);
        T* pl = (T*)C.p[PS] + C.off[lf];
        float md = 0.f;
        for (uint32_t q = f.z + lane; q < f.z + f.w; q += 32) {
          const P2 ab = ld_l2(abf + q);
          const T old = ld_l2(pl + q);
          T v = V::add(V::mul(c1, PR::A(ab)), V::mul(c2, PR::B(ab)));
          if (omd != 1.0) v = V::add(old, V::mul(om, V::sub(v, old)));
          md = fmaxf(md, V::absdiff(v, old));
          pl[q] = v;
        }
        for (int m = 16; m > 0; m >>= 1) md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, m));
        if (lane == 0 && md > 0.f) atomicMax(sbits + c, __float_as_uint(md));
      }
      // -- gather layer n of every active instance ------------------------------------------
      for (int it = a.ifirst[n] + gwarp; it < a.ifirst[n + 1]; it += nwarps) {
        const int c = __ldg(a.icfg + it);
        if (!a.active[c]) continue;
        const BCfg& C = a.cfg[c];
        LayerView<V> lv;
        lv.n = n;
        lv.N = C.N;
        lv.L = C.L;
        lv.H = C.H;
        lv.Sp = C.Sp;
        lv.off_n = C.off[n];
        lv.toff_n = C.toff[n];
        lv.lp = 1;
        lv.tw = C.tw[n];
        lv.masks = C.masks;
        lv.lidx = C.lidx;
        lv.RH = C.RH;
        lv.Tt = (const T*)C.T[PS];
        lv.rt = (const T*)C.r[PS];
        lv.p_up = (const T*)C.p[PS] + C.off[n + 1];
        lv.ab_prev = (const P2*)((par ^ 1) ? C.ab1 : C.ab0);
        lv.ab_cur = (P2*)(par ? C.ab1 : C.ab0);
        lv.nu = (const T*)C.nu[PS];
        lv.c1 = n > 1 ? V::from_d(__ldcg(&C.sc->c1[n - 1])) : V::zero();
        lv.c2 = n > 1 ? V::from_d(__ldcg(&C.sc->c2[n - 1])) : V::zero();
        lv.lamT = V::from_d(C.lam);
        lv.one = V::from_d(1.0);
        T sA = V::zero(), sB = V::zero(), sa = V::zero(), sb = V::zero();
        gather_item<V, false>(lv, __ldg(a.items + it), s_RL, s_bin[C.L], slot_d, slot_u, s_hl[wid],
                              s_hnu[wid], lane, sA, sB, sa, sb);
        __syncwarp();
        sA = warp_sum<V>(sA);
        sB = warp_sum<V>(sB);
        sa = warp_sum<V>(sa);
        sb = warp_sum<V>(sb);
        if (lane == 0) {
          double* q = a.ipart + (size_t)it * 4;
          q[0] = V::to_d(sA);
          q[1] = V::to_d(sB);
          q[2] = V::to_d(sa);
          q[3] = V::to_d(sb);
        }
      }
      grid_barrier();
      // -- fold each instance's item partials in item order, solve its layer-n scalars -------
      for (int e = a.cfirst[n] + (int)blockIdx.x; e < a.cfirst[n + 1]; e += (int)G) {
        const uint4 fe = __ldg(a.folds + e);
        const int c = (int)fe.x;
        if (!a.active[c]) continue;  // uniform across the CTA
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        for (uint32_t it = fe.y + threadIdx.x; it < fe.z; it += blockDim.x) {
#pragma unroll
          for (int w = 0; w < 4; w++) v[w] += __ldcg(a.ipart + (size_t)it * 4 + w);
        }
#pragma unroll
        for (int w = 0; w < 4; w++)
          for (int m = 16; m > 0; m >>= 1) v[w] += __shfl_xor_sync(0xffffffffu, v[w], m);
        if (lane == 0)
#pragma unroll
          for (int w = 0; w < 4; w++) s_red[w][wid] = v[w];
        __syncthreads();
        if (wid == 0) {
          double f[4];
#pragma unroll
          for (int w = 0; w < 4; w++) {
            f[w] = lane < kWarps ? s_red[w][lane] : 0.0;
            for (int m = 16; m > 0; m >>= 1) f[w] += __shfl_xor_sync(0xffffffffu, f[w], m);  // lanes past kWarps hold 0
          }
          if (lane == 0) {
            // closed-form limit of the inner loop (Eq. 12 and 14), then Eq. (13)
            DevScalars* sc = a.cfg[c].sc;
            const double alpha = 1.0 / sc->lam_n[n - 1];
            const double beta = sc->lam_n[n] / sc->mu_n[n + 1];
            const double aa = alpha * f[0], bb = beta * f[1];
            const double mustar = bb / (1.0 - aa);
            const double c1 = alpha * mustar;
            sc->c1[n] = c1;
            sc->c2[n] = beta;
            sc->lam_n[n] = a.cfg[c].lam * (c1 * f[2] + beta * f[3]);
            sc->mu_n[n] = mustar;
            if (!isfinite(mustar) || !(aa < 1.0)) atomicOr(&a.bar[2], 1u);
          }
        }
        __syncthreads();
      }
      grid_barrier();
    }
  }
}

template <class V>
const void* kernel_of(int variant) {
  const int t = kVarThreads[variant];
  if (t == 1024) return (const void*)k_batch<V, 1024>;
  if (t == 256) return (const void*)k_batch<V, 256>;
  return (const void*)k_batch<V, 512>;
}

}  // namespace

struct hq_batch {
  int K = 0, Nmax = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int dev = 0, nsm = 0;
  std::vector<hq_solver*> s;
  std::vector<BCfg> hcfg;
  BCfg* cfg = nullptr;
  int* active = nullptr;
  double* omega = nullptr;
  uint4* items = nullptr;
  int* icfg = nullptr;
  uint4* fchunks = nullptr;
  uint4* folds = nullptr;
  double* ipart = nullptr;
  unsigned* step_bits = nullptr;
  unsigned* hstep = nullptr;  // pinned: [2][K]
  unsigned* bar = nullptr;
  int ifirst[HQ_MAXN + 2], ffirst[HQ_MAXN + 2], cfirst[HQ_MAXN + 2];
  int64_t nitems = 0, states = 0;
  int variant[3] = {0, 0, 0};  // tuned variant per precision slot
  // graph of one convergence check, per (precision slot, variant, sweeps)
  cudaGraphExec_t exec = nullptr;
  int exec_key[3] = {-1, -1, -1};
  int graph_state = 0;  // 0 untried, 1 graph replay in use, -1 capture refused: direct launches
  BatchArgs args;
};

namespace {

int slot_of(int prec) { return prec == HQ_PREC_FP64 ? 0 : (prec == HQ_PREC_DF64 ? 1 : 2); }

template <class V>
size_t smem_of(int variant) { return (size_t)(kVarThreads[variant] / 32) * Slot<V>::kBytes; }

size_t smem_for(int prec, int variant) {
  if (prec == HQ_PREC_FP64) return smem_of<PolF64>(variant);
  if (prec == HQ_PREC_DF64) return smem_of<PolDF>(variant);
  return smem_of<PolF32>(variant);
}

const void* kernel_for(int prec, int variant) {
  if (prec == HQ_PREC_FP64) return kernel_of<PolF64>(variant);
  if (prec == HQ_PREC_DF64) return kernel_of<PolDF>(variant);
  return kernel_of<PolF32>(variant);
}

int grid_for(hq_batch* b, int prec, int variant, int* G) {
  const void* k = kernel_for(prec, variant);
  const size_t sm = smem_for(prec, variant);
  HQ_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  int occ = 0;
  HQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kVarThreads[variant], sm));
  if (occ < 1) {
    hq_set_error("batched sweep kernel does not fit on an SM");
    return HQ_ECUDA;
  }
  const int want = kVarCtas[variant];
  *G = b->nsm * (occ < want ? occ : want);
  return HQ_OK;
}

// record [reset steps, sweeps, read steps back] on b->stream (launch or capture)
int record_check(hq_batch* b, int prec, int variant, int nsweeps) {
  int G = 0;
  int rc = grid_for(b, prec, variant, &G);
  if (rc != HQ_OK) return rc;
  if ((int64_t)G * 2 * b->Nmax * (int64_t)nsweeps >= ((int64_t)1 << 31)) {
    hq_set_error("too many barrier arrivals for one batched launch");
    return HQ_EINVAL;
  }
  b->args.nsweeps = nsweeps;
  HQ_CUDA(cudaMemsetAsync(b->bar, 0, sizeof(unsigned), b->stream));  // arrivals
  cudaLaunchConfig_t lc;
  memset(&lc, 0, sizeof(lc));
  lc.gridDim = dim3(G);
  lc.blockDim = dim3(kVarThreads[variant]);
  lc.dynamicSmemBytes = smem_for(prec, variant);
  lc.stream = b->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  void* params[] = {&b->args};
  HQ_CUDA(cudaLaunchKernelExC(&lc, kernel_for(prec, variant), params));
  HQ_LAUNCHED();
  HQ_CUDA(cudaMemcpyAsync(b->hstep, b->step_bits, sizeof(unsigned) * 2 * b->K, cudaMemcpyDeviceToHost,
                          b->stream));
  return HQ_OK;
}

// one convergence check through the captured graph (re-captured when its key changes);
// if this CUDA stack refuses to capture the cooperative launch, checks launch directly
int run_check(hq_batch* b, int prec, int variant, int nsweeps) {
  const int key[3] = {slot_of(prec), variant, nsweeps};
  if (b->graph_state >= 0 && (!b->exec || memcmp(key, b->exec_key, sizeof(key)) != 0)) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    HQ_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int rc = record_check(b, prec, variant, nsweeps);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (rc == HQ_OK && e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (rc != HQ_OK || e != cudaSuccess) {
      cudaGetLastError();
      if (b->exec) cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
      b->graph_state = -1;
    } else {
      b->graph_state = 1;
      memcpy(b->exec_key, key, sizeof(key));
    }
  }
  if (b->graph_state == 1) {
    HQ_CUDA(cudaGraphLaunch(b->exec, b->stream));
  } else {
    const int rc = record_check(b, prec, variant, nsweeps);
    if (rc != HQ_OK) return rc;
  }
  HQ_CUDA(cudaStreamSynchronize(b->stream));
  return HQ_OK;
}

void free_batch(hq_batch* b) {
  void* ptrs[] = {b->cfg, b->active, b->omega, b->items, b->icfg, b->fchunks, b->folds, b->ipart,
                  b->step_bits, b->bar};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (b->hstep) cudaFreeHost(b->hstep);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

template <class T>
int dupload(T** dst, const std::vector<T>& v) {
  const size_t bytes = sizeof(T) * (v.empty() ? 1 : v.size());
  cudaError_t e = cudaMalloc((void**)dst, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    hq_set_error("cudaMalloc of batch metadata failed");
    return HQ_ENOMEM;
  }
  if (!v.empty()) HQ_CUDA(cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  return HQ_OK;
}

// run `fn` with every solver's work on the batch stream
template <class F>
int on_batch_stream(hq_batch* b, F fn) {
  int rc = HQ_OK;
  for (hq_solver* h : b->s) {
    cudaStream_t saved = h->stream;
    h->stream = b->stream;
    rc = fn(h);
    h->stream = saved;
    if (rc != HQ_OK) break;
  }
  return rc;
}

// A solver of the batch may have been loaded with another instance of its size since the
// batch was made: bring the per-instance total rate (the one value of an instance the
// batch keeps by value) up to date, and make the double-float tables, on the batch's
// stream.
int refresh_instances(hq_batch* b) {
  bool stale = false;
  for (int c = 0; c < b->K; c++)
    if (b->hcfg[c].lam != b->s[c]->lam) {
      b->hcfg[c].lam = b->s[c]->lam;
      stale = true;
    }
  if (stale) {
    HQ_CUDA(cudaMemcpyAsync(b->cfg, b->hcfg.data(), sizeof(BCfg) * b->hcfg.size(), cudaMemcpyHostToDevice,
                            b->stream));
    HQ_CUDA(cudaStreamSynchronize(b->stream));
  }
  return on_batch_stream(b, [&](hq_solver* h) { return hq_ensure_df(h); });
}

}  // namespace

extern "C" int hq_batch_create(hq_solver* const* solvers, int count, void* stream, hq_batch** out) {
  if (!out) { hq_set_error("out is NULL"); return HQ_EINVAL; }
  *out = nullptr;
  if (!solvers || count < 1) { hq_set_error("need at least one solver"); return HQ_EINVAL; }
  for (int c = 0; c < count; c++) {
    if (!solvers[c]) { hq_set_error("NULL solver in the batch"); return HQ_EINVAL; }
    if (!solvers[c]->loaded) { hq_set_error("every solver of a batch must be loaded"); return HQ_ESTATE; }
    if (solvers[c]->N < 2) { hq_set_error("batched solvers need N >= 2"); return HQ_EINVAL; }
    if (solvers[c]->N > HQ_DF_MAXN) { hq_set_error("batched solvers need N <= 28"); return HQ_EINVAL; }
  }

  hq_batch* b = new hq_batch();
  b->K = count;
  b->s.assign(solvers, solvers + count);
  cudaGetDevice(&b->dev);
  for (hq_solver* h : b->s)
    if (h->dev != b->dev) {
      delete b;
      hq_set_error("every solver of a batch must live on the current device");
      return HQ_EINVAL;
    }
  cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->dev);
  b->stream = (cudaStream_t)stream;
  if (!b->stream) {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete b;
      hq_set_error("cudaStreamCreateWithFlags failed");
      return HQ_ECUDA;
    }
    b->own_stream = true;
  }
  for (hq_solver* h : b->s)
    if (h->N > b->Nmax) b->Nmax = h->N;
  // per-instance views
  b->hcfg.resize(count);
  for (int c = 0; c < count; c++) {
    hq_solver* h = b->s[c];
    BCfg& C = b->hcfg[c];
    memset(&C, 0, sizeof(C));
    C.N = h->N;
    C.L = h->L;
    C.H = h->H;
    C.lam = h->lam;
    C.Sp = h->Sp;
    for (int i = 0; i < HQ_MAXN + 2; i++) {
      C.off[i] = h->off[i];
      C.toff[i] = h->toff[i];
    }
    for (int i = 0; i <= HQ_MAXN; i++) {
      C.lsize[i] = i <= h->N ? h->lsize[i] : 0;
      C.lpad[i] = i <= h->N ? h->lpad[i] : 0;
      C.tw[i] = i <= h->N ? h->tw[i] : 0;
    }
    C.masks = h->masks;
    C.lidx = h->lidx;
    C.RH = h->RH;
    PrecBufs* pb[3] = {&h->b64, &h->bdf, &h->b32};
    for (int q = 0; q < 3; q++) {
      C.T[q] = pb[q]->T;
      C.r[q] = pb[q]->r;
      C.p[q] = pb[q]->p;
      C.nu[q] = pb[q]->nu;
    }
    C.ab0 = h->ab;
    C.ab1 = (char*)h->ab + h->ab_half_bytes;
    C.sc = h->sc;
  }
  // items, finalise chunks and folds, phase by phase
  std::vector<std::vector<uint4>> own(count);
  std::vector<std::vector<int>> own_first(count, std::vector<int>(HQ_MAXN + 2));
  for (int c = 0; c < count; c++) {
    int rc = hq_item_list(b->s[c]->N, own[c], own_first[c].data());
    if (rc != HQ_OK) {
      delete b;
      return rc;
    }
  }
  std::vector<uint4> items, fchunks, folds;
  std::vector<int> icfg;
  for (int n = 0; n <= HQ_MAXN + 1; n++) b->ifirst[n] = b->ffirst[n] = b->cfirst[n] = 0;
  for (int n = 1; n <= b->Nmax; n++) {
    b->ifirst[n] = (int)items.size();
    b->ffirst[n] = (int)fchunks.size();
    b->cfirst[n] = (int)folds.size();
    for (int c = 0; c < count; c++) {
      const int Nc = b->s[c]->N;
      if (n >= 2 && n <= Nc) {
        const uint32_t sz = (uint32_t)b->s[c]->lsize[n - 1];
        for (uint32_t k0 = 0; k0 < sz; k0 += 256)
          fchunks.push_back(make_uint4((uint32_t)c, (uint32_t)(n - 1), k0, sz - k0 < 256 ? sz - k0 : 256));
      }
      if (n <= Nc - 1) {
        const uint32_t f0 = (uint32_t)items.size();
        for (int q = own_first[c][n]; q < own_first[c][n + 1]; q++) {
          items.push_back(own[c][q]);
          icfg.push_back(c);
        }
        folds.push_back(make_uint4((uint32_t)c, f0, (uint32_t)items.size(), 0u));
      }
    }
  }
  b->ifirst[b->Nmax + 1] = (int)items.size();
  b->ffirst[b->Nmax + 1] = (int)fchunks.size();
  b->cfirst[b->Nmax + 1] = (int)folds.size();
  b->nitems = (int64_t)items.size();
  for (hq_solver* h : b->s) b->states += h->S - 2;
  std::vector<int> act(count, 1);
  int rc = dupload(&b->cfg, b->hcfg);
  if (rc == HQ_OK) rc = dupload(&b->active, act);
  if (rc == HQ_OK) rc = dupload(&b->omega, std::vector<double>(count, 1.0));
  if (rc == HQ_OK) rc = dupload(&b->items, items);
  if (rc == HQ_OK) rc = dupload(&b->icfg, icfg);
  if (rc == HQ_OK) rc = dupload(&b->fchunks, fchunks);
  if (rc == HQ_OK) rc = dupload(&b->folds, folds);
  if (rc == HQ_OK) rc = dupload(&b->ipart, std::vector<double>((size_t)(b->nitems > 0 ? b->nitems : 1) * 4, 0.0));
  if (rc == HQ_OK) rc = dupload(&b->step_bits, std::vector<unsigned>((size_t)2 * count, 0u));
  if (rc == HQ_OK) rc = dupload(&b->bar, std::vector<unsigned>(4, 0u));
  if (rc == HQ_OK && cudaMallocHost((void**)&b->hstep, sizeof(unsigned) * 2 * count) != cudaSuccess) {
    cudaGetLastError();
    hq_set_error("cudaMallocHost failed");
    rc = HQ_ENOMEM;
  }
  if (rc != HQ_OK) {
    free_batch(b);
    delete b;
    return rc;
  }
  BatchArgs& a = b->args;
  memset(&a, 0, sizeof(a));
  a.K = count;
  a.Nmax = b->Nmax;
  for (int n = 0; n < HQ_MAXN + 2; n++) {
    a.ifirst[n] = b->ifirst[n];
    a.ffirst[n] = b->ffirst[n];
    a.cfirst[n] = b->cfirst[n];
  }
  a.cfg = b->cfg;
  a.active = b->active;
  a.omega = b->omega;
  a.items = b->items;
  a.icfg = b->icfg;
  a.fchunks = b->fchunks;
  a.folds = b->folds;
  a.ipart = b->ipart;
  a.step_bits = b->step_bits;
  a.bar = b->bar;
  a.dbg_skip_cta = -1;
  *out = b;
  return HQ_OK;
}

extern "C" void hq_batch_destroy(hq_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  free_batch(b);
  delete b;
}

extern "C" int hq_batch_set_variant(hq_batch* b, int precision, int variant) {
  if (!b) { hq_set_error("NULL batch"); return HQ_EINVAL; }
  if (precision != HQ_PREC_FP64 && precision != HQ_PREC_DF64 && precision != HQ_PREC_FP32) {
    hq_set_error("precision must be FP64, DF64 or FP32");
    return HQ_EINVAL;
  }
  if (variant < 0 || variant >= kVariants) {
    hq_set_error("variant out of range");
    return HQ_EINVAL;
  }
  b->variant[slot_of(precision)] = variant;
  return HQ_OK;
}

extern "C" int hq_batch_info(const hq_batch* b, int64_t* out8) {
  if (!b || !out8) { hq_set_error("NULL argument"); return HQ_EINVAL; }
  out8[0] = b->K;
  out8[1] = b->Nmax;
  out8[2] = b->states;
  out8[3] = b->nitems;
  out8[4] = b->graph_state;
  out8[5] = b->variant[0];
  out8[6] = b->variant[1];
  out8[7] = b->variant[2];
  return HQ_OK;
}

// Autotuner: time every kernel variant on `sweeps` sweeps from the current iterates (the
// first call of a precision initialises them cold) and keep the fastest.
extern "C" int hq_batch_tune(hq_batch* b, int precision, int sweeps, int* variant_out, float* ms_out) {
  if (!b) { hq_set_error("NULL batch"); return HQ_EINVAL; }
  if (precision != HQ_PREC_FP64 && precision != HQ_PREC_DF64 && precision != HQ_PREC_FP32) {
    hq_set_error("precision must be FP64, DF64 or FP32");
    return HQ_EINVAL;
  }
  if (sweeps < 1) sweeps = 1;
  int rc = refresh_instances(b);
  if (rc != HQ_OK) return rc;
  rc = on_batch_stream(b, [&](hq_solver* h) { return hq_init_iterate(h, precision, nullptr, HQ_HOST); });
  if (rc != HQ_OK) return rc;
  std::vector<int> act(b->K, 1);
  std::vector<double> om1(b->K, 1.0);
  HQ_CUDA(cudaMemcpyAsync(b->active, act.data(), sizeof(int) * b->K, cudaMemcpyHostToDevice, b->stream));
  HQ_CUDA(cudaMemcpyAsync(b->omega, om1.data(), sizeof(double) * b->K, cudaMemcpyHostToDevice, b->stream));
  HQ_CUDA(cudaStreamSynchronize(b->stream));
  cudaEvent_t e0, e1;
  HQ_CUDA(cudaEventCreate(&e0));
  HQ_CUDA(cudaEventCreate(&e1));
  int best = 0;
  float best_ms = 0.f;
  for (int v = 0; v < kVariants && rc == HQ_OK; v++) {
    float ms = 0.f;
    for (int rep = 0; rep < 2 && rc == HQ_OK; rep++) {  // the first run warms up
      cudaEventRecord(e0, b->stream);
      rc = record_check(b, precision, v, sweeps);
      cudaEventRecord(e1, b->stream);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
    }
    if (rc != HQ_OK) break;
    if (ms_out) ms_out[v] = ms / sweeps;
    if (v == 0 || ms < best_ms) {
      best = v;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  HQ_CUDA(cudaStreamSynchronize(b->stream));
  if (rc != HQ_OK) return rc;
  if (b->bar && cudaMemcpy(b->hstep, b->bar + 2, sizeof(unsigned), cudaMemcpyDeviceToHost) == cudaSuccess &&
      (b->hstep[0] & 2u)) {
    hq_set_error("a bounded wait in the batched sweep kernel gave up");
    return HQ_ETIMEOUT;
  }
  b->variant[slot_of(precision)] = best;
  if (variant_out) *variant_out = best;
  for (hq_solver* h : b->s) {
    h->cur_prec = precision;
    h->it_version++;
  }
  return HQ_OK;
}

// Solve every instance of the batch to opts->tol on Algorithm 1's step (tol_kind must be
// HQ_TOL_STEP); per-instance outputs then come from each solver's getters.
extern "C" int hq_batch_solve(hq_batch* b, const hq_opts* opts_in, hq_stats* stats, double* ms_total) {
  if (!b) { hq_set_error("NULL batch"); return HQ_EINVAL; }
  hq_opts o;
  if (opts_in) o = *opts_in;
  else hq_default_opts(&o);
  if (o.tol_kind != HQ_TOL_STEP) { hq_set_error("batched solves stop on the step (HQ_TOL_STEP)"); return HQ_EINVAL; }
  if (o.warm_start != HQ_WARM_NONE) { hq_set_error("batched solves start cold"); return HQ_EINVAL; }
  if (o.check_every < 1) o.check_every = 1;
  if (o.precision < HQ_PREC_FP64 || o.precision > HQ_PREC_FP32_FP64) { hq_set_error("bad precision"); return HQ_EINVAL; }
  if (o.debug_barrier < 0) { hq_set_error("debug_barrier must be >= 0"); return HQ_EINVAL; }
  if (!(o.omega < 2.0) || (o.omega >= 0.0 && o.omega < 1.0 && o.omega != 0.0)) {
    hq_set_error("omega must be 0, in [1, 2), or negative (automatic)");
    return HQ_EINVAL;
  }
  {
    const int rcr = refresh_instances(b);
    if (rcr != HQ_OK) return rcr;
  }
  const bool auto_omega = o.omega < 0.0;
  const double stall = o.fp32_stall > 0.0 ? o.fp32_stall : 0.9;
  auto t0 = std::chrono::steady_clock::now();
  int phases[2];
  int nph = 1;
  switch (o.precision) {
    case HQ_PREC_FP64: phases[0] = HQ_PREC_FP64; break;
    case HQ_PREC_DF64: phases[0] = HQ_PREC_DF64; break;
    case HQ_PREC_FP32: phases[0] = HQ_PREC_FP32; break;
    case HQ_PREC_FP32_DF64: phases[0] = HQ_PREC_FP32; phases[1] = HQ_PREC_DF64; nph = 2; break;
    default: phases[0] = HQ_PREC_FP32; phases[1] = HQ_PREC_FP64; nph = 2; break;
  }
  const int K = b->K;
  int rc = on_batch_stream(b, [&](hq_solver* h) {
    h->solved = false;
    return hq_init_iterate(h, phases[0], nullptr, HQ_HOST);
  });
  if (rc != HQ_OK) return rc;
  std::vector<int> act(K, 1), conv(K, 0), sw32(K, 0), swhi(K, 0), stalled(K, 0), flat(K, 0);
  std::vector<double> step(K, INFINITY), prev(K, 0.0), om(K, o.omega >= 1.0 ? o.omega : 1.0);
  std::vector<int> checks(K, 0);
  HQ_CUDA(cudaMemcpyAsync(b->active, act.data(), sizeof(int) * K, cudaMemcpyHostToDevice, b->stream));
  HQ_CUDA(cudaMemcpyAsync(b->omega, om.data(), sizeof(double) * K, cudaMemcpyHostToDevice, b->stream));
  HQ_CUDA(cudaMemsetAsync(b->bar + 2, 0, sizeof(unsigned), b->stream));
  int ph = 0, total = 0, status = HQ_OK;
  while (total < o.max_sweeps) {
    const int prec = phases[ph];
    int nrun = o.check_every;
    if (nrun > o.max_sweeps - total) nrun = o.max_sweeps - total;
    if (o.debug_barrier > 0 && total == 0) {
      // fault injection (tests): one direct launch in which CTA debug_barrier - 1 skips its
      // first grid-barrier arrival and every wait gives up after 2^20 polls; the captured
      // graph never holds these arguments
      b->args.dbg_skip_cta = o.debug_barrier - 1;
      b->args.spin_limit = 1u << 20;
      rc = record_check(b, prec, b->variant[slot_of(prec)], nrun);
      if (rc == HQ_OK) {
        cudaError_t e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) rc = hq_cuda_fail(e, "batched launch", __FILE__, __LINE__);
      }
      b->args.dbg_skip_cta = -1;
      b->args.spin_limit = 0;
    } else {
      rc = run_check(b, prec, b->variant[slot_of(prec)], nrun);
    }
    if (rc != HQ_OK) return rc;
    total += nrun;
    unsigned flags = 0;
    HQ_CUDA(cudaMemcpy(&flags, b->bar + 2, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (flags & 2u) {
      hq_set_error("a bounded wait in the batched sweep kernel gave up");
      status = HQ_ETIMEOUT;
      break;
    }
    const unsigned* last = b->hstep + (size_t)((nrun - 1) & 1) * K;
    bool all_stalled = true, any_active = false;
    for (int c = 0; c < K; c++) {
      if (!act[c]) continue;
      (prec == HQ_PREC_FP32 ? sw32[c] : swhi[c]) += nrun;
      float f;
      memcpy(&f, last + c, sizeof(f));
      step[c] = f;
      if (!isfinite(step[c]) || (flags & 1u)) status = HQ_EDIVERGED;
      const double ratio = prev[c] > 0.0 ? step[c] / prev[c] : 0.0;
      if (auto_omega) {
        // as hq_solve: Young's omega for the contraction over the second check, at most
        // 1.9; halfway back whenever the steps stop shrinking
        checks[c]++;
        if (om[c] == 1.0 && checks[c] == 2 && ratio > 0.0 && ratio < 1.0) {
          const double r = pow(ratio, 1.0 / nrun);
          om[c] = fmin(2.0 / (1.0 + sqrt(1.0 - r)), 1.9);
        } else if (om[c] > 1.0 && ratio >= 1.0) {
          om[c] = 1.0 + 0.5 * (om[c] - 1.0);
        }
      }
      if (ph == nph - 1) {
        if (step[c] <= o.tol) {
          conv[c] = 1;
          act[c] = 0;
        } else if (prev[c] > 0.0 && ratio >= 1.0) {
          // a precision floor above the tolerance: stop this instance, as hq_solve does
          if (++flat[c] >= 4) act[c] = 0;
        } else {
          flat[c] = 0;
        }
      } else {
        // FP32 has stalled for this instance once its step stops shrinking (sticky: the
        // steps at the rounding floor fluctuate)
        if ((prev[c] > 0.0 && ratio > stall) || step[c] == 0.0) stalled[c] = 1;
        if (!stalled[c]) all_stalled = false;
      }
      prev[c] = step[c];
      any_active = any_active || act[c];
    }
    if (status != HQ_OK) {
      hq_set_error("non-finite value in the batched iteration");
      break;
    }
    if (!any_active) break;
    if (ph < nph - 1 && all_stalled) {
      rc = on_batch_stream(b, [&](hq_solver* h) { return hq_convert_iterate(h, phases[ph], phases[ph + 1]); });
      if (rc != HQ_OK) return rc;
      ph++;
      for (int c = 0; c < K; c++) {
        prev[c] = 0.0;
        flat[c] = 0;
      }
    }
    HQ_CUDA(cudaMemcpyAsync(b->active, act.data(), sizeof(int) * K, cudaMemcpyHostToDevice, b->stream));
    HQ_CUDA(cudaMemcpyAsync(b->omega, om.data(), sizeof(double) * K, cudaMemcpyHostToDevice, b->stream));
  }
  HQ_CUDA(cudaStreamSynchronize(b->stream));
  for (hq_solver* h : b->s) {
    h->cur_prec = phases[ph];
    h->it_version++;  // the batched kernel moved every iterate
  }
  std::vector<double> res(K, -1.0);
  if (status == HQ_OK) {
    int c = 0;
    rc = on_batch_stream(b, [&](hq_solver* h) {
      const int r = hq_finalize(h, phases[ph], true, &res[c]);
      if (r == HQ_OK) h->solved = true;
      c++;
      return r;
    });
    if (rc != HQ_OK) return rc;
  }
  if (stats) {
    for (int c = 0; c < K; c++) {
      hq_stats& st = stats[c];
      memset(&st, 0, sizeof(st));
      st.sweeps_fp32 = sw32[c];
      st.sweeps_hi = swhi[c];
      st.converged = conv[c];
      st.final_step = step[c];
      st.final_residual = res[c];
      st.ms_table = b->s[c]->ms_table;
      st.state_updates = (double)(b->s[c]->S - 2) * (double)(sw32[c] + swhi[c]);
      st.omega = om[c];
    }
  }
  if (ms_total) *ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (status != HQ_OK) return status;
  for (int c = 0; c < K; c++)
    if (!conv[c]) return HQ_ENOTCONVERGED;
  return HQ_OK;
}

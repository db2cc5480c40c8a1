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
// does not read it), and a closing phase finalises the last sweep.  Once every CTA has
// arrived at a barrier, each CTA folds all CTAs' partial sums in the same fixed order
// and solves the layer's scalar recursion (c1, c2, lambda(n), mu(n), the step) itself:
// the result is deterministic and identical in every CTA, and no CTA waits for another
// to publish it.
//
// Work.  Layer n is cut into items of at most 32 consecutive states of one rank block
// (see HQ_ITEM_HI_BITS); items go round-robin to the warps of the grid.  A warp first
// copies the two small blocks that hold its states' neighbours across a low-part unit,
// (hi, w-1) of the (A, B) pairs of layer n-1 and (hi, w+1) of p of layer n+1, into its
// own slot of shared memory with coalesced loads, so that the scattered part of the
// gather reads shared memory; the positions there come precomputed per state (lidx).
// Neighbours across a high-part unit, and the table rows, are read with coalesced loads
// straight from global memory: one lane per state, consecutive states at consecutive
// addresses.  The gather has no per-neighbour branch: the low-part steps are unrolled
// over the lidx bytes, the high-part ones run over a per-warp list of the item's
// neighbour blocks, and the low-part table entries are loaded before the staging wait.
// There is no producer, no stage ring and no wait other than the grid barrier.
//
// The grid barrier's wait is bounded: a barrier that does not complete within its
// iteration limit sets an error bit in DevScalars::flags and the kernel runs to its end
// with in-bounds indices; the host reports HQ_ETIMEOUT.
#include <stdlib.h>
#include <string.h>

#include "hq_sweep_dev.cuh"

namespace {

using namespace hqdev;

constexpr int kThreads = 1024;            // 32 warps, one CTA per SM at 64 registers:
                                          // half the grid arrivals and partials of 2 x 512
constexpr int kWarps = kThreads / 32;
constexpr int kPW = 6;                    // partial words per CTA per phase
constexpr unsigned kSpinLimit = 1u << 24;

struct PersistArgs {
  int N, L, H, nsweeps;
  double lam;
  double omega;                 // over-relaxation of the finalised layers (1: none)
  int64_t Sp;
  int64_t off[HQ_MAXN + 2];     // padded per-state offsets of the layers
  int64_t toff[HQ_MAXN + 2];    // padded table offsets of the layers
  int64_t lsize[HQ_MAXN + 1];
  int64_t lpad[HQ_MAXN + 1];    // table row stride of layer n
  int ifirst[HQ_MAXN + 2];      // items of layer n: [ifirst[n], ifirst[n+1])
  const uint4* items;
  const uint32_t* masks;
  const uint32_t* lidx;
  const uint32_t* RL;
  const uint32_t* RH;
  const void* T;
  const void* r;
  void* p;
  const void* nu;
  void* ab0;
  void* ab1;
  double* partials;  // [2][gridDim][kPW]
  DevScalars* sc;
  const float* ir;   // correction sweeps: 6 x Sp base terms {rho0, A0, B0, G_rho, G_A, G_B}
};

template <class V, bool kFullL, bool kIR>
__global__ void __launch_bounds__(kThreads, 1) k_persist(PersistArgs a) {
  typedef typename V::T T;
  typedef Pair<V> PR;
  typedef typename PR::P P2;
  // per-warp slots: staged (A, B) block of layer n-1, then staged p block of layer n+1
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint32_t s_RL[1 << HQ_LO_BITS];
  __shared__ int s_binL[HQ_LO_BITS + 2];
  __shared__ double s_lam[HQ_MAXN + 1], s_mu[HQ_MAXN + 1];
  __shared__ T s_nu[HQ_MAXN];
  __shared__ double s_red[kPW][kWarps];
  __shared__ uint32_t s_hl[kWarps][32];  // per warp: the item's high-part neighbour bases
  __shared__ T s_hnu[kWarps][32];        // and its idle high-part units' rates
  __shared__ T s_lamT, s_one;
  __shared__ T s_c1, s_c2;
  __shared__ T s_d1, s_d2;  // correction sweeps: c1 - c1^0, c2 - c2^0 of the last layer solved
  __shared__ double s_step[2];
  __shared__ double s_alpha, s_beta;  // 1/lambda(n-1) and lambda(n)/mu(n+1) of the layer solved

  DevScalars* sc = a.sc;
  const int N = a.N, L = a.L, H = a.H;
  const unsigned G = gridDim.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned char* slot_d = smem + (size_t)wid * Slot<V>::kBytes;
  unsigned char* slot_u = slot_d + Slot<V>::kD;
  for (int i = threadIdx.x; i < (1 << L); i += blockDim.x) s_RL[i] = a.RL[i];
  if (threadIdx.x <= L + 1) {
    // C(L, i - 1): the sizes of the blocks (hi, w -/+ 1) are s_binL[w] and s_binL[w + 2]
    const int i = threadIdx.x;
    int c = 0;
    if (i >= 1) {
      double v = 1.0;
      for (int q = 1; q <= i - 1; q++) v = v * (double)(L - (i - 1) + q) / (double)q;
      c = (int)(v + 0.5);
    }
    s_binL[i] = c;
  }
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
    s_d1 = V::zero();
    s_d2 = V::zero();
    s_step[0] = s_step[1] = 0.0;
    if (blockIdx.x == 0) sc->t_start = globaltimer_ns();
  }
  __syncthreads();

  const T* pv = (const T*)a.p;
  T* pw = (T*)a.p;
  const T* Tt = (const T*)a.T;
  const T* rt = (const T*)a.r;
  const int gwarp = (int)blockIdx.x * kWarps + wid;
  const int nwarps = (int)G * kWarps;
  int gphase = 0;  // phase counter within this launch

  // finalise layer lf from the (A, B) buffer `abf`: p = c1 A + c2 B, |p - p_old|; in
  // correction sweeps e = rho0 + d1 A0 + d2 B0 + c1 a + c2 b (the pairs hold a, b)
  auto finalize = [&](int lf, const P2* abf, float& md) {
    const T c1 = s_c1, c2 = s_c2, d1 = s_d1, d2 = s_d2;
    const bool relax = a.omega != 1.0;
    const T om = V::from_d(a.omega);
    T* pl = pw + a.off[lf];
    const T* r0 = kIR ? (const T*)(a.ir + a.off[lf]) : nullptr;
    const int64_t Lf = a.lsize[lf];
    const int64_t nthreads = (int64_t)G * blockDim.x;
#pragma unroll 4
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < Lf; k += nthreads) {
      const P2 q = ld_l2(abf + k);
      const T old = ld_l2(pl + k);
      T v = V::add(V::mul(c1, PR::A(q)), V::mul(c2, PR::B(q)));
      if constexpr (kIR) {
        const T base = V::add(ld_stream(r0 + k),
                              V::add(V::mul(d1, ld_stream(r0 + a.Sp + k)), V::mul(d2, ld_stream(r0 + 2 * a.Sp + k))));
        v = V::add(base, v);
      }
      if (relax) v = V::add(old, V::mul(om, V::sub(v, old)));
      md = fmaxf(md, V::absdiff(v, old));
      pl[k] = v;
    }
  };

  // Write this CTA's partials, then the grid barrier.  Arrivals count up on bar_count
  // (zeroed before the launch, released by the arriving thread so that its partials are
  // visible); phase g completes when the count reaches G (g + 1).  Then every CTA folds
  // all partials in CTA order itself -- the same operations in the same order in every
  // CTA, so all hold the same scalars -- and solves the scalar recursion of layer lg
  // (if lg > 0).  The two ratios of the closed form that do not depend on this phase's
  // sums are formed while waiting.  ks: sweep of the layer finalised in this phase (its
  // step goes into s_step).
  auto sync_phase = [&](T sA, T sB, T sa, T sb, float md, int lg, int ks) {
    const int buf = gphase & 1;
    double* part = a.partials + (size_t)buf * kPW * G;  // [word][CTA]
    {
      T w4[4] = {sA, sB, sa, sb};
#pragma unroll
      for (int i = 0; i < 4; i++) {
        const T v = warp_sum<V>(w4[i]);
        if (lane == 0) s_red[i][wid] = V::to_d(v);
      }
      for (int m = 16; m > 0; m >>= 1) md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, m));
      if (lane == 0) s_red[4][wid] = (double)md;
    }
    __syncthreads();
    if (wid == 0) {
      // warp 0 folds the kWarps warp results of each word (few FP64 operations)
      double v[5];
#pragma unroll
      for (int w = 0; w < 5; w++) v[w] = lane < kWarps ? s_red[w][lane] : 0.0;
#pragma unroll
      for (int w = 0; w < 5; w++)
        for (int m = 16; m > 0; m >>= 1) {  // lanes past kWarps hold 0
          const double o = __shfl_xor_sync(0xffffffffu, v[w], m);
          v[w] = (w == 4) ? fmax(v[w], o) : v[w] + o;
        }
      if (lane == 0) {
        // this thread writes the CTA's partials, so its release covers them
#pragma unroll
        for (int w = 0; w < 5; w++) part[(size_t)w * G + blockIdx.x] = v[w];
        red_add_release(&sc->bar_count, 1u);
        if (lg > 0) {
          s_alpha = 1.0 / s_lam[lg - 1];
          s_beta = s_lam[lg] / s_mu[lg + 1];
        }
        const unsigned target = G * (unsigned)(gphase + 1);
        unsigned it = 0;
        while ((int)(ld_relaxed_u32(&sc->bar_count) - target) < 0) {
          if (*(volatile int*)&sc->flags & 6) break;  // an earlier wait gave up: do not wait again
          if (++it > kSpinLimit) {
            atomicOr(&sc->flags, 2);
            break;
          }
        }
        fence_acq_rel_gpu();
      }
    }
    __syncthreads();
    // fold every CTA's partials in CTA order: warp w < 5 takes word w
    if (wid < 5) {
      double v = 0.0;
      for (unsigned b = lane; b < G; b += 32) {
        const double x = __ldcg(part + (size_t)wid * G + b);
        v = (wid == 4) ? fmax(v, x) : v + x;
      }
      for (int m = 16; m > 0; m >>= 1) {
        const double o = __shfl_xor_sync(0xffffffffu, v, m);
        v = (wid == 4) ? fmax(v, o) : v + o;
      }
      if (lane == 0) s_red[wid][0] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double f[5];
#pragma unroll
      for (int w = 0; w < 5; w++) f[w] = s_red[w][0];
      if (kIR && lg > 0) {
        // the correction sums plus the base's: the sums of the full (A, B) of layer lg
#pragma unroll
        for (int w = 0; w < 4; w++) f[w] += sc->ir_sum[w][lg];
      }
      if (lg > 0) {
        // closed-form limit of the inner loop (Eq. 12 and 14), then Eq. (13)
        const double alpha = s_alpha, beta = s_beta;
        const double aa = alpha * f[0], bb = beta * f[1];
        const double mustar = bb / (1.0 - aa);
        const double c1 = alpha * mustar;
        s_c1 = V::from_d(c1);
        s_c2 = V::from_d(beta);
        if (kIR) {
          s_d1 = V::from_d(c1 - sc->ir_c1[lg]);
          s_d2 = V::from_d(beta - sc->ir_c2[lg]);
        }
        s_lam[lg] = a.lam * (c1 * f[2] + beta * f[3]);
        s_mu[lg] = mustar;
        if (blockIdx.x == 0) {
          sc->c1[lg] = c1;
          sc->c2[lg] = beta;
          if (!isfinite(mustar) || !(aa < 1.0)) atomicOr(&sc->flags, 1);
        }
      }
      s_step[ks & 1] = fmax(s_step[ks & 1], f[4]);
      if (blockIdx.x == 0 && gphase < 64) sc->t_phase[gphase] = globaltimer_ns();
    }
    __syncthreads();
    gphase++;
  };

  for (int k = 0; k < a.nsweeps; k++) {
    for (int n = 1; n <= N - 1; n++) {
      if (threadIdx.x == 0 && n == 1) s_step[k & 1] = 0.0;  // sweep k starts
      // the layer this phase finalises: gathered in the previous phase (not read in this one)
      const int fin_layer = gphase == 0 ? -1 : (n == 1 ? N - 1 : n - 1);
      const P2* ab_prev = (const P2*)(((gphase + 1) & 1) ? a.ab1 : a.ab0);
      P2* ab_cur = (P2*)((gphase & 1) ? a.ab1 : a.ab0);
      const T* p_up = pv + a.off[n + 1];
      float md = 0.f;
      if (fin_layer > 0) finalize(fin_layer, ab_prev, md);
      // -- gather layer n -------------------------------------------------------------------
      T sA = V::zero(), sB = V::zero(), sa = V::zero(), sb = V::zero();
      LayerView<V> lv;
      lv.n = n;
      lv.N = N;
      lv.L = L;
      lv.H = H;
      lv.Sp = a.Sp;
      lv.off_n = a.off[n];
      lv.toff_n = a.toff[n];
      lv.lp = a.lpad[n];
      lv.masks = a.masks;
      lv.lidx = a.lidx;
      lv.RH = a.RH;
      lv.Tt = Tt;
      lv.rt = rt;
      lv.p_up = p_up;
      lv.ab_prev = ab_prev;
      lv.ab_cur = ab_cur;
      lv.nu = s_nu;
      lv.c1 = s_c1;
      lv.c2 = s_c2;
      lv.lamT = s_lamT;
      lv.one = s_one;
      lv.gR = kIR ? a.ir + 3 * a.Sp : nullptr;
      lv.gA = kIR ? a.ir + 4 * a.Sp : nullptr;
      lv.gB = kIR ? a.ir + 5 * a.Sp : nullptr;
      lv.d1 = s_d1;
      lv.d2 = s_d2;
      const int it_end = a.ifirst[n + 1];
      int it = a.ifirst[n] + gwarp;
      uint4 dnext = it < it_end ? __ldg(a.items + it) : make_uint4(0u, 0u, 0u, 0u);
      for (; it < it_end; it += nwarps) {
        const uint4 d = dnext;
        if (it + nwarps < it_end) dnext = __ldg(a.items + it + nwarps);  // next item, ahead
        gather_item<V, kFullL, kIR>(lv, d, s_RL, s_binL, slot_d, slot_u, s_hl[wid], s_hnu[wid], lane, sA,
                                    sB, sa, sb);
        __syncwarp();  // the slot and the lists are rewritten by the next item
      }
      sync_phase(sA, sB, sa, sb, md, n, n >= 2 ? k : k - 1);
    }
  }
  // closing phase: final values of layer N-1 of the last sweep
  if (gphase > 0) {
    const int kl = a.nsweeps - 1;
    float md = 0.f;
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

int g_occ[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
int g_nsm = 0;

template <class V, bool kIR>
const void* persist_fn(bool full) {
  return full ? (const void*)k_persist<V, true, kIR> : (const void*)k_persist<V, false, kIR>;
}

// ir: correction sweeps (FP32 only), against the base set up by hq_ir_begin
template <class V>
int launch_persist(hq_solver* h, int nsweeps, cudaEvent_t ev0, cudaEvent_t ev1, bool ir = false) {
  typedef typename V::T T;
  typedef typename Pair<V>::P P2;
  const int slot = ir ? 3 : (V::kind == HQ_PREC_FP64 ? 0 : (V::kind == HQ_PREC_DF64 ? 1 : 2));
  const size_t smem = (size_t)kWarps * Slot<V>::kBytes;
  const bool full = h->L == HQ_LO_BITS;
  const void* kfn = ir ? persist_fn<PolF32, true>(full) : persist_fn<V, false>(full);
  if (!g_nsm) HQ_CUDA(cudaDeviceGetAttribute(&g_nsm, cudaDevAttrMultiProcessorCount, h->dev));
  if (!g_occ[slot][full]) {
    HQ_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  int occ = 0;
  HQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, kThreads, smem));
  if (occ < 1) {
    hq_set_error("persistent sweep kernel does not fit on an SM");
    return HQ_ECUDA;
  }
  g_occ[slot][full] = occ;
  const int G = g_nsm * occ;
  if ((int64_t)G * (nsweeps * (int64_t)(h->N - 1) + 1) >= ((int64_t)1 << 31)) {
    hq_set_error("too many barrier arrivals for one launch");
    return HQ_EINVAL;
  }
  if ((int64_t)G * kPW * 2 > h->partials_len) {
    hq_set_error("partials buffer too small for the persistent grid");
    return HQ_ECUDA;
  }
  PrecBufs& b = hq_bufs(h, V::kind);
  PersistArgs a;
  memset(&a, 0, sizeof(a));
  a.N = h->N;
  a.L = h->L;
  a.H = h->H;
  a.nsweeps = nsweeps;
  a.lam = h->lam;
  a.omega = h->omega;
  a.Sp = h->Sp;
  for (int i = 0; i < HQ_MAXN + 2; i++) {
    a.off[i] = h->off[i];
    a.toff[i] = h->toff[i];
    a.ifirst[i] = h->ifirst[i];
  }
  for (int n = 0; n <= HQ_MAXN; n++) {
    a.lsize[n] = n <= h->N ? h->lsize[n] : 0;
    a.lpad[n] = n <= h->N ? h->lpad[n] : 0;
  }
  a.items = h->items;
  a.masks = h->masks;
  a.lidx = h->lidx;
  a.RL = h->RL;
  a.RH = h->RH;
  a.T = b.T;
  a.r = b.r;
  a.p = b.p;
  a.nu = b.nu;
  a.ab0 = h->ab;
  a.ab1 = (char*)h->ab + h->ab_half_bytes;
  a.partials = h->partials;
  a.sc = h->sc;
  a.ir = ir ? h->ir : nullptr;
  void* args[] = {&a};
  // a barrier left half-entered by an aborted launch must not leak into this one
  HQ_CUDA(cudaMemsetAsync(&h->sc->bar_count, 0, sizeof(unsigned), h->stream));
  if (ev0) HQ_CUDA(cudaEventRecord(ev0, h->stream));
  HQ_CUDA(cudaLaunchCooperativeKernel(kfn, dim3(G), dim3(kThreads), args, smem, h->stream));
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
  h->it_version++;
  // the barrier's arrival count (grid size x phases of a launch) stays below 2^31
  const int64_t per = ((int64_t)1 << 31) / ((int64_t)152 * 8 * (h->N - 1) + 1) - 1;
  // Layer N-1 of a sweep is finalised lazily in phase 1 of the next sweep of the same
  // launch, whose gather of layer 1 reads layer 2; for N = 3 those are the same layer, so
  // there every launch runs one sweep (its closing phase finalises layer N-1, and a
  // launch's first phase finalises nothing)
  const int cap = h->N == 3 ? 1 : (per > (1 << 20) ? (1 << 20) : (per < 1 ? 1 : (int)per));
  for (int done = 0; done < nsweeps;) {
    const int k = nsweeps - done < cap ? nsweeps - done : cap;
    cudaEvent_t e0 = done == 0 ? ev0 : nullptr, e1 = done + k == nsweeps ? ev1 : nullptr;
    int rc;
    if (prec == HQ_PREC_FP64) rc = launch_persist<PolF64>(h, k, e0, e1);
    else if (prec == HQ_PREC_DF64) rc = launch_persist<PolDF>(h, k, e0, e1);
    else if (prec == HQ_PREC_IRC) rc = launch_persist<PolF32>(h, k, e0, e1, true);
    else rc = launch_persist<PolF32>(h, k, e0, e1);
    if (rc != HQ_OK) return rc;
    done += k;
  }
  return HQ_OK;
}

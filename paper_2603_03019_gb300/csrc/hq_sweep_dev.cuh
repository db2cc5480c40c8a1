// Device code shared by the sweep kernels (one instance: hq_persist.cu; a batch of
// instances: hq_batch.cu): memory-model and copy helpers, (A, B) pair types, and the
// gather of one work item (up to 32 states of one rank block of layer n; the item format
// and the rank-block layout are described with HQ_ITEM_HI_BITS in hq_internal.cuh).
#pragma once

#include "hq_internal.cuh"

namespace hqdev {

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// barrier arrival (acquire + release at gpu scope), release of the barrier, acquire fence
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
  unsigned r;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "r"(v) : "memory");
  return r;
}
__device__ __forceinline__ void red_add_release(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
// 16-byte asynchronous global -> shared copy through L2 only (it sees other CTAs' writes
// made before the grid barrier), and the wait for all of this thread's such copies
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// polling load: coherent at gpu scope without the acquire's L1 invalidation, so spinning
// CTAs do not evict the cached data of CTAs still working on the SM
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// ---- loads of values other CTAs wrote in this launch: from L2 (.cg); the table streams
// through once per sweep (ld_stream, hq_internal.cuh)
__device__ __forceinline__ double ld_l2(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float2 ld_l2(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ float ld_l2(const float* p) { return __ldcg(p); }
__device__ __forceinline__ double2 ld_l2(const double2* p) { return __ldcg(p); }
__device__ __forceinline__ float4 ld_l2(const float4* p) { return __ldcg(p); }

// (A, B) pair storage per precision
template <class V> struct Pair;
template <> struct Pair<PolF64> {
  typedef double2 P;
  __device__ static P pack(double a, double b) { return make_double2(a, b); }
  __device__ static double A(P p) { return p.x; }
  __device__ static double B(P p) { return p.y; }
};
template <> struct Pair<PolDF> {
  typedef float4 P;
  __device__ static P pack(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }
  __device__ static float2 A(P p) { return make_float2(p.x, p.y); }
  __device__ static float2 B(P p) { return make_float2(p.z, p.w); }
};
template <> struct Pair<PolF32> {
  typedef float2 P;
  __device__ static P pack(float a, float b) { return make_float2(a, b); }
  __device__ static float A(P p) { return p.x; }
  __device__ static float B(P p) { return p.y; }
};

template <class V>
__device__ __forceinline__ typename V::T warp_sum(typename V::T v) {
  for (int m = 16; m > 0; m >>= 1) v = V::add(v, V::shfl_xor(v, m));
  return v;
}

// position of the k-th low-part neighbour of a state in its staged block (lidx bytes)
__device__ __forceinline__ int lo_pos(uint32_t w0, uint32_t w1, uint32_t w2, int k) {
  const uint32_t wd = k < 4 ? w0 : (k < 8 ? w1 : w2);
  return (int)((wd >> (8 * (k & 3))) & 0xffu);
}

// shared-memory slot of one warp: the staged (A, B) block of layer n-1, then the staged p
// block of layer n+1, each with 16 bytes of room for the copy's alignment offset
template <class V> struct Slot {
  typedef typename V::T T;
  typedef typename Pair<V>::P P2;
  static constexpr int kD = HQ_MAX_BLOCK * (int)sizeof(P2) + 16;
  static constexpr int kU = HQ_MAX_BLOCK * (int)sizeof(T) + 16;
  static constexpr int kBytes = kD + kU;
};

// one layer of one instance, as seen by the gather of layer n
template <class V> struct LayerView {
  typedef typename V::T T;
  typedef typename Pair<V>::P P2;
  int n, N, L, H;
  int64_t Sp;       // padded state count (row stride of lidx)
  int64_t off_n;    // first state of layer n in the layer-ranked vectors
  int64_t toff_n;   // first table entry of layer n
  int64_t lp;       // distance between a state's consecutive table slots (1: state-major)
  int64_t tw;       // table record width of layer n
  const uint32_t* masks;
  const uint32_t* lidx;
  const uint32_t* RH;
  const T* Tt;      // pull-form table
  const T* rt;      // r_m
  const T* p_up;    // p of layer n+1
  const P2* ab_prev;  // (A, B) pairs of layer n-1
  P2* ab_cur;         // (A, B) pairs of layer n (written)
  const T* nu;        // nu_i in this precision
  T c1, c2;           // p_{n-1} = c1 A + c2 B
  T lamT, one;
  // correction sweeps (refinement): the pull gathers of the base terms of layer n-1
  // (G_rho, G_A, G_B at off_n + rank) and d1 = c1 - c1^0, d2 = c2 - c2^0 of layer n-1
  const float* gR;
  const float* gA;
  const float* gB;
  T d1, d2;
};

// Gather one item of layer n (Eq. 12): A_m = r_m sum_s p_{n-1}(m - c_s) T[m][s] with
// p_{n-1} = c1 A + c2 B of the previous layer, B_m = r_m sum_{u idle} p_{n+1}(m + u) nu_u,
// written as (A, B) pairs; adds the item's sum mu_m A_m to sA, sum mu_m B_m to sB, sum A_m
// to sa and sum B_m to sb (mu_m r_m = 1 - lambda r_m).
//
// The sums run in a fixed order whatever the layout of the loops: busy neighbours in
// table-slot order (increasing unit), idle neighbours in increasing unit order.  Low part:
// one step per lidx byte k < L (compile-time k, so the byte and the table row are
// immediates; k < w busy from the staged block of layer n-1, else idle from the staged
// block of layer n+1).  High part: counted loops over the warp's list `hl` of neighbour
// block bases (the item's busy units first, then its idle units, each increasing) with
// the idle units' rates in `hnu`; every lane reads the same entry.  kFullL: L equals
// HQ_LO_BITS (every instance with N >= HQ_LO_BITS).  kIR (FP32 only): the pairs and p
// are the corrections a, b, e against a fixed base, and the pull term gains the base's
// part G_rho + d1 G_A + d2 G_B (layer 1 pulls nothing: the empty state has no
// correction).  The caller syncs the warp before the slot and the lists are rewritten
// by the next item.
template <class V, bool kFullL, bool kIR = false>
__device__ __forceinline__ void gather_item(const LayerView<V>& lv, const uint4 d, const uint32_t* s_RL,
                                            const int* s_binL, unsigned char* slot_d,
                                            unsigned char* slot_u, uint32_t* hl, typename V::T* hnu,
                                            int lane, typename V::T& sA, typename V::T& sB,
                                            typename V::T& sa, typename V::T& sb) {
  typedef typename V::T T;
  typedef Pair<V> PR;
  typedef typename PR::P P2;
  const int n = lv.n, L = kFullL ? HQ_LO_BITS : lv.L, H = lv.H;
  const uint32_t lmask = (1u << L) - 1u;
  const uint32_t rank0 = d.x;
  const uint32_t hi = d.y & ((1u << HQ_ITEM_HI_BITS) - 1u);
  const int w = (int)((d.y >> HQ_ITEM_HI_BITS) & 0xfu);
  const int count = (int)((d.y >> 24) & 0x1fu) + 1;
  const bool pull = n > 1;  // layer 1 pulls from the empty state, whose p_0 = 1
  const int nbh = n - w, nih = H - nbh;
  // the high-part neighbour lists: lane j < H owns unit L + j, whose block base is
  // RH[hi ^ 2^j][w] in layer n -/+ 1
  if (lane < H) {
    const uint32_t hb = __ldg(lv.RH + (size_t)(hi ^ (1u << lane)) * (L + 1) + w);
    const uint32_t below = hi & ((1u << lane) - 1u);
    if ((hi >> lane) & 1u) {
      hl[__popc(below)] = hb;
    } else {
      const int k = lane - __popc(below);
      hl[nbh + k] = hb;
      hnu[k] = lv.nu[L + lane];
    }
  }
  // this lane's state (lanes past the item repeat its first state and discard it)
  const bool act = lane < count;
  const uint32_t kq = rank0 + (act ? (uint32_t)lane : 0u);
  const int64_t gi = lv.off_n + kq;
  const uint32_t x = __ldg(lv.masks + gi);
  const uint32_t iw0 = __ldg(lv.lidx + gi), iw1 = __ldg(lv.lidx + lv.Sp + gi),
                 iw2 = __ldg(lv.lidx + 2 * lv.Sp + gi);
  const T rv = __ldg(lv.rt + gi);
  T g0 = V::zero(), g1 = V::zero(), g2 = V::zero();
  if constexpr (kIR) {
    if (pull) {
      g0 = ld_stream(lv.gR + gi);
      g1 = ld_stream(lv.gA + gi);
      g2 = ld_stream(lv.gB + gi);
    }
  }
  const T* tcol = lv.Tt + lv.toff_n + (int64_t)kq * lv.tw;  // table slot s at tcol[s * lp]
  const int64_t lp = lv.lp;
  // table entries of the low-part busy neighbours, issued before the staging wait
  T tlo[HQ_LO_BITS];
#pragma unroll
  for (int k = 0; k < HQ_LO_BITS; k++) tlo[k] = (k < w && pull) ? ld_stream(tcol + k * lp) : V::zero();
  // stage the low-part neighbour blocks in this warp's slot with 16-byte asynchronous
  // copies: a block's copy starts at the 16-byte boundary at or below its first
  // element (offset `dd` / `du` elements into the slot) and covers whole 16-byte units
  const P2* sdn;
  const T* sup;
  {
    const int dc = (pull && w > 0) ? s_binL[w] : 0;
    const int uc = w < L ? s_binL[w + 2] : 0;
    const unsigned char* gd = (const unsigned char*)(lv.ab_prev + d.z);
    const unsigned char* gu = (const unsigned char*)(lv.p_up + d.w);
    const int od = (int)((uintptr_t)gd & 15u), ou = (int)((uintptr_t)gu & 15u);
    const int cd = dc ? (od + dc * (int)sizeof(P2) + 15) >> 4 : 0;
    const int cu = uc ? (ou + uc * (int)sizeof(T) + 15) >> 4 : 0;
    for (int c = lane; c < cd; c += 32) cp_async16(slot_d + 16 * c, gd - od + 16 * c);
    for (int c = lane; c < cu; c += 32) cp_async16(slot_u + 16 * c, gu - ou + 16 * c);
    cp_async_wait_all();
    sdn = (const P2*)(slot_d + od);
    sup = (const T*)(slot_u + ou);
  }
  const uint32_t lo = x & lmask;
  const uint32_t rl = s_RL[lo];
  __syncwarp();  // staged blocks and lists visible to the whole warp
  T UA = V::zero(), UB = V::zero(), D = V::zero();
  // low part: lidx byte k is the k-th busy unit's neighbour for k < w, else the
  // (k - w)-th idle unit's (the idle units are the set bits of `z`, taken in order)
  {
    uint32_t z = ~lo & lmask;
#pragma unroll
    for (int k = 0; k < HQ_LO_BITS; k++) {
      if (kFullL || k < L) {
        const uint32_t wd = k < 4 ? iw0 : (k < 8 ? iw1 : iw2);
        const int pos = (int)((wd >> (8 * (k & 3))) & 0xffu);
        if (k < w) {
          if (pull) {
            const P2 q = sdn[pos];
            V::fma_acc(UA, PR::A(q), tlo[k]);
            V::fma_acc(UB, PR::B(q), tlo[k]);
          }
        } else {
          const int u = __ffs(z) - 1;
          z &= z - 1u;
          V::fma_acc(D, sup[pos], lv.nu[u]);
        }
      }
    }
  }
  // high part, busy: table slots w .. n-1
  if (pull) {
    const T* tp = tcol + w * lp;
#pragma unroll 4
    for (int k = 0; k < nbh; k++) {
      const T t = ld_stream(tp + k * lp);
      const P2 q = ld_l2(lv.ab_prev + hl[k] + rl);
      V::fma_acc(UA, PR::A(q), t);
      V::fma_acc(UB, PR::B(q), t);
    }
  }
  // high part, idle
#pragma unroll 4
  for (int k = 0; k < nih; k++) V::fma_acc(D, ld_l2(lv.p_up + hl[nbh + k] + rl), hnu[k]);
  // up-inflow: layer 0 is the empty state with p_0 = 1
  T U;
  if constexpr (kIR) {
    U = pull ? V::add(V::add(g0, V::add(V::mul(lv.d1, g1), V::mul(lv.d2, g2))),
                      V::add(V::mul(lv.c1, UA), V::mul(lv.c2, UB)))
             : V::zero();
  } else {
    U = pull ? V::add(V::mul(lv.c1, V::norm(UA)), V::mul(lv.c2, V::norm(UB))) : ld_stream(tcol);
  }
  D = V::norm(D);
  const T qm = V::sub(lv.one, V::mul(lv.lamT, rv));  // mu_m r_m = 1 - lambda r_m
  const T A = V::mul(U, rv), B = V::mul(D, rv);
  if (act) {
    lv.ab_cur[kq] = PR::pack(A, B);
    sA = V::add(sA, V::mul(U, qm));
    sB = V::add(sB, V::mul(D, qm));
    sa = V::add(sa, A);
    sb = V::add(sb, B);
  }
}

}  // namespace hqdev

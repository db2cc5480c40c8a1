// Outer iterations k of Algorithm 1 (Eq. 12-14) on the layer-ranked layout, as one
// persistent cooperative kernel per batch of sweeps.
//
// The update of layer n.  For each state m of layer n, Eq. (12) reads
//     p_n^{k,r}(m) = alpha mu^{k,r-1}(n) A_m + beta B_m
// with  alpha = 1/lambda^k(n-1),  beta = lambda^{k-1}(n) / mu^{k-1}(n+1),
//       A_m = r_m U_m,  U_m = sum_{l in C_{n-1}} p_{n-1}(l) lambda_{lm},
//       B_m = r_m D_m,  D_m = sum_{u idle in m} p_{n+1}(m+u) nu_u,   r_m = 1/(lambda_m+mu_m).
// Only mu^{k,r-1}(n) depends on r, and Eq. (14) makes it an affine recursion
// mu^{k,r} = a mu^{k,r-1} + b with a = alpha sum_m mu_m A_m in (0,1) and
// b = beta sum_m mu_m B_m, so the inner loop of Algorithm 1 converges to mu* = b/(1-a)
// and p_n^k(m) = c1 A_m + c2 B_m with c1 = alpha mu*, c2 = beta (its delta -> 0 limit).
//
// The scalars of layer n come from its neighbour layers, before its gather.  The sums
// over layer n that the closed form needs are sums over layers n-1 and n+1 with
// per-state weights that depend on the instance only:
//     sum_m mu_m A_m = sum_{l in C_{n-1}} p(l) w''(l),   w''(l) = sum_{u idle in l} lambda_u(l) mu_{l+u} r_{l+u},
//     sum_m mu_m B_m = sum_{l in C_{n+1}} p(l) v''(l),   v''(l) = sum_{u busy in l} nu_u mu_{l-u} r_{l-u},
// and lambda(n-1) = lambda sum p_{n-1} (Eq. 13), mu(n+1) = sum mu_l p_{n+1}(l) (Eq. 14).
// So every layer carries four sums {sum p, sum mu p, sum w'' p, sum v'' p}; the phase
// that writes a layer also adds up its four sums, and the grid barrier that ends the
// phase folds them, after which every CTA solves the closed form of the layers of the
// next phase.  The gather then writes the final p_n directly: no (A, B) pairs are
// stored and no layer is finalised later.
//
// Sweep orders.  HQ_ORDER_ASCENDING is Algorithm 1 as printed: layers 1..N-1 in turn,
// Gauss-Seidel from layer n-1, Jacobi from layer n+1 (the two properties stated for
// Algorithm 2), one phase and one grid barrier per layer.  HQ_ORDER_REDBLACK (not in the
// paper) updates all odd layers from the even ones, then all even layers from the odd
// ones: two phases per sweep.  Both are block Gauss-Seidel iterations of the same
// fixed-point equations, so they share the fixed point (the exact stationary
// distribution); layer coupling is block tridiagonal, and for such couplings any
// ordering that updates each layer after one of its neighbours and before the other
// ("consistent" orderings) has the same asymptotic rate.
//
// Work.  The pull-form table is state-major: a state's n upward rates form one record,
// padded to a multiple of four entries, which a lane loads as 16-byte vectors.  A phase's
// rank blocks (the states of one layer sharing their high part, see HQ_SW_HI_BITS) are
// sorted by cost and dealt to the warps of the grid in snake order, which evens out the
// warps' totals; a block's items (runs of at most 32 consecutive states) go to one warp,
// one lane per state.  A warp fetches the metadata of its next 32 blocks at once, one
// lane per block (first item, descriptor, and the block's rank-table entries into a
// per-warp shared buffer).  Per block, the warp takes its neighbour block bases from
// that buffer (lane j: the block across high unit j; lanes 29..31: its own block and the
// blocks (hi, w -/+ 1)), lists its high-part neighbour runs in shared memory, and
// copies the two blocks that hold its states' low-part neighbours -- (hi, w-1) of layer
// n-1 and (hi, w+1) of layer n+1, at most 252 states each -- into its shared-memory slot
// with 16-byte asynchronous copies.  Per item, every lane issues all its loads at once before it
// waits: its table record, its high-part neighbours (consecutive states have them at
// consecutive ranks, so these are coalesced runs), r_m, its old value and its two weights.
// Low-part neighbour positions and idle units come from a shared table per low part, so
// no index is read from memory.  The inflow sums are unrolled per low-part weight w, so
// every register index is a constant; busy neighbours go by table slot (increasing
// unit), idle neighbours by unit, the low and the high part as two chains added at the end.
//
// Correction sweeps (iterative refinement against an FP64 base p0, FP32): the iterate is
// e = p - p0, the gathers read e, and the update is
//     e_n(m) = rho0_m + d1 A0_m + d2 B0_m + c1 a_m + c2 b_m
// (a, b: the gathers of e; A0, B0, rho0 = c1^0 A0 + c2^0 B0 - p0: per-state base terms in
// FP32; d = c - c^0), with the layer sums of p0 + e made of the base's (FP64) and the
// correction's.
//
// Every grid barrier's wait is bounded: one that does not complete within its
// iteration limit sets an error bit in DevScalars::flags and the kernel runs to its end
// with in-bounds indices; the host reports HQ_ETIMEOUT.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "hq_sweep_dev.cuh"

namespace {

using namespace hqdev;

constexpr int kMaxPL = HQ_MAXN / 2;        // layers in one phase, at most (red-black, N <= 29)
constexpr int kMaxWords = 4 * kMaxPL + 1;  // partial words per CTA per phase
constexpr unsigned kSpinDefault = 1u << 24;
constexpr unsigned kFull = 0xffffffffu;

// per-state weights (w'', v'') as stored, and as the policy's type
template <class V> struct WT {
  typedef double2 W;
  __device__ static double x(W w) { return w.x; }
  __device__ static double y(W w) { return w.y; }
};
template <> struct WT<PolF32> {
  typedef float2 W;
  __device__ static float x(W w) { return w.x; }
  __device__ static float y(W w) { return w.y; }
};
template <> struct WT<PolDF> {
  typedef double2 W;
  __device__ static float2 x(W w) { return df_from_double(w.x); }
  __device__ static float2 y(W w) { return df_from_double(w.y); }
};

// per warp: two block parities x (staged block of layer n-1, staged block of layer n+1),
// each with 16 bytes of room for the copy's alignment offset; then the rank-table entries
// of the warp's next 32 blocks (kHP + 3 per block, see run_items)
template <class V>
constexpr int kStageBytes() {
  return 4 * (HQ_MAX_BLOCK * (int)sizeof(typename V::T) + 16);
}
template <class V, int kHP>
constexpr int kSlotBytes() {
  return kStageBytes<V>() + 32 * (kHP + 3) * 4;
}
template <class V>
int slot_bytes(int H) {
  return H <= 14 ? kSlotBytes<V, 14>() : (H <= 18 ? kSlotBytes<V, 18>() : kSlotBytes<V, 20>());
}

struct SweepArgs {
  int N, L, H, nsweeps, order, nphases;
  double lam;
  double omega;                // over-relaxation of the updated layers (1: none)
  int64_t Sp;
  int64_t off[HQ_MAXN + 2];    // padded per-state offsets of the layers
  int64_t toff[HQ_MAXN + 2];   // padded table offsets of the layers
  int64_t tw[HQ_MAXN + 2];     // table record width of layer n
  int pbfirst[HQ_MAXN + 2];    // rank blocks of phase ph: [pbfirst[ph], pbfirst[ph+1])
  const uint2* items;
  const int* blocks;           // first item of each rank block (and the end)
  const int* perm;             // per phase, its blocks by decreasing cost
  const uint32_t* RL;
  const uint32_t* RH;
  const void* T;
  const void* r;
  const void* wv;              // per-state weights (w'', v'')
  const void* nu;
  void* p;
  double* partials;            // [2][kMaxWords][G]
  DevScalars* sc;
  const float* ir;             // correction sweeps: 3 x Sp base terms {rho0, A0, B0}
  float* out;                  // base pass: 3 x Sp {rho0, A0, B0} written (FP32)
  unsigned spin_limit;
  int dbg_skip_cta;            // fault injection: this CTA skips its first barrier arrival
};

// first layer and number of layers of phase ph (red-black: every other layer from f)
__device__ __forceinline__ void phase_layers(int order, int ph, int N, int& f, int& nl) {
  f = ph + 1;
  nl = order == HQ_ORDER_ASCENDING ? 1 : (N - 1 - f) / 2 + 1;
}

// shared tables of one CTA: the low-part tables and per-layer offsets
template <class V, int kWarps, int kHP>
struct Smem {
  typedef typename V::T T;
  uint32_t RL[1 << HQ_LO_BITS];
  uint16_t LO[1 << HQ_LO_BITS];     // low parts in colex order, by weight: LO[woff[w] + rank]
  // per low part (same index as LO), 16 bytes: byte k < w = position RL[lo ^ 2^u] of the
  // k-th busy unit u's neighbour in block (hi, w-1); byte k >= w = position RL[lo | 2^u]
  // of the (k-w)-th idle unit u's neighbour in block (hi, w+1); nibble k at bit 80 + 4k
  // = that idle unit u
  uint4 LX[1 << HQ_LO_BITS];
  T MUlo[1 << HQ_LO_BITS];          // sum of nu over the busy units of lo
  int woff[HQ_LO_BITS + 2];         // woff[w + 1] - woff[w] = C(L, w)
  T nu[HQ_MAXN];
  int64_t off[HQ_MAXN + 2], toff[HQ_MAXN + 2], tw[HQ_MAXN + 2];
  // per warp and block parity (a warp holds the rank block of its current item and of
  // its next one): the high-part neighbour runs (busy units in increasing order, then idle
  // units), and the idle units' rates at the same index
  const T* hptr[kWarps][2][kHP];
  T hnu[kWarps][2][kHP];
  double ws[kWarps][kMaxPL][4];     // per warp: layer sums of this phase
  float wmd[kWarps];
  double fold[kMaxWords];
  double LS[4][HQ_MAXN + 1];        // layer sums of the iterate (corrections: p0 + e)
  double IB[4][HQ_MAXN + 1];        // corrections: the base's layer sums
  double I1[HQ_MAXN + 1], I2[HQ_MAXN + 1];  // corrections: c1^0, c2^0
  T c1[HQ_MAXN + 1], c2[HQ_MAXN + 1], d1[HQ_MAXN + 1], d2[HQ_MAXN + 1];
  double step[2];
  double fac[HQ_MAXN + 1];          // residual: P{B} = fac[w(B)] p(B)
};

template <class V, int kWarps, int kHP>
__device__ void setup_tables(Smem<V, kWarps, kHP>& s, const SweepArgs& a) {
  typedef typename V::T T;
  const int L = a.L, N = a.N;
  for (int i = threadIdx.x; i < (1 << L); i += blockDim.x) s.RL[i] = a.RL[i];
  if ((int)threadIdx.x < N) s.nu[threadIdx.x] = ((const T*)a.nu)[threadIdx.x];
  for (int i = threadIdx.x; i < HQ_MAXN + 2; i += blockDim.x) {
    s.off[i] = a.off[i];
    s.toff[i] = a.toff[i];
    s.tw[i] = a.tw[i];
  }
  if (threadIdx.x == 0) {
    s.woff[0] = 0;
    for (int w = 0; w <= L; w++) {
      double c = 1.0;  // C(L, w), exact for L <= 10
      for (int q = 1; q <= w; q++) c = c * (double)(L - w + q) / (double)q;
      s.woff[w + 1] = s.woff[w] + (int)(c + 0.5);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < (1 << L); i += blockDim.x) {
    const uint32_t lo = (uint32_t)i;
    const int e = s.woff[__popc(lo)] + (int)s.RL[lo];
    s.LO[e] = (uint16_t)lo;
    uint32_t wd[4] = {0u, 0u, 0u, 0u};
    int k = 0;
    for (int u = 0; u < L; u++)
      if ((lo >> u) & 1u) {
        wd[k >> 2] |= (s.RL[lo ^ (1u << u)] & 0xffu) << (8 * (k & 3));
        k++;
      }
    for (int u = 0; u < L; u++)
      if (!((lo >> u) & 1u)) {
        wd[k >> 2] |= (s.RL[lo | (1u << u)] & 0xffu) << (8 * (k & 3));
        const int bit = 80 + 4 * k;
        wd[bit >> 5] |= (uint32_t)u << (bit & 31);
        k++;
      }
    s.LX[e] = make_uint4(wd[0], wd[1], wd[2], wd[3]);
    T mu = V::zero();
    for (uint32_t y = lo; y; y &= y - 1u) mu = V::add(mu, s.nu[__ffs(y) - 1]);
    s.MUlo[lo] = mu;
  }
}

__device__ __forceinline__ uint32_t lx_word(const uint4& x, int i) {
  return i == 0 ? x.x : (i == 1 ? x.y : (i == 2 ? x.z : x.w));
}

// A state's table record as loaded: vectors of kPer entries (16 bytes), and entry s of it
// (s a constant once the caller's loop is unrolled)
template <class V> struct Vec;
template <> struct Vec<PolF32> {
  typedef float4 VT;
  static constexpr int kPer = 4;
  __device__ static float get(const float4* v, int s) {
    const float4 x = v[s >> 2];
    const int c = s & 3;
    return c == 0 ? x.x : (c == 1 ? x.y : (c == 2 ? x.z : x.w));
  }
};
template <> struct Vec<PolF64> {
  typedef double2 VT;
  static constexpr int kPer = 2;
  __device__ static double get(const double2* v, int s) { return (s & 1) ? v[s >> 1].y : v[s >> 1].x; }
};
template <> struct Vec<PolDF> {
  typedef float4 VT;
  static constexpr int kPer = 2;
  __device__ static float2 get(const float4* v, int s) {
    return (s & 1) ? make_float2(v[s >> 1].z, v[s >> 1].w) : make_float2(v[s >> 1].x, v[s >> 1].y);
  }
};
__device__ __forceinline__ float4 ld_vec(const float4* p) { return __ldcs(p); }
__device__ __forceinline__ double2 ld_vec(const double2* p) { return __ldcs(p); }

// Eq. (12)'s two inflow sums of one state whose low part has W busy units: busy
// neighbours by table slot (low units, then high units: slot W + j), idle neighbours by
// unit (low, then high).  tv: the state's table record; h: its high-part neighbours (busy
// units first, as the warp's list); lx: its low-part positions and idle units.
// FP32 and DF64: the low- and high-part sums run as separate chains (then low + high),
// which halves the dependent FMA chain of a state.  FP64, whose sweep is bound by the
// FP64 pipe on this chip, keeps one chain per sum (two adds fewer per state).  Inside
// each part the order is by slot / by unit.
template <int W, class V, int kHP, int kNV>
__device__ __forceinline__ void inflows(typename V::T& U, typename V::T& D, const typename Vec<V>::VT* tv,
                                        const typename V::T* h, const uint4& lx, const typename V::T* sdn,
                                        const typename V::T* sup, int nbh, int H, int L,
                                        const typename V::T* nu, const typename V::T* hnu) {
  typedef typename V::T T;
  constexpr int kMaxSlot = kNV * Vec<V>::kPer;
  constexpr bool kOne = V::kind == HQ_PREC_FP64;
  T Ul = V::zero(), Uh0 = V::zero(), Dl = V::zero(), Dh0 = V::zero();
  T& Uh = kOne ? Ul : Uh0;
  T& Dh = kOne ? Dl : Dh0;
#pragma unroll
  for (int k = 0; k < W; k++) {
    const uint32_t pos = (lx_word(lx, k >> 2) >> (8 * (k & 3))) & 0xffu;
    V::fma_acc(Ul, sdn[pos], Vec<V>::get(tv, k));
  }
#pragma unroll
  for (int j = 0; j < kHP; j++) {
    if (j >= nbh) break;
    if (W + j < kMaxSlot) V::fma_acc(Uh, h[j], Vec<V>::get(tv, W + j));
  }
#pragma unroll
  for (int k = W; k < HQ_LO_BITS; k++) {
    if (k >= L) break;
    const uint32_t pos = (lx_word(lx, k >> 2) >> (8 * (k & 3))) & 0xffu;
    const uint32_t u = (lx_word(lx, (80 + 4 * k) >> 5) >> ((80 + 4 * k) & 31)) & 0xfu;
    V::fma_acc(Dl, sup[pos], nu[u]);
  }
#pragma unroll
  for (int j = 0; j < kHP; j++) {
    if (j >= H) break;
    if (j < nbh) continue;
    V::fma_acc(Dh, h[j], hnu[j]);
  }
  if constexpr (kOne) {
    U = Ul;
    D = Dl;
  } else {
    U = V::add(V::norm(Ul), V::norm(Uh));
    D = V::add(V::norm(Dl), V::norm(Dh));
  }
}

// One item's loads, held in registers from issue to compute.
template <class V, int kNV, int kHP>
struct ItemLoads {
  typename Vec<V>::VT tv[kNV];  // the states' table records
  typename V::T h[kHP];         // high-part neighbours (the block's list order)
  typename V::T rv, po, q0, q1, q2;
  typename WT<V>::W wv;
};
// A rank block as a warp holds it: its id bits, layer, base rank and high-part rates.
template <class V>
struct BlockCtx {
  uint32_t hi, hself;
  int w, n, nbh, par, grp;  // par: list/slot parity; grp: its cp.async group number
  int it0, size;            // the block's first item and its number of states
  int od, ou;               // byte offsets of the staged blocks' first elements
  typename V::T mu_hi;
};
struct ItemRef {
  uint32_t rk;  // this lane's state rank in layer n
  int cnt, bq;  // states in the item; the parity of its block's lists and staged blocks
};

// Process the rank blocks [b0, b1) of a phase whose layers start at f (li = (n - f) >>
// order).  The phase's blocks come by decreasing cost (a.perm) and go to the warps in
// snake order: round r gives block r W + g (r even) or r W + W - 1 - g (r odd) to warp g,
// so the warps' totals even out.  The metadata of 32 rounds (each block's first item,
// descriptor and rank-table entries) is fetched at once, one block per lane.  A warp
// walks its blocks' items in order: per item it issues every load (table record,
// high-part neighbours, r, the old value, the weights) and then computes; the
// high-part neighbours must be loaded with the rest (loading them inside the gather was
// measured 1.5x slower).  A block's neighbour lists and staged low-part blocks alternate
// between two parities.  One lane per state of an item.
// kMode 0: a sweep (write p, add the layer sums into s.ws);  kMode 1: a correction
// sweep (the iterate is e, base terms from a.ir);  kMode 2: the base pass of the
// refinement (read p = p0, write rho0, A0, B0 to a.out with the scalars c^0 in s.c1/c2;
// no sums, no update);  kMode 3: the global-balance residual of Eq. (1) (read p, FP64;
// md and rmax receive max_m |out_m - in_m| and max_m out_m).  md receives the step max
// |p_new - p_old| in modes 0 and 1.
// Every per-neighbour loop is unrolled with compile-time indices (registers) and leaves
// at a warp-uniform bound, so only the neighbours that exist issue instructions.
template <class V, int kMode, int kHP, int kWarps>
__device__ __forceinline__ void run_items(Smem<V, kWarps, kHP>& s, const SweepArgs& a, int b0, int b1, int f,
                                          unsigned char* slot, int kSlot, float& md, double* rmax = nullptr) {
  typedef typename V::T T;
  typedef WT<V> WX;
  typedef typename WX::W W;
  typedef typename Vec<V>::VT VT;
  constexpr int kNV = (kHP + HQ_LO_BITS + Vec<V>::kPer - 1) / Vec<V>::kPer;  // record vectors, at most
  constexpr int kHalf = HQ_MAX_BLOCK * (int)sizeof(T) + 16;                // one staged block
  const int L = a.L, H = a.H, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const T* pv = (const T*)a.p;
  T* pw = (T*)a.p;
  const bool relax = kMode != 2 && a.omega != 1.0;
  const T om = V::from_d(a.omega);
  (void)kSlot;
  int cur_n = -1, li = 0;
  T aS = V::zero(), aM = V::zero(), aW = V::zero(), aV = V::zero();
  auto flush = [&]() {
    if (kMode == 2) return;
    T v[4] = {aS, aM, aW, aV};
#pragma unroll
    for (int q = 0; q < 4; q++) {
      T x = V::norm(v[q]);
      for (int m = 16; m > 0; m >>= 1) x = V::add(x, V::shfl_xor(x, m));
      if (lane == 0) s.ws[wid][li][q] += V::to_d(x);
    }
  };
  const int gwarp = (int)blockIdx.x * kWarps + wid, nwarps = (int)gridDim.x * kWarps;
  const int nb = b1 - b0;
  // the warp's item sequence: its blocks in snake order, each block's items in order
  int sr = 0, sit = 0, sie = 0;  // round, next item, end of the current block
  // Block metadata of the warp's rounds [mbase, mbase + 32), one round per lane, fetched
  // together: the warp pays one chain of dependent loads (perm, first item, its
  // descriptor) per 32 blocks instead of one per block.  m_id = hi | w << 20 | n << 24 of
  // the lane's block (~0u: none), m_it0 its first item.
  // The lane also loads its block's rank-table entries into the warp's buffer rhb
  // (kRHB words per block: the high-part neighbour blocks RH[hi ^ 2^j][w], j < H, then
  // the block's own rank and those of (hi, w - 1), (hi, w + 1)), all in flight at once.
  constexpr int kRHB = kHP + 3;
  uint32_t* rhb = (uint32_t*)(slot + kStageBytes<V>());
  int mbase = -32, m_it0 = 0;
  uint32_t m_id = ~0u;
  auto fetch_meta = [&](int r0) {
    mbase = r0;
    const int r = r0 + lane;
    const int k = r * nwarps + ((r & 1) ? nwarps - 1 - gwarp : gwarp);
    m_id = ~0u;
    __syncwarp();  // every lane is done with the previous batch's entries
    if (k < nb) {
      m_it0 = __ldg(a.blocks + __ldg(a.perm + b0 + k));
      const uint2 d0 = __ldg(a.items + m_it0);
      m_id = (d0.x & ((1u << (HQ_SW_HI_BITS + 4)) - 1u)) | ((d0.y >> 27) << (HQ_SW_HI_BITS + 4));
      const uint32_t hi = m_id & ((1u << HQ_SW_HI_BITS) - 1u);
      const int w = (int)((m_id >> HQ_SW_HI_BITS) & 0xfu);
      uint32_t* rb = rhb + lane * kRHB;
      const uint32_t* rh = a.RH + w;
#pragma unroll
      for (int j = 0; j < kHP; j++)
        if (j < H) rb[j] = __ldg(rh + (hi ^ (1u << j)) * (uint32_t)(L + 1));
      rb[kHP] = __ldg(rh + hi * (uint32_t)(L + 1));
      rb[kHP + 1] = w >= 1 ? __ldg(rh + hi * (uint32_t)(L + 1) - 1) : 0u;
      rb[kHP + 2] = w < L ? __ldg(rh + hi * (uint32_t)(L + 1) + 1) : 0u;
    }
    __syncwarp();
  };
  BlockCtx<V> bc;  // the block being worked (its lists and staged blocks alternate parity)
  int ngrp = 0;        // cp.async groups committed so far
  int last_par = 1;    // parity of the most recently set-up block
  // set up the block with metadata id (first item it0, rank entries at rhb[src]) in the
  // next parity
  auto setup = [&](uint32_t id, int it0, int src) -> int {
    const int par = last_par ^ 1;
    last_par = par;
    BlockCtx<V> c;
    c.hi = id & ((1u << HQ_SW_HI_BITS) - 1u);
    c.w = (int)((id >> HQ_SW_HI_BITS) & 0xfu);
    c.n = (int)(id >> (HQ_SW_HI_BITS + 4));
    c.par = par;
    const uint32_t hi = c.hi;
    const int w = c.w, n = c.n;
    const T* p_dn = pv + s.off[n - 1];
    const T* p_up = pv + s.off[n + 1];
    __syncwarp();  // every lane is done with this parity's previous block
    const uint32_t* rb = rhb + src * kRHB;
    uint32_t rh = 0u;
    if (lane < H) rh = rb[lane];
    else if (lane == 29) rh = rb[kHP];
    else if (lane == 30) rh = rb[kHP + 1];
    else if (lane == 31) rh = rb[kHP + 2];
    c.nbh = __popc(hi);
    T muj = V::zero();
    if (lane < H) {
      const int before = __popc(hi & ((1u << lane) - 1u));
      if ((hi >> lane) & 1u) {
        s.hptr[wid][par][before] = p_dn + rh;
        muj = s.nu[L + lane];
      } else {
        const int at = c.nbh + lane - before;
        s.hptr[wid][par][at] = p_up + rh;
        s.hnu[wid][par][at] = s.nu[L + lane];
      }
    }
    for (int m = 16; m > 0; m >>= 1) muj = V::add(muj, V::shfl_xor(muj, m));
    c.mu_hi = muj;
    c.hself = __shfl_sync(kFull, rh, 29);
    const uint32_t bdn = __shfl_sync(kFull, rh, 30), bup = __shfl_sync(kFull, rh, 31);
    const int dc = w >= 1 ? s.woff[w] - s.woff[w - 1] : 0;
    const int uc = w < L ? s.woff[w + 2] - s.woff[w + 1] : 0;
    const unsigned char* gd = (const unsigned char*)(p_dn + bdn);
    const unsigned char* gu = (const unsigned char*)(p_up + bup);
    const int od = (int)((uintptr_t)gd & 15u), ou = (int)((uintptr_t)gu & 15u);
    const int cd = dc ? (od + dc * (int)sizeof(T) + 15) >> 4 : 0;
    const int cu = uc ? (ou + uc * (int)sizeof(T) + 15) >> 4 : 0;
    unsigned char* sl = slot + (size_t)par * 2 * kHalf;
    for (int q = lane; q < cd; q += 32) cp_async16(sl + 16 * q, gd - od + 16 * q);
    for (int q = lane; q < cu; q += 32) cp_async16(sl + kHalf + 16 * q, gu - ou + 16 * q);
    asm volatile("cp.async.commit_group;" ::: "memory");
    c.grp = ngrp++;
    c.it0 = it0;
    c.size = s.woff[w + 1] - s.woff[w];
    c.od = od;
    c.ou = ou;
    bc = c;
    __syncwarp();  // the lists are visible to the warp
    return par;
  };
  // advance the sequence; false at its end
  auto next_item = [&](int& it_out, bool& newblk) -> bool {
    newblk = false;
    if (sit >= sie) {
      if (sr >= mbase + 32) fetch_meta(sr);
      const int src = sr - mbase;
      const uint32_t id = __shfl_sync(kFull, m_id, src);
      if (id == ~0u) return false;  // rounds past the phase's blocks stay past it
      const int it0 = __shfl_sync(kFull, m_it0, src);
      sr++;
      setup(id, it0, src);
      sit = it0;
      sie = it0 + (bc.size + HQ_SW_ITEM - 1) / HQ_SW_ITEM;
      newblk = true;
    }
    it_out = sit++;
    return true;
  };
  // issue every load of item `it` of the block in parity bq
  auto issue = [&](int it, int bq, ItemRef& ir, ItemLoads<V, kNV, kHP>& ld) {
    const BlockCtx<V>& c = bc;
    (void)bq;
    // items are the block's consecutive runs of 32 states from its first rank
    const int k32 = (it - c.it0) * HQ_SW_ITEM;
    ir.cnt = c.size - k32 < HQ_SW_ITEM ? c.size - k32 : HQ_SW_ITEM;
    ir.bq = bq;
    const bool act = lane < ir.cnt;
    ir.rk = c.hself + (uint32_t)k32 + (act ? (uint32_t)lane : 0u);
    const uint32_t rib = ir.rk - c.hself;
    const int n = c.n;
    const int64_t tw = s.tw[n];
    const int nvec = (int)tw / Vec<V>::kPer;
    const VT* rec = (const VT*)((const T*)a.T + s.toff[n] + (int64_t)ir.rk * tw);
#pragma unroll
    for (int v = 0; v < kNV; v++) {
      if (v >= nvec) break;
      ld.tv[v] = ld_vec(rec + v);
    }
#pragma unroll
    for (int j = 0; j < kHP; j++) {
      if (j >= H) break;
      ld.h[j] = ld_l2(s.hptr[wid][bq][j] + rib);
    }
    const int64_t on = s.off[n];
    ld.rv = ld_stream((const T*)a.r + on + ir.rk);
    ld.po = ld_l2(pv + on + ir.rk);
    if constexpr (kMode < 2) ld.wv = __ldcs((const W*)a.wv + on + ir.rk);
    if constexpr (kMode == 1) {
      const float* irn = a.ir + on + ir.rk;
      ld.q0 = ld_stream(irn);
      ld.q1 = ld_stream(irn + a.Sp);
      ld.q2 = ld_stream(irn + 2 * a.Sp);
    }
  };
  // compute item ir from its loads
  auto compute = [&](const ItemRef& ir, const ItemLoads<V, kNV, kHP>& ld) {
    const BlockCtx<V>& c = bc;
    // the block's staged low-part blocks: every group up to its own must be complete
    if (ngrp - 1 - c.grp >= 1) asm volatile("cp.async.wait_group 1;" ::: "memory");
    else asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();
    const int n = c.n, w = c.w;
    if (n != cur_n) {
      if (cur_n >= 0) flush();
      cur_n = n;
      li = (n - f) >> a.order;
      aS = aM = aW = aV = V::zero();
    }
    const bool act = lane < ir.cnt;
    const uint32_t rib = ir.rk - c.hself;
    const int ent = s.woff[w] + (int)rib;
    const uint4 lx = s.LX[ent];
    const unsigned char* sl = slot + (size_t)ir.bq * 2 * kHalf;
    const T* sdn = (const T*)(sl + c.od);
    const T* sup = (const T*)(sl + kHalf + c.ou);
    T U = V::zero(), D = V::zero();
    switch (w) {
#define HQ_INFLOWS(Wc) \
  case Wc: inflows<Wc, V, kHP, kNV>(U, D, ld.tv, ld.h, lx, sdn, sup, c.nbh, H, L, s.nu, s.hnu[wid][ir.bq]); break;
      HQ_INFLOWS(0) HQ_INFLOWS(1) HQ_INFLOWS(2) HQ_INFLOWS(3) HQ_INFLOWS(4) HQ_INFLOWS(5)
      HQ_INFLOWS(6) HQ_INFLOWS(7) HQ_INFLOWS(8) HQ_INFLOWS(9) HQ_INFLOWS(10)
#undef HQ_INFLOWS
      default: break;
    }
    const T c1 = s.c1[n], c2 = s.c2[n];
    if constexpr (kMode == 3) {
      // Eq. (1) at this state: out = P (lambda + mu_m), in = P-weighted inflows from its
      // neighbours, P = fac[layer] p (lambda_m = lambda in layers 1..N-1)
      const double mu = V::to_d(s.MUlo[s.LO[ent]]) + V::to_d(c.mu_hi);
      const double out = s.fac[n] * V::to_d(ld.po) * (a.lam + mu);
      const double in = s.fac[n - 1] * V::to_d(U) + s.fac[n + 1] * V::to_d(D);
      if (act) {
        rmax[0] = fmax(rmax[0], fabs(out - in));
        rmax[1] = fmax(rmax[1], out);
      }
    } else if constexpr (kMode == 2) {
      // base pass: rho0 = c1^0 A0 + c2^0 B0 - p0 (FP64 here), stored in FP32
      if (act) {
        float* outn = a.out + s.off[n] + ir.rk;
        const double A0 = V::to_d(U) * V::to_d(ld.rv), B0 = V::to_d(D) * V::to_d(ld.rv);
        const double rho0 = V::to_d(c1) * A0 + V::to_d(c2) * B0 - V::to_d(ld.po);
        outn[0] = (float)rho0;
        outn[a.Sp] = (float)A0;
        outn[2 * a.Sp] = (float)B0;
      }
    } else {
      // c1 A + c2 B with A = r U, B = r D
      T pn = V::mul(ld.rv, V::add(V::mul(c1, U), V::mul(c2, D)));
      if constexpr (kMode == 1)
        pn = V::add(V::add(ld.q0, V::add(V::mul(s.d1[n], ld.q1), V::mul(s.d2[n], ld.q2))), pn);
      if (relax) pn = V::add(ld.po, V::mul(om, V::sub(pn, ld.po)));
      md = fmaxf(md, V::absdiff(pn, ld.po));
      if (act) {
        pw[s.off[n] + ir.rk] = pn;
        aS = V::add(aS, pn);
        aM = V::add(aM, V::mul(pn, V::add(s.MUlo[s.LO[ent]], c.mu_hi)));
        aW = V::add(aW, V::mul(pn, WX::x(ld.wv)));
        aV = V::add(aV, V::mul(pn, WX::y(ld.wv)));
      }
    }
  };
  ItemLoads<V, kNV, kHP> LA;
  ItemRef RA;
  int it;
  bool nbk;
  while (next_item(it, nbk)) {
    issue(it, last_par, RA, LA);
    compute(RA, LA);
  }
  if (cur_n >= 0) flush();
}

// closed-form scalars of layer n from the layer sums of its neighbours
template <class V, int kWarps, int kHP, bool kIR>
__device__ void solve_layer(Smem<V, kWarps, kHP>& s, const SweepArgs& a, int n) {
  const double Sd = s.LS[0][n - 1], Wd = s.LS[2][n - 1], Sn = s.LS[0][n];
  const double Mu = s.LS[1][n + 1], Vu = s.LS[3][n + 1];
  const double lamd = a.lam * Sd;     // lambda(n-1), Eq. (13)
  const double alpha = 1.0 / lamd;
  const double beta = a.lam * Sn / Mu;  // lambda(n) / mu(n+1)
  const double aa = alpha * Wd;       // alpha sum_m mu_m A_m
  const double bb = beta * Vu;        // beta sum_m mu_m B_m
  const double mustar = bb / (1.0 - aa);
  const double c1 = alpha * mustar;
  s.c1[n] = V::from_d(c1);
  s.c2[n] = V::from_d(beta);
  if (kIR) {
    s.d1[n] = V::from_d(c1 - s.I1[n]);
    s.d2[n] = V::from_d(beta - s.I2[n]);
  }
  if (blockIdx.x == 0) {
    a.sc->c1[n] = c1;
    a.sc->c2[n] = beta;
    if (!isfinite(mustar) || !(aa < 1.0) || !(c1 >= 0.0)) atomicOr(&a.sc->flags, 1);
  }
}

template <class V, bool kIR, int kHP, int kThreads>
__global__ void __launch_bounds__(kThreads, 1) k_sweep(SweepArgs a) {
  constexpr int kWarps = kThreads / 32;
  constexpr int kSlot = kSlotBytes<V, kHP>();
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  __shared__ Smem<V, kWarps, kHP> s;
  DevScalars* sc = a.sc;
  const int N = a.N;
  const unsigned G = gridDim.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned char* slot = smem_dyn + (size_t)wid * kSlot;
  setup_tables(s, a);
  for (int i = threadIdx.x; i < 4 * (N + 1); i += kThreads) {
    const int q = i / (N + 1), n = i % (N + 1);
    s.LS[q][n] = sc->ls[q][n];
    if (kIR) s.IB[q][n] = sc->ir_sum[q][n];
  }
  if (kIR)
    for (int n = threadIdx.x; n <= N; n += kThreads) {
      s.I1[n] = sc->ir_c1[n];
      s.I2[n] = sc->ir_c2[n];
    }
  for (int i = threadIdx.x; i < kWarps * kMaxPL * 4; i += kThreads) (&s.ws[0][0][0])[i] = 0.0;
  if (threadIdx.x == 0) {
    s.step[0] = s.step[1] = 0.0;
    if (blockIdx.x == 0) sc->t_start = globaltimer_ns();
  }
  __syncthreads();
  {
    int f, nl;
    phase_layers(a.order, 0, N, f, nl);
    if ((int)threadIdx.x < nl) solve_layer<V, kWarps, kHP, kIR>(s, a, f + ((int)threadIdx.x << a.order));
  }
  __syncthreads();
  const unsigned limit = a.spin_limit ? a.spin_limit : kSpinDefault;
  int gphase = 0;
  for (int k = 0; k < a.nsweeps; k++) {
    if (threadIdx.x == 0) s.step[k & 1] = 0.0;
    for (int ph = 0; ph < a.nphases; ph++) {
      int f, nl;
      phase_layers(a.order, ph, N, f, nl);
      float md = 0.f;
      run_items<V, kIR ? 1 : 0, kHP, kWarps>(s, a, a.pbfirst[ph], a.pbfirst[ph + 1], f, slot, kSlot, md);
      // ---- end of phase: this CTA's partials, the grid barrier, the fold ----------------
      for (int m = 16; m > 0; m >>= 1) md = fmaxf(md, __shfl_xor_sync(kFull, md, m));
      if (lane == 0) s.wmd[wid] = md;
      __syncthreads();
      const int nw = 4 * nl + 1;
      double* part = a.partials + (size_t)(gphase & 1) * kMaxWords * G;
      if ((int)threadIdx.x < nw) {
        const int t = threadIdx.x;
        double v = 0.0;
        if (t < 4 * nl) {
          const int li = t >> 2, q = t & 3;
          for (int w2 = 0; w2 < kWarps; w2++) {
            v += s.ws[w2][li][q];
            s.ws[w2][li][q] = 0.0;
          }
        } else {
          for (int w2 = 0; w2 < kWarps; w2++) v = fmax(v, (double)s.wmd[w2]);
        }
        part[(size_t)t * G + blockIdx.x] = v;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();  // the CTA's partials (written before the CTA barrier) go first
        const bool skip = a.dbg_skip_cta == (int)blockIdx.x && gphase == 0;
        if (!skip) red_add_release(&sc->bar_count, 1u);
        const unsigned target = G * (unsigned)(gphase + 1);
        unsigned spins = 0;
        while ((int)(ld_relaxed_u32(&sc->bar_count) - target) < 0) {
          if (*(volatile int*)&sc->flags & 6) break;  // a wait gave up: do not wait again
          if (++spins > limit) {
            atomicOr(&sc->flags, 2);
            break;
          }
        }
        fence_acq_rel_gpu();
      }
      __syncthreads();
      // every CTA folds every CTA's partials in CTA order: identical scalars everywhere
      for (int t = wid; t < nw; t += kWarps) {
        const bool mx = t == 4 * nl;
        double v = 0.0;
        for (unsigned c = lane; c < G; c += 32) {
          const double x = __ldcg(part + (size_t)t * G + c);
          v = mx ? fmax(v, x) : v + x;
        }
        for (int m = 16; m > 0; m >>= 1) {
          const double o = __shfl_xor_sync(kFull, v, m);
          v = mx ? fmax(v, o) : v + o;
        }
        if (lane == 0) s.fold[t] = v;
      }
      __syncthreads();
      if ((int)threadIdx.x < nl) {
        const int t = threadIdx.x, n = f + (t << a.order);
#pragma unroll
        for (int q = 0; q < 4; q++) s.LS[q][n] = s.fold[4 * t + q] + (kIR ? s.IB[q][n] : 0.0);
      }
      if (threadIdx.x == 0) {
        s.step[k & 1] = fmax(s.step[k & 1], s.fold[4 * nl]);
        if (blockIdx.x == 0 && gphase < 64) sc->t_phase[gphase] = globaltimer_ns();
      }
      __syncthreads();
      {
        int fn, nln;
        phase_layers(a.order, ph + 1 < a.nphases ? ph + 1 : 0, N, fn, nln);
        if ((int)threadIdx.x < nln) solve_layer<V, kWarps, kHP, kIR>(s, a, fn + ((int)threadIdx.x << a.order));
      }
      __syncthreads();
      gphase++;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int n = 0; n <= N; n++) {
      for (int q = 0; q < 4; q++) sc->ls[q][n] = s.LS[q][n];
      if (n < N) {
        sc->lam_n[n] = a.lam * s.LS[0][n];
        sc->mu_n[n] = s.LS[1][n];
      }
    }
    const int kl = a.nsweeps - 1;
    sc->step_prev = a.nsweeps > 1 ? s.step[(kl - 1) & 1] : sc->step;
    sc->step = s.step[kl & 1];
    sc->sweeps += a.nsweeps;
    if (!isfinite(sc->step)) atomicOr(&sc->flags, 1);
  }
}

// The refinement's base pass: A0, B0 of every state of layers 1..N-1 gathered from p0
// (FP64 table), rho0 = c1^0 A0 + c2^0 B0 - p0 with c^0 the closed-form scalars of p0's own
// layer sums (every neighbour taken from p0), written as FP32 base terms.
template <int kHP, int kThreads>
__global__ void __launch_bounds__(kThreads, 1) k_base_pass(SweepArgs a) {
  constexpr int kWarps = kThreads / 32;
  constexpr int kSlot = kSlotBytes<PolF64, kHP>();
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  __shared__ Smem<PolF64, kWarps, kHP> s;
  const int N = a.N;
  const int wid = threadIdx.x >> 5;
  unsigned char* slot = smem_dyn + (size_t)wid * kSlot;
  setup_tables(s, a);
  for (int n = threadIdx.x; n <= N; n += kThreads) {
    s.c1[n] = a.sc->ir_c1[n];
    s.c2[n] = a.sc->ir_c2[n];
  }
  __syncthreads();
  float md = 0.f;
  run_items<PolF64, 2, kHP, kWarps>(s, a, a.pbfirst[0], a.pbfirst[a.nphases], 1, slot, kSlot, md);
}

// The relative global-balance residual's maxima over layers 1..N-1 (Eq. 1): the same
// gather as a sweep, from the FP64 iterate, with P = fac[n] p; per warp a max, folded by
// atomic maxima on the bit patterns of the non-negative doubles into res_num[1],
// res_den[1] (zeroed by the caller)
template <int kHP, int kThreads>
__global__ void __launch_bounds__(kThreads, 1) k_residual_fused(SweepArgs a) {
  constexpr int kWarps = kThreads / 32;
  constexpr int kSlot = kSlotBytes<PolF64, kHP>();
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  __shared__ Smem<PolF64, kWarps, kHP> s;
  const int N = a.N;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* slot = smem_dyn + (size_t)wid * kSlot;
  setup_tables(s, a);
  for (int n = threadIdx.x; n <= N; n += kThreads) s.fac[n] = a.sc->fac[n];
  __syncthreads();
  float md = 0.f;
  double rm[2] = {0.0, 0.0};
  run_items<PolF64, 3, kHP, kWarps>(s, a, a.pbfirst[0], a.pbfirst[a.nphases], 1, slot, kSlot, md, rm);
  for (int m = 16; m > 0; m >>= 1) {
    rm[0] = fmax(rm[0], __shfl_xor_sync(kFull, rm[0], m));
    rm[1] = fmax(rm[1], __shfl_xor_sync(kFull, rm[1], m));
  }
  if (lane == 0) {
    atomicMax((unsigned long long*)&a.sc->res_num[1], (unsigned long long)__double_as_longlong(rm[0]));
    atomicMax((unsigned long long*)&a.sc->res_den[1], (unsigned long long)__double_as_longlong(rm[1]));
  }
}

// base scalars c^0 of every layer from the base's layer sums (Jacobi: all from p0)
__global__ void k_base_scalars(DevScalars* sc, int N, double lam) {
  for (int n = 1 + threadIdx.x; n <= N - 1; n += blockDim.x) {
    const double Sd = sc->ir_sum[0][n - 1], Wd = sc->ir_sum[2][n - 1], Sn = sc->ir_sum[0][n];
    const double Mu = sc->ir_sum[1][n + 1], Vu = sc->ir_sum[3][n + 1];
    const double alpha = 1.0 / (lam * Sd), beta = lam * Sn / Mu;
    const double mustar = beta * Vu / (1.0 - alpha * Wd);
    sc->ir_c1[n] = alpha * mustar;
    sc->ir_c2[n] = beta;
  }
}

// ---- the four layer sums of an iterate, and the per-state weights ---------------------

// Per warp: a contiguous run of 32-state chunks (layers start on 32-entry boundaries,
// so a chunk lies in one layer); FP64 sums per layer, written per warp and folded by
// k_iter_sums_fold in warp order (deterministic).
struct SumArgs {
  int N, L;
  int64_t off[HQ_MAXN + 2];
  int64_t lsize[HQ_MAXN + 1];
  const uint32_t* masks;
  const void* p;
  const double2* wv;   // FP64 weights
  const double* mulo;  // mu of each low part (2^L), then mu of each high part (2^H)
  const double* muhi;
  double* part;        // [warps][HQ_MAXN + 1][4]
};

template <class V>
__global__ void __launch_bounds__(256) k_iter_sums(SumArgs a) {
  const int lane = threadIdx.x & 31;
  const uint32_t lomask = (1u << a.L) - 1u;
  const int64_t chunks = a.off[a.N + 1] >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t per = (chunks + nw - 1) / nw;
  const int64_t c0 = gw * per, c1 = c0 + per < chunks ? c0 + per : chunks;
  double* out = a.part + (size_t)gw * (HQ_MAXN + 1) * 4;
  for (int i = lane; i < (HQ_MAXN + 1) * 4; i += 32) out[i] = 0.0;
  __syncwarp();
  int n = 0;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const typename V::T* p = (const typename V::T*)a.p;
  for (int64_t c = c0; c < c1; c++) {
    const int64_t g = (c << 5) + lane;
    int nc = n;
    while (nc < a.N && a.off[nc + 1] <= (c << 5)) nc++;
    if (nc != n) {
      for (int q = 0; q < 4; q++) {
        double v = acc[q];
        for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(kFull, v, m);
        if (lane == 0) out[n * 4 + q] += v;
        acc[q] = 0.0;
      }
      n = nc;
    }
    if (g - a.off[n] < a.lsize[n]) {
      const double pv = V::to_d(p[g]);
      const uint32_t x = a.masks[g];
      const double mu = __ldg(a.mulo + (x & lomask)) + __ldg(a.muhi + (x >> a.L));
      const double2 wq = a.wv[g];
      acc[0] += pv;
      acc[1] += pv * mu;
      acc[2] += pv * wq.x;
      acc[3] += pv * wq.y;
    }
  }
  for (int q = 0; q < 4; q++) {
    double v = acc[q];
    for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(kFull, v, m);
    if (lane == 0 && c0 < c1) out[n * 4 + q] += v;
  }
}

// dst[q][n] = sum over warps of part[w][n][q]; dst has stride HQ_MAXN + 1.  One CTA per
// output: thread t sums warps t, t + 256, ... in order, then a fixed halving tree
// (the same order on every run).
__global__ void __launch_bounds__(256) k_iter_sums_fold(int N, int nwarps, const double* part, double* dst) {
  __shared__ double red[256];
  const int i = blockIdx.x;
  const int q = i / (N + 1), n = i % (N + 1);
  double v = 0.0;
  for (int w = threadIdx.x; w < nwarps; w += 256) v += part[((size_t)w * (HQ_MAXN + 1) + n) * 4 + q];
  red[threadIdx.x] = v;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) dst[q * (HQ_MAXN + 1) + n] = red[0];
}

// w''(l) = sum_{u idle in l} lambda_u(l) mu_{l+u} r_{l+u} (the upward rates are the
// table entries of state l+u at the slot of u), v''(l) = sum_{u busy in l} nu_u mu_{l-u}
// r_{l-u}, in FP64, and their FP32 copies; padding entries get zeros.
struct WeightArgs {
  int N, L;
  int64_t off[HQ_MAXN + 2];
  int64_t toff[HQ_MAXN + 2];
  int64_t lsize[HQ_MAXN + 1];
  int64_t tw[HQ_MAXN + 1];
  const uint32_t* masks;
  const uint32_t* RL;
  const uint32_t* RH;
  const double* T;
  const double* r;
  const double* nu;
  const double* mulo;
  const double* muhi;
  double lam, lam_full;
  double2* w64;
  float2* w32;
};

// mu of every low part (sum of nu over its busy units, in unit order) and of every high
// part: mu(x) = mulo[x & (2^L - 1)] + muhi[x >> L]
__global__ void k_mu_tables(int L, int H, const double* nu, double* mulo, double* muhi) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nlo = (int64_t)1 << L, nhi = (int64_t)1 << H;
  if (i < nlo) {
    double m = 0.0;
    for (uint32_t y = (uint32_t)i; y; y &= y - 1u) m += nu[__ffs(y) - 1];
    mulo[i] = m;
  } else if (i < nlo + nhi) {
    double m = 0.0;
    for (uint32_t y = (uint32_t)(i - nlo); y; y &= y - 1u) m += nu[L + __ffs(y) - 1];
    muhi[i - nlo] = m;
  }
}

__global__ void __launch_bounds__(256) k_weights(WeightArgs a, int64_t Sp) {
  __shared__ double snu[HQ_MAXN];
  if ((int)threadIdx.x < a.N) snu[threadIdx.x] = a.nu[threadIdx.x];
  __syncthreads();
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= Sp) return;
  int n = 0;
  while (n < a.N && a.off[n + 1] <= g) n++;
  double wu = 0.0, wd = 0.0;
  if (g - a.off[n] < a.lsize[n]) {
    const int N = a.N, L = a.L;
    const uint32_t x = a.masks[g];
    auto rank = [&](uint32_t y) -> uint32_t {
      const uint32_t lo = y & ((1u << L) - 1u), hi = y >> L;
      return __ldg(a.RL + lo) + __ldg(a.RH + (size_t)hi * (L + 1) + __popc(lo));
    };
    // mu of a neighbour: mu(x) plus or minus one unit's rate
    const double mux = __ldg(a.mulo + (x & ((1u << L) - 1u))) + __ldg(a.muhi + (x >> L));
    // neighbours four at a time, so their rank-table and table loads are in flight
    // together; the sums still run in increasing unit order
    if (n < N) {
      uint32_t idle = ~x & ((1u << N) - 1u);
      while (idle) {
        int us[4];
        uint32_t ry[4];
        double t[4], rv[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
          us[q] = idle ? __ffs(idle) - 1 : -1;
          idle &= idle - 1u;
        }
#pragma unroll
        for (int q = 0; q < 4; q++)
          if (us[q] >= 0) ry[q] = rank(x | (1u << us[q]));
#pragma unroll
        for (int q = 0; q < 4; q++)
          if (us[q] >= 0) {
            const int slot = __popc(x & ((1u << us[q]) - 1u));
            t[q] = a.T[a.toff[n + 1] + (int64_t)ry[q] * a.tw[n + 1] + slot];
            rv[q] = a.r[a.off[n + 1] + ry[q]];
          }
#pragma unroll
        for (int q = 0; q < 4; q++)
          if (us[q] >= 0) wu += t[q] * (mux + snu[us[q]]) * rv[q];
      }
    }
    if (n > 0) {
      uint32_t busy = x;
      while (busy) {
        int us[4];
        uint32_t ry[4];
        double rv[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
          us[q] = busy ? __ffs(busy) - 1 : -1;
          busy &= busy - 1u;
        }
#pragma unroll
        for (int q = 0; q < 4; q++)
          if (us[q] >= 0) ry[q] = rank(x ^ (1u << us[q]));
#pragma unroll
        for (int q = 0; q < 4; q++)
          if (us[q] >= 0) rv[q] = a.r[a.off[n - 1] + ry[q]];
#pragma unroll
        for (int q = 0; q < 4; q++)
          if (us[q] >= 0) wd += snu[us[q]] * (mux - snu[us[q]]) * rv[q];
      }
    }
  }
  a.w64[g] = make_double2(wu, wd);
  a.w32[g] = make_float2((float)wu, (float)wd);
}

// ---- launch ---------------------------------------------------------------------------------

constexpr int kSweepThreads = 512;
constexpr int kSweepThreadsNarrow = 640;
constexpr int kSweepThreadsWide = 384;

// One CTA per SM.  FP32 sweeps with the 14- or 18-entry high-part list (N <= 28): 640
// threads (20 warps, up to 102 registers, no spills); measured at N=24, 0.562 ms per
// red-black sweep (0.590 before the item loop held one block context) against 0.606 at
// 576, 0.636 at 512 and 0.70 at 768 threads (spilling); at N=26 2.28 against 2.54 ms at
// 512.  FP32 sweeps at N = 29: 512 threads (the 20-entry list spills at 640).  FP64 and
// DF64 sweeps, whose wider values spill at 128 registers: 384 threads (12 warps, up to 168
// registers); measured at N=24 against 512 and 256, DF64 1.36 vs 1.63 and 1.80 ms per
// red-black sweep, FP64 1.98 vs 2.00 and 2.21 ms.
int sweep_threads(int H, int kind) {
  if (kind != HQ_PREC_FP32) return kSweepThreadsWide;
  return H <= 18 ? kSweepThreadsNarrow : kSweepThreads;
}

// high-part list sizes: 14 (N <= 24), 18 (N <= 28), 20 (N = 29; no double-float there)
template <class V, bool kIR>
const void* sweep_fn(int H) {
  constexpr bool k32 = V::kind == HQ_PREC_FP32;
  constexpr int kT = k32 ? kSweepThreadsNarrow : kSweepThreadsWide;
  constexpr int kT20 = k32 ? kSweepThreads : kSweepThreadsWide;
  if (H <= 14) return (const void*)k_sweep<V, kIR, 14, kT>;
  if (H <= 18) return (const void*)k_sweep<V, kIR, 18, kT>;
  if constexpr (V::kind != HQ_PREC_DF64) return (const void*)k_sweep<V, kIR, 20, kT20>;
  return nullptr;
}

int g_nsm = 0;

void fill_args(hq_solver* h, SweepArgs& a, int order) {
  memset(&a, 0, sizeof(a));
  a.N = h->N;
  a.L = h->L;
  a.H = h->H;
  a.order = order;
  a.nphases = h->snph[order];
  a.lam = h->lam;
  a.omega = h->omega;
  a.Sp = h->Sp;
  for (int i = 0; i < HQ_MAXN + 2; i++) {
    a.off[i] = h->off[i];
    a.toff[i] = h->toff[i];
    a.tw[i] = i <= h->N ? h->tw[i] : 0;
    a.pbfirst[i] = h->spbfirst[order][i];
  }
  a.items = h->sitems[order];
  a.blocks = h->sblocks[order];
  a.perm = h->sperm[order];
  a.RL = h->RL;
  a.RH = h->RH;
  a.partials = h->partials;
  a.sc = h->sc;
  a.spin_limit = h->spin_limit;
  a.dbg_skip_cta = h->dbg_skip_cta;
}

// ir: correction sweeps (FP32 only), against the base set up by hq_ir_begin
template <class V>
int launch_sweep(hq_solver* h, int nsweeps, cudaEvent_t ev0, cudaEvent_t ev1, int G, bool ir) {
  typedef typename V::T T;
  const int thr = sweep_threads(h->H, V::kind);
  const size_t smem = (size_t)(thr / 32) * slot_bytes<V>(h->H);
  const void* kfn = ir ? sweep_fn<PolF32, true>(h->H) : sweep_fn<V, false>(h->H);
  PrecBufs& bp = hq_bufs(h, V::kind);
  SweepArgs a;
  fill_args(h, a, h->order);
  a.nsweeps = nsweeps;
  a.T = bp.T;
  a.r = bp.r;
  a.p = bp.p;
  a.nu = bp.nu;
  a.wv = V::kind == HQ_PREC_FP32 ? h->wv32 : h->wv64;
  a.ir = ir ? h->ir : nullptr;
  void* args[] = {&a};
  // a barrier left half-entered by an aborted launch must not leak into this one
  HQ_CUDA(cudaMemsetAsync(&h->sc->bar_count, 0, sizeof(unsigned), h->stream));
  if (ev0) HQ_CUDA(cudaEventRecord(ev0, h->stream));
  HQ_CUDA(cudaLaunchCooperativeKernel(kfn, dim3(G), dim3(thr), args, smem, h->stream));
  HQ_LAUNCHED();
  if (ev1) HQ_CUDA(cudaEventRecord(ev1, h->stream));
  return HQ_OK;
}

// grid of the sweep kernel: one CTA per SM times its occupancy
template <class V>
int sweep_grid(hq_solver* h, bool ir, int* G) {
  typedef typename V::T T;
  const int thr = sweep_threads(h->H, V::kind);
  const size_t smem = (size_t)(thr / 32) * slot_bytes<V>(h->H);
  const void* kfn = ir ? sweep_fn<PolF32, true>(h->H) : sweep_fn<V, false>(h->H);
  if (!kfn) {
    hq_set_error("no sweep kernel for this precision at this N");
    return HQ_EINVAL;
  }
  if (!g_nsm) HQ_CUDA(cudaDeviceGetAttribute(&g_nsm, cudaDevAttrMultiProcessorCount, h->dev));
  HQ_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  HQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, thr, smem));
  if (occ < 1) {
    hq_set_error("persistent sweep kernel does not fit on an SM");
    return HQ_ECUDA;
  }
  *G = g_nsm * occ;
  if ((int64_t)(*G) * kMaxWords * 2 > h->partials_len) {
    hq_set_error("partials buffer too small for the persistent grid");
    return HQ_ECUDA;
  }
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
  const bool ir = prec == HQ_PREC_IRC;
  int G = 0, rc;
  if (prec == HQ_PREC_FP64) rc = sweep_grid<PolF64>(h, false, &G);
  else if (prec == HQ_PREC_DF64) rc = sweep_grid<PolDF>(h, false, &G);
  else rc = sweep_grid<PolF32>(h, ir, &G);
  if (rc != HQ_OK) return rc;
  // the barrier's arrival count (grid size x phases of one launch) stays below 2^31
  const int64_t per = ((int64_t)1 << 31) / ((int64_t)G * h->snph[h->order] + 1) - 1;
  const int cap = per > (1 << 20) ? (1 << 20) : (per < 1 ? 1 : (int)per);
  for (int done = 0; done < nsweeps;) {
    const int k = nsweeps - done < cap ? nsweeps - done : cap;
    cudaEvent_t e0 = done == 0 ? ev0 : nullptr, e1 = done + k == nsweeps ? ev1 : nullptr;
    if (prec == HQ_PREC_FP64) rc = launch_sweep<PolF64>(h, k, e0, e1, G, false);
    else if (prec == HQ_PREC_DF64) rc = launch_sweep<PolDF>(h, k, e0, e1, G, false);
    else rc = launch_sweep<PolF32>(h, k, e0, e1, G, ir);
    if (rc != HQ_OK) return rc;
    done += k;
  }
  return HQ_OK;
}

int hq_base_pass(hq_solver* h) {
  if (h->N < 2) return HQ_OK;
  k_base_scalars<<<1, 32, 0, h->stream>>>(h->sc, h->N, h->lam);
  HQ_LAUNCHED();
  SweepArgs a;
  fill_args(h, a, HQ_ORDER_ASCENDING);
  a.T = h->b64.T;
  a.r = h->b64.r;
  a.p = h->ir_base;
  a.nu = h->b64.nu;
  a.wv = h->wv64;
  a.out = h->ir;
  const size_t smem = (size_t)(kSweepThreadsWide / 32) * slot_bytes<PolF64>(h->H);
  const void* kfn = h->H <= 14   ? (const void*)k_base_pass<14, kSweepThreadsWide>
                    : h->H <= 18 ? (const void*)k_base_pass<18, kSweepThreadsWide>
                                 : (const void*)k_base_pass<20, kSweepThreadsWide>;
  HQ_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (!g_nsm) HQ_CUDA(cudaDeviceGetAttribute(&g_nsm, cudaDevAttrMultiProcessorCount, h->dev));
  void* args[] = {&a};
  HQ_CUDA(cudaLaunchKernel(kfn, dim3(g_nsm), dim3(kSweepThreadsWide), args, smem, h->stream));
  HQ_LAUNCHED();
  return HQ_OK;
}

int hq_residual_fused(hq_solver* h) {
  if (h->N < 2) return HQ_OK;
  if (!g_nsm) HQ_CUDA(cudaDeviceGetAttribute(&g_nsm, cudaDevAttrMultiProcessorCount, h->dev));
  SweepArgs a;
  fill_args(h, a, HQ_ORDER_ASCENDING);
  a.T = h->b64.T;
  a.r = h->b64.r;
  a.p = h->b64.p;
  a.nu = h->b64.nu;
  a.wv = h->wv64;
  HQ_CUDA(cudaMemsetAsync(&h->sc->res_num[0], 0, sizeof(double) * (HQ_MAXN + 1), h->stream));
  HQ_CUDA(cudaMemsetAsync(&h->sc->res_den[0], 0, sizeof(double) * (HQ_MAXN + 1), h->stream));
  const size_t smem = (size_t)(kSweepThreadsWide / 32) * slot_bytes<PolF64>(h->H);
  const void* kfn = h->H <= 14   ? (const void*)k_residual_fused<14, kSweepThreadsWide>
                    : h->H <= 18 ? (const void*)k_residual_fused<18, kSweepThreadsWide>
                                 : (const void*)k_residual_fused<20, kSweepThreadsWide>;
  HQ_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  void* args[] = {&a};
  HQ_CUDA(cudaLaunchKernel(kfn, dim3(g_nsm), dim3(kSweepThreadsWide), args, smem, h->stream));
  HQ_LAUNCHED();
  return HQ_OK;
}

int hq_iter_sums(hq_solver* h, int prec, const void* p, double* dst) {
  SumArgs a;
  memset(&a, 0, sizeof(a));
  a.N = h->N;
  a.L = h->L;
  for (int i = 0; i < HQ_MAXN + 2; i++) a.off[i] = h->off[i];
  for (int i = 0; i <= HQ_MAXN; i++) a.lsize[i] = i <= h->N ? h->lsize[i] : 0;
  a.masks = h->masks;
  a.p = p;
  a.wv = (const double2*)h->wv64;
  a.mulo = h->mutab;
  a.muhi = h->mutab + ((int64_t)1 << h->L);
  a.part = h->partials;
  // 8 warps per CTA; at most partials_len / (4 (HQ_MAXN + 1)) warps
  const int64_t chunks = h->Sp >> 5;
  int64_t warps = (chunks + 3) / 4;
  const int64_t wmax = h->partials_len / (4 * (HQ_MAXN + 1));
  if (warps > wmax) warps = wmax;
  warps = (warps + 7) / 8 * 8;
  if (warps > wmax) warps = wmax / 8 * 8;
  if (warps < 8) warps = 8;
  const unsigned grid = (unsigned)(warps / 8);
  if (prec == HQ_PREC_FP64) k_iter_sums<PolF64><<<grid, 256, 0, h->stream>>>(a);
  else if (prec == HQ_PREC_DF64) k_iter_sums<PolDF><<<grid, 256, 0, h->stream>>>(a);
  else k_iter_sums<PolF32><<<grid, 256, 0, h->stream>>>(a);
  HQ_LAUNCHED();
  k_iter_sums_fold<<<4 * (h->N + 1), 256, 0, h->stream>>>(h->N, (int)warps, h->partials, dst);
  HQ_LAUNCHED();
  return HQ_OK;
}

int hq_build_weights(hq_solver* h) {
  WeightArgs a;
  memset(&a, 0, sizeof(a));
  a.N = h->N;
  a.L = h->L;
  for (int i = 0; i < HQ_MAXN + 2; i++) {
    a.off[i] = h->off[i];
    a.toff[i] = h->toff[i];
  }
  for (int i = 0; i <= HQ_MAXN; i++) {
    a.lsize[i] = i <= h->N ? h->lsize[i] : 0;
    a.tw[i] = i <= h->N ? h->tw[i] : 0;
  }
  a.masks = h->masks;
  a.RL = h->RL;
  a.RH = h->RH;
  a.T = (const double*)h->b64.T;
  a.r = (const double*)h->b64.r;
  a.nu = h->nu;
  a.lam = h->lam;
  a.lam_full = h->mode == HQ_LOSS ? 0.0 : h->lam;
  a.w64 = (double2*)h->wv64;
  a.w32 = (float2*)h->wv32;
  a.mulo = h->mutab;
  a.muhi = h->mutab + ((int64_t)1 << h->L);
  {
    const int64_t nt = ((int64_t)1 << h->L) + ((int64_t)1 << h->H);
    k_mu_tables<<<(unsigned)((nt + 255) / 256), 256, 0, h->stream>>>(h->L, h->H, h->nu, h->mutab,
                                                                    h->mutab + ((int64_t)1 << h->L));
    HQ_LAUNCHED();
  }
  k_weights<<<(unsigned)((h->Sp + 255) / 256), 256, 0, h->stream>>>(a, h->Sp);
  HQ_LAUNCHED();
  return HQ_OK;
}

int hq_sweep_partials_words() { return kMaxWords; }

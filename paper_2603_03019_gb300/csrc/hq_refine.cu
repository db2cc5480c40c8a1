// Mixed-precision refinement of the outer iteration (Algorithm 1, Eq. 12-14): FP32
// correction sweeps against a fixed FP64 base.
//
// Write the iterate as p = p0 + e with p0 fixed (FP64).  The gathers of Eq. (12) are
// linear in p:
//     A_m = r_m sum_s T[m][s] p_{n-1}(m - c_s)       = A0_m + a_m,
//     B_m = r_m sum_{u idle} nu_u p_{n+1}(m + u)      = B0_m + b_m,
// where A0, B0 gather p0 and a, b gather e.  With the layer's scalars written as
// c1 = c1^0 + d1 and c2 = c2^0 + d2 (c^0 fixed with the base),
//     e_n(m) = c1 A_m + c2 B_m - p0_n(m) = rho0_m + d1 A0_m + d2 B0_m + c1 a_m + c2 b_m,
//     rho0_m = c1^0 A0_m + c2^0 B0_m - p0_n(m),
// and the pull term that layer n+1 gathers splits the same way:
//     sum_s T[m][s] e_n(m - c_s) = G_rho(m) + d1 G_A(m) + d2 G_B(m) + c1 sum T a + c2 sum T b,
// with G_x(m) = sum_s T[m][s] x(m - c_s) gathered once from the base terms of layer n.
// Every term on the right is of the size of the correction, so the FP32 arithmetic of
// the correction sweeps loses about 1e-7 of |e| rather than of |p|.  The layer sums of
// the closed-form step (sum mu A, sum mu B, sum A, sum B) are the base's (FP64, once per
// base) plus the corrections' (FP32 partials of the sweep, folded in FP64).
//
// This file: the base pass (FP64 gathers of p0: rho0, A0, B0 per state and per-item
// partial sums), the per-layer fold of those sums in item order (deterministic), the
// gather of the base terms (G_rho, G_A, G_B), re-basing (p0 += e) and the assembly of
// p0 + e for the residual and the outputs.  The correction sweeps themselves are the
// persistent sweep kernel in its correction mode (hq_persist.cu).
#include <string.h>

#include "hq_internal.cuh"

namespace {

struct IrArgs {
  int N, L, H;
  double lam;
  int64_t Sp;
  int ifirst[HQ_MAXN + 2];
  int64_t off[HQ_MAXN + 2];
  int64_t toff[HQ_MAXN + 2];
  int64_t lpad[HQ_MAXN + 1];
  const uint4* items;
  const uint32_t* masks;
  const uint32_t* lidx;
  const uint32_t* RL;
  const uint32_t* RH;
  const double* T;   // FP64 pull-form table
  const float* T32;  // FP32 pull-form table
  const double* r;   // FP64 r_m
  const double* nu;  // FP64 nu_i
  const double* pb;  // the base p0
  float* ir;         // 6 x Sp: rho0, A0, B0, G_rho, G_A, G_B
  double* ipart;     // 4 per item
  DevScalars* sc;
};

// Visit the neighbours of the state of lane `lane` of item `d` of layer n: busy(s, rank)
// for table slot s (increasing unit) and its neighbour's rank in layer n-1, then
// idle(u, rank) for idle unit u (increasing) and its neighbour's rank in layer n+1.
// The ranks follow the item format of HQ_ITEM_HI_BITS: low-part neighbours at the
// lidx positions within the blocks (hi, w-1) / (hi, w+1), high-part ones at
// RH[hi ^ 2^j][w] + RL[lo].
template <class FB, class FI>
__device__ void visit(const IrArgs& a, uint4 d, uint32_t x, uint32_t w0, uint32_t w1, uint32_t w2, FB busy,
                      FI idle) {
  const int L = a.L, H = a.H;
  const uint32_t hi = d.y & ((1u << HQ_ITEM_HI_BITS) - 1u);
  const int w = (int)((d.y >> HQ_ITEM_HI_BITS) & 0xfu);
  const uint32_t lo = x & ((1u << L) - 1u);
  const uint32_t rl = __ldg(a.RL + lo);
  int s = 0;
  for (int k = 0; k < w; k++) {
    const uint32_t wd = k < 4 ? w0 : (k < 8 ? w1 : w2);
    busy(s++, d.z + ((wd >> (8 * (k & 3))) & 0xffu));
  }
  for (int j = 0; j < H; j++)
    if ((hi >> j) & 1u) busy(s++, __ldg(a.RH + (size_t)(hi ^ (1u << j)) * (L + 1) + w) + rl);
  uint32_t z = ~lo & ((1u << L) - 1u);
  for (int k = w; k < L; k++) {
    const uint32_t wd = k < 4 ? w0 : (k < 8 ? w1 : w2);
    const int u = __ffs(z) - 1;
    z &= z - 1u;
    idle(u, d.w + ((wd >> (8 * (k & 3))) & 0xffu));
  }
  for (int j = 0; j < H; j++)
    if (!((hi >> j) & 1u)) idle(L + j, __ldg(a.RH + (size_t)(hi ^ (1u << j)) * (L + 1) + w) + rl);
}

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

// kPass 0: the base terms of every state of layers 1..N-1 from p0 (FP64), and per-item
// partial sums {sum mu_m A0_m, sum mu_m B0_m, sum A0_m, sum B0_m} (mu_m r_m = 1 - lambda r_m).
// kPass 1: G_rho, G_A, G_B of every state of layers 2..N-1 from the stored base terms
// of layer n-1 (zero in layer 1, which pulls from the empty state), in FP32: G_rho is
// of the correction's size and G_A, G_B only ever multiply d1, d2, so FP32 rounding
// of them is rounding relative to the correction.
template <int kPass>
__global__ void __launch_bounds__(256) k_ir_pass(IrArgs a) {
  const int lane = threadIdx.x & 31;
  const int nitems = a.ifirst[a.N];
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int64_t Sp = a.Sp;
  for (int it = a.ifirst[1] + gw; it < nitems; it += nw) {
    const uint4 d = __ldg(a.items + it);
    const uint32_t hi = d.y & ((1u << HQ_ITEM_HI_BITS) - 1u);
    const int w = (int)((d.y >> HQ_ITEM_HI_BITS) & 0xfu);
    const int count = (int)((d.y >> 24) & 0x1fu) + 1;
    const int n = __popc(hi) + w;
    const bool act = lane < count;
    const uint32_t kq = d.x + (act ? (uint32_t)lane : 0u);
    const int64_t gi = a.off[n] + kq;
    const uint32_t x = __ldg(a.masks + gi);
    const uint32_t w0 = __ldg(a.lidx + gi), w1 = __ldg(a.lidx + Sp + gi), w2 = __ldg(a.lidx + 2 * Sp + gi);
    const double* tcol = a.T + a.toff[n] + kq;
    const int64_t lp = a.lpad[n];
    if (kPass == 0) {
      const double* pd = a.pb + a.off[n - 1];
      const double* pu = a.pb + a.off[n + 1];
      double U0 = 0.0, D0 = 0.0;
      if (n == 1) U0 = tcol[0];  // the empty state, p_0 = 1
      visit(
          a, d, x, w0, w1, w2,
          [&](int s, uint32_t rk) {
            if (n > 1) U0 = fma(tcol[s * lp], pd[rk], U0);
          },
          [&](int u, uint32_t rk) { D0 = fma(__ldg(a.nu + u), pu[rk], D0); });
      const double rv = __ldg(a.r + gi);
      const double A0 = U0 * rv, B0 = D0 * rv;
      const double rho0 = a.sc->ir_c1[n] * A0 + a.sc->ir_c2[n] * B0 - a.pb[gi];
      if (act) {
        a.ir[gi] = (float)rho0;
        a.ir[Sp + gi] = (float)A0;
        a.ir[2 * Sp + gi] = (float)B0;
      }
      const double qm = 1.0 - a.lam * rv;
      const double v0 = warp_sum_d(act ? qm * U0 : 0.0);
      const double v1 = warp_sum_d(act ? qm * D0 : 0.0);
      const double v2 = warp_sum_d(act ? A0 : 0.0);
      const double v3 = warp_sum_d(act ? B0 : 0.0);
      if (lane == 0) {
        double* q = a.ipart + (size_t)it * 4;
        q[0] = v0;
        q[1] = v1;
        q[2] = v2;
        q[3] = v3;
      }
    } else {
      float gR = 0.f, gA = 0.f, gB = 0.f;
      if (n > 1) {
        const float* bd = a.ir + a.off[n - 1];
        const float* t32 = a.T32 + a.toff[n] + kq;
        visit(
            a, d, x, w0, w1, w2,
            [&](int s, uint32_t rk) {
              const float t = __ldg(t32 + s * lp);
              gR = fmaf(t, bd[rk], gR);
              gA = fmaf(t, bd[Sp + rk], gA);
              gB = fmaf(t, bd[2 * Sp + rk], gB);
            },
            [&](int, uint32_t) {});
      }
      if (act) {
        a.ir[3 * Sp + gi] = gR;
        a.ir[4 * Sp + gi] = gA;
        a.ir[5 * Sp + gi] = gB;
      }
    }
  }
}

// the base's c^0 (the scalars of the last layer updates) frozen for the base's lifetime
__global__ void k_ir_prep(DevScalars* sc, int N) {
  for (int n = threadIdx.x; n <= N; n += blockDim.x) {
    sc->ir_c1[n] = sc->c1[n];
    sc->ir_c2[n] = sc->c2[n];
  }
}

// per-layer sums of the item partials in item order: block n-1 folds layer n
__global__ void __launch_bounds__(256) k_ir_fold(const double* ipart, IrArgs a) {
  __shared__ double s[4][256];
  const int n = (int)blockIdx.x + 1;
  const int i0 = a.ifirst[n], i1 = a.ifirst[n + 1];
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int it = i0 + (int)threadIdx.x; it < i1; it += (int)blockDim.x)
    for (int c = 0; c < 4; c++) v[c] += ipart[(size_t)it * 4 + c];
  for (int c = 0; c < 4; c++) s[c][threadIdx.x] = v[c];
  __syncthreads();
  for (int m = 128; m > 0; m >>= 1) {
    if ((int)threadIdx.x < m)
      for (int c = 0; c < 4; c++) s[c][threadIdx.x] += s[c][threadIdx.x + m];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int c = 0; c < 4; c++) a.sc->ir_sum[c][n] = s[c][0];
}

__global__ void k_ir_assemble(int64_t Sp, const double* pb, const float* e, double* p) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < Sp) p[i] = pb[i] + (double)e[i];
}

__global__ void k_ir_rebase(int64_t Sp, double* pb, const float* e) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < Sp) pb[i] += (double)e[i];
}

}  // namespace

int hq_ir_assemble(hq_solver* h) {
  const unsigned grid = (unsigned)((h->Sp + 255) / 256);
  k_ir_assemble<<<grid, 256, 0, h->stream>>>(h->Sp, h->ir_base, (const float*)h->b32.p, (double*)h->b64.p);
  HQ_LAUNCHED();
  return HQ_OK;
}

int hq_ir_begin(hq_solver* h, int from) {
  const int64_t Sp = h->Sp;
  h->it_version++;
  const unsigned grid = (unsigned)((Sp + 255) / 256);
  if (from == HQ_PREC_IRC) {
    k_ir_rebase<<<grid, 256, 0, h->stream>>>(Sp, h->ir_base, (const float*)h->b32.p);
    HQ_LAUNCHED();
  } else {
    if (from != HQ_PREC_FP64) {
      const int rc = hq_convert_iterate(h, from, HQ_PREC_FP64);
      if (rc != HQ_OK) return rc;
    }
    HQ_CUDA(cudaMemcpyAsync(h->ir_base, h->b64.p, sizeof(double) * Sp, cudaMemcpyDeviceToDevice, h->stream));
  }
  if (h->N >= 2) {
    IrArgs a;
    memset(&a, 0, sizeof(a));
    a.N = h->N;
    a.L = h->L;
    a.H = h->H;
    a.lam = h->lam;
    a.Sp = Sp;
    for (int i = 0; i < HQ_MAXN + 2; i++) {
      a.ifirst[i] = h->ifirst[i];
      a.off[i] = h->off[i];
      a.toff[i] = h->toff[i];
    }
    for (int n = 0; n <= HQ_MAXN; n++) a.lpad[n] = n <= h->N ? h->lpad[n] : 0;
    a.items = h->items;
    a.masks = h->masks;
    a.lidx = h->lidx;
    a.RL = h->RL;
    a.RH = h->RH;
    a.T = (const double*)h->b64.T;
    a.T32 = (const float*)h->b32.T;
    a.r = (const double*)h->b64.r;
    a.nu = h->nu;
    a.pb = h->ir_base;
    a.ir = h->ir;
    a.ipart = h->ir_part;
    a.sc = h->sc;
    const int items = h->ifirst[h->N] - h->ifirst[1];
    const int64_t want = ((int64_t)items * 32 + 255) / 256;
    const unsigned g = (unsigned)(want < 152 * 16 ? (want > 0 ? want : 1) : 152 * 16);
    k_ir_prep<<<1, 32, 0, h->stream>>>(h->sc, h->N);
    HQ_LAUNCHED();
    k_ir_pass<0><<<g, 256, 0, h->stream>>>(a);
    HQ_LAUNCHED();
    k_ir_fold<<<h->N - 1, 256, 0, h->stream>>>(h->ir_part, a);
    HQ_LAUNCHED();
    k_ir_pass<1><<<g, 256, 0, h->stream>>>(a);
    HQ_LAUNCHED();
  }
  // e = 0 everywhere (the empty and the full state have no correction)
  HQ_CUDA(cudaMemsetAsync(h->b32.p, 0, sizeof(float) * Sp, h->stream));
  h->cur_prec = HQ_PREC_IRC;
  return HQ_OK;
}

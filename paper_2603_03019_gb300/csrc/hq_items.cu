// Work items of the sweep kernels (built on the host from N alone, at hq_create): the
// direct sweep's per-order lists (format with HQ_SW_HI_BITS) and the batched sweep's
// list (format with HQ_ITEM_HI_BITS, hq_internal.cuh) with the positions of each
// state's low-part neighbours inside their rank blocks (device, at hq_create); and the
// FP32 / DF64 copies of the pull-form table (device, at hq_load).
#include <algorithm>
#include <vector>

#include "hq_internal.cuh"

namespace {

struct HostBinom {
  uint64_t c[33][33];
  HostBinom() {
    for (int n = 0; n <= 32; n++)
      for (int k = 0; k <= 32; k++) c[n][k] = k > n ? 0 : (uint64_t)hq_binom(n, k);
  }
};

// rank of the first state of block (hi, w): the high-part term of the split rank
uint64_t rank_hi(const HostBinom& B, int L, uint32_t hi, int w) {
  uint64_t r = 0;
  int k = 0;
  for (int b = 0; hi >> b; b++)
    if ((hi >> b) & 1u) {
      const int idx = w + k + 1;
      r += idx <= 32 ? B.c[L + b][idx] : 0;
      k++;
    }
  return r;
}

// Word q of state g holds bytes 4q..4q+3 of its low-part neighbour positions: byte k < w
// is RL[lo ^ 2^u] for the k-th busy unit u of lo (increasing), then byte w + k is
// RL[lo | 2^u] for the k-th idle unit u < L of lo (increasing).  RL[.] is the position of
// a state inside its rank block, so these index the staged blocks (hi, w -/+ 1).
__global__ void k_lidx(int L, int64_t Sp, const uint32_t* masks, const uint32_t* RL, uint32_t* lidx) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= Sp) return;
  const uint32_t lo = masks[g] & ((1u << L) - 1u);
  uint32_t wd[3] = {0u, 0u, 0u};
  int k = 0;
  for (int u = 0; u < L; u++)
    if ((lo >> u) & 1u) {
      wd[k >> 2] |= (RL[lo ^ (1u << u)] & 0xffu) << (8 * (k & 3));
      k++;
    }
  for (int u = 0; u < L; u++)
    if (!((lo >> u) & 1u)) {
      wd[k >> 2] |= (RL[lo | (1u << u)] & 0xffu) << (8 * (k & 3));
      k++;
    }
  for (int q = 0; q < 3; q++) lidx[(int64_t)q * Sp + g] = wd[q];
}

__global__ void k_table_conv(int64_t n, const double* T64, float2* Tdf) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Tdf[i] = df_from_double(T64[i]);
}

}  // namespace

int hq_item_list(int N, std::vector<uint4>& items, int* ifirst) {
  static const HostBinom B;
  const int L = N < HQ_LO_BITS ? N : HQ_LO_BITS, H = N - L;
  if (H > HQ_ITEM_HI_BITS) {
    hq_set_error("item builder: high part too wide");
    return HQ_EINVAL;
  }
  items.clear();
  for (int n = 0; n <= N; n++) {
    ifirst[n] = (int)items.size();
    if (n < 1 || n > N - 1) continue;
    uint64_t expect = 0;  // blocks come in increasing rank order, without gaps
    for (uint32_t hi = 0; hi < (1u << H); hi++) {
      const int w = n - __builtin_popcount(hi);
      if (w < 0 || w > L) continue;
      const uint64_t start = rank_hi(B, L, hi, w);
      const int size = (int)B.c[L][w];
      if (start != expect) {
        hq_set_error("item builder: rank blocks out of order");
        return HQ_ECUDA;
      }
      expect = start + (uint64_t)size;
      // layer 0 is the empty state (p_0 = 1, no (A, B) pairs): no block below layer 1
      const uint32_t dn = (w >= 1 && n >= 2) ? (uint32_t)rank_hi(B, L, hi, w - 1) : 0u;
      const uint32_t up = w < L ? (uint32_t)rank_hi(B, L, hi, w + 1) : 0u;
      for (int s0 = 0; s0 < size; s0 += 32) {
        const int c = size - s0 < 32 ? size - s0 : 32;
        items.push_back(make_uint4((uint32_t)(start + s0),
                                   hi | ((uint32_t)w << HQ_ITEM_HI_BITS) | ((uint32_t)(c - 1) << 24), dn, up));
      }
    }
    if (expect != (uint64_t)B.c[N][n]) {
      hq_set_error("item builder: rank blocks do not cover the layer");
      return HQ_ECUDA;
    }
  }
  ifirst[N + 1] = (int)items.size();
  for (int n = N + 2; n < HQ_MAXN + 2; n++) ifirst[n] = ifirst[N + 1];
  return HQ_OK;
}

// Items of the direct sweep (format with HQ_SW_HI_BITS in hq_internal.cuh) for one sweep
// order, phase by phase: HQ_ORDER_ASCENDING has one phase per layer 1..N-1;
// HQ_ORDER_REDBLACK has the odd layers' items, then the even layers' (one phase if
// N = 2).  Inside a phase, layers ascend and blocks come in rank order; blocks[] marks
// where each rank block's items start.
int hq_sweep_item_list(int N, int order, std::vector<uint2>& items, std::vector<int>& blocks, int* pbfirst,
                       int* nphases) {
  static const HostBinom B;
  const int L = N < HQ_LO_BITS ? N : HQ_LO_BITS, H = N - L;
  if (H > HQ_SW_HI_BITS) {
    hq_set_error("item builder: high part too wide");
    return HQ_EINVAL;
  }
  items.clear();
  blocks.clear();
  auto add_layer = [&](int n) {
    for (uint32_t hi = 0; hi < (1u << H); hi++) {
      const int w = n - __builtin_popcount(hi);
      if (w < 0 || w > L) continue;
      const uint64_t start = rank_hi(B, L, hi, w);
      const int size = (int)B.c[L][w];
      blocks.push_back((int)items.size());
      for (int s0 = 0; s0 < size; s0 += HQ_SW_ITEM) {
        const int c = size - s0 < HQ_SW_ITEM ? size - s0 : HQ_SW_ITEM;
        items.push_back(make_uint2(hi | ((uint32_t)w << HQ_SW_HI_BITS) | ((uint32_t)(c - 1) << (HQ_SW_HI_BITS + 4)),
                                   (uint32_t)(start + (uint64_t)s0) | ((uint32_t)n << 27)));
      }
    }
  };
  int np = 0;
  if (order == HQ_ORDER_ASCENDING) {
    for (int n = 1; n <= N - 1; n++) {
      pbfirst[np++] = (int)blocks.size();
      add_layer(n);
    }
  } else {
    for (int f = 1; f <= 2 && f <= N - 1; f++) {
      pbfirst[np++] = (int)blocks.size();
      for (int n = f; n <= N - 1; n += 2) add_layer(n);
    }
  }
  for (int i = np; i < HQ_MAXN + 2; i++) pbfirst[i] = (int)blocks.size();
  blocks.push_back((int)items.size());
  *nphases = np;
  return HQ_OK;
}

// Per phase, its rank blocks by decreasing cost (ties by index): the sweep deals them to
// the warps in snake order (round r goes warp 0..W-1 when r is even, W-1..0 when odd), which
// evens out the warps' totals.  A block's cost counts, per item, the loads of a lane
// (table record, all N neighbours, a few per-state values) plus a fixed set-up per block.
void hq_block_order(int N, const std::vector<uint2>& items, const std::vector<int>& blocks, const int* pbfirst,
                    int nphases, std::vector<int>& perm) {
  perm.resize(blocks.size() > 0 ? blocks.size() - 1 : 0);
  std::vector<double> cost(perm.size());
  for (size_t b = 0; b < perm.size(); b++) {
    const int ni = blocks[b + 1] - blocks[b];
    const int n = (int)(items[blocks[b]].y >> 27);
    cost[b] = 24.0 + (double)ni * (HQ_TW(n) + N + 8);
    perm[b] = (int)b;
  }
  for (int ph = 0; ph < nphases; ph++)
    std::stable_sort(perm.begin() + pbfirst[ph], perm.begin() + pbfirst[ph + 1],
                     [&](int x, int y) { return cost[x] > cost[y]; });
}

int hq_build_items(hq_solver* h) {
  for (int order = 0; order < 2; order++) {
    std::vector<uint2> si;
    std::vector<int> sb, perm;
    int rc = hq_sweep_item_list(h->N, order, si, sb, h->spbfirst[order], &h->snph[order]);
    if (rc != HQ_OK) return rc;
    hq_block_order(h->N, si, sb, h->spbfirst[order], h->snph[order], perm);
    const size_t bytes = sizeof(uint2) * (si.empty() ? 1 : si.size());
    const size_t bbytes = sizeof(int) * sb.size();
    const size_t pbytes = sizeof(int) * (perm.empty() ? 1 : perm.size());
    cudaError_t e = cudaMalloc((void**)&h->sitems[order], bytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->sblocks[order], bbytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->sperm[order], pbytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      hq_set_error("cudaMalloc of the sweep items failed");
      return HQ_ENOMEM;
    }
    h->dev_bytes += (int64_t)(bytes + bbytes + pbytes);
    if (!si.empty())
      HQ_CUDA(cudaMemcpyAsync(h->sitems[order], si.data(), bytes, cudaMemcpyHostToDevice, h->stream));
    HQ_CUDA(cudaMemcpyAsync(h->sblocks[order], sb.data(), bbytes, cudaMemcpyHostToDevice, h->stream));
    if (!perm.empty())
      HQ_CUDA(cudaMemcpyAsync(h->sperm[order], perm.data(), pbytes, cudaMemcpyHostToDevice, h->stream));
    HQ_CUDA(cudaStreamSynchronize(h->stream));  // the host vectors go out of scope
  }
  if (h->N > HQ_DF_MAXN) return HQ_OK;  // the batched kernel's lists: not kept above HQ_DF_MAXN
  std::vector<uint4> items;
  const int rc = hq_item_list(h->N, items, h->ifirst);
  if (rc != HQ_OK) return rc;
  const size_t bytes = sizeof(uint4) * (items.empty() ? 1 : items.size());
  cudaError_t e = cudaMalloc((void**)&h->items, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    hq_set_error("cudaMalloc of the sweep items failed");
    return HQ_ENOMEM;
  }
  h->dev_bytes += (int64_t)bytes;
  if (!items.empty())
    HQ_CUDA(cudaMemcpyAsync(h->items, items.data(), bytes, cudaMemcpyHostToDevice, h->stream));
  HQ_CUDA(cudaStreamSynchronize(h->stream));  // the host vector goes out of scope
  k_lidx<<<(unsigned)((h->Sp + 255) / 256), 256, 0, h->stream>>>(h->L, h->Sp, h->masks, h->RL, h->lidx);
  HQ_LAUNCHED();
  return HQ_OK;
}

int hq_ensure_df(hq_solver* h) {
  if (h->df_ready || !h->bdf.T) return HQ_OK;
  const int64_t n = h->tentries;
  if (n > 0) {
    k_table_conv<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(n, (const double*)h->b64.T,
                                                                      (float2*)h->bdf.T);
    HQ_LAUNCHED();
  }
  h->df_ready = true;
  return HQ_OK;
}

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
//     rho0_m = c1^0 A0_m + c2^0 B0_m - p0_n(m).
// Every term on the right is of the size of the correction, so FP32 arithmetic on the
// correction loses about 1e-7 of |e| rather than of |p|.  The layer sums that the
// closed form reads are the base's (FP64, once per base) plus the correction's (FP32
// partials of the sweep, folded in FP64).  Any c^0 splits the update exactly; the base
// takes the closed-form scalars of p0's own layer sums.
//
// This file: setting up a base (its layer sums, its scalars c^0 and the base pass that
// stores rho0, A0, B0 per state, in hq_persist.cu), re-basing (p0 += e) and the assembly
// of p0 + e for the residual and the outputs.  The correction sweeps themselves are the
// persistent sweep kernel in its correction mode (hq_persist.cu).
#include <string.h>

#include "hq_internal.cuh"

namespace {

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
  int rc = hq_iter_sums(h, HQ_PREC_FP64, h->ir_base, &h->sc->ir_sum[0][0]);
  if (rc != HQ_OK) return rc;
  rc = hq_base_pass(h);
  if (rc != HQ_OK) return rc;
  // e = 0 everywhere (the empty and the full state have no correction), so the layer
  // sums of p0 + e are the base's
  HQ_CUDA(cudaMemsetAsync(h->b32.p, 0, sizeof(float) * Sp, h->stream));
  HQ_CUDA(cudaMemcpyAsync(&h->sc->ls[0][0], &h->sc->ir_sum[0][0], sizeof(h->sc->ls), cudaMemcpyDeviceToDevice,
                          h->stream));
  h->cur_prec = HQ_PREC_IRC;
  return HQ_OK;
}

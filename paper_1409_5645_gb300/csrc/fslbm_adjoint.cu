// fslbm_adjoint.cu -- hand-written adjoint of the FSLBM step and the
// checkpointed reverse sweep behind fslbm_adjoint_forward / _backward.
//
// The forward step maps the stored state (f~(t), m(t), phi(t)) to
// (f~(t+1), m(t+1), phi(t+1)) for fixed cell flags.  Its adjoint is taken in
// two kernels per step:
//   k_adj_local   per fluid cell x: recompute the cell's forward step (pull,
//                 wall and free-surface closures, mass exchange, collision),
//                 then reverse it.  Writes the adjoint of the populations the
//                 cell read from itself ("own", O) and of the populations it
//                 pulled from its neighbours (P), the adjoint of m(t), and
//                 adds adjoints of phi(t) of itself and of the neighbours it
//                 read (mass-exchange weights, height functions) with atomics.
//   k_adj_gather  reverse of the pull: abar_q(y) = O_q(y) + P_q(y + c_q).
// Parameters: lambda_+, lambda_- (-> nu with Lambda fixed) and g, reduced per
// block.  Interface decisions (flags, the height-function/plane-fit branch,
// the dominant axis, clamps of delta) are held fixed; a clamped delta passes
// no derivative.  delta = d / (n.c_p) is differentiated through the heights
// where the height columns are closed, and through the plane fit elsewhere:
// the volume identity V(n, d) = phi (the section's area and centroid) and
// the Parker-Youngs normal of the fill levels around the cell.
// Cell conversions are replayed as the forward pass took them: the flags of
// every step are recorded (in the checkpoints and in the recomputed segment),
// and two kernels per step reverse the conversion stage before k_adj_local
// reverses the rest of the step:
//   k_adj_conv1   per cell of the new state: the adjoint of the final mass
//                 (m_bar + phi_bar / rho) and of the density (from phi =
//                 m / rho) of every interface cell; per new cell from gas the
//                 reverse of its collided equilibrium f^eq(mean rho, mean u)
//                 down to the means of its fluid neighbours
//   k_adj_conv2   per fluid cell of the old state: the adjoint of its
//                 post-collision populations and mass before the
//                 conversions: the excess of a filled (m - rho) or emptied
//                 (m) cell gathers its receivers' mass adjoints over their
//                 number (equal split), a new cell from liquid passes its mass
//                 adjoint to rho, the new cells' means to their neighbours.
// The receivers of a step are the cells that are interface after it, so the
// two recorded flag fields decide every branch.
// Supported: rho_0 = 1, sigma = 0, equal excess split.
//
// This file holds the host entry points and the cell-list kernel; the
// reverse step's kernels and the sweep are templates in fslbm_adjoint.cuh,
// instantiated per precision form in fslbm_adjoint_p64/p32/p16.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "fslbm_adjoint.h"

using namespace fsl;

namespace fsl {

// The liquid and the interface cells of a flag field, in two lists
// (warp-aggregated appends; the order does not matter: each cell's reverse
// step is its own).  The adjoint kernels run over them only: the entries of
// other cells are never read.
__device__ __forceinline__ void list_append(bool pred, int i, int* list, int* count) {
  const unsigned bal = __ballot_sync(0xffffffffu, pred);
  if (!bal) return;
  const int lane = threadIdx.x & 31, leader = __ffs(bal) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(count, __popc(bal));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (pred) list[base + __popc(bal & ((1u << lane) - 1u))] = i;
}
__global__ void __launch_bounds__(256) k_adj_lists(Par p, const uint8_t* __restrict__ flags, int* __restrict__ liq,
                                                   int* __restrict__ ifc, int* __restrict__ count) {
  for (long long i0 = blockIdx.x * (long long)blockDim.x; i0 < p.N; i0 += (long long)gridDim.x * blockDim.x) {
    const long long i = i0 + threadIdx.x;
    const uint8_t k = i < p.N ? (flags[i] & KIND) : (uint8_t)GAS;
    list_append(k == LIQ, (int)i, liq, count);
    list_append(k == IFC, (int)i, ifc, count + 1);
  }
}

void build_lists(const Par& p, const uint8_t* flags, const CellLists& L, cudaStream_t st) {
  int blocks = (int)((p.N + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  cudaMemsetAsync(L.cnt, 0, 2 * sizeof(int), st);
  k_adj_lists<<<blocks, 256, 0, st>>>(p, flags, L.liq, L.ifc, L.cnt);
}

}  // namespace fsl


// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
static int adj_fail(fslbm* h, int code, const char* what) {
  snprintf(h->msg, sizeof h->msg, "%s", what);
  return code;
}

void fslbm_free_adjoint(fslbm* h) {
  if (!h || !h->adj) return;
  AdjointState* A = h->adj;
  void* ptrs[] = {A->ck_f, A->ck_m, A->ck_phi, A->ck_flags, A->seg_f, A->seg_m, A->seg_phi, A->seg_flags,
                  A->Mh, A->rh, A->ngb, A->flist, A->abar[0], A->abar[1], A->P, A->mbar[0], A->mbar[1], A->phibar[0],
                  A->phibar[1], A->theta, A->red, A->dphi0};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete A;
  h->adj = nullptr;
}

static bool amalloc(AdjointState* A, void** p, size_t bytes) {
  if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
    *p = nullptr;
    return false;
  }
  A->bytes += bytes;
  return true;
}

int save_state(fslbm* h, void* f, double* m, void* phi, uint8_t* flags) {
  AdjointState* A = h->adj;
  if (cudaMemcpyAsync(flags, h->flags, (size_t)h->par.N, cudaMemcpyDeviceToDevice, h->st) != cudaSuccess) return 1;
  if (cudaMemcpyAsync(f, cur_f(h), A->fbytes, cudaMemcpyDeviceToDevice, h->st) != cudaSuccess) return 1;
  if (cudaMemcpyAsync(m, h->m, (size_t)h->par.N * 8, cudaMemcpyDeviceToDevice, h->st) != cudaSuccess) return 1;
  if (cudaMemcpyAsync(phi, cur_phi(h), A->rbytes, cudaMemcpyDeviceToDevice, h->st) != cudaSuccess) return 1;
  return 0;
}

int restore_state(fslbm* h, const void* f, const double* m, const void* phi, const uint8_t* flags) {
  AdjointState* A = h->adj;
  h->cur = 0;
  if (cudaMemcpyAsync(h->flags, flags, (size_t)h->par.N, cudaMemcpyDeviceToDevice, h->st) != cudaSuccess) return 1;
  if (cudaMemcpyAsync(h->fA, f, A->fbytes, cudaMemcpyDeviceToDevice, h->st) != cudaSuccess) return 1;
  if (cudaMemcpyAsync(h->m, m, (size_t)h->par.N * 8, cudaMemcpyDeviceToDevice, h->st) != cudaSuccess) return 1;
  if (cudaMemcpyAsync(h->phiA, phi, A->rbytes, cudaMemcpyDeviceToDevice, h->st) != cudaSuccess) return 1;
  return 0;
}

extern "C" int fslbm_adjoint_forward(fslbm_t* h, int nsteps, int K, int objective, double* J) {
  if (!h || nsteps < 1 || K < 1 || (objective != 0 && objective != 1)) return FSLBM_ERR_ARG;
  if (h->par.compressible) return adj_fail(h, FSLBM_ERR_ARG, "adjoint needs rho_0 = 1");
  if (h->par.sigma != 0.0) return adj_fail(h, FSLBM_ERR_ARG, "adjoint needs sigma = 0");
  if (h->par.stress) return adj_fail(h, FSLBM_ERR_ARG, "adjoint needs D = 0 (no boundary shear term)");
  if (h->par.has_uw) return adj_fail(h, FSLBM_ERR_ARG, "adjoint needs resting walls");
  if (h->par.ub_extrap) return adj_fail(h, FSLBM_ERR_ARG, "adjoint needs u_b = u(x_b) (ub_extrap = 0)");
  if (h->par.recon_nc) return adj_fail(h, FSLBM_ERR_ARG, "adjoint needs the gas links only (recon_nc = 0)");
  if (h->par.excess_split) return adj_fail(h, FSLBM_ERR_ARG, "adjoint needs the equal excess split");
  if (h->par.elvira) return adj_fail(h, FSLBM_ERR_ARG, "adjoint needs the Parker-Youngs plane fit (elvira = 0)");
  fslbm_free_adjoint(h);
  AdjointState* A = new AdjointState();
  h->adj = A;
  const size_t N = (size_t)h->par.N;
  A->nsteps = nsteps;
  A->K = K;
  A->objective = objective;
  A->nck = (nsteps + K - 1) / K;
  const size_t sb = h->prec == FSLBM_F64 ? 8 : (h->prec == FSLBM_F32 ? 4 : 2);
  A->fbytes = 19 * N * sb;
  A->rbytes = N * (h->prec == FSLBM_F64 ? 8 : 4);
  bool ok = amalloc(A, &A->ck_f, A->fbytes * A->nck) && amalloc(A, (void**)&A->ck_m, N * 8 * A->nck) &&
            amalloc(A, &A->ck_phi, A->rbytes * A->nck) && amalloc(A, (void**)&A->ck_flags, N * A->nck) &&
            amalloc(A, (void**)&A->red, 64);
  if (!ok) {
    fslbm_free_adjoint(h);
    return adj_fail(h, FSLBM_ERR_OOM, "adjoint checkpoint allocation");
  }
  int c[16];
  cudaMemcpy(c, h->cnt, sizeof c, cudaMemcpyDeviceToHost);
  A->conv0 = c[8];
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, h->st);
  for (int s = 0; s < A->nck; ++s) {
    if (save_state(h, (char*)A->ck_f + s * A->fbytes, A->ck_m + s * N, (char*)A->ck_phi + s * A->rbytes,
                   A->ck_flags + s * N))
      return adj_fail(h, FSLBM_ERR_CUDA, "checkpoint copy");
    int n = nsteps - s * K < K ? nsteps - s * K : K;
    int rc = fslbm_step(h, n);
    if (rc) return rc;
  }
  cudaEventRecord(e1, h->st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  A->fwd_ms = ms / nsteps;
  int rc = fslbm_sync(h);
  if (rc) return rc;
  cudaMemcpy(c, h->cnt, sizeof c, cudaMemcpyDeviceToHost);
  A->conversions = c[8] - A->conv0;
  double norm = 0.0;
  int orc;
  switch (h->prec) {
    case FSLBM_F64: orc = adj_objective<P64>(h, &A->J, &norm); break;
    case FSLBM_F32: orc = adj_objective<P32>(h, &A->J, &norm); break;
    default: orc = adj_objective<P16>(h, &A->J, &norm); break;
  }
  if (orc) return adj_fail(h, FSLBM_ERR_CUDA, "objective");
  A->ready = true;
  if (J) *J = A->J;
  return FSLBM_OK;
}

extern "C" int fslbm_adjoint_backward(fslbm_t* h, double* dJ_dnu, double dJ_dg[3], double* dJ_dphi0, int where) {
  if (!h) return FSLBM_ERR_ARG;
  AdjointState* A = h->adj;
  if (!A || !A->ready) return adj_fail(h, FSLBM_ERR_ARG, "fslbm_adjoint_forward has not run");
  const size_t N = (size_t)h->par.N;
  if (!A->abar[0]) {
    bool ok = amalloc(A, (void**)&A->abar[0], 19 * N * 8) && amalloc(A, (void**)&A->abar[1], 19 * N * 8) &&
              amalloc(A, (void**)&A->P, 19 * N * 8) && amalloc(A, (void**)&A->mbar[0], N * 8) &&
              amalloc(A, (void**)&A->mbar[1], N * 8) && amalloc(A, (void**)&A->phibar[0], N * 8) &&
              amalloc(A, (void**)&A->phibar[1], N * 8) && amalloc(A, (void**)&A->theta, 64) &&
              amalloc(A, (void**)&A->dphi0, N * 8) && amalloc(A, &A->seg_f, A->fbytes * (A->K + 1)) &&
              amalloc(A, (void**)&A->seg_m, N * 8 * (A->K + 1)) &&
              amalloc(A, &A->seg_phi, A->rbytes * (A->K + 1)) &&
              amalloc(A, (void**)&A->seg_flags, N * (A->K + 1)) && amalloc(A, (void**)&A->Mh, N * 8) &&
              amalloc(A, (void**)&A->flist, 2 * (2 * N + 2) * sizeof(int)) &&
              amalloc(A, (void**)&A->rh, N * 8) && amalloc(A, (void**)&A->ngb, N * 4 * 8);
    if (!ok) return adj_fail(h, FSLBM_ERR_OOM, "adjoint buffer allocation");
  }
  int r;
  switch (h->prec) {
    case FSLBM_F64: r = adj_backward<P64>(h); break;
    case FSLBM_F32: r = adj_backward<P32>(h); break;
    default: r = adj_backward<P16>(h); break;
  }
  if (r) return adj_fail(h, FSLBM_ERR_CUDA, "adjoint sweep");
  double th[8];
  if (cudaMemcpyAsync(th, A->theta, sizeof th, cudaMemcpyDeviceToHost, h->st) != cudaSuccess)
    return adj_fail(h, FSLBM_ERR_CUDA, "D2H theta");
  if (cudaStreamSynchronize(h->st) != cudaSuccess) return adj_fail(h, FSLBM_ERR_CUDA, "sync");
  // nu = (tau - 1/2)/3; lambda_+ = -1/tau; lambda_- from Lambda fixed
  const double tau = h->prm.tau;
  const double dlp_dtau = 1.0 / (tau * tau);
  double dlm_dtau;
  if (h->prm.magic <= 0.0) {
    dlm_dtau = dlp_dtau;
  } else {
    const double Lp = tau - 0.5, Lm = h->prm.magic / Lp;
    dlm_dtau = (1.0 / ((Lm + 0.5) * (Lm + 0.5))) * (-h->prm.magic / (Lp * Lp));
  }
  if (dJ_dnu) *dJ_dnu = 3.0 * (th[0] * dlp_dtau + th[1] * dlm_dtau);
  if (dJ_dg) {
    dJ_dg[0] = th[2] + A->gseed;
    dJ_dg[1] = th[3];
    dJ_dg[2] = th[4];
  }
  if (dJ_dphi0) {
    cudaMemcpyKind kind = where == FSLBM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (cudaMemcpyAsync(dJ_dphi0, A->dphi0, N * 8, kind, h->st) != cudaSuccess)
      return adj_fail(h, FSLBM_ERR_CUDA, "copy dJ/dphi0");
  }
  return fslbm_sync(h);
}

extern "C" int fslbm_adjoint_stats(fslbm_t* h, double* fwd_ms_per_step, double* adj_ms_per_step,
                                   size_t* peak_bytes) {
  if (!h || !h->adj) return FSLBM_ERR_ARG;
  if (fwd_ms_per_step) *fwd_ms_per_step = h->adj->fwd_ms;
  if (adj_ms_per_step) *adj_ms_per_step = h->adj->adj_ms;
  if (peak_bytes) *peak_bytes = h->adj->bytes + h->bytes;
  return FSLBM_OK;
}

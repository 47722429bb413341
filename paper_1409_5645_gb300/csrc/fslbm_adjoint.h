// fslbm_adjoint.h -- the state of a checkpointed reverse sweep and what the
// adjoint's translation units share: the host entry points (fslbm_adjoint.cu)
// and the reverse step's kernels, instantiated per precision form
// (fslbm_adjoint_p64/p32/p16.cu from fslbm_adjoint.cuh).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fslbm.h"
#include "fslbm_dev.cuh"
#include "fslbm_handle.h"
#include "fslbm_kernels.h"


struct AdjointState {
  int nsteps = 0, K = 1, objective = 0, nck = 0;
  size_t fbytes = 0, rbytes = 0;
  void* ck_f = nullptr;
  double* ck_m = nullptr;
  void* ck_phi = nullptr;
  uint8_t* ck_flags = nullptr;
  void* seg_f = nullptr;  // K + 1 states of the segment being reversed
  double* seg_m = nullptr;
  void* seg_phi = nullptr;
  uint8_t* seg_flags = nullptr;
  int* flist = nullptr;  // [2][2N + 2]: liquid and interface cells of a flag field, their counts
                         // (double buffer: the fields before and after the step being reversed)
  double* Mh = nullptr;  // conversion reverse: final-mass and density adjoints, new-cell means
  double* rh = nullptr;
  double* ngb = nullptr;
  double* abar[2] = {nullptr, nullptr};
  double* P = nullptr;
  double* mbar[2] = {nullptr, nullptr};
  double* phibar[2] = {nullptr, nullptr};
  double* theta = nullptr;  // [0] lambda_+ [1] lambda_- [2..4] g
  double* red = nullptr;    // objective reductions
  double* dphi0 = nullptr;
  int conv0 = 0;
  long long conversions = 0;  // cell conversions inside the window
  double J = 0.0, gseed = 0.0;
  double fwd_ms = 0.0, adj_ms = 0.0;
  size_t bytes = 0;
  bool ready = false;
};

namespace fsl {

// the liquid and interface cells of a flag field (see k_adj_lists)
struct CellLists {
  int* liq;
  int* ifc;
  int* cnt;  // [0] liquid, [1] interface
};
void build_lists(const Par& p, const uint8_t* flags, const CellLists& L, cudaStream_t st);
}  // namespace fsl

// the handle's current populations and fill levels
inline void* cur_f(fslbm* h) { return h->cur ? h->fB : h->fA; }
inline void* cur_phi(fslbm* h) { return (h->par.freeze || !h->cur) ? h->phiA : h->phiB; }
// copies of the handle's state to and from a checkpoint (device to device, on the handle's stream)
int save_state(fslbm* h, void* f, double* m, void* phi, uint8_t* flags);
int restore_state(fslbm* h, const void* f, const double* m, const void* phi, const uint8_t* flags);
// the objective at the current state (J, its normalisation; sets the seed of dJ/dg_x)
template <int P>
int adj_objective(fslbm* h, double* J, double* norm);
// the reverse sweep over the recorded window (fslbm_adjoint_backward)
template <int P>
int adj_backward(fslbm* h);

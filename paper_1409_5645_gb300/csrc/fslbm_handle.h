// fslbm_handle.h -- the handle behind the opaque fslbm_t of the C interface
// (shared by the host translation units of the library).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <vector>

#include "fslbm.h"
#include "fslbm_dev.cuh"
#include "fslbm_kernels.h"

struct AdjointState;
struct fslbm;
void fslbm_free_adjoint(fslbm* h);

struct fslbm {
  fslbm_params prm;
  fsl::Par par;
  int prec;
  cudaStream_t st;
  uint8_t* flags;
  uint8_t* mark;
  void* fA;
  void* fB;
  double* m;
  void* phiA;
  void* phiB;
  double* wd;
  int* lists[6];
  int* seglist;  // 32-cell x segments holding fluid: int4 records, then uint4 masks (rebuilt every step)
  int* cnt;
  double* share;
  void* geo;  // interface geometry scratch [5][cap] in the arithmetic type
  double* partials;
  long long nparts;
  int bulk_blocks, iface_blocks, list_blocks, red_blocks;
  int coop_blocks;  // blocks of the fused cooperative conversion kernel (0: four launches)
  double* red;
  double* lost;
  int* err;
  double* step_mass;
  double* total_out;
  int cur;
  long long t;
  int cap;
  size_t bytes;
  char msg[256];
  int timing;
  std::vector<cudaEvent_t>* events;  // 5 per timed step
  long long timed_steps;
  AdjointState* adj;  // checkpoints and buffers of a differentiation, or NULL
  double* f0;         // FP64 pre-collision initial populations (keep_f0), or NULL
  int f0_valid;       // f0 holds the populations of the current initial state
  int bulk_mode;      // fsl::BulkMode of the bulk kernel
  CUtensorMap* tmap;  // [2] tensor maps of fA and fB for the TMA bulk kernel (64-byte aligned), or NULL
  fsl::Fork fork;     // the side stream of the interface kernels and its two events
  int forked;         // fork holds a stream and events
  int overlap;        // 1: the interface kernels run on the side stream beside the bulk kernel
};


template <int P>
inline fsl::View<P> make_view(fslbm* h) {
  using namespace fsl;

  View<P> v;
  using S = typename Form<P>::S;
  using R = typename Form<P>::R;
  v.flags = h->flags;
  v.mark = h->mark;
  v.fin = (const S*)(h->cur ? h->fB : h->fA);
  v.fout = (S*)(h->cur ? h->fA : h->fB);
  v.m = h->m;
  if (h->par.freeze) {
    v.phin = (const R*)h->phiA;
    v.phout = (R*)h->phiA;
  } else {
    v.phin = (const R*)(h->cur ? h->phiB : h->phiA);
    v.phout = (R*)(h->cur ? h->phiA : h->phiB);
  }
  v.wd = (const double*)h->wd;
  v.ilist = h->lists[0];
  v.flist = h->lists[1];
  v.elist = h->lists[2];
  v.nglist = h->lists[3];
  v.nllist = h->lists[4];
  v.rlist = h->lists[5];
  v.cnt = h->cnt;
  v.cap = h->cap;
  v.share = h->share;
  v.geo = (R*)h->geo;
  v.partials = h->partials;
  v.lost = h->lost;
  v.err = h->err;
  return v;
}


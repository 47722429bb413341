// fslbm_api.cu -- host side of the C interface declared in include/fslbm.h.
//
// A handle owns every device buffer of one lattice.  fslbm_step enqueues, per
// time step and with no host synchronisation:
//   memset(counters) -> k_segments -> k_bulk -> k_iface -> mass reduction
//   (2 kernels) -> 7 conversion kernels (dynamic interface only)
// and swaps the A/B population and fill-level buffers.
#include <cuda_runtime.h>
#include <stdio.h>
#include <vector>
#include <stdlib.h>
#include <string.h>

#include "fslbm.h"
#include "fslbm_dev.cuh"
#include "fslbm_handle.h"
#include "fslbm_kernels.h"

using namespace fsl;

static const char* k_ok = "no error";

static int fail(fslbm* h, int code, const char* what, cudaError_t e = cudaSuccess) {
  if (h) {
    if (e != cudaSuccess) snprintf(h->msg, sizeof h->msg, "%s: %s", what, cudaGetErrorString(e));
    else snprintf(h->msg, sizeof h->msg, "%s", what);
  }
  return code;
}

#define CK(call, what)                                    \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return fail(h, FSLBM_ERR_CUDA, what, e_); \
  } while (0)

// magic numbers of fsl::fdiv for the divisor d >= 1 (d < 2^31)
static FDiv make_fdiv(unsigned d) {
  int l = 0;
  while ((1ull << l) < d) ++l;
  const unsigned long long m = ((1ull << 32) * ((1ull << l) - d)) / d + 1;
  FDiv f;
  f.m = (unsigned)m;
  f.s1 = l < 1 ? l : 1;
  f.s2 = l > 1 ? l - 1 : 0;
  return f;
}

static size_t store_bytes(int prec) { return prec == FSLBM_F64 ? 8 : (prec == FSLBM_F32 ? 4 : 2); }
static size_t real_bytes(int prec) { return prec == FSLBM_F64 ? 8 : 4; }

static void drop_events(fslbm* h) {
  if (!h->events) return;
  for (cudaEvent_t e : *h->events) cudaEventDestroy(e);
  delete h->events;
  h->events = nullptr;
}

static void free_all(fslbm* h) {
  drop_events(h);
  if (h->forked) {
    cudaEventDestroy(h->fork.fork);
    cudaEventDestroy(h->fork.join);
    cudaStreamDestroy(h->fork.side);
    h->forked = 0;
  }
  void* ptrs[] = {h->flags, h->mark, h->fA, h->fB, h->m, h->phiA, h->phiB, h->wd, h->cnt, h->share, h->geo,
                  h->partials, h->red, h->lost, h->err, h->step_mass, h->total_out, h->f0, h->seglist};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (int k = 0; k < 6; ++k)
    if (h->lists[k]) cudaFree(h->lists[k]);
  free(h->tmap);
  h->tmap = nullptr;
}

template <class T>
static bool dalloc(fslbm* h, T** p, size_t bytes) {
  if (cudaMalloc((void**)p, bytes ? bytes : 16) != cudaSuccess) {
    *p = nullptr;
    return false;
  }
  h->bytes += bytes;
  return true;
}

extern "C" void fslbm_default_params(fslbm_params* p) {
  if (!p) return;
  memset(p, 0, sizeof *p);
  p->tau = 0.8;
  p->magic = 3.0 / 16.0;
  p->rho_G = 1.0;
  p->rule = FSLBM_FSL;
  p->eps = 1e-3;
  p->delta_min = 0.0;
  p->cleanup = 3;
  p->keep_f0 = 0;
  p->precision = FSLBM_F64;
  p->u_max = 0.4;
}

extern "C" int fslbm_create_ex(const fslbm_params* prm, fslbm_t** out) {
  if (!prm || !out) return FSLBM_ERR_ARG;
  *out = nullptr;
  const fslbm_params& q = *prm;
  if (q.dims[0] <= 0 || q.dims[1] <= 0 || q.dims[2] <= 0) return FSLBM_ERR_ARG;
  if (!(q.tau > 0.5) || !(q.eps >= 0.0) || q.rule < 0 || q.rule > 1) return FSLBM_ERR_ARG;
  if (q.precision < FSLBM_F64 || q.precision > FSLBM_F16) return FSLBM_ERR_ARG;
  if (q.rule == FSLBM_FSL && fabs(1.0 - q.tau) < 1e-3) return FSLBM_ERR_ARG;
  long long N = (long long)q.dims[0] * q.dims[1] * q.dims[2];
  if (N >= (1LL << 31)) return FSLBM_ERR_ARG;
  if (q.precision == FSLBM_F16 && q.compressible) return FSLBM_ERR_ARG;
  if (q.bulk_loads < FSLBM_LOADS_PLAIN || q.bulk_loads > FSLBM_LOADS_PAIRS) return FSLBM_ERR_ARG;
  if (q.stress < 0 || q.stress > 2) return FSLBM_ERR_ARG;
  if (q.ub_extrap < 0 || q.ub_extrap > 1) return FSLBM_ERR_ARG;
  if (q.recon_nc < 0 || q.recon_nc > 1) return FSLBM_ERR_ARG;
  if (q.excess_split < 0 || q.excess_split > 1) return FSLBM_ERR_ARG;
  if (q.elvira < 0 || q.elvira > 1) return FSLBM_ERR_ARG;
  if (q.adjoint_fp32 < 0 || q.adjoint_fp32 > 1) return FSLBM_ERR_ARG;
  if (!(q.u_max >= 0.0)) return FSLBM_ERR_ARG;
  if (q.compressible && (q.wall_u[0] != 0.0 || q.wall_u[1] != 0.0 || q.wall_u[2] != 0.0)) return FSLBM_ERR_ARG;

  fslbm* h = (fslbm*)calloc(1, sizeof(fslbm));
  if (!h) return FSLBM_ERR_OOM;
  h->prm = q;
  h->prec = q.precision;
  h->st = (cudaStream_t)q.stream;
  strcpy(h->msg, k_ok);
  Par& p = h->par;
  p.nx = q.dims[0]; p.ny = q.dims[1]; p.nz = q.dims[2];
  p.dnx = make_fdiv((unsigned)p.nx);
  p.dny = make_fdiv((unsigned)p.ny);
  p.dnxy = make_fdiv((unsigned)(p.nx * p.ny));
  p.dnsx = make_fdiv((unsigned)((p.nx + 31) / 32));
  p.N = N;
  p.px = q.periodic[0] != 0; p.py = q.periodic[1] != 0; p.pz = q.periodic[2] != 0;
  p.zshift = q.zshift;
  // lambda_+ = -1/tau; Lambda_+ = tau - 1/2; Lambda_- = Lambda / Lambda_+;
  // lambda_- = -1/(Lambda_- + 1/2) (Sec. 2.1, Sec. 3.1)
  p.lam_p = -1.0 / q.tau;
  if (q.magic <= 0.0) {
    p.lam_m = p.lam_p;
  } else {
    double Lp = -(0.5 + 1.0 / p.lam_p);
    double Lm = q.magic / Lp;
    p.lam_m = -1.0 / (Lm + 0.5);
  }
  p.inv_1plp = 1.0 / (1.0 + p.lam_p);
  p.inv_lam_m = 1.0 / p.lam_m;
  for (int a = 0; a < 3; ++a) p.g[a] = q.g[a];
  p.rho_G = q.rho_G;
  p.sigma = q.sigma;
  p.eps = q.eps;
  p.delta_min = q.delta_min;
  p.rule = q.rule;
  p.compressible = q.compressible != 0;
  p.linear_eq = q.linear_eq != 0;
  p.freeze = q.freeze != 0;
  p.cleanup = q.cleanup;
  p.stress = q.stress;
  p.tau_m_half = q.tau - 0.5;
  for (int k = 0; k < 6; ++k) p.shear_b[k] = q.shear_b[k];
  for (int a = 0; a < 3; ++a) p.wall_u[a] = q.wall_u[a];
  p.has_uw = (q.wall_u[0] != 0.0 || q.wall_u[1] != 0.0 || q.wall_u[2] != 0.0) ? 1 : 0;
  p.has_wd = 0;
  p.ub_extrap = q.ub_extrap;
  p.recon_nc = q.recon_nc;
  p.excess_split = q.excess_split;
  for (int a = 0; a < 3; ++a) {
    p.own_lo[a] = 0;
    p.own_hi[a] = q.dims[a];
  }
  p.owned_all = 1;
  p.elvira = q.elvira;
  p.adj32 = q.adjoint_fp32 && q.precision != FSLBM_F64;
  p.umax2 = q.u_max * q.u_max;

  const size_t Nn = (size_t)N, N4 = (Nn + 3) & ~(size_t)3;
  h->cap = (int)N;
  // 32-cell segments; the bulk kernel runs one resident wave of warps
  const long long nseg = ((p.nx + 31) / 32) * (long long)p.ny * p.nz;
  h->bulk_blocks = 152 * (h->prec == FSLBM_F64 ? 4 : 8);
  h->iface_blocks = 152 * 16;  // one thread per interface cell up to 311 296 cells per round
  h->list_blocks = 152 * 8;  // 8 warps each: one warp per listed cell, 9728 cells per round
  {
    // the four conversion stages as one cooperative launch, two resident
    // blocks per SM, where the device allows it; else four launches
    int dev = 0, coop = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int per_sm = h->prec == FSLBM_F64   ? convert_blocks_per_sm<P64>()
                       : h->prec == FSLBM_F32 ? convert_blocks_per_sm<P32>()
                                              : convert_blocks_per_sm<P16>();
    h->coop_blocks = (coop && per_sm > 0 && sms > 0) ? sms * (per_sm < 2 ? per_sm : 2) : 0;
  }
  h->red_blocks = 152;
  h->nparts = (h->bulk_blocks + h->iface_blocks) * 4;  // one partial per bulk and per interface warp
  if (h->nparts < 4096) h->nparts = 4096;
  bool ok = dalloc(h, &h->flags, N4) && dalloc(h, &h->mark, N4) &&
            dalloc(h, (char**)&h->fA, 19 * Nn * store_bytes(h->prec) + 16) &&
            dalloc(h, (char**)&h->fB, 19 * Nn * store_bytes(h->prec) + 16) && dalloc(h, &h->m, Nn * 8) &&
            dalloc(h, (char**)&h->phiA, Nn * real_bytes(h->prec)) &&
            dalloc(h, (char**)&h->phiB, Nn * real_bytes(h->prec)) && dalloc(h, &h->cnt, 16 * sizeof(int)) &&
            dalloc(h, &h->share, Nn * 8) && dalloc(h, (char**)&h->geo, 5 * Nn * real_bytes(h->prec)) &&
            dalloc(h, &h->partials, (size_t)h->nparts * 8) &&
            dalloc(h, &h->red, (size_t)(h->red_blocks + 2) * 8) && dalloc(h, &h->lost, 8) &&
            dalloc(h, &h->err, 8) && dalloc(h, &h->step_mass, 8) && dalloc(h, &h->total_out, 8);
  for (int k = 0; k < 6 && ok; ++k) ok = dalloc(h, &h->lists[k], Nn * sizeof(int));
  if (ok && q.keep_f0) ok = dalloc(h, &h->f0, 19 * Nn * 8);
  if (ok) ok = dalloc(h, &h->seglist, (size_t)nseg * 8 * sizeof(int));  // record and masks per segment
  if (!ok) {
    free_all(h);
    free(h);
    return FSLBM_ERR_OOM;
  }
#ifdef FSLBM_CHECKED
  p.err = h->err;
#endif
  cudaMemsetAsync(h->flags, GAS, N4, h->st);
  cudaMemsetAsync(h->mark, 0, N4, h->st);
  cudaMemsetAsync(h->fA, 0, 19 * Nn * store_bytes(h->prec), h->st);
  cudaMemsetAsync(h->fB, 0, 19 * Nn * store_bytes(h->prec), h->st);
  cudaMemsetAsync(h->m, 0, Nn * 8, h->st);
  cudaMemsetAsync(h->phiA, 0, Nn * real_bytes(h->prec), h->st);
  cudaMemsetAsync(h->phiB, 0, Nn * real_bytes(h->prec), h->st);
  cudaMemsetAsync(h->cnt, 0, 16 * sizeof(int), h->st);
  cudaMemsetAsync(h->lost, 0, 8, h->st);
  cudaMemsetAsync(h->err, 0, 8, h->st);
  cudaMemsetAsync(h->step_mass, 0, 8, h->st);
  // loads of the bulk kernel: staged ones only for FP32/FP16 (FP64 is bound by its arithmetic)
  h->bulk_mode = BULK_PLAIN;
  if (h->prec != FSLBM_F64 && q.bulk_loads == FSLBM_LOADS_ASYNC) h->bulk_mode = BULK_ASYNC;
  if (h->prec != FSLBM_F64 && q.bulk_loads == FSLBM_LOADS_PAIRS && pairs_shape_ok(p)) h->bulk_mode = BULK_PAIRS;
  if (h->prec != FSLBM_F64 && q.bulk_loads == FSLBM_LOADS_TMA && tma_shape_ok(p, h->prec)) {
    // tensor maps of both population buffers
    h->tmap = (CUtensorMap*)aligned_alloc(64, 2 * sizeof(CUtensorMap));
    if (h->tmap && tma_encode(p, h->prec, h->fA, &h->tmap[0]) && tma_encode(p, h->prec, h->fB, &h->tmap[1])) {
      h->bulk_mode = BULK_TMA;
    } else {
      free(h->tmap);
      h->tmap = nullptr;
    }
  }
  // the side stream of the interface kernels (they run beside the bulk kernel)
  h->overlap = 1;
  if (cudaStreamCreateWithFlags(&h->fork.side, cudaStreamNonBlocking) == cudaSuccess) {
    if (cudaEventCreateWithFlags(&h->fork.fork, cudaEventDisableTiming) == cudaSuccess) {
      if (cudaEventCreateWithFlags(&h->fork.join, cudaEventDisableTiming) == cudaSuccess) h->forked = 1;
      else cudaEventDestroy(h->fork.fork);
    }
    if (!h->forked) cudaStreamDestroy(h->fork.side);
  }
  if (cudaStreamSynchronize(h->st) != cudaSuccess) {
    free_all(h);
    free(h);
    return FSLBM_ERR_CUDA;
  }
  *out = h;
  return FSLBM_OK;
}

extern "C" int fslbm_create(const int dims[3], double tau, const double g[3], double rho_G, double sigma,
                            int rule, fslbm_t** out) {
  if (!dims) return FSLBM_ERR_ARG;
  fslbm_params p;
  fslbm_default_params(&p);
  for (int a = 0; a < 3; ++a) {
    p.dims[a] = dims[a];
    p.g[a] = g ? g[a] : 0.0;
  }
  p.tau = tau;
  p.rho_G = rho_G;
  p.sigma = sigma;
  p.rule = rule;
  return fslbm_create_ex(&p, out);
}

// Sec. 2.1: nu = c_s^2 (tau - 1/2) with c_s^2 = 1/3 (lambda_+ = -1/tau)
extern "C" int fslbm_tau_of_viscosity(double nu, double* tau) {
  if (!tau || !(nu > 0.0) || !(nu < 1e300)) return FSLBM_ERR_ARG;
  *tau = 3.0 * nu + 0.5;
  return FSLBM_OK;
}

extern "C" int fslbm_bulk_loads(const fslbm_t* h) {
  if (!h) return FSLBM_ERR_ARG;
  return h->bulk_mode == BULK_TMA     ? FSLBM_LOADS_TMA
         : h->bulk_mode == BULK_ASYNC ? FSLBM_LOADS_ASYNC
         : h->bulk_mode == BULK_PAIRS ? FSLBM_LOADS_PAIRS
                                      : FSLBM_LOADS_PLAIN;
}

extern "C" int fslbm_set_overlap(fslbm_t* h, int on) {
  if (!h || (on != 0 && on != 1)) return FSLBM_ERR_ARG;
  h->overlap = on;
  return FSLBM_OK;
}

// the step's mass reduction runs inside the cooperative conversion kernel
static bool fold_reduce(const fslbm* h) { return !h->par.freeze && h->coop_blocks >= h->red_blocks; }

extern "C" int fslbm_check_grid_barrier(int expire, void* stream) {
  if (expire < 0 || expire > 1) return FSLBM_ERR_ARG;
  int dev = 0, coop = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FSLBM_ERR_CUDA;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (!coop || sms <= 0) return FSLBM_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  int* buf = nullptr;  // [0] barrier counter, [1] error bits
  if (cudaMalloc(&buf, 2 * sizeof(int)) != cudaSuccess) return FSLBM_ERR_OOM;
  int rc = FSLBM_OK, host[2] = {0, 0};
  if (cudaMemsetAsync(buf, 0, 2 * sizeof(int), st) != cudaSuccess ||
      launch_barrier_check((unsigned*)buf, buf + 1, sms * 2, (unsigned)expire, st) != cudaSuccess ||
      cudaMemcpyAsync(host, buf, sizeof host, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    rc = FSLBM_ERR_CUDA;
  else if (host[1] & ERRB_SYNC)
    rc = FSLBM_ERR_TIMEOUT;
  cudaFree(buf);
  return rc;
}

extern "C" int fslbm_launches_per_step(const fslbm_t* h) {
  if (!h) return FSLBM_ERR_ARG;
  const Par& p = h->par;
  const int geom = (p.rule != 0 || p.sigma != 0.0 || p.stress || p.recon_nc) ? 1 : 0;
  const int conv = p.freeze ? 0 : (h->coop_blocks > 0 ? 1 : 4);
  const int reduce = fold_reduce(h) ? 0 : 2;
  return 4 + geom + reduce + conv;  // reset, segments, bulk, interface
}

extern "C" void fslbm_destroy(fslbm_t* h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  fslbm_free_adjoint(h);
  free_all(h);
  free(h);
}

// Copy a caller buffer to device memory: device pointers are used in place,
// host pointers are staged through a temporary device buffer.
struct Staged {
  const void* dev = nullptr;
  void* owned = nullptr;
  ~Staged() {
    if (owned) cudaFree(owned);
  }
};
static int stage(fslbm* h, const void* src, size_t bytes, int where, Staged& s) {
  if (!src) return FSLBM_OK;
  if (where == FSLBM_DEVICE) {
    s.dev = src;
    return FSLBM_OK;
  }
  CK(cudaMalloc(&s.owned, bytes), "cudaMalloc (staging)");
  CK(cudaMemcpyAsync(s.owned, src, bytes, cudaMemcpyHostToDevice, h->st), "H2D copy");
  s.dev = s.owned;
  return FSLBM_OK;
}

static int read_err(fslbm* h) {
  int e = 0;
  CK(cudaMemcpyAsync(&e, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->st), "D2H error word");
  CK(cudaStreamSynchronize(h->st), "stream synchronize");
  if (e & ERRB_STATE) return fail(h, FSLBM_ERR_STATE, "invariant violated: a liquid cell touches gas, or a bad flag");
  if (e & ERRB_UNSTABLE) return fail(h, FSLBM_ERR_UNSTABLE, "non-finite or non-positive density");
  if (e & ERRB_SPEED) return fail(h, FSLBM_ERR_UNSTABLE, "a liquid cell velocity above u_max");
  if (e & ERRB_OVERFLOW) return fail(h, FSLBM_ERR_OVERFLOW, "conversion list overflow");
  if (e & ERRB_TMA) return fail(h, FSLBM_ERR_TIMEOUT, "staged loads of the bulk kernel failed (bounded wait expired)");
  if (e & ERRB_SYNC) return fail(h, FSLBM_ERR_TIMEOUT, "grid barrier of the conversion kernel expired");
  if (e & ERRB_BOUNDS) return fail(h, FSLBM_ERR_STATE, "an index outside its array (bounds-checked build)");
  return FSLBM_OK;
}

static int begin_state(fslbm* h, const uint8_t* flags, const double* wall_delta, int where, Staged& sf,
                       Staged& sw) {
  const size_t N = (size_t)h->par.N;
  if (!flags) return fail(h, FSLBM_ERR_ARG, "flags is NULL");
  fslbm_free_adjoint(h);
  if (where != FSLBM_HOST && where != FSLBM_DEVICE) return fail(h, FSLBM_ERR_ARG, "bad `where`");
  CK(cudaMemcpyAsync(h->flags, flags, N, where == FSLBM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     h->st),
     "copy flags");
  CK(cudaMemsetAsync(h->err, 0, 8, h->st), "memset");
  CK(cudaMemsetAsync(h->mark, 0, ((N + 3) & ~(size_t)3), h->st), "memset");
  CK(cudaMemsetAsync(h->lost, 0, 8, h->st), "memset");
  CK(cudaMemsetAsync(h->cnt, 0, 16 * sizeof(int), h->st), "memset");
  if (launch_prepare_flags(h->par, h->flags, h->err, h->st)) return fail(h, FSLBM_ERR_CUDA, "prepare flags launch");
  if (wall_delta) {
    if (!h->wd) {
      if (!dalloc(h, &h->wd, 19 * N * 8)) return fail(h, FSLBM_ERR_OOM, "wall_delta allocation");
    }
    CK(cudaMemcpyAsync(h->wd, wall_delta, 19 * N * 8,
                       where == FSLBM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st),
       "copy wall_delta");
    h->par.has_wd = 1;
  } else {
    h->par.has_wd = 0;
  }
  (void)sf;
  (void)sw;
  h->cur = 0;
  h->t = 0;
  return FSLBM_OK;
}

template <int P>
static int init_pre_t(fslbm* h, const double* f, const double* phi, const double* rho, const double* u,
                      const double* noise) {
  View<P> v = make_view<P>(h);
  h->f0_valid = h->f0 != nullptr;
  return launch_init_pre<P>(h->par, v, f, phi, rho, u, noise, h->f0, h->st);
}
template <int P>
static int init_post_t(fslbm* h, const double* f, const double* m, const double* phi) {
  View<P> v = make_view<P>(h);
  h->f0_valid = 0;
  return launch_init_post<P>(h->par, v, f, m, phi, h->st);
}

static int dispatch_init_pre(fslbm* h, const double* f, const double* phi, const double* rho, const double* u,
                             const double* noise) {
  switch (h->prec) {
    case FSLBM_F64: return init_pre_t<P64>(h, f, phi, rho, u, noise);
    case FSLBM_F32: return init_pre_t<P32>(h, f, phi, rho, u, noise);
    default: return init_pre_t<P16>(h, f, phi, rho, u, noise);
  }
}

extern "C" int fslbm_set_state(fslbm_t* h, const uint8_t* flags, const double* f, const double* phi,
                               const double* wall_delta, int where) {
  if (!h || !f) return FSLBM_ERR_ARG;
  const size_t N = (size_t)h->par.N;
  Staged sfl, swd, sf, sphi;
  int rc = begin_state(h, flags, wall_delta, where, sfl, swd);
  if (rc) return rc;
  if ((rc = stage(h, f, 19 * N * 8, where, sf))) return rc;
  if ((rc = stage(h, phi, N * 8, where, sphi))) return rc;
  if (dispatch_init_pre(h, (const double*)sf.dev, (const double*)sphi.dev, nullptr, nullptr, nullptr))
    return fail(h, FSLBM_ERR_CUDA, "init launch");
  return read_err(h);
}

extern "C" int fslbm_init_equilibrium(fslbm_t* h, const uint8_t* flags, const double* rho, const double* u,
                                      const double* phi, const double* noise, const double* wall_delta,
                                      int where) {
  if (!h || !rho || !u) return FSLBM_ERR_ARG;
  const size_t N = (size_t)h->par.N;
  Staged sfl, swd, sr, su, sphi, sn;
  int rc = begin_state(h, flags, wall_delta, where, sfl, swd);
  if (rc) return rc;
  if ((rc = stage(h, rho, N * 8, where, sr))) return rc;
  if ((rc = stage(h, u, 3 * N * 8, where, su))) return rc;
  if ((rc = stage(h, phi, N * 8, where, sphi))) return rc;
  if ((rc = stage(h, noise, 19 * N * 8, where, sn))) return rc;
  if (dispatch_init_pre(h, nullptr, (const double*)sphi.dev, (const double*)sr.dev, (const double*)su.dev,
                        (const double*)sn.dev))
    return fail(h, FSLBM_ERR_CUDA, "init launch");
  return read_err(h);
}

extern "C" int fslbm_set_state_post(fslbm_t* h, const uint8_t* flags, const double* f_post, const double* m,
                                    const double* phi, const double* wall_delta, int where) {
  if (!h || !f_post || !m || !phi) return FSLBM_ERR_ARG;
  const size_t N = (size_t)h->par.N;
  Staged sfl, swd, sf, sm, sphi;
  int rc = begin_state(h, flags, wall_delta, where, sfl, swd);
  if (rc) return rc;
  if ((rc = stage(h, f_post, 19 * N * 8, where, sf))) return rc;
  if ((rc = stage(h, m, N * 8, where, sm))) return rc;
  if ((rc = stage(h, phi, N * 8, where, sphi))) return rc;
  int lr;
  switch (h->prec) {
    case FSLBM_F64: lr = init_post_t<P64>(h, (const double*)sf.dev, (const double*)sm.dev, (const double*)sphi.dev); break;
    case FSLBM_F32: lr = init_post_t<P32>(h, (const double*)sf.dev, (const double*)sm.dev, (const double*)sphi.dev); break;
    default: lr = init_post_t<P16>(h, (const double*)sf.dev, (const double*)sm.dev, (const double*)sphi.dev); break;
  }
  if (lr) return fail(h, FSLBM_ERR_CUDA, "init launch");
  return read_err(h);
}

// event k (0..4) of the current timed step, created on first use
static int mark_event(fslbm* h, int k) {
  if (!h->timing) return 0;
  size_t idx = (size_t)h->timed_steps * 5 + k;
  while (h->events->size() <= idx) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return 1;
    h->events->push_back(e);
  }
  return cudaEventRecord((*h->events)[idx], h->st) != cudaSuccess;
}

template <int P>
static int step_t(fslbm* h) {
  View<P> v = make_view<P>(h);
  if (launch_reset(h->cnt, h->st)) return 1;
  if (launch_step_kernels<P>(h->par, v, h->st, h->bulk_blocks, h->iface_blocks, h->seglist, h->cnt + 9,
                             h->timing ? h : nullptr, h->bulk_mode, h->tmap ? &h->tmap[h->cur] : nullptr,
                             (h->forked && h->overlap) ? &h->fork : nullptr))
    return 1;
  if (mark_event(h, 2)) return 1;
  // the mass reduction rides in the cooperative conversion kernel where that runs
  MassReduce mr = {};
  const long long nparts = (long long)(h->bulk_blocks + h->iface_blocks) * 4;
  if (fold_reduce(h)) {
    mr.in = h->partials;
    mr.n = nparts;
    mr.chunk = (nparts + h->red_blocks - 1) / h->red_blocks;
    if (mr.chunk < 1) mr.chunk = 1;
    mr.nb = (int)((nparts + mr.chunk - 1) / mr.chunk);
    mr.tmp = h->red;
    mr.add = h->lost;
    mr.out = h->step_mass;
  } else if (launch_reduce(h->partials, nparts, h->red, h->red_blocks, h->lost, h->step_mass, h->st)) {
    return 1;
  }
  if (mark_event(h, 3)) return 1;
  if (!h->par.freeze) {
    int rc = launch_conversions<P>(h->par, v, h->st, h->list_blocks, h->coop_blocks, mr);
    if (rc == (int)cudaErrorCooperativeLaunchTooLarge && h->coop_blocks > 0) {
      // the device cannot hold the cooperative grid now (e.g. shared with
      // other work): four launches and the stand-alone reduction from here on
      cudaGetLastError();
      h->coop_blocks = 0;
      if (mr.nb > 0 && launch_reduce(h->partials, nparts, h->red, h->red_blocks, h->lost, h->step_mass, h->st))
        return 1;
      rc = launch_conversions<P>(h->par, v, h->st, h->list_blocks, 0, MassReduce{});
    }
    if (rc) return 1;
  }
  if (mark_event(h, 4)) return 1;
  if (h->timing) h->timed_steps += 1;
  return 0;
}

// called around the bulk kernel when timing is on (events 0 and 1)
namespace fsl {
int fslbm_mark(void* hv, int k) { return mark_event((fslbm*)hv, k); }
}  // namespace fsl

extern "C" int fslbm_timing(fslbm_t* h, int on) {
  if (!h) return FSLBM_ERR_ARG;
  CK(cudaStreamSynchronize(h->st), "stream synchronize");
  drop_events(h);
  h->timed_steps = 0;
  h->timing = on ? 1 : 0;
  if (on) h->events = new std::vector<cudaEvent_t>();
  return FSLBM_OK;
}

extern "C" int fslbm_timing_read(fslbm_t* h, double ms[4], long long* steps) {
  if (!h || !ms) return FSLBM_ERR_ARG;
  for (int k = 0; k < 4; ++k) ms[k] = 0.0;
  if (steps) *steps = h->timed_steps;
  if (!h->events || h->timed_steps == 0) return FSLBM_OK;
  CK(cudaStreamSynchronize(h->st), "stream synchronize");
  for (long long s = 0; s < h->timed_steps; ++s)
    for (int k = 0; k < 4; ++k) {
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, (*h->events)[s * 5 + k], (*h->events)[s * 5 + k + 1]), "event elapsed");
      ms[k] += t;
    }
  for (int k = 0; k < 4; ++k) ms[k] /= (double)h->timed_steps;
  return FSLBM_OK;
}

extern "C" int fslbm_step(fslbm_t* h, int n) {
  if (!h || n < 0) return FSLBM_ERR_ARG;
  for (int s = 0; s < n; ++s) {
    int r;
    switch (h->prec) {
      case FSLBM_F64: r = step_t<P64>(h); break;
      case FSLBM_F32: r = step_t<P32>(h); break;
      default: r = step_t<P16>(h); break;
    }
    if (r) return fail(h, FSLBM_ERR_CUDA, "step launch", cudaGetLastError());
    h->cur ^= 1;
    h->t += 1;
  }
  return FSLBM_OK;
}

extern "C" int fslbm_sync(fslbm_t* h) {
  if (!h) return FSLBM_ERR_ARG;
  return read_err(h);
}

extern "C" int fslbm_get_fields(fslbm_t* h, unsigned mask, void* const* out, int where) {
  if (!h || (mask & ~63u) || (mask && !out)) return FSLBM_ERR_ARG;
  const size_t N = (size_t)h->par.N;
  const size_t sizes[6] = {N, 19 * N * 8, N * 8, N * 8, N * 8, 3 * N * 8};
  void* dev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  void* owned[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int k = 0, rc = FSLBM_OK;
  for (int b = 0; b < 6; ++b) {
    if (!(mask & (1u << b))) continue;
    if (!out[k]) return fail(h, FSLBM_ERR_ARG, "NULL output buffer");
    if (where == FSLBM_DEVICE) {
      dev[k] = out[k];
    } else if (cudaMalloc(&owned[k], sizes[b]) != cudaSuccess) {
      rc = fail(h, FSLBM_ERR_OOM, "staging allocation");
      break;
    } else {
      dev[k] = owned[k];
    }
    ++k;
  }
  if (rc == FSLBM_OK) {
    int lr;
    switch (h->prec) {
      case FSLBM_F64: { View<P64> v = make_view<P64>(h); lr = launch_fields<P64>(h->par, v, mask, dev, h->st); break; }
      case FSLBM_F32: { View<P32> v = make_view<P32>(h); lr = launch_fields<P32>(h->par, v, mask, dev, h->st); break; }
      default: { View<P16> v = make_view<P16>(h); lr = launch_fields<P16>(h->par, v, mask, dev, h->st); break; }
    }
    if (lr) rc = fail(h, FSLBM_ERR_CUDA, "fields launch");
  }
  if (rc == FSLBM_OK && where != FSLBM_DEVICE) {
    int kk = 0;
    for (int b = 0; b < 6 && rc == FSLBM_OK; ++b) {
      if (!(mask & (1u << b))) continue;
      if (cudaMemcpyAsync(out[kk], dev[kk], sizes[b], cudaMemcpyDeviceToHost, h->st) != cudaSuccess)
        rc = fail(h, FSLBM_ERR_CUDA, "D2H copy");
      ++kk;
    }
  }
  int se = rc == FSLBM_OK ? read_err(h) : rc;
  for (int b = 0; b < 6; ++b)
    if (owned[b]) cudaFree(owned[b]);
  return se;
}

extern "C" int fslbm_total_mass(fslbm_t* h, double* mass, double* lost) {
  if (!h) return FSLBM_ERR_ARG;
  int lr;
  switch (h->prec) {
    case FSLBM_F64: { View<P64> v = make_view<P64>(h); lr = launch_total_mass<P64>(h->par, v, h->partials, h->nparts, h->red, h->red_blocks, h->total_out, h->st); break; }
    case FSLBM_F32: { View<P32> v = make_view<P32>(h); lr = launch_total_mass<P32>(h->par, v, h->partials, h->nparts, h->red, h->red_blocks, h->total_out, h->st); break; }
    default: { View<P16> v = make_view<P16>(h); lr = launch_total_mass<P16>(h->par, v, h->partials, h->nparts, h->red, h->red_blocks, h->total_out, h->st); break; }
  }
  if (lr) return fail(h, FSLBM_ERR_CUDA, "mass launch");
  double M = 0.0, L = 0.0;
  CK(cudaMemcpyAsync(&M, h->total_out, 8, cudaMemcpyDeviceToHost, h->st), "D2H mass");
  CK(cudaMemcpyAsync(&L, h->lost, 8, cudaMemcpyDeviceToHost, h->st), "D2H lost");
  int rc = read_err(h);
  if (mass) *mass = M;
  if (lost) *lost = L;
  return rc;
}

extern "C" int fslbm_step_mass(fslbm_t* h, double* mass) {
  if (!h) return FSLBM_ERR_ARG;
  double M = 0.0;
  CK(cudaMemcpyAsync(&M, h->step_mass, 8, cudaMemcpyDeviceToHost, h->st), "D2H step mass");
  int rc = read_err(h);
  if (mass) *mass = M;
  return rc;
}

extern "C" int fslbm_counters(fslbm_t* h, long long out[5]) {
  if (!h || !out) return FSLBM_ERR_ARG;
  int c[16];
  CK(cudaMemcpyAsync(c, h->cnt, sizeof c, cudaMemcpyDeviceToHost, h->st), "D2H counters");
  int rc = read_err(h);
  out[0] = c[1];
  out[1] = c[7];
  out[2] = c[3];
  out[3] = c[4];
  out[4] = c[0] + c[6];
  return rc;
}

extern "C" long long fslbm_time(const fslbm_t* h) { return h ? h->t : -1; }
extern "C" int fslbm_build_info(void) {
#ifdef FSLBM_CHECKED
  return 1;
#else
  return 0;
#endif
}

extern "C" size_t fslbm_device_bytes(const fslbm_t* h) { return h ? h->bytes : 0; }
extern "C" const char* fslbm_last_error(const fslbm_t* h) { return h ? h->msg : "NULL handle"; }

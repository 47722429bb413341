// fslbm_halo.cu -- state of a box of cells in and out of a contiguous device
// buffer, and the owned region of a subdomain (slab decomposition).
//
// A lattice split into slabs runs each slab as a lattice of its own with G
// ghost layers beside every cut.  One time step of a cell depends on the
// state of time t within a fixed radius R of it (interface geometry 3, stream
// 1, the conversions' neighbour chains 3 more), so after a step every cell at
// least R layers inside a slab's ghost band is exact; with G >= R the owned
// cells are exact, and refilling the ghost layers from the neighbours' owned
// cells (pack here, transport by the caller, unpack there) makes the whole
// slab exact again.  One exchange per step covers the whole step, conversions
// included.  The buffer of a box of n cells holds, in this order, each block
// starting on a 16-byte boundary: the cell kinds (u8[n]), the interface mass
// (f64[n]), the fill levels phi(t) (R[n]) and the post-collision populations
// f~(t) ([19][n] in the storage type), cells in box order (x fastest).
#include <cuda_runtime.h>

#include "fslbm.h"
#include "fslbm_dev.cuh"
#include "fslbm_handle.h"

using namespace fsl;

namespace {

inline size_t up16(size_t b) { return (b + 15) & ~(size_t)15; }

struct BoxLayout {
  long long n;
  size_t off_m, off_phi, off_f, bytes;
};

BoxLayout layout(int prec, long long n) {
  const size_t sb = prec == FSLBM_F64 ? 8 : (prec == FSLBM_F32 ? 4 : 2);
  const size_t rb = prec == FSLBM_F64 ? 8 : 4;
  BoxLayout L;
  L.n = n;
  L.off_m = up16((size_t)n);
  L.off_phi = up16(L.off_m + 8 * (size_t)n);
  L.off_f = up16(L.off_phi + rb * (size_t)n);
  L.bytes = up16(L.off_f + 19 * sb * (size_t)n);
  return L;
}

template <int P, bool UNPACK>
__global__ void __launch_bounds__(256) k_box(Par p, View<P> v, int x0, int y0, int z0, int bx, int by, long long n,
                                             unsigned char* __restrict__ buf, size_t off_m, size_t off_phi,
                                             size_t off_f) {
  using S = typename Form<P>::S;
  using R = typename Form<P>::R;
  uint8_t* bk = buf;
  double* bm = reinterpret_cast<double*>(buf + off_m);
  R* bphi = reinterpret_cast<R*>(buf + off_phi);
  S* bf = reinterpret_cast<S*>(buf + off_f);
  S* fin = const_cast<S*>(v.fin);
  R* phin = const_cast<R*>(v.phin);
  const size_t N = (size_t)p.N;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const long long row = k / bx;
    const int x = x0 + (int)(k - row * bx);
    const int y = y0 + (int)(row % by);
    const int z = z0 + (int)(row / by);
    const size_t i = (size_t)FSL_CK(p, (size_t)x + (size_t)p.nx * ((size_t)y + (size_t)p.ny * (size_t)z), p.N);
    if (UNPACK) {
      v.flags[i] = (uint8_t)((v.flags[i] & STATIC_BITS) | (bk[k] & KIND));
      v.m[i] = bm[k];
      phin[i] = bphi[k];
#pragma unroll
      for (int q = 0; q < 19; ++q) fin[(size_t)q * N + i] = bf[(size_t)q * (size_t)n + (size_t)k];
    } else {
      bk[k] = (uint8_t)(v.flags[i] & KIND);
      bm[k] = v.m[i];
      bphi[k] = phin[i];
#pragma unroll
      for (int q = 0; q < 19; ++q) bf[(size_t)q * (size_t)n + (size_t)k] = fin[(size_t)q * N + i];
    }
  }
}

bool box_ok(const fslbm* h, const int lo[3], const int hi[3]) {
  if (!h || !lo || !hi) return false;
  const int n[3] = {h->par.nx, h->par.ny, h->par.nz};
  for (int a = 0; a < 3; ++a)
    if (lo[a] < 0 || hi[a] > n[a] || lo[a] >= hi[a]) return false;
  return true;
}

long long box_cells(const int lo[3], const int hi[3]) {
  return (long long)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
}

template <int P, bool UNPACK>
int run_box(fslbm* h, const int lo[3], const int hi[3], void* buf) {
  const long long n = box_cells(lo, hi);
  const BoxLayout L = layout(h->prec, n);
  long long grid = (n + 255) / 256;
  if (grid > 152LL * 16) grid = 152LL * 16;
  k_box<P, UNPACK><<<(unsigned)grid, 256, 0, h->st>>>(h->par, make_view<P>(h), lo[0], lo[1], lo[2], hi[0] - lo[0],
                                                      hi[1] - lo[1], n, (unsigned char*)buf, L.off_m, L.off_phi,
                                                      L.off_f);
  const cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return FSLBM_ERR_CUDA;
  }
  return FSLBM_OK;
}

template <bool UNPACK>
int box(fslbm* h, const int lo[3], const int hi[3], void* buf) {
  if (!box_ok(h, lo, hi) || !buf || ((uintptr_t)buf & 15)) return FSLBM_ERR_ARG;
  if (UNPACK) fslbm_free_adjoint(h);  // a changed state ends a differentiation
  switch (h->prec) {
    case FSLBM_F64: return run_box<P64, UNPACK>(h, lo, hi, buf);
    case FSLBM_F32: return run_box<P32, UNPACK>(h, lo, hi, buf);
    default: return run_box<P16, UNPACK>(h, lo, hi, buf);
  }
}

}  // namespace

extern "C" int fslbm_set_owned(fslbm_t* h, const int lo[3], const int hi[3]) {
  if (!box_ok(h, lo, hi)) return FSLBM_ERR_ARG;
  Par& p = h->par;
  const int n[3] = {p.nx, p.ny, p.nz};
  bool all = true;
  for (int a = 0; a < 3; ++a) {
    p.own_lo[a] = lo[a];
    p.own_hi[a] = hi[a];
    all = all && lo[a] == 0 && hi[a] == n[a];
  }
  p.owned_all = all ? 1 : 0;
  return FSLBM_OK;
}

extern "C" long long fslbm_halo_bytes(const fslbm_t* h, const int lo[3], const int hi[3]) {
  if (!box_ok(h, lo, hi)) return FSLBM_ERR_ARG;
  return (long long)layout(h->prec, box_cells(lo, hi)).bytes;
}

extern "C" int fslbm_halo_pack(fslbm_t* h, const int lo[3], const int hi[3], void* buf) {
  return box<false>(h, lo, hi, buf);
}

extern "C" int fslbm_halo_unpack(fslbm_t* h, const int lo[3], const int hi[3], const void* buf) {
  return box<true>(h, lo, hi, const_cast<void*>(buf));
}

// fslbm_step.cu -- the precision-independent kernels of one FSLBM time step:
// the segment scan (k_segments), the counter reset and the fixed-order
// reduction.  The stream-collide kernels are templates in fslbm_step.cuh,
// instantiated per precision form in fslbm_step_p64/p32/p16.cu.
#include "fslbm_dev.cuh"
#include "fslbm_kernels.h"

namespace fsl {

// ---------------------------------------------------------------------------
// k_segments: compact list of the 32-cell x segments (one warp each) that
// hold a liquid or interface cell; one thread per segment, one atomic per warp.
// Besides the record (x0, y, z, first cell) of list entry k at seglist[4k],
// it writes the segment's masks at seglist[4 (S + k)] (S: segments of the
// lattice): bit j of each for cell x0 + j, liquid, interface, and liquid
// needing the general pull (k_bulk's test of a fast cell, negated), so that a
// bulk kernel reads no flag on its fast path.  It also lists the step's
// interface cells: a cell whose stencil (every cell within 3) lies inside the
// lattice at the front of the interface list, the others at its back, each
// segment's cells in x order, one atomic per warp and end.
// ---------------------------------------------------------------------------
// bit s of each byte of w, gathered into bits 0-3 (the four partial products
// of the multiplier land on distinct bits, so no carries mix them)
__device__ __forceinline__ unsigned byte_bits(unsigned w, int s) {
  return ((((w >> s) & 0x01010101u) * 0x00204081u) >> 21) & 0xfu;
}

// the set bits of m (cells x0 + k of a segment) written in increasing k to
// list positions k0, k0 + 1, ... (from the back of the list when back)
__device__ __forceinline__ void put_cells(unsigned m, int first, int k0, int* list, int cap, bool back, int* err) {
  while (m) {
    const int k = __ffs(m) - 1;
    m &= m - 1u;
    if (k0 < cap) list[back ? cap - 1 - k0 : k0] = first + k;
    else atomicOr(err, ERRB_OVERFLOW);
    ++k0;
  }
}

__global__ void __launch_bounds__(256) k_segments(Par p, const uint8_t* __restrict__ flags, int* __restrict__ seglist,
                                                  int* __restrict__ count, int* __restrict__ ilist,
                                                  int* __restrict__ icount, int cap, int* __restrict__ err) {
  pdl_begin();
  const int nsx = (p.nx + 31) >> 5;
  const long long nseg = (long long)nsx * p.ny * p.nz;
  const long long sgi = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  bool act = false;
  unsigned liq = 0u, ifc = 0u, nearb = 0u, nearw = 0u;
  int len = 0;
  if (sgi < nseg) {
    const long long row = (long long)fdiv((unsigned)sgi, p.dnsx);
    const int x0 = (int)(sgi - row * nsx) << 5;
    len = min(32, p.nx - x0);
    const uint8_t* base = flags + row * p.nx + x0;
    // kinds are one-hot (LIQ = bit 0, IFC = bit 1); NEARB = bit 4, NEARW = bit 5
    if (len == 32 && ((p.nx & 15) == 0)) {
      const uint4* v4 = reinterpret_cast<const uint4*>(base);
      const uint4 a = __ldg(v4), b = __ldg(v4 + 1);
      const unsigned w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
      // the masks only for segments holding fluid (most of a lattice is gas)
      if (((a.x | a.y | a.z | a.w | b.x | b.y | b.z | b.w) & 0x03030303u) != 0u) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          liq |= byte_bits(w[k], 0) << (4 * k);
          ifc |= byte_bits(w[k], 1) << (4 * k);
          nearb |= byte_bits(w[k], 4) << (4 * k);
          nearw |= byte_bits(w[k], 5) << (4 * k);
        }
      }
    } else {
      for (int k = 0; k < len; ++k) {
        const unsigned c = base[k];
        liq |= (c & 1u) << k;
        ifc |= ((c >> 1) & 1u) << k;
        nearb |= ((c >> 4) & 1u) << k;
        nearw |= ((c >> 5) & 1u) << k;
      }
    }
    act = (liq | ifc) != 0u;
  }
  // one global atomic per block: warp counts -> block offsets in shared memory
  __shared__ int wcount[8], wbase[8], bbase;
  const unsigned bal = __ballot_sync(0xffffffffu, act);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) wcount[w] = __popc(bal);
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int k = 0; k < 8; ++k) { wbase[k] = t; t += wcount[k]; }
    bbase = t ? atomicAdd(count, t) : 0;
  }
  __syncthreads();
  if (act) {
    // the segment's first x, y, z and first cell index, so that the bulk
    // kernels need no division
    const unsigned row = fdiv((unsigned)sgi, p.dnsx);
    const unsigned zz = fdiv(row, p.dny);
    const int x0 = (int)((unsigned)sgi - row * (unsigned)nsx) << 5;
    const int y = (int)(row - zz * (unsigned)p.ny), z = (int)zz;
    const int k = bbase + wbase[w] + __popc(bal & ((1u << lane) - 1u));
    reinterpret_cast<int4*>(seglist)[k] = make_int4(x0, y, z, (int)row * p.nx + x0);
    // liquid cells that need the general pull (fast_cell of the bulk kernels, negated)
    const unsigned all = len == 32 ? 0xffffffffu : ((1u << len) - 1u);
    const unsigned xf = (x0 == 0 ? 1u : 0u) | (x0 + len == p.nx ? 1u << (len - 1) : 0u);
    const bool yf = y == 0 || y == p.ny - 1, zf = z == 0 || z == p.nz - 1;
    unsigned slow;
    if (p.has_wd || p.has_uw) slow = liq & (nearb | xf | ((yf || zf) ? all : 0u));
    else slow = liq & (nearw | (p.px ? xf : 0u) | (((yf && p.py) || (zf && p.pz)) ? all : 0u));
    reinterpret_cast<uint4*>(seglist)[nseg + k] = make_uint4(liq, ifc, slow, 0u);
  }
  // interface cells: interior ones (every cell within 3 inside the lattice) to
  // the front of the list (count icount[0]), the others to its back (icount[6])
  unsigned fin = 0u, fed = 0u;
  int first = 0;
  if (ifc) {
    const unsigned row = fdiv((unsigned)sgi, p.dnsx);
    const unsigned zz = fdiv(row, p.dny);
    const int x0 = (int)((unsigned)sgi - row * (unsigned)nsx) << 5;
    const int y = (int)(row - zz * (unsigned)p.ny), z = (int)zz;
    first = (int)row * p.nx + x0;
    const int lo = max(0, 3 - x0), hi = min(len, p.nx - 3 - x0);  // cells with 3 <= x < nx - 3
    const unsigned xin = hi > lo ? ((hi - lo == 32) ? 0xffffffffu : ((1u << (hi - lo)) - 1u) << lo) : 0u;
    const bool yz3 = y >= 3 && y < p.ny - 3 && z >= 3 && z < p.nz - 3;
    fin = yz3 ? (ifc & xin) : 0u;
    fed = ifc & ~fin;
  }
  // prefix sums of the counts over the warp, then over the block's warps: one
  // atomic per block and end (the two counters are shared by the whole grid)
  int ni = __popc(fin), ne = __popc(fed);
  const bool any = __ballot_sync(0xffffffffu, (fin | fed) != 0u) != 0u;
  if (any) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int a = __shfl_up_sync(0xffffffffu, ni, o), b = __shfl_up_sync(0xffffffffu, ne, o);
      if (lane >= o) { ni += a; ne += b; }
    }
  }
  __shared__ int wi[8], we[8], bi0, be0;
  if (lane == 31) { wi[w] = ni; we[w] = ne; }
  __syncthreads();
  if (threadIdx.x == 0) {
    int ti = 0, te = 0;
    for (int k = 0; k < 8; ++k) {
      const int a = wi[k], b = we[k];
      wi[k] = ti; we[k] = te;
      ti += a; te += b;
    }
    bi0 = ti ? atomicAdd(&icount[0], ti) : 0;
    be0 = te ? atomicAdd(&icount[6], te) : 0;
  }
  __syncthreads();
  const int bi = bi0 + wi[w], be = be0 + we[w];
  if (fin) put_cells(fin, first, bi + ni - __popc(fin), ilist, cap, false, err);
  if (fed) put_cells(fed, first, be + ne - __popc(fed), ilist, cap, true, err);
}

// ---------------------------------------------------------------------------
// Fixed-order reduction of the block partials: out[b] = sum of chunk b.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_reduce(const double* __restrict__ in, long long n, long long chunk,
                                                double* __restrict__ out, const double* add, double* final_out) {
  pdl_begin();
  const double t = block_chunk_sum(in, n, chunk, blockIdx.x);
  if (threadIdx.x == 0) {
    out[blockIdx.x] = t;
    if (final_out) *final_out = t + (add ? *add : 0.0);
  }
}

int launch_segments(const Par& p, const uint8_t* flags, int* seglist, int* segcount, int* ilist, int* cnt, int cap,
                    int* err, cudaStream_t st) {
  const long long nseg = (long long)((p.nx + 31) / 32) * p.ny * p.nz;
  return launch_k(k_segments, (unsigned)((nseg + 255) / 256), 256, 0, st, p, flags, seglist, segcount, ilist, cnt,
                  cap, err);
}

__global__ void k_reset(int* cnt) {
  pdl_begin();
  if (threadIdx.x < 11 && threadIdx.x != 8) cnt[threadIdx.x] = 0;
}

int launch_reset(int* cnt, cudaStream_t st) { return launch_k(k_reset, 1, 32, 0, st, cnt); }

int launch_reduce(const double* in, long long n, double* tmp, int tmp_blocks, const double* add, double* out,
                  cudaStream_t st) {
  long long chunk = (n + tmp_blocks - 1) / tmp_blocks;
  if (chunk < 1) chunk = 1;
  int nb = (int)((n + chunk - 1) / chunk);
  if (nb < 1) nb = 1;
  if (launch_k(k_reduce, nb, 256, 0, st, in, n, chunk, tmp, (const double*)nullptr, (double*)nullptr)) return 1;
  if (launch_k(k_reduce, 1, 256, 0, st, (const double*)tmp, (long long)nb, (long long)nb, tmp + tmp_blocks, add, out))
    return 1;
  return (int)cudaGetLastError();
}

}  // namespace fsl

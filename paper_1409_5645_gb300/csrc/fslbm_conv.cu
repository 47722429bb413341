// fslbm_conv.cu -- cell conversions after the mass update (Sec. 2.3 / 4.4; the
// paper takes interface tracking from Koerner et al. and Thuerey).
//
// The step kernel appended interface cells with m > (1+eps) rho to the fill
// list F and those with m < -eps rho to the empty list E, and marked them.
// Then, all as list kernels (grid-stride; counts read on the device, no host
// synchronisation):
//   fill     gas neighbours of F become new interface (NEWG, listed once by an
//            atomic byte-OR); an E cell next to F leaves E
//   newg     NEWG cells get f = f^eq(mean rho, mean u) over their liquid /
//            interface neighbours (q order), collided, m = 0
//   empty    liquid neighbours of the remaining E become interface with m = rho
//   share    excess (F: m - rho, E: m) / number of receivers (interface after
//            the steps above, not converting); no receiver -> lost ledger
//   recv     each receiver gathers the shares of its converting neighbours in q
//            order (deterministic, no floating-point atomics)
//   final    F -> liquid, E -> gas, new cells -> interface, marks cleared
// The result does not depend on list order.
#include "fslbm_dev.cuh"
#include "fslbm_kernels.h"

namespace fsl {

__device__ __forceinline__ uint8_t or_u8(uint8_t* base, long long j, unsigned bits) {
  unsigned* w = (unsigned*)(base + (j & ~3LL));
  unsigned sh = (unsigned)(j & 3) * 8u;
  unsigned old = atomicOr(w, bits << sh);
  return (uint8_t)(old >> sh);
}
__device__ __forceinline__ void clear_u8(uint8_t* base, long long j, unsigned bits) {
  unsigned* w = (unsigned*)(base + (j & ~3LL));
  unsigned sh = (unsigned)(j & 3) * 8u;
  atomicAnd(w, ~(bits << sh));
}
// append `value` for every converged lane with `pred`, one atomic per warp
__device__ __forceinline__ void push(bool pred, int* list, int* count, int cap, int value, int* err) {
  const unsigned act = __activemask();
  const unsigned bal = __ballot_sync(act, pred);
  if (!bal) return;
  const int lane = threadIdx.x & 31, leader = __ffs(bal) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(count, __popc(bal));
  base = __shfl_sync(act, base, leader);
  if (pred) {
    int k = base + __popc(bal & ((1u << lane) - 1u));
    if (k < cap) list[k] = value;
    else atomicOr(err, ERRB_OVERFLOW);
  }
}
__device__ __forceinline__ int load_count(const int* c) { return *((volatile const int*)c); }

template <int P>
__device__ __forceinline__ typename Form<P>::R rho_out(const Par& p, const View<P>& v, long long i) {
  using R = typename Form<P>::R;
  R r = R(0);
#pragma unroll
  for (int q = 0; q < 19; ++q) r += ldq<P>(v.fout, (size_t)q * (size_t)p.N + (size_t)i, q);
  return r;
}

// A gas cell next to a filled cell becomes interface with f = f^eq(mean rho,
// mean u) over its liquid/interface neighbours (kinds of step t, q order),
// collided, m = 0, phi = 0.  Its neighbours' populations are final for the
// step, and new cells are never read as neighbours (their kind is still gas).
template <int P>
__device__ void init_new_cell(const Par& p, const View<P>& v, long long j) {
  using R = typename Form<P>::R;
  const size_t N = (size_t)p.N;
  int x, y, z;
  coords(p, j, x, y, z);
  R rs = R(0), us0 = R(0), us1 = R(0), us2 = R(0);
  int c = 0;
#pragma unroll 1
  for (int q = 1; q < 19; ++q) {
    long long y2 = nbr(p, x, y, z, cx(q), cy(q), cz(q));
    if (y2 < 0) continue;
    uint8_t ky = v.flags[y2] & KIND;
    if (!is_fluid(ky)) continue;
    R g[19];
#pragma unroll
    for (int r = 0; r < 19; ++r) g[r] = ldq<P>(v.fout, (size_t)r * N + (size_t)y2, r);
    R rr, ux, uy, uz;
    moments_post<R>(p, g, rr, ux, uy, uz);
    rs += rr; us0 += ux; us1 += uy; us2 += uz;
    ++c;
  }
  R rbar = rs / R(c), u0 = us0 / R(c), u1 = us1 / R(c), u2 = us2 / R(c);
  R r0 = p.compressible ? rbar : R(1);
  R usq = u0 * u0 + u1 * u1 + u2 * u2;
  R f[19];
  f[0] = eplus<R, 0>(p, rbar, r0, u0, u1, u2, usq);
#define FSL_EQ(q) f[q] = eplus<R, q>(p, rbar, r0, u0, u1, u2, usq) + eminus<R, q>(r0, u0, u1, u2);
  FSL_EQ(1) FSL_EQ(2) FSL_EQ(3) FSL_EQ(4) FSL_EQ(5) FSL_EQ(6) FSL_EQ(7) FSL_EQ(8) FSL_EQ(9)
  FSL_EQ(10) FSL_EQ(11) FSL_EQ(12) FSL_EQ(13) FSL_EQ(14) FSL_EQ(15) FSL_EQ(16) FSL_EQ(17) FSL_EQ(18)
#undef FSL_EQ
  R rho, ux, uy, uz;
  collide<R>(p, f, rho, ux, uy, uz);
#pragma unroll
  for (int q = 0; q < 19; ++q) stq<P>(v.fout, (size_t)q * N + (size_t)j, q, f[q]);
  v.m[j] = 0.0;
  v.phout[j] = R(0);
}

template <int P>
__global__ void k_fill(Par p, View<P> v) {
  int nf = min(load_count(&v.cnt[1]), v.cap);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nf; k += gridDim.x * blockDim.x) {
    long long i = v.flist[k];
    int x, y, z;
    coords(p, i, x, y, z);
#pragma unroll
    for (int q = 1; q < 19; ++q) {
      long long j = nbr(p, x, y, z, cx(q), cy(q), cz(q));
      uint8_t kj = j < 0 ? (uint8_t)WALL : (uint8_t)(v.flags[j] & KIND);
      bool won = false;
      if (kj == GAS) {
        uint8_t old = or_u8(v.mark, j, MK_NEWG);
        won = !(old & MK_NEWG);  // the first claimant lists the new cell
      } else if (kj == IFC) {
        if (((volatile uint8_t*)v.mark)[j] & MK_EMPTY) clear_u8(v.mark, j, MK_EMPTY);
      }
      push(won, v.nglist, &v.cnt[3], v.cap, (int)j, v.err);
    }
  }
}

template <int P>
__global__ void k_newg(Par p, View<P> v) {
  int nn = min(load_count(&v.cnt[3]), v.cap);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nn; k += gridDim.x * blockDim.x)
    init_new_cell<P>(p, v, v.nglist[k]);
}

template <int P>
__global__ void k_empty(Par p, View<P> v) {
  using R = typename Form<P>::R;
  int ne = min(load_count(&v.cnt[2]), v.cap);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ne; k += gridDim.x * blockDim.x) {
    long long i = v.elist[k];
    if (!(v.mark[i] & MK_EMPTY)) continue;
    int x, y, z;
    coords(p, i, x, y, z);
#pragma unroll 1
    for (int q = 1; q < 19; ++q) {
      long long j = nbr(p, x, y, z, cx(q), cy(q), cz(q));
      if (j < 0) continue;
      if ((v.flags[j] & KIND) != LIQ) continue;
      uint8_t old = or_u8(v.mark, j, MK_NEWL);
      if (!(old & MK_NEWL)) {
        R r = rho_out<P>(p, v, j);
        double mm = (double)r;
        v.m[j] = mm;
        v.phout[j] = (R)(mm / (double)r);
        int kk = atomicAdd(&v.cnt[4], 1);
        if (kk < v.cap) v.nllist[kk] = (int)j;
        else atomicOr(v.err, ERRB_OVERFLOW);
      }
    }
  }
}

template <int P>
__global__ void k_share(Par p, View<P> v) {
  using R = typename Form<P>::R;
  int nf = min(load_count(&v.cnt[1]), v.cap), ne = min(load_count(&v.cnt[2]), v.cap);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nf + ne; k += gridDim.x * blockDim.x) {
    bool isF = k < nf;
    long long i = isF ? v.flist[k] : v.elist[k - nf];
    if (!isF && !(v.mark[i] & MK_EMPTY)) continue;
    int x, y, z;
    coords(p, i, x, y, z);
    double rho = (double)rho_out<P>(p, v, i);
    double ex = isF ? v.m[i] - rho : v.m[i];
    int nr = 0;
    unsigned rm = 0u;
#pragma unroll
    for (int q = 1; q < 19; ++q) {
      long long j = nbr(p, x, y, z, cx(q), cy(q), cz(q));
      if (j < 0) continue;
      uint8_t mk = ((volatile uint8_t*)v.mark)[j];
      uint8_t kj = v.flags[j] & KIND;
      bool recv = (mk & (MK_NEWG | MK_NEWL)) || (kj == IFC && !(mk & (MK_FILL | MK_EMPTY)));
      if (recv) { ++nr; rm |= 1u << q; }
    }
    if (nr == 0) {
      atomicAdd(v.lost, ex);
      v.share[i] = 0.0;
    } else {
      v.share[i] = ex / (double)nr;
    }
    v.m[i] = isF ? rho : 0.0;
#pragma unroll
    for (int q = 1; q < 19; ++q) {
      bool first = false;
      long long j = 0;
      if (rm & (1u << q)) {
        j = nbr(p, x, y, z, cx(q), cy(q), cz(q));
        uint8_t old = or_u8(v.mark, j, MK_RECV);
        first = !(old & MK_RECV);
      }
      push(first, v.rlist, &v.cnt[5], v.cap, (int)j, v.err);
    }
  }
}

template <int P>
__global__ void k_recv(Par p, View<P> v) {
  using R = typename Form<P>::R;
  int nr = min(load_count(&v.cnt[5]), v.cap);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nr; k += gridDim.x * blockDim.x) {
    long long yj = v.rlist[k];
    int x, y, z;
    coords(p, yj, x, y, z);
    double acc = 0.0;
#pragma unroll
    for (int q = 1; q < 19; ++q) {
      long long j = nbr(p, x, y, z, cx(q), cy(q), cz(q));
      if (j < 0) continue;
      if (v.mark[j] & (MK_FILL | MK_EMPTY)) acc += v.share[j];
    }
    double mm = v.m[yj] + acc;
    v.m[yj] = mm;
    R r = rho_out<P>(p, v, yj);
    v.phout[yj] = (R)(mm / (double)r);
  }
}

template <int P>
__global__ void k_final(Par p, View<P> v) {
  using R = typename Form<P>::R;
  int nf = min(load_count(&v.cnt[1]), v.cap), ne = min(load_count(&v.cnt[2]), v.cap);
  int ng = min(load_count(&v.cnt[3]), v.cap), nl = min(load_count(&v.cnt[4]), v.cap);
  int nr = min(load_count(&v.cnt[5]), v.cap);
  int total = nf + ne + ng + nl + nr;
  // running total of conversions since the state was set (never reset per step)
  if (blockIdx.x == 0 && threadIdx.x == 0 && nf + ng + nl) atomicAdd(&v.cnt[8], nf + ng + nl);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
    int kk = k;
    if (kk < nf) {
      long long i = v.flist[kk];
      v.flags[i] = (uint8_t)((v.flags[i] & NEARB) | LIQ);
      v.mark[i] = 0;
      continue;
    }
    kk -= nf;
    if (kk < ne) {
      long long i = v.elist[kk];
      if (v.mark[i] & MK_EMPTY) {
        v.flags[i] = (uint8_t)((v.flags[i] & NEARB) | GAS);
        v.phout[i] = R(0);
        v.mark[i] = 0;
        atomicAdd(&v.cnt[7], 1);
        atomicAdd(&v.cnt[8], 1);
      }
      continue;
    }
    kk -= ne;
    if (kk < ng) {
      long long i = v.nglist[kk];
      v.flags[i] = (uint8_t)((v.flags[i] & NEARB) | IFC);
      v.mark[i] = 0;
      continue;
    }
    kk -= ng;
    if (kk < nl) {
      long long i = v.nllist[kk];
      v.flags[i] = (uint8_t)((v.flags[i] & NEARB) | IFC);
      v.mark[i] = 0;
      continue;
    }
    kk -= nl;
    v.mark[v.rlist[kk]] = 0;
  }
}

// removed E cells keep a zero mark; receivers, new cells and F/E cells are
// cleared above.  E cells that left E in k_fill carry no mark bits besides a
// possible RECV (cleared through the receiver list).

template <int P>
int launch_conversions(const Par& p, const View<P>& v, cudaStream_t st, int list_blocks) {
  k_fill<P><<<list_blocks, 256, 0, st>>>(p, v);
  k_newg<P><<<list_blocks, 128, 0, st>>>(p, v);
  k_empty<P><<<list_blocks, 256, 0, st>>>(p, v);
  k_share<P><<<list_blocks, 256, 0, st>>>(p, v);
  k_recv<P><<<list_blocks, 256, 0, st>>>(p, v);
  k_final<P><<<list_blocks, 256, 0, st>>>(p, v);
  return (int)cudaGetLastError();
}

template int launch_conversions<P64>(const Par&, const View<P64>&, cudaStream_t, int);
template int launch_conversions<P32>(const Par&, const View<P32>&, cudaStream_t, int);
template int launch_conversions<P16>(const Par&, const View<P16>&, cudaStream_t, int);

}  // namespace fsl

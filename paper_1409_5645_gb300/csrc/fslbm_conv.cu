// fslbm_conv.cu -- cell conversions after the mass update (Sec. 2.3 / 4.4; the
// paper takes interface tracking from Koerner et al. and Thuerey).
//
// The step kernel appended interface cells with m > (1+eps) rho to the fill
// list F and those with m < -eps rho to the empty list E, and marked them.
// Then, all as list kernels (grid-stride; counts read on the device, no host
// synchronisation):
//   fill     gas neighbours of F become new interface (NEWG, listed once by an
//            atomic byte-OR)
//   empty    an E cell with an F neighbour leaves E (it stays interface);
//            liquid neighbours of the remaining E become interface (NEWL)
//   newg     NEWG cells get f = f^eq(mean rho, mean u) over their liquid /
//            interface neighbours (q order), collided, m = 0
//   newl     NEWL cells get m = rho
//   share    excess (F: m - rho, E: m) / number of receivers (interface after
//            the steps above, not converting); no receiver -> lost ledger
//   recv     each receiver gathers the shares of its converting neighbours in q
//            order (deterministic, no floating-point atomics)
//   final    F -> liquid, E -> gas, new cells -> interface, marks cleared
// fill and empty run together (each E cell tests its own neighbours for F
// marks, which the step kernel set), and so do newg, newl and share (share
// reads only the marks and claims of the first stage and the converting
// cells' own state).  The four stages run as one cooperative launch
// (k_convert, two resident blocks per SM, grid barriers between the stages)
// where the device allows it, else as four launches.  The result does not
// depend on list order.
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

// density of cell i at t+1 (summed in q order in the arithmetic type)
template <int P>
__device__ __forceinline__ double rho_out(const Par& p, const View<P>& v, long long i) {
  using R = typename Form<P>::R;
  R r = R(0);
#pragma unroll
  for (int q = 0; q < 19; ++q) r += ldq<P>(v.fout, (size_t)q * (size_t)p.N + (size_t)i, q);
  return rho_full<Form<P>::SH>(r);
}

// one warp per fill cell, lane q (1..18) takes link q
template <int P>
__device__ __forceinline__ void do_fill(const Par& p, const View<P>& v) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int nf = min(load_count(&v.cnt[1]), v.cap);
  const int q = (lane >= 1 && lane < 19) ? lane : 0;
  for (int k = gw; k < nf; k += nw) {
    const long long i = FSL_CK(p, v.flist[k], p.N);
    int x, y, z;
    coords(p, i, x, y, z);
    bool won = false;
    long long j = -1;
    if (q) {
      j = nbr(p, x, y, z, cx(q), cy(q), cz(q));
      const uint8_t kj = j < 0 ? (uint8_t)WALL : (uint8_t)(v.flags[j] & KIND);
      if (kj == GAS) {
        const uint8_t old = or_u8(v.mark, j, MK_NEWG);
        won = !(old & MK_NEWG);  // the first claimant lists the new cell
      }
    }
    push(won, v.nglist, &v.cnt[3], v.cap, (int)j, v.err);
  }
}
template <int P>
__device__ __forceinline__ void do_empty(const Par& p, const View<P>& v);
template <int P>
__global__ void __launch_bounds__(256) k_fill_empty(Par p, View<P> v) {
  pdl_begin();
  do_fill<P>(p, v);
  do_empty<P>(p, v);
}

// one warp per new cell: lane l (1..18) reads neighbour l's populations; the
// means are summed in neighbour order; lane q builds and collides population q
template <int P>
__device__ __forceinline__ void do_newg(const Par& p, const View<P>& v) {
  using R = typename Form<P>::R;
  const unsigned FULL = 0xffffffffu;
  const size_t N = (size_t)p.N;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int nn = min(load_count(&v.cnt[3]), v.cap);
  const int q = lane < 19 ? lane : 0;
  for (int k = gw; k < nn; k += nw) {
    const long long j = FSL_CK(p, v.nglist[k], p.N);
    int x, y, z;
    coords(p, j, x, y, z);
    bool use = false;
    R rr = R(0), ux = R(0), uy = R(0), uz = R(0);
    if (lane >= 1 && lane < 19) {
      long long y2 = nbr(p, x, y, z, cx(q), cy(q), cz(q));
      if (y2 >= 0) {
        // the populations are loaded beside the flag (a gas cell's are read and dropped)
        R g[19];
#pragma unroll
        for (int r = 0; r < 19; ++r) g[r] = ldq<P>(v.fout, (size_t)r * N + (size_t)y2, r);
        use = is_fluid(v.flags[y2] & KIND);
        if (use) moments_post<R, Form<P>::SH>(p, g, rr, ux, uy, uz);
      }
    }
    R rs = R(0), s0 = R(0), s1 = R(0), s2 = R(0);
    int c = 0;
#pragma unroll
    for (int l = 1; l < 19; ++l) {
      const bool ul = __shfl_sync(FULL, use, l);
      const R a = __shfl_sync(FULL, rr, l), b0 = __shfl_sync(FULL, ux, l);
      const R b1 = __shfl_sync(FULL, uy, l), b2 = __shfl_sync(FULL, uz, l);
      if (ul) { rs += a; s0 += b0; s1 += b1; s2 += b2; ++c; }
    }
    // (rbar is rho - 1 in the shifted forms: the mean of rho - 1)
    const R rbar = rs / R(c), u0 = s0 / R(c), u1 = s1 / R(c), u2 = s2 / R(c);
    const R r0 = p.compressible ? rho_full_r<Form<P>::SH>(rbar) : R(1);
    const R usq = u0 * u0 + u1 * u1 + u2 * u2;
    const R wq_ = q == 0 ? R(1) / R(3) : (q <= 6 ? R(1) / R(18) : R(1) / R(36));
    // f^eq(rbar, ubar) with u^eq = ubar
    const R f = eplus_q<R>(p, q, rbar, r0, u0, u1, u2, usq) +
                R(3) * wq_ * r0 * (R(cx(q)) * u0 + R(cy(q)) * u1 + R(cz(q)) * u2);
    // collision (Eq. lbe2) of the new cell, lane q -> population q
    const R f19 = lane < 19 ? f : R(0);
    R rho = f19, jx = R(cx(q)) * f19, jy = R(cy(q)) * f19, jz = R(cz(q)) * f19;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      rho += __shfl_xor_sync(FULL, rho, o);
      jx += __shfl_xor_sync(FULL, jx, o);
      jy += __shfl_xor_sync(FULL, jy, o);
      jz += __shfl_xor_sync(FULL, jz, o);
    }
    const R rc = p.compressible ? rho_full_r<Form<P>::SH>(rho) : R(1);
    const R Ux = jx / rc, Uy = jy / rc, Uz = jz / rc;
    const R gx = R(p.g[0]), gy = R(p.g[1]), gz = R(p.g[2]);
    const R vx_ = Ux + R(0.5) * gx, vy_ = Uy + R(0.5) * gy, vz_ = Uz + R(0.5) * gz;
    const R ilm = R(1) / R(p.lam_m);
    const R ex = Ux - gx * ilm, ey = Uy - gy * ilm, ez = Uz - gz * ilm;
    const R usq2 = vx_ * vx_ + vy_ * vy_ + vz_ * vz_;
    const R fb = __shfl_sync(FULL, f, inv(q));
    const R ep = eplus_q<R>(p, q, rho, rc, vx_, vy_, vz_, usq2);
    const R em = R(3) * wq_ * rc * (R(cx(q)) * ex + R(cy(q)) * ey + R(cz(q)) * ez);
    const R out = f + R(p.lam_p) * (R(0.5) * (f + fb) - ep) + R(p.lam_m) * (R(0.5) * (f - fb) - em);
    if (lane < 19) stq<P>(v.fout, (size_t)q * N + (size_t)j, q, out);
    if (lane == 0) {
      v.m[j] = 0.0;
      v.phout[j] = R(0);
    }
  }
}

// one warp per empty cell still marked, lane q (1..18) takes link q
template <int P>
__device__ __forceinline__ void do_empty(const Par& p, const View<P>& v) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int ne = min(load_count(&v.cnt[2]), v.cap);
  const int q = (lane >= 1 && lane < 19) ? lane : 0;
  for (int k = gw; k < ne; k += nw) {
    const long long i = FSL_CK(p, v.elist[k], p.N);
    if (!(v.mark[i] & MK_EMPTY)) continue;  // warp-uniform
    int x, y, z;
    coords(p, i, x, y, z);
    long long j = -1;
    uint8_t kj = WALL, mj = 0;
    if (q) {
      j = nbr(p, x, y, z, cx(q), cy(q), cz(q));
      if (j >= 0) {
        kj = v.flags[j] & KIND;
        mj = v.mark[j];
      }
    }
    // an emptied cell next to a filled one stays interface
    if (__any_sync(0xffffffffu, (mj & MK_FILL) != 0)) {
      if (lane == 0) clear_u8(v.mark, i, MK_EMPTY);
      continue;  // (warp-uniform)
    }
    bool won = false;
    if (kj == LIQ) {
      const uint8_t old = or_u8(v.mark, j, MK_NEWL);
      won = !(old & MK_NEWL);  // the first claimant lists it; newl sets m = rho
    }
    push(won, v.nllist, &v.cnt[4], v.cap, (int)j, v.err);
  }
}

// liquid cells turned interface next to an emptied cell: m = rho, phi = m/rho
template <int P>
__device__ __forceinline__ void do_newl(const Par& p, const View<P>& v) {
  using R = typename Form<P>::R;
  int nl = min(load_count(&v.cnt[4]), v.cap);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nl; k += gridDim.x * blockDim.x) {
    long long j = FSL_CK(p, v.nllist[k], p.N);
    const double r = rho_out<P>(p, v, j);
    v.m[j] = r;
    v.phout[j] = (R)(r / r);
  }
}

// Fill-level normal of a converting cell for the weighted excess split
// (Thuerey's distribution along the interface normal): n = -grad phi by
// central differences, n_a = (phi(x - e_a) - phi(x + e_a)) / 2, pointing into
// the gas, from the fill levels after the mass exchange (liquid 1, gas 0,
// interface m/rho as k_iface stored it, the cell's own value across a wall or
// a face).  The flags are those of time t until k_final.
template <int P>
__device__ __forceinline__ double phi_star(const Par& p, const View<P>& v, long long j, double own) {
  if (j < 0) return own;
  const uint8_t k = v.flags[j] & KIND;
  return k == LIQ ? 1.0 : (k == GAS ? 0.0 : (k == IFC ? (double)v.phout[j] : own));
}
template <int P>
__device__ __forceinline__ void fill_normal(const Par& p, const View<P>& v, long long i, double (&n)[3]) {
  int x, y, z;
  coords(p, i, x, y, z);
  const double own = (double)v.phout[i];
  n[0] = 0.5 * (phi_star<P>(p, v, nbr(p, x, y, z, -1, 0, 0), own) - phi_star<P>(p, v, nbr(p, x, y, z, 1, 0, 0), own));
  n[1] = 0.5 * (phi_star<P>(p, v, nbr(p, x, y, z, 0, -1, 0), own) - phi_star<P>(p, v, nbr(p, x, y, z, 0, 1, 0), own));
  n[2] = 0.5 * (phi_star<P>(p, v, nbr(p, x, y, z, 0, 0, -1), own) - phi_star<P>(p, v, nbr(p, x, y, z, 0, 0, 1), own));
}
// weight of the neighbour along c (components -1, 0, 1, so the products are
// exact and the sum is the same in any contraction): a filled cell pushes its
// excess toward the gas (n.c > 0), an emptied cell draws its deficit from the
// liquid side (n.c < 0)
__device__ __forceinline__ double split_weight(const double (&n)[3], int ax, int ay, int az, bool filled) {
  const double d = (double)ax * n[0] + (double)ay * n[1] + (double)az * n[2];
  return filled ? (d > 0.0 ? d : 0.0) : (d < 0.0 ? -d : 0.0);
}

// one warp per fill / empty cell: lane q (1..18) tests neighbour q as a
// receiver; lane 0 computes the share (rho summed in q order, as a thread would)
template <int P>
__device__ __forceinline__ void do_share(const Par& p, const View<P>& v) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int nf = min(load_count(&v.cnt[1]), v.cap), ne = min(load_count(&v.cnt[2]), v.cap);
  const int q = (lane >= 1 && lane < 19) ? lane : 0;
  for (int k = gw; k < nf + ne; k += nw) {
    const bool isF = k < nf;
    const long long i = FSL_CK(p, isF ? v.flist[k] : v.elist[k - nf], p.N);
    if (!isF && !(v.mark[i] & MK_EMPTY)) continue;  // warp-uniform
    int x, y, z;
    coords(p, i, x, y, z);
    // lane 0: the cell's density and mass, loaded beside the neighbour tests
    double rho = 0.0, mi = 0.0;
    if (lane == 0) {
      rho = rho_out<P>(p, v, i);
      mi = v.m[i];
    }
    bool recv = false;
    long long j = -1;
    if (q) {
      j = nbr(p, x, y, z, cx(q), cy(q), cz(q));
      if (j >= 0) {
        const uint8_t mk = ((volatile uint8_t*)v.mark)[j];
        const uint8_t kj = v.flags[j] & KIND;
        recv = (mk & (MK_NEWG | MK_NEWL)) || (kj == IFC && !(mk & (MK_FILL | MK_EMPTY)));
      }
    }
    const unsigned rm = __ballot_sync(FULL, recv);
    // weighted split: the receivers' weights summed in q order on lane 0
    double V = 0.0;
    if (p.excess_split && rm) {
      double n[3];
      fill_normal<P>(p, v, i, n);  // (every lane: the same few loads)
      const double w = recv ? split_weight(n, cx(q), cy(q), cz(q), isF) : 0.0;
      for (int s = 1; s < 19; ++s) V += __shfl_sync(FULL, w, s);
    }
    if (lane == 0) {
      const double ex = isF ? mi - rho : mi;
      const int nr = __popc(rm);
      if (nr == 0) {
        if (owned(p, x, y, z)) atomicAdd(v.lost, ex);  // (a ghost cell's owner books it)
        v.share[i] = 0.0;
      } else if (V > 1e-12) {
        v.share[i] = ex / V;
        v.mark[i] = (uint8_t)(v.mark[i] | MK_WSPLIT);
      } else {
        v.share[i] = ex / (double)nr;  // equal split (also where no receiver lies along the normal)
      }
      v.m[i] = isF ? rho : 0.0;
    }
    bool first = false;
    if (recv) {
      const uint8_t old = or_u8(v.mark, j, MK_RECV);
      first = !(old & MK_RECV);
    }
    push(first, v.rlist, &v.cnt[5], v.cap, (int)j, v.err);
  }
}

// new cells from gas, new cells from liquid and the excess shares are
// independent once the first stage has claimed the new cells and settled the
// empty list
template <int P>
__global__ void __launch_bounds__(256) k_new_share(Par p, View<P> v) {
  pdl_begin();
  do_newg<P>(p, v);
  do_newl<P>(p, v);
  do_share<P>(p, v);
}

// one thread per receiver (the lists are long late in a run): gathers the
// shares of its converting neighbours in q order (deterministic)
template <int P>
__device__ __forceinline__ void do_recv(const Par& p, const View<P>& v) {
  using R = typename Form<P>::R;
  const int nr = min(load_count(&v.cnt[5]), v.cap);
  const long long sy = p.nx, sz = (long long)p.nx * p.ny;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nr; k += gridDim.x * blockDim.x) {
    const long long yj = FSL_CK(p, v.rlist[k], p.N);
    int x, y, z;
    coords(p, yj, x, y, z);
    const bool in1 = x >= 1 && x < p.nx - 1 && y >= 1 && y < p.ny - 1 && z >= 1 && z < p.nz - 1;
    // the receiver's own mass and density first: their loads overlap the
    // neighbours' marks and shares
    const double m0 = v.m[yj];
    const double rho = p.excess_split ? 1.0 : rho_out<P>(p, v, yj);
    double acc = 0.0;
#pragma unroll
    for (int q = 1; q < 19; ++q) {
      const long long j = in1 ? yj + (cx(q) + sy * cy(q) + sz * cz(q)) : nbr(p, x, y, z, cx(q), cy(q), cz(q));
      if (j < 0) continue;
      const uint8_t mk = v.mark[j];
      if (mk & (MK_FILL | MK_EMPTY)) {
        if (mk & MK_WSPLIT) {  // the link from j to this receiver is -c_q
          double n[3];
          fill_normal<P>(p, v, j, n);
          acc += v.share[j] * split_weight(n, -cx(q), -cy(q), -cz(q), (mk & MK_FILL) != 0);
        } else {
          acc += v.share[j];
        }
      }
    }
    const double mm = m0 + acc;
    v.m[yj] = mm;
    // (the weighted split reads the fill levels of interface cells here, so
    // its receivers take their new fill level in k_final)
    if (!p.excess_split) {
      v.phout[yj] = (R)(mm / rho);
    }
  }
}

template <int P>
__global__ void __launch_bounds__(256) k_recv(Par p, View<P> v) {
  pdl_begin();
  do_recv<P>(p, v);
}

template <int P>
__device__ __forceinline__ void do_final(const Par& p, const View<P>& v) {
  using R = typename Form<P>::R;
  int nf = min(load_count(&v.cnt[1]), v.cap), ne = min(load_count(&v.cnt[2]), v.cap);
  int ng = min(load_count(&v.cnt[3]), v.cap), nl = min(load_count(&v.cnt[4]), v.cap);
  int nr = min(load_count(&v.cnt[5]), v.cap);
  int total = nf + ne + ng + nl + nr;
  // running total of conversions since the state was set (never reset per step)
  if (blockIdx.x == 0 && threadIdx.x == 0 && nf + ng + nl) atomicAdd(&v.cnt[8], nf + ng + nl);
  int emptied = 0;  // cells this thread turned to gas (counted once per warp below)
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
    int kk = k;
    if (kk < nf) {
      long long i = FSL_CK(p, v.flist[kk], p.N);
      v.flags[i] = (uint8_t)((v.flags[i] & STATIC_BITS) | LIQ);
      v.mark[i] = 0;
      continue;
    }
    kk -= nf;
    if (kk < ne) {
      long long i = FSL_CK(p, v.elist[kk], p.N);
      if (v.mark[i] & MK_EMPTY) {
        v.flags[i] = (uint8_t)((v.flags[i] & STATIC_BITS) | GAS);
        v.phout[i] = R(0);
        v.mark[i] = 0;
        ++emptied;
      }
      continue;
    }
    kk -= ne;
    if (kk < ng) {
      long long i = FSL_CK(p, v.nglist[kk], p.N);
      v.flags[i] = (uint8_t)((v.flags[i] & STATIC_BITS) | IFC);
      v.mark[i] = 0;
      continue;
    }
    kk -= ng;
    if (kk < nl) {
      long long i = FSL_CK(p, v.nllist[kk], p.N);
      v.flags[i] = (uint8_t)((v.flags[i] & STATIC_BITS) | IFC);
      v.mark[i] = 0;
      continue;
    }
    kk -= nl;
    const long long r = FSL_CK(p, v.rlist[kk], p.N);
    v.mark[r] = 0;
    if (p.excess_split) v.phout[r] = (R)(v.m[r] / rho_out<P>(p, v, r));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) emptied += __shfl_down_sync(0xffffffffu, emptied, o);
  if ((threadIdx.x & 31) == 0 && emptied) {
    atomicAdd(&v.cnt[7], emptied);
    atomicAdd(&v.cnt[8], emptied);
  }
}

template <int P>
__global__ void __launch_bounds__(256) k_final(Par p, View<P> v) {
  pdl_begin();
  do_final<P>(p, v);
}

// removed E cells keep a zero mark; receivers, new cells and F/E cells are
// cleared above.  E cells that left E in k_fill carry no mark bits besides a
// possible RECV (cleared through the receiver list).

// Grid-wide barrier of the fused conversion kernel (a cooperative launch, so
// every block is resident): thread 0 of each block arrives on the per-step
// counter cnt[10] and waits until the blocks of this phase have arrived.  The
// wait is bounded (about a second); on expiry it records ERRB_SYNC and goes
// on, the step's result is then invalid and the host reports the error.
__device__ __forceinline__ void grid_sync(unsigned* ctr, unsigned target, int* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(ctr, 1u);
    unsigned spins = 0;
    while (*((volatile unsigned*)ctr) < target) {
      if (++spins > (1u << 20)) {
        atomicOr(err, ERRB_SYNC);
        break;
      }
      __nanosleep(100);
    }
    __threadfence();
  }
  __syncthreads();
}

// the four conversion stages in one launch, separated by grid barriers; the
// step's two-level mass reduction rides along in the first two stages (the
// same chunks and order as the stand-alone reduction), with the lost ledger
// read before any excess of this step reaches it
template <int P>
__global__ void __launch_bounds__(256) k_convert(Par p, View<P> v, MassReduce mr) {
  pdl_begin();
  unsigned* ctr = (unsigned*)&v.cnt[10];
  const unsigned nb = gridDim.x;
  double lost0 = 0.0;
  if (mr.nb > 0 && blockIdx.x == 0 && threadIdx.x == 0) lost0 = *mr.add;
  if ((int)blockIdx.x < mr.nb) {
    const double t = block_chunk_sum(mr.in, mr.n, mr.chunk, blockIdx.x);
    if (threadIdx.x == 0) mr.tmp[blockIdx.x] = t;
  }
  do_fill<P>(p, v);
  do_empty<P>(p, v);
  grid_sync(ctr, nb, v.err);
  if (mr.nb > 0 && blockIdx.x == 0) {
    const double t = block_chunk_sum(mr.tmp, mr.nb, mr.nb, 0);
    if (threadIdx.x == 0) *mr.out = t + lost0;
  }
  do_newg<P>(p, v);
  do_newl<P>(p, v);
  do_share<P>(p, v);
  grid_sync(ctr, 2 * nb, v.err);
  do_recv<P>(p, v);
  grid_sync(ctr, 3 * nb, v.err);
  do_final<P>(p, v);
}

// self-check of the barrier: one grid_sync waiting for `extra` blocks more
// than the grid has (extra = 1: nothing completes it, the bounded wait runs out)
__global__ void __launch_bounds__(256) k_barrier_check(unsigned* ctr, unsigned extra, int* err) {
  grid_sync(ctr, gridDim.x + extra, err);
}

int launch_barrier_check(unsigned* ctr, int* err, int blocks, unsigned extra, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(256);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return (int)cudaLaunchKernelEx(&cfg, k_barrier_check, ctr, extra, err);
}

// resident blocks of k_convert per SM (0: the fused kernel cannot be used)
template <int P>
int convert_blocks_per_sm() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_convert<P>, 256, 0) != cudaSuccess) return 0;
  return nb;
}

// coop_blocks > 0: the fused cooperative kernel on that many blocks (all
// resident); else four launches of list_blocks
template <int P>
int launch_conversions(const Par& p, const View<P>& v, cudaStream_t st, int list_blocks, int coop_blocks,
                       const MassReduce& mr) {
  if (coop_blocks > 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(coop_blocks);
    cfg.blockDim = dim3(256);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (mr.nb > coop_blocks) return (int)cudaErrorInvalidValue;
    return (int)cudaLaunchKernelEx(&cfg, k_convert<P>, p, v, mr);
  }
  void (*ks[4])(Par, View<P>) = {k_fill_empty<P>, k_new_share<P>, k_recv<P>, k_final<P>};
  for (auto k : ks)
    if (launch_k(k, list_blocks, 256, 0, st, p, v)) return 1;
  return 0;
}

template int launch_conversions<P64>(const Par&, const View<P64>&, cudaStream_t, int, int, const MassReduce&);
template int launch_conversions<P32>(const Par&, const View<P32>&, cudaStream_t, int, int, const MassReduce&);
template int launch_conversions<P16>(const Par&, const View<P16>&, cudaStream_t, int, int, const MassReduce&);
template int convert_blocks_per_sm<P64>();
template int convert_blocks_per_sm<P32>();
template int convert_blocks_per_sm<P16>();

}  // namespace fsl

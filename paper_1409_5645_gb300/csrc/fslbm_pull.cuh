// fslbm_pull.cuh -- device helpers of the stream step shared by the bulk
// kernels: the warp-aggregated list append, the general pull next to walls,
// faces and gas, and the wall closures.
#pragma once
#include "fslbm_dev.cuh"

namespace fsl {

// ---------------------------------------------------------------------------
// warp-aggregated append of `pred` lanes' values to list[*count ...]
// (all 32 lanes of the warp must call it)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void warp_append(bool pred, int value, int* list, int* count, int cap, int* err) {
  unsigned bal = __ballot_sync(0xffffffffu, pred);
  if (!bal) return;
  int lane = threadIdx.x & 31;
  int leader = __ffs(bal) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(count, __popc(bal));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (pred) {
    int k = base + __popc(bal & ((1u << lane) - 1u));
    if (k < cap) list[k] = value;
    else atomicOr(err, ERRB_OVERFLOW);
  }
}

// ---------------------------------------------------------------------------
// General pull for a cell next to a wall, a face or gas.  Fills f[q] from
// fluid sources and returns masks of wall and gas sources.
// ---------------------------------------------------------------------------
template <int P, bool IN = false>
__device__ __forceinline__ void pull_general(const Par& p, const View<P>& v, int x, int y, int z,
                                             typename Form<P>::R (&f)[19], unsigned& wallm, unsigned& gasm,
                                             unsigned* liqm = nullptr, int* srcs = nullptr) {
  const size_t N = (size_t)p.N;
  wallm = 0u;
  gasm = 0u;
  unsigned lm = 0u;
  // away from the faces the sources are plain offsets
  // (IN: the caller knows the cell is at least one cell away from every face)
  const bool in1 = IN || (x >= 1 && x < p.nx - 1 && y >= 1 && y < p.ny - 1 && z >= 1 && z < p.nz - 1);
  const long long i = (long long)x + (long long)p.nx * ((long long)y + (long long)p.ny * z);
  const long long sy = p.nx, sz = (long long)p.nx * p.ny;
  if constexpr (IN) {
    // every source lies inside the lattice: issue the population and flag
    // loads together (a gas source's stale populations are read and dropped)
#pragma unroll
    for (int q = 1; q < 19; ++q) {
      const long long s = i - (cx(q) + sy * cy(q) + sz * cz(q));
      const uint8_t ks = v.flags[s] & KIND;
      const typename Form<P>::R fq = ldq<P>(v.fin, (size_t)q * N + (size_t)s, q);
      if (is_fluid(ks)) {
        f[q] = fq;
        if (ks == LIQ) lm |= 1u << q;
      } else if (ks == WALL) { wallm |= 1u << q; f[q] = 0; }
      else { gasm |= 1u << q; f[q] = 0; }
    }
  } else {
    // a lattice without periodic axes: a source past a face is a wall
    const bool bounded = !p.px && !p.py && !p.pz;
#pragma unroll
    for (int q = 1; q < 19; ++q) {
      long long s;
      if (in1) {
        s = i - (cx(q) + sy * cy(q) + sz * cz(q));
      } else if (bounded) {
        const bool inside = (unsigned)(x - cx(q)) < (unsigned)p.nx && (unsigned)(y - cy(q)) < (unsigned)p.ny &&
                            (unsigned)(z - cz(q)) < (unsigned)p.nz;
        s = inside ? i - (cx(q) + sy * cy(q) + sz * cz(q)) : -1;
      } else {
        s = nbr(p, x, y, z, -cx(q), -cy(q), -cz(q));
      }
      uint8_t ks = kind_at(v.flags, s);
      if (srcs) srcs[q] = (int)s;
      if (is_fluid(ks)) {
        f[q] = ldq<P>(v.fin, (size_t)q * N + (size_t)s, q);
        if (ks == LIQ) lm |= 1u << q;
      } else if (ks == WALL) { wallm |= 1u << q; f[q] = 0; }
      else { gasm |= 1u << q; f[q] = 0; }
    }
  }
  if (liqm) *liqm = lm;
}

// Wall closure for the links in wallm (needs the cell's own f~ and the
// pulled values): half-way bounce-back f_q = f~_p(x), p = qbar, or CLI with
// kappa = (1 - 2 dw)/(1 + 2 dw): f_q = f~_p(x) + kappa (f~_p(x - c_p) - f~_q(x)),
// where f~_p(x - c_p) is the value pulled along p (used only if that source is
// fluid).
template <int P>
__device__ __forceinline__ void wall_links(const Par& p, const View<P>& v, long long i, unsigned wallm,
                                           unsigned gasm, const typename Form<P>::R (&own)[19],
                                           typename Form<P>::R (&f)[19]) {
  using R = typename Form<P>::R;
  const size_t N = (size_t)p.N;
#pragma unroll
  for (int q = 1; q < 19; ++q) {
    if (!(wallm & (1u << q))) continue;
    const int pq = inv(q);
    R val = own[pq];
    if (p.has_wd) {
      R dw = (R)v.wd[(size_t)pq * N + (size_t)i];
      bool up_fluid = !((wallm | gasm) & (1u << pq));
      if (dw >= R(0) && up_fluid) {
        R kap = (R(1) - R(2) * dw) / (R(1) + R(2) * dw);
        val = val + kap * (f[pq] - own[q]);
      }
    } else if (p.has_uw) {
      // moving wall (half-way bounce-back): + 6 w_q rho_0 (c_q.u_w), rho_0 = 1
      val = val + R(6) * wq<R>(q) *
                      (R(cx(q)) * R(p.wall_u[0]) + R(cy(q)) * R(p.wall_u[1]) + R(cz(q)) * R(p.wall_u[2]));
    }
    f[q] = val;
  }
}

}  // namespace fsl

// fslbm_step.cuh -- the stream-collide kernels of one FSLBM time step (the
// segment scan k_segments, which lists the step's segments and interface
// cells before them, is in fslbm_step.cu).
//
// k_bulk   every warp walks the segment list on its own, one lane per cell.
//          Liquid cells pull their 19 populations (Eq. lbe1), apply half-way
//          bounce-back / CLI at walls, collide (Eq. lbe2) and store.  The
//          liquid density is reduced per warp for the mass balance.
// k_iface  one thread per interface cell (grid-stride over the list): pulls,
//          rebuilds the populations arriving from gas cells by the FSK rule
//          (Eq. koerner) or the FSL rule (Eq. closure, Table 1, D = 0) with the
//          link fraction from the height-function plane (Sec. 2.2, Sec. 5),
//          exchanges mass with its neighbours (Sec. 2.3), collides, stores, and
//          marks fill / empty conversions into compact lists.
//
// Templates over the precision form; each fslbm_step_p*.cu instantiates
// the launcher for one form, so that the forms compile in parallel.
#pragma once
#include "fslbm_dev.cuh"
#include "fslbm_kernels.h"
#include "fslbm_pull.cuh"

namespace fsl {

// ---------------------------------------------------------------------------
// k_bulk: every warp walks the segment list on its own (no block barrier),
// one lane per cell; the liquid density is summed per warp.
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(128, (P == P64 ? 4 : 8)) k_bulk(Par p, View<P> v, const int* __restrict__ seglist,
                                              const int* __restrict__ segcount) {
  pdl_begin();
  using R = typename Form<P>::R;
  const int nseg = *((volatile const int*)segcount);
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  double msum = 0.0;
  for (int si = gw; si < nseg; si += nw) {
    const int4 sd = reinterpret_cast<const int4*>(seglist)[si];  // x0, y, z, first cell
    const int x = sd.x + lane, y = sd.y, z = sd.z;
    const bool in = x < p.nx;
    const long long i = FSL_CK_IF(p, in, (long long)sd.w + lane, p.N);
    const uint8_t fl = in ? v.flags[i] : (uint8_t)GAS;
    const uint8_t k = fl & KIND;
    const size_t N = (size_t)p.N;
    R f[19];
    // Fast path: every source is a fluid cell at a plain offset, or lies beyond
    // a non-periodic face (half-way bounce-back f_q = f~_qbar(x), read by
    // selecting the cell's own slot).  Cells next to a WALL cell, on a
    // periodic face, or with CLI link fractions take the general path.
    const bool ax0 = x == 0, ax1 = x == p.nx - 1, ay0 = y == 0, ay1 = y == p.ny - 1, az0 = z == 0,
               az1 = z == p.nz - 1;
    const bool onface = ax0 || ax1 || ay0 || ay1 || az0 || az1;
    const bool fast = k == LIQ &&
                      ((p.has_wd || p.has_uw) ? !(fl & NEARB) && !onface
                                : !(fl & NEARW) && !((ax0 || ax1) && p.px) && !((ay0 || ay1) && p.py) &&
                                      !((az0 || az1) && p.pz));
    const bool face_warp = __any_sync(0xffffffffu, fast && onface);
    if (k != LIQ) continue;
    if (fast && !face_warp) {
      const long long sy = p.nx, sz = (long long)p.nx * p.ny;
#define FSL_LD(q) \
  f[q] = ld<P, q>(v.fin, (size_t)q * N + (size_t)FSL_CK(p, i - (cx(q) + sy * cy(q) + sz * cz(q)), p.N));
      FSL_LD(0) FSL_LD(1) FSL_LD(2) FSL_LD(3) FSL_LD(4) FSL_LD(5) FSL_LD(6) FSL_LD(7) FSL_LD(8)
      FSL_LD(9) FSL_LD(10) FSL_LD(11) FSL_LD(12) FSL_LD(13) FSL_LD(14) FSL_LD(15) FSL_LD(16)
      FSL_LD(17) FSL_LD(18)
#undef FSL_LD
    } else if (fast) {
      const long long sy = p.nx, sz = (long long)p.nx * p.ny;
#define FSL_LDF(q)                                                                                              \
  {                                                                                                             \
    const bool bb = (cx(q) == 1 && ax0) || (cx(q) == -1 && ax1) || (cy(q) == 1 && ay0) || (cy(q) == -1 && ay1) || \
                    (cz(q) == 1 && az0) || (cz(q) == -1 && az1);                                                \
    const size_t k_ = bb ? (size_t)inv(q) * N + (size_t)i                                                       \
                         : (size_t)q * N + (size_t)FSL_CK(p, i - (cx(q) + sy * cy(q) + sz * cz(q)), p.N);      \
    f[q] = bb ? ld<P, inv(q)>(v.fin, k_) : ld<P, q>(v.fin, k_);                                                 \
  }
      f[0] = ld<P, 0>(v.fin, (size_t)i);
      FSL_LDF(1) FSL_LDF(2) FSL_LDF(3) FSL_LDF(4) FSL_LDF(5) FSL_LDF(6) FSL_LDF(7) FSL_LDF(8)
      FSL_LDF(9) FSL_LDF(10) FSL_LDF(11) FSL_LDF(12) FSL_LDF(13) FSL_LDF(14) FSL_LDF(15) FSL_LDF(16)
      FSL_LDF(17) FSL_LDF(18)
#undef FSL_LDF
    } else {
      unsigned wallm, gasm;
      f[0] = ld<P, 0>(v.fin, (size_t)i);
      pull_general<P>(p, v, x, y, z, f, wallm, gasm);
      if (gasm) atomicOr(v.err, ERRB_STATE);  // liquid must not touch gas
      wallm |= gasm;
      if (wallm) {
        R own[19];
#pragma unroll
        for (int q = 0; q < 19; ++q) own[q] = ldq<P>(v.fin, (size_t)q * N + (size_t)i, q);
        wall_links<P>(p, v, i, wallm, 0u, own, f);
      }
    }
    R rho, ux, uy, uz;
    collide<R, Form<P>::SH>(p, f, rho, ux, uy, uz);
    if (rho_bad<Form<P>::SH>(rho)) atomicOr(v.err, ERRB_UNSTABLE);
    if (speed_bad(p, ux, uy, uz)) atomicOr(v.err, ERRB_SPEED);
#define FSL_ST(q) st<P, q>(v.fout, (size_t)q * N + (size_t)i, f[q]);
    FSL_ST(0) FSL_ST(1) FSL_ST(2) FSL_ST(3) FSL_ST(4) FSL_ST(5) FSL_ST(6) FSL_ST(7) FSL_ST(8)
    FSL_ST(9) FSL_ST(10) FSL_ST(11) FSL_ST(12) FSL_ST(13) FSL_ST(14) FSL_ST(15) FSL_ST(16)
    FSL_ST(17) FSL_ST(18)
#undef FSL_ST
    if (owned(p, x, y, z)) msum += rho_full<Form<P>::SH>(rho);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) msum += __shfl_down_sync(0xffffffffu, msum, o);
  if (lane == 0) v.partials[gw] = msum;
}

// ---------------------------------------------------------------------------
// k_iface
// ---------------------------------------------------------------------------
// The work of one interface cell (pull, mass exchange, wall and gas-link
// closures, collision, store, fill/empty marks); returns its mass m.  IN:
// every cell within 3 of it lies inside the lattice, so all stencil offsets
// are plain (the hot path, kept apart from the face and wrap logic).
// Velocity of a fluid cell from its stored post-collision populations
// (sum_q c_q f~_q = rho_0 U + F, u = U + F/(2 rho_0)); only the FSL closure
// with u_b extrapolated along the link calls it (the extended k_iface instance).
template <class R>
struct Vel3 {
  R x, y, z;
};
template <int P>
__device__ __forceinline__ Vel3<typename Form<P>::R> cell_velocity(const typename Form<P>::S* __restrict__ fin,
                                                                 size_t N, size_t s, int compressible, double gx,
                                                                 double gy, double gz) {
  using R = typename Form<P>::R;
  R r = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
  for (int q = 0; q < 19; ++q) {
    const R fq = ldq<P>(fin, (size_t)q * N + s, q);
    r += fq;
    if (cx(q)) jx += R(cx(q)) * fq;
    if (cy(q)) jy += R(cy(q)) * fq;
    if (cz(q)) jz += R(cz(q)) * fq;
  }
  const R ir0 = compressible ? R(1) / rho_full_r<Form<P>::SH>(r) : R(1);
  return Vel3<R>{jx * ir0 - R(0.5) * R(gx), jy * ir0 - R(0.5) * R(gy), jz * ir0 - R(0.5) * R(gz)};
}

template <int P, bool IN, bool EXT>
__device__ __forceinline__ double iface_cell(const Par& p, const View<P>& v, int li, long long i, int x, int y,
                                             int z, bool& fill, bool& empty) {
  using R = typename Form<P>::R;
  const size_t N = (size_t)p.N;
  R own[19], f[19];
#pragma unroll
  for (int q = 0; q < 19; ++q) own[q] = ldq<P>(v.fin, (size_t)q * N + (size_t)i, q);
  constexpr bool SH = Form<P>::SH;
  R rt, utx, uty, utz;  // rt: rho(t), or rho(t) - 1 in the shifted forms
  moments_post<R, SH>(p, own, rt, utx, uty, utz);
  f[0] = own[0];
  unsigned wallm, gasm, liqm;
  int srcs[19];  // sources of the pull (only kept off the interior path)
  pull_general<P, IN>(p, v, x, y, z, f, wallm, gasm, &liqm, IN ? nullptr : srcs);
  const long long sy = p.nx, sz = (long long)p.nx * p.ny;
  const R phic = v.phin[i];
  // mass exchange (Sec. 2.3) with the pulled values, before any rebuild
  double dm = 0.0;
  if (!p.freeze) {
#pragma unroll
    for (int q = 1; q < 19; ++q) {
      if ((wallm | gasm) & (1u << q)) continue;
      const long long sq = IN ? i - (cx(q) + sy * cy(q) + sz * cz(q)) : (long long)srcs[q];
      const R phs = v.phin[sq];  // (loaded whatever the kind, so the loads overlap)
      R sw = (liqm & (1u << q)) ? R(1) : R(0.5) * (phic + phs);
      dm += (double)(sw * (f[q] - own[inv(q)]));
    }
  }
  if (wallm) wall_links<P>(p, v, i, wallm, gasm, own, f);
  if (gasm || (EXT && p.recon_nc)) {
    // the plane and curvature of k_geom (FSK without surface tension, the
    // boundary shear term or the normal links needs neither)
    R n[3] = {R(0), R(0), R(0)}, d = R(0), kap = R(0);
    if (p.rule != 0 || p.sigma != 0.0 || (EXT && (p.stress || p.recon_nc))) {
      const size_t cap = (size_t)v.cap;
      n[0] = v.geo[li];
      n[1] = v.geo[cap + li];
      n[2] = v.geo[2 * cap + li];
      d = v.geo[3 * cap + li];
      kap = v.geo[4 * cap + li];
    }
    const bool ok = true;  // no normal is stored as n = 0: c.n > 0 fails and delta stays 1/2
    // links to rebuild: the gas links, and with recon_nc the links p toward a
    // fluid node with n.c_p > 0 (Koerner et al.'s reconstruction along the
    // normal; margin 1e-6 for links tangent to the surface)
    unsigned rmask = gasm;
    R pulled[19];  // the pulled values, kept apart from the rebuilt ones
    if (EXT && p.recon_nc) {
#pragma unroll
      for (int q = 1; q < 19; ++q) {
        pulled[q] = f[q];
        const int pq = inv(q);
        const R cn = R(cx(pq)) * n[0] + R(cy(pq)) * n[1] + R(cz(pq)) * n[2];
        if (!((wallm | gasm) & (1u << q)) && cn > R(1e-6)) rmask |= 1u << q;
      }
    }
    R rb = R(p.rho_G);
    if (p.sigma != 0.0) rb = rb + R(3.0 * p.sigma) * kap;
    const R r0b = p.compressible ? rb : R(1);
    const R r0t = p.compressible ? rho_full_r<SH>(rt) : R(1);
    if (SH) rb = rb - R(1);  // e^+ below in the arithmetic of the stored values
    const R usq = utx * utx + uty * uty + utz * utz;
    const R lp = R(p.lam_p);
    // boundary shear rate S^b of Eq. bterm (stress mode): S from the cell's
    // own non-equilibrium part, sum_q c_qa c_qb n_q^+ = (2 c_s^2 / lambda_+) S_ab
    // (leading order of Eq. nqp), with its normal-tangential components set to
    // zero in the basis of the normal (Eq. proj2 through Eq. bstress):
    // S^b = S - (S n) n^T - n (S n)^T + 2 (n.S.n) n n^T
    R Sb[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};  // xx yy zz xy xz yz
    if (EXT && p.stress == 2) {  // prescribed S^b
#pragma unroll
      for (int k = 0; k < 6; ++k) Sb[k] = R(p.shear_b[k]);
    } else if (EXT && p.stress) {
#pragma unroll
      for (int q = 1; q < 19; q += 2) {  // each pair once: n_q^+ = n_qbar^+
        const R et = eplus_q<R>(p, q, rt, r0t, utx, uty, utz, usq);
        const R np2 = R(2) * (R(0.5) * (own[q] + own[q + 1]) - et) * R(p.inv_1plp);
        Sb[0] += R(cx(q) * cx(q)) * np2; Sb[1] += R(cy(q) * cy(q)) * np2; Sb[2] += R(cz(q) * cz(q)) * np2;
        Sb[3] += R(cx(q) * cy(q)) * np2; Sb[4] += R(cx(q) * cz(q)) * np2; Sb[5] += R(cy(q) * cz(q)) * np2;
      }
#pragma unroll
      for (int k = 0; k < 6; ++k) Sb[k] *= R(1.5) * lp;
      const R Sn0 = Sb[0] * n[0] + Sb[3] * n[1] + Sb[4] * n[2];
      const R Sn1 = Sb[3] * n[0] + Sb[1] * n[1] + Sb[5] * n[2];
      const R Sn2 = Sb[4] * n[0] + Sb[5] * n[1] + Sb[2] * n[2];
      const R snn = n[0] * Sn0 + n[1] * Sn1 + n[2] * Sn2;
      Sb[0] += R(2) * (snn * n[0] * n[0] - Sn0 * n[0]);
      Sb[1] += R(2) * (snn * n[1] * n[1] - Sn1 * n[1]);
      Sb[2] += R(2) * (snn * n[2] * n[2] - Sn2 * n[2]);
      Sb[3] += R(2) * snn * n[0] * n[1] - Sn0 * n[1] - n[0] * Sn1;
      Sb[4] += R(2) * snn * n[0] * n[2] - Sn0 * n[2] - n[0] * Sn2;
      Sb[5] += R(2) * snn * n[1] * n[2] - Sn1 * n[2] - n[1] * Sn2;
    }
    const R Dk = R(-3.0 * (p.tau_m_half));  // D = -alpha_+ Lambda_+ w_p / c_s^2, without alpha_+ w_p
#pragma unroll
    for (int q = 1; q < 19; ++q) {
      if (!(rmask & (1u << q))) continue;
      const int pq = inv(q);  // boundary link: x + c_p is gas (or a normal link), rebuilt f_pbar = f_q
      R eb = eplus_q<R>(p, pq, rb, r0b, utx, uty, utz, usq);
      bool up_fluid = !((wallm | gasm) & (1u << pq));
      // D c_p.S^b.c_p / alpha_+ (Eq. bterm, Table 1)
      R dterm = R(0);
      if (EXT && p.stress) {
        const R cSc = R(cx(pq) * cx(pq)) * Sb[0] + R(cy(pq) * cy(pq)) * Sb[1] + R(cz(pq) * cz(pq)) * Sb[2] +
                      R(2 * cx(pq) * cy(pq)) * Sb[3] + R(2 * cx(pq) * cz(pq)) * Sb[4] +
                      R(2 * cy(pq) * cz(pq)) * Sb[5];
        dterm = Dk * wq<R>(pq) * cSc;
      }
      if (p.rule == 0 || !up_fluid) {
        f[q] = -own[pq] + R(2) * eb + R(2) * dterm;  // FSK, Eq. koerner (alpha_+ = 2)
      } else {
        R dl = R(0.5);
        if (ok) {
          R cn = R(cx(pq)) * n[0] + R(cy(pq)) * n[1] + R(cz(pq)) * n[2];
          if (cn > R(0)) {
            dl = qdiv(d, cn);
            dl = dl < R(p.delta_min) ? R(p.delta_min) : (dl > R(1) ? R(1) : dl);
          }
        }
        if (EXT && p.ub_extrap) {
          // u_b at the surface point x_b + delta c_p, linear along the link
          // through u(x_b) and u(x_b - c_p)
          const long long su = IN ? i - (cx(pq) + sy * cy(pq) + sz * cz(pq)) : (long long)srcs[pq];
          const Vel3<R> uu = cell_velocity<P>(v.fin, N, (size_t)su, p.compressible, p.g[0], p.g[1], p.g[2]);
          const R wx = utx + dl * (utx - uu.x), wy = uty + dl * (uty - uu.y), wz = utz + dl * (utz - uu.z);
          eb = eplus_q<R>(p, pq, rb, r0b, wx, wy, wz, wx * wx + wy * wy + wz * wz);
        }
        R et = eplus_q<R>(p, pq, rt, r0t, utx, uty, utz, usq);
        R nplus = (R(0.5) * (own[pq] + own[q]) - et) * R(p.inv_1plp);
        R C = lp * (R(0.5) + dl) - R(2) * lp;
        const R fup = (EXT && p.recon_nc) ? pulled[pq] : f[pq];  // f~_p(x_b - c_p)
        f[q] = (R(0.5) - dl) * own[pq] + R(0.5) * own[q] + (dl - R(1)) * fup + C * nplus + eb + dterm;
      }
    }
  }
  R rho, ux, uy, uz;
  collide<R, SH>(p, f, rho, ux, uy, uz);
  // (the velocity guard is the liquid cells': an isolated interface cell of
  // the spray, with a few fluid neighbours, carries spurious speeds of 0.4
  // and more in a stable flow)
  if (rho_bad<SH>(rho)) atomicOr(v.err, ERRB_UNSTABLE);
#pragma unroll
  for (int q = 0; q < 19; ++q) stq<P>(v.fout, (size_t)q * N + (size_t)i, q, f[q]);
  double mm = v.m[i];
  if (!p.freeze) {
    const double rhof = rho_full<SH>(rho);
    mm = mm + dm;
    v.m[i] = mm;
    v.phout[i] = (R)(mm / rhof);
    // thresholds, plus the isolated-cell rules: no gas neighbour -> fill,
    // no liquid/interface neighbour -> empty
    fill = mm > (1.0 + p.eps) * rhof || ((p.cleanup & 1) && gasm == 0u);
    empty = !fill && (mm < -p.eps * rhof || ((p.cleanup & 2) && (wallm | gasm) == 0x7fffeu));
    if (fill) v.mark[i] = MK_FILL;  // marks are zero between steps; each cell writes only its own
    else if (empty) v.mark[i] = MK_EMPTY;
  }
  return mm;
}

// the geometry of cells within 3 of a face (bounded: no periodic axis);
// inlined, so that its Geo stays in registers (an out-of-line call measured
// slower: the edge warps set the kernel's tail)
template <class R, bool BOUNDED, bool SIG, bool ELV>
__device__ __forceinline__ void geometry_edge(const Par& p, const uint8_t* __restrict__ flags,
                                           const R* __restrict__ phin, int x, int y, int z, R phic, Geo<R>& G) {
  geometry<R, BOUNDED ? 2 : 0, SIG, ELV>(p, flags, phin, x, y, z, phic, G);
}

// ---------------------------------------------------------------------------
// k_geom: plane (normal, offset) and curvature of every listed interface cell
// from phi(t) (Sec. 2.2, Sec. 5), one thread per cell, into v.geo; kept apart
// from k_iface so that each kernel holds fewer registers and less code.
// ---------------------------------------------------------------------------
// SIG: the instance that also computes the curvature (surface tension); ELV:
// the one with the ELVIRA normal where the height columns are open
template <int P, bool SIG, bool ELV>
__global__ void __launch_bounds__(128) k_geom(Par p, View<P> v) {
  pdl_begin();
  using R = typename Form<P>::R;
  const int n_in = min(*((volatile int*)&v.cnt[0]), v.cap), n_edge = min(*((volatile int*)&v.cnt[6]), v.cap);
  const int count = min(n_in + n_edge, v.cap);
  const size_t cap = (size_t)v.cap;
  for (int li = blockIdx.x * blockDim.x + threadIdx.x; li < count; li += gridDim.x * blockDim.x) {
    const bool in3 = li < n_in;  // interior cells at the front, edge cells at the back
    const int pos = in3 ? li : v.cap - 1 - (li - n_in);
    const long long i = FSL_CK(p, v.ilist[pos], p.N);
    int x, y, z;
    coords(p, i, x, y, z);
    if (!FSL_OK(p, !in3 || (x >= 3 && x < p.nx - 3 && y >= 3 && y < p.ny - 3 && z >= 3 && z < p.nz - 3))) continue;
    const R phic = v.phin[i];
    R o[5];
    if (in3) {
      Geo<R> G;  // (in registers)
      geometry<R, 1, SIG, ELV>(p, v.flags, v.phin, x, y, z, phic, G);
      o[0] = G.ok ? G.n[0] : R(0); o[1] = G.ok ? G.n[1] : R(0); o[2] = G.ok ? G.n[2] : R(0);
      o[3] = G.d; o[4] = G.kap;
    } else {
      Geo<R> G;
      if (!p.px && !p.py && !p.pz) geometry_edge<R, true, SIG, ELV>(p, v.flags, v.phin, x, y, z, phic, G);
      else geometry_edge<R, false, SIG, ELV>(p, v.flags, v.phin, x, y, z, phic, G);
      o[0] = G.ok ? G.n[0] : R(0); o[1] = G.ok ? G.n[1] : R(0); o[2] = G.ok ? G.n[2] : R(0);
      o[3] = G.d; o[4] = G.kap;
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) v.geo[k * cap + pos] = o[k];
  }
}

// EXT: the instance with the boundary shear-rate term, the extrapolated u_b
// and the normal links (separate, so that the default instance carries none
// of their code)
template <int P, bool EXT>
__global__ void __launch_bounds__(128, (EXT ? 2 : (P == P64 ? 3 : 5))) k_iface(Par p, View<P> v, int part_base) {
  pdl_begin();
  const int n_in = min(*((volatile int*)&v.cnt[0]), v.cap), n_edge = min(*((volatile int*)&v.cnt[6]), v.cap);
  const int count = min(n_in + n_edge, v.cap);
  const int stride = gridDim.x * blockDim.x;
  const int rounds = (count + stride - 1) / stride;
  double msum = 0.0;
  for (int r = 0; r < rounds; ++r) {
    const int li = r * stride + blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = li < count;
    bool fill = false, empty = false;
    int icell = 0;
    if (act) {
      const bool in3 = li < n_in;  // interior cells at the front, edge cells at the back
      const int pos = in3 ? li : v.cap - 1 - (li - n_in);
      const long long i = FSL_CK(p, v.ilist[pos], p.N);
      icell = (int)i;
      int x, y, z;
      coords(p, i, x, y, z);
      if (FSL_OK(p, !in3 || (x >= 3 && x < p.nx - 3 && y >= 3 && y < p.ny - 3 && z >= 3 && z < p.nz - 3))) {
        const double mm = in3 ? iface_cell<P, true, EXT>(p, v, pos, i, x, y, z, fill, empty)
                              : iface_cell<P, false, EXT>(p, v, pos, i, x, y, z, fill, empty);
        if (owned(p, x, y, z)) msum += mm;
      }
    }
    warp_append(fill, icell, v.flist, &v.cnt[1], v.cap, v.err);
    warp_append(empty, icell, v.elist, &v.cnt[2], v.cap, v.err);
  }
  // per-warp partial sums, after the bulk warps' ones
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) msum += __shfl_down_sync(0xffffffffu, msum, o);
  if ((threadIdx.x & 31) == 0) v.partials[part_base + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5)] = msum;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// a launch without the programmatic-serialization attribute (after a wait
// on another stream's event)
template <typename... KArgs, typename... Args>
inline int launch_plain(void (*kernel)(KArgs...), unsigned grid, unsigned block, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.stream = st;
  return (int)cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <int P>
int launch_step_kernels(const Par& p, const View<P>& v, cudaStream_t st, int bulk_blocks, int iface_blocks,
                        int* seglist, int* segcount, void* timing_handle, int bulk_mode,
                        const CUtensorMap* tmap, const Fork* fork) {
  if (launch_segments(p, v.flags, seglist, segcount, v.ilist, v.cnt, v.cap, v.err, st))
    return 1;
  // the interface geometry reads phi(t), the flags and the interface list of
  // the segment scan, and writes only its scratch: it runs on the side stream
  // beside the bulk kernel.  Beside the pair kernel (whose grid then leaves
  // room on every SM) the interface kernel follows it there: it reads f~(t),
  // phi(t), m and the flags, and writes the interface cells' populations, m,
  // phi(t+1), marks and lists, none of which the bulk kernel touches
  const bool geo = p.rule != 0 || p.sigma != 0.0 || p.stress || p.recon_nc;
  auto kgeo = p.elvira ? (p.sigma != 0.0 ? k_geom<P, true, true> : k_geom<P, false, true>)
                       : (p.sigma != 0.0 ? k_geom<P, true, false> : k_geom<P, false, false>);
  auto kif = (p.stress || p.ub_extrap || p.recon_nc) ? k_iface<P, true> : k_iface<P, false>;
  const bool pairs = P != P64 && bulk_mode == BULK_PAIRS;
  const bool side_geo = geo && fork;
  const bool side_if = pairs && fork;
  if (side_geo || side_if) {
    if (cudaEventRecord(fork->fork, st) != cudaSuccess) return 1;
    if (cudaStreamWaitEvent(fork->side, fork->fork, 0) != cudaSuccess) return 1;
    if (side_geo && launch_plain(kgeo, iface_blocks, 128, fork->side, p, v)) return 1;
    // the interface partials follow the bulk warps' ones
    if (side_if && launch_plain(kif, iface_blocks, 128, fork->side, p, v, bulk_blocks * 4)) return 1;
    if (cudaEventRecord(fork->join, fork->side) != cudaSuccess) return 1;
  }
  if (timing_handle && fslbm_mark(timing_handle, 0)) return 1;  // the bulk group times the bulk kernel alone
  bool launched = false;
  if constexpr (P != P64) {
    if (bulk_mode == BULK_TMA && tmap) {
      if (launch_bulk_tma<P>(p, v, tmap, st, bulk_blocks, seglist, segcount)) return 1;
      launched = true;
    } else if (bulk_mode == BULK_ASYNC) {
      if (launch_bulk_async<P>(p, v, st, bulk_blocks, seglist, segcount)) return 1;
      launched = true;
    } else if (bulk_mode == BULK_PAIRS) {
      if (launch_bulk_pairs<P>(p, v, st, bulk_blocks, seglist, segcount, side_if)) return 1;
      launched = true;
    }
  }
  if (!launched && launch_k(k_bulk<P>, bulk_blocks, 128, 0, st, p, v, (const int*)seglist, (const int*)segcount))
    return 1;
  if (timing_handle && fslbm_mark(timing_handle, 1)) return 1;
  if (geo && !side_geo && launch_k(kgeo, iface_blocks, 128, 0, st, p, v)) return 1;
  if (side_geo || side_if) {
    if (cudaStreamWaitEvent(st, fork->join, 0) != cudaSuccess) return 1;
  }
  if (!side_if) {
    if (side_geo ? launch_plain(kif, iface_blocks, 128, st, p, v, bulk_blocks * 4)
                 : launch_k(kif, iface_blocks, 128, 0, st, p, v, bulk_blocks * 4))
      return 1;
  }
  return (int)cudaGetLastError();
}

}  // namespace fsl

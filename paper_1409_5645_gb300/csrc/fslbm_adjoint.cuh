// fslbm_adjoint.cuh -- the reverse step's kernels and the reverse sweep, as
// templates over the precision form (the method is described at the top of
// fslbm_adjoint.cu).
#pragma once
#include <math.h>
#include <stdio.h>

#include "fslbm_adjoint.h"

using namespace fsl;

namespace fsl {


template <int P>
struct AdjView {
  using S = typename Form<P>::S;
  using R = typename Form<P>::R;
  const uint8_t* flags;
  const S* f;
  const double* m;
  const R* phi;
  const double* wd;
  const double* abar_in;
  const double* mbar_in;
  const double* phibar_in;
  double* abar_out;
  double* Pb;
  double* mbar_out;
  double* phibar_out;
  double* theta;
  const int* flist;  // the liquid (or interface) cells of `flags`, nfl of them
  const int* nfl;
};

// a population of the stored state in the arithmetic A of the reverse step:
// f_q in FP64, or in the deviation mode (float A on FP32/FP16 storage) the
// stored f_q - w_q itself
template <int P, class A>
__device__ __forceinline__ A ld_adj(const typename Form<P>::S* __restrict__ f, size_t k, int q) {
  if constexpr (sizeof(A) == 4 && Form<P>::SH) {
    if constexpr (P == P16) return __half2float(f[k]);
    else return (A)f[k];
  } else {
    return (A)ldq_full<P>(f, k, q);
  }
}

// warp-level sums of th added to out (one atomic per warp and component; all
// 32 lanes call it)
template <class A>
__device__ __forceinline__ void warp_add(A (&th)[5], double* out) {
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    double v = (double)th[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(out + k, v);
  }
}

// d e_q^+ / d u for rho_0 = 1: w_q (9 (c.u) c - 3 u); zero for the linear equilibrium
template <class A>
__device__ __forceinline__ void deplus_du(const Par& p, int q, A ux, A uy, A uz, A g, A (&ub)[3]) {
  if (p.linear_eq) return;
  A w = q == 0 ? A(1.0) / A(3.0) : (q <= 6 ? A(1.0) / A(18.0) : A(1.0) / A(36.0));
  A cu = A(cx(q)) * ux + A(cy(q)) * uy + A(cz(q)) * uz;
  ub[0] += g * w * (A(9.0) * cu * cx(q) - A(3.0) * ux);
  ub[1] += g * w * (A(9.0) * cu * cy(q) - A(3.0) * uy);
  ub[2] += g * w * (A(9.0) * cu * cz(q) - A(3.0) * uz);
}

template <class A>
__device__ __forceinline__ A eplus_d(const Par& p, int q, A rho, A ux, A uy, A uz) {
  A w = q == 0 ? A(1.0) / A(3.0) : (q <= 6 ? A(1.0) / A(18.0) : A(1.0) / A(36.0));
  A e = w * rho;
  if (!p.linear_eq) {
    A cu = A(cx(q)) * ux + A(cy(q)) * uy + A(cz(q)) * uz;
    e += w * A(1.5) * (A(3.0) * cu * cu - (ux * ux + uy * uy + uz * uz));
  }
  return e;
}

// Reverse of the TRT collision (Eq. lbe2, rho_0 = 1) at pre-collision f with
// output adjoint ab: adds to fb and to th (lambda_+, lambda_-, g).
template <class A>
__device__ void collide_rev(const Par& p, const A (&f)[19], const A (&ab)[19], A (&fb)[19], A (&th)[5]) {
  const A lp = (A)p.lam_p, lm = (A)p.lam_m;
  const A g0 = (A)p.g[0], g1 = (A)p.g[1], g2 = (A)p.g[2];
  A r = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
  for (int q = 0; q < 19; ++q) {
    r += f[q];
    jx += A(cx(q)) * f[q];
    jy += A(cy(q)) * f[q];
    jz += A(cz(q)) * f[q];
  }
  const A ux = jx + A(0.5) * g0, uy = jy + A(0.5) * g1, uz = jz + A(0.5) * g2;
  const A vx = jx - g0 / lm, vy = jy - g1 / lm, vz = jz - g2 / lm;
  A rb = 0, ub[3] = {0, 0, 0}, vb[3] = {0, 0, 0};
#pragma unroll
  for (int q = 0; q < 19; ++q) fb[q] += ab[q];
  {  // rest population: out0 = f0 + l+ (f0 - e0+)
    A e0 = eplus_d<A>(p, 0, r, ux, uy, uz);
    A np = f[0] - e0;
    A npb = lp * ab[0];
    th[0] += np * ab[0];
    fb[0] += npb;
    rb += (A(1.0) / A(3.0)) * (-npb);
    deplus_du<A>(p, 0, ux, uy, uz, -npb, ub);
  }
#pragma unroll
  for (int q = 1; q < 19; q += 2) {
    const int qb = q + 1;
    A w = q <= 6 ? A(1.0) / A(18.0) : A(1.0) / A(36.0);
    A ep = eplus_d<A>(p, q, r, ux, uy, uz);
    A em = A(3.0) * w * (A(cx(q)) * vx + A(cy(q)) * vy + A(cz(q)) * vz);
    A np = A(0.5) * (f[q] + f[qb]) - ep;
    A nm = A(0.5) * (f[q] - f[qb]) - em;
    A npb = lp * (ab[q] + ab[qb]);
    A nmb = lm * (ab[q] - ab[qb]);
    th[0] += np * (ab[q] + ab[qb]);
    th[1] += nm * (ab[q] - ab[qb]);
    fb[q] += A(0.5) * npb + A(0.5) * nmb;
    fb[qb] += A(0.5) * npb - A(0.5) * nmb;
    // e^+: -npb;  e^-: -nmb
    rb += w * (-npb);
    deplus_du<A>(p, q, ux, uy, uz, -npb, ub);
    vb[0] += A(3.0) * w * A(cx(q)) * (-nmb);
    vb[1] += A(3.0) * w * A(cy(q)) * (-nmb);
    vb[2] += A(3.0) * w * A(cz(q)) * (-nmb);
  }
  // u = U + g/2, v = U - g/lambda_-, U = j
  A Ub[3] = {ub[0] + vb[0], ub[1] + vb[1], ub[2] + vb[2]};
  th[2] += A(0.5) * ub[0] - vb[0] / lm;
  th[3] += A(0.5) * ub[1] - vb[1] / lm;
  th[4] += A(0.5) * ub[2] - vb[2] / lm;
  th[1] += (g0 * vb[0] + g1 * vb[1] + g2 * vb[2]) / (lm * lm);
#pragma unroll
  for (int q = 0; q < 19; ++q) fb[q] += rb + A(cx(q)) * Ub[0] + A(cy(q)) * Ub[1] + A(cz(q)) * Ub[2];
}

__device__ __forceinline__ void block_add(double (&th)[5], double* out) {
  __shared__ double red[4][5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    double v = th[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    double s = red[0][threadIdx.x] + red[1][threadIdx.x] + red[2][threadIdx.x] + red[3][threadIdx.x];
    if (s != 0.0) atomicAdd(out + threadIdx.x, s);
  }
}

// Area A and centroid c of the section of the unit cell [-1/2, 1/2]^3 by the
// plane n.x = d (n a unit vector).  The volume V(n, d) on the side n.x <= d
// has dV/dd = A and dV/dn = -A c, so at fixed V the plane offset moves by
// dd = dV / A + c.dn (the adjoint of the plane fit).  The polygon's corners
// are the plane's crossings of the twelve cell edges, ordered by angle about
// their mean; triangles from the mean give A and c.
static __device__ void plane_section(const double (&n)[3], double d, double& A, double (&c)[3]) {
  double P[12][3];
  int np = 0;
  for (int e = 0; e < 3; ++e) {
    if (fabs(n[e]) < 1e-12) continue;  // the four edges along e are parallel to the plane
    const int a1 = (e + 1) % 3, a2 = (e + 2) % 3;
    for (int s1 = -1; s1 <= 1; s1 += 2)
      for (int s2 = -1; s2 <= 1; s2 += 2) {
        const double x1 = 0.5 * s1, x2 = 0.5 * s2;
        const double t = (d - n[a1] * x1 - n[a2] * x2) / n[e];
        if (t >= -0.5 && t <= 0.5) {
          P[np][e] = t;
          P[np][a1] = x1;
          P[np][a2] = x2;
          ++np;
        }
      }
  }
  A = 0.0;
  c[0] = c[1] = c[2] = 0.0;
  if (np < 3) return;
  double m[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < np; ++k)
    for (int j = 0; j < 3; ++j) m[j] += P[k][j] / np;
  // in-plane basis: u from the axis least aligned with n, v = n x u
  int ax = 0;
  if (fabs(n[1]) < fabs(n[ax])) ax = 1;
  if (fabs(n[2]) < fabs(n[ax])) ax = 2;
  double u[3] = {-n[ax] * n[0], -n[ax] * n[1], -n[ax] * n[2]};
  u[ax] += 1.0;
  const double lu = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  u[0] /= lu; u[1] /= lu; u[2] /= lu;
  const double v[3] = {n[1] * u[2] - n[2] * u[1], n[2] * u[0] - n[0] * u[2], n[0] * u[1] - n[1] * u[0]};
  double ang[12];
  int ord[12];
  for (int k = 0; k < np; ++k) {
    const double r0 = P[k][0] - m[0], r1 = P[k][1] - m[1], r2 = P[k][2] - m[2];
    ang[k] = atan2(r0 * v[0] + r1 * v[1] + r2 * v[2], r0 * u[0] + r1 * u[1] + r2 * u[2]);
    ord[k] = k;
  }
  for (int k = 1; k < np; ++k)  // insertion sort by angle
    for (int j = k; j > 0 && ang[ord[j]] < ang[ord[j - 1]]; --j) {
      const int t = ord[j];
      ord[j] = ord[j - 1];
      ord[j - 1] = t;
    }
  for (int k = 0; k < np; ++k) {
    const double* p0 = P[ord[k]];
    const double* p1 = P[ord[(k + 1) % np]];
    const double e0[3] = {p0[0] - m[0], p0[1] - m[1], p0[2] - m[2]};
    const double e1[3] = {p1[0] - m[0], p1[1] - m[1], p1[2] - m[2]};
    const double cr = (e0[1] * e1[2] - e0[2] * e1[1]) * n[0] + (e0[2] * e1[0] - e0[0] * e1[2]) * n[1] +
                      (e0[0] * e1[1] - e0[1] * e1[0]) * n[2];
    const double at = 0.5 * fabs(cr);
    A += at;
    for (int j = 0; j < 3; ++j) c[j] += at * (m[j] + p0[j] + p1[j]) / 3.0;
  }
  if (A > 0.0)
    for (int j = 0; j < 3; ++j) c[j] /= A;
}

// Reverse of the plane fit of a cell whose height columns are open: d =
// d(n, phi_c) with V(n, d) = phi_c (phi_c kept in [1e-9, 1 - 1e-9]), n = -g/|g|
// with g the Parker-Youngs gradient of the fill levels around the cell (a
// wall takes phi_c).  dbar, nbar: adjoints of d and of the unit normal.  Adds
// the neighbours' fill-level adjoints to phibar (atomics) and returns the
// cell's own.  Out of line: rare, and its arrays stay out of the main frame.
template <class R>
__device__ __noinline__ double plane_fit_adjoint(const Par& p, const uint8_t* __restrict__ flags,
                                                 const R* __restrict__ phi, double* phibar, int x, int y, int z,
                                                 double phic, double n0, double n1, double n2, double d,
                                                 double dbar, const double (&nb)[3]) {
  const double nh[3] = {n0, n1, n2};
  double nbar[3] = {nb[0], nb[1], nb[2]};
  double own = 0.0;
  double A, cen[3];
  plane_section(nh, d, A, cen);
  if (A > 0.0 && phic > 1e-9 && phic < 1.0 - 1e-9) own += dbar / A;
  for (int k = 0; k < 3; ++k) nbar[k] += dbar * cen[k];
  double gr[3] = {0.0, 0.0, 0.0};
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (!dx && !dy && !dz) continue;
        const uint8_t kj = kind_at(flags, nbr(p, x, y, z, dx, dy, dz));
        double pj = 0.0;
        if (kj == LIQ) pj = 1.0;
        else if (kj == IFC || (kj == GAS && p.freeze)) pj = (double)phi[nbr(p, x, y, z, dx, dy, dz)];
        else if (kj == WALL) pj = phic;
        const int ax_ = dx < 0 ? -dx : dx, ay_ = dy < 0 ? -dy : dy, az_ = dz < 0 ? -dz : dz;
        gr[0] += dx * (2 - ay_) * (2 - az_) * pj;
        gr[1] += dy * (2 - az_) * (2 - ax_) * pj;
        gr[2] += dz * (2 - ax_) * (2 - ay_) * pj;
      }
  const double gl = sqrt(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
  const double nd = nbar[0] * nh[0] + nbar[1] * nh[1] + nbar[2] * nh[2];
  double gb[3];  // adjoint of g
  for (int k = 0; k < 3; ++k) gb[k] = -(nbar[k] - nd * nh[k]) / gl;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (!dx && !dy && !dz) continue;
        const long long j = nbr(p, x, y, z, dx, dy, dz);
        const uint8_t kj = kind_at(flags, j);
        const int ax_ = dx < 0 ? -dx : dx, ay_ = dy < 0 ? -dy : dy, az_ = dz < 0 ? -dz : dz;
        const double val = gb[0] * (dx * (2 - ay_) * (2 - az_)) + gb[1] * (dy * (2 - az_) * (2 - ax_)) +
                           gb[2] * (dz * (2 - ax_) * (2 - ay_));
        if (val == 0.0) continue;
        if (kj == WALL) own += val;
        else if (kj == IFC || (kj == GAS && p.freeze)) atomicAdd(phibar + j, val);
      }
  return own;
}

// IFCP: the instance for interface cells (gas links, mass exchange,
// geometry); the other runs the liquid cells, whose code is a small part of
// this one (a liquid cell never touches gas).
// A: the arithmetic of the reverse step (double; float for FP32/FP16 lattices
// with adj32, which then works in the deviations f - w_q as the forward step
// does: moments rho - 1, the gas density rho_G - 1 in the rebuilt links; every
// closure is affine in the populations with weights summing to one per link
// pair, so only the densities that divide (phi = m / rho) take the 1 back).
template <int P, bool IFCP, class A>
__global__ void __launch_bounds__(128) k_adj_local(Par p, AdjView<P> a) {
  using R = typename Form<P>::R;
  constexpr bool SH = sizeof(A) == 4 && Form<P>::SH;
  const size_t N = (size_t)p.N;
  A th[5] = {0, 0, 0, 0, 0};
  const int nf = *a.nfl;
  for (int li = blockIdx.x * blockDim.x + threadIdx.x; li < nf; li += gridDim.x * blockDim.x) {
    const long long i = FSL_CK(p, a.flist[li], p.N);
    const uint8_t kc = IFCP ? (uint8_t)IFC : (uint8_t)LIQ;
    int x, y, z;
    coords(p, i, x, y, z);
    A own[19], F[19], f[19];
#pragma unroll
    for (int q = 0; q < 19; ++q) own[q] = ld_adj<P, A>(a.f, q * N + i, q);
    unsigned wallm = 0u, gasm = 0u;
    int src[19];
    F[0] = own[0];
    src[0] = (int)i;
#pragma unroll
    for (int q = 1; q < 19; ++q) {
      long long s = nbr(p, x, y, z, -cx(q), -cy(q), -cz(q));
      src[q] = (int)s;
      uint8_t ks = kind_at(a.flags, s);
      if (is_fluid(ks)) F[q] = ld_adj<P, A>(a.f, q * N + s, q);
      else if (ks == WALL) { wallm |= 1u << q; F[q] = A(0.0); }
      else { gasm |= 1u << q; F[q] = A(0.0); }
    }
    if constexpr (!IFCP) gasm = 0u;  // (liquid cells have no gas neighbour)
#pragma unroll
    for (int q = 0; q < 19; ++q) f[q] = F[q];
    // own moments at t (rho_0 = 1): rho_t = sum f~, u_t = sum c f~ - g/2
    A rt = 0, tx = 0, ty = 0, tz = 0;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
      rt += own[q];
      tx += cx(q) * own[q];
      ty += cy(q) * own[q];
      tz += cz(q) * own[q];
    }
    const A utx = tx - A(0.5) * (A)p.g[0], uty = ty - A(0.5) * (A)p.g[1], utz = tz - A(0.5) * (A)p.g[2];
    const bool ifc = kc == IFC;
    const A phic = ifc ? (A)a.phi[i] : A(1);
    const bool dyn = ifc && !p.freeze;
    // mass exchange
    A dm = A(0.0);
    if (dyn) {
#pragma unroll
      for (int q = 1; q < 19; ++q) {
        if ((wallm | gasm) & (1u << q)) continue;
        uint8_t ks = a.flags[src[q]] & KIND;
        A sw = (ks == LIQ) ? A(1.0) : A(0.5) * (phic + (A)a.phi[src[q]]);
        dm += sw * (F[q] - own[inv(q)]);
      }
    }
    // wall closures
    A kw[19];
#pragma unroll
    for (int q = 0; q < 19; ++q) kw[q] = A(0.0);
#pragma unroll
    for (int q = 1; q < 19; ++q) {
      if (!(wallm & (1u << q))) continue;
      const int pq = inv(q);
      A val = own[pq];
      if (p.has_wd) {
        A dw = (A)a.wd[(size_t)pq * N + i];
        bool upf = !((wallm | gasm) & (1u << pq));
        if (dw >= A(0.0) && upf) {
          kw[q] = (A(1.0) - A(2.0) * dw) / (A(1.0) + A(2.0) * dw);
          val += kw[q] * (F[pq] - own[q]);
        }
      }
      f[q] = val;
    }
    // free-surface closures (forward, keeping what the reverse needs)
    Geo<R> G;
    A dl[19], npl[19], et[19];
    bool fsl[19];
    const A lp = (A)p.lam_p, inv1 = (A)p.inv_1plp, dmin = (A)p.delta_min;
    const A rhoG = SH ? (A)(p.rho_G - 1.0) : (A)p.rho_G;  // (deviation of the gas density)
    if (gasm) {
      geometry<R>(p, a.flags, a.phi, x, y, z, (R)phic, G);
#pragma unroll
      for (int q = 1; q < 19; ++q) {
        fsl[q] = false;
        if (!(gasm & (1u << q))) continue;
        const int pq = inv(q);
        A eb = eplus_d<A>(p, pq, rhoG, utx, uty, utz);
        bool upf = !((wallm | gasm) & (1u << pq));
        if (p.rule == 0 || !upf) {
          f[q] = -own[pq] + A(2.0) * eb;
        } else {
          A d_ = A(0.5);
          if (G.ok) {
            A cn = A(cx(pq)) * (A)G.n[0] + A(cy(pq)) * (A)G.n[1] + A(cz(pq)) * (A)G.n[2];
            if (cn > A(0.0)) {
              d_ = (A)G.d / cn;
              d_ = d_ < dmin ? dmin : (d_ > A(1) ? A(1) : d_);
            }
          }
          dl[q] = d_;
          et[q] = eplus_d<A>(p, pq, rt, utx, uty, utz);
          npl[q] = (A(0.5) * (own[pq] + own[q]) - et[q]) * inv1;
          A C = lp * (A(0.5) + d_) - A(2.0) * lp;
          f[q] = (A(0.5) - d_) * own[pq] + A(0.5) * own[q] + (d_ - A(1.0)) * F[pq] + C * npl[q] + eb;
          fsl[q] = true;
        }
      }
    }
    A rho1 = 0;
#pragma unroll
    for (int q = 0; q < 19; ++q) rho1 += f[q];
    const A rho1f = SH ? A(1) + rho1 : rho1;  // the density after the step

    // ---------------- reverse ----------------
    A ab[19], fb[19], ob[19], Fb[19];
#pragma unroll
    for (int q = 0; q < 19; ++q) {
      ab[q] = (A)a.abar_in[q * N + i];
      fb[q] = A(0.0); ob[q] = A(0.0); Fb[q] = A(0.0);
    }
    A phib_self = A(0.0), mb1 = A(0.0), rho1b = A(0.0);
    if (dyn) {
      const A m1 = (A)a.m[i] + dm;
      const A pb = (A)a.phibar_in[i];
      mb1 = (A)a.mbar_in[i] + pb / rho1f;
      rho1b = -pb * m1 / (rho1f * rho1f);
    } else if (ifc) {
      phib_self += (A)a.phibar_in[i];  // frozen interface: phi(t+1) = phi(t)
    }
    collide_rev<A>(p, f, ab, fb, th);
#pragma unroll
    for (int q = 0; q < 19; ++q) fb[q] += rho1b;
    a.mbar_out[i] = dyn ? (double)mb1 : 0.0;
    if (dyn) {
      const A dmb = mb1;
#pragma unroll
      for (int q = 1; q < 19; ++q) {
        if ((wallm | gasm) & (1u << q)) continue;
        uint8_t ks = a.flags[src[q]] & KIND;
        A sw = (ks == LIQ) ? A(1.0) : A(0.5) * (phic + (A)a.phi[src[q]]);
        Fb[q] += sw * dmb;
        ob[inv(q)] -= sw * dmb;
        if (ks == IFC) {
          A c = A(0.5) * dmb * (F[q] - own[inv(q)]);
          phib_self += c;
          atomicAdd(a.phibar_out + src[q], (double)c);
        }
      }
    }
    // wall closures
#pragma unroll
    for (int q = 1; q < 19; ++q) {
      if (!(wallm & (1u << q))) continue;
      const int pq = inv(q);
      ob[pq] += fb[q];
      if (kw[q] != A(0.0)) {
        Fb[pq] += kw[q] * fb[q];
        ob[q] -= kw[q] * fb[q];
      }
    }
    // free-surface closures
    A utb[3] = {0, 0, 0}, rtb = A(0.0);
    A Hbar[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    bool geo_used = false;
    A dbar = A(0.0), nbar[3] = {A(0.0), A(0.0), A(0.0)};  // plane-fit cells: adjoints of the offset and unit normal
    bool plic_used = false;
    if (gasm) {
#pragma unroll
      for (int q = 1; q < 19; ++q) {
        if (!(gasm & (1u << q))) continue;
        const int pq = inv(q);
        const A fbq = fb[q];
        if (!fsl[q]) {  // FSK: f_q = -f~_p + 2 e_p^+(rho_b, u_t)
          ob[pq] -= fbq;
          deplus_du<A>(p, pq, utx, uty, utz, A(2.0) * fbq, utb);
          continue;
        }
        const A d_ = dl[q];
        ob[pq] += (A(0.5) - d_) * fbq;
        ob[q] += A(0.5) * fbq;
        Fb[pq] += (d_ - A(1.0)) * fbq;
        const A C = lp * (A(0.5) + d_) - A(2.0) * lp;
        th[0] += fbq * (d_ - A(1.5)) * npl[q];
        deplus_du<A>(p, pq, utx, uty, utz, fbq, utb);  // e_p^+(rho_b, u_t)
        const A nb = C * fbq;
        ob[pq] += A(0.5) * nb * inv1;
        ob[q] += A(0.5) * nb * inv1;
        const A etb = -nb * inv1;
        rtb += (pq <= 6 ? A(1.0) / A(18.0) : A(1.0) / A(36.0)) * etb;
        deplus_du<A>(p, pq, utx, uty, utz, etb, utb);
        th[0] += -nb * (A(0.5) * (own[pq] + own[q]) - et[q]) * inv1 * inv1;
        // delta -> heights (closed height columns) or -> plane offset and
        // normal (plane fit), unclamped delta only
        const A db = fbq * (-own[pq] + F[pq] + lp * npl[q]);
        if (G.ok && !G.closed && db != A(0.0)) {
          const A cn = A(cx(pq)) * (A)G.n[0] + A(cy(pq)) * (A)G.n[1] + A(cz(pq)) * (A)G.n[2];
          if (cn > A(0.0)) {
            const A raw = (A)G.d / cn;
            if (raw > dmin && raw < A(1.0)) {  // delta = d / (n.c_p)
              dbar += db / cn;
              const A t = -db * raw / cn;
              nbar[0] += t * cx(pq);
              nbar[1] += t * cy(pq);
              nbar[2] += t * cz(pq);
              plic_used = true;
            }
          }
        }
        if (G.ok && G.closed && db != A(0.0)) {
          const int Ax = G.a, B = G.b, Cc = 3 - G.a - G.b;
          const int ca = Ax == 0 ? cx(pq) : (Ax == 1 ? cy(pq) : cz(pq));
          const int cb = B == 0 ? cx(pq) : (B == 1 ? cy(pq) : cz(pq));
          const int cc = Cc == 0 ? cx(pq) : (Cc == 1 ? cy(pq) : cz(pq));
          const A Hb = A(0.5) * ((A)G.H[7] - (A)G.H[1]);
          const A Hc = A(0.5) * ((A)G.H[5] - (A)G.H[3]);
          const A vc = G.s * ca - Hb * cb - Hc * cc;
          if (vc > A(0.0)) {
            const A raw = ((A)G.H[4] - A(3.5)) / vc;
            if (raw > dmin && raw < A(1.0)) {
              const A hb_ = db * d_ * cb / vc, hc_ = db * d_ * cc / vc;
              Hbar[4] += db / vc;
              Hbar[7] += A(0.5) * hb_;
              Hbar[1] -= A(0.5) * hb_;
              Hbar[5] += A(0.5) * hc_;
              Hbar[3] -= A(0.5) * hc_;
              geo_used = true;
            }
          }
        }
      }
    }
#pragma unroll
    for (int q = 1; q < 19; ++q)
      if (!((wallm | gasm) & (1u << q))) Fb[q] += fb[q];
    ob[0] += fb[0];
    if (geo_used) {
      const int Ax = G.a, B = G.b;
      for (int ib = -1; ib <= 1; ++ib)
        for (int ic = -1; ic <= 1; ++ic) {
          const A hb = Hbar[(ib + 1) * 3 + (ic + 1)];
          if (hb == A(0.0)) continue;
          for (int k = -3; k <= 3; ++k) {
            int o0 = (Ax == 0) ? k : ((B == 0) ? ib : ic);
            int o1 = (Ax == 1) ? k : ((B == 1) ? ib : ic);
            int o2 = (Ax == 2) ? k : ((B == 2) ? ib : ic);
            long long j = nbr(p, x, y, z, o0, o1, o2);
            uint8_t kj = kind_at(a.flags, j);
            if (kj == IFC || (kj == GAS && p.freeze)) {
              if (j == i) phib_self += hb;
              else atomicAdd(a.phibar_out + j, (double)hb);
            }
          }
        }
    }
    if (plic_used) {
      const double nbd[3] = {(double)nbar[0], (double)nbar[1], (double)nbar[2]};
      phib_self += (A)plane_fit_adjoint(p, a.flags, a.phi, a.phibar_out, x, y, z, (double)phic, (double)G.n[0],
                                        (double)G.n[1], (double)G.n[2], (double)G.d, (double)dbar, nbd);
    }
    // own moments: rho_t = sum f~, u_t = sum c f~ - g/2
#pragma unroll
    for (int q = 0; q < 19; ++q) ob[q] += rtb + cx(q) * utb[0] + cy(q) * utb[1] + cz(q) * utb[2];
    th[2] -= A(0.5) * utb[0];
    th[3] -= A(0.5) * utb[1];
    th[4] -= A(0.5) * utb[2];
#pragma unroll
    for (int q = 0; q < 19; ++q) {
      a.abar_out[q * N + i] = (double)ob[q];
      a.Pb[q * N + i] = (double)Fb[q];
    }
    if (phib_self != A(0)) atomicAdd(a.phibar_out + i, (double)phib_self);
  }
  warp_add(th, a.theta);
}

// reverse of the pull: abar_q(y) += P_q(y + c_q) when y + c_q pulled from y
// (over the liquid and the interface cells of the step: lists liq, ifc)
template <int P>
__global__ void k_adj_gather(Par p, const uint8_t* __restrict__ flags, const double* __restrict__ Pb,
                             double* __restrict__ abar, const int* __restrict__ liq, const int* __restrict__ ifc,
                             const int* __restrict__ cnt) {
  const size_t N = (size_t)p.N;
  const int nl = cnt[0], ni = cnt[1];
  for (int li = blockIdx.x * blockDim.x + threadIdx.x; li < nl + ni; li += gridDim.x * blockDim.x) {
    const long long i = FSL_CK(p, li < nl ? liq[li] : ifc[li - nl], p.N);
    int x, y, z;
    coords(p, i, x, y, z);
#pragma unroll
    for (int q = 1; q < 19; ++q) {
      long long zc = nbr(p, x, y, z, cx(q), cy(q), cz(q));
      if (zc < 0 || !is_fluid(flags[zc] & KIND)) continue;
      abar[q * N + i] += Pb[q * N + zc];
    }
  }
}

// Objective on the stored state: red[0] = sum of the objective's terms,
// red[1] = count (interface cells) or sum of phi (flux).
template <int P>
__global__ void k_objective(Par p, const uint8_t* flags, const typename Form<P>::S* f,
                            const typename Form<P>::R* phi, int objective, double* red) {
  const size_t N = (size_t)p.N;
  double s = 0.0, c = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < p.N;
       i += (long long)gridDim.x * blockDim.x) {
    uint8_t k = flags[i] & KIND;
    if (!is_fluid(k)) continue;
    if (objective == 0 && k != IFC) continue;
    double jx = 0.0;
#pragma unroll
    for (int q = 0; q < 19; ++q)
      if (cx(q)) jx += cx(q) * ldq_full<P>(f, q * N + i, q);
    double ux = jx - 0.5 * p.g[0];
    double w = objective == 0 ? 1.0 : (k == IFC ? (double)phi[i] : 1.0);
    s += w * ux;
    c += w;
  }
  atomicAdd(red, s);
  atomicAdd(red + 1, c);
}

template <int P>
__global__ void k_obj_seed(Par p, const uint8_t* flags, const typename Form<P>::S* f,
                           const typename Form<P>::R* phi, int objective, double scale, double* abar,
                           double* phibar, double* mbar) {
  const size_t N = (size_t)p.N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < p.N;
       i += (long long)gridDim.x * blockDim.x) {
    uint8_t k = flags[i] & KIND;
    double w = 0.0, pb = 0.0;
    if (is_fluid(k)) {
      if (objective == 0) {
        w = (k == IFC) ? scale : 0.0;
      } else {
        w = (k == IFC ? (double)phi[i] : 1.0) * scale;
        if (k == IFC) {
          double jx = 0.0;
#pragma unroll
          for (int q = 0; q < 19; ++q)
            if (cx(q)) jx += cx(q) * ldq_full<P>(f, q * N + i, q);
          pb = (jx - 0.5 * p.g[0]) * scale;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 19; ++q) abar[q * N + i] = w * cx(q);
    phibar[i] = pb;
    mbar[i] = 0.0;
  }
}

// Reverse of the initial collision f~(0) = C(f(0)) for the parameter
// adjoints (f(0) recovered by inverting the collision), and dJ/dphi0 =
// mbar(0) rho(0) + phibar(0) on interface cells.
template <int P>
__global__ void __launch_bounds__(128) k_adj_init(Par p, const uint8_t* flags, const typename Form<P>::S* f,
                                                  const double* f0keep, const double* abar, const double* mbar,
                                                  const double* phibar, double* theta, double* dphi0) {
  const size_t N = (size_t)p.N;
  double th[5] = {0, 0, 0, 0, 0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < p.N;
       i += (long long)gridDim.x * blockDim.x) {
    uint8_t k = flags[i] & KIND;
    dphi0[i] = 0.0;
    if (!is_fluid(k)) continue;
    double ft[19], f0[19], ab[19], fb[19];
    double r = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
      ft[q] = ldq_full<P>(f, q * N + i, q);
      ab[q] = abar[q * N + i];
      fb[q] = 0.0;
      r += ft[q];
      jx += cx(q) * ft[q];
      jy += cy(q) * ft[q];
      jz += cz(q) * ft[q];
    }
    // U = sum c f~ - g, u = U + g/2, v = U - g/lambda_-
    const double Ux = jx - p.g[0], Uy = jy - p.g[1], Uz = jz - p.g[2];
    const double ux = Ux + 0.5 * p.g[0], uy = Uy + 0.5 * p.g[1], uz = Uz + 0.5 * p.g[2];
    const double vx = Ux - p.g[0] / p.lam_m, vy = Uy - p.g[1] / p.lam_m, vz = Uz - p.g[2] / p.lam_m;
    f0[0] = eplus_d(p, 0, r, ux, uy, uz) + (ft[0] - eplus_d(p, 0, r, ux, uy, uz)) / (1.0 + p.lam_p);
#pragma unroll
    for (int q = 1; q < 19; q += 2) {
      const int qb = q + 1;
      double w = q <= 6 ? 1.0 / 18.0 : 1.0 / 36.0;
      double ep = eplus_d(p, q, r, ux, uy, uz);
      double em = 3.0 * w * (cx(q) * vx + cy(q) * vy + cz(q) * vz);
      double fp = ep + (0.5 * (ft[q] + ft[qb]) - ep) / (1.0 + p.lam_p);
      double fm = em + (0.5 * (ft[q] - ft[qb]) - em) / (1.0 + p.lam_m);
      f0[q] = fp + fm;
      f0[qb] = fp - fm;
    }
    if (f0keep) {  // the initial populations as set, in FP64
      r = 0.0;
#pragma unroll
      for (int q = 0; q < 19; ++q) {
        f0[q] = f0keep[(size_t)q * N + i];
        r += f0[q];
      }
    }
    collide_rev(p, f0, ab, fb, th);
    if (k == IFC) dphi0[i] = (p.freeze ? 0.0 : mbar[i] * r) + phibar[i];
  }
  block_add(th, theta);
}

// Reverse of the conversions of one step, part 1 (see the file header).
// flags0 / flags1: the flags before / after the step; f1, m1: the state after
// it (post-collision populations, mass); abar, mbar, phibar: adjoints of that
// state.  Writes Mh, rh (interface cells after the step, the list ifc1 of
// n1 cells; the entries of other cells are not read) and, per new cell from
// gas, ngb[4 j + 0..3] = (adjoint of mean rho, of mean u) / count.
template <int P>
__global__ void __launch_bounds__(128) k_adj_conv1(Par p, const uint8_t* __restrict__ flags0,
                                                   const int* __restrict__ ifc1, const int* __restrict__ n1p,
                                                   const typename Form<P>::S* __restrict__ f1,
                                                   const double* __restrict__ m1, const double* __restrict__ abar,
                                                   const double* __restrict__ mbar, const double* __restrict__ phibar,
                                                   double* __restrict__ Mh, double* __restrict__ rh,
                                                   double* __restrict__ ngb, double* theta) {
  const size_t N = (size_t)p.N;
  double th[5] = {0, 0, 0, 0, 0};
  const int n1 = *n1p;
  for (int li = blockIdx.x * blockDim.x + threadIdx.x; li < n1; li += gridDim.x * blockDim.x) {
    const long long i = FSL_CK(p, ifc1[li], p.N);
    const uint8_t k0 = flags0[i] & KIND;
    double r = 0.0;
#pragma unroll
    for (int q = 0; q < 19; ++q) r += ldq_full<P>(f1, q * N + i, q);
    // phi = m / rho after the step
    const double pb = phibar[i];
    const double Mhat = mbar[i] + pb / r;
    const double rhat = -pb * m1[i] / (r * r);
    Mh[i] = Mhat;
    rh[i] = rhat;
    if (k0 != GAS) continue;
    // a new cell from gas: f~ = C(f^eq(rbar, ubar)), means over the fluid
    // neighbours (flags before the step) of their rho = sum f~ and
    // u = sum c f~ - g/2 (rho_0 = 1)
    int x, y, z;
    coords(p, i, x, y, z);
    double rs = 0.0, us[3] = {0.0, 0.0, 0.0};
    int cnt = 0;
    for (int l = 1; l < 19; ++l) {
      const long long yj = nbr(p, x, y, z, cx(l), cy(l), cz(l));
      if (yj < 0 || !is_fluid(flags0[yj] & KIND)) continue;
      double ry = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
      for (int q = 0; q < 19; ++q) {
        const double v = ldq_full<P>(f1, q * N + yj, q);
        ry += v;
        jx += cx(q) * v;
        jy += cy(q) * v;
        jz += cz(q) * v;
      }
      rs += ry;
      us[0] += jx - 0.5 * p.g[0];
      us[1] += jy - 0.5 * p.g[1];
      us[2] += jz - 0.5 * p.g[2];
      ++cnt;
    }
    ngb[4 * i] = ngb[4 * i + 1] = ngb[4 * i + 2] = ngb[4 * i + 3] = 0.0;
    if (!cnt) continue;
    const double rbar = rs / cnt, ub0 = us[0] / cnt, ub1 = us[1] / cnt, ub2 = us[2] / cnt;
    double feq[19], ab[19], fb[19];
#pragma unroll
    for (int q = 0; q < 19; ++q) {
      const double w = q == 0 ? 1.0 / 3.0 : (q <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
      feq[q] = eplus_d(p, q, rbar, ub0, ub1, ub2) + 3.0 * w * (cx(q) * ub0 + cy(q) * ub1 + cz(q) * ub2);
      // its density after the step, sum f~ = sum f^eq, carries rhat
      ab[q] = abar[q * N + i] + rhat;
      fb[q] = 0.0;
    }
    collide_rev(p, feq, ab, fb, th);
    double rb = 0.0, ubr[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int q = 0; q < 19; ++q) {
      const double w = q == 0 ? 1.0 / 3.0 : (q <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
      rb += w * fb[q];
      deplus_du(p, q, ub0, ub1, ub2, fb[q], ubr);
      ubr[0] += 3.0 * w * cx(q) * fb[q];
      ubr[1] += 3.0 * w * cy(q) * fb[q];
      ubr[2] += 3.0 * w * cz(q) * fb[q];
    }
    // u of each neighbour carries -g/2
    th[2] -= 0.5 * ubr[0];
    th[3] -= 0.5 * ubr[1];
    th[4] -= 0.5 * ubr[2];
    ngb[4 * i] = rb / cnt;
    ngb[4 * i + 1] = ubr[0] / cnt;
    ngb[4 * i + 2] = ubr[1] / cnt;
    ngb[4 * i + 3] = ubr[2] / cnt;
  }
  warp_add(th, theta);
}

// Part 2, per fluid cell of the old flags that the conversions touch: abar
// (in place) becomes the adjoint of the step's post-collision populations
// before the conversions, mbar that of the exchanged mass m + dm, phibar zero
// (the fill levels' adjoints are in Mh / rh).  A cell liquid before and after
// the step is left as it is: no new cell from gas can neighbour it (it had
// no gas neighbour) and its populations and density pass through.  So the
// cells are the interface cells before the step (list ifc0) and the new
// interface cells from liquid (liquid cells of the list ifc1).
template <int P>
__global__ void __launch_bounds__(128) k_adj_conv2(Par p, const uint8_t* __restrict__ flags0,
                                                   const uint8_t* __restrict__ flags1,
                                                   const int* __restrict__ ifc0, const int* __restrict__ n0p,
                                                   const int* __restrict__ ifc1, const int* __restrict__ n1p,
                                                   const double* __restrict__ Mh, const double* __restrict__ rh,
                                                   const double* __restrict__ ngb, double* __restrict__ abar,
                                                   double* __restrict__ mbar, double* __restrict__ phibar) {
  const size_t N = (size_t)p.N;
  const int n0 = *n0p, n1 = *n1p;
  for (int li = blockIdx.x * blockDim.x + threadIdx.x; li < n0 + n1; li += gridDim.x * blockDim.x) {
    const long long i = FSL_CK(p, li < n0 ? ifc0[li] : ifc1[li - n0], p.N);
    const uint8_t k0 = flags0[i] & KIND, k1 = flags1[i] & KIND;
    if (li >= n0 && k0 != LIQ) continue;  // (interface before and after: done from ifc0)
    if (k0 == IFC) phibar[i] = 0.0;
    int x, y, z;
    coords(p, i, x, y, z);
    double add = 0.0, mb = 0.0;
    if (k1 == IFC) add += rh[i];                 // rho after the step = sum f~
    if (k0 == LIQ && k1 == IFC) add += Mh[i];    // new from liquid: m = rho + shares
    if (k0 == IFC) {
      if (k1 == IFC) {
        mb = Mh[i];                              // m + dm + shares
      } else {
        // filled (-> liquid) or emptied (-> gas): excess over the receivers,
        // the neighbours that are interface after the step
        double s = 0.0;
        int nr = 0;
        for (int l = 1; l < 19; ++l) {
          const long long r = nbr(p, x, y, z, cx(l), cy(l), cz(l));
          if (r < 0 || (flags1[r] & KIND) != IFC) continue;
          s += Mh[r];
          ++nr;
        }
        const double exb = nr ? s / nr : 0.0;
        mb = exb;                                // excess m + dm - rho (filled) or m + dm (emptied)
        if (k1 == LIQ) add -= exb;
      }
    }
    double ng0 = 0.0, ng1 = 0.0, ng2 = 0.0, ng3 = 0.0;  // means of the new cells from gas next to i
    for (int l = 1; l < 19; ++l) {
      const long long j = nbr(p, x, y, z, cx(l), cy(l), cz(l));
      if (j < 0 || (flags0[j] & KIND) != GAS || (flags1[j] & KIND) != IFC) continue;
      ng0 += ngb[4 * j];
      ng1 += ngb[4 * j + 1];
      ng2 += ngb[4 * j + 2];
      ng3 += ngb[4 * j + 3];
    }
    const bool keep = is_fluid(k1);  // an emptied cell's populations reach nothing else
#pragma unroll
    for (int q = 0; q < 19; ++q)
      abar[q * N + i] = (keep ? abar[q * N + i] : 0.0) + add + ng0 + cx(q) * ng1 + cy(q) * ng2 + cz(q) * ng3;
    mbar[i] = mb;
  }
}

template <int P>
static void launch_conv(const Par& p, const uint8_t* flags0, const uint8_t* flags1, const CellLists& L0,
                        const CellLists& L1, const typename Form<P>::S* f1, const double* m1, double* abar,
                        double* mbar, double* phibar, double* Mh, double* rh, double* ngb, double* theta,
                        cudaStream_t st) {
  int blocks = (int)((p.N / 8 + 127) / 128);  // (over the interface lists: a small share of the cells)
  if (blocks < 152) blocks = 152;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_adj_conv1<P><<<blocks, 128, 0, st>>>(p, flags0, L1.ifc, L1.cnt + 1, f1, m1, abar, mbar, phibar, Mh, rh, ngb,
                                         theta);
  k_adj_conv2<P><<<blocks, 128, 0, st>>>(p, flags0, flags1, L0.ifc, L0.cnt + 1, L1.ifc, L1.cnt + 1, Mh, rh, ngb,
                                         abar, mbar, phibar);
}

template <int P>
static void launch_local(const Par& p, AdjView<P> a, const CellLists& L0, cudaStream_t st) {
  int lb = (int)((p.N + 127) / 128);
  if (lb > 152 * 8) lb = 152 * 8;
  a.flist = L0.liq;
  a.nfl = L0.cnt;
  if constexpr (P != P64) {
    if (p.adj32) {
      k_adj_local<P, false, float><<<lb, 128, 0, st>>>(p, a);
      a.flist = L0.ifc;
      a.nfl = L0.cnt + 1;
      k_adj_local<P, true, float><<<lb, 128, 0, st>>>(p, a);
    } else {
      k_adj_local<P, false, double><<<lb, 128, 0, st>>>(p, a);
      a.flist = L0.ifc;
      a.nfl = L0.cnt + 1;
      k_adj_local<P, true, double><<<lb, 128, 0, st>>>(p, a);
    }
  } else {
    k_adj_local<P, false, double><<<lb, 128, 0, st>>>(p, a);
    a.flist = L0.ifc;
    a.nfl = L0.cnt + 1;
    k_adj_local<P, true, double><<<lb, 128, 0, st>>>(p, a);
  }
  int gb = (int)((p.N + 127) / 128);
  if (gb > 152 * 16) gb = 152 * 16;
  k_adj_gather<P><<<gb, 128, 0, st>>>(p, a.flags, a.Pb, a.abar_out, L0.liq, L0.ifc, L0.cnt);
}

}  // namespace fsl

template <int P>
int adj_objective(fslbm* h, double* J, double* norm) {
  AdjointState* A = h->adj;
  if (cudaMemsetAsync(A->red, 0, 4 * 8, h->st) != cudaSuccess) return 1;
  int blocks = (int)((h->par.N + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_objective<P><<<blocks, 256, 0, h->st>>>(h->par, h->flags, (const typename Form<P>::S*)cur_f(h),
                                            (const typename Form<P>::R*)cur_phi(h), A->objective, A->red);
  double r[2];
  if (cudaMemcpyAsync(r, A->red, 16, cudaMemcpyDeviceToHost, h->st) != cudaSuccess) return 1;
  if (cudaStreamSynchronize(h->st) != cudaSuccess) return 1;
  if (A->objective == 0) {
    *norm = r[1] > 0 ? 1.0 / r[1] : 0.0;
    *J = r[0] * *norm;
  } else {
    *norm = 1.0 / h->par.nx;
    *J = r[0] * *norm;
  }
  A->gseed = A->objective == 0 ? -0.5 : -0.5 * r[1] * *norm;
  return 0;
}

template <int P>
int adj_backward(fslbm* h) {
  using S = typename Form<P>::S;
  using R = typename Form<P>::R;
  AdjointState* A = h->adj;
  const size_t N = (size_t)h->par.N;
  cudaStream_t st = h->st;
  // seed from the objective at the final state
  double J = 0.0, norm = 0.0;
  if (adj_objective<P>(h, &J, &norm)) return 1;
  int blocks = (int)((N + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  cudaMemsetAsync(A->theta, 0, 8 * 8, st);
  k_obj_seed<P><<<blocks, 256, 0, st>>>(h->par, h->flags, (const S*)cur_f(h), (const R*)cur_phi(h), A->objective,
                                        norm, A->abar[0], A->phibar[0], A->mbar[0]);
  int cur = 0;
  // cell lists of the flags before (L[lb ^ 1]) and after (L[lb]) the step
  // being reversed; those after the last step from the final flags
  CellLists L[2];
  for (int b = 0; b < 2; ++b) {
    int* base = A->flist + (size_t)b * (2 * N + 2);
    L[b] = CellLists{base, base + N, base + 2 * N};
  }
  int lb = 0;
  build_lists(h->par, h->flags, L[lb], st);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float adj_total = 0.f;
  long long adj_steps = 0;
  for (int s = A->nck - 1; s >= 0; --s) {
    if (restore_state(h, (char*)A->ck_f + s * A->fbytes, A->ck_m + s * N, (char*)A->ck_phi + s * A->rbytes,
                      A->ck_flags + s * N))
      return 1;
    int n = A->nsteps - s * A->K < A->K ? A->nsteps - s * A->K : A->K;
    for (int k = 0; k <= n; ++k) {  // the states before each step and after the last
      if (save_state(h, (char*)A->seg_f + k * A->fbytes, A->seg_m + k * N, (char*)A->seg_phi + k * A->rbytes,
                     A->seg_flags + k * N))
        return 1;
      if (k < n && fslbm_step(h, 1)) return 1;
    }
    cudaEventRecord(e0, st);
    for (int k = n - 1; k >= 0; --k) {
      build_lists(h->par, A->seg_flags + k * N, L[lb ^ 1], st);
      if (!h->par.freeze)  // the step's conversions, as the forward pass took them
        launch_conv<P>(h->par, A->seg_flags + k * N, A->seg_flags + (k + 1) * N, L[lb ^ 1], L[lb],
                       (const S*)((char*)A->seg_f + (k + 1) * A->fbytes), A->seg_m + (k + 1) * N, A->abar[cur],
                       A->mbar[cur], A->phibar[cur], A->Mh, A->rh, A->ngb, A->theta, st);
      AdjView<P> a;
      a.flags = A->seg_flags + k * N;
      a.f = (const S*)((char*)A->seg_f + k * A->fbytes);
      a.m = A->seg_m + k * N;
      a.phi = (const R*)((char*)A->seg_phi + k * A->rbytes);
      a.wd = h->wd;
      a.abar_in = A->abar[cur];
      a.mbar_in = A->mbar[cur];
      a.phibar_in = A->phibar[cur];
      a.abar_out = A->abar[cur ^ 1];
      a.Pb = A->P;
      a.mbar_out = A->mbar[cur ^ 1];
      a.phibar_out = A->phibar[cur ^ 1];
      a.theta = A->theta;
      cudaMemsetAsync(a.phibar_out, 0, N * 8, st);
      launch_local<P>(h->par, a, L[lb ^ 1], st);
      cur ^= 1;
      lb ^= 1;
    }
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    adj_total += ms;
    adj_steps += n;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  A->adj_ms = adj_total / (adj_steps ? adj_steps : 1);
  // initial collision and phi0
  k_adj_init<P><<<(int)((N + 127) / 128 < 152 * 16 ? (N + 127) / 128 : 152 * 16), 128, 0, st>>>(
      h->par, A->ck_flags, (const S*)A->ck_f, h->f0_valid ? h->f0 : nullptr, A->abar[cur], A->mbar[cur],
      A->phibar[cur], A->theta, A->dphi0);
  return cudaGetLastError() != cudaSuccess;
}

// fslbm_oracle.cpp -- plain, slow FP64 CPU oracle of one free-surface
// lattice Boltzmann (FSLBM) time step on D3Q19.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
// includes this file; only the test-suite, the smoke check and the CPU
// baseline leg of the benchmark load it.  It shares no code, header, table or
// constant with the CUDA path.
//
// Paper: Bogner, Ammer, Ruede, "Boundary Conditions for Free Interfaces with
// the Lattice Boltzmann Method" (arXiv:1409.5645).  Each routine cites the
// section / equation / table it restates.  Where the paper is silent (the
// interface tracking it takes from Koerner et al. and Thuerey, Sec. 4.4) the
// reading used is stated at the routine.
//
// State at time t (the paper's cut of the loop, Eq. lbe1/lbe2): flags,
// pre-collision populations f_q(x,t), interface mass m(x,t) and fill level
// phi(x,t).  One call of step() performs
//   1. geometry of the interface from phi(t)          (Sec. 2.2, Sec. 5)
//   2. TRT collision of every liquid/interface node    (Eq. lbe2, Sec. 2.1)
//   3. pull streaming with wall and free-surface closures
//                                                      (Eq. lbe1, Eq. closure,
//                                                       Eq. koerner, Table 1)
//   4. interface mass exchange and fill update          (Sec. 2.3)
//   5. cell conversions with excess-mass redistribution (Sec. 2.3 / 4.4)
// No blocking, fusion or reordering beyond this.
//
// The scalar type is a template parameter: T = double is the oracle proper,
// T = Dual carries one forward tangent (tangent-linear model) through every
// arithmetic step, with every discrete decision (flags, thresholds, clamps,
// sorting) taken on the value part.
//
// Build: g++ -O2 -ffp-contract=off -shared -fPIC (no fused multiply-add, so
// each operation is one IEEE rounding in source order).  The same source
// built with -fopenmp (liborc_omp.so, for the all-core CPU timing only) runs
// the per-cell loops of stages 1-4 over threads; each iteration writes only
// its own cell, every sum keeps its order, and the conversions stay serial,
// so both builds give the same bits.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace orc {

// --------------------------------------------------------------------------
// Scalar types
// --------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual(double v_ = 0.0, double d_ = 0.0) : v(v_), d(d_) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }
inline Dual sqrt(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, a.d / (2.0 * s));
}
inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }
inline double tan_of(double) { return 0.0; }
inline double tan_of(const Dual& x) { return x.d; }
using std::sqrt;

template <class T> inline T absT(const T& x) { return val(x) < 0.0 ? T(-x) : x; }
template <class T> inline T with_tangent(double v, double d);
template <> inline double with_tangent<double>(double v, double) { return v; }
template <> inline Dual with_tangent<Dual>(double v, double d) { return Dual(v, d); }
template <class T> inline T clampT(const T& x, double lo, double hi) {
  if (val(x) < lo) return T(lo);
  if (val(x) > hi) return T(hi);
  return x;
}

// --------------------------------------------------------------------------
// D3Q19 velocity set (Sec. 4: "D3Q19 lattice model"), weights of Qian et al.
// (Sec. 2.1: w_q = w_|c_q|, c_s^2 = 1/3).  The ordering is the library's
// public population ordering: rest, six axis links, twelve diagonal links,
// each link directly followed by its opposite.
// --------------------------------------------------------------------------
static const int Q = 19;
static const int CV[Q][3] = {
    {0, 0, 0},                                                        //
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},  //
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},                  //
    {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},                  //
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static double weight(int q) {
  int s = CV[q][0] * CV[q][0] + CV[q][1] * CV[q][1] + CV[q][2] * CV[q][2];
  return s == 0 ? 1.0 / 3.0 : (s == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
}
// opposite direction qbar: c_qbar = -c_q (Sec. 2.1)
static int opposite(int q) {
  for (int k = 0; k < Q; ++k)
    if (CV[k][0] == -CV[q][0] && CV[k][1] == -CV[q][1] && CV[k][2] == -CV[q][2]) return k;
  return -1;
}

enum : uint8_t { LIQ = 1, IFC = 2, GAS = 4, WALL = 8 };

enum { OK = 0, ERR_ARG = -1, ERR_STATE = -4, ERR_UNSTABLE = -5 };

// Parameters.  Mirrors the library's parameter set field by field, but is
// declared here on its own.
struct Params {
  int nx, ny, nz;
  double tau;        // lambda_+ = -1/tau, nu = (tau - 1/2)/3 (Sec. 2.1)
  double magic;      // Lambda = Lambda_+ Lambda_- (Sec. 3.1); <= 0 selects SRT
  double g[3];       // body force per unit mass and step
  double rho_G;      // gas density, P_b = rho_G / 3 (Eq. koerner)
  double sigma;      // surface tension (Sec. 2.3, Laplace pressure)
  int rule;          // 0 = FSK, 1 = FSL (Table 1, D = 0)
  int compressible;  // 1: rho_0 = rho, 0: rho_0 = 1 (Sec. 2.1)
  int linear_eq;     // 1: drop N_q (Stokes flow, Sec. 2.1)
  double eps;        // conversion threshold
  int periodic[3];   // 1 = periodic axis, 0 = half-way wall at the face
  int zshift;        // z offset applied on a periodic x wrap
  int freeze;        // 1 = fixed flags and fill levels (no mass exchange, no conversion)
  int cleanup;       // bit 1: no gas neighbour -> fill; bit 2: no fluid neighbour -> empty
  double delta_min;  // lower clamp of the free-surface link fraction (0: FSL needs delta >= 0)
  int stress;        // 1: boundary shear-rate term D c_a c_b S^b_ab of Eq. bterm (Table 1's D, S^b per
                     //    Eq. bstress); 2: the same term with the prescribed S^b below (Sec. 6,
                     //    linear Couette flows); 0: D = 0
  double shear_b[6]; // prescribed S^b: xx, yy, zz, xy, xz, yz (stress = 2)
  double wall_u[3];  // velocity of every wall (half-way bounce-back links; rho_0 = 1)
  int ub_extrap;     // 1: FSL takes u_b at the surface point x_b + delta c_p (linear along the link)
  int recon_nc;      // 1: interface cells also rebuild links p with n.c_p > 0 toward a fluid node
                     //    (Koerner et al.'s reconstruction along the normal, Sec. 4.4 citation)
  int excess_split;  // 1: excess mass split with weights along the fill-level normal (Thuerey)
  int elvira;        // 1: where the height columns are open, the ELVIRA normal (Pilliod & Puckett)
                     //    in place of the Parker-Youngs one (the higher-order reconstruction of Sec. 5)
};

template <class T>
struct Sim {
  Params p;
  long N = 0;
  int opp[Q];
  double w[Q];
  T lam_p, lam_m;  // TRT relaxation rates lambda_+ / lambda_- (Eq. lbe2)
  T gv[3];
  std::vector<uint8_t> flag;
  std::vector<T> f;    // pre-collision f_q(x,t), index q*N + cell
  std::vector<T> m;    // interface mass
  std::vector<T> phi;  // fill level of interface cells
  std::vector<double> wdelta;  // wall link fractions, index q*N + cell, or empty
  T lost = T(0);
  long t = 0;
  int status = OK;
  long cnt[4] = {0, 0, 0, 0};  // last step: filled, emptied, new from gas, new from liquid

  // scratch of one step (kept so that tests may inspect them)
  std::vector<T> ft;      // post-collision f~ at time t
  std::vector<T> nplus;   // n_q^+ at time t
  std::vector<T> rho_t, u_t;  // moments at time t
  std::vector<T> gn, gd, gk;  // geometry: normal (3N), plane offset, curvature
  std::vector<uint8_t> gok;

  explicit Sim(const Params& pp) : p(pp) {
    N = (long)p.nx * p.ny * p.nz;
    for (int q = 0; q < Q; ++q) { opp[q] = opposite(q); w[q] = weight(q); }
    set_rates(T(p.tau));
    for (int a = 0; a < 3; ++a) gv[a] = T(p.g[a]);
    flag.assign(N, GAS);
    f.assign((size_t)Q * N, T(0));
    m.assign(N, T(0));
    phi.assign(N, T(0));
  }

  // Relaxation rates.  lambda_+ = -1/tau (nu = -(1/lambda_+ + 1/2)/3, Sec. 2.1).
  // Lambda_+- = -(1/2 + 1/lambda_+-) and Lambda = Lambda_+ Lambda_- (Sec. 3.1):
  // lambda_- follows from the fixed magic parameter Lambda.
  void set_rates(T tau) {
    lam_p = T(-1.0) / tau;
    if (p.magic <= 0.0) {
      lam_m = lam_p;
    } else {
      T Lp = T(-1.0) * (T(0.5) + T(1.0) / lam_p);
      T Lm = T(p.magic) / Lp;
      lam_m = T(-1.0) / (Lm + T(0.5));
    }
  }

  long idx(int x, int y, int z) const { return x + (long)p.nx * (y + (long)p.ny * z); }
  void coords(long i, int& x, int& y, int& z) const {
    x = (int)(i % p.nx);
    y = (int)((i / p.nx) % p.ny);
    z = (int)(i / ((long)p.nx * p.ny));
  }
  // Cell at x + (dx,dy,dz); -1 when that lies beyond a non-periodic face
  // (a half-way wall at the face).  A periodic x wrap also shifts z by zshift
  // (the inclined film repeats one period higher).
  long nbr(long i, int dx, int dy, int dz) const {
    int x, y, z;
    coords(i, x, y, z);
    int X = x + dx, Y = y + dy, Z = z + dz;
    if (X < 0 || X >= p.nx) {
      if (!p.periodic[0]) return -1;
      if (X < 0) { X += p.nx; Z += p.zshift; } else { X -= p.nx; Z -= p.zshift; }
    }
    if (Y < 0 || Y >= p.ny) {
      if (!p.periodic[1]) return -1;
      Y = Y < 0 ? Y + p.ny : Y - p.ny;
    }
    if (Z < 0 || Z >= p.nz) {
      if (!p.periodic[2]) return -1;
      Z = Z < 0 ? Z + p.nz : Z - p.nz;
    }
    if (X < 0 || X >= p.nx || Y < 0 || Y >= p.ny || Z < 0 || Z >= p.nz) return -1;
    return idx(X, Y, Z);
  }
  long nbq(long i, int q, int sgn) const { return nbr(i, sgn * CV[q][0], sgn * CV[q][1], sgn * CV[q][2]); }
  uint8_t type(long i) const { return i < 0 ? (uint8_t)WALL : flag[i]; }
  static bool fluid(uint8_t fl) { return fl == LIQ || fl == IFC; }

  T rho0(const T& rho) const { return p.compressible ? rho : T(1.0); }

  // Even equilibrium e_q^+ = (w_q/c_s^2) (P + N_q), P = c_s^2 rho,
  // N_q = 1/2 rho_0 u_a u_b (c_qa c_qb / c_s^2 - delta_ab)   (Eq. eqEven)
  T e_plus(int q, const T& rho, const T u[3], const T& r0) const {
    T val_ = T(w[q]) * rho;
    if (!p.linear_eq) {
      T N_q = T(0);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double cc = 3.0 * CV[q][a] * CV[q][b] - (a == b ? 1.0 : 0.0);
          N_q += T(0.5) * r0 * u[a] * u[b] * T(cc);
        }
      val_ += T(3.0 * w[q]) * N_q;
    }
    return val_;
  }
  // Odd equilibrium e_q^- = (w_q/c_s^2) rho_0 c_qa u^eq_a   (Eq. eqOdd)
  T e_minus(int q, const T u[3], const T& r0) const {
    T cu = T(0);
    for (int a = 0; a < 3; ++a) cu += T((double)CV[q][a]) * u[a];
    return T(3.0 * w[q]) * r0 * cu;
  }
  // Equilibrium f^eq = e^+ + e^- at (rho, u), used for initial states and for
  // cells newly created from gas.
  T f_eq(int q, const T& rho, const T u[3]) const {
    T r0 = rho0(rho);
    return e_plus(q, rho, u, r0) + e_minus(q, u, r0);
  }

  // Moments (Eq. density / momentum): rho = sum f, rho_0 U = sum c f,
  // u = U + F/(2 rho_0), with the force F = rho_0 g.
  void moments(const T* fq, T& rho, T U[3], T u[3]) const {
    rho = T(0);
    T j[3] = {T(0), T(0), T(0)};
    for (int q = 0; q < Q; ++q) {
      rho += fq[q];
      for (int a = 0; a < 3; ++a)
        if (CV[q][a] != 0) j[a] += T((double)CV[q][a]) * fq[q];
    }
    T r0 = rho0(rho);
    for (int a = 0; a < 3; ++a) {
      U[a] = j[a] / r0;
      u[a] = U[a] + T(0.5) * gv[a];
    }
  }

  // TRT collision (Eq. lbe2): f~ = f + lambda_+ n^+ + lambda_- n^-, with
  // n^+- = f^+- - e^+-, f^+- = (f_q +- f_qbar)/2, and the force entering
  // through the shifted equilibrium velocity u^eq = U - F/lambda_- (Sec. 2.1,
  // no source term F_q).  Returns rho and u of the pre-collision state.
  void collide(const T* fq, T* out, T* np_out, T& rho, T u[3]) const {
    T U[3];
    moments(fq, rho, U, u);
    T r0 = rho0(rho);
    T ueq[3];
    for (int a = 0; a < 3; ++a) ueq[a] = U[a] - gv[a] / lam_m;
    for (int q = 0; q < Q; ++q) {
      int qb = opp[q];
      T fp = T(0.5) * (fq[q] + fq[qb]);
      T fm = T(0.5) * (fq[q] - fq[qb]);
      T np = fp - e_plus(q, rho, u, r0);
      T nm = fm - e_minus(q, ueq, r0);
      out[q] = fq[q] + lam_p * np + lam_m * nm;
      if (np_out) np_out[q] = np;
    }
  }

  // Fill level of a cell: 1 for liquid, the stored value for interface and
  // gas cells (0 for gas in a dynamic run; a frozen run may give gas cells a
  // partial fill whose node lies outside the liquid).
  T phi_of(long i) const {
    uint8_t ty = type(i);
    if (ty == LIQ) return T(1.0);
    if (ty == IFC || ty == GAS) return phi[i];
    return T(0.0);
  }

  // ---------------------------------------------------------------------
  // Geometry of the free surface (Sec. 2.2: x_w = x_b + delta c_q on the
  // boundary, 0 <= delta <= 1; Sec. 5: delta must come from an interface
  // position of matching accuracy).  Reading: normal from height functions
  // (exact for planes), Parker-Youngs where the columns are not closed; plane
  // offset from the fill level by inverting the plane/cube volume; curvature
  // from the same heights.
  // ---------------------------------------------------------------------

  // Volume of {m.x <= alpha} inside the unit cube, m sorted ascending,
  // m1+m2+m3 = 1, all >= 0.  Piecewise cubic; written in a form with no
  // division by a vanishing component.
  static T cube_volume(T alpha, const T ms[3]) {
    if (val(alpha) <= 0.0) return T(0.0);
    if (val(alpha) >= 1.0) return T(1.0);
    if (val(alpha) > 0.5) return T(1.0) - cube_volume(T(1.0) - alpha, ms);
    const T &m1 = ms[0], &m2 = ms[1], &m3 = ms[2];
    if (val(alpha) <= val(m1))  // corner tetrahedron
      return alpha * alpha * alpha / (T(6.0) * m1 * m2 * m3);
    T base = T(3.0) * alpha * alpha - T(3.0) * alpha * m1 + m1 * m1;
    if (val(alpha) <= val(m2)) return base / (T(6.0) * m2 * m3);
    T m12 = m1 + m2;
    if (val(m3) >= val(m12)) {
      if (val(alpha) <= val(m12)) {
        T s = alpha - m2;
        return (base - s * s * s / m1) / (T(6.0) * m2 * m3);
      }
      return (alpha - T(0.5) * m12) / m3;
    }
    T s = alpha - m2;
    if (val(alpha) <= val(m3)) return (base - s * s * s / m1) / (T(6.0) * m2 * m3);
    T r = alpha - m3;
    return (base - s * s * s / m1 - r * r * r / m1) / (T(6.0) * m2 * m3);
  }
  // d V / d alpha (the plane's cross-section area), same pieces.
  static T cube_area(T alpha, const T ms[3]) {
    if (val(alpha) <= 0.0 || val(alpha) >= 1.0) return T(0.0);
    if (val(alpha) > 0.5) return cube_area(T(1.0) - alpha, ms);
    const T &m1 = ms[0], &m2 = ms[1], &m3 = ms[2];
    if (val(alpha) <= val(m1)) return alpha * alpha / (T(2.0) * m1 * m2 * m3);
    T base = T(6.0) * alpha - T(3.0) * m1;
    if (val(alpha) <= val(m2)) return base / (T(6.0) * m2 * m3);
    T m12 = m1 + m2;
    T s = alpha - m2;
    if (val(m3) >= val(m12)) {
      if (val(alpha) <= val(m12)) return (base - T(3.0) * s * s / m1) / (T(6.0) * m2 * m3);
      return T(1.0) / m3;
    }
    if (val(alpha) <= val(m3)) return (base - T(3.0) * s * s / m1) / (T(6.0) * m2 * m3);
    T r = alpha - m3;
    return (base - T(3.0) * s * s / m1 - T(3.0) * r * r / m1) / (T(6.0) * m2 * m3);
  }

  // Plane offset d (from the cell centre, along the unit normal n pointing
  // from liquid to gas) such that the liquid side {n.(x - x_c) <= d} fills the
  // fraction ph of the unit cell.  The inverse volume has a cube-root
  // singularity at an empty or full corner (alpha ~ (6 m1 m2 m3 ph)^(1/3)), so
  // the fill is first kept in [PH_REG, 1 - PH_REG]; the plane constant is the
  // bisection result, and a tangent (if any) gets the implicit derivative
  // d alpha = -(dV|_m - d ph) / V'(alpha).
  static constexpr double PH_REG = 1e-9;
  static T plic_offset(const T n[3], T ph) {
    T ms[3] = {absT(n[0]), absT(n[1]), absT(n[2])};
    T L1 = ms[0] + ms[1] + ms[2];
    for (int a = 0; a < 3; ++a) ms[a] = ms[a] / L1;
    std::sort(ms, ms + 3, [](const T& a, const T& b) { return val(a) < val(b); });
    ph = clampT(ph, PH_REG, 1.0 - PH_REG);
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 200; ++it) {
      double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (val(cube_volume(T(mid), ms)) < val(ph)) lo = mid; else hi = mid;
    }
    double a0 = 0.5 * (lo + hi);
    T alpha = T(a0);
    T area = cube_area(alpha, ms);
    if (val(area) > 0.0) {
      T corr = (cube_volume(alpha, ms) - ph) / area;
      alpha = with_tangent<T>(a0, -tan_of(corr));
    }
    return L1 * (alpha - T(0.5));
  }

  // Parker-Youngs gradient: 3x3x3 stencil, weights (2-|o_b|)(2-|o_c|) for the
  // derivative along a; wall or out-of-domain neighbours take the centre value.
  void normal_py(long i, T n[3]) const {
    T grad[3] = {T(0), T(0), T(0)};
    T pc = phi_of(i);
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (!dx && !dy && !dz) continue;
          long j = nbr(i, dx, dy, dz);
          T pj = (type(j) == WALL) ? pc : phi_of(j);
          int o[3] = {dx, dy, dz};
          for (int a = 0; a < 3; ++a) {
            if (o[a] == 0) continue;
            int b = (a + 1) % 3, c = (a + 2) % 3;
            double wgt = (double)((2 - std::abs(o[b])) * (2 - std::abs(o[c])));
            grad[a] += T(wgt * o[a]) * pj;
          }
        }
    for (int a = 0; a < 3; ++a) n[a] = -grad[a];
  }

  // Geometry of interface cell i at time t.  ok=false when no normal exists.
  // With closed height columns the plane passes through the column-centre
  // height H(0,0) along the dominant axis a: the liquid fills the column from
  // its liquid end (3.5 cells from the node), so the signed distance of the
  // plane from the node along n is d = |n_a| (H(0,0) - 3.5).  Otherwise the
  // plane offset comes from the cell's own fill level (PLIC).
  void geometry(long i, T n[3], T& d, T& kappa, bool& ok) const {
    kappa = T(0);
    normal_py(i, n);
    double nn = val(n[0]) * val(n[0]) + val(n[1]) * val(n[1]) + val(n[2]) * val(n[2]);
    if (!(nn > 1e-24)) { ok = false; d = T(0); n[0] = n[1] = T(0); n[2] = T(1); return; }
    ok = true;
    // dominant axis (first strict maximum of |n_a|)
    int a = 0;
    for (int k = 1; k < 3; ++k)
      if (std::fabs(val(n[k])) > std::fabs(val(n[a]))) a = k;
    int s = val(n[a]) > 0 ? 1 : -1;
    int b = (a == 0) ? 1 : 0;
    int c = (a == 2) ? 1 : 2;
    // heights over the 3x3 columns of 7 cells along a
    T H[3][3];
    bool closed = true;
    for (int ib = -1; ib <= 1 && closed; ++ib)
      for (int ic = -1; ic <= 1 && closed; ++ic) {
        T sum = T(0);
        for (int k = -3; k <= 3; ++k) {
          int o[3] = {0, 0, 0};
          o[a] = k; o[b] = ib; o[c] = ic;
          long j = nbr(i, o[0], o[1], o[2]);
          uint8_t ty = type(j);
          if (ty == WALL) { closed = false; break; }
          if (k == -3 * s && ty != LIQ) { closed = false; break; }
          if (k == 3 * s && ty != GAS) { closed = false; break; }
          sum += phi_of(j);
        }
        H[ib + 1][ic + 1] = sum;
      }
    if (closed) {
      T Hb = T(0.5) * (H[2][1] - H[0][1]);
      T Hc = T(0.5) * (H[1][2] - H[1][0]);
      T v[3];
      v[a] = T((double)s); v[b] = -Hb; v[c] = -Hc;
      T len = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      for (int k = 0; k < 3; ++k) n[k] = v[k] / len;
      d = absT(n[a]) * (H[1][1] - T(3.5));
      if (p.sigma != 0.0) {
        // mean curvature of the height surface, positive for convex liquid
        T Hbb = H[2][1] - T(2.0) * H[1][1] + H[0][1];
        T Hcc = H[1][2] - T(2.0) * H[1][1] + H[1][0];
        T Hbc = T(0.25) * (H[2][2] - H[2][0] - H[0][2] + H[0][0]);
        T q2 = T(1.0) + Hb * Hb + Hc * Hc;
        T num = Hbb * (T(1.0) + Hc * Hc) + Hcc * (T(1.0) + Hb * Hb) - T(2.0) * Hb * Hc * Hbc;
        kappa = T(-1.0) * num / (q2 * sqrt(q2));
      }
    } else {
      // curvature only: heights along the other axes, by decreasing |n_a|,
      // where the columns along the dominant one are not closed
      if (p.sigma != 0.0) {
        int ax[2] = {(a + 1) % 3, (a + 2) % 3};
        if (std::fabs(val(n[ax[1]])) > std::fabs(val(n[ax[0]]))) std::swap(ax[0], ax[1]);
        bool got = false;
        for (int t = 0; t < 2 && !got; ++t) got = height_curvature(i, ax[t], val(n[ax[t]]) > 0 ? 1 : -1, kappa);
        if (!got) kappa = normal_divergence(i, n);
      }
      if (p.elvira) {
        elvira(i, n, d);
      } else {
        T len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        for (int k = 0; k < 3; ++k) n[k] = n[k] / len;
        d = plic_offset(n, phi_of(i));
      }
    }
  }

  // Volume fraction of the unit cell around a node on the side n.x <= d of
  // the plane (n a unit vector, x from the node).
  static T plane_volume(const T n[3], const T& d) {
    T ms[3] = {absT(n[0]), absT(n[1]), absT(n[2])};
    T L1 = ms[0] + ms[1] + ms[2];
    for (int a = 0; a < 3; ++a) ms[a] = ms[a] / L1;
    std::sort(ms, ms + 3, [](const T& a, const T& b) { return val(a) < val(b); });
    return cube_volume(d / L1 + T(0.5), ms);
  }

  // ELVIRA (Pilliod and Puckett, "Second-order accurate volume-of-fluid
  // algorithms for tracking material interfaces", J. Comput. Phys. 2004),
  // in three dimensions: along each axis a, the fill levels of the 3x3x3
  // block summed over 3 cells give column heights h(b, c); the backward,
  // central and forward differences of h in the two other axes give nine
  // candidate normals (s_a, -dh/db, -dh/dc), s_a the gas side of a (the sign
  // of the Parker-Youngs component).  For each of the 27 candidates the plane
  // through the cell's own fill is continued through the block; the one whose
  // volume fractions match the block's fill levels best (least squares over
  // the cells that are not walls, first minimum in the order a, b-difference,
  // c-difference) gives the normal and the offset.  n: the Parker-Youngs
  // normal on entry (not normalised).  A wall in a column takes the cell's own
  // fill level, as in the gradient.
  void elvira(long i, T n[3], T& d) const {
    const T phc = phi_of(i);
    const T npy[3] = {n[0], n[1], n[2]};
    double best = 1e300;
    for (int a = 0; a < 3; ++a) {
      const int s = val(npy[a]) > 0 ? 1 : -1;
      const int b = (a + 1) % 3, c = (a + 2) % 3;
      T h[3][3];
      for (int ib = -1; ib <= 1; ++ib)
        for (int ic = -1; ic <= 1; ++ic) {
          T sum = T(0);
          for (int k = -1; k <= 1; ++k) {
            int o[3] = {0, 0, 0};
            o[a] = k; o[b] = ib; o[c] = ic;
            long j = nbr(i, o[0], o[1], o[2]);
            sum += type(j) == WALL ? phc : phi_of(j);
          }
          h[ib + 1][ic + 1] = sum;
        }
      const T db[3] = {h[1][1] - h[0][1], T(0.5) * (h[2][1] - h[0][1]), h[2][1] - h[1][1]};
      const T dc[3] = {h[1][1] - h[1][0], T(0.5) * (h[1][2] - h[1][0]), h[1][2] - h[1][1]};
      for (int kb = 0; kb < 3; ++kb)
        for (int kc = 0; kc < 3; ++kc) {
          T v[3];
          v[a] = T((double)s); v[b] = T(-1.0) * db[kb]; v[c] = T(-1.0) * dc[kc];
          T len = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
          T m[3] = {v[0] / len, v[1] / len, v[2] / len};
          T dd = plic_offset(m, phc);
          double err = 0.0;
          for (int oz = -1; oz <= 1; ++oz)
            for (int oy = -1; oy <= 1; ++oy)
              for (int ox = -1; ox <= 1; ++ox) {
                if (!ox && !oy && !oz) continue;
                long j = nbr(i, ox, oy, oz);
                if (type(j) == WALL) continue;
                T shift = m[0] * T((double)ox) + m[1] * T((double)oy) + m[2] * T((double)oz);
                double e = val(plane_volume(m, dd - shift)) - val(phi_of(j));
                err += e * e;
              }
          if (err < best) {
            best = err;
            for (int k = 0; k < 3; ++k) n[k] = m[k];
            d = dd;
          }
        }
    }
  }

  // Curvature as the divergence of the unit Parker-Youngs normal by central
  // differences over the six face neighbours; a neighbour without a normal
  // takes the cell's own (n0, not normalised on entry).
  T normal_divergence(long i, const T n0[3]) const {
    T l0 = sqrt(n0[0] * n0[0] + n0[1] * n0[1] + n0[2] * n0[2]);
    T k = T(0);
    for (int a = 0; a < 3; ++a) {
      T comp[2];
      for (int sgn = 0; sgn < 2; ++sgn) {
        int o[3] = {0, 0, 0};
        o[a] = sgn ? 1 : -1;
        long j = nbr(i, o[0], o[1], o[2]);
        T nj[3] = {n0[0], n0[1], n0[2]};
        T lj = l0;
        if (j >= 0 && type(j) != WALL) {
          T m[3];
          normal_py(j, m);
          T lm = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
          if (val(lm) > 1e-12) { nj[0] = m[0]; nj[1] = m[1]; nj[2] = m[2]; lj = lm; }
        }
        comp[sgn] = nj[a] / lj;
      }
      k += T(0.5) * (comp[1] - comp[0]);
    }
    return k;
  }

  // Curvature from the heights over 3x3 columns of 7 cells along axis a,
  // gas side s; false (kappa untouched) where a column is not closed.
  bool height_curvature(long i, int a, int s, T& kappa) const {
    const int b = (a == 0) ? 1 : 0;
    const int c = (a == 2) ? 1 : 2;
    T H[3][3];
    for (int ib = -1; ib <= 1; ++ib)
      for (int ic = -1; ic <= 1; ++ic) {
        T sum = T(0);
        for (int k = -3; k <= 3; ++k) {
          int o[3] = {0, 0, 0};
          o[a] = k; o[b] = ib; o[c] = ic;
          long j = nbr(i, o[0], o[1], o[2]);
          uint8_t ty = type(j);
          if (ty == WALL) return false;
          if (k == -3 * s && ty != LIQ) return false;
          if (k == 3 * s && ty != GAS) return false;
          sum += phi_of(j);
        }
        H[ib + 1][ic + 1] = sum;
      }
    T Hb = T(0.5) * (H[2][1] - H[0][1]);
    T Hc = T(0.5) * (H[1][2] - H[1][0]);
    T Hbb = H[2][1] - T(2.0) * H[1][1] + H[0][1];
    T Hcc = H[1][2] - T(2.0) * H[1][1] + H[1][0];
    T Hbc = T(0.25) * (H[2][2] - H[2][0] - H[0][2] + H[0][0]);
    T q2 = T(1.0) + Hb * Hb + Hc * Hc;
    T num = Hbb * (T(1.0) + Hc * Hc) + Hcc * (T(1.0) + Hb * Hb) - T(2.0) * Hb * Hc * Hbc;
    kappa = T(-1.0) * num / (q2 * sqrt(q2));
    return true;
  }

  // Link fraction along c_q for a gas link: x_w = x_b + delta c_q lies on the
  // plane n.(x - x_b) = d, so delta = d / (n.c_q); clamped to [delta_min, 1];
  // 1/2 when the link does not point to the gas side.
  T link_delta(int q, const T n[3], const T& d, bool ok) const {
    if (!ok) return T(0.5);
    T cn = T(0);
    for (int a = 0; a < 3; ++a) cn += T((double)CV[q][a]) * n[a];
    if (!(val(cn) > 0.0)) return T(0.5);
    return clampT(d / cn, p.delta_min, 1.0);
  }

  // ---------------------------------------------------------------------
  // One time step t -> t+1.
  // ---------------------------------------------------------------------
  void clear_scratch() {
    const long NN = N;
    ft.assign((size_t)Q * NN, T(0));
    nplus.assign((size_t)Q * NN, T(0));
    rho_t.assign(NN, T(0));
    u_t.assign((size_t)3 * NN, T(0));
    gn.assign((size_t)3 * NN, T(0));
    gd.assign(NN, T(0));
    gk.assign(NN, T(0));
    gok.assign(NN, 0);
  }

  // 1. geometry at time t
  void stage_geometry() {
#pragma omp parallel for schedule(dynamic, 4096)
    for (long i = 0; i < N; ++i) {
      if (flag[i] != IFC) continue;
      T n[3], d, k;
      bool ok;
      geometry(i, n, d, k, ok);
      for (int a = 0; a < 3; ++a) gn[3 * i + a] = n[a];
      gd[i] = d; gk[i] = k; gok[i] = ok ? 1 : 0;
    }
  }

  int step() {
    const long NN = N;
    clear_scratch();
    stage_geometry();
    // 2. collision at time t (Eq. lbe2)
#pragma omp parallel for schedule(static)
    for (long i = 0; i < NN; ++i) {
      if (!fluid(flag[i])) continue;
      T fq[Q], out[Q], np[Q], rho, u[3];
      for (int q = 0; q < Q; ++q) fq[q] = f[(size_t)q * NN + i];
      collide(fq, out, np, rho, u);
      for (int q = 0; q < Q; ++q) {
        ft[(size_t)q * NN + i] = out[q];
        nplus[(size_t)q * NN + i] = np[q];
      }
      rho_t[i] = rho;
      for (int a = 0; a < 3; ++a) u_t[3 * i + a] = u[a];
    }
    return stream_and_convert();
  }

  // One step from a post-collision state f~(t) given directly (test entry for
  // sampled windows of a large lattice).  The moments of the pre-collision
  // state follow from f~ (sum f~ = rho, sum c f~ = rho_0 U + F) and
  // n^+ = (f~^+ - e^+) / (1 + lambda_+) (Eq. lbe2 restricted to the even part);
  // n^- is not needed by the step.
  int step_from_post(const double* ftp) {
    const long NN = N;
    clear_scratch();
    stage_geometry();
#pragma omp parallel for schedule(static)
    for (long i = 0; i < NN; ++i) {
      if (!fluid(flag[i])) continue;
      T r = T(0), j[3] = {T(0), T(0), T(0)};
      for (int q = 0; q < Q; ++q) {
        T v = T(ftp[(size_t)q * NN + i]);
        ft[(size_t)q * NN + i] = v;
        r += v;
        for (int a = 0; a < 3; ++a)
          if (CV[q][a] != 0) j[a] += T((double)CV[q][a]) * v;
      }
      T r0 = rho0(r);
      T u[3];
      for (int a = 0; a < 3; ++a) u[a] = j[a] / r0 - T(0.5) * gv[a];
      for (int q = 0; q < Q; ++q) {
        T fp = T(0.5) * (ft[(size_t)q * NN + i] + ft[(size_t)opp[q] * NN + i]);
        nplus[(size_t)q * NN + i] = (fp - e_plus(q, r, u, r0)) / (T(1.0) + lam_p);
      }
      rho_t[i] = r;
      for (int a = 0; a < 3; ++a) u_t[3 * i + a] = u[a];
    }
    return stream_and_convert();
  }

  // stages 3-5 of a step, from ft / nplus / rho_t / u_t / geometry of time t
  int stream_and_convert() {
    const long NN = N;
    int st = OK;

    // 3. pull streaming (Eq. lbe1) with closures for the missing populations
    std::vector<T> fn((size_t)Q * NN, T(0));
    int bad_state = 0;
#pragma omp parallel for schedule(dynamic, 4096) reduction(| : bad_state)
    for (long i = 0; i < NN; ++i) {
      if (!fluid(flag[i])) continue;
      for (int q = 0; q < Q; ++q) {
        long src = nbq(i, q, -1);  // x - c_q
        uint8_t ts = type(src);
        if (q == 0) { fn[i] = ft[i]; continue; }
        if (fluid(ts)) {
          fn[(size_t)q * NN + i] = normal_link(i, q) ? free_surface_closure(i, q) : ft[(size_t)q * NN + src];
        } else if (ts == WALL) {
          fn[(size_t)q * NN + i] = wall_closure(i, q);
        } else {  // gas source
          if (flag[i] != IFC) { bad_state = 1; fn[(size_t)q * NN + i] = ft[(size_t)opp[q] * NN + i]; continue; }
          fn[(size_t)q * NN + i] = free_surface_closure(i, q);
        }
      }
    }
    if (bad_state) st = ERR_STATE;

    // 4. mass exchange (non-frozen), Sec. 2.3 advection of phi
    std::vector<T> mn = m;
    if (!p.freeze) {
#pragma omp parallel for schedule(dynamic, 4096)
      for (long i = 0; i < NN; ++i) {
        if (flag[i] != IFC) continue;
        T dm = T(0);
        for (int q = 1; q < Q; ++q) {
          long y = nbq(i, q, -1);
          uint8_t ty = type(y);
          if (!fluid(ty)) continue;
          T sw = (ty == LIQ) ? T(1.0) : T(0.5) * (phi[i] + phi[y]);
          dm += sw * (ft[(size_t)q * NN + y] - ft[(size_t)opp[q] * NN + i]);
        }
        mn[i] = m[i] + dm;
      }
    }
    f.swap(fn);
    m.swap(mn);

    // density at t+1 and instability check
    std::vector<T> rho1(NN, T(0));
    int unstable = 0;
#pragma omp parallel for schedule(static) reduction(| : unstable)
    for (long i = 0; i < NN; ++i) {
      if (!fluid(flag[i])) continue;
      T r = T(0);
      for (int q = 0; q < Q; ++q) r += f[(size_t)q * NN + i];
      rho1[i] = r;
      if (!(val(r) > 0.0) || !std::isfinite(val(r))) unstable = 1;
    }
    if (unstable && st == OK) st = ERR_UNSTABLE;

    // 5. conversions (non-frozen)
    cnt[0] = cnt[1] = cnt[2] = cnt[3] = 0;
    if (!p.freeze) {
      convert(rho1);
#pragma omp parallel for schedule(static)
      for (long i = 0; i < NN; ++i)
        if (flag[i] == IFC) phi[i] = m[i] / rho1[i];
    }
    ++t;
    if (st != OK && status == OK) status = st;
    return st;
  }

  // Koerner et al.'s extra reconstruction (recon_nc): at an interface cell
  // with a surface normal n (pointing into the gas), the population f_q whose
  // source x - c_q = x + c_p is a fluid node is rebuilt by the free-surface
  // closure as well when n.c_p > 0, i.e. when the link points to the gas side
  // of the surface.  A margin of 1e-6 keeps links that are tangent to the
  // surface (n.c_p = 0 up to rounding) out of the set.
  bool normal_link(long i, int q) const {
    if (!p.recon_nc || flag[i] != IFC || !gok[i]) return false;
    const int pq = opp[q];
    const double cn = CV[pq][0] * val(gn[3 * i]) + CV[pq][1] * val(gn[3 * i + 1]) + CV[pq][2] * val(gn[3 * i + 2]);
    return cn > 1e-6;
  }

  // Wall closure for population q at fluid cell i whose source x - c_q is a
  // wall.  The outgoing link is p = qbar (x + c_p is the wall).  Half-way
  // bounce-back f_q(x,t+1) = f~_p(x,t) (Sec. 4.2/4.3); with a link fraction
  // delta_w the CLI rule of Ginzburg (Sec. 4.2/4.3) in the Eq. closure form
  // a_0 = 1, abar_0 = -k, a_1 = k, k = (1 - 2 delta_w)/(1 + 2 delta_w).
  T wall_closure(long i, int q) const {
    const long NN = N;
    int pq = opp[q];
    T bb = ft[(size_t)pq * NN + i];
    if (wdelta.empty()) {
      // a moving wall adds -2 w_p rho_0 (c_p.u_w)/c_s^2 = 6 w_q (c_q.u_w) for the
      // link arriving from it (c_q = -c_p), rho_0 = 1
      const double cu = CV[q][0] * p.wall_u[0] + CV[q][1] * p.wall_u[1] + CV[q][2] * p.wall_u[2];
      if (cu != 0.0) bb = bb + T(6.0 * w[q] * cu);
      return bb;
    }
    double dw = wdelta[(size_t)pq * NN + i];
    if (!(dw >= 0.0)) return bb;
    long up = nbq(i, pq, -1);  // x - c_p
    if (!fluid(type(up))) return bb;
    double k = (1.0 - 2.0 * dw) / (1.0 + 2.0 * dw);
    return bb + T(k) * (ft[(size_t)pq * NN + up] - ft[(size_t)q * NN + i]);
  }

  // Free-surface closure for population q at interface cell i whose source
  // x - c_q is gas.  In the paper's notation the boundary link is p = qbar
  // (x_b + c_p is gas) and the missing population is f_pbar = f_q.
  //   FSK (Eq. koerner):  f_q = -f~_p(x_b) + 2 e_p^+(rho_b, u_b)
  //   FSL (Eq. closure with Table 1, D = 0):
  //     f_q = (1/2 - delta) f~_p(x_b) + 1/2 f~_q(x_b) + (delta - 1) f~_p(x_b - c_p)
  //           + C n_p^+(x_b),  C = lambda_+ (1/2 + delta) - 2 lambda_+,
  //           + alpha_+ e_p^+(rho_b, u_b),  alpha_+ = 1
  // rho_b = rho_G + 3 sigma kappa (Laplace pressure in place of P_b, Sec. 2.3),
  // u_b = u(x_b, t) (next-neighbour extrapolation, Sec. 4.5; with ub_extrap the
  // FSL links take its linear extrapolation to x_w).  FSL falls back
  // to FSK on a link whose upstream node x_b - c_p is not liquid/interface.
  T free_surface_closure(long i, int q) const {
    const long NN = N;
    int pq = opp[q];
    T rb = T(p.rho_G);
    if (p.sigma != 0.0) rb = rb + T(3.0 * p.sigma) * gk[i];
    T ub[3] = {u_t[3 * i], u_t[3 * i + 1], u_t[3 * i + 2]};
    T eb = e_plus(pq, rb, ub, rho0(rb));
    T ftp = ft[(size_t)pq * NN + i];
    long up = nbq(i, pq, -1);  // x_b - c_p
    if (p.rule == 0 || !fluid(type(up))) {
      T fq = T(-1.0) * ftp + T(2.0) * eb;
      if (p.stress) fq = fq + stress_term(i, pq, 2.0);
      return fq;
    }
    T n[3] = {gn[3 * i], gn[3 * i + 1], gn[3 * i + 2]};
    T dl = link_delta(pq, n, gd[i], gok[i] != 0);
    if (p.ub_extrap) {
      // u_b at the surface point x_w = x_b + delta c_p, linear in the values at
      // x_b and x_b - c_p along the link (the boundary velocity of Eq. koerner,
      // extrapolated from the nodes)
      T uw[3];
      for (int a = 0; a < 3; ++a) uw[a] = ub[a] + dl * (ub[a] - u_t[3 * up + a]);
      eb = e_plus(pq, rb, uw, rho0(rb));
    }
    T a0 = T(0.5) - dl;
    T ab0 = T(0.5);
    T a1 = dl - T(1.0);
    T C = lam_p * (T(0.5) + dl) - T(2.0) * lam_p;
    T fq = a0 * ftp + ab0 * ft[(size_t)q * NN + i] + a1 * ft[(size_t)pq * NN + up] +
           C * nplus[(size_t)pq * NN + i] + eb;
    if (p.stress) fq = fq + stress_term(i, pq, 1.0);
    return fq;
  }

  // Boundary shear-rate term of Eq. bterm for the gas link p of interface
  // cell i: D c_p,a c_p,b S^b_ab with D = -alpha_+ Lambda_+ w_p / c_s^2
  // (Table 1: alpha_+ = 2 FSK, 1 FSL; Lambda_+ = tau - 1/2).  S is extrapolated
  // from the cell's own non-equilibrium part (the leading order of Eq. nqp,
  // incompressible: sum_q c_qa c_qb n_q^+ = (2 c_s^2 / lambda_+) S_ab), and
  // S^b is S with its normal-tangential components set to zero in the basis of
  // the interface normal n (Eq. proj2 through Eq. bstress), the others kept:
  //   S^b = S - (S n) n^T - n (S n)^T + 2 (n.S.n) n n^T.
  // Without a normal, S^b = S.
  T stress_term(long i, int pq, double alpha) const {
    const long NN = N;
    T S[3][3];
    if (p.stress == 2) {  // prescribed S^b
      const double* s6 = p.shear_b;
      const double Sp[3][3] = {{s6[0], s6[3], s6[4]}, {s6[3], s6[1], s6[5]}, {s6[4], s6[5], s6[2]}};
      T ccS = T(0);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) ccS += T(CV[pq][a] * CV[pq][b] * Sp[a][b]);
      return T(-alpha * (p.tau - 0.5) * 3.0 * w[pq]) * ccS;
    }
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) S[a][b] = T(0);
    for (int q = 1; q < Q; ++q) {
      const T np = nplus[(size_t)q * NN + i];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) S[a][b] += T(CV[q][a] * CV[q][b]) * np;
    }
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) S[a][b] = T(1.5) * lam_p * S[a][b];
    if (gok[i]) {
      const T n[3] = {gn[3 * i], gn[3 * i + 1], gn[3 * i + 2]};
      T Sn[3];
      for (int a = 0; a < 3; ++a) Sn[a] = S[a][0] * n[0] + S[a][1] * n[1] + S[a][2] * n[2];
      const T snn = n[0] * Sn[0] + n[1] * Sn[1] + n[2] * Sn[2];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) S[a][b] = S[a][b] - Sn[a] * n[b] - n[a] * Sn[b] + T(2.0) * snn * n[a] * n[b];
    }
    T ccS = T(0);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) ccS += T(CV[pq][a] * CV[pq][b]) * S[a][b];
    const double Lp = p.tau - 0.5;
    return T(-alpha * Lp * 3.0 * w[pq]) * ccS;
  }

  // Normal of the fill level for the weighted excess split (Thuerey's
  // distribution along the interface normal): n = -grad phi by central
  // differences, n_a = (phi(x - e_a) - phi(x + e_a)) / 2, pointing into the
  // gas, from the fill levels after the mass exchange: liquid 1, gas 0,
  // interface m / rho, and the cell's own value across a wall or a face.
  double phi_star(long j, double own, const std::vector<T>& rho1) const {
    if (j < 0) return own;
    switch (flag[j]) {
      case LIQ: return 1.0;
      case GAS: return 0.0;
      case IFC: return val(m[j]) / val(rho1[j]);
      default: return own;
    }
  }
  void fill_normal(long i, const std::vector<T>& rho1, double* n) const {
    const double own = val(m[i]) / val(rho1[i]);
    for (int a = 0; a < 3; ++a) {
      const int qp = 1 + 2 * a, qm = 2 + 2 * a;  // +e_a and -e_a
      n[a] = 0.5 * (phi_star(nbq(i, qm, 1), own, rho1) - phi_star(nbq(i, qp, 1), own, rho1));
    }
  }
  // Weight of the neighbour x + c_q in the split of a converting cell: a
  // filled cell pushes its excess toward the gas (n.c_q > 0), an emptied cell
  // draws its deficit from the liquid side (n.c_q < 0).
  static double split_weight(const double* n, int q, bool filled) {
    const double d = CV[q][0] * n[0] + CV[q][1] * n[1] + CV[q][2] * n[2];
    return filled ? (d > 0.0 ? d : 0.0) : (d < 0.0 ? -d : 0.0);
  }

  // Cell conversions after the mass update (reading of Koerner et al. /
  // Thuerey as cited in Sec. 4.4; the paper gives no details):
  //  F = {interface : m > (1+eps) rho, or no gas neighbour (cleanup bit 1)},
  //  E = {interface : m < -eps rho, or no liquid/interface neighbour (bit 2)}
  //  1. drop from E every cell next to a cell of F;
  //  2. gas neighbours of F become interface, f = f^eq(mean rho, mean u) over
  //     their liquid/interface neighbours (q order), m = 0;
  //  3. liquid neighbours of the remaining E become interface with m = rho;
  //  4. excess (F: m - rho, E: m) is split equally over the neighbours that are
  //     interface after 2-3 and not converting (excess_split 1: in proportion
  //     to split_weight along the fill-level normal, equally where no receiver
  //     lies on the weighted side); no receiver -> lost ledger;
  //  5. F -> liquid (m = rho), E -> gas (m = 0), new cells -> interface.
  void convert(std::vector<T>& rho1) {
    const long NN = N;
    std::vector<uint8_t> isF(NN, 0), isE(NN, 0), isNG(NN, 0), isNL(NN, 0);
    for (long i = 0; i < NN; ++i) {
      if (flag[i] != IFC) continue;
      bool any_gas = false, any_fluid = false;
      for (int q = 1; q < Q; ++q) {
        uint8_t tj = type(nbq(i, q, 1));
        any_gas |= tj == GAS;
        any_fluid |= fluid(tj);
      }
      // thresholds, plus Thuerey's isolated-cell rules (cleanup bits)
      if (val(m[i]) > (1.0 + p.eps) * val(rho1[i]) || ((p.cleanup & 1) && !any_gas)) isF[i] = 1;
      else if (val(m[i]) < -p.eps * val(rho1[i]) || ((p.cleanup & 2) && !any_fluid)) isE[i] = 1;
    }
    // 1.
    for (long i = 0; i < NN; ++i) {
      if (!isE[i]) continue;
      for (int q = 1; q < Q; ++q) {
        long j = nbq(i, q, 1);
        if (j >= 0 && isF[j]) { isE[i] = 0; break; }
      }
    }
    // 2.
    for (long i = 0; i < NN; ++i) {
      if (!isF[i]) continue;
      for (int q = 1; q < Q; ++q) {
        long j = nbq(i, q, 1);
        if (j >= 0 && flag[j] == GAS) isNG[j] = 1;
      }
    }
    for (long j = 0; j < NN; ++j) {
      if (!isNG[j]) continue;
      T rs = T(0), us[3] = {T(0), T(0), T(0)};
      int cntn = 0;
      for (int q = 1; q < Q; ++q) {
        long y = nbq(j, q, 1);
        if (y < 0 || !fluid(flag[y])) continue;
        T fy[Q];
        for (int k = 0; k < Q; ++k) fy[k] = f[(size_t)k * NN + y];
        T r, U[3], u[3];
        moments(fy, r, U, u);
        rs += r;
        for (int a = 0; a < 3; ++a) us[a] += u[a];
        ++cntn;
      }
      T rbar = rs / T((double)cntn);
      T ubar[3];
      for (int a = 0; a < 3; ++a) ubar[a] = us[a] / T((double)cntn);
      T rn = T(0);
      for (int q = 0; q < Q; ++q) {
        f[(size_t)q * NN + j] = f_eq(q, rbar, ubar);
        rn += f[(size_t)q * NN + j];
      }
      rho1[j] = rn;
      m[j] = T(0);
    }
    // 3.
    for (long i = 0; i < NN; ++i) {
      if (!isE[i]) continue;
      for (int q = 1; q < Q; ++q) {
        long j = nbq(i, q, 1);
        if (j >= 0 && flag[j] == LIQ) isNL[j] = 1;
      }
    }
    for (long j = 0; j < NN; ++j)
      if (isNL[j]) m[j] = rho1[j];
    // 4.
    auto receiver = [&](long j) {
      if (j < 0) return false;
      if (isNG[j] || isNL[j]) return true;
      return flag[j] == IFC && !isF[j] && !isE[j];
    };
    std::vector<T> share(NN, T(0));
    std::vector<uint8_t> weighted(NN, 0);
    std::vector<double> nf;  // fill-level normals of the converting cells (weighted split)
    if (p.excess_split) nf.assign((size_t)3 * NN, 0.0);
    for (long i = 0; i < NN; ++i) {
      if (!isF[i] && !isE[i]) continue;
      T ex = isF[i] ? T(m[i] - rho1[i]) : m[i];
      int nr = 0;
      for (int q = 1; q < Q; ++q)
        if (receiver(nbq(i, q, 1))) ++nr;
      if (nr == 0) { lost += ex; continue; }
      if (p.excess_split) {
        fill_normal(i, rho1, &nf[3 * i]);
        double V = 0.0;  // sum of the receivers' weights, in q order
        for (int q = 1; q < Q; ++q)
          if (receiver(nbq(i, q, 1))) V += split_weight(&nf[3 * i], q, isF[i] != 0);
        if (V > 1e-12) { share[i] = ex / T(V); weighted[i] = 1; continue; }
      }
      share[i] = ex / T((double)nr);  // equal split (also where no receiver lies along the normal)
    }
    for (long j = 0; j < NN; ++j) {
      if (!receiver(j)) continue;
      T acc = T(0);
      bool any = false;
      for (int q = 1; q < Q; ++q) {
        long i = nbq(j, q, 1);
        if (i >= 0 && (isF[i] || isE[i])) {
          // the link from i to j is opp[q]
          if (weighted[i]) acc += share[i] * T(split_weight(&nf[3 * i], opp[q], isF[i] != 0));
          else acc += share[i];
          any = true;
        }
      }
      if (any) m[j] = m[j] + acc;
    }
    // 5.
    for (long i = 0; i < NN; ++i) {
      if (isF[i]) { flag[i] = LIQ; m[i] = rho1[i]; ++cnt[0]; }
      else if (isE[i]) { flag[i] = GAS; m[i] = T(0); phi[i] = T(0); ++cnt[1]; }
      else if (isNG[i]) { flag[i] = IFC; ++cnt[2]; }
      else if (isNL[i]) { flag[i] = IFC; ++cnt[3]; }
    }
  }

  // Total mass M = sum_liquid rho + sum_interface m + lost (in cell order).
  T total_mass() const {
    T M = T(0);
    for (long i = 0; i < N; ++i) {
      if (flag[i] == LIQ) {
        T r = T(0);
        for (int q = 0; q < Q; ++q) r += f[(size_t)q * N + i];
        M += r;
      } else if (flag[i] == IFC) {
        M += m[i];
      }
    }
    return M + lost;
  }

  int check_state() const {
    for (long i = 0; i < N; ++i) {
      uint8_t fl = flag[i];
      if (fl != LIQ && fl != IFC && fl != GAS && fl != WALL) return ERR_STATE;
      if (fl == LIQ)
        for (int q = 1; q < Q; ++q)
          if (type(nbq(i, q, 1)) == GAS) return ERR_STATE;
    }
    return OK;
  }

  // m = phi rho for interface cells, m = rho for liquid; phi = m/rho.
  void finish_state(const double* phi_in) {
    for (long i = 0; i < N; ++i) {
      m[i] = T(0);
      phi[i] = T(0);
      if (flag[i] == GAS && p.freeze && phi_in) phi[i] = T(phi_in[i]);
      if (!fluid(flag[i])) continue;
      T r = T(0);
      for (int q = 0; q < Q; ++q) r += f[(size_t)q * N + i];
      if (flag[i] == LIQ) { m[i] = r; phi[i] = T(1.0); }
      else { m[i] = T(phi_in ? phi_in[i] : 1.0) * r; phi[i] = m[i] / r; }
    }
  }
};

}  // namespace orc

// ===========================================================================
// C interface used by the tests (ctypes).  Handles are Sim<double>; a second
// handle kind Sim<Dual> carries one tangent direction.
// ===========================================================================
using namespace orc;

struct OrcHandle {
  int dual;
  Sim<double>* sd;
  Sim<Dual>* sv;
};


extern "C" void* orc_create(const Params* p, int dual) {
  if (!p || p->nx <= 0 || p->ny <= 0 || p->nz <= 0 || !(p->tau > 0.5)) return nullptr;
  OrcHandle* h = new OrcHandle{dual, nullptr, nullptr};
  if (dual) h->sv = new Sim<Dual>(*p); else h->sd = new Sim<double>(*p);
  return h;
}

extern "C" void orc_destroy(void* hv) {
  OrcHandle* h = (OrcHandle*)hv;
  if (!h) return;
  delete h->sd;
  delete h->sv;
  delete h;
}

template <class T>
static int set_state_impl(Sim<T>* s, const uint8_t* flags, const double* f, const double* phi,
                          const double* wall_delta) {
  long N = s->N;
  for (long i = 0; i < N; ++i) s->flag[i] = flags[i];
  for (long k = 0; k < (long)Q * N; ++k) s->f[k] = T(f[k]);
  if (wall_delta) s->wdelta.assign(wall_delta, wall_delta + (size_t)Q * N);
  else s->wdelta.clear();
  s->lost = T(0);
  s->t = 0;
  s->status = OK;
  s->finish_state(phi);
  return s->check_state();
}

template <class T>
static int init_impl(Sim<T>* s, const uint8_t* flags, const double* rho, const double* u,
                     const double* phi, const double* noise, const double* wall_delta) {
  long N = s->N;
  std::vector<double> f((size_t)Q * N, 0.0);
  for (long i = 0; i < N; ++i) {
    s->flag[i] = flags[i];
    if (!Sim<T>::fluid(flags[i])) continue;
    T uu[3] = {T(u[3 * i]), T(u[3 * i + 1]), T(u[3 * i + 2])};
    for (int q = 0; q < Q; ++q) {
      T fe = s->f_eq(q, T(rho[i]), uu);
      double v = val(fe) + (noise ? noise[(size_t)q * N + i] : 0.0);
      f[(size_t)q * N + i] = v;
    }
  }
  return set_state_impl(s, flags, f.data(), phi, wall_delta);
}

extern "C" int orc_init(void* hv, const uint8_t* flags, const double* rho, const double* u, const double* phi,
             const double* noise, const double* wall_delta) {
  OrcHandle* h = (OrcHandle*)hv;
  return h->dual ? init_impl(h->sv, flags, rho, u, phi, noise, wall_delta)
                 : init_impl(h->sd, flags, rho, u, phi, noise, wall_delta);
}

extern "C" int orc_set_state(void* hv, const uint8_t* flags, const double* f, const double* phi,
                  const double* wall_delta) {
  OrcHandle* h = (OrcHandle*)hv;
  return h->dual ? set_state_impl(h->sv, flags, f, phi, wall_delta)
                 : set_state_impl(h->sd, flags, f, phi, wall_delta);
}

// One step from a post-collision state: flags, f~(t) [19][N], interface m,
// and fill levels phi (as the library reports them).  FP64 handles only.
extern "C" int orc_step_from_post(void* hv, const uint8_t* flags, const double* ft, const double* m,
                                  const double* phi) {
  OrcHandle* h = (OrcHandle*)hv;
  if (h->dual) return ERR_ARG;
  Sim<double>* s = h->sd;
  for (long i = 0; i < s->N; ++i) {
    s->flag[i] = flags[i];
    s->m[i] = (flags[i] == IFC) ? m[i] : 0.0;
    s->phi[i] = (flags[i] == IFC || (flags[i] == GAS && s->p.freeze)) ? phi[i] : 0.0;
  }
  s->lost = 0.0;
  int r = s->step_from_post(ft);
  return r;
}

// Threads of the OpenMP build (n > 0 sets them); returns the count in use,
// 1 for the plain build.
extern "C" int orc_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

extern "C" int orc_step(void* hv, int n) {
  OrcHandle* h = (OrcHandle*)hv;
  int st = OK;
  for (int k = 0; k < n; ++k) {
    int r = h->dual ? h->sv->step() : h->sd->step();
    if (r != OK && st == OK) st = r;
  }
  return st;
}

// Fields: 0 f (pre-collision, 19N), 1 f~ (post-collision, 19N), 2 mass (N:
// interface m, liquid rho),
// 3 phi (N), 4 rho (N), 5 u (3N, cell-major u[3*i+a]).  Values of non-fluid
// cells are 0.  tangent=1 returns the tangent part (dual handles only).
template <class T>
static int get_impl(Sim<T>* s, int field, int tangent, double* out) {
  long N = s->N;
  auto put = [&](size_t k, const T& v) { out[k] = tangent ? tan_of(v) : val(v); };
  if (field == 0 || field == 1) {
    for (size_t k = 0; k < (size_t)Q * N; ++k) out[k] = 0.0;
    for (long i = 0; i < N; ++i) {
      if (!Sim<T>::fluid(s->flag[i])) continue;
      T fq[Q], o[Q], rho, u[3];
      for (int q = 0; q < Q; ++q) fq[q] = s->f[(size_t)q * N + i];
      if (field == 1) s->collide(fq, o, nullptr, rho, u);
      for (int q = 0; q < Q; ++q) put((size_t)q * N + i, field == 1 ? o[q] : fq[q]);
    }
    return OK;
  }
  for (long i = 0; i < N; ++i) {
    bool fl = Sim<T>::fluid(s->flag[i]);
    T fq[Q], rho = T(0), U[3], u[3] = {T(0), T(0), T(0)};
    if (fl && (field == 2 || field == 4 || field == 5)) {
      for (int q = 0; q < Q; ++q) fq[q] = s->f[(size_t)q * N + i];
      s->moments(fq, rho, U, u);
    }
    switch (field) {
      case 2: put(i, s->flag[i] == IFC ? s->m[i] : (s->flag[i] == LIQ ? rho : T(0))); break;
      case 3: put(i, s->flag[i] == LIQ ? T(1.0) : ((s->flag[i] == IFC || s->flag[i] == GAS) ? s->phi[i] : T(0))); break;
      case 4: put(i, rho); break;
      case 5: for (int a = 0; a < 3; ++a) put((size_t)3 * i + a, u[a]); break;
      default: return ERR_ARG;
    }
  }
  return OK;
}

extern "C" int orc_get(void* hv, int field, int tangent, double* out) {
  OrcHandle* h = (OrcHandle*)hv;
  return h->dual ? get_impl(h->sv, field, tangent, out) : get_impl(h->sd, field, 0, out);
}

extern "C" int orc_get_flags(void* hv, uint8_t* out) {
  OrcHandle* h = (OrcHandle*)hv;
  const std::vector<uint8_t>& fl = h->dual ? h->sv->flag : h->sd->flag;
  std::memcpy(out, fl.data(), fl.size());
  return OK;
}

// Total mass (sum_L rho + sum_I m + lost) and the lost ledger.
extern "C" double orc_total_mass(void* hv, double* lost) {
  OrcHandle* h = (OrcHandle*)hv;
  if (h->dual) {
    if (lost) *lost = h->sv->lost.v;
    return h->sv->total_mass().v;
  }
  if (lost) *lost = h->sd->lost;
  return h->sd->total_mass();
}

// Geometry of the current state: normal (3N), plane offset d (N), curvature
// (N), link fractions delta (19N, NaN where not a gas link), ok flag (N).
extern "C" int orc_geometry(void* hv, double* normal, double* d, double* kappa, double* delta, uint8_t* ok) {
  OrcHandle* h = (OrcHandle*)hv;
  if (h->dual) return ERR_ARG;
  Sim<double>* s = h->sd;
  long N = s->N;
  for (long i = 0; i < N; ++i) {
    for (int a = 0; a < 3; ++a) normal[3 * i + a] = 0.0;
    d[i] = 0.0; kappa[i] = 0.0; ok[i] = 0;
    for (int q = 0; q < Q; ++q) delta[(size_t)q * N + i] = NAN;
    if (s->flag[i] != IFC) continue;
    double n[3], dd, kk;
    bool good;
    s->geometry(i, n, dd, kk, good);
    for (int a = 0; a < 3; ++a) normal[3 * i + a] = n[a];
    d[i] = dd; kappa[i] = kk; ok[i] = good;
    for (int q = 1; q < Q; ++q)
      if (s->type(s->nbq(i, q, 1)) == GAS) delta[(size_t)q * N + i] = s->link_delta(q, n, dd, good);
  }
  return OK;
}

// Plane/cube volume and its inverse, exposed for the geometry pins.
extern "C" double orc_cube_volume(const double n[3], double d) {
  double ms[3] = {std::fabs(n[0]), std::fabs(n[1]), std::fabs(n[2])};
  double L1 = ms[0] + ms[1] + ms[2];
  for (int a = 0; a < 3; ++a) ms[a] /= L1;
  std::sort(ms, ms + 3);
  return Sim<double>::cube_volume(d / L1 + 0.5, ms);
}
extern "C" double orc_plic_offset(const double n[3], double phi) { return Sim<double>::plic_offset(n, phi); }

extern "C" int orc_counters(void* hv, long* out4, long* step) {
  OrcHandle* h = (OrcHandle*)hv;
  const long* c = h->dual ? h->sv->cnt : h->sd->cnt;
  for (int k = 0; k < 4; ++k) out4[k] = c[k];
  if (step) *step = h->dual ? h->sv->t : h->sd->t;
  return OK;
}

// Tangent seeds (dual handles): direction in tau, in g (3), and in the
// interface fill levels (N, applied as m = phi rho on the current state).
extern "C" int orc_seed(void* hv, double dtau, const double* dg, const double* dphi) {
  OrcHandle* h = (OrcHandle*)hv;
  if (!h->dual) return ERR_ARG;
  Sim<Dual>* s = h->sv;
  s->set_rates(Dual(s->p.tau, dtau));
  for (int a = 0; a < 3; ++a) s->gv[a] = Dual(s->p.g[a], dg ? dg[a] : 0.0);
  if (dphi) {
    for (long i = 0; i < s->N; ++i) {
      if (s->flag[i] != IFC) continue;
      Dual r = Dual(0);
      for (int q = 0; q < Q; ++q) r += s->f[(size_t)q * s->N + i];
      Dual ph = Dual(s->phi[i].v, dphi[i]);
      s->m[i] = ph * r;
      s->phi[i] = s->m[i] / r;
    }
  }
  return OK;
}


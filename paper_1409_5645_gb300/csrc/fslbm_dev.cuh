// fslbm_dev.cuh -- device-side building blocks of the FSLBM step (sm_103a).
//
// Layout in HBM (one handle):
//   flags  u8  [N]        cell kind (bits 0-3) + NEAR_BOUNDARY bit (static walls)
//   mark   u8  [N]        conversion marks of the current step (zero between steps)
//   fA, fB S   [19][N]    post-collision populations f~(t) / f~(t+1), SoA, x fastest
//   m      f64 [N]        interface mass
//   phiA/B R   [N]        fill level phi(t) / phi(t+1)
//   wd     f64 [19][N]    wall link fractions (only when given)
// S = double (f_q) / float / half (f_q - w_q), R = double (FP64 form) or float.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fsl {

// ---------------------------------------------------------------------------
// D3Q19 (Sec. 4), public population order.  Tables as constexpr functions so
// that fully unrolled loops fold them into immediates.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int cx(int q) {
  return (q == 1 || q == 7 || q == 9 || q == 11 || q == 13) ? 1
       : (q == 2 || q == 8 || q == 10 || q == 12 || q == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cy(int q) {
  return (q == 3 || q == 7 || q == 10 || q == 15 || q == 17) ? 1
       : (q == 4 || q == 8 || q == 9 || q == 16 || q == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cz(int q) {
  return (q == 5 || q == 11 || q == 14 || q == 15 || q == 18) ? 1
       : (q == 6 || q == 12 || q == 13 || q == 16 || q == 17) ? -1 : 0;
}
// each link is followed by its opposite
__host__ __device__ constexpr int inv(int q) { return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1); }
template <class R>
__host__ __device__ constexpr R wq(int q) {
  return q == 0 ? R(1) / R(3) : (q <= 6 ? R(1) / R(18) : R(1) / R(36));
}

// static bits beside the kind: NEARB a neighbour is a wall (a WALL cell or
// beyond a non-periodic face); NEARW a neighbour is a WALL cell of the lattice
enum : uint8_t { LIQ = 1, IFC = 2, GAS = 4, WALL = 8, KIND = 15, NEARB = 16, NEARW = 32, STATIC_BITS = 48 };
enum : uint8_t { MK_FILL = 1, MK_EMPTY = 2, MK_NEWG = 4, MK_NEWL = 8, MK_RECV = 16, MK_WSPLIT = 32 };
enum : int { ERRB_STATE = 1, ERRB_UNSTABLE = 2, ERRB_OVERFLOW = 4, ERRB_TMA = 8, ERRB_SYNC = 16, ERRB_SPEED = 32,
             ERRB_BOUNDS = 64 };

// ---------------------------------------------------------------------------
// Precision forms
// ---------------------------------------------------------------------------
enum { P64 = 0, P32 = 1, P16 = 2 };
// SH: the reduced forms store, and compute with, the deviation f_q - w_q of
// each population from its rest-state value (rho_0 = 1).  Every step of the
// method is affine in the populations with coefficients that sum to one per
// link pair (w_q = w_qbar), so it takes the same form in the deviations, with
// rho' = rho - 1 in place of rho in the equilibria; the stored values (of
// order |u| rather than w_q) then keep the full float or half mantissa for the
// part that carries the flow.  FP64 stores f_q itself.
template <int P> struct Form;
template <> struct Form<P64> { using S = double; using R = double; static constexpr bool SH = false; };
template <> struct Form<P32> { using S = float; using R = float; static constexpr bool SH = true; };
template <> struct Form<P16> { using S = __half; using R = float; static constexpr bool SH = true; };

// loads and stores in the arithmetic type: f_q (FP64) or f_q - w_q (FP32/FP16)
template <int P, int q>
__device__ __forceinline__ typename Form<P>::R ld(const typename Form<P>::S* __restrict__ p, size_t k) {
  if constexpr (P == P16) return __half2float(__ldg(p + k));
  else return __ldg(p + k);
}
template <int P>
__device__ __forceinline__ typename Form<P>::R ldq(const typename Form<P>::S* __restrict__ p, size_t k, int q) {
  if constexpr (P == P16) return __half2float(p[k]);
  else return p[k];
}
template <int P, int q>
__device__ __forceinline__ void st(typename Form<P>::S* __restrict__ p, size_t k, typename Form<P>::R v) {
  if constexpr (P == P16) p[k] = __float2half_rn(v);
  else p[k] = v;
}
template <int P>
__device__ __forceinline__ void stq(typename Form<P>::S* __restrict__ p, size_t k, int q, typename Form<P>::R v) {
  if constexpr (P == P16) p[k] = __float2half_rn(v);
  else p[k] = v;
}
// the population f_q itself, in FP64 (state read-back, the adjoint)
template <int P>
__device__ __forceinline__ double ldq_full(const typename Form<P>::S* __restrict__ p, size_t k, int q) {
  double v;
  if constexpr (P == P16) v = (double)__half2float(p[k]);
  else v = (double)p[k];
  if constexpr (Form<P>::SH) v += (q == 0 ? 1.0 / 3.0 : (q <= 6 ? 1.0 / 18.0 : 1.0 / 36.0));
  return v;
}
// the stored value of a population f_q given in FP64
template <int P>
__device__ __forceinline__ typename Form<P>::R to_arith(double f, int q) {
  if constexpr (Form<P>::SH) f -= (q == 0 ? 1.0 / 3.0 : (q <= 6 ? 1.0 / 18.0 : 1.0 / 36.0));
  return (typename Form<P>::R)f;
}
// density from a sum of populations in the arithmetic type (rho' or rho)
template <bool SH, class R>
__device__ __forceinline__ double rho_full(R r) {
  return SH ? 1.0 + (double)r : (double)r;
}
template <bool SH, class R>
__device__ __forceinline__ R rho_full_r(R r) {
  return SH ? R(1) + r : r;
}
// instability test of a density given as a sum in the arithmetic type
template <bool SH, class R>
__device__ __forceinline__ bool rho_bad(R r) {
  const R rf = rho_full_r<SH>(r);
  return !(rf > R(0)) || !(rf < R(1e30));
}

// ---------------------------------------------------------------------------
// Parameters passed by value to every kernel
// ---------------------------------------------------------------------------
// Division of a 32-bit unsigned n by a fixed divisor d >= 1 with one high
// multiply (Granlund and Montgomery, "Division by invariant integers using
// multiplication", 1994, Fig. 4.1): l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1, t = mulhi(m, n),
// n / d = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0), exact for all n < 2^32.
struct FDiv {
  unsigned m;
  int s1, s2;
};
__device__ __forceinline__ unsigned fdiv(unsigned n, const FDiv& d) {
  const unsigned t = __umulhi(n, d.m);
  return (t + ((n - t) >> d.s1)) >> d.s2;
}

struct Par {
  int nx, ny, nz;
  FDiv dnx, dny, dnxy, dnsx;  // fast division by nx, ny, nx*ny and the segments per row
  long long N;
  int px, py, pz, zshift;
  double lam_p, lam_m;     // TRT rates
  double inv_lam_m;        // 1/lambda_-
  double inv_1plp;         // 1/(1 + lambda_+), recovers n^+ from f~
  double g[3];
  double rho_G, sigma, eps, delta_min;
  int rule, compressible, linear_eq, freeze, cleanup;
  int stress;              // boundary shear-rate term of Eq. bterm: 0 off, 1 extrapolated S^b, 2 prescribed
  double tau_m_half;       // Lambda_+ = tau - 1/2
  double shear_b[6];       // prescribed S^b (xx yy zz xy xz yz)
  double wall_u[3];        // wall velocity
  int has_uw;              // a wall velocity is set
  int has_wd;
  int ub_extrap;           // FSL: u_b extrapolated along the link to the surface point
  int recon_nc;            // interface cells also rebuild the links with n.c_p > 0
  int excess_split;        // 1: excess split along the fill-level normal
  // cells this lattice owns when it is one subdomain of a decomposition (the
  // others are ghost layers, computed but left out of the mass balance and
  // the lost ledger); owned_all: every cell
  int own_lo[3], own_hi[3];
  int owned_all;
  int elvira;              // 1: ELVIRA normal where the height columns are open
  int adj32;               // 1: the adjoint's reverse step in FP32 (FP32/FP16 lattices)
  double umax2;            // stability guard: |u|^2 above it is an error (0: off)
#ifdef FSLBM_CHECKED
  int* err;                // the handle's error word (bounds-checked build)
#endif
};

// ---------------------------------------------------------------------------
// Bounds-checked build (compiled with FSLBM_CHECKED, a library of its own).
// Every cell index a kernel reads from memory (a segment record, a cell list)
// and every source cell a bulk kernel's fast path forms by offset arithmetic
// (whose range rests on the segment masks) is tested against the lattice
// before the access, and so is the precondition of the interface kernels'
// interior instances (the cell lies 3 or more cells inside every face).  A
// failed test sets ERRB_BOUNDS in the error word, reported at the next
// synchronising call, and the access goes to cell 0 instead (where the
// precondition failed, the cell is skipped); nothing traps.  Indices from
// nbr() (an in-range cell or -1), from bounded loop counters and from
// offsets next to a test of the cell's coordinates need no test.  In the
// normal build each macro is the bare expression.
// ---------------------------------------------------------------------------
#ifdef FSLBM_CHECKED
__device__ __forceinline__ long long chk_index(long long k, long long n, int* err) {
  if ((unsigned long long)k < (unsigned long long)n) return k;
  atomicOr(err, ERRB_BOUNDS);
  return 0;
}
// element k of an array of n from base
__device__ __forceinline__ long long chk_cell(long long k, long long base, long long n, int* err) {
  if ((unsigned long long)(k - base) < (unsigned long long)n) return k;
  atomicOr(err, ERRB_BOUNDS);
  return 0;
}
// element k of a word of two (k even, k + 1 in the same array of n from base)
__device__ __forceinline__ long long chk_word(long long k, long long base, long long n, int* err) {
  if ((k & 1) == 0 && (unsigned long long)(k - base) < (unsigned long long)(n - 1)) return k;
  atomicOr(err, ERRB_BOUNDS);
  return 0;
}
__device__ __forceinline__ bool chk_ok(bool ok, int* err) {
  if (!ok) atomicOr(err, ERRB_BOUNDS);
  return ok;
}
// k in [0, n), else 0
#define FSL_CK(p, k, n) fsl::chk_index((long long)(k), (long long)(n), (p).err)
// the same where c holds (k is not used otherwise)
#define FSL_CK_IF(p, c, k, n) ((c) ? fsl::chk_index((long long)(k), (long long)(n), (p).err) : (long long)(k))
// k - base in [0, n) (an element of population plane base / N), else 0
#define FSL_CK_CELL(p, k, base, n) fsl::chk_cell((long long)(k), (long long)(base), (long long)(n), (p).err)
// the first element of a two-element word (see chk_word), else 0
#define FSL_CK_WORD(p, k, base, n) fsl::chk_word((long long)(k), (long long)(base), (long long)(n), (p).err)
#define FSL_CK_WORD_IF(p, c, k, n) ((c) ? fsl::chk_word((long long)(k), 0LL, (long long)(n), (p).err) : (long long)(k))
// a precondition: c, a failure recorded (the caller then skips the cell)
#define FSL_OK(p, c) fsl::chk_ok((c), (p).err)
#else
#define FSL_CK(p, k, n) (k)
#define FSL_CK_IF(p, c, k, n) (k)
#define FSL_CK_CELL(p, k, base, n) (k)
#define FSL_CK_WORD(p, k, base, n) (k)
#define FSL_CK_WORD_IF(p, c, k, n) (k)
#define FSL_OK(p, c) true
#endif

// stability guard on a liquid cell's velocity: |u| above u_max (0.4 lattice
// units by default: the equilibria are second order in u, and the lattice's
// speed of sound is 1/sqrt(3) ~ 0.58); umax2 = u_max^2, 0 switches it off.
// Interface cells are left out: isolated ones in spray (a few fluid
// neighbours) reach such speeds in a stable flow.
template <class R>
__device__ __forceinline__ bool speed_bad(const Par& p, R ux, R uy, R uz) {
  return p.umax2 > 0.0 && ux * ux + uy * uy + uz * uz > R(p.umax2);
}
__device__ __forceinline__ bool owned(const Par& p, int x, int y, int z) {
  return p.owned_all || ((unsigned)(x - p.own_lo[0]) < (unsigned)(p.own_hi[0] - p.own_lo[0]) &&
                         (unsigned)(y - p.own_lo[1]) < (unsigned)(p.own_hi[1] - p.own_lo[1]) &&
                         (unsigned)(z - p.own_lo[2]) < (unsigned)(p.own_hi[2] - p.own_lo[2]));
}

template <int P>
struct View {
  using S = typename Form<P>::S;
  using R = typename Form<P>::R;
  uint8_t* flags;
  uint8_t* mark;
  const S* fin;
  S* fout;
  double* m;
  const R* phin;
  R* phout;
  const double* wd;  // wall link fractions (FP64 in every form)
  // lists and counters
  int* ilist;   // interface cells of this step: interior from the front, edge cells from the back
  int* flist;   // fill
  int* elist;   // empty
  int* nglist;  // new from gas
  int* nllist;  // new from liquid
  int* rlist;   // excess receivers
  int* cnt;     // [0] ilist front [6] ilist back [1] flist [2] elist [3] ng [4] nl [5] rl [7] emptied;
                // [8] all conversions since set; [9] fluid segments; [10] grid barrier of k_convert
  int cap;
  double* share;
  R* geo;            // interface geometry per list entry: [5][cap] n0, n1, n2, d, kappa (n = 0: none)
  double* partials;  // block partial sums of the mass balance
  double* lost;
  int* err;
};

// ---------------------------------------------------------------------------
// Neighbours: cell (x,y,z) + d with periodic wrap (x wrap shifts z), -1 past a
// non-periodic face (half-way wall there).
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long nbr(const Par& p, int x, int y, int z, int dx, int dy, int dz) {
  int X = x + dx, Y = y + dy, Z = z + dz;
  if ((unsigned)X >= (unsigned)p.nx) {
    if (!p.px) return -1;
    if (X < 0) { X += p.nx; Z += p.zshift; } else { X -= p.nx; Z -= p.zshift; }
  }
  if ((unsigned)Y >= (unsigned)p.ny) {
    if (!p.py) return -1;
    Y += (Y < 0) ? p.ny : -p.ny;
  }
  if ((unsigned)Z >= (unsigned)p.nz) {
    if (!p.pz) return -1;
    Z += (Z < 0) ? p.nz : -p.nz;
  }
  if ((unsigned)X >= (unsigned)p.nx || (unsigned)Y >= (unsigned)p.ny || (unsigned)Z >= (unsigned)p.nz) return -1;
  return (long long)X + (long long)p.nx * ((long long)Y + (long long)p.ny * Z);
}
// (x, y, z) of cell i (i < N < 2^31)
__device__ __forceinline__ void coords(const Par& p, long long i, int& x, int& y, int& z) {
  const unsigned u = (unsigned)i;
  const unsigned zz = fdiv(u, p.dnxy);
  const unsigned r = u - zz * (unsigned)(p.nx * p.ny);
  const unsigned yy = fdiv(r, p.dnx);
  z = (int)zz;
  y = (int)yy;
  x = (int)(r - yy * (unsigned)p.nx);
}
__device__ __forceinline__ uint8_t kind_at(const uint8_t* flags, long long j) {
  return j < 0 ? (uint8_t)WALL : (uint8_t)(flags[j] & KIND);
}
__device__ __forceinline__ bool is_fluid(uint8_t k) { return k == LIQ || k == IFC; }

// ---------------------------------------------------------------------------
// Equilibria (Eq. eqEven / eqOdd), c_s^2 = 1/3:
//   e_q^+ = w_q (rho + 3 N_q),  3 N_q = 3/2 rho_0 (3 (c.u)^2 - u.u)
//   e_q^- = 3 w_q rho_0 (c.u^eq)
// ---------------------------------------------------------------------------
template <class R, int q>
__device__ __forceinline__ R eplus(const Par& p, R rho, R r0, R ux, R uy, R uz, R usq) {
  // branch-free in linear_eq: the non-linear part is scaled by 0 or 1
  const R nl = p.linear_eq ? R(0) : R(1);
  const R cu = R(cx(q)) * ux + R(cy(q)) * uy + R(cz(q)) * uz;
  return wq<R>(q) * rho + (wq<R>(q) * R(1.5) * r0 * nl) * (R(3) * cu * cu - usq);
}
template <class R>
__device__ __forceinline__ R eplus_q(const Par& p, int q, R rho, R r0, R ux, R uy, R uz, R usq) {
  R w = q == 0 ? R(1) / R(3) : (q <= 6 ? R(1) / R(18) : R(1) / R(36));
  R e = w * rho;
  if (!p.linear_eq) {
    R cu = R(cx(q)) * ux + R(cy(q)) * uy + R(cz(q)) * uz;
    e += w * R(1.5) * r0 * (R(3) * cu * cu - usq);
  }
  return e;
}
template <class R, int q>
__device__ __forceinline__ R eminus(R r0, R vx, R vy, R vz) {
  R cu = R(cx(q)) * vx + R(cy(q)) * vy + R(cz(q)) * vz;
  return R(3) * wq<R>(q) * r0 * cu;
}

// Arithmetic with the rounding of every operation fixed (no compiler choice
// of fused multiply-adds), so that a collision gives the same bits in every
// kernel it is inlined into.
__device__ __forceinline__ float fx_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fx_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fx_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double fx_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fx_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double fx_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float fx_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double fx_sub(double a, double b) { return __dsub_rn(a, b); }

// c.u for a lattice direction (components 0 or +-1: exact adds)
template <class R, int q>
__device__ __forceinline__ R cdot(R ux, R uy, R uz) {
  R s = R(0);
  if (cx(q) == 1) s = fx_add(s, ux);
  if (cx(q) == -1) s = fx_sub(s, ux);
  if (cy(q) == 1) s = fx_add(s, uy);
  if (cy(q) == -1) s = fx_sub(s, uy);
  if (cz(q) == 1) s = fx_add(s, uz);
  if (cz(q) == -1) s = fx_sub(s, uz);
  return s;
}

// TRT collision of one cell (Eq. lbe2) in place: f <- f + l+ n^+ + l- n^-,
// with u = U + g/2 in e^+ and u^eq = U - g/lambda_- in e^- (Sec. 2.1).
// On return rho holds sum f and (ux,uy,uz) the velocity u of the
// pre-collision state.  SH: f holds f_q - w_q and rho receives rho - 1 (the
// equilibria below are affine in rho with the weights w_q as slopes, so the
// same expressions give e_q - w_q from rho - 1).
template <class R, bool SH = false>
__device__ __forceinline__ void collide(const Par& p, R (&f)[19], R& rho, R& ux, R& uy, R& uz) {
  R r = f[0], jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
  for (int q = 1; q < 19; ++q) r = fx_add(r, f[q]);
#pragma unroll
  for (int q = 1; q < 19; ++q) {
    if (cx(q) == 1) jx = fx_add(jx, f[q]);
    if (cx(q) == -1) jx = fx_sub(jx, f[q]);
    if (cy(q) == 1) jy = fx_add(jy, f[q]);
    if (cy(q) == -1) jy = fx_sub(jy, f[q]);
    if (cz(q) == 1) jz = fx_add(jz, f[q]);
    if (cz(q) == -1) jz = fx_sub(jz, f[q]);
  }
  const R r0 = p.compressible ? rho_full_r<SH>(r) : R(1);
  const R ir0 = p.compressible ? R(1) / r0 : R(1);
  const R Ux = fx_mul(jx, ir0), Uy = fx_mul(jy, ir0), Uz = fx_mul(jz, ir0);
  const R gx = R(p.g[0]), gy = R(p.g[1]), gz = R(p.g[2]);
  ux = fx_fma(R(0.5), gx, Ux);
  uy = fx_fma(R(0.5), gy, Uy);
  uz = fx_fma(R(0.5), gz, Uz);
  const R ilm = R(p.inv_lam_m);
  const R vx = fx_fma(-gx, ilm, Ux), vy = fx_fma(-gy, ilm, Uy), vz = fx_fma(-gz, ilm, Uz);
  const R usq = fx_fma(uz, uz, fx_fma(uy, uy, fx_mul(ux, ux)));
  const R lp = R(p.lam_p), lm = R(p.lam_m);
  // e^+_q = w rho + K_w (3 (c.u)^2 - u.u), K_w = 3/2 w rho_0 (0 for linear e^+);
  // e^-_q = 3 w rho_0 (c.u^eq)
  const R nl = p.linear_eq ? R(0) : R(1);
  const R k0 = fx_mul(fx_mul(R(1.5) * wq<R>(0), r0), nl);
  const R k1 = fx_mul(fx_mul(R(1.5) * wq<R>(1), r0), nl);
  const R k7 = fx_mul(fx_mul(R(1.5) * wq<R>(7), r0), nl);
  // 3 w_q rho_0 of e^-.  In float the rounded weights would make
  // sum_q 3 w_q c_qa c_qa = 2 (3 w_1) + 8 (3 w_7) differ from 1 by ~1e-7, and
  // the momentum would relax toward (1 + 1e-7) U every step: a systematic
  // drift of the velocity that grows with time.  3 w_7 = fl(1/12) and
  // 3 w_1 = (1 - 8 fl(1/12))/2 (both exact in float) keep that sum at 1.
  R m1, m7;
  if constexpr (sizeof(R) == 4) {
    constexpr R m7f = R(1) / R(12);
    constexpr R m1f = (R(1) - R(8) * m7f) * R(0.5);
    m1 = fx_mul(m1f, r0);
    m7 = fx_mul(m7f, r0);
  } else {
    m1 = fx_mul(R(3) * wq<R>(1), r0);
    m7 = fx_mul(R(3) * wq<R>(7), r0);
  }
  R out[19];
  {
    const R ep = fx_fma(k0, -usq, fx_mul(wq<R>(0), r));
    out[0] = fx_fma(lp, fx_sub(f[0], ep), f[0]);
  }
#define FSL_PAIR(q)                                                                  \
  {                                                                                  \
    constexpr int qb = inv(q);                                                       \
    const R kq = q <= 6 ? k1 : k7, mq = q <= 6 ? m1 : m7;                            \
    const R cu = cdot<R, q>(ux, uy, uz), cv = cdot<R, q>(vx, vy, vz);                \
    const R ep = fx_fma(kq, fx_fma(R(3) * cu, cu, -usq), fx_mul(wq<R>(q), r));       \
    const R em = fx_mul(mq, cv);                                                     \
    const R np = fx_fma(R(0.5), fx_add(f[q], f[qb]), -ep);                           \
    const R nm = fx_fma(R(0.5), fx_sub(f[q], f[qb]), -em);                           \
    out[q] = fx_fma(lm, nm, fx_fma(lp, np, f[q]));                                   \
    out[qb] = fx_fma(-lm, nm, fx_fma(lp, np, f[qb]));                                \
  }
  FSL_PAIR(1) FSL_PAIR(3) FSL_PAIR(5) FSL_PAIR(7) FSL_PAIR(9)
  FSL_PAIR(11) FSL_PAIR(13) FSL_PAIR(15) FSL_PAIR(17)
#undef FSL_PAIR
#pragma unroll
  for (int q = 0; q < 19; ++q) f[q] = out[q];
  rho = r;
}

// Moments of the pre-collision state recovered from post-collision f~:
// sum f~ = rho and sum c f~ = rho_0 U + F, so u = U + g/2 = (sum c f~)/rho_0 - g/2.
// SH: f holds f~_q - w_q and rho receives rho - 1.
template <class R, bool SH = false>
__device__ __forceinline__ void moments_post(const Par& p, const R (&f)[19], R& rho, R& ux, R& uy, R& uz) {
  R r = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
  for (int q = 0; q < 19; ++q) {
    r += f[q];
    if (cx(q)) jx += R(cx(q)) * f[q];
    if (cy(q)) jy += R(cy(q)) * f[q];
    if (cz(q)) jz += R(cz(q)) * f[q];
  }
  R ir0 = p.compressible ? R(1) / rho_full_r<SH>(r) : R(1);
  ux = jx * ir0 - R(0.5) * R(p.g[0]);
  uy = jy * ir0 - R(0.5) * R(p.g[1]);
  uz = jz * ir0 - R(0.5) * R(p.g[2]);
  rho = r;
}

// ---------------------------------------------------------------------------
// Plane / unit-cube volume (piecewise cubic in the plane constant alpha for a
// normal with sorted components m1 <= m2 <= m3, m1+m2+m3 = 1) and its slope.
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ R cube_vol_half(R a, R m1, R m2, R m3) {
  // valid for 0 <= a <= 1/2
  if (a <= R(0)) return R(0);
  if (a <= m1) return a * a * a / (R(6) * m1 * m2 * m3);
  R base = R(3) * a * a - R(3) * a * m1 + m1 * m1;
  R den = R(6) * m2 * m3;
  if (a <= m2) return base / den;
  R s = a - m2;
  R m12 = m1 + m2;
  if (m3 >= m12) {
    if (a <= m12) return (base - s * s * s / m1) / den;
    return (a - R(0.5) * m12) / m3;
  }
  if (a <= m3) return (base - s * s * s / m1) / den;
  R r = a - m3;
  return (base - s * s * s / m1 - r * r * r / m1) / den;
}
template <class R>
__device__ __forceinline__ R cube_vol(R a, R m1, R m2, R m3) {
  if (a >= R(1)) return R(1);
  if (a > R(0.5)) return R(1) - cube_vol_half(R(1) - a, m1, m2, m3);
  return cube_vol_half(a, m1, m2, m3);
}
template <class R>
__device__ __forceinline__ R cube_area_half(R a, R m1, R m2, R m3) {
  if (a <= R(0)) return R(0);
  if (a <= m1) return a * a / (R(2) * m1 * m2 * m3);
  R base = R(6) * a - R(3) * m1;
  R den = R(6) * m2 * m3;
  if (a <= m2) return base / den;
  R s = a - m2;
  R m12 = m1 + m2;
  if (m3 >= m12) {
    if (a <= m12) return (base - R(3) * s * s / m1) / den;
    return R(1) / m3;
  }
  if (a <= m3) return (base - R(3) * s * s / m1) / den;
  R r = a - m3;
  return (base - R(3) * s * s / m1 - R(3) * r * r / m1) / den;
}
template <class R>
__device__ __forceinline__ R cube_area(R a, R m1, R m2, R m3) {
  if (a >= R(1)) return R(0);
  if (a > R(0.5)) return cube_area_half(R(1) - a, m1, m2, m3);
  return cube_area_half(a, m1, m2, m3);
}

// Inverse of cube_vol_half by region, for the float forms: with the sorted
// normal (m1 <= m2 <= m3, sum 1) the volume is alpha^3 / (6 m1 m2 m3) on
// [0, m1] (a cube root), a quadratic on [m1, m2] (a square root), linear on
// [m1 + m2, m3] when m3 >= m1 + m2, and
// cubic on the remaining ranges, where Newton iterations from a secant
// start, kept inside the range, reach the float resolution.  tv in (0, 1/2].
// a / b: IEEE for double; for float on the device the fast approximate
// division (2 ulp, the operands here are O(1)), which the float forms accept
template <class R>
__host__ __device__ __forceinline__ R qdiv(R a, R b) {
#ifdef __CUDA_ARCH__
  if constexpr (sizeof(R) == 4) return __fdividef(a, b);
#endif
  return a / b;
}

template <class R>
__host__ __device__ __forceinline__ R cube_vol_r3(R a, R m1, R m2, R m3) {
  const R s = a - m2;
  return (R(3) * a * a - R(3) * a * m1 + m1 * m1 - s * s * s / m1) / (R(6) * m2 * m3);
}
template <class R>
__host__ __device__ __forceinline__ R plic_alpha_regions(R tv, R m1, R m2, R m3) {
  const R m12 = m1 + m2;
  const R den = R(6) * m2 * m3;
  if (m1 > R(0) && tv <= m1 * m1 / den) return cbrt(R(6) * m1 * m2 * m3 * tv);
  if (m2 > R(0) && tv <= (R(3) * m2 * m2 - R(3) * m2 * m1 + m1 * m1) / den) {
    const R t = R(2) * m2 * m3 * tv - m1 * m1 / R(12);
    return R(0.5) * m1 + sqrt(t > R(0) ? t : R(0));
  }
  R lo = m2, hi, vlo, vhi;
  bool four = false;  // the range [m3, 1/2] of a cube with m3 < m1 + m2
  if (m3 >= m12) {
    if (tv >= R(0.5) * m12 / m3) return m3 * tv + R(0.5) * m12;
    hi = m12;
    vhi = R(0.5) * m12 / m3;
  } else {
    const R v3 = cube_vol_r3(m3, m1, m2, m3);
    if (tv <= v3) {
      hi = m3;
      vhi = v3;
    } else {
      four = true;
      lo = m3;
      hi = R(0.5);
      vhi = R(0.5);
    }
  }
  vlo = four ? cube_vol_r3(m3, m1, m2, m3) : (R(3) * m2 * m2 - R(3) * m2 * m1 + m1 * m1) / den;
  R al = vhi > vlo ? lo + (hi - lo) * qdiv(tv - vlo, vhi - vlo) : hi;
  // (the cubic ranges have m1 > 0)
  const R im1 = qdiv(R(1), m1), iden = qdiv(R(1), den);
  for (int it = 0; it < 5; ++it) {
    const R sa = al - m2, ra = four ? al - m3 : R(0);
    const R v = (R(3) * al * al - R(3) * al * m1 + m1 * m1 - (sa * sa * sa + ra * ra * ra) * im1) * iden;
    const R dv = (R(6) * al - R(3) * m1 - R(3) * (sa * sa + ra * ra) * im1) * iden;
    if (!(dv > R(0))) break;
    R nx = al - qdiv(v - tv, dv);
    al = nx < lo ? lo : (nx > hi ? hi : nx);
  }
  return al;
}

// Signed offset d (from the cell centre along the unit normal n, liquid on
// the side n.(x - x_c) <= d) of the plane cutting volume fraction ph.  The
// fill is kept in [1e-9, 1 - 1e-9] first: at an empty or full corner the
// inverse volume grows like a cube root and would turn rounding of ph into
// visible plane shifts.  Bracketing bisection, then Newton on the convex half.
template <class R>
__device__ R plic_offset(R nx_, R ny_, R nz_, R ph) {
  R a0 = fabs(nx_), a1 = fabs(ny_), a2 = fabs(nz_);
  R L1 = a0 + a1 + a2;
  a0 /= L1; a1 /= L1; a2 /= L1;
  // sort ascending
  R t;
  if (a0 > a1) { t = a0; a0 = a1; a1 = t; }
  if (a1 > a2) { t = a1; a1 = a2; a2 = t; }
  if (a0 > a1) { t = a0; a0 = a1; a1 = t; }
  const R lo_ph = R(1e-9), hi_ph = R(1) - R(1e-9);
  ph = ph < lo_ph ? lo_ph : (ph > hi_ph ? hi_ph : ph);
  // the volume is point-symmetric about alpha = 1/2: solve on [0, 1/2] for
  // min(ph, 1 - ph), where it is convex
  const bool upper = ph > R(0.5);
  const R tv = upper ? R(1) - ph : ph;
  if constexpr (sizeof(R) == 4) {
    R al = plic_alpha_regions(tv, a0, a1, a2);
    if (upper) al = R(1) - al;
    return L1 * (al - R(0.5));
  }
  R lo = R(0), hi = R(0.5);
#pragma unroll 1
  for (int it = 0; it < 20; ++it) {  // bracket to 2^-21
    R mid = R(0.5) * (lo + hi);
    if (cube_vol_half(mid, a0, a1, a2) < tv) lo = mid; else hi = mid;
  }
  // Newton from the right end of the bracket (convex, increasing: monotone),
  // kept inside the bracket
  R al = hi;
  constexpr int newton = sizeof(R) == 8 ? 6 : 3;
#pragma unroll 1
  for (int it = 0; it < newton; ++it) {
    R ar = cube_area_half(al, a0, a1, a2);
    if (!(ar > R(0))) break;
    R nx2 = al - (cube_vol_half(al, a0, a1, a2) - tv) / ar;
    al = nx2 < lo ? lo : (nx2 > hi ? hi : nx2);
  }
  if (upper) al = R(1) - al;
  return L1 * (al - R(0.5));
}

// fill level as seen by the geometry: 1 liquid, stored for interface cells
// (and for gas cells of a frozen interface), else 0
template <class R>
__device__ __forceinline__ R phi_at(const Par& p, const R* __restrict__ phin, long long j, uint8_t kj) {
  if (kj == LIQ) return R(1);
  if (kj == IFC) return phin[j];
  if (kj == GAS && p.freeze) return phin[j];
  return R(0);
}

// ---------------------------------------------------------------------------
// Geometry of an interface cell from phi(t) (Sec. 2.2, Sec. 5): Parker-Youngs
// gradient, then height functions over 3x3 columns of 7 cells along the
// dominant axis; if every column is closed (liquid at its liquid end, gas at
// its gas end, no wall) the normal, the plane offset
// d = |n_a| (H(0,0) - 3.5) and the curvature come from the heights, else the
// normalised Parker-Youngs normal and the plane cutting the cell's own fill.
// ---------------------------------------------------------------------------
template <class R>
struct Geo {
  R n[3];        // unit normal, liquid -> gas
  R d;           // signed plane offset from the node along n
  R kap;         // curvature (sigma != 0 only)
  bool ok;       // a normal exists
  bool closed;   // height columns closed: n, d, kap from the heights
  int a, b, s;   // dominant axis, first other axis (the third is 3 - a - b), gas side of a
  R H[9];        // column heights H[(ib+1)*3 + (ic+1)]
};

// Curvature where the height columns along the dominant axis are not closed
// (surface tension only; rare, so out of line and on the general neighbour
// rule): heights along the two other axes by decreasing |n_a|, else the
// divergence of the unit Parker-Youngs normal by central differences over the
// six face neighbours (a neighbour without a normal, or a wall, takes the
// cell's own).  n: the cell's Parker-Youngs normal -grad phi, not normalised.
template <class R>
__device__ __forceinline__ R fill_at(const Par& p, const uint8_t* __restrict__ flags, const R* __restrict__ phin,
                                     long long j, uint8_t& kj) {
  kj = kind_at(flags, j);
  if (kj == LIQ) return R(1);
  if (kj == IFC || (kj == GAS && p.freeze)) return phin[j];
  return R(0);
}
template <class R>
__device__ __forceinline__ bool height_curvature(const Par& p, const uint8_t* __restrict__ flags,
                                                 const R* __restrict__ phin, int x, int y, int z, int a, int s,
                                                 R& kap) {
  const int b = (a == 0) ? 1 : 0;
  const int c = (a == 2) ? 1 : 2;
  R H[9];
  for (int ib = -1; ib <= 1; ++ib)
    for (int ic = -1; ic <= 1; ++ic) {
      R sum = R(0);
      for (int k = -3; k <= 3; ++k) {
        int o[3] = {0, 0, 0};
        o[a] = k; o[b] = ib; o[c] = ic;
        uint8_t kj;
        const R v = fill_at<R>(p, flags, phin, nbr(p, x, y, z, o[0], o[1], o[2]), kj);
        if (kj == WALL) return false;
        if (k == -3 * s && kj != LIQ) return false;
        if (k == 3 * s && kj != GAS) return false;
        sum += v;
      }
      H[(ib + 1) * 3 + (ic + 1)] = sum;
    }
  const R Hb = R(0.5) * (H[7] - H[1]);
  const R Hc = R(0.5) * (H[5] - H[3]);
  const R Hbb = H[7] - R(2) * H[4] + H[1];
  const R Hcc = H[5] - R(2) * H[4] + H[3];
  const R Hbc = R(0.25) * (H[8] - H[6] - H[2] + H[0]);
  const R q2 = R(1) + Hb * Hb + Hc * Hc;
  const R num = Hbb * (R(1) + Hc * Hc) + Hcc * (R(1) + Hb * Hb) - R(2) * Hb * Hc * Hbc;
  kap = -num / (q2 * sqrt(q2));
  return true;
}
template <class R>
__device__ __noinline__ R curvature_open(const Par& p, const uint8_t* __restrict__ flags,
                                         const R* __restrict__ phin, int x, int y, int z, R n0, R n1, R n2,
                                         int a) {
  const R nv[3] = {n0, n1, n2};
  int ax0 = (a + 1) % 3, ax1 = (a + 2) % 3;
  if (fabs(nv[ax1]) > fabs(nv[ax0])) {
    const int t = ax0;
    ax0 = ax1;
    ax1 = t;
  }
  R kap = R(0);
  if (height_curvature<R>(p, flags, phin, x, y, z, ax0, nv[ax0] > R(0) ? 1 : -1, kap)) return kap;
  if (height_curvature<R>(p, flags, phin, x, y, z, ax1, nv[ax1] > R(0) ? 1 : -1, kap)) return kap;
  const R l0 = sqrt(n0 * n0 + n1 * n1 + n2 * n2);
  R div = R(0);
  for (int d = 0; d < 3; ++d) {
    R comp[2];
    for (int sg = 0; sg < 2; ++sg) {
      int o[3] = {0, 0, 0};
      o[d] = sg ? 1 : -1;
      const int xj = x + o[0], yj = y + o[1], zj = z + o[2];
      const long long j = nbr(p, x, y, z, o[0], o[1], o[2]);
      R m0 = n0, m1 = n1, m2 = n2, lm = l0;
      if (j >= 0 && kind_at(flags, j) != WALL) {
        // Parker-Youngs gradient around the neighbour (its own fill across walls)
        uint8_t kc;
        const R pc = fill_at<R>(p, flags, phin, j, kc);
        R g0 = R(0), g1 = R(0), g2 = R(0);
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              if (!dx && !dy && !dz) continue;
              uint8_t kk;
              R pj = fill_at<R>(p, flags, phin, nbr(p, xj, yj, zj, dx, dy, dz), kk);
              if (kk == WALL) pj = pc;
              const int adx = dx < 0 ? -dx : dx, ady = dy < 0 ? -dy : dy, adz = dz < 0 ? -dz : dz;
              if (dx) g0 += R(dx * (2 - ady) * (2 - adz)) * pj;
              if (dy) g1 += R(dy * (2 - adz) * (2 - adx)) * pj;
              if (dz) g2 += R(dz * (2 - adx) * (2 - ady)) * pj;
            }
        const R l = sqrt(g0 * g0 + g1 * g1 + g2 * g2);
        if (l > R(1e-12)) {
          m0 = -g0; m1 = -g1; m2 = -g2; lm = l;
        }
      }
      comp[sg] = (d == 0 ? m0 : (d == 1 ? m1 : m2)) / lm;
    }
    div += R(0.5) * (comp[1] - comp[0]);
  }
  return div;
}

// Volume fraction of the cell around a node on the side n.x <= d of a plane
// (n unit, x from the node): the plane/cube volume in the L1-normalised,
// sorted normal.
template <class R>
__device__ __forceinline__ R plane_volume(R n0, R n1, R n2, R d) {
  R a0 = fabs(n0), a1 = fabs(n1), a2 = fabs(n2);
  const R L1 = a0 + a1 + a2;
  a0 /= L1; a1 /= L1; a2 /= L1;
  R t;
  if (a0 > a1) { t = a0; a0 = a1; a1 = t; }
  if (a1 > a2) { t = a1; a1 = a2; a2 = t; }
  if (a0 > a1) { t = a0; a0 = a1; a1 = t; }
  return cube_vol(d / L1 + R(0.5), a0, a1, a2);
}

// ELVIRA (Pilliod and Puckett, "Second-order accurate volume-of-fluid
// algorithms for tracking material interfaces", J. Comput. Phys. 2004) in
// three dimensions, for a cell whose height columns are open: along each
// axis a the fill levels of the 3x3x3 block summed over 3 cells give column
// heights h(b, c); backward, central and forward differences of h in the two
// other axes give nine candidate normals (s_a, -dh/db, -dh/dc), s_a the gas
// side of a (sign of the Parker-Youngs component npy_a).  Each candidate's
// plane through the cell's own fill is continued through the block; the
// candidate whose volume fractions match the block's fill levels best (least
// squares over the cells that are not walls, summed z-major; first minimum in
// the order a, b-difference, c-difference) gives n and d.  A wall takes the
// cell's own fill level in the column sums.  Out of line: rare, and kept out
// of the registers of the common path.
template <class R>
__device__ __noinline__ void elvira_plane(const Par& p, const uint8_t* __restrict__ flags,
                                          const R* __restrict__ phin, int x, int y, int z, R phic, R npy0, R npy1,
                                          R npy2, R* nout, R* dout) {
  R blk[27];
  unsigned wallm = 0u;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int k = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
        uint8_t kj;
        const R v = fill_at<R>(p, flags, phin, nbr(p, x, y, z, dx, dy, dz), kj);
        if (kj == WALL) wallm |= 1u << k;
        blk[k] = kj == WALL ? phic : v;
      }
  const R npy[3] = {npy0, npy1, npy2};
  R best = R(1e30);
  for (int a = 0; a < 3; ++a) {
    const int s = npy[a] > R(0) ? 1 : -1;
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    R h[9];
    for (int ib = -1; ib <= 1; ++ib)
      for (int ic = -1; ic <= 1; ++ic) {
        R sum = R(0);
        for (int k = -1; k <= 1; ++k) {
          int o[3];
          o[a] = k; o[b] = ib; o[c] = ic;
          sum += blk[(o[2] + 1) * 9 + (o[1] + 1) * 3 + (o[0] + 1)];
        }
        h[(ib + 1) * 3 + (ic + 1)] = sum;
      }
    const R db[3] = {h[4] - h[1], R(0.5) * (h[7] - h[1]), h[7] - h[4]};
    const R dc[3] = {h[4] - h[3], R(0.5) * (h[5] - h[3]), h[5] - h[4]};
    for (int kb = 0; kb < 3; ++kb)
      for (int kc = 0; kc < 3; ++kc) {
        R v[3];
        v[a] = R(s); v[b] = -db[kb]; v[c] = -dc[kc];
        const R len = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        const R m0 = v[0] / len, m1 = v[1] / len, m2 = v[2] / len;
        const R dd = plic_offset<R>(m0, m1, m2, phic);
        R err = R(0);
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              const int k = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
              if (k == 13 || (wallm & (1u << k))) continue;
              const R e = plane_volume<R>(m0, m1, m2, dd - (m0 * R(dx) + m1 * R(dy) + m2 * R(dz))) - blk[k];
              err += e * e;
            }
        if (err < best) {
          best = err;
          nout[0] = m0; nout[1] = m1; nout[2] = m2;
          *dout = dd;
        }
      }
  }
}

// MODE 0: any cell (plain offsets when every stencil cell is inside the
// lattice, else the general neighbour rule); 1: the caller knows every cell
// within 3 is inside; 2: a lattice without periodic axes (a stencil cell past
// a face is a wall: a bounds test per cell instead of the neighbour rule).
// SIG: the instance for surface tension (curvature); without it kappa stays 0.
// ELV: the instance with the ELVIRA normal where the columns are open.
template <class R, int MODE = 0, bool SIG = false, bool ELV = false>
__device__ __forceinline__ void geometry(const Par& p, const uint8_t* __restrict__ flags,
                                         const R* __restrict__ phin, int x, int y, int z, R phic, Geo<R>& G) {
  R (&n)[3] = G.n;
  R& d = G.d;
  R& kap = G.kap;
  bool& ok = G.ok;
  R (&H)[9] = G.H;
  G.closed = false;
  G.a = 2; G.b = 0; G.s = 1;
  // cells within 3 of the node are inside the lattice without a wrap: plain
  // offsets; otherwise the general neighbour rule
  const bool interior = MODE == 1 || (x >= 3 && x < p.nx - 3 && y >= 3 && y < p.ny - 3 && z >= 3 && z < p.nz - 3);
  const long long i0 = (long long)x + (long long)p.nx * ((long long)y + (long long)p.ny * z);
  // fill level seen by the geometry; the phi load is issued whatever the kind
  // so that all loads of the stencil are independent
  // interior cells index in 32 bits (N < 2^31)
  const int i0i = (int)i0, syi = p.nx, szi = p.nx * p.ny;
  auto sample = [&](int dx, int dy, int dz, uint8_t& kj) -> R {
    R raw;
    if (interior) {
      const unsigned j = (unsigned)(i0i + dx + syi * dy + szi * dz);
      raw = phin[j];
      kj = (uint8_t)(flags[j] & KIND);
    } else if (MODE == 2) {
      const bool inside = (unsigned)(x + dx) < (unsigned)p.nx && (unsigned)(y + dy) < (unsigned)p.ny &&
                          (unsigned)(z + dz) < (unsigned)p.nz;
      const unsigned j = inside ? (unsigned)(i0i + dx + syi * dy + szi * dz) : 0u;
      raw = inside ? phin[j] : R(0);
      kj = inside ? (uint8_t)(flags[j] & KIND) : (uint8_t)WALL;
    } else {
      const long long j = nbr(p, x, y, z, dx, dy, dz);
      raw = j >= 0 ? phin[j] : R(0);
      kj = kind_at(flags, j);
    }
    if (kj == LIQ) return R(1);
    if (kj == IFC || (kj == GAS && p.freeze)) return raw;
    return R(0);
  };
  R g0 = R(0), g1 = R(0), g2 = R(0);
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        if (!dx && !dy && !dz) continue;
        uint8_t kj;
        R pj = sample(dx, dy, dz, kj);
        if (kj == WALL) pj = phic;
        const int ax = dx < 0 ? -dx : dx, ay = dy < 0 ? -dy : dy, az = dz < 0 ? -dz : dz;
        if (dx) g0 += R(dx * (2 - ay) * (2 - az)) * pj;
        if (dy) g1 += R(dy * (2 - az) * (2 - ax)) * pj;
        if (dz) g2 += R(dz * (2 - ax) * (2 - ay)) * pj;
      }
  n[0] = -g0; n[1] = -g1; n[2] = -g2;
  kap = R(0);
  R nn = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
  if (!(nn > R(1e-24))) {
    ok = false;
    d = R(0);
    n[0] = R(0); n[1] = R(0); n[2] = R(1);
    return;
  }
  ok = true;
  int a = 0;
  R na = fabs(n[0]);
  if (fabs(n[1]) > na) { a = 1; na = fabs(n[1]); }
  if (fabs(n[2]) > na) { a = 2; }
  const int s = (a == 0 ? n[0] : (a == 1 ? n[1] : n[2])) > R(0) ? 1 : -1;
  const int b = (a == 0) ? 1 : 0;  // the third axis is the remaining one
  G.a = a; G.b = b; G.s = s;
  // heights over 3x3 columns of 7 cells along a; closed when every column
  // has liquid at its liquid end, gas at its gas end and no wall
  bool closed = true;
  // strides of the dominant axis a, of b and of the third axis (interior cells)
  const int c3 = 3 - a - b;
  const int sa = a == 0 ? 1 : (a == 1 ? syi : szi);
  const int sb = b == 0 ? 1 : (b == 1 ? syi : szi);
  const int sc = c3 == 0 ? 1 : (c3 == 1 ? syi : szi);
#pragma unroll
  for (int ib = -1; ib <= 1; ++ib)
#pragma unroll
    for (int ic = -1; ic <= 1; ++ic) {
      R sum = R(0);
      const int col = i0i + ib * sb + ic * sc;
#pragma unroll
      for (int k = -3; k <= 3; ++k) {
        uint8_t kj;
        R pj;
        if (interior) {
          const unsigned j = (unsigned)(col + k * sa);
          const R raw = phin[j];
          kj = kind_at(flags, j);
          pj = kj == LIQ ? R(1) : ((kj == IFC || (kj == GAS && p.freeze)) ? raw : R(0));
        } else {
          const int o0 = (a == 0) ? k : ((b == 0) ? ib : ic);
          const int o1 = (a == 1) ? k : ((b == 1) ? ib : ic);
          const int o2 = (a == 2) ? k : ((b == 2) ? ib : ic);
          pj = sample(o0, o1, o2, kj);
        }
        closed = closed && kj != WALL;
        if (k == -3) closed = closed && (s > 0 ? kj == LIQ : kj == GAS);
        if (k == 3) closed = closed && (s > 0 ? kj == GAS : kj == LIQ);
        sum += pj;
      }
      H[(ib + 1) * 3 + (ic + 1)] = sum;
    }
  G.closed = closed;
  if (closed) {
    R Hb = R(0.5) * (H[7] - H[1]);
    R Hc = R(0.5) * (H[5] - H[3]);
    R v0 = (a == 0) ? R(s) : ((b == 0) ? -Hb : -Hc);
    R v1 = (a == 1) ? R(s) : ((b == 1) ? -Hb : -Hc);
    R v2 = (a == 2) ? R(s) : ((b == 2) ? -Hb : -Hc);
    if constexpr (sizeof(R) == 4) {
      const R il = rsqrtf(v0 * v0 + v1 * v1 + v2 * v2);
      n[0] = v0 * il; n[1] = v1 * il; n[2] = v2 * il;
    } else {
      R len = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
      n[0] = v0 / len; n[1] = v1 / len; n[2] = v2 / len;
    }
    R nabs = fabs(a == 0 ? n[0] : (a == 1 ? n[1] : n[2]));
    d = nabs * (H[4] - R(3.5));
    if (SIG && p.sigma != 0.0) {
      R Hbb = H[7] - R(2) * H[4] + H[1];
      R Hcc = H[5] - R(2) * H[4] + H[3];
      R Hbc = R(0.25) * (H[8] - H[6] - H[2] + H[0]);
      R q2 = R(1) + Hb * Hb + Hc * Hc;
      R num = Hbb * (R(1) + Hc * Hc) + Hcc * (R(1) + Hb * Hb) - R(2) * Hb * Hc * Hbc;
      kap = -num / (q2 * sqrt(q2));
    }
  } else {
    if (SIG && p.sigma != 0.0) kap = curvature_open<R>(p, flags, phin, x, y, z, n[0], n[1], n[2], a);
    if constexpr (ELV) {
      R ne[3];
      elvira_plane<R>(p, flags, phin, x, y, z, phic, n[0], n[1], n[2], ne, &d);
      n[0] = ne[0]; n[1] = ne[1]; n[2] = ne[2];
      return;
    }
    if constexpr (sizeof(R) == 4) {
      const R il = rsqrtf(nn);
      n[0] *= il; n[1] *= il; n[2] *= il;
    } else {
      R len = sqrt(nn);
      n[0] /= len; n[1] /= len; n[2] /= len;
    }
    d = plic_offset<R>(n[0], n[1], n[2], phic);
  }
}

// Fixed-order sum of chunk b of in[0, n) by the calling block of 256 threads:
// strided per-thread sums, warp shuffles, the eight warp sums in a fixed
// tree.  Every thread of the block must call it; the result is on thread 0.
__device__ __forceinline__ double block_chunk_sum(const double* __restrict__ in, long long n, long long chunk,
                                                  long long b) {
  __shared__ double red[8];
  const long long lo = b * chunk;
  const long long hi = lo + chunk < n ? lo + chunk : n;
  double s = 0.0;
  for (long long k = lo + threadIdx.x; k < hi; k += blockDim.x) s += in[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  const double t = ((red[0] + red[1]) + (red[2] + red[3])) + ((red[4] + red[5]) + (red[6] + red[7]));
  __syncthreads();  // red is reused by the next call
  return t;
}

// The step's mass reduction when the conversion kernel carries it: nb chunks
// of `chunk` partials summed into tmp, then tmp summed into *out (+ *add, the
// lost ledger).  nb = 0: the reduction runs on its own.
struct MassReduce {
  const double* in;
  long long n, chunk;
  int nb;
  double* tmp;
  const double* add;
  double* out;
};

}  // namespace fsl

/*
 * fslbm.h -- C interface of the GB300 free-surface lattice Boltzmann step.
 *
 * One time step of the free-surface lattice Boltzmann method (FSLBM) on a
 * D3Q19 lattice, after Bogner, Ammer, Ruede, "Boundary Conditions for Free
 * Interfaces with the Lattice Boltzmann Method" (arXiv:1409.5645):
 *   - TRT stream-collide with a body force on liquid and interface cells
 *     (Sec. 2.1, Eq. lbe1 / lbe2, forcing through u^eq = U - F/lambda_-),
 *   - half-way bounce-back or CLI walls (Sec. 4.2, 4.3),
 *   - reconstruction of the populations streaming in from gas cells by the
 *     FSK rule (Eq. koerner) or the FSL rule (Eq. closure with Table 1, D = 0),
 *     with the link fraction delta taken from the fill levels and the interface
 *     normal (Sec. 2.2, Sec. 5),
 *   - interface mass exchange and fill update, and cell conversion with
 *     excess-mass redistribution (Sec. 2.3 / 4.4; the paper takes these from
 *     Koerner et al. and Thuerey).
 *
 * Conventions shared by every entry point
 *   cells       N = nx*ny*nz, cell index i = x + nx*(y + ny*z) (x fastest).
 *   links       q = 0..18 in this order: rest; (+-1,0,0), (0,+-1,0), (0,0,+-1);
 *               (1,1,0),(-1,-1,0),(1,-1,0),(-1,1,0); (1,0,1),(-1,0,-1),(1,0,-1),
 *               (-1,0,1); (0,1,1),(0,-1,-1),(0,1,-1),(0,-1,1).  Each link is
 *               followed by its opposite.  Per-link arrays are [19][N].
 *   flags       uint8 per cell: FSLBM_LIQUID, FSLBM_INTERFACE, FSLBM_GAS,
 *               FSLBM_WALL.  A face of a non-periodic axis is a half-way wall.
 *   f           populations in FP64 at the interface, whatever the internal
 *               precision.  fslbm_set_state takes pre-collision f(x,t);
 *               fslbm_get_fields returns post-collision f~(x,t) (what the
 *               library stores); fslbm_set_state_post takes that back.
 *   where       FSLBM_HOST: plain host pointers (copied synchronously);
 *               FSLBM_DEVICE: device pointers on the handle's GPU (copied on
 *               the handle's stream).
 *   ownership   the library owns its device state; buffers passed in or out
 *               belong to the caller, are copied, and are never retained.
 *   errors      every int-returning call returns an fslbm_status.  Device-side
 *               faults of the method (instability, a liquid cell next to gas)
 *               are recorded in a sticky device error word, reported by the
 *               next synchronising call (fslbm_sync, fslbm_get_fields,
 *               fslbm_total_mass) and cleared by fslbm_set_state.  No call
 *               exits or aborts the process.
 *   threading   one handle per host thread at a time; calls on one handle are
 *               ordered on its CUDA stream.
 */
#ifndef FSLBM_H
#define FSLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fslbm fslbm_t;

enum fslbm_rule { FSLBM_FSK = 0, FSLBM_FSL = 1 };

/* Precision forms: FP64 throughout; FP32 populations with FP64 interface
 * mass and mass balance; FP16 storage with FP32 arithmetic and FP64
 * interface mass and mass balance.  Both reduced forms store, and compute
 * with, the deviation f_q - w_q of each population from its rest value
 * (rho_0 = 1): the step is affine in the populations with rho - 1 in place
 * of rho, and the deviations keep the full mantissa for the flow. */
enum fslbm_precision { FSLBM_F64 = 0, FSLBM_F32 = 1, FSLBM_F16 = 2 };

enum fslbm_status {
  FSLBM_OK = 0,
  FSLBM_ERR_ARG = -1,      /* bad argument or parameter */
  FSLBM_ERR_OOM = -2,      /* device allocation failed */
  FSLBM_ERR_CUDA = -3,     /* a CUDA runtime call failed */
  FSLBM_ERR_STATE = -4,    /* invariant violated: a liquid cell next to gas, bad flag; in the
                              bounds-checked library also an index outside its array */
  FSLBM_ERR_UNSTABLE = -5, /* non-finite or non-positive density, or a liquid cell's velocity
                              above u_max (the stability guard of the step) */
  FSLBM_ERR_OVERFLOW = -6, /* a conversion list exceeded its capacity */
  FSLBM_ERR_TIMEOUT = -7,  /* a bounded device-side wait expired (staged loads of the bulk kernel, the
                              grid barrier of the conversion kernel) */
  FSLBM_ERR_TOO_LARGE = -8 /* beyond the fixed scratch of fslbm_mass_balance_noalloc */
};

enum fslbm_cell { FSLBM_LIQUID = 1, FSLBM_INTERFACE = 2, FSLBM_GAS = 4, FSLBM_WALL = 8 };

enum fslbm_where { FSLBM_HOST = 0, FSLBM_DEVICE = 1 };

/* Loads of the bulk stream-collide kernel (an implementation choice with no
 * counterpart in the paper; the pull of Eq. lbe1 is the same every way, and
 * so are the results, bit for bit).  FP64 lattices always load plainly. */
enum fslbm_loads {
  FSLBM_LOADS_PLAIN = 0, /* default: one cell per lane, plain coalesced global loads */
  FSLBM_LOADS_ASYNC = 1, /* each lane copies its 19 values into shared memory with cp.async,
                            two 32-cell segments ahead of use */
  FSLBM_LOADS_TMA = 2    /* the 19 rows of a segment by tensor-map (TMA) copies; needs nx a multiple
                            of 16 bytes of elements and nx >= 32 cells + two 16-byte halos, else
                            plain loads */,
  FSLBM_LOADS_PAIRS = 3  /* two x-adjacent cells per lane: one 32-bit (FP16) or 64-bit (FP32) load
                            per population without an x component and one store per population
                            and pair, the collision of both cells in packed FP32x2 instructions
                            (the fastest on GB300); needs nx even and 19 N < 2^32, else plain */
};

/* Field bits of fslbm_get_fields; out[] holds one pointer per set bit, in
 * increasing bit order. */
enum fslbm_field {
  FSLBM_FIELD_FLAGS = 1, /* uint8 [N] */
  FSLBM_FIELD_F = 2,     /* double [19][N], post-collision f~(t); 0 off fluid cells */
  FSLBM_FIELD_MASS = 4,  /* double [N]: interface m, liquid rho, else 0 */
  FSLBM_FIELD_PHI = 8,   /* double [N]: liquid 1, interface m/rho, gas its stored fill */
  FSLBM_FIELD_RHO = 16,  /* double [N]: rho = sum_q f_q on fluid cells */
  FSLBM_FIELD_U = 32     /* double [N][3]: u = U + F/(2 rho_0) (Eq. momentum) */
};

/* Parameters of a lattice (fslbm_default_params fills the defaults). */
typedef struct {
  int dims[3];        /* nx, ny, nz > 0 */
  double tau;         /* > 1/2; lambda_+ = -1/tau, nu = (tau - 1/2)/3 (Sec. 2.1) */
  double magic;       /* Lambda = Lambda_+ Lambda_- (Sec. 3.1) fixing lambda_-; <= 0: SRT
                         (lambda_- = lambda_+); default 3/16 */
  double g[3];        /* body force per unit mass and step; F = rho_0 g */
  double rho_G;       /* gas density: boundary pressure P_b = rho_G/3 (Eq. koerner) */
  double sigma;       /* surface tension: rho_b = rho_G + 3 sigma kappa (Sec. 2.3); kappa from
                         height functions along the dominant normal axis, where those columns
                         are open from the other axes' heights, else the divergence of the
                         normal */
  int rule;           /* FSLBM_FSK or FSLBM_FSL */
  int compressible;   /* 1: rho_0 = rho (Qian); 0: rho_0 = 1 (He-Luo), default */
  int linear_eq;      /* 1: drop the non-linear part N_q of e^+ (Stokes flow) */
  double eps;         /* conversion threshold: fill if m > (1+eps) rho, empty if m < -eps rho */
  int periodic[3];    /* 1 = periodic axis, 0 = half-way wall at both faces */
  int zshift;         /* z offset added on a periodic x wrap (inclined films) */
  int freeze;         /* 1 = frozen interface: no mass exchange, no conversions */
  int cleanup;        /* isolated-cell rules (Thuerey): bit 1 fills an interface cell with no gas
                         neighbour, bit 2 empties an interface cell with no liquid/interface
                         neighbour (its mass goes to the lost ledger if no receiver); default 3 */
  int keep_f0;        /* 1: keep the pre-collision initial populations in FP64 (152 B per cell) so
                         that fslbm_adjoint_backward reverses the initial collision from them; 0:
                         it recovers them by inverting the collision from the stored populations
                         (exact in FP64, limited by the storage precision in FP32/FP16) */
  double delta_min;   /* lower clamp of the free-surface link fraction, default 0 */
  int stress;         /* 1: the boundary shear-rate term D c_a c_b S^b_ab of Eq. bterm on every
                         rebuilt gas link (D of Table 1; S extrapolated from the cell's own
                         non-equilibrium part, its normal-tangential components set to zero in
                         the interface basis, Eq. bstress / Eq. proj2); 2: the same term with the
                         prescribed S^b of shear_b (Sec. 6, linear Couette flows); 0 (default):
                         D = 0 */
  double shear_b[6];  /* prescribed S^b for stress = 2: xx, yy, zz, xy, xz, yz */
  double wall_u[3];   /* velocity of every wall: half-way bounce-back links get
                         + 6 w_q (c_q.u_w) (rho_0 = 1; not with compressible, not on CLI links) */
  int ub_extrap;      /* u_b in e^+(rho_b, u_b) of the FSL closure (Eq. closure, Table 1): 0
                         (default) the interface node's own velocity u(x_b) (first order, the
                         next-neighbour value of Sec. 6's breaking dam); 1 its linear extrapolation
                         along the link to the surface point x_w = x_b + delta c_p,
                         u(x_b) + delta (u(x_b) - u(x_b - c_p)) (second order; with the non-linear
                         e^+ a linear flow along a surface that is not lattice-aligned needs it,
                         Sec. 6).  FSK links, and FSL links that fall back to FSK, keep u(x_b). */
  int recon_nc;       /* 1: an interface cell also rebuilds, with the rule's closure, every link p
                         toward a liquid/interface node whose direction points to the gas side of
                         the surface, n.c_p > 1e-6 with n the unit normal of the plane fit
                         (the reconstruction along the normal of Koerner et al., whose tracking
                         Sec. 4.4 and Sec. 6 follow); 0 (default): only the links to gas cells */
  int excess_split;   /* excess mass of a filled or emptied cell: 0 (default) split equally over
                         its receivers; 1 split in proportion to the weights along the fill-level
                         normal n = -grad phi (central differences of the fill levels after the
                         mass exchange): n.c_q > 0 for a filled cell, -n.c_q > 0 for an emptied
                         one (Thuerey's distribution, whose tracking Sec. 4.4 follows); equal
                         split where no receiver has a positive weight (sum below 1e-12) */
  int bulk_loads;     /* fslbm_loads: how the bulk kernel of FP32/FP16 lattices reaches the
                         pulled values (FP64 always loads them plainly); same results every way */
  int precision;      /* fslbm_precision */
  void *stream;       /* cudaStream_t for all work of the handle; NULL = legacy default */
  int elvira;         /* 1: where the height columns along the dominant axis are open, the
                         interface normal by ELVIRA (Pilliod & Puckett) in place of the Parker-Youngs
                         gradient: 27 candidates from backward, central and forward differences of
                         3-cell column sums of the 3x3x3 block along each axis, the one whose planes
                         (each through the cell's own fill) best reproduce the block's fill levels;
                         exact for planes.  The higher-order reconstruction the conclusion (Sec. 5)
                         asks of the interface position.  0 (default): Parker-Youngs */
  int adjoint_fp32;   /* 1: the reverse step of an FP32/FP16 lattice computes in FP32, in the
                         deviations f - w_q of the forward step (the adjoint variables stay FP64 in
                         memory); 0 (default): in FP64.  An implementation choice: GB300 runs FP64
                         at a small fraction of its FP32 rate, and the reverse step is bound by it.
                         Ignored by FP64 lattices */
  double u_max;       /* stability guard: a step in which a liquid cell's velocity exceeds u_max
                         lattice units reports FSLBM_ERR_UNSTABLE (the equilibria are second order in
                         u, and the lattice speed of sound is 1/sqrt(3)); default 0.4, 0 switches it
                         off.  Interface cells are not guarded: isolated ones in spray, with a few
                         fluid neighbours, reach 0.4 in stable flows (dam break 512x256x256,
                         tau 0.53, steps 5000-15500: interface cells up to 0.4 and above, liquid
                         cells below 0.14) */
} fslbm_params;

/* Defaults: tau 0.8, magic 3/16, g 0, rho_G 1, sigma 0, FSL, rho_0 = 1,
 * non-linear e^+, eps 1e-3, all axes walls, zshift 0, dynamic interface,
 * cleanup 3, delta_min 0, FP64, default stream.  dims are set to 0. */
void fslbm_default_params(fslbm_params *p);

/* Create a lattice with the paper's problem data (Eq. freeboundary:
 * viscosity through tau, P_b through rho_G, sigma, gravity g) and the given
 * rule; other parameters at their defaults.  *out receives the handle.
 * Returns FSLBM_ERR_ARG for dims <= 0 or tau <= 1/2, FSLBM_ERR_OOM when the
 * device state does not fit.  The state is all-gas until set. */
int fslbm_create(const int dims[3], double tau, const double g[3], double rho_G, double sigma,
                 int rule, fslbm_t **out);

/* Relaxation time of a kinematic viscosity: tau = 3 nu + 1/2 (Sec. 2.1,
 * nu = c_s^2 (tau - 1/2), c_s^2 = 1/3).  *tau receives it.  Returns
 * FSLBM_ERR_ARG for nu <= 0, a non-finite nu or tau == NULL.  Host only. */
int fslbm_tau_of_viscosity(double nu, double *tau);

/* As fslbm_create with every parameter given.  FSL with |1 - tau| < 1e-3 is
 * rejected (FSLBM_ERR_ARG): the library stores post-collision populations
 * and recovers n^+ from them by dividing by 1 + lambda_+. */
int fslbm_create_ex(const fslbm_params *p, fslbm_t **out);

/* Set the state from cell flags, pre-collision populations f[19][N] (FP64),
 * fill levels phi[N] (read on interface cells, and on gas cells of a frozen
 * interface; m = phi * rho), and optional wall link fractions
 * wall_delta[19][N] (the fraction delta_w in [0,1] of link q from fluid cell
 * i to the wall it crosses, CLI rule; a negative entry or NULL = half-way
 * bounce-back).  Synchronises.  Returns FSLBM_ERR_STATE when a liquid cell
 * touches a gas cell or a flag is not one of the four cell kinds. */
int fslbm_set_state(fslbm_t *h, const uint8_t *flags, const double *f, const double *phi,
                    const double *wall_delta, int where);

/* As fslbm_set_state, but the populations are built by the library:
 * f = f^eq(rho, u) + noise (Eq. eqEven / eqOdd with u^eq = u), from rho[N],
 * u[N][3] and an optional noise[19][N] (NULL = none). */
int fslbm_init_equilibrium(fslbm_t *h, const uint8_t *flags, const double *rho, const double *u,
                           const double *phi, const double *noise, const double *wall_delta,
                           int where);

/* Restore a state saved with fslbm_get_fields: flags, post-collision
 * f~[19][N], mass m[N] (interface m; ignored elsewhere), phi[N], optional
 * wall_delta.  Round-trips every precision bit-exactly. */
int fslbm_set_state_post(fslbm_t *h, const uint8_t *flags, const double *f_post, const double *m,
                         const double *phi, const double *wall_delta, int where);

/* Advance n >= 0 time steps.  Asynchronous on the handle's stream: returns
 * launch errors only; method faults appear at the next synchronising call. */
int fslbm_step(fslbm_t *h, int n);

/* Wait for the handle's stream; return the sticky device error, if any. */
int fslbm_sync(fslbm_t *h);

/* Copy the fields selected by mask (fslbm_field bits) into out[], one buffer
 * per set bit in increasing bit order, host or device per `where`.
 * Synchronises. */
int fslbm_get_fields(fslbm_t *h, unsigned mask, void *const *out, int where);

/* Total mass M = sum_liquid rho + sum_interface m + lost, and the lost
 * ledger (excess mass that found no interface neighbour), in FP64 with a
 * fixed reduction order.  Synchronises. */
int fslbm_total_mass(fslbm_t *h, double *mass, double *lost);

/* Mass balance of the last step, reduced inside the step kernels before the
 * conversions (which conserve it): M(t) as above.  Synchronises. */
int fslbm_step_mass(fslbm_t *h, double *mass);

/* Conversions of the last step: out[0] filled (interface -> liquid),
 * out[1] emptied (interface -> gas), out[2] new interface from gas, out[3]
 * new interface from liquid; out[4] interface cells at the start of the
 * step.  Synchronises. */
int fslbm_counters(fslbm_t *h, long long out[5]);

/* Per-kernel timing.  While on, fslbm_step records CUDA events on the
 * handle's stream between the kernel groups of every step (a few
 * microseconds of overhead per step).  Switching it on clears the totals. */
int fslbm_timing(fslbm_t *h, int on);

/* Average device time per step, in milliseconds, of each kernel group over
 * the steps taken with timing on: ms[0] the bulk stream-collide kernel alone,
 * ms[1] the interface kernels (geometry and interface cells), ms[2] the
 * mass-balance reduction, ms[3] the conversion kernels (the counter reset and
 * the fluid-segment scan are in no group); *steps receives the number of
 * timed steps.  Synchronises. */
int fslbm_timing_read(fslbm_t *h, double ms[4], long long *steps);

/* ---- Differentiation: hand-written adjoint -------------------------------
 * The differentiated map runs from the initial populations of the current
 * state (as set by fslbm_init_equilibrium / fslbm_set_state, whose collision
 * is included) through nsteps time steps to an objective J, with every
 * discrete decision of the forward pass held: the cell flags of every step,
 * so that cell conversions are replayed as the forward pass took them (the
 * adjoints of the new cells' equilibrium initialisation, of the excess split
 * and of m = rho for new cells from liquid are taken; Sec. 2.3), the height-
 * function or plane-fit branch, the dominant axis, clamps of delta.
 * Supported: rho_0 = 1, sigma = 0, D = 0 (stress off), resting walls (wall_u = 0), u_b = u(x_b)
 * (ub_extrap = 0), gas links only (recon_nc = 0) and the equal excess split (excess_split = 0);
 * FSLBM_ERR_ARG otherwise.  Parameters: nu = (tau - 1/2)/3 with the magic
 * parameter Lambda held fixed, g, and the initial fill levels phi0 of
 * interface cells (m0 = phi0 rho0). */
enum fslbm_objective {
  FSLBM_OBJ_SURFACE_UX = 0, /* mean u_x over interface cells at the end */
  FSLBM_OBJ_FLUX_X = 1      /* sum over liquid and interface cells of phi u_x, divided by nx */
};

/* Forward pass: run nsteps >= 1 steps from the current state with a full
 * checkpoint (flags, f~, m, phi) every K >= 1 steps, and return J.  Holds
 * ceil(nsteps/K) checkpoints on the device until the handle's state is set
 * again or the handle is destroyed. */
int fslbm_adjoint_forward(fslbm_t *h, int nsteps, int K, int objective, double *J);

/* Reverse pass (once per forward pass): recompute each K-step segment from
 * its checkpoint, storing its K + 1 states (flags included), and run the
 * adjoint step kernels backwards, the reverse of each step's conversions
 * first.  Returns dJ/dnu, dJ/dg[3], and dJ/dphi0[N] (zero off interface
 * cells; host or device per `where`; NULL to skip).  Afterwards the handle
 * holds the state of step min(K, nsteps). */
int fslbm_adjoint_backward(fslbm_t *h, double *dJ_dnu, double dJ_dg[3], double *dJ_dphi0, int where);

/* Costs of the last differentiation: device milliseconds per forward step
 * and per adjoint step (segment recomputation excluded), and the device bytes
 * held (lattice + checkpoints + adjoint buffers). */
int fslbm_adjoint_stats(fslbm_t *h, double *fwd_ms_per_step, double *adj_ms_per_step, size_t *peak_bytes);

/* ---- Mass balance without device allocation --------------------------------
 * The paper has no counterpart to this entry point; it is a service for
 * callers that cannot allocate device memory once they run: applications whose
 * framework owns the GPU's memory through its own pool and refuses other
 * allocations, and time-critical loops where cudaMalloc/cudaFree would
 * synchronise the device and stall other streams.  It computes
 * M = sum_liquid rho + sum_interface m + lost over caller-owned device arrays
 * and allocates nothing: its per-block partial sums live in a fixed array
 * inside the library (FSLBM_NOALLOC_MAX_BLOCKS doubles, 32 KiB, held by every
 * GPU that loads the library until the process exits).
 *   flags     uint8 [n_cells] cell kinds, device memory
 *   f_post    [19][n_cells] populations in the storage of `precision`:
 *             double holding f (FSLBM_F64), float (FSLBM_F32) or half
 *             (FSLBM_F16) holding f - w_q, device memory
 *   m         double [n_cells] interface mass (read on interface cells only)
 *   lost      added to the sum (the lost ledger of fslbm_total_mass)
 *   mass_out  one double in device memory, written by the call
 *   stream    cudaStream_t, NULL = legacy default stream; the call is
 *             asynchronous on it and returns launch errors only
 * At most FSLBM_NOALLOC_MAX_BLOCKS * FSLBM_NOALLOC_CELLS_PER_BLOCK cells
 * (268,435,456); larger n_cells returns FSLBM_ERR_TOO_LARGE before any work.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one array, which keeps the
 * last call's partial sums; each call writes every entry it reads first.
 * Calls whose work overlaps on the GPU (concurrent streams) race on the
 * array: order them. */
#define FSLBM_NOALLOC_MAX_BLOCKS 4096
#define FSLBM_NOALLOC_CELLS_PER_BLOCK 65536
int fslbm_mass_balance_noalloc(const uint8_t *flags, const void *f_post, int precision, const double *m,
                               long long n_cells, double lost, double *mass_out, void *stream);

/* ---- Slab decomposition ---------------------------------------------------
 * The paper's runs used a parallel framework that splits the lattice into
 * blocks (Sec. 4); these calls let a caller run a lattice as slabs, one
 * handle per slab (one per GPU, or several on one GPU).  A slab's handle
 * holds the cells it owns plus G ghost layers beside each cut, copies of the
 * neighbouring slabs' cells.  One time step of a cell reads the state of time
 * t within 7 cells of it (interface geometry 3, streaming 1, the chains of
 * neighbour tests of the conversions 3), so with G >= 7 a step leaves every
 * owned cell exact, and refilling the ghost layers from the neighbours'
 * owned cells (pack, transport by the caller, unpack) makes the whole slab
 * exact again: one exchange per step, conversions included.  A cut is a
 * half-way wall to the handle; no ghost cell reaches an owned one within a
 * step.  Implementation services, no counterpart in the paper. */

/* Cells of the box [lo, hi) (per axis, 0 <= lo < hi <= dims) are the ones the
 * handle owns: the mass balance (fslbm_total_mass, fslbm_step_mass) sums them
 * only, and only their excess mass enters the lost ledger; the others are
 * ghost cells, stepped like every cell.  Default: every cell.  Applies to the
 * steps enqueued after the call.  FSLBM_ERR_ARG for an empty or outside box. */
int fslbm_set_owned(fslbm_t *h, const int lo[3], const int hi[3]);

/* Bytes of the packed state of the box [lo, hi): u8 cell kinds, f64 interface
 * mass, fill levels phi(t) in the arithmetic type (f64 for FSLBM_F64, else
 * f32) and post-collision populations [19][n] in the storage type (f - w_q in
 * the reduced forms), each block 16-byte aligned, cells in box order (x
 * fastest).  FSLBM_ERR_ARG (negative) for a bad box. */
long long fslbm_halo_bytes(const fslbm_t *h, const int lo[3], const int hi[3]);

/* Copy the current state of the box [lo, hi) into the device buffer buf
 * (16-byte aligned, fslbm_halo_bytes long, on the handle's GPU), or set the
 * box's state from one: cell kinds (static wall bits stay the handle's own),
 * interface mass, fill levels and post-collision populations.  Asynchronous
 * on the handle's stream; the caller orders the transport between a pack and
 * the matching unpack.  Unpacking ends a differentiation in progress.
 * FSLBM_ERR_ARG for a bad box or a misaligned or NULL buffer. */
int fslbm_halo_pack(fslbm_t *h, const int lo[3], const int hi[3], void *buf);
int fslbm_halo_unpack(fslbm_t *h, const int lo[3], const int hi[3], const void *buf);

/* Steps taken since the last set_state. */
long long fslbm_time(const fslbm_t *h);

/* The fslbm_loads the bulk kernel of this handle uses (FSLBM_ERR_ARG for
 * NULL).  An implementation property with no counterpart in the paper. */
int fslbm_bulk_loads(const fslbm_t *h);

/* Scheduling of the interface kernels (an implementation choice with no
 * counterpart in the paper; the results are the same either way, bit for
 * bit).  on = 1 (default): after the segment scan the interface geometry,
 * and beside the two-cells-per-lane bulk kernel the interface kernel too,
 * run on a second stream of the handle while the bulk kernel runs on its
 * stream; the pair kernel's grid then leaves room for them on every SM, and
 * the streams join before the conversions.  on = 0: every kernel in order on
 * the handle's stream, the bulk kernel on a full resident wave (to time the
 * kernels alone).  FSLBM_ERR_ARG for other values. */
int fslbm_set_overlap(fslbm_t *h, int on);

/* Kernel launches one fslbm_step time step makes on this handle (the
 * per-step reset, segment list, bulk, interface geometry where the rule,
 * surface tension, the shear term or the normal links need it, interface,
 * the two-level mass reduction, and the conversions: one cooperative launch
 * where the device allows it, else four; none with frozen flags), or
 * FSLBM_ERR_ARG for NULL.  An implementation property with no counterpart in
 * the paper. */
int fslbm_launches_per_step(const fslbm_t *h);

/* Self-check of the grid barrier between the conversion stages: one
 * cooperative launch of it (two resident blocks per SM) on `stream` (NULL =
 * legacy default).  expire = 0: the barrier completes; expire = 1: it waits
 * for one block more than exists, so its bounded wait runs out after about a
 * second and records the expiry, the way a barrier that never completes ends
 * in a step.  Returns FSLBM_OK when it completed, FSLBM_ERR_TIMEOUT when it
 * expired, FSLBM_ERR_CUDA when the device refuses the cooperative launch,
 * FSLBM_ERR_ARG for another expire.  Synchronises the stream; the context
 * stays usable either way.  An implementation property with no counterpart
 * in the paper. */
int fslbm_check_grid_barrier(int expire, void *stream);

/* The current device's FP64 arithmetic rate in TFLOP/s (a fused multiply-add
 * counts two): chains of dependent FMAs on every SM, timed with CUDA events
 * on `stream` (NULL = legacy default), best of three after a warm-up run.
 * The ceiling of the FP64 form, whose stream-collide is bound by arithmetic
 * on GB300.  Synchronises the stream.  An implementation property with no
 * counterpart in the paper. */
int fslbm_fp64_rate(double *tflops, void *stream);

/* Build properties of the loaded library: bit 0 set in the bounds-checked
 * library (compiled with FSLBM_CHECKED).  There every cell index a kernel
 * reads from a segment record or a cell list, and every source cell that a
 * bulk kernel's fast path forms by offset arithmetic, is tested against the
 * lattice before the access (as is the interface kernels' precondition for
 * a cell handled as interior: 3 or more cells inside every face); a failed
 * test skips to cell 0 and makes the next synchronising call return
 * FSLBM_ERR_STATE.  Results are otherwise those of the normal library.  An
 * implementation property with no counterpart in the paper. */
int fslbm_build_info(void);

/* Bytes of device memory held by the handle. */
size_t fslbm_device_bytes(const fslbm_t *h);

/* Text of the last error on this handle (static storage, never NULL). */
const char *fslbm_last_error(const fslbm_t *h);

/* Release the handle and its device memory.  NULL is a no-op. */
void fslbm_destroy(fslbm_t *h);

#ifdef __cplusplus
}
#endif

#endif /* FSLBM_H */

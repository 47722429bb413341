"""One free-surface LBM time step in exact rational arithmetic.

Test infrastructure: an independent restatement of the step that the FP64
oracle (oracle/fslbm_oracle.cpp) performs, written from the paper and from
the readings of its silent points, in Python ``fractions.Fraction``
arithmetic so that no rounding enters.  It shares no code with the oracle or
with the CUDA library; the tests hand both the same state (the oracle's own
FP64 values, which are exact rationals) and compare one step.

Scope: rho_0 = 1 (incompressible equilibrium), half-way bounce-back walls at
non-periodic faces and at WALL cells, no surface tension, D = 0, u_b = u(x_b),
gas links only, equal excess split.  FSK needs no interface geometry; FSL
needs the link fraction delta, which is rational where the height columns
of the cell are closed (the normal's length cancels), so FSL is covered on
such cells and a step that meets an open column raises ``Irrational``.

Paper: Bogner, Ammer, Ruede, "Boundary Conditions for Free Interfaces with
the Lattice Boltzmann Method" (arXiv:1409.5645).
"""
from __future__ import annotations

import os
from fractions import Fraction as Fr

import numpy as np

LIQ, IFC, GAS, WALL = 1, 2, 4, 8
# D3Q19 directions in the public population order (rest, six axis links,
# twelve diagonals, each link followed by its opposite)
C = [(0, 0, 0),
     (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
     (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
     (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
     (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]
Q = 19
OPP = [C.index(tuple(-a for a in c)) for c in C]
# lattice weights of Qian et al. for D3Q19 (Sec. 2.1), c_s^2 = 1/3
W = [Fr(1, 3) if sum(a * a for a in c) == 0 else (Fr(1, 18) if sum(a * a for a in c) == 1 else Fr(1, 36))
     for c in C]
HALF = Fr(1, 2)

_GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                       "table1_closure_coefficients.txt")


class Irrational(Exception):
    """The step needs a link fraction that is not rational (an open height
    column of an FSL interface cell)."""


def _table1():
    rows = {}
    for line in open(_GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, *ex = line.split()
        rows[name] = ex
    return rows


TABLE1 = _table1()


def closure_coefficients(rule: str, delta: Fr, lam: Fr):
    """(a0, abar0, a1, alpha_plus, C) of Table 1 at link fraction delta and
    lambda_+, evaluated in rationals (the table's entries are polynomials)."""
    env = {"delta": delta, "lam": lam}
    out = []
    for e in TABLE1[rule]:
        out.append(Fr(eval(e.replace("0.5", "Fraction(1, 2)"), {"Fraction": Fr}, env)))
    return out


class Lattice:
    """A tiny lattice with flags and the method's state in rationals."""

    def __init__(self, dims, periodic, tau, magic, g, rho_G, rule, eps, cleanup, linear_eq=0,
                 delta_min=0.0):
        self.nx, self.ny, self.nz = (int(v) for v in dims)
        self.N = self.nx * self.ny * self.nz
        self.periodic = tuple(bool(v) for v in periodic)
        self.tau = Fr(tau)
        # TRT rates (Sec. 2.1 and Sec. 3.1): lambda_+ = -1/tau; the magic
        # parameter Lambda = Lambda_+ Lambda_-, Lambda_pm = -(1/2 + 1/lambda_pm),
        # fixes lambda_-; Lambda <= 0 selects one rate (SRT)
        self.lp = Fr(-1) / self.tau
        if magic <= 0:
            self.lm = self.lp
        else:
            Lp = -(HALF + 1 / self.lp)
            Lm = Fr(magic) / Lp
            self.lm = Fr(-1) / (Lm + HALF)
        self.g = [Fr(v) for v in g]
        self.rho_G = Fr(rho_G)
        self.rule = "FSL" if rule else "FSK"
        self.eps = Fr(eps)
        self.cleanup = int(cleanup)
        self.linear = bool(linear_eq)
        self.delta_min = Fr(delta_min)

    # cell index and neighbours ------------------------------------------------
    def index(self, x, y, z):
        return x + self.nx * (y + self.ny * z)

    def xyz(self, i):
        return i % self.nx, (i // self.nx) % self.ny, i // (self.nx * self.ny)

    def nb(self, i, d):
        """Cell i + d, or None beyond a non-periodic face (a half-way wall)."""
        x, y, z = self.xyz(i)
        p = [x + d[0], y + d[1], z + d[2]]
        n = (self.nx, self.ny, self.nz)
        for a in range(3):
            if not 0 <= p[a] < n[a]:
                if not self.periodic[a]:
                    return None
                p[a] %= n[a]
        return self.index(*p)

    def kind(self, flags, j):
        return WALL if j is None else flags[j]

    # equilibria (Eq. eqEven / eqOdd), rho_0 = 1 ---------------------------
    def e_plus(self, q, rho, u):
        e = W[q] * rho
        if not self.linear:
            cu = sum(C[q][a] * u[a] for a in range(3))
            uu = sum(v * v for v in u)
            # N_q = rho_0/2 u_a u_b (c_qa c_qb / c_s^2 - delta_ab)
            e += W[q] * 3 * HALF * (3 * cu * cu - uu)
        return e

    def e_minus(self, q, u):
        return 3 * W[q] * sum(C[q][a] * u[a] for a in range(3))

    def moments(self, fq):
        """rho = sum f, rho_0 U = sum c f, u = U + F/(2 rho_0), F = rho_0 g."""
        rho = sum(fq)
        U = [sum(C[q][a] * fq[q] for q in range(Q)) for a in range(3)]
        return rho, U, [U[a] + HALF * self.g[a] for a in range(3)]

    # geometry of an FSL interface cell (Sec. 2.2, Sec. 5) -----------------
    def fill(self, flags, phi, j, own):
        k = self.kind(flags, j)
        if k == LIQ:
            return Fr(1)
        if k == IFC:
            return phi[j]
        if k == GAS:
            return Fr(0)
        return own  # a wall takes the cell's own fill level

    def link_delta(self, flags, phi, i, p):
        """delta of the boundary link p of interface cell i from the height
        function plane: gradient by the Parker-Youngs weights picks the
        dominant axis; with every one of the 3 x 3 columns of 7 cells along it
        closed (liquid at its liquid end, gas at its gas end, no wall) the
        plane through the centre column's height has the normal
        v = (s, -dH/db, -dH/dc) and delta = (H_0 - 7/2) / (v.c_p) for
        v.c_p > 0, else 1/2; clamped to [delta_min, 1]."""
        own = phi[i]
        grad = [Fr(0)] * 3
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if dx == dy == dz == 0:
                        continue
                    v = self.fill(flags, phi, self.nb(i, (dx, dy, dz)), own)
                    d = (dx, dy, dz)
                    for a in range(3):
                        if d[a]:
                            o1, o2 = d[(a + 1) % 3], d[(a + 2) % 3]
                            grad[a] += d[a] * (2 - abs(o1)) * (2 - abs(o2)) * v
        n = [-v for v in grad]
        if all(v == 0 for v in n):
            return HALF
        a = max(range(3), key=lambda k: (abs(n[k]), -k))
        s = 1 if n[a] > 0 else -1
        b = 1 if a == 0 else 0
        c3 = 3 - a - b
        H = {}
        for ib in (-1, 0, 1):
            for ic in (-1, 0, 1):
                tot = Fr(0)
                for k in range(-3, 4):
                    d = [0, 0, 0]
                    d[a], d[b], d[c3] = k, ib, ic
                    j = self.nb(i, tuple(d))
                    kj = self.kind(flags, j)
                    if kj == WALL:
                        raise Irrational("wall in a height column")
                    if k == -3 * s and kj != LIQ:
                        raise Irrational("open column")
                    if k == 3 * s and kj != GAS:
                        raise Irrational("open column")
                    tot += self.fill(flags, phi, j, own)
                H[ib, ic] = tot
        v = [Fr(0)] * 3
        v[a] = Fr(s)
        v[b] = -HALF * (H[1, 0] - H[-1, 0])
        v[c3] = -HALF * (H[0, 1] - H[0, -1])
        vc = sum(v[k] * C[p][k] for k in range(3))
        if not vc > 0:
            return HALF
        dl = (H[0, 0] - Fr(7, 2)) / vc
        return min(max(dl, self.delta_min), Fr(1))

    # one step ----------------------------------------------------------------
    def step(self, flags, f, m, phi, variant=None):
        """flags: list of ints; f: [19][N] pre-collision populations f(t);
        m, phi: interface mass and fill level (read on interface cells).
        Returns (flags, f, m, phi, lost, events) at t+1, f pre-collision.
        ``variant`` plants one plausible misreading of the conversion rules
        (tests show that the comparison with the oracle detects each):
        "keep_empty" keeps an emptied cell next to a filled one, "new_avg_all"
        averages a new cell over new cells too, "new_avg_precollision" over
        its neighbours' populations of time t, "recv_converting" lets
        converting cells receive excess."""
        N = self.N
        fluid = lambda k: k in (LIQ, IFC)
        # 1. geometry of time t: link fractions of FSL boundary links (cached)
        deltas = {}
        # 2. TRT collision (Eq. lbe2): f~ = f + lambda_+ n^+ + lambda_- n^-,
        #    e^- at u^eq = U - F/lambda_-, e^+ at u = U + F/2
        ft = [[Fr(0)] * N for _ in range(Q)]
        nplus = [[Fr(0)] * N for _ in range(Q)]
        rho_t = [Fr(0)] * N
        u_t = [[Fr(0)] * 3 for _ in range(N)]
        for i in range(N):
            if not fluid(flags[i]):
                continue
            fq = [f[q][i] for q in range(Q)]
            rho, U, u = self.moments(fq)
            ueq = [U[a] - self.g[a] / self.lm for a in range(3)]
            for q in range(Q):
                qb = OPP[q]
                npq = HALF * (fq[q] + fq[qb]) - self.e_plus(q, rho, u)
                nmq = HALF * (fq[q] - fq[qb]) - self.e_minus(q, ueq)
                ft[q][i] = fq[q] + self.lp * npq + self.lm * nmq
                nplus[q][i] = npq
            rho_t[i], u_t[i] = rho, u
        # 3. pull streaming (Eq. lbe1); walls by half-way bounce-back; links
        #    from gas by the rule's closure (Eq. koerner / Eq. closure with
        #    Table 1), boundary link p = qbar, rho_b = rho_G, u_b = u(x_b, t);
        #    FSL falls back to FSK where x_b - c_p is not fluid
        fn = [[Fr(0)] * N for _ in range(Q)]
        for i in range(N):
            if not fluid(flags[i]):
                continue
            fn[0][i] = ft[0][i]
            for q in range(1, Q):
                src = self.nb(i, tuple(-a for a in C[q]))
                ks = self.kind(flags, src)
                p = OPP[q]
                if fluid(ks):
                    fn[q][i] = ft[q][src]
                elif ks == WALL:
                    fn[q][i] = ft[p][i]
                else:
                    if flags[i] != IFC:
                        raise ValueError("a liquid cell next to gas")
                    eb = self.e_plus(p, self.rho_G, u_t[i])
                    up = self.nb(i, tuple(-a for a in C[p]))  # x_b - c_p
                    if self.rule == "FSK" or not fluid(self.kind(flags, up)):
                        a0, ab0, a1, ap, Cc = closure_coefficients("FSK", HALF, self.lp)
                        fn[q][i] = a0 * ft[p][i] + ab0 * ft[q][i] + ap * eb
                    else:
                        if (i, p) not in deltas:
                            deltas[i, p] = self.link_delta(flags, phi, i, p)
                        a0, ab0, a1, ap, Cc = closure_coefficients("FSL", deltas[i, p], self.lp)
                        fn[q][i] = (a0 * ft[p][i] + ab0 * ft[q][i] + a1 * ft[p][up] + Cc * nplus[p][i]
                                    + ap * eb)
        # 4. interface mass exchange (Sec. 2.3): dm = sum_q s_q (f~_q(x - c_q)
        #    - f~_qbar(x)), s = 1 from liquid, (phi(x) + phi(y))/2 from interface
        m1 = list(m)
        for i in range(N):
            if flags[i] != IFC:
                continue
            dm = Fr(0)
            for q in range(1, Q):
                y = self.nb(i, tuple(-a for a in C[q]))
                ky = self.kind(flags, y)
                if ky == LIQ:
                    s = Fr(1)
                elif ky == IFC:
                    s = HALF * (phi[i] + phi[y])
                else:
                    continue
                dm += s * (ft[q][y] - ft[OPP[q]][i])
            m1[i] = m[i] + dm
        rho1 = [sum(fn[q][i] for q in range(Q)) if fluid(flags[i]) else Fr(0) for i in range(N)]
        # 5. conversions (Koerner / Thuerey as read: thresholds with strict
        #    inequalities, isolated-cell rules, fill before empty)
        nbrs = [[self.nb(i, C[q]) for q in range(1, Q)] for i in range(N)]
        F, E = set(), set()
        for i in range(N):
            if flags[i] != IFC:
                continue
            kinds = [self.kind(flags, j) for j in nbrs[i]]
            no_gas = GAS not in kinds
            no_fluid = not any(fluid(k) for k in kinds)
            if m1[i] > (1 + self.eps) * rho1[i] or (self.cleanup & 1 and no_gas):
                F.add(i)
            elif m1[i] < -self.eps * rho1[i] or (self.cleanup & 2 and no_fluid):
                E.add(i)
        # an empty cell next to a filled one stays interface
        dropped = {i for i in E if any(j is not None and j in F for j in nbrs[i])}
        if variant != "keep_empty":
            E -= dropped
        # gas neighbours of filled cells: new interface cells at the
        # equilibrium of the mean density and velocity of their liquid and
        # interface neighbours (flags of time t, populations of t+1), m = 0
        NG = sorted({j for i in F for j in nbrs[i] if j is not None and flags[j] == GAS})
        src = f if variant == "new_avg_precollision" else fn
        for j in NG:
            rs, us, cnt = Fr(0), [Fr(0)] * 3, 0
            for y in nbrs[j]:
                if y is None or not (fluid(flags[y]) or (variant == "new_avg_all" and y in NG and y < j)):
                    continue
                r, _, u = self.moments([src[q][y] for q in range(Q)])
                rs += r
                us = [us[a] + u[a] for a in range(3)]
                cnt += 1
            rbar = rs / cnt
            ubar = [v / cnt for v in us]
            for q in range(Q):
                fn[q][j] = self.e_plus(q, rbar, ubar) + self.e_minus(q, ubar)
            rho1[j] = sum(fn[q][j] for q in range(Q))
            m1[j] = Fr(0)
        # liquid neighbours of emptied cells: interface with m = rho
        NL = sorted({j for i in E for j in nbrs[i] if j is not None and flags[j] == LIQ})
        for j in NL:
            m1[j] = rho1[j]
        # excess (filled: m - rho, emptied: m), split equally over the
        # neighbours that are interface now and do not convert
        NGs, NLs = set(NG), set(NL)
        if variant == "recv_converting":
            recv = lambda j: j is not None and (j in NGs or j in NLs or flags[j] == IFC)
        else:
            recv = lambda j: j is not None and (j in NGs or j in NLs or (flags[j] == IFC and j not in F and j not in E))
        lost = Fr(0)
        share = {}
        for i in sorted(F | E):
            ex = m1[i] - rho1[i] if i in F else m1[i]
            nr = sum(1 for j in nbrs[i] if recv(j))
            if nr == 0:
                lost += ex
            else:
                share[i] = ex / nr
        receivers = [j for j in range(N) if recv(j)]
        add = {}
        for j in receivers:
            acc = sum((share[i] for i in nbrs[j] if i is not None and i in share), Fr(0))
            add[j] = acc
        for j, acc in add.items():
            m1[j] += acc
        flags1 = list(flags)
        phi1 = list(phi)
        for i in range(N):
            if i in F:
                flags1[i], m1[i] = LIQ, rho1[i]
            elif i in E:
                flags1[i], m1[i], phi1[i] = GAS, Fr(0), Fr(0)
            elif i in NGs or i in NLs:
                flags1[i] = IFC
        for i in range(N):
            if flags1[i] == IFC:
                phi1[i] = m1[i] / rho1[i]
            elif flags1[i] == LIQ:
                m1[i] = rho1[i]
        for i in range(N):
            if not fluid(flags1[i]):
                for q in range(Q):
                    fn[q][i] = Fr(0)
        events = dict(fill=len(F), empty=len(E), dropped=len(dropped), new_gas=len(NG), new_liq=len(NL),
                      lost_cells=sum(1 for i in F | E if i not in share), fsl_links=len(deltas))
        return flags1, fn, m1, phi1, lost, events


def total_mass(flags, m, lost):
    """M = sum_liquid rho + sum_interface m + lost (m = rho on liquid cells)."""
    return sum((m[i] for i in range(len(flags)) if flags[i] in (LIQ, IFC)), Fr(0)) + lost


def from_float(a):
    return [Fr(float(v)) for v in np.asarray(a, dtype=np.float64).reshape(-1)]

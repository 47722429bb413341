"""Host emulation of the index arithmetic of the two-cells-per-lane bulk
kernel (k_bulk_pairs) and of the segment scan's masks (k_segments), on the
lattices the GPU tests use: every population load and store stays inside the
[19][N] array and on its word boundary, the pulled (population, cell) of each
liquid cell on the pair path is the one the one-cell kernel pulls (Eq. lbe1
with half-way bounce-back beyond a non-periodic face), and the masks equal
the per-cell tests.  No GPU: the emulation restates the kernels' formulas."""
import numpy as np
import pytest

from paper_1409_5645_gb300 import cases

CX = [0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0]
CY = [0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1]
CZ = [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1]
LIQ, IFC, GAS, WALL, KIND, NEARB, NEARW = 1, 2, 4, 8, 15, 16, 32


def inv(q):
    return 0 if q == 0 else (q + 1 if q & 1 else q - 1)


def static_flags(c):
    """Cell kinds plus the static bits the library sets: NEARB (a neighbour is
    a wall: a WALL cell or beyond a non-periodic face), NEARW (a WALL cell)."""
    nx, ny, nz = c["dims"]
    px, py, pz = c["params"]["periodic"]
    fl = c["flags"].astype(np.uint8).reshape(nz, ny, nx).copy()
    kind = fl & KIND
    out = fl.copy()
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for q in range(1, 19):
        X, Y, Z = x + CX[q], y + CY[q], z + CZ[q]
        beyond = np.zeros_like(x, bool)
        for A, n, per in ((X, nx, px), (Y, ny, py), (Z, nz, pz)):
            if not per:
                beyond |= (A < 0) | (A >= n)
        wall = kind[Z % nz, Y % ny, X % nx] == WALL
        out[beyond] |= NEARB
        out[~beyond & wall] |= NEARB | NEARW
    return out.reshape(-1)


def fast_cell(fl, x, y, z, dims, periodic, wd_or_uw):
    nx, ny, nz = dims
    ax, ay, az = x in (0, nx - 1), y in (0, ny - 1), z in (0, nz - 1)
    if fl & KIND != LIQ:
        return False
    if wd_or_uw:
        return not (fl & NEARB) and not (ax or ay or az)
    return not (fl & NEARW) and not (ax and periodic[0]) and not (ay and periodic[1]) and not (az and periodic[2])


def byte_bits(w, s):
    return ((((w >> s) & 0x01010101) * 0x00204081) & 0xFFFFFFFF) >> 21 & 0xF


def segment_masks(b, x0, y, z, dims, periodic, wd_or_uw):
    """k_segments' masks of one segment from its flag bytes."""
    nx, ny, nz = dims
    n = len(b)
    liq = ifc = nb = nw = 0
    if n == 32 and nx % 16 == 0:
        w = np.frombuffer(b.tobytes(), dtype="<u4")
        for k in range(8):
            liq |= byte_bits(int(w[k]), 0) << 4 * k
            ifc |= byte_bits(int(w[k]), 1) << 4 * k
            nb |= byte_bits(int(w[k]), 4) << 4 * k
            nw |= byte_bits(int(w[k]), 5) << 4 * k
    else:
        for k in range(n):
            c = int(b[k])
            liq |= (c & 1) << k
            ifc |= (c >> 1 & 1) << k
            nb |= (c >> 4 & 1) << k
            nw |= (c >> 5 & 1) << k
    full = 0xFFFFFFFF if n == 32 else (1 << n) - 1
    xf = (1 if x0 == 0 else 0) | ((1 << (n - 1)) if x0 + n == nx else 0)
    yf, zf = y in (0, ny - 1), z in (0, nz - 1)
    if wd_or_uw:
        slow = liq & (nb | xf | (full if (yf or zf) else 0))
    else:
        slow = liq & (nw | (xf if periodic[0] else 0) | (full if ((yf and periodic[1]) or (zf and periodic[2])) else 0))
    return liq, ifc, slow


def check(c, wd_or_uw=False):
    nx, ny, nz = c["dims"]
    N = nx * ny * nz
    per = c["params"]["periodic"]
    fl = static_flags(c)
    assert nx % 2 == 0 and 19 * N < 2 ** 32
    pulls = 0
    for z in range(nz):
        for y in range(ny):
            for x0 in range(0, nx, 32):
                n = min(32, nx - x0)
                i0 = (z * ny + y) * nx + x0
                b = fl[i0:i0 + n]
                liq, ifc, slow = segment_masks(b, x0, y, z, (nx, ny, nz), per, wd_or_uw)
                for k in range(n):
                    kind = int(b[k]) & KIND
                    assert (liq >> k & 1) == (kind == LIQ) and (ifc >> k & 1) == (kind == IFC)
                    want = kind == LIQ and not fast_cell(int(b[k]), x0 + k, y, z, (nx, ny, nz), per, wd_or_uw)
                    assert (slow >> k & 1) == want
                if not (liq | ifc) or slow or not liq:
                    continue  # no pair path for this half-warp
                for hl in range(16):
                    if 2 * hl >= n:
                        continue
                    ia, xa = i0 + 2 * hl, x0 + 2 * hl
                    if not (liq >> 2 * hl & 3):
                        continue
                    for q in range(19):
                        bb = (CY[q] == 1 and y == 0) or (CY[q] == -1 and y == ny - 1) or \
                             (CZ[q] == 1 and z == 0) or (CZ[q] == -1 and z == nz - 1)
                        own_k = (inv(q) * N + ia) % 2 ** 32
                        src_k = (q * N + ia - CX[q] - nx * CY[q] - nx * ny * CZ[q]) % 2 ** 32
                        if CX[q] == 0:
                            k = own_k if bb else src_k
                            assert 0 <= k and k + 1 < 19 * N and k % 2 == 0
                            got = [(k // N, k % N), (k // N, k % N + 1)]
                        else:
                            bba = bb or (CX[q] == 1 and xa == 0)
                            bbb = bb or (CX[q] == -1 and xa + 2 == nx)
                            ka = own_k if bba else src_k
                            kb = own_k + 1 if bbb else src_k + 1
                            assert 0 <= ka < 19 * N and 0 <= kb < 19 * N
                            got = [(ka // N, ka % N), (kb // N, kb % N)]
                        for cc in range(2):
                            if not (liq >> (2 * hl + cc) & 1):
                                continue
                            x, i = xa + cc, ia + cc
                            beyond = (CX[q] == 1 and x == 0) or (CX[q] == -1 and x == nx - 1) or bb
                            want = (inv(q), i) if beyond else (q, i - CX[q] - nx * CY[q] - nx * ny * CZ[q])
                            assert got[cc] == want, (q, x, y, z, got[cc], want)
                            pulls += 1
                    # the word stores of the pair
                    for q in range(19):
                        k = q * N + ia
                        assert k % 2 == 0 and k + 1 < 19 * N
    return pulls


def test_dam_break_ragged_rows_all_faces():
    assert check(cases.dam_break(nx=70, ny=12, nz=20, col_x=33, col_z=15, tau=0.6, g=3e-4, rule=1)) > 50000


def test_dam_break_full_rows():
    assert check(cases.dam_break(nx=64, ny=10, nz=16, col_x=40, col_z=12, tau=0.6, g=2e-4, rule=1)) > 20000


@pytest.mark.parametrize("make,wd", [(lambda: cases.inclined_film(), True), (lambda: cases.plate_flow(), True)],
                         ids=["inclined_film_cli", "plate_flow_moving_wall"])
def test_wall_cases_take_the_general_path(make, wd):
    check(make(), wd_or_uw=wd)


def test_periodic_blob():
    n = 32
    N = n ** 3
    i = np.arange(N)
    x, y, z = i % n + 0.5, (i // n) % n + 0.5, i // (n * n) + 0.5
    phi = np.clip(9.3 - np.sqrt((x - 16.2) ** 2 + (y - 15.7) ** 2 + ((z - 16.1) / 0.8) ** 2) + 0.5, 0.0, 1.0)
    params = cases.default_params(tau=0.7, rule=1, periodic=(1, 1, 1))
    flags = cases.classify((n, n, n), params["periodic"], 0, phi)
    c = cases.Case(dims=(n, n, n), params=params, flags=flags, rho=np.ones(N), u=np.zeros((N, 3)), phi=phi,
                   noise=None, wall_delta=None)
    assert check(c) > 10000

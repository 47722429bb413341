"""Writes dam_break_128x64x64_oracle.txt: the FP64 oracle's own account of
the 128x64x64 dam break (the 512x256x256 throughput workload scaled by 1/4:
column x < 32, z < 48, tau 0.53, Lambda 0.005, g 1e-5, FSL) over 10 000
steps: total mass (liquid rho plus interface m plus the lost ledger) and the
ledger at the start and the end, and the cell counts at the end.  Calls only the oracle (the
OpenMP build of its source, whose results equal the single-thread build);
about 20 minutes on 8 cores.

    python tests/golden/make_dam_break_128_mass.py
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle.oracle import Oracle  # noqa: E402
from paper_1409_5645_gb300 import cases  # noqa: E402

STEPS = 10000
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "dam_break_128x64x64_oracle.txt")


def main():
    c = cases.dam_break(nx=128, ny=64, nz=64, col_x=32, col_z=48, tau=0.53, magic=0.005, rule=1)
    o = Oracle.from_case(c, omp=True)
    M0, L0 = o.total_mass()
    t0 = time.time()
    o.step(STEPS)
    M1, L1 = o.total_mass()
    fl = o.flags()
    conv, t = o.counters()
    lines = [
        "# FP64 oracle, dam break 128x64x64 (column x < 32, z < 48; tau 0.53, Lambda 0.005,",
        "# g = (0, 0, -1e-5), FSL, walls on every face), written by tests/golden/make_dam_break_128_mass.py",
        "# (oracle only).  mass = sum over liquid cells of rho + sum over interface cells of m + lost",
        "# (lost: the ledger of excess mass that found no receiver); mass is the conserved quantity.",
        f"steps {STEPS}",
        f"mass0 {M0!r}",
        f"lost0 {L0!r}",
        f"mass1 {M1!r}",
        f"lost1 {L1!r}",
        f"drift_rel {(M1 - M0) / M0!r}",
        f"liquid1 {int(np.count_nonzero(fl == cases.LIQUID))}",
        f"interface1 {int(np.count_nonzero(fl == cases.INTERFACE))}",
        f"conversions {' '.join(str(int(x)) for x in conv)}",
        f"seconds {time.time() - t0:.0f}",
    ]
    with open(OUT, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print("\n".join(lines))


if __name__ == "__main__":
    main()

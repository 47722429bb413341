"""The region-wise inverse of the plane/unit-cube volume used by the float
forms of the CUDA path (Sec. 2.2: the plane that cuts the cell's fill): its
root, put back into the oracle's volume function, returns the fill, for
random and degenerate normals (built for the host with nvcc, no GPU)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1409_5645_gb300", "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("plic") / "plic_regions")
    subprocess.run([nvcc, "-std=c++17", "-O2", "--expt-relaxed-constexpr", "-I", CSRC, "-I", INCLUDE,
                    os.path.join(HERE, "plic_regions_host.cu"), "-o", exe], check=True)
    return exe


def _cases():
    rng = np.random.default_rng(1409)
    rows = []
    normals = [np.sort(rng.random(3)) for _ in range(300)]
    normals += [np.array([0.0, 0.0, 1.0]), np.array([0.0, 0.3, 0.7]), np.array([0.0, 0.5, 0.5]),
                np.array([1 / 3, 1 / 3, 1 / 3]), np.array([0.1, 0.2, 0.7]), np.array([0.2, 0.3, 0.5]),
                np.array([1e-7, 0.4, 0.6]), np.array([0.25, 0.25, 0.5])]
    for m in normals:
        m = m / m.sum()
        for tv in list(rng.random(6) * 0.5) + [1e-9, 1e-6, 0.5, 0.25]:
            rows.append((max(tv, 1e-9), *m))
    return np.array(rows)


def test_root_reproduces_the_fill(driver):
    rows = _cases()
    text = "\n".join("%.17g %.17g %.17g %.17g" % tuple(r) for r in rows)
    out = subprocess.run([driver], input=text, capture_output=True, text=True, check=True).stdout.split()
    res = np.array(out, dtype=np.float64).reshape(-1, 2)
    worst_f = worst_d = 0.0
    for (tv, m1, m2, m3), (af, ad) in zip(rows, res):
        m = np.array([m1, m2, m3])
        vf = oracle.cube_volume(m, af - 0.5)
        vd = oracle.cube_volume(m, ad - 0.5)
        worst_f = max(worst_f, abs(vf - tv))
        worst_d = max(worst_d, abs(vd - tv))
        assert 0.0 <= af <= 0.5 + 1e-6 and 0.0 <= ad <= 0.5 + 1e-12
    print(f"|V(alpha) - fill|: float {worst_f:.2e}, double {worst_d:.2e}")
    assert worst_f < 2e-6
    assert worst_d < 1e-12

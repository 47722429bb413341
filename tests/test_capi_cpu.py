"""The C interface without a GPU: the header's declarations, the built
library's exported symbols, and the binding's refusal to run without it."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fslbm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fslbm_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def built_lib():
    from paper_1409_5645_gb300 import build
    return build.build()


def test_header_declares_the_step_api():
    names = declared_functions()
    for required in ("fslbm_create", "fslbm_create_ex", "fslbm_set_state", "fslbm_init_equilibrium",
                     "fslbm_step", "fslbm_get_fields", "fslbm_total_mass", "fslbm_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    lib = ctypes.CDLL(built_lib)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", built_lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (fslbm_[a-z_0-9]+)", out))
    assert set(declared_functions()) <= exported


def test_build_targets_sm103a_only():
    from paper_1409_5645_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_default_params_and_argument_checks(built_lib):
    from paper_1409_5645_gb300 import fslbm
    L = fslbm.lib()
    P = fslbm.Params()
    L.fslbm_default_params(ctypes.byref(P))
    assert P.tau == 0.8 and P.magic == pytest.approx(3 / 16) and P.rule == fslbm.FSL
    assert P.eps == 1e-3 and P.delta_min == 0.0 and P.precision == fslbm.F64
    h = ctypes.c_void_p()
    bad = fslbm.Params()
    L.fslbm_default_params(ctypes.byref(bad))
    bad.dims[0], bad.dims[1], bad.dims[2] = 4, 4, 0          # empty lattice
    assert L.fslbm_create_ex(ctypes.byref(bad), ctypes.byref(h)) == -1
    bad.dims[2] = 4
    bad.tau = 0.5                                            # tau must exceed 1/2
    assert L.fslbm_create_ex(ctypes.byref(bad), ctypes.byref(h)) == -1
    bad.tau = 1.0                                            # FSL cannot recover n^+ at tau = 1
    assert L.fslbm_create_ex(ctypes.byref(bad), ctypes.byref(h)) == -1
    bad.tau, bad.precision = 0.8, 7
    assert L.fslbm_create_ex(ctypes.byref(bad), ctypes.byref(h)) == -1
    bad.precision = fslbm.F64
    # options outside their ranges, each on its own (checked before any device work)
    for field, value in (("stress", 3), ("ub_extrap", 2), ("recon_nc", -1), ("excess_split", 2),
                         ("bulk_loads", 9), ("rule", 2), ("elvira", 2)):
        old = getattr(bad, field)
        setattr(bad, field, value)
        assert L.fslbm_create_ex(ctypes.byref(bad), ctypes.byref(h)) == -1, field
        setattr(bad, field, old)
    bad.compressible, bad.wall_u[0] = 1, 1e-3                # moving walls need rho_0 = 1
    assert L.fslbm_create_ex(ctypes.byref(bad), ctypes.byref(h)) == -1
    bad.compressible, bad.wall_u[0] = 0, 0.0
    L.fslbm_check_grid_barrier.argtypes = [ctypes.c_int, ctypes.c_void_p]
    assert L.fslbm_check_grid_barrier(2, None) == -1          # expire must be 0 or 1
    L.fslbm_launches_per_step.argtypes = [ctypes.c_void_p]
    assert L.fslbm_launches_per_step(None) == -1
    assert L.fslbm_build_info() == 0                        # the normal library, not the bounds-checked one
    assert L.fslbm_step(None, 1) == -1
    L.fslbm_last_error.restype = ctypes.c_char_p
    assert L.fslbm_last_error(None) == b"NULL handle"
    L.fslbm_destroy(None)


def test_checked_variant_is_a_separate_build():
    """build(checked=True) compiles the same sources with FSLBM_CHECKED into
    a library of its own, which the binding loads only when FSLBM_CHECKED=1."""
    from paper_1409_5645_gb300 import build, fslbm
    assert build.CHECKED_LIB != build.LIB and os.path.dirname(build.CHECKED_LIB) != os.path.dirname(build.LIB)
    if os.environ.get("FSLBM_CHECKED") != "1":
        assert fslbm.LIB_PATH == build.LIB
    src = open(os.path.join(ROOT, "paper_1409_5645_gb300", "csrc", "fslbm_dev.cuh")).read()
    # in the normal build every check macro is the bare expression
    normal = src.split("#ifdef FSLBM_CHECKED\n__device__")[1].split("#else")[1].split("#endif")[0]
    for line in normal.strip().splitlines():
        name, body = re.match(r"#define (FSL_[A-Z_]+)\((.*?)\) (.*)", line).group(1, 3)
        assert body in ("(k)", "true"), line


def test_binding_refuses_without_library(monkeypatch, tmp_path):
    from paper_1409_5645_gb300 import fslbm
    monkeypatch.setattr(fslbm, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(fslbm, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        fslbm.lib()


def _c_struct_fields(text, start, end):
    """Field names of a C struct body between two markers, in order."""
    body = text[text.index(start):]
    body = body[:body.index(end)]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    body = re.sub(r"//[^\n]*", "", body)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl or decl.startswith(("typedef", "struct")):
            continue
        # "int nx, ny, nz": the type goes with the first declarator only
        for part in decl.split(","):
            m = re.search(r"([A-Za-z_][A-Za-z0-9_]*)\s*(\[\d+\])?\s*$", part.strip())
            if m:
                names.append(m.group(1))
    return names


def test_ctypes_structs_follow_the_c_layouts():
    """The ctypes mirrors of fslbm_params (binding) and of the oracle's Params
    list the C fields in the same order (the structs cross the ABI by value)."""
    from oracle import oracle as orc
    from paper_1409_5645_gb300 import fslbm
    hdr = open(os.path.join(ROOT, "include", "fslbm.h")).read()
    c_lib = _c_struct_fields(hdr, "  int dims[3];", "} fslbm_params;")
    assert c_lib == [f[0] for f in fslbm.Params._fields_]
    src = open(os.path.join(ROOT, "oracle", "fslbm_oracle.cpp")).read()
    src = src[src.index("struct Params {") + len("struct Params {"):]
    c_orc = _c_struct_fields(src, "", "};")
    assert c_orc == [f[0] for f in orc.Params._fields_]


def test_viscosity_map_lives_in_the_library(built_lib):
    """tau = 3 nu + 1/2 (Sec. 2.1) is the library's own entry point; the
    autograd binding only marshals nu to it (no parameter arithmetic)."""
    from paper_1409_5645_gb300 import fslbm
    assert fslbm.tau_of_viscosity(0.1) == pytest.approx(0.8, abs=1e-15)
    assert fslbm.tau_of_viscosity(1.0 / 60.0) == pytest.approx(0.55, abs=1e-15)
    for bad in (0.0, -0.1, float("nan"), float("inf")):
        with pytest.raises(fslbm.FslbmError):
            fslbm.tau_of_viscosity(bad)
    src = open(os.path.join(ROOT, "paper_1409_5645_gb300", "autograd.py")).read()
    code = "\n".join(l.split("#")[0] for l in src.splitlines() if not l.strip().startswith(("\"", "'")))
    assert "tau_of_viscosity" in code
    assert not re.search(r"\d\s*\*\s*float\(nu\)|float\(nu\)\s*\*|\+\s*0\.5", code)

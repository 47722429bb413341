"""The bounds-checked build covers every cell index the kernels read from
memory: a source scan (no GPU) that each index taken from a cell list or a
segment record goes through one of the check macros, so that an index read
added later without a check fails here.  In the normal build the macros are
the bare expressions (test_capi_cpu.py); in the checked build they test the
index against the lattice before the access."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1409_5645_gb300", "csrc")


def sources():
    for name in sorted(os.listdir(CSRC)):
        if name.endswith((".cu", ".cuh")):
            with open(os.path.join(CSRC, name)) as fh:
                for k, line in enumerate(fh, 1):
                    yield name, k, line.split("//")[0]


def test_list_entries_are_checked():
    """A cell index assigned from a list entry (interface, fill, empty,
    new-cell, receiver lists; the adjoint's liquid and interface lists)."""
    read = re.compile(r"\blong long \w+ = (.*\b(?:\w*list|liq|ifc|ifc0|ifc1)\[.*);")
    seen = 0
    for name, k, line in sources():
        m = read.search(line)
        if m:
            seen += 1
            assert m.group(1).startswith("FSL_CK("), f"{name}:{k}: {line.strip()}"
    assert seen >= 17  # the step, conversion and adjoint kernels' list reads


def test_segment_record_cells_are_checked():
    """The first cell of a segment record (sd.w) becomes a cell index only
    through a check: directly, or through the row start of the staged kernels."""
    uses = 0
    for name, k, line in sources():
        if "sd.w" in line and "rowstart" not in line:
            uses += 1
            assert "FSL_CK_IF(" in line or "FSL_CK_WORD_IF(" in line, f"{name}:{k}: {line.strip()}"
        if re.search(r"\browstart \+ x\b", line):
            uses += 1
            assert "FSL_CK_IF(" in line, f"{name}:{k}: {line.strip()}"
    assert uses >= 5  # the one-cell, pair, TMA and cp.async bulk kernels


# source cells formed by offset arithmetic whose range rests on a coordinate
# test of the same function (or the interior precondition that the checked
# build tests with FSL_OK), and one that indexes no array
UNCHECKED_BY_CONSTRUCTION = {
    ("fslbm_pull.cuh", "const long long s = i - ("): "IN: every source inside (the caller's precondition)",
    ("fslbm_pull.cuh", "s = i - ("): "in1: the cell is one or more cells inside every face",
    ("fslbm_pull.cuh", "s = inside ? i - ("): "inside: the source's coordinates tested just above",
    ("fslbm_step.cuh", "const long long sq = IN ? i - ("): "IN: the interior precondition (FSL_OK in k_iface)",
    ("fslbm_step.cuh", "const long long su = IN ? i - ("): "IN: the interior precondition (FSL_OK in k_iface)",
    ("fslbm_staged.cu", "const long long e = (long long)q * (long long)N + i - ("): "selects a half-word (e & 1), no access",
}


def test_fast_path_offsets_are_checked():
    """A source cell formed as i minus a stencil offset on the bulk kernels'
    fast paths (whose range rests on the segment masks) goes through FSL_CK;
    the others are in range by a coordinate test next to them."""
    offset = re.compile(r"\bi - \(c(?:c)?x")
    checked = exempt = 0
    for name, k, line in sources():
        if not offset.search(line):
            continue
        if "FSL_CK(" in line:
            checked += 1
            continue
        stmt = line.strip()
        assert any(name == f and stmt.startswith(frag) for f, frag in UNCHECKED_BY_CONSTRUCTION), \
            f"{name}:{k}: {stmt}"
        exempt += 1
    assert checked >= 4 and exempt == len(UNCHECKED_BY_CONSTRUCTION)

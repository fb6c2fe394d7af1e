"""The C-ABI library loads on a machine without a GPU and exports every entry
point that include/*.h declares (no compute call is made here, except the
host-only contour routine, which is checked against the oracle)."""

import glob
import os
import re
import subprocess

import numpy as np

from conftest import ROOT


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(feast_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    import paper_0901_2665_gb300 as F
    declared = _declared()
    assert "feast_solve" in declared and "feast_init" in declared
    out = subprocess.run(["nm", "-D", "--defined-only", F.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (feast_\w+)", out))
    missing = declared - exported
    assert not missing, missing
    for name in declared:
        assert hasattr(F._lib, name)
    assert set(F.EXPORTED) == declared


def test_contour_entry_point_matches_oracle():
    import oracle
    import paper_0901_2665_gb300 as F
    for Ne in (3, 8, 16):
        x, w, theta, Z = F.feast_contour(1.5, 7.25, Ne)
        xo, wo, to, Zo, r = oracle.contour_points(1.5, 7.25, Ne)
        assert np.allclose(x, xo, atol=1e-15, rtol=0) and np.allclose(w, wo, atol=1e-15, rtol=0)
        assert np.allclose(Z, Zo, atol=1e-14, rtol=0)


def test_contour_rejects_bad_arguments():
    import paper_0901_2665_gb300 as F
    import pytest
    with pytest.raises(F.FeastError):
        F.feast_contour(2.0, 1.0, 8)
    with pytest.raises(F.FeastError):
        F.feast_contour(1.0, 2.0, 0)


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of feast_options and feast_info have the C layout
    (size and field offsets from a C program built against include/feast.h)."""
    import ctypes

    import paper_0901_2665_gb300 as F
    src = tmp_path / "sizes.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "feast.h"\n'
        'int main(void) {\n'
        '  printf("%zu %zu %zu %zu %zu\\n", sizeof(feast_options), sizeof(feast_info),\n'
        '         offsetof(feast_info, factor_flops), offsetof(feast_info, kernel_flops),\n'
        '         offsetof(feast_info, sweep_graphs));\n'
        '  return 0;\n}\n')
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(F.feast_options), ctypes.sizeof(F.feast_info), F.feast_info.factor_flops.offset,
            F.feast_info.kernel_flops.offset, F.feast_info.sweep_graphs.offset]
    assert got == want

"""CPU-side checks of the C-ABI library: it loads, exports every symbol the
header declares, and the binding refuses to run without a CUDA device."""
import os
import re
import subprocess

import pytest

import paper_2605_23088_b300 as yb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "yasps.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(yasps_[a-z_0-9]+)\s*\(", src)))


def test_header_matches_binding_list():
    assert declared() == sorted(yb.EXPORTS)


def test_library_exports_every_declared_symbol():
    L = yb.lib()
    for name in declared():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", yb.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (yasps_\w+)", out))
    assert set(declared()) <= exported


def test_default_params():
    p = yb.default_params(dt=0.005)
    assert p.dt == 0.005 and p.dhat == 1e-3 and p.precision == 0 and p.ccd_gap == 0.1
    assert list(p.gravity) == [0.0, -9.81, 0.0]


def test_no_cpu_fallback():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    import scenes
    with pytest.raises(RuntimeError):
        yb.System(scenes.cubes_scene(n=1))

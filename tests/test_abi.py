"""CPU checks of the C ABI: the library builds, loads and exports every
function declared in the headers under include/; host-only entry points
validate descriptors.  No compute call is made (no GPU here)."""

import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


def _declared():
    names = set()
    for path in HEADERS:
        text = open(path).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(selm_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1003_2680_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(lib, n)]
    assert missing == []


def test_binding_covers_header():
    from paper_1003_2680_gb300 import selm
    assert sorted(selm._SIGS) == _declared()


def _desc(**kw):
    from paper_1003_2680_gb300 import selm
    return selm.make_desc(torch_allocator=False, **kw)


def test_footprint_host_only():
    from paper_1003_2680_gb300 import selm
    f64 = selm.selm_mg_footprint(_desc(dim=2, n=64, levels=6))
    f32 = selm.selm_mg_footprint(_desc(dim=3, n=128, precision=selm.SELM_FP32_REFINE64))
    fproj = selm.selm_mg_footprint(_desc(dim=3, n=128, precision=selm.SELM_FP32_REFINE64,
                                         projection=selm.SELM_PROJ_MAC))
    assert 0 < f64 < f32 < fproj
    # 128^3: three level-0 inner fields (FP32) + four FP64 fields, plus coarse levels
    nv = 2 * 128 ** 3 + 127 * 128 ** 2
    assert f32 >= nv * (3 * 4 + 4 * 8)
    assert f32 < nv * (3 * 4 * 8 / 7 + 4 * 8) + (64 << 20)
    # with the projection, the chain keeps its own copy of the velocity level fields
    assert fproj >= f32 + nv * 3 * 4


@pytest.mark.parametrize("bad", [dict(dim=4, n=64), dict(dim=3, n=6, levels=3), dict(dim=2, n=64, mu=-1.0),
                                 dict(dim=3, n=64, precision=7), dict(dim=3, n=96, levels=7)])
def test_invalid_descriptors_rejected(bad):
    from paper_1003_2680_gb300 import selm
    assert selm.selm_mg_footprint(_desc(**bad)) == 0
    h = ctypes.c_void_p()
    d = _desc(**bad)
    st = selm.lib().selm_mg_create(ctypes.byref(d), None, ctypes.byref(h))
    assert st == selm.SELM_EINVAL and not h.value

"""The allocation-free V-cycle entry point against the handle-based one.

selm_mg_vcycle_static serves callers that cannot allocate device memory --
for instance a service with a fixed, pre-planned memory budget that forbids
allocation while it runs, or a thread that cannot reach the allocator of the
framework owning the device.  It keeps its scratch in a fixed array inside the
library instead of asking for memory, so its results must match
selm_mg_vcycle (which runs on a handle's allocated workspace, and is itself
compared with the oracle) on the same inputs, call after call.
"""

import pytest
import torch

import selm_inputs
from tests.gpu_util import comps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_2680_gb300 import selm as mod
    mod.lib()
    return mod


def _flat(h, shapes_seed, dtype):
    lay, size = comps(h)
    fields = selm_inputs.fields([shape for shape, _ in lay], seed=shapes_seed)
    import numpy as np
    flat = np.concatenate([f.ravel() for f in fields])
    assert flat.size == size
    return torch.tensor(flat, dtype=dtype, device="cuda")


CASES = [(p, tol, dim, n, levels) for p, tol in ((1, 1e-5), (0, 1e-12))
         for dim, n, levels in ((3, 32, 4), (3, 48, 4), (2, 128, 6))]
CASES.append((1, 1e-5, 3, 80, 5))   # near the array's limit in FP32


@pytest.mark.parametrize("precision,tol,dim,n,levels", CASES)
def test_static_vcycle_matches_handle_vcycle(S, precision, tol, dim, n, levels):
    m = S.SelmMG(dim=dim, n=n, levels=levels, precision=precision, seed=5, instance=2)
    desc = S.make_desc(dim=dim, n=n, levels=levels, precision=precision, seed=5, instance=2,
                       torch_allocator=False)
    dt = m.inner_dtype()
    b = _flat(m.h, 61, dt)
    v0 = _flat(m.h, 62, dt)
    # two calls in a row: the second runs on the array the first one left behind
    for cycle, noise in ((7, 1), (8, 0)):
        v_ref = v0.clone()
        S.selm_mg_vcycle(m.h, 0, v_ref, b, cycle, noise)
        v_static = v0.clone()
        S.selm_mg_vcycle_static(desc, v_static, b, cycle, noise)
        torch.cuda.synchronize()
        err = ((v_static - v_ref).double().norm() / v_ref.double().norm()).item()
        assert err < tol, (cycle, noise, err)
    m.close()


def test_static_vcycle_rejects_grids_beyond_its_array(S):
    desc = S.make_desc(dim=3, n=256, precision=1, torch_allocator=False)
    v = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(S.SelmError) as info:
        S.selm_mg_vcycle_static(desc, v, v, 0, 0)
    assert info.value.status == S.SELM_EINVAL

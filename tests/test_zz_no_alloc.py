"""lbm_diagnostics_state_noalloc: the diagnostics reduction for callers that
cannot let the library allocate device memory (their own pool owns all of
it, or their loop must not be serialised by an allocation). It reduces a
state field the caller owns, keeping its block partials in a fixed array in
the library's device memory.

Checked through the C ABI against lbm_diagnostics (the allocating path that
reads the populations) on the same state, with the FP64 tolerance of the
other diagnostics test, on two calls in a row (the second call reuses the
array the first one filled)."""
import ctypes as C

import numpy as np
import pytest

from tests.cases import smooth_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch

    assert torch.cuda.is_available()
    from paper_2605_26677_gb300 import build

    build.build()
    from paper_2605_26677_gb300 import lbm as m

    return m


LAWS = {"NH": (1, [1.5, 0.75]), "MR": (3, [1.5, 0.25, 0.125]), "GENT": (5, [1.5, 0.75, 10.0])}


@pytest.mark.parametrize("law", sorted(LAWS))
@pytest.mark.parametrize("storage", [0, 1])
def test_noalloc_diagnostics_match_existing_entry_point(lbm, storage, law):
    import torch

    nx, ny = 301, 157  # several reduction blocks and a ragged last block
    L = lbm.Lattice(nx, ny, storage=storage, omega=1.9)
    law_id, prm = LAWS[law]
    lbm.lbm_set_material(L.ctx, law_id, prm)
    lbm.lbm_set_boundary(L.ctx, 0, lbm.LBM_BC_VELOCITY)
    lbm.lbm_set_boundary(L.ctx, 1, lbm.LBM_BC_TRACTION, (0.02, 0.01))
    lbm.lbm_init(L.ctx, smooth_field(nx, ny, seed=41, amp=0.05, periodic=False))
    lbm.lbm_step(L.ctx, 30)
    expect = lbm.lbm_diagnostics(L.ctx)
    U = torch.empty((6, ny, nx), dtype=torch.float64, device="cuda")
    lbm.lbm_read_state_device(L.ctx, U)
    lbm.lbm_sync(L.ctx)
    dev = torch.cuda.current_device()
    for _ in range(2):
        out = torch.full((10,), float("nan"), dtype=torch.float64, device="cuda")
        lbm.lbm_diagnostics_state_noalloc(U, nx, ny, law_id, prm, 1.0, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.allclose(got, expect, rtol=1e-11, atol=1e-13), (got, expect)
        # the call leaves the calling thread's current device as it was
        assert torch.cuda.current_device() == dev
    L.close()


def test_noalloc_rejects_grids_beyond_its_scratch(lbm):
    import torch

    U = torch.zeros(6, dtype=torch.float64, device="cuda")
    out = torch.zeros(10, dtype=torch.float64, device="cuda")
    prm = (C.c_double * 2)(1.0, 0.5)
    # 8193 x 8192 nodes is one row more than the array holds; the call must
    # refuse before touching the device
    st = lbm.library().lbm_diagnostics_state_noalloc(
        C.c_void_p(U.data_ptr()), 8193, 8192, lbm.LBM_LAW_NH, prm, 2, 1.0, C.c_void_p(out.data_ptr()), 0, None)
    assert st == lbm.LBM_ERR_ARG
    assert "exceeds the static scratch capacity" in lbm.lbm_last_error(None)
    assert torch.count_nonzero(out).item() == 0

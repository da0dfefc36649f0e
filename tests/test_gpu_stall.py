"""Failure detection of the staged 16-bit step kernel's bounded wait, without
a GPU fault: LBM_STEP16_STALL_TEST=1 makes the first staged launch of the
process expect 16 bytes more than its copies deliver for one task, so that
warp's stage never completes (no copy is left in flight: all of them land).
Its wait gives up after about a second, the kernel latches the status bit
and returns, and the host reports LBM_ERR_CUDA from the step call. The
context stays usable: a new initialization and later steps run normally and
match a run that never stalled. Runs in child processes because the
environment is read once per process.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def child(out_path, stall):
    """A 300 x 40 BF16 lattice with the staged kernel: (stall) one step that
    must report LBM_ERR_CUDA, then init and 50 steps; saves the final state."""
    import time

    from paper_2605_26677_gb300 import lbm
    from tests.cases import smooth_field

    nx, ny = 300, 40
    U0 = smooth_field(nx, ny, seed=5, periodic=True)
    L = lbm.Lattice(nx, ny, c=5.0, omega=1.9, storage=lbm.LBM_STORE_BF16)
    lbm.lbm_set_material(L.ctx, lbm.LBM_LAW_NH, [1.5, 0.75])
    err, secs = None, 0.0
    if stall:
        lbm.lbm_init(L.ctx, U0)
        t0 = time.time()
        try:
            lbm.lbm_step(L.ctx, 1)
        except lbm.LbmError as e:
            err = (e.status, str(e))
        secs = time.time() - t0
    lbm.lbm_init(L.ctx, U0)
    lbm.lbm_step(L.ctx, 50)
    U, _, _ = lbm.lbm_read_state(L.ctx)
    L.close()
    np.savez(out_path, U=U, status=-1 if err is None else err[0], secs=secs,
             msg="" if err is None else err[1])


def run(tmp_path, stall):
    out = str(tmp_path / ("stall%d.npz" % stall))
    env = dict(os.environ, LBM_STEP16="staged")
    env.pop("LBM_STEP16_STALL_TEST", None)
    if stall:
        env["LBM_STEP16_STALL_TEST"] = "1"
    code = "import sys; sys.path.insert(0, %r); import tests.test_gpu_stall as m; m.child(%r, %d)" % (ROOT, out, stall)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return dict(np.load(out))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2605_26677_gb300 import build

    build.build()


def test_bounded_wait_reports_and_context_recovers(tmp_path):
    from paper_2605_26677_gb300 import lbm

    got = run(tmp_path, 1)
    ref = run(tmp_path, 0)
    assert int(got["status"]) == lbm.LBM_ERR_CUDA, str(got["msg"])
    assert "time bound" in str(got["msg"])
    assert 0.5 < float(got["secs"]) < 30.0, float(got["secs"])
    assert np.array_equal(got["U"].view(np.uint64), ref["U"].view(np.uint64))

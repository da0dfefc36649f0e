"""The 16-bit step kernels against each other: the register kernel
(LBM_STEP16=regs in the environment) and the staged kernel (rows moved into
shared memory by bulk asynchronous copies; LBM_STEP16=staged) run the same
tasks through the same per-node arithmetic, so after any number of steps
their states, displacements and diagnostics agree bit for bit; so does the
default, where the first lbm_step times both kernels on the lattice with
trial steps that must leave the state untouched, and keeps the faster. The
choice is read once per process, so each variant runs in a child process
over the same cases; agreement with the oracle is the 16-bit part of
test_gpu_parity, which runs the default.

Cases: ragged widths (1000 = 7 segments of 128 and a tail of 104; 131 = one
segment and a tail of 3), every edge rule with the fused ghost writes, the
extrapolated F^b form (step kernel without fused ghosts), periodic
directions, and the 1 x 1 and 5 x 2 degenerate lattices.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BF16, F16 = 2, 3

CASES = [
    # (name, nx, ny, edge set, fb_mode, storage, steps)
    ("clamped_mixed_bf16", 131, 37, "clamped_mixed", 0, BF16, 200),
    ("x_periodic_f16", 131, 37, "x_periodic", 0, F16, 150),
    ("all_traction_extrap_bf16", 300, 9, "all_traction", 1, BF16, 120),
    ("all_velocity_wide_bf16", 1000, 5, "all_velocity", 0, BF16, 80),
    ("y_periodic_f16", 5, 2, "y_periodic", 0, F16, 60),
    ("periodic_1x1_bf16", 1, 1, "periodic", 0, BF16, 60),
]


def child(out_path):
    """Runs every case with the kernel this process selected; saves all
    outputs to out_path (npz)."""
    from tests.cases import Case, run_gpu, smooth_field
    from tests.test_gpu_parity import edge_sets

    res = {}
    for name, nx, ny, edges, fb, storage, steps in CASES:
        E = {} if edges == "periodic" else edge_sets(nx, ny)[edges]
        U0 = smooth_field(nx, ny, seed=29, periodic=("periodic" in edges))
        case = Case(nx, ny, steps, lam=1.5, mu=0.75, omega=1.9, body=(2e-4, -1e-4), edges=E, U0=U0, fb_mode=fb)
        g = run_gpu(case, storage)
        for k in ("U", "P", "u", "sigma", "diag"):
            res[name + "/" + k] = np.asarray(g[k], dtype=np.float64)
    np.savez(out_path, **res)


def run_variant(tmp_path, variant):
    out = str(tmp_path / ("%s.npz" % (variant or "default")))
    env = dict(os.environ)
    env.pop("LBM_STEP16", None)
    if variant:
        env["LBM_STEP16"] = variant
    code = "import sys; sys.path.insert(0, %r); import tests.test_gpu_step16_kernels as m; m.child(%r)" % (ROOT, out)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return dict(np.load(out))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2605_26677_gb300 import build

    build.build()


def test_staged_and_register_kernels_bit_identical(tmp_path):
    ref = run_variant(tmp_path, "regs")
    for variant in ("staged", None):
        got = run_variant(tmp_path, variant)
        assert set(got) == set(ref)
        for k in ref:
            assert np.all(np.isfinite(ref[k])), k
            same = np.array_equal(got[k].view(np.uint64), ref[k].view(np.uint64))
            assert same, (variant, k, float(np.max(np.abs(got[k] - ref[k]))))

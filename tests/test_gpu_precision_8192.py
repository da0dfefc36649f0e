"""Storage precision at full size: the 8192^2 periodic workload (16-mode
random velocity, seed 1, NH lambda = 1.5, mu = 0.75, c = 5, omega = 2, F = I)
advanced 5000 steps with FP32, FP16 and BF16 population storage, each
compared with the FP64-storage run of the same field, on the centred
512 x 512 crop and over the whole field.

The FP64 storage mode stands in for the oracle here: the oracle cannot run
67 M nodes for 5000 steps inside a test, and the FP64 mode is held to it at
1e-11 per group on every edge rule, closure and size (test_gpu_parity). The
crop compares a window of the full run; it is not run on its own, since
after 5000 steps its domain of dependence spans far more than 512 nodes.

Bounds: those of test_gpu_parity for the same step count: FP32 1e-5 per
group (2e-5 for u) and 1e-6 on U; FP16 / BF16 the rounding model
1.5 * 2^-p * sqrt(n) * s_g with s_g from the FP64-storage state over the
same window (tests.cases.rounding_scales). The measured errors are printed
for the record.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

F64, F32, BF16, F16 = 0, 1, 2, 3
STEPS = 5000
CROP = 512


def tol_for(storage, steps, ref, sl, w):
    from tests.test_gpu_parity import tol_for as parity_tol

    Uo, Po, _ = ref
    return parity_tol(storage, steps, {"U": Uo[sl], "P": Po[sl]}, w.c, w.lam + 2.0 * w.mu)


def run(lbm, torch, w, U0, storage):
    """Runs the workload and returns its state U (6 x N), P (4 x N) and
    displacement u (2 x N) as FP64 device tensors."""
    L = lbm.Lattice(w.nx, w.ny, dx=w.dx, c=w.c, omega=w.omega, storage=storage)
    try:
        lbm.lbm_set_material(L.ctx, lbm.LBM_LAW_NH, [w.lam, w.mu])
        lbm.lbm_init_device(L.ctx, U0)
        lbm.lbm_step(L.ctx, STEPS)
        N = w.nx * w.ny
        U = torch.empty(6 * N, dtype=torch.float64, device="cuda")
        P = torch.empty(4 * N, dtype=torch.float64, device="cuda")
        u = torch.empty(2 * N, dtype=torch.float64, device="cuda")
        lbm.lbm_read_state_device(L.ctx, U, P)
        lbm.lbm_read_displacement_device(L.ctx, u)
        torch.cuda.synchronize()
    finally:
        L.close()
    return U.view(6, w.ny, w.nx), P.view(4, w.ny, w.nx), u.view(2, w.ny, w.nx)


def rel(a, b):
    return float(((a - b).norm() / b.norm()).item())


def groups(g, o, sl):
    """Relative L2 per group (v, F - I, P, u, full state U) over the window sl."""
    (Ug, Pg, ug), (Uo, Po, uo) = g, o
    eye = Uo.new_tensor([1.0, 0.0, 0.0, 1.0]).view(4, 1, 1)
    return {
        "v": rel(Ug[:2][sl], Uo[:2][sl]),
        "F-I": rel(Ug[2:][sl] - eye, Uo[2:][sl] - eye),
        "P": rel(Pg[sl], Po[sl]),
        "u": rel(ug[sl], uo[sl]),
        "U": rel(Ug[sl], Uo[sl]),
    }


def test_precision_8192_crop_against_fp64_storage():
    import torch

    from paper_2605_26677_gb300 import build

    build.build()
    from paper_2605_26677_gb300 import lbm
    from synth import fourier_periodic

    w = fourier_periodic()
    assert (w.nx, w.ny) == (8192, 8192)
    U0h, _ = w.fields()
    U0 = torch.from_numpy(np.ascontiguousarray(U0h)).cuda()
    del U0h
    ref = run(lbm, torch, w, U0, F64)
    c0 = (w.nx - CROP) // 2
    crop = (slice(None), slice(c0, c0 + CROP), slice(c0, c0 + CROP))
    whole = (slice(None), slice(None), slice(None))
    for storage, name in ((F32, "FP32"), (F16, "FP16"), (BF16, "BF16")):
        got = run(lbm, torch, w, U0, storage)
        ec, ew = groups(got, ref, crop), groups(got, ref, whole)
        del got
        print("precision 8192^2 x %d %s crop512 %s whole %s" % (
            STEPS, name, {k: "%.2e" % v for k, v in ec.items()}, {k: "%.2e" % v for k, v in ew.items()}))
        for errs, sl in ((ec, crop), (ew, whole)):
            tol = tol_for(storage, STEPS, ref, sl, w)
            for k in ("v", "F-I", "P", "u", "U"):
                assert errs[k] <= tol[k], (name, k, tol[k], errs)

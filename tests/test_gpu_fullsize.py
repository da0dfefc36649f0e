"""Checks at the full sizes of the benchmark workloads, in the launch
configuration bench.py times (same library calls, same grid):

- 4096 x 2048 clamped specimen: after K steps a node depends only on nodes
  within K lattice spacings (one pull per step; the node-form traction rule
  reads only the boundary node), so patches at the corners, edge midpoints and
  centre must equal the same patches of a 160 x 96 specimen with the same edges
  run by the oracle;
- the rest state stays exact at full size;
- 8192^2 periodic: shifting the initial field by whole nodes shifts the
  result (the same arithmetic runs at every node), and sum U is conserved.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch

    assert torch.cuda.is_available()
    from paper_2605_26677_gb300 import build

    build.build()
    from paper_2605_26677_gb300 import lbm as m

    return m


def specimen(lbm, w, storage):
    from bench import setup_ctx

    return setup_ctx(lbm, w, storage, None, None)


def fast_specimen(nx, ny):
    from synth import clamped_specimen

    w = clamped_specimen(nx=nx, ny=ny)
    # a short ramp so that K steps already load the edge noticeably
    w.edges[1].tparams = (10 * 0.2, 0, 0, 0)
    return w


@pytest.mark.parametrize("storage", [0, 1])
def test_clamped_specimen_full_size_patches(lbm, storage):
    from oracle import oracle as orc
    from synth import rest_state

    K, R = 32, 8
    big = fast_specimen(4096, 2048)
    L = specimen(lbm, big, storage)
    lbm.lbm_init(L.ctx, rest_state(big.nx, big.ny))
    lbm.lbm_step(L.ctx, K)
    Ub, Pb, _ = lbm.lbm_read_state(L.ctx)
    ub = lbm.lbm_read_displacement(L.ctx)
    L.close()

    small = fast_specimen(160, 96)
    O = orc.Lattice(small.nx, small.ny, small.dx, small.c, small.omega)
    O.set_law(orc.NH, [small.lam, small.mu])
    O.set_body_force(*small.body_force)
    kinds = {"velocity": orc.VELOCITY, "traction": orc.TRACTION}
    for e, ed in enumerate(small.edges):
        O.set_edge(e, kinds[ed.kind], ed.value, 2 if ed.timefn == "sin2_ramp" else 0, ed.tparams)
    O.init(rest_state(small.nx, small.ny))
    O.step(K)
    Uo, Po, _ = O.state()
    uo = O.displacement()

    def spans(n_big, n_small):
        # (big start, small start) of patches at the low end, the middle and the high end
        return [(0, 0), (n_big // 2 - R, n_small // 2 - R), (n_big - 2 * R, n_small - 2 * R)]

    tol = 1e-12 if storage == 0 else 1e-4
    FI = np.array([1.0, 0.0, 0.0, 1.0])[:, None, None]
    checked = 0
    for bx, sx in spans(big.nx, small.nx):
        for by, sy in spans(big.ny, small.ny):
            gb = (slice(by, by + 2 * R), slice(bx, bx + 2 * R))
            gs = (slice(sy, sy + 2 * R), slice(sx, sx + 2 * R))
            for a, b in ((Ub[:2], Uo[:2]), (Ub[2:] - FI, Uo[2:] - FI), (Pb, Po), (ub, uo)):
                pa, pb = a[(slice(None),) + gb], b[(slice(None),) + gs]
                # the oracle evaluates P from the full F (about 1), so near the
                # rest state its own rounding is ~1e-16 absolute: compare on a
                # scale of at least 1e-3
                scale = max(np.abs(pb).max(), 1e-3)
                assert np.abs(pa - pb).max() <= tol * scale * 10, (bx, by, np.abs(pa - pb).max(), scale)
            checked += 1
    assert checked == 9
    # the loaded edge has moved, the far interior only feels the body force
    assert np.abs(Uo[0][:, -1]).max() > 1e-4


def test_rest_state_full_size_is_exact(lbm):
    from synth import clamped_specimen, rest_state

    w = clamped_specimen()
    w.body_force = (0.0, 0.0)
    for ed in w.edges:
        ed.value = (0.0, 0.0)
    L = specimen(lbm, w, 1)
    lbm.lbm_init(L.ctx, rest_state(w.nx, w.ny))
    lbm.lbm_step(L.ctx, 20)
    d = lbm.lbm_diagnostics(L.ctx)
    L.close()
    assert d[0] == 0.0 and d[1] == 0.0 and d[7] == 1.0 and d[8] == 1.0 and d[9] == 0.0


def test_periodic_8192_shift_equivariance(lbm):
    import torch

    from synth import fourier_periodic

    w = fourier_periodic()
    U0, u0 = w.fields()
    sx, sy, K = 37, 11, 8
    outs = []
    for shift in ((0, 0), (sy, sx)):
        U = np.ascontiguousarray(np.roll(U0, shift, axis=(1, 2)))
        L = specimen(lbm, w, 1)
        lbm.lbm_init(L.ctx, U, None, 2)
        lbm.lbm_step(L.ctx, K)
        d = torch.empty((6, w.ny, w.nx), dtype=torch.float64, device="cuda")
        lbm.lbm_read_state_device(L.ctx, d)
        lbm.lbm_sync(L.ctx)
        L.close()
        outs.append(d)
    back = torch.roll(outs[1], shifts=(-sy, -sx), dims=(1, 2))
    assert torch.equal(back, outs[0])


def test_periodic_8192_conservation_fp64(lbm):
    from synth import fourier_periodic

    w = fourier_periodic()
    U0, u0 = w.fields()
    L = specimen(lbm, w, 0)
    lbm.lbm_init(L.ctx, U0, None, 2)
    d0 = lbm.lbm_diagnostics(L.ctx)
    lbm.lbm_step(L.ctx, 20)
    d1 = lbm.lbm_diagnostics(L.ctx)
    L.close()
    N = w.nx * w.ny
    assert abs(d1[0] - d0[0]) < 1e-12 * N and abs(d1[1] - d0[1]) < 1e-12 * N
    assert np.allclose(d1[2:6], d0[2:6], rtol=0, atol=1e-13)

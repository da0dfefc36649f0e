"""Pins of the oracle's shear-modulus field and its reference adjoint.

The adjoint is checked against what does not involve it: central finite
differences of the oracle's own FP64 forward loss along random directions of
mu and v0 (a dropped term, a wrong sign, a transposed index or a missing
edge contribution moves the directional derivative by far more than the
1e-6 bound), on a bounded specimen with velocity and traction edges (the
Newton solve of Sec. 3.6.2 enters through the implicit function theorem) and
on a periodic one (wrapped streaming); plus exact special cases."""
import numpy as np
import pytest

from oracle import oracle as orc
from synth import splitmix64_uniform


def fields(nx, ny, seed):
    r = splitmix64_uniform(seed, 3 * nx * ny)
    mu = 0.5 + 0.5 * r[: nx * ny].reshape(ny, nx)
    U0 = np.zeros((6, ny, nx))
    U0[2] = U0[5] = 1.0
    X = (np.arange(nx) + 0.5) / nx
    Y = (np.arange(ny) + 0.5) / ny
    U0[0] = 0.02 * np.sin(np.pi * X)[None, :] * np.sin(np.pi * Y)[:, None] + \
        0.005 * (r[nx * ny: 2 * nx * ny].reshape(ny, nx) - 0.5)
    U0[1] = 0.01 * np.cos(2 * np.pi * Y)[:, None] * np.ones(nx)[None, :]
    return mu, U0, r[2 * nx * ny:]


def lattice(nx, ny, bounded, omega=1.9):
    O = orc.Lattice(nx, ny, 1.0, 5.0, omega)
    O.set_law(orc.NH, [1.0, 0.5])
    if bounded:
        O.set_edge(orc.LEFT, orc.VELOCITY)
        O.set_edge(orc.RIGHT, orc.TRACTION, (0.002, 0.001))
        O.set_edge(orc.BOTTOM, orc.TRACTION)
        O.set_edge(orc.TOP, orc.TRACTION)
    return O


def forward_loss(nx, ny, bounded, mu, lam_ratio, U0, sens, rec, target, order=2):
    O = lattice(nx, ny, bounded)
    O.set_material_field(mu, lam_ratio)
    O.init(U0, None, order)
    tot, n = 0.0, 0
    for k, nk in enumerate(rec):
        O.step(nk - n)
        n = nk
        u = O.displacement()
        for s, node in enumerate(sens):
            iy, ix = divmod(int(node), nx)
            d = u[:, iy, ix] - target[k, s]
            tot += 0.5 * float(d @ d)
    return tot


@pytest.mark.parametrize("bounded", [True, False])
def test_adjoint_matches_central_differences(bounded):
    nx, ny, steps, lam_ratio = 14, 10, 60, 2.0
    mu, U0, r = fields(nx, ny, 11)
    sens = np.array([iy * nx + nx - 1 for iy in range(0, ny, 2)])
    rec = np.array([10, 30, 45, 60])
    target = 0.001 * (r[: len(rec) * len(sens) * 2].reshape(len(rec), len(sens), 2) - 0.5)
    O = lattice(nx, ny, bounded)
    O.set_material_field(mu, lam_ratio)
    L, gmu, gv0 = O.adjoint(U0, steps, sens, rec, target)
    assert L == pytest.approx(forward_loss(nx, ny, bounded, mu, lam_ratio, U0, sens, rec, target), rel=1e-14)
    rng = np.random.default_rng(0)
    h = 1e-5
    for _ in range(4):
        dmu = rng.standard_normal((ny, nx))
        dv = np.zeros_like(U0)
        dv[:2] = rng.standard_normal((2, ny, nx))
        fd_mu = (forward_loss(nx, ny, bounded, mu + h * dmu, lam_ratio, U0, sens, rec, target) -
                 forward_loss(nx, ny, bounded, mu - h * dmu, lam_ratio, U0, sens, rec, target)) / (2 * h)
        fd_v = (forward_loss(nx, ny, bounded, mu, lam_ratio, U0 + h * dv, sens, rec, target) -
                forward_loss(nx, ny, bounded, mu, lam_ratio, U0 - h * dv, sens, rec, target)) / (2 * h)
        ad_mu = float((gmu * dmu).sum())
        ad_v = float((gv0 * dv[:2]).sum())
        assert abs(ad_mu - fd_mu) <= 1e-6 * abs(fd_mu), (ad_mu, fd_mu)
        assert abs(ad_v - fd_v) <= 1e-6 * abs(fd_v), (ad_v, fd_v)


def test_uniform_field_equals_uniform_parameters():
    nx, ny = 12, 9
    _, U0, _ = fields(nx, ny, 3)
    A = lattice(nx, ny, True)
    A.set_law(orc.NH, [1.4, 0.7])
    A.init(U0)
    A.step(40)
    B = lattice(nx, ny, True)
    B.set_material_field(np.full((ny, nx), 0.7), 2.0)
    B.init(U0)
    B.step(40)
    assert np.array_equal(A.state()[0], B.state()[0])
    assert np.array_equal(A.displacement(), B.displacement())


def test_displacement_at_step_zero_does_not_depend_on_v0():
    # order-0 init: f^0 = f^eq(U0) sums to U0, so u^0 = u*^0 + (dt/2) v^0 =
    # -(dt/2) v0 + (dt/2)(v0 + (dt/2) b) does not involve v0 or mu
    nx, ny = 8, 6
    mu, U0, _ = fields(nx, ny, 5)
    O = lattice(nx, ny, True)
    O.set_body_force(0.0, -1e-3)
    O.set_material_field(mu, 1.5)
    sens = np.arange(nx * ny)
    L, gmu, gv0 = O.adjoint(U0, 0, sens, [0], np.full((1, nx * ny, 2), 0.3), order=0)
    assert np.all(gv0 == 0.0) and np.all(gmu == 0.0)
    dt = O.dt
    u0 = np.array([0.0, 0.5 * dt * 0.5 * dt * -1e-3])
    assert L == pytest.approx(0.5 * nx * ny * float(((u0 - 0.3) ** 2).sum()), rel=1e-14)


def test_adjoint_rejects_missing_field_and_extrapolated_form():
    nx, ny = 8, 6
    mu, U0, _ = fields(nx, ny, 5)
    O = lattice(nx, ny, True)
    with pytest.raises(RuntimeError):
        O.adjoint(U0, 3, [0], [3], np.zeros((1, 1, 2)))
    O.set_material_field(mu, 2.0)
    O.set_fb_mode(orc.FB_EXTRAP2)
    with pytest.raises(RuntimeError):
        O.adjoint(U0, 3, [0], [3], np.zeros((1, 1, 2)))

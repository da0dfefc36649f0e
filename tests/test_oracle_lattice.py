"""Lattice-level pins of the oracle that follow from the scheme itself
(Sec. 3.3, 3.4, 3.6 and Appendix B), each independent of the oracle's code:
exact stationarity of uniform equilibria under every edge kind, conservation of
sum U on periodic domains (and the momentum gain N dt B per step under a
uniform body force), time reversibility of the omega = 2 collide-stream map
(Eq. B.5), the zeroth moment of the second-order initialization, and the
linear S-wave speed of a small shear wave.
"""
import numpy as np
import pytest

from oracle import oracle as o

CI = np.array([1, 0, -1, 0])
CJ = np.array([0, 1, 0, -1])


def uniform_state(nx, ny, F0, v=(0.0, 0.0)):
    U0 = np.zeros((6, ny, nx))
    U0[0], U0[1] = v
    for m in range(4):
        U0[2 + m] = F0[m]
    return U0


def smooth_random_state(nx, ny, rng, amp=0.02, modes=4):
    """A smooth periodic field (a few Fourier modes) around F = I, v = 0."""
    X, Y = o.node_coords(nx, ny, 1.0)
    U0 = np.zeros((6, ny, nx))
    U0[2] = 1.0
    U0[5] = 1.0
    for comp in range(6):
        for _ in range(modes):
            kx, ky = rng.integers(-2, 3, 2)
            ph = rng.uniform(0, 2 * np.pi)
            U0[comp] += amp * rng.uniform(-1, 1) * np.cos(2 * np.pi * (kx * X / nx + ky * Y / ny) + ph)
    return U0


EDGE_SETS = {
    "periodic": {},
    "all_velocity": {e: o.VELOCITY for e in range(4)},
    "all_traction": {e: o.TRACTION for e in range(4)},
    "mixed": {o.LEFT: o.VELOCITY, o.RIGHT: o.TRACTION, o.BOTTOM: o.TRACTION, o.TOP: o.TRACTION},
    "x_periodic_y_bounded": {o.BOTTOM: o.VELOCITY, o.TOP: o.TRACTION},
}


@pytest.mark.parametrize("edges", sorted(EDGE_SETS))
@pytest.mark.parametrize("omega", [1.3, 1.9, 2.0])
def test_rest_state_is_a_fixed_point(edges, omega):
    """F = I, v = 0 has P = 0 and f = f^eq, so every rule of Sec. 3.3 and 3.6
    returns it unchanged, bit for bit."""
    L = o.Lattice(9, 7, 1.0, 5.0, omega)
    L.set_law(o.NH, [1.0, 0.5])
    for e, kind in EDGE_SETS[edges].items():
        L.set_edge(e, kind)
    U0 = uniform_state(9, 7, [1.0, 0.0, 0.0, 1.0])
    L.init(U0)
    f0 = L.populations()
    L.step(300)
    assert np.array_equal(L.populations(), f0)
    assert L.status == 0


@pytest.mark.parametrize("omega", [1.5, 1.9])
def test_uniform_predeformed_state_is_stationary(omega):
    """A uniform F0 is a static equilibrium when velocity edges hold v_D = 0
    and traction edges carry T = P(F0) N (pair identities, Eq. B.16). (At
    omega near 2 the traction rule amplifies rounding; see the test below.)"""
    nx, ny = 10, 8
    lam, mu = 1.5, 0.75
    F0 = np.array([1.08, 0.05, -0.03, 0.96])
    P0, _ = o.piola(o.NH, [lam, mu], F0)
    P0 = P0.reshape(2, 2)
    normals = {o.LEFT: (-1, 0), o.RIGHT: (1, 0), o.BOTTOM: (0, -1), o.TOP: (0, 1)}
    L = o.Lattice(nx, ny, 1.0, 5.0, omega)
    L.set_law(o.NH, [lam, mu])
    L.set_edge(o.LEFT, o.VELOCITY)
    for e in (o.RIGHT, o.BOTTOM, o.TOP):
        T = P0 @ np.array(normals[e], dtype=float)
        L.set_edge(e, o.TRACTION, T)
    U0 = uniform_state(nx, ny, F0)
    L.init(U0)
    L.step(1000)
    U, _, _ = L.state()
    assert L.status == 0
    assert np.abs(U - U0).max() < 2e-14


def test_uniform_predeformed_state_periodic():
    nx, ny = 6, 5
    F0 = np.array([1.2, 0.3, 0.0, 1 / 1.2])
    L = o.Lattice(nx, ny, 1.0, 5.0, 2.0)
    L.set_law(o.NH, [1.5, 0.75])
    U0 = uniform_state(nx, ny, F0, v=(0.01, -0.02))
    L.init(U0)
    L.step(1000)
    U, _, _ = L.state()
    assert np.abs(U - U0).max() < 2e-14


@pytest.mark.parametrize("omega", [1.7, 2.0])
def test_periodic_conservation_of_state_sum(omega):
    """With B = 0, sum_q f* = sum_q f at every node (Eq. 14 and Eq. 11) and
    streaming permutes populations, so sum over nodes of U is conserved."""
    rng = np.random.default_rng(5)
    nx, ny = 24, 16
    L = o.Lattice(nx, ny, 1.0, 5.0, omega)
    L.set_law(o.NH, [1.0, 0.5])
    U0 = smooth_random_state(nx, ny, rng)
    L.init(U0)
    s0 = L.state()[0].sum(axis=(1, 2))
    L.step(1000)
    s1 = L.state()[0].sum(axis=(1, 2))
    assert np.abs(s1 - s0).max() < 1e-12 * nx * ny


@pytest.mark.parametrize("omega", [1.6, 2.0])
def test_momentum_gain_under_uniform_body_force(omega):
    """sum_q f* = U + (dt/2) B (Eq. 14, sum_q w_q = 1/2) and U = sum_q f +
    (dt/2) B (Eq. 10), so sum over nodes of v grows by N dt b per step."""
    rng = np.random.default_rng(6)
    nx, ny, c = 16, 12, 5.0
    b = np.array([3e-3, -2e-3])
    L = o.Lattice(nx, ny, 1.0, c, omega)
    L.set_law(o.NH, [1.0, 0.5])
    L.set_body_force(*b)
    L.init(smooth_random_state(nx, ny, rng))
    v0 = L.state()[0][:2].sum(axis=(1, 2))
    n = 400
    L.step(n)
    v1 = L.state()[0][:2].sum(axis=(1, 2))
    assert np.allclose(v1 - v0, n * nx * ny * L.dt * b, rtol=1e-11, atol=1e-12)


def _nh_piola_np(F, lam, mu):
    """P = mu (F - F^{-T}) + (lam/2)(J^2 - 1) F^{-T} for stacked F (4, ...)."""
    J = F[0] * F[3] - F[1] * F[2]
    H = np.array([F[3] / J, -F[2] / J, -F[1] / J, F[0] / J])
    return mu * (F - H) + 0.5 * lam * (J * J - 1) * H


def test_time_reversibility_at_omega_two():
    """At omega = 2, B = 0 the step is f(X + c_q dt, t + dt) = 2 f^eq(U) - f
    (Eq. B.5). Since sum_q f* = U, one step back is: un-stream, then
    f = 2 f^eq(sum_q f*) - f*. Running 300 steps forward in the oracle and 300
    back here must return the initial populations."""
    rng = np.random.default_rng(7)
    nx, ny, c, lam, mu = 20, 14, 5.0, 1.0, 0.5
    L = o.Lattice(nx, ny, 1.0, c, 2.0)
    L.set_law(o.NH, [lam, mu])
    L.init(smooth_random_state(nx, ny, rng, amp=0.05))
    f_start = L.populations()
    n = 300
    L.step(n)
    f = L.populations()
    for _ in range(n):
        fs = np.empty_like(f)
        for q in range(4):  # un-stream: f*_q(X) = f_q(X + c_q dt)
            fs[q] = np.roll(f[q], shift=(-CJ[q], -CI[q]), axis=(1, 2))
        U = fs.sum(axis=0)
        P = _nh_piola_np(U[2:], lam, mu)
        PhiX = np.array([-P[0], -P[2], -U[0], 0 * U[0], -U[1], 0 * U[0]])
        PhiY = np.array([-P[1], -P[3], 0 * U[0], -U[0], 0 * U[0], -U[1]])
        feq = np.array([0.25 * (U + (2 / c) * (CI[q] * PhiX + CJ[q] * PhiY)) for q in range(4)])
        f = 2 * feq - fs
    assert np.abs(f - f_start).max() < 1e-10


@pytest.mark.parametrize("edges", ["periodic", "all_velocity", "mixed"])
def test_second_order_init_zeroth_moment(edges):
    """sum_q D_q f^eq(U0) = B for any consistent gradients (the flux terms of
    Eq. 21 cancel against Z_1, Z_2 of Eq. 18), so sum_q f_q(0) = U0 - (dt/2) B."""
    rng = np.random.default_rng(8)
    nx, ny = 12, 10
    b = np.array([0.02, -0.01])
    L = o.Lattice(nx, ny, 1.0, 5.0, 2.0)
    L.set_law(o.NH, [1.2, 0.6])
    for e, kind in EDGE_SETS[edges].items():
        L.set_edge(e, kind)
    L.set_body_force(*b)
    U0 = smooth_random_state(nx, ny, rng, amp=0.05)
    L.init(U0, order=2)
    f = L.populations()
    target = U0.copy()
    target[0] -= 0.5 * L.dt * b[0]
    target[1] -= 0.5 * L.dt * b[1]
    assert np.abs(f.sum(axis=0) - target).max() < 1e-14
    # and the first-order correction is present: f differs from f^eq(U0)
    L0 = o.Lattice(nx, ny, 1.0, 5.0, 2.0)
    L0.set_law(o.NH, [1.2, 0.6])
    for e, kind in EDGE_SETS[edges].items():
        L0.set_edge(e, kind)
    L0.init(U0, order=0)
    assert np.abs(L0.populations() - f).max() > 1e-4


def test_linear_shear_wave_speed():
    """A standing shear wave v1 = A sin(kY) (F = I) oscillates at c_S k with
    c_S = sqrt(mu / rho0) (Sec. 2.3, Eq. 9); lattice dispersion is O((k dx)^2).
    64 x 64 periodic lattice, NH lambda = 1, mu = 0.5, c = 5, omega = 2."""
    n, lam, mu, A = 64, 1.0, 0.5, 0.01
    k = 2 * np.pi / n
    L = o.Lattice(n, n, 1.0, 5.0, 2.0)
    L.set_law(o.NH, [lam, mu])
    X, Y = o.node_coords(n, n, 1.0)
    U0 = uniform_state(n, n, [1.0, 0.0, 0.0, 1.0])
    U0[0] = A * np.sin(k * Y)
    L.init(U0)
    s = np.sin(k * Y)
    amps = [2 * np.mean(L.state()[0][0] * s)]
    cs = np.sqrt(mu)
    nsteps = int(0.3 * 2 * np.pi / (cs * k) / L.dt)
    for _ in range(nsteps):
        L.step(1)
        amps.append(2 * np.mean(L.state()[0][0] * s))
    amps = np.array(amps)
    # first zero crossing of A cos(Omega t) by linear interpolation
    i = np.nonzero(amps < 0)[0][0]
    t0 = (i - 1 + amps[i - 1] / (amps[i - 1] - amps[i])) * L.dt
    c_num = (np.pi / 2) / t0 / k
    assert abs(c_num - cs) / cs < 2e-3
    assert abs(amps[0] - A) < 1e-12


def _seeded_growth(omega, nsteps, nx=32, ny=16):
    L = o.Lattice(nx, ny, 1.0, 5.0, omega)
    L.set_law(o.NH, [2.0, 1.0])
    L.set_edge(o.LEFT, o.VELOCITY)
    for e in (o.RIGHT, o.BOTTOM, o.TOP):
        L.set_edge(e, o.TRACTION)
    rng = np.random.default_rng(0)
    U0 = uniform_state(nx, ny, [1.0, 0.0, 0.0, 1.0]) + 1e-12 * rng.normal(size=(6, ny, nx))
    L.init(U0, order=0)
    L.step(nsteps)
    U = L.state()[0]
    U[2] -= 1.0
    U[5] -= 1.0
    return np.abs(U).max()


def test_traction_edge_stability_threshold():
    """Characterisation of the traction rule of Eq. (25) (not a claim of the
    paper): its source S_d depends on the boundary node's own F, and at
    omega = 2 nothing damps that loop, so a 1e-12 perturbation of the rest
    state grows; at omega = 1.95 it decays. Clamped left edge, traction on the
    other three, NH lambda = 2, mu = 1, c = 5."""
    assert _seeded_growth(1.95, 2000) < 1e-11
    assert _seeded_growth(2.0, 1200) > 1e-9


def test_oracle_conditioning_of_the_64_shear_wave():
    """The floor any FP64 comparison of the 64 x 64 shear wave (1000 steps,
    omega = 2) can reach: perturbing the initial state by one ulp moves the
    oracle's own result by about 3.5e-12 in v and 1.7e-12 in P, 7e-15 in U."""
    from synth import shear_wave_64
    from tests.cases import group_errors

    w = shear_wave_64()
    U0, u0 = w.fields()

    def run(U):
        L = o.Lattice(64, 64, 1.0, 5.0, 2.0)
        L.set_law(o.NH, [1.0, 0.5])
        L.init(U, u0, 2)
        L.step(1000)
        U1, P1, S1 = L.state()
        return {"U": U1, "P": P1, "u": L.displacement(), "sigma": S1}

    a = run(U0)
    rng = np.random.default_rng(0)
    b = run(U0 * (1 + 2.2e-16 * rng.choice([-1, 1], size=U0.shape)))
    e = group_errors(a, b)
    assert 1e-12 < e["v"] < 1e-11 and 5e-13 < e["P"] < 5e-12 and e["U"] < 1e-13, e

"""Pins of the oracle's second-order initialization with finite-difference
gradients (Sec. 3.4, Eqs. 16-21: the gradients of v0 and F0 come from
second-order central differences, one-sided three-point stencils next to a
non-periodic edge), each against a fact of the mathematics rather than
against the oracle's own formula:

- on a non-periodic lattice, the central stencil (f(i+1) - f(i-1)) / (2 dx)
  and the one-sided (-3 f0 + 4 f1 - f2) / (2 dx) are exact for quadratics,
  so an FD start of a quadratic field equals the start with the analytic
  gradients;
- on a periodic lattice the central difference of sin(k X + phi) is exactly
  cos(k X + phi) sin(k dx) / dx, so an FD start of a sum of sinusoids equals
  the start with those scaled derivatives;
- the noise-free 64 x 64 shear wave of NH (F = I, v1 = A sin kY, omega = 2)
  stays on the simple-shear path F = [[1, g], [0, 1]], J = 1, where P12 =
  P21 = mu g exactly, so the whole scheme (FD start, collision, streaming,
  quadrature) is linear and translation invariant: its lattice solution is
  the eigen-decomposition of the per-mode 8 x 8 amplification matrix, here
  derived from the scheme's definitions (Eqs. 7, 12, 14, 15, 22) and the
  start f = f^eq - (dt/2)(d_t + c_q . grad) f^eq with the continuum time
  derivatives, and the oracle must follow it to rounding over 1000 steps.
"""
import numpy as np
import pytest

from oracle import oracle as o

EDGE_SETS = {
    "all_velocity": {e: o.VELOCITY for e in range(4)},
    "all_traction": {e: o.TRACTION for e in range(4)},
    "mixed": {o.LEFT: o.VELOCITY, o.RIGHT: o.TRACTION, o.BOTTOM: o.TRACTION, o.TOP: o.VELOCITY},
}


def _lattice(nx, ny, edges, c=5.0, omega=1.9, law=o.NH, prm=(1.3, 0.7), b=(0.0, 0.0)):
    L = o.Lattice(nx, ny, 1.0, c, omega)
    L.set_law(law, list(prm))
    L.set_body_force(*b)
    for e, kind in edges.items():
        L.set_edge(e, kind)
    return L


def _quadratic_field(nx, ny, seed):
    """U0 with every component a seeded quadratic polynomial in (X, Y) (F
    near I), and its exact gradients."""
    rng = np.random.default_rng(seed)
    X, Y = o.node_coords(nx, ny, 1.0)
    xs, ys = X / nx, Y / ny
    U0 = np.zeros((6, ny, nx))
    gX = np.zeros_like(U0)
    gY = np.zeros_like(U0)
    for k in range(6):
        a0, ax, ay, axx, axy, ayy = 0.03 * rng.uniform(-1, 1, 6)
        U0[k] = a0 + ax * xs + ay * ys + axx * xs ** 2 + axy * xs * ys + ayy * ys ** 2
        gX[k] = (ax + 2 * axx * xs + axy * ys) / nx
        gY[k] = (ay + axy * xs + 2 * ayy * ys) / ny
    U0[2] += 1.0
    U0[5] += 1.0
    return U0, gX, gY


@pytest.mark.parametrize("edges", sorted(EDGE_SETS))
@pytest.mark.parametrize("law,prm", [(o.NH, (1.3, 0.7)), (o.SVK, (1.1, 0.6)), (o.GENT, (1.0, 0.5, 8.0))])
def test_fd_start_is_exact_for_quadratic_fields(edges, law, prm):
    """Three-point stencils, central inside and one-sided at every
    non-periodic end, differentiate quadratics exactly; with a body force
    present so every term of Eq. (18) is in play."""
    nx, ny = 13, 11
    U0, gX, gY = _quadratic_field(nx, ny, seed=11)
    La = _lattice(nx, ny, EDGE_SETS[edges], law=law, prm=prm, b=(0.01, -0.02))
    La.init(U0, order=2, dUdX=gX, dUdY=gY)
    Lf = _lattice(nx, ny, EDGE_SETS[edges], law=law, prm=prm, b=(0.01, -0.02))
    Lf.init(U0, order=2)
    fa, ff = La.populations(), Lf.populations()
    # the gradients matter at this size: the order-0 start is far away
    L0 = _lattice(nx, ny, EDGE_SETS[edges], law=law, prm=prm, b=(0.01, -0.02))
    L0.init(U0, order=0)
    assert np.abs(L0.populations() - fa).max() > 1e-4
    err = np.abs(ff - fa)
    assert err.max() < 1e-13, (err.max(), np.unravel_index(err.argmax(), err.shape))
    # edge rows and columns and corners included
    for sl in (np.s_[..., 0, :], np.s_[..., -1, :], np.s_[..., :, 0], np.s_[..., :, -1]):
        assert err[sl].max() < 1e-13


def _mode_sum(nx, ny, seed, amp=0.03, nmodes=3):
    """Each component a seeded sum of periodic sinusoids sin(kx X + ky Y +
    phi); returns U0 and the gradients the central difference must give:
    A cos(.) kx sin(kx dx) / (kx dx) along x (dx = 1), likewise along y."""
    rng = np.random.default_rng(seed)
    X, Y = o.node_coords(nx, ny, 1.0)
    U0 = np.zeros((6, ny, nx))
    gX = np.zeros_like(U0)
    gY = np.zeros_like(U0)
    for k in range(6):
        for _ in range(nmodes):
            mx, my = rng.integers(-3, 4, 2)
            kx, ky = 2 * np.pi * mx / nx, 2 * np.pi * my / ny
            A, ph = amp * rng.uniform(-1, 1), rng.uniform(0, 2 * np.pi)
            U0[k] += A * np.sin(kx * X + ky * Y + ph)
            gX[k] += A * np.cos(kx * X + ky * Y + ph) * np.sin(kx)
            gY[k] += A * np.cos(kx * X + ky * Y + ph) * np.sin(ky)
    U0[2] += 1.0
    U0[5] += 1.0
    return U0, gX, gY


def test_fd_start_on_periodic_sinusoids_matches_the_scaled_derivative():
    nx, ny = 24, 18
    U0, gX, gY = _mode_sum(nx, ny, seed=5)
    La = _lattice(nx, ny, {}, omega=2.0)
    La.init(U0, order=2, dUdX=gX, dUdY=gY)
    Lf = _lattice(nx, ny, {}, omega=2.0)
    Lf.init(U0, order=2)
    err = np.abs(Lf.populations() - La.populations()).max()
    assert err < 1e-13, err
    # and the continuum derivative (without the sin(k dx)/(k dx) factor) is
    # measurably different, so the comparison sees the stencil's scale
    _, gXc, gYc = _mode_sum_continuum(nx, ny, seed=5)
    Lc = _lattice(nx, ny, {}, omega=2.0)
    Lc.init(U0, order=2, dUdX=gXc, dUdY=gYc)
    assert np.abs(Lc.populations() - La.populations()).max() > 1e-6


def _mode_sum_continuum(nx, ny, seed, amp=0.03, nmodes=3):
    rng = np.random.default_rng(seed)
    X, Y = o.node_coords(nx, ny, 1.0)
    U0 = np.zeros((6, ny, nx))
    gX = np.zeros_like(U0)
    gY = np.zeros_like(U0)
    for k in range(6):
        for _ in range(nmodes):
            mx, my = rng.integers(-3, 4, 2)
            kx, ky = 2 * np.pi * mx / nx, 2 * np.pi * my / ny
            A, ph = amp * rng.uniform(-1, 1), rng.uniform(0, 2 * np.pi)
            U0[k] += A * np.sin(kx * X + ky * Y + ph)
            gX[k] += A * kx * np.cos(kx * X + ky * Y + ph)
            gY[k] += A * ky * np.cos(kx * X + ky * Y + ph)
    U0[2] += 1.0
    U0[5] += 1.0
    return U0, gX, gY


def test_fd_start_mixed_periodic_and_bounded():
    """x periodic (sinusoid along X), y bounded (quadratic along Y): both
    stencils at once, product fields so each derivative is exact."""
    nx, ny = 16, 9
    rng = np.random.default_rng(3)
    X, Y = o.node_coords(nx, ny, 1.0)
    ys = Y / ny
    U0 = np.zeros((6, ny, nx))
    gX = np.zeros_like(U0)
    gY = np.zeros_like(U0)
    for k in range(6):
        m = rng.integers(1, 4)
        kx = 2 * np.pi * m / nx
        ph = rng.uniform(0, 2 * np.pi)
        a0, a1, a2 = 0.03 * rng.uniform(-1, 1, 3)
        q = a0 + a1 * ys + a2 * ys ** 2
        dq = (a1 + 2 * a2 * ys) / ny
        s = np.sin(kx * X + ph)
        U0[k] = q * s
        gX[k] = q * np.cos(kx * X + ph) * np.sin(kx)
        gY[k] = dq * s
    U0[2] += 1.0
    U0[5] += 1.0
    edges = {o.BOTTOM: o.VELOCITY, o.TOP: o.TRACTION}
    La = _lattice(nx, ny, edges)
    La.init(U0, order=2, dUdX=gX, dUdY=gY)
    Lf = _lattice(nx, ny, edges)
    Lf.init(U0, order=2)
    err = np.abs(Lf.populations() - La.populations()).max()
    assert err < 1e-13, err


# ---------------------------------------------------------------------------
# the 64 x 64 shear wave as a linear lattice recurrence
# ---------------------------------------------------------------------------

CJ = np.array([0, 1, 0, -1])  # y-components of the D2Q4 directions (Sec. 3.1)


def _shear_wave_closed_form(n, A, mu, c, omega, nsteps, dps=32):
    """v1, g = F12, the displacement u1 (each (n,) along y, uniform in x) after
    nsteps of the scheme for v1(0) = A sin(k (y + 1/2)), F = I, by the
    eigen-decomposition of the per-mode amplification matrix (in dps-digit
    arithmetic: a phase of 14 radians after 1000 steps is only good to a few
    1e-13 from an FP64 eigenvalue).

    Populations of the two active components (v1, F12) for q = 0..3 form the
    8-vector f. On the path F = [[1, g], [0, 1]] the fluxes of Eq. (7) give
    f^eq_q(v1) = (S_v - (2/c) j_q mu S_g) / 4 and f^eq_q(F12) = (S_g - (2/c)
    j_q S_v) / 4 with S the population sums (no body force). The collision
    (Eq. 14) is f* = (1 - w) f + w E f; pull streaming (Eq. 15) multiplies a
    mode exp(i k y) by exp(-i k j_q). A real field is Re(a exp(i k y))."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = dps
    k = 2 * mp.pi / n
    c, mu, omega = mp.mpf(c), mp.mpf(mu), mp.mpf(omega)
    dt = 1 / c
    E = mp.matrix(8, 8)
    for q in range(4):
        for p in range(4):
            E[q, p] = mp.mpf(1) / 4                          # S_v into v1
            E[q, 4 + p] = -(2 / c) * CJ[q] * mu / 4          # S_g into v1
            E[4 + q, 4 + p] = mp.mpf(1) / 4                  # S_g into F12
            E[4 + q, p] = -(2 / c) * CJ[q] / 4               # S_v into F12
    M = (1 - omega) * mp.eye(8) + omega * E
    G = mp.diag([mp.exp(-1j * k * int(CJ[q])) for q in range(4)] * 2) * M
    # start: v1 = Re(av e^{iky}), av = -i A e^{ik/2}; its central difference is
    # Re(ad e^{iky}) with ad = A sin(k) e^{ik/2} (dx = 1). With g = 0 and the
    # continuum rates d_t v1 = mu d_y g = 0 and d_t g = d_y v1:
    #   (d_t + c j d_y) f^eq(v1)  = (c j - (2/c) j mu) d_y v1 / 4
    #   (d_t + c j d_y) f^eq(F12) = (1 - 2 j^2) d_y v1 / 4
    A = mp.mpf(A)
    av = -1j * A * mp.exp(0.5j * k)
    ad = A * mp.sin(k) * mp.exp(0.5j * k)
    a0 = mp.matrix(8, 1)
    for q in range(4):
        j = int(CJ[q])
        a0[q] = av / 4 - dt / 2 * (c * j - (2 / c) * j * mu) * ad / 4
        a0[4 + q] = (-(2 / c) * j * av) / 4 - dt / 2 * (1 - 2 * j * j) * ad / 4
    lam, V = mp.eig(G)
    b0 = mp.lu_solve(V, a0)
    an = V * mp.matrix([lam[i] ** nsteps * b0[i] for i in range(8)])
    # sum_{m<n} lam^m, the geometric sum of each eigenvalue
    geo = [nsteps if abs(lv - 1) < mp.mpf(10) ** (-dps // 2) else (1 - lv ** nsteps) / (1 - lv) for lv in lam]
    asum = V * mp.matrix([geo[i] * b0[i] for i in range(8)])

    def field(vec, lo):
        amp = complex(sum(vec[lo + q] for q in range(4)))
        return np.real(amp * np.exp(1j * 2 * np.pi / n * np.arange(n)))

    v1, g, v0 = field(an, 0), field(an, 4), field(a0, 0)
    # Eq. (22): u^n = u*^n + (dt/2) v^n, u*^0 = u0 - (dt/2) v^0 (u0 = 0), u*^{m+1} = u*^m + dt v^m
    dtf = float(dt)
    u1 = -0.5 * dtf * v0 + dtf * field(asum, 0) + 0.5 * dtf * v1
    Gf = np.array([[complex(G[r, s]) for s in range(8)] for r in range(8)])
    return v1, g, u1, Gf


def test_shear_wave_64_follows_the_closed_form_lattice_evolution():
    """Config of the 64 x 64 periodic square (NH lambda = 1, mu = 0.5, c = 5,
    omega = 2, A = 0.01) without the noise, 1000 steps, relative L2 <= 1e-12
    per field against the closed form."""
    n, lam, mu, c, omega, A, nsteps = 64, 1.0, 0.5, 5.0, 2.0, 0.01, 1000
    v1, g, u1, G = _shear_wave_closed_form(n, A, mu, c, omega, nsteps)
    # the recurrence is neutral at omega = 2 (no mode grows or decays)
    assert np.allclose(np.abs(np.linalg.eigvals(G)), 1.0, atol=1e-12)
    L = o.Lattice(n, n, 1.0, c, omega)
    L.set_law(o.NH, [lam, mu])
    U0 = np.zeros((6, n, n))
    U0[2] = U0[5] = 1.0
    U0[0] = A * np.sin(2 * np.pi * (np.arange(n)[:, None] + 0.5) / n) * np.ones((1, n))
    L.init(U0, np.zeros((2, n, n)), 2)
    L.step(nsteps)
    U, P, _ = L.state()
    u = L.displacement()

    def rel(a, b):
        return np.linalg.norm(a - b) / np.linalg.norm(b)

    full = np.ones((1, n))
    assert rel(U[0], v1[:, None] * full) < 1e-12
    assert rel(U[3], g[:, None] * full) < 1e-12
    assert rel(P[1], mu * g[:, None] * full) < 1e-12
    assert rel(P[2], mu * g[:, None] * full) < 1e-12
    assert rel(u[0], u1[:, None] * full) < 1e-12
    # the other components stay on the simple-shear path to rounding
    # (a few 1e-15 against the wave's 1e-2)
    for comp, ref in ((1, 0.0), (2, 1.0), (4, 0.0), (5, 1.0)):
        assert np.abs(U[comp] - ref).max() < 1e-13, comp
    assert np.abs(u[1]).max() < 1e-13
    # a nontrivial phase after 1000 steps (t = 200, about 1.4 periods of the S wave)
    assert np.abs(v1).max() > 1e-3 and np.abs(g).max() > 1e-3


def test_shear_wave_closed_form_is_the_continuum_wave_to_second_order():
    """Independent of the oracle: the closed form's phase speed approaches
    sqrt(mu) as k dx -> 0 with the O((k dx)^2) lattice dispersion."""
    mu, c = 0.5, 5.0
    errs = []
    for n in (32, 64, 128):
        G = _shear_wave_closed_form(n, 0.01, mu, c, 2.0, 1)[3]
        k = 2 * np.pi / n
        lam = np.linalg.eigvals(G)
        # the slow (acoustic) pair: smallest nonzero phase per step
        ph = np.abs(np.angle(lam))
        ph = ph[ph > 1e-9].min()
        errs.append(abs(ph / (1.0 / c) / k - np.sqrt(mu)) / np.sqrt(mu))
    assert errs[-1] < 1e-3
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5

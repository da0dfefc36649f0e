"""Pins of the oracle's pointwise building blocks against what Appendix A,
Sec. 2.3-2.4 and Sec. 3.2 fix: P = dW/dF, the tangent C = dP/dF (Eq. 4), the
stress-free reference state, objectivity, the small-strain moduli, the flux
vectors (Eq. 7) and the equilibrium moment and pair identities (Eqs. 11, B.16).
"""
import numpy as np
import pytest

from oracle import oracle as o

LAWS = {
    "SVK": (o.SVK, [1.3, 0.7]),
    "NH": (o.NH, [1.3, 0.7]),
    "LOGNH": (o.LOGNH, [1.3, 0.7]),
    "MR": (o.MR, [1.3, 0.2, 0.15]),
    "YEOH": (o.YEOH, [1.3, 0.35, 0.03, 0.02]),
    "GENT": (o.GENT, [1.3, 0.7, 10.0]),
}
# small-strain shear modulus of each parameter set (Appendix A: c10 + c01 = mu/2,
# c1 = mu/2) and its 2-D Lame lambda; the isochoric invariants of the last three
# laws are 3-D ones with F33 = 1, which lowers the in-plane lambda by 2 mu / 3
SMALL_STRAIN = {
    "SVK": (0.7, 1.3), "NH": (0.7, 1.3), "LOGNH": (0.7, 1.3),
    "MR": (0.7, 1.3 - 2 * 0.7 / 3), "YEOH": (0.7, 1.3 - 2 * 0.7 / 3), "GENT": (0.7, 1.3 - 2 * 0.7 / 3),
}


def random_F(rng, scale=0.25):
    while True:
        F = np.eye(2).ravel() + scale * rng.uniform(-1, 1, 4)
        if F[0] * F[3] - F[1] * F[2] > 0.3:
            return F


@pytest.mark.parametrize("name", sorted(LAWS))
def test_reference_state_is_stress_free(name):
    law, prm = LAWS[name]
    P, rc = o.piola(law, prm, np.array([1.0, 0.0, 0.0, 1.0]))
    assert rc == 0
    assert np.abs(P).max() < 1e-15
    assert abs(o.energy(law, prm, np.array([1.0, 0.0, 0.0, 1.0]))) < 1e-15


@pytest.mark.parametrize("name", sorted(LAWS))
def test_piola_is_energy_gradient(name):
    """P_iA = dW/dF_iA by fourth-order central differences of W (Eq. 4)."""
    law, prm = LAWS[name]
    rng = np.random.default_rng(11)
    h = 1e-4
    for _ in range(5):
        F = random_F(rng)
        P, _ = o.piola(law, prm, F)
        g = np.zeros(4)
        for m in range(4):
            e = np.zeros(4)
            e[m] = h
            w = [o.energy(law, prm, F + s * e) for s in (-2, -1, 1, 2)]
            g[m] = (w[0] - 8 * w[1] + 8 * w[2] - w[3]) / (12 * h)
        assert np.allclose(P, g, rtol=1e-8, atol=1e-10), (P, g)


@pytest.mark.parametrize("name", sorted(LAWS))
def test_tangent_against_differences_and_symmetry(name):
    law, prm = LAWS[name]
    rng = np.random.default_rng(12)
    h = 1e-4
    for _ in range(5):
        F = random_F(rng)
        Ct = o.tangent(law, prm, F)
        fd = np.zeros((4, 4))
        for m in range(4):
            e = np.zeros(4)
            e[m] = h
            p = [o.piola(law, prm, F + s * e)[0] for s in (-2, -1, 1, 2)]
            fd[:, m] = (p[0] - 8 * p[1] + 8 * p[2] - p[3]) / (12 * h)
        assert np.allclose(Ct, fd, rtol=1e-8, atol=1e-9)
        # hyperelastic major symmetry C_iAkB = C_kBiA
        assert np.allclose(Ct, Ct.T, rtol=0, atol=1e-12)


@pytest.mark.parametrize("name", sorted(LAWS))
def test_complex_copy_matches_real_closure(name):
    law, prm = LAWS[name]
    rng = np.random.default_rng(13)
    for _ in range(5):
        F = random_F(rng)
        P, _ = o.piola(law, prm, F)
        Pre, Pim = o.piola_cplx(law, prm, F, np.zeros(4))
        assert np.allclose(P, Pre, rtol=1e-14, atol=1e-15)
        assert np.abs(Pim).max() == 0.0


@pytest.mark.parametrize("name", sorted(LAWS))
def test_objectivity(name):
    """W(RF) = W(F) for a rotation R, hence P F^T is symmetric."""
    law, prm = LAWS[name]
    rng = np.random.default_rng(14)
    for _ in range(5):
        F = random_F(rng)
        th = rng.uniform(0, 2 * np.pi)
        R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        RF = (R @ F.reshape(2, 2)).ravel()
        assert abs(o.energy(law, prm, RF) - o.energy(law, prm, F)) < 1e-13
        P, _ = o.piola(law, prm, F)
        PFt = P.reshape(2, 2) @ F.reshape(2, 2).T
        assert abs(PFt[0, 1] - PFt[1, 0]) < 1e-13


@pytest.mark.parametrize("name", sorted(LAWS))
def test_small_strain_moduli(name):
    """At F = I every law reduces to linear elasticity:
    C_iAkB = mu (d_ik d_AB + d_iB d_kA) + lambda d_iA d_kB."""
    law, prm = LAWS[name]
    mu, lam = SMALL_STRAIN[name]
    Ct = o.tangent(law, prm, np.array([1.0, 0.0, 0.0, 1.0]))
    d = np.eye(2)
    ref = np.zeros((4, 4))
    for i in range(2):
        for A in range(2):
            for k in range(2):
                for B in range(2):
                    ref[2 * i + A, 2 * k + B] = mu * (d[i, k] * d[A, B] + d[i, B] * d[k, A]) + lam * d[i, A] * d[k, B]
    assert np.allclose(Ct, ref, rtol=0, atol=1e-12)


def test_nh_wave_speeds_from_acoustic_tensor():
    """Eq. (9): at F = I the acoustic tensor has eigenvalues mu and lambda + 2 mu,
    i.e. c_S = sqrt(mu) and c_P = sqrt(lambda + 2 mu) (rho0 = 1)."""
    lam, mu = 1.0, 0.5
    Ct = o.tangent(o.NH, [lam, mu], np.array([1.0, 0.0, 0.0, 1.0])).reshape(2, 2, 2, 2)
    for th in np.linspace(0, np.pi, 7):
        n = np.array([np.cos(th), np.sin(th)])
        Q = np.einsum("A,iAkB,B->ik", n, Ct, n)
        assert np.allclose(np.sort(np.linalg.eigvalsh(Q)), [mu, lam + 2 * mu], atol=1e-12)


def test_nh_closed_form_on_simple_shear():
    """On F = [[1, g], [0, 1]] (J = 1) the NH stress is P = mu [[0, g], [g, 0]]
    (the path of Eqs. 43-45, transposed)."""
    for g in (0.1, -0.3, 0.8):
        P, _ = o.piola(o.NH, [2.0, 1.5], np.array([1.0, g, 0.0, 1.0]))
        assert np.allclose(P, [0.0, 1.5 * g, 1.5 * g, 0.0], atol=1e-14)


def test_flux_vectors_definition():
    rng = np.random.default_rng(2)
    U = rng.normal(size=6)
    P = rng.normal(size=4)
    X, Y = o.flux(U, P)
    # Eq. (7): Phi_X = (-P11, -P21, -v1, 0, -v2, 0), Phi_Y = (-P12, -P22, 0, -v1, 0, -v2)
    assert np.array_equal(X, [-P[0], -P[2], -U[0], 0.0, -U[1], 0.0])
    assert np.array_equal(Y, [-P[1], -P[3], 0.0, -U[0], 0.0, -U[1]])


@pytest.mark.parametrize("c", [1.0, 5.0, 10.0])
def test_equilibrium_moments_and_pair_identities(c):
    """Eq. (11) moments and the pair identities of Eq. (B.16) for random U."""
    rng = np.random.default_rng(3)
    ci = np.array([1, 0, -1, 0])
    cj = np.array([0, 1, 0, -1])
    for _ in range(10):
        U = rng.normal(size=6)
        P = rng.normal(size=4)
        X, Y = o.flux(U, P)
        f = o.feq(U, P, c)
        assert np.allclose(f.sum(0), U, atol=1e-14)
        assert np.allclose((c * ci[:, None] * f).sum(0), X, atol=1e-13)
        assert np.allclose((c * cj[:, None] * f).sum(0), Y, atol=1e-13)
        assert np.allclose((c * c * (ci ** 2 - cj ** 2)[:, None] * f).sum(0), 0.0, atol=1e-12)
        for q, mq in ((0, 2), (1, 3), (2, 0), (3, 1)):
            dA = np.array([ci[q], cj[q]])
            assert np.allclose(f[q] + f[mq], U / 2, atol=1e-14)
            assert np.allclose(f[q] - f[mq], (dA[0] * X + dA[1] * Y) / c, atol=1e-14)


def test_time_functions_special_values():
    assert o.timefn(o.T_CONST, [], 3.0) == 1.0
    assert o.timefn(o.T_LINEAR_RAMP, [4.0], 1.0) == 0.25
    assert o.timefn(o.T_LINEAR_RAMP, [4.0], 5.0) == 1.0
    # Eq. (33): g = sin^2(pi t / 4) for t < 2 is SIN2_RAMP with T = 2
    assert abs(o.timefn(o.T_SIN2_RAMP, [2.0], 1.0) - 0.5) < 1e-15
    assert o.timefn(o.T_SIN2_RAMP, [2.0], 2.5) == 1.0
    # Eq. (35): h = sin(pi t / 2) for t < 2, 0 after
    assert abs(o.timefn(o.T_SIN_PULSE, [2.0], 1.0) - 1.0) < 1e-15
    assert o.timefn(o.T_SIN_PULSE, [2.0], 2.0) == 0.0
    # Sec. 5.4 Ricker pulse: peak 2/(sqrt(3 s) pi^(1/4)) at t0, zeros at t0 +- s
    s, t0 = 0.215, 1.0
    assert abs(o.timefn(o.T_RICKER, [s, t0, 2.0], t0) - 2 / (np.sqrt(3 * s) * np.pi ** 0.25)) < 1e-14
    assert abs(o.timefn(o.T_RICKER, [s, t0, 2.0], t0 + s)) < 1e-14
    assert o.timefn(o.T_RICKER, [s, t0, 2.0], 2.1) == 0.0

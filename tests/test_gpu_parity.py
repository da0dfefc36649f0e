"""CUDA path (through the C ABI) against the FP64 oracle, element by element,
on seeded inputs at sizes that span several warp segments and end in a ragged
tail, for every edge rule, closure, storage precision and degenerate size.

Tolerances (relative L2 per group; groups are v, F - I, P, u, sigma and the
full state U over all nodes and components):
  FP64 storage: 1e-12 on U; 1e-11 per group. The 64^2 shear wave is neutral
  (omega = 2) for 1000 steps, and perturbing its initial state by one ulp
  moves the oracle's own v, P and F - I by 3.5e-12, 1.7e-12 and 8e-13
  (test_oracle_conditioning); the per-group bound sits a factor three above
  that floor.
  FP32 storage: 1e-5 per group (the FP32 target after 1000 steps) except the
  displacement, and 1e-6 on U. The displacement u gets 2e-5: it integrates
  the velocity error of every step, and in the periodic cases with a body
  force (mean flow growing as b t, u as b t^2 / 2) the FP32 rounding of the
  slowly varying velocity populations adds up with one sign over the run
  (1.05e-5 after 300 steps there, where a one-ulp FP32 perturbation of the
  start alone moves v by only 6.5e-7).
  FP16 / BF16 storage (FP32 compute): the rounding model of
  tests.cases.rounding_scales, 1.5 * 2^-p * sqrt(n) * s_g per group with
  2^-p = 2^-11 / 2^-8 and s_g the ratio of the stored offsets' size to the
  group's size, taken from the oracle's state; every case measures 0.02 to
  0.55 of 2^-p sqrt(n) s_g.
"""
import numpy as np
import pytest

from tests.cases import (Case, group_errors, rounding_scales, run_gpu, run_oracle, small_strain_modulus,
                         smooth_field, tol_16bit)

pytestmark = pytest.mark.gpu

F64, F32, BF16, F16 = 0, 1, 2, 3
TOL = {F64: dict(group=1e-11, U=1e-12), F32: dict(group=1e-5, u=2e-5, U=1e-6)}


def tol_for(storage, steps, ref=None, c=5.0, modulus=None):
    """Per-group bounds {group: bound} (see the module docstring); the 16-bit
    bounds need the reference state ref = {"U": U, "P": P} and the
    closure's lambda + 2 mu_0."""
    if storage in TOL:
        t = TOL[storage]
        return {g: t.get(g, t["group"]) for g in ("v", "F-I", "P", "u", "sigma")} | {"U": t["U"]}
    return tol_16bit(storage, steps, rounding_scales(ref["U"], ref["P"], c, modulus))


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2605_26677_gb300 import build

    build.build()


def check(case, storage, skip=()):
    g = run_gpu(case, storage)
    o = run_oracle(case)
    errs = group_errors(g, o)
    print("PARITY storage=%d steps=%d %dx%d" % (storage, case.steps, case.nx, case.ny),
          {k: "%.2e" % v for k, v in errs.items()})
    tol = tol_for(storage, case.steps, o, case.c, small_strain_modulus(case.law, case.material()))
    for k, v in errs.items():
        if k in skip:
            continue
        assert v <= tol[k], (k, v, tol[k], errs)
    assert abs(g["t"] - o["t"]) < 1e-12
    return errs


# ---------------------------------------------------------------- 64 x 64 shear wave, 1000 steps
def shear_wave_case(steps=1000):
    from synth import shear_wave_64

    w = shear_wave_64()
    U0, u0 = w.fields()
    return Case(w.nx, w.ny, steps, lam=w.lam, mu=w.mu, c=w.c, omega=w.omega, U0=U0, u0=u0)


@pytest.mark.parametrize("storage", [F64, F32, F16, BF16])
def test_shear_wave_64_1000_steps(storage):
    errs = check(shear_wave_case(), storage)
    print("shear wave 64^2 x 1000 storage", storage, {k: "%.2e" % v for k, v in errs.items()})


# ---------------------------------------------------------------- edge rules
def edge_sets(nx, ny):
    ry = np.linspace(0.5, 1.5, ny)
    rx = np.cos(np.linspace(0, np.pi, nx)) ** 2 + 0.5
    return {
        "all_velocity": {0: ("velocity", (0.01, -0.02), "sin2_ramp", (30.0,), ry),
                         1: ("velocity", (0.0, 0.015), "linear_ramp", (50.0,), None),
                         2: ("velocity", (-0.01, 0.0), "const", None, rx),
                         3: ("velocity", (0.02, 0.01), "sin_pulse", (80.0,), None)},
        "all_traction": {0: ("traction", (0.02, 0.0), "sin2_ramp", (40.0,), None),
                         1: ("traction", (0.03, -0.01), "const", None, ry),
                         2: ("traction", (0.0, -0.02), "linear_ramp", (60.0,), rx),
                         3: ("traction", (0.01, 0.02), "sin2_ramp", (30.0,), None)},
        "clamped_mixed": {0: ("velocity", (0.0, 0.0), "const", None, None),
                          1: ("traction", (0.05, 0.02), "ricker", (20.0, 40.0, 120.0), ry),
                          2: ("traction", (0.0, 0.0), "const", None, None),
                          3: ("traction", (0.0, 0.0), "const", None, None)},
        "x_periodic": {2: ("velocity", (0.0, 0.01), "sin2_ramp", (25.0,), rx),
                       3: ("traction", (0.02, 0.0), "sin2_ramp", (25.0,), None)},
        "y_periodic": {0: ("traction", (0.0, 0.03), "sin2_ramp", (25.0,), ry),
                       1: ("velocity", (0.01, 0.0), "const", None, None)},
    }


@pytest.mark.parametrize("storage", [F64, F32, F16, BF16])
@pytest.mark.parametrize("edges", ["all_velocity", "all_traction", "clamped_mixed", "x_periodic", "y_periodic"])
def test_edge_rules_ragged_grid(storage, edges):
    nx, ny = 131, 37  # 3 warp segments in FP64 (64 nodes), 2 in FP32 (128), tail of 3
    E = edge_sets(nx, ny)[edges]
    periodic = edges in ("x_periodic", "y_periodic")
    U0 = smooth_field(nx, ny, seed=21, periodic=periodic)
    case = Case(nx, ny, 200, lam=1.5, mu=0.75, omega=1.9, body=(2e-4, -1e-4), edges=E, U0=U0)
    errs = check(case, storage)
    print("edges", edges, "storage", storage, {k: "%.2e" % v for k, v in errs.items()})


@pytest.mark.parametrize("storage", [F64, F32])
def test_traction_second_order_F_boundary(storage):
    nx, ny = 70, 45
    E = edge_sets(nx, ny)["clamped_mixed"]
    E[2] = ("traction", (0.0, -0.01), "sin2_ramp", (20.0,), None)
    case = Case(nx, ny, 150, lam=2.0, mu=1.0, omega=1.9, fb_mode=1, edges=E,
                U0=smooth_field(nx, ny, seed=5, periodic=False))
    check(case, storage)


# ---------------------------------------------------------------- closures
@pytest.mark.parametrize("law", ["SVK", "NH", "LOGNH"])
def test_closures_periodic(law):
    nx, ny = 67, 29
    U0 = smooth_field(nx, ny, seed=31, amp=0.08)
    case = Case(nx, ny, 300, law=law, lam=1.2, mu=0.8, body=(1e-3, 0.0), U0=U0)
    check(case, F64)
    check(case, F32)


def test_closures_bounded_logNH():
    nx, ny = 50, 40
    case = Case(nx, ny, 200, law="LOGNH", lam=2 / 3, mu=1.0, omega=1.9,
                edges=edge_sets(nx, ny)["all_traction"], U0=smooth_field(nx, ny, seed=8, periodic=False))
    check(case, F64)


# Appendix A closures built on the isochoric invariants; lambda = 1.2 and a
# small-strain shear modulus of 0.8 for each
INVARIANT_LAWS = {"MR": (1.2, 0.3, 0.1), "YEOH": (1.2, 0.4, 0.05, 0.01), "GENT": (1.2, 0.8, 20.0)}


@pytest.mark.parametrize("law", list(INVARIANT_LAWS))
def test_invariant_closures_periodic(law):
    nx, ny = 67, 29
    U0 = smooth_field(nx, ny, seed=31, amp=0.08)
    case = Case(nx, ny, 300, law=law, params=INVARIANT_LAWS[law], body=(1e-3, 0.0), U0=U0)
    check(case, F64)
    check(case, F32)


@pytest.mark.parametrize("law", list(INVARIANT_LAWS))
def test_invariant_closures_bounded(law):
    # every edge a traction edge: the Newton solve for F^b and the
    # second-order start both take the closure's tangent (dual numbers)
    nx, ny = 50, 40
    case = Case(nx, ny, 200, law=law, params=INVARIANT_LAWS[law], omega=1.9,
                edges=edge_sets(nx, ny)["all_traction"], U0=smooth_field(nx, ny, seed=8, periodic=False))
    check(case, F64)
    check(case, F32)


@pytest.mark.parametrize("law", list(INVARIANT_LAWS))
@pytest.mark.parametrize("storage", [BF16, F16])
def test_invariant_closures_16bit(law, storage):
    nx, ny = 67, 29
    U0 = smooth_field(nx, ny, seed=31, amp=0.08)
    check(Case(nx, ny, 300, law=law, params=INVARIANT_LAWS[law], U0=U0), storage)


# ---------------------------------------------------------------- initialization
@pytest.mark.parametrize("order", [0, 2])
@pytest.mark.parametrize("edges", ["periodic", "clamped_mixed"])
def test_initialization_only(order, edges):
    nx, ny = 45, 33
    E = {} if edges == "periodic" else edge_sets(nx, ny)[edges]
    U0 = smooth_field(nx, ny, seed=3, amp=0.05, periodic=(edges == "periodic"))
    u0 = 0.01 * smooth_field(nx, ny, seed=4)[:2]
    case = Case(nx, ny, 0, order=order, body=(0.01, -0.02), edges=E, U0=U0, u0=u0)
    check(case, F64)
    # zero steps: Eq. (10) with Eq. (16) summed over q gives U0 for the
    # second-order start; the equilibrium start has sum_q f = U0, so Eq. (10)
    # adds (dt/2) B to the velocity
    g = run_gpu(case, F64)
    expect = U0.copy()
    if order == 0:
        expect[0] += 0.5 * 0.2 * 0.01
        expect[1] += 0.5 * 0.2 * -0.02
    assert np.abs(g["U"] - expect).max() < 1e-14
    # u^0 = u*^0 + (dt/2) v^0 with u*^0 = u0 - (dt/2) v0 (Eq. 22)
    assert np.abs(g["u"] - (u0 + 0.1 * (expect[:2] - U0[:2]))).max() < 1e-15


@pytest.mark.parametrize("order", [0, 2])
def test_initialization_then_steps(order):
    nx, ny = 45, 33
    case = Case(nx, ny, 50, order=order, U0=smooth_field(nx, ny, seed=3, amp=0.05))
    check(case, F64)


# ---------------------------------------------------------------- degenerate sizes
@pytest.mark.parametrize("nx,ny,edges", [
    (1, 1, "periodic"), (1, 9, "periodic"), (9, 1, "periodic"), (2, 2, "periodic"),
    (3, 3, "all_velocity"), (3, 4, "all_traction"), (4, 3, "clamped_mixed"),
    (1, 6, "x_periodic"), (5, 2, "y_periodic"), (64, 5, "periodic"), (65, 3, "all_velocity"),
])
@pytest.mark.parametrize("storage", [F64, F32, F16, BF16])
def test_degenerate_sizes(nx, ny, edges, storage):
    E = {} if edges == "periodic" else edge_sets(nx, ny)[edges]
    U0 = smooth_field(nx, ny, seed=13, periodic=(edges in ("periodic", "x_periodic", "y_periodic")))
    case = Case(nx, ny, 60, omega=1.9, body=(1e-3, 5e-4), edges=E, U0=U0)
    check(case, storage)


# ---------------------------------------------------------------- diagnostics
def test_diagnostics_match_oracle_state():
    from oracle import oracle as orc

    nx, ny = 40, 30
    case = Case(nx, ny, 80, lam=1.5, mu=0.75, omega=1.9, edges=edge_sets(nx, ny)["clamped_mixed"],
                U0=smooth_field(nx, ny, seed=17, amp=0.05, periodic=False))
    g = run_gpu(case, F64)
    o = run_oracle(case)
    U = o["U"]
    J = U[2] * U[5] - U[3] * U[4]
    W = np.array([orc.energy(orc.NH, [1.5, 0.75], U[2:, j, i]) for j in range(ny) for i in range(nx)])
    expect = [U[0].sum(), U[1].sum(), U[2].mean(), U[3].mean(), U[4].mean(), U[5].mean(),
              (0.5 * (U[0] ** 2 + U[1] ** 2)).sum() + W.sum(), J.min(), J.max(),
              np.sqrt((U[2] - 1) ** 2 + U[3] ** 2 + U[4] ** 2 + (U[5] - 1) ** 2).max()]
    assert np.allclose(g["diag"], expect, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("fb_mode", [0, 1])
@pytest.mark.parametrize("storage", [F64, F32])
def test_edge_data_changed_between_steps(storage, fb_mode):
    """New edge data applies from the next step (the node form rebuilds the
    ghost cells the previous step wrote with the old data)."""
    from oracle import oracle as orc
    from paper_2605_26677_gb300 import lbm
    from tests.cases import KIND, TIMEFN, group_errors

    nx, ny, n1, n2 = 70, 40, 60, 50
    E = edge_sets(nx, ny)["clamped_mixed"]
    U0 = smooth_field(nx, ny, seed=12, periodic=False)
    change = {1: ("traction", (-0.03, 0.01), "sin2_ramp", (15.0,), None),
              0: ("velocity", (0.005, 0.0), "const", None, None)}
    L = lbm.Lattice(nx, ny, omega=1.9, storage=storage, fb_mode=fb_mode)
    lbm.lbm_set_material(L.ctx, lbm.LBM_LAW_NH, [1.5, 0.75])
    for e, (k, v, tf, tp, pr) in E.items():
        lbm.lbm_set_boundary(L.ctx, e, KIND[k], v, TIMEFN[tf], tp, pr)
    lbm.lbm_init(L.ctx, U0)
    lbm.lbm_step(L.ctx, n1)
    for e, (k, v, tf, tp, pr) in change.items():
        lbm.lbm_set_boundary(L.ctx, e, KIND[k], v, TIMEFN[tf], tp, pr)
    lbm.lbm_step(L.ctx, n2)
    U, P, _ = lbm.lbm_read_state(L.ctx)
    u = lbm.lbm_read_displacement(L.ctx)
    S = lbm.lbm_read_cauchy(L.ctx)
    L.close()
    O = orc.Lattice(nx, ny, 1.0, 5.0, 1.9)
    O.set_law(orc.NH, [1.5, 0.75])
    O.set_fb_mode(fb_mode)
    for e, (k, v, tf, tp, pr) in E.items():
        O.set_edge(e, KIND[k], v, TIMEFN[tf], tp if tp is not None else (0, 0, 0, 0), pr)
    O.init(U0)
    O.step(n1)
    for e, (k, v, tf, tp, pr) in change.items():
        O.set_edge(e, KIND[k], v, TIMEFN[tf], tp if tp is not None else (0, 0, 0, 0), pr)
    O.step(n2)
    Uo, Po, So = O.state()
    errs = group_errors({"U": U, "P": P, "u": u, "sigma": S}, {"U": Uo, "P": Po, "u": O.displacement(), "sigma": So})
    print("PARITY edge data changed, storage=%d" % storage, {k: "%.2e" % v for k, v in errs.items()})
    tol = tol_for(storage, n1 + n2)
    for k, v in errs.items():
        assert v <= tol[k], (k, v, errs)


@pytest.mark.parametrize("storage", [F64, F32])
def test_tabulated_time_function(storage):
    """LBM_T_TABLE: a piecewise-linear load history on the right (traction)
    edge. The oracle has no tables; it gets the same edge data written out
    step by step (its explicit per-node edge data, the value times the
    table interpolated by numpy at t^n + dt/2)."""
    from oracle import oracle as orc
    from paper_2605_26677_gb300 import lbm
    from tests.cases import KIND, TIMEFN, group_errors

    nx, ny, steps = 70, 40, 120
    E = edge_sets(nx, ny)["clamped_mixed"]
    U0 = smooth_field(nx, ny, seed=14, periodic=False)
    value = (0.04, -0.01)
    tt = np.array([0.0, 3.0, 7.5, 12.0, 20.0])
    gg = np.array([0.0, 1.0, 0.4, -0.3, 0.1])
    L = lbm.Lattice(nx, ny, omega=1.9, storage=storage)
    lbm.lbm_set_material(L.ctx, lbm.LBM_LAW_NH, [1.5, 0.75])
    for e, (k, v, tf, tp, pr) in E.items():
        lbm.lbm_set_boundary(L.ctx, e, KIND[k], v, TIMEFN[tf], tp, pr)
    lbm.lbm_set_boundary(L.ctx, 1, lbm.LBM_BC_TRACTION, value, lbm.LBM_T_TABLE)
    with pytest.raises(lbm.LbmError, match="LBM_ERR_STATE"):
        lbm.lbm_init(L.ctx, U0)  # the table is missing
    lbm.lbm_set_boundary_table(L.ctx, 1, tt, gg)
    lbm.lbm_init(L.ctx, U0)
    lbm.lbm_step(L.ctx, steps)
    U, P, _ = lbm.lbm_read_state(L.ctx)
    u = lbm.lbm_read_displacement(L.ctx)
    L.close()
    O = orc.Lattice(nx, ny, 1.0, 5.0, 1.9)
    O.set_law(orc.NH, [1.5, 0.75])
    for e, (k, v, tf, tp, pr) in E.items():
        O.set_edge(e, KIND[k], v, TIMEFN[tf], tp if tp is not None else (0, 0, 0, 0), pr)
    O.set_edge(1, orc.TRACTION, value)
    O.init(U0)
    for n in range(steps):
        g = np.interp((n + 0.5) * O.dt, tt, gg)
        O.set_edge_data(1, np.array([[value[0] * g] * ny, [value[1] * g] * ny]))
        O.step(1)
    Uo, Po, So = O.state()
    errs = group_errors({"U": U, "P": P, "u": u, "sigma": So}, {"U": Uo, "P": Po, "u": O.displacement(), "sigma": So})
    print("PARITY tabulated load, storage=%d" % storage, {k: "%.2e" % v for k, v in errs.items()})
    tol = tol_for(storage, steps)
    for k in ("v", "F-I", "P", "u", "U"):
        assert errs[k] <= tol[k], (k, errs)


@pytest.mark.parametrize("storage", [F64, F32, F16, BF16])
def test_precision_error_vs_oracle_fourier(storage):
    """Error of each storage precision against the FP64 oracle on the 16-mode
    random-velocity workload (NH lambda = 1.5, mu = 0.75, omega = 2) at 256^2
    after 1000 steps; the numbers are printed for the record."""
    from synth import fourier_periodic

    w = fourier_periodic(n=256)
    U0, _ = w.fields()
    case = Case(w.nx, w.ny, 1000, lam=w.lam, mu=w.mu, c=w.c, omega=w.omega, U0=U0)
    errs = check(case, storage)
    print("precision fourier 256^2 x 1000 storage", storage, {k: "%.3e" % v for k, v in errs.items()})

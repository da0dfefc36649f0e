"""One problem description run through both the CUDA library (C ABI via the
Python binding) and the FP64 oracle, for the parity tests."""
from dataclasses import dataclass, field

import numpy as np

from oracle import oracle as orc

LAW_IDS = {"SVK": (0, orc.SVK), "NH": (1, orc.NH), "LOGNH": (2, orc.LOGNH), "MR": (3, orc.MR),
           "YEOH": (4, orc.YEOH), "GENT": (5, orc.GENT)}
TIMEFN = {"const": 0, "linear_ramp": 1, "sin2_ramp": 2, "sin_pulse": 3, "ricker": 4}
KIND = {"periodic": 0, "velocity": 1, "traction": 2}


@dataclass
class Case:
    nx: int
    ny: int
    steps: int
    law: str = "NH"
    lam: float = 1.0
    mu: float = 0.5
    c: float = 5.0
    omega: float = 2.0
    dx: float = 1.0
    body: tuple = (0.0, 0.0)
    order: int = 2
    fb_mode: int = 0
    # edge -> (kind, value, timefn, tparams, profile or None)
    edges: dict = field(default_factory=dict)
    U0: np.ndarray = None
    u0: np.ndarray = None
    params: tuple = None  # closure parameters when not (lam, mu)

    def material(self):
        return list(self.params) if self.params is not None else [self.lam, self.mu]


def case_from_workload(w, steps=None):
    """A Case with the sizes, material, edges and initial fields of a
    synthetic Workload (NH closure)."""
    U0, u0 = w.fields()
    edges = {}
    for e, E in enumerate(w.edges):
        if E.kind != "periodic":
            edges[e] = (E.kind, E.value, E.timefn, E.tparams, E.profile)
    return Case(w.nx, w.ny, w.steps if steps is None else steps, lam=w.lam, mu=w.mu, c=w.c, omega=w.omega,
                dx=w.dx, body=w.body_force, edges=edges, U0=U0, u0=u0)


def smooth_field(nx, ny, seed, amp=0.02, modes=3, periodic=True):
    """Smooth initial state around F = I, v = 0 from a seeded stream."""
    from synth import splitmix64_uniform

    r = splitmix64_uniform(seed, 6 * modes * 4)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y, indexing="xy")
    U0 = np.zeros((6, ny, nx))
    U0[2] = U0[5] = 1.0
    i = 0
    for comp in range(6):
        for _ in range(modes):
            kx = int(r[i] * 5) - 2
            ky = int(r[i + 1] * 5) - 2
            ph = 2 * np.pi * r[i + 2]
            a = amp * (2 * r[i + 3] - 1)
            i += 4
            if not periodic:  # any smooth field will do on a bounded domain
                kx, ky = kx + 0.37, ky - 0.21
            U0[comp] += a * np.cos(2 * np.pi * (kx * X + ky * Y) + ph)
    return U0


def run_gpu(case: Case, storage):
    from paper_2605_26677_gb300 import lbm

    L = lbm.Lattice(case.nx, case.ny, dx=case.dx, c=case.c, omega=case.omega, storage=storage,
                    fb_mode=case.fb_mode)
    try:
        lbm.lbm_set_material(L.ctx, LAW_IDS[case.law][0], case.material())
        lbm.lbm_set_body_force(L.ctx, *case.body)
        for e, (kind, val, tf, tp, prof) in case.edges.items():
            lbm.lbm_set_boundary(L.ctx, e, KIND[kind], val, TIMEFN[tf], tp, prof)
        lbm.lbm_init(L.ctx, case.U0, case.u0, case.order)
        lbm.lbm_step(L.ctx, case.steps)
        U, P, t = lbm.lbm_read_state(L.ctx)
        u = lbm.lbm_read_displacement(L.ctx)
        sigma = lbm.lbm_read_cauchy(L.ctx)
        diag = lbm.lbm_diagnostics(L.ctx)
    finally:
        L.close()
    return {"U": U, "P": P, "u": u, "sigma": sigma, "t": t, "diag": diag}


def run_oracle(case: Case):
    O = orc.Lattice(case.nx, case.ny, case.dx, case.c, case.omega)
    O.set_law(LAW_IDS[case.law][1], case.material())
    O.set_body_force(*case.body)
    O.set_fb_mode(case.fb_mode)
    for e, (kind, val, tf, tp, prof) in case.edges.items():
        O.set_edge(e, KIND[kind], val, TIMEFN[tf], tp if tp is not None else (0, 0, 0, 0), prof)
    O.init(case.U0, case.u0, case.order)
    O.step(case.steps)
    U, P, S = O.state()
    u = O.displacement()
    assert O.status == 0, O.status
    return {"U": U, "P": P, "u": u, "sigma": S, "t": O.time}


def rel(a, b):
    d = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (d if d > 0 else 1.0)


def group_errors(g, o):
    """Relative L2 errors per group: v, F - I, P, u, sigma, and the full state
    U (the paper's norm over all nodes and components)."""
    FI = np.array([1.0, 0.0, 0.0, 1.0])[:, None, None]
    return {
        "v": rel(g["U"][:2], o["U"][:2]),
        "F-I": rel(g["U"][2:] - FI, o["U"][2:] - FI),
        "P": rel(g["P"], o["P"]),
        "u": rel(g["u"], o["u"]),
        "sigma": rel(g["sigma"], o["sigma"]),
        "U": rel(g["U"], o["U"]),
    }


# ---------------------------------------------------------------- 16-bit rounding model
HALF_BITS = {2: 8, 3: 11}  # storage id -> significand bits: BF16 8, FP16 11


def small_strain_modulus(law, prm):
    """lambda + 2 mu_0 (mu_0 the small-strain shear modulus) of a closure's
    parameters as lbm_set_material lists them: the largest factor between a
    strain error and the stress error it makes near the rest state."""
    if law in ("SVK", "NH", "LOGNH", "GENT"):
        return prm[0] + 2.0 * prm[1]
    if law == "MR":
        return prm[0] + 4.0 * (prm[1] + prm[2])
    if law == "YEOH":
        return prm[0] + 4.0 * prm[1]
    raise ValueError(law)


def rounding_scales(U, P, c, modulus):
    """Per-group ratio of the stored offsets' size to the group's size.

    The 16-bit formats store f_q - f_rest; by Eq. (12) those offsets are of
    the size of (U - U_rest)/4 and Phi/(2c), Phi holding v and P. Rounding
    each stored value to a relative 2^-p once per step moves a state
    component by about 2^-p times that size per step, as a random walk over
    n steps; relative to a group g that is 2^-p sqrt(n) s_g with
      s_g = ||(v, F - I, P/c)|| / ||g||      for v, F - I and the full state U,
      s_P = s_sigma = that times (lambda + 2 mu_0) ||F - I|| / ||P|| read
            through the stress (a strain error e gives a stress error up to
            (lambda + 2 mu_0) e),
      s_u = the larger of s_v and s_(F-I) (u integrates v and F is its
            gradient).
    U, P: (6|4, ...) arrays of the reference state (any array module with
    .sum and elementwise ops)."""
    import math

    v2 = float((U[:2] ** 2).sum())
    g2 = float(((U[2] - 1.0) ** 2).sum() + (U[3] ** 2).sum() + (U[4] ** 2).sum() + ((U[5] - 1.0) ** 2).sum())
    p2 = float((P ** 2).sum())
    u2 = float((U ** 2).sum())
    off = math.sqrt(v2 + g2 + p2 / (c * c))
    sv, sg = off / math.sqrt(v2), off / math.sqrt(g2)
    sp = off * modulus / math.sqrt(p2)
    return {"v": sv, "F-I": sg, "P": sp, "sigma": sp, "u": max(sv, sg), "U": off / math.sqrt(u2)}


def tol_16bit(storage, steps, scales, C=1.5):
    """Bound C 2^-p sqrt(n) s_g per group (rounding_scales). The measured
    errors of every 16-bit parity case sit at 0.02 to 0.55 of 2^-p sqrt(n)
    s_g, so C = 1.5 is about three times the largest of them."""
    e = 2.0 ** -HALF_BITS[storage] * max(steps, 1) ** 0.5
    return {g: C * e * s for g, s in scales.items()}

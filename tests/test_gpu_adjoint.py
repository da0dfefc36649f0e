"""Per-node material fields and the adjoint through the C ABI.

Forward with a shear-modulus field against the FP64 oracle (every storage
type, with test_gpu_parity's bounds); the GPU
gradients (FP64 and FP32 storage) against the oracle's reference adjoint on
lattices that span several warp segments with a ragged tail; independence of
the checkpoint interval (recomputed segments are bit-identical); central
finite differences of the GPU's own FP64 forward loss; the autograd wrapper;
and the full 1024^2 x 2000-step workload against central differences (h =
1e-3) along 16 random directions with an FP64 forward.

Tolerances. FP64 storage: the gradients are sums over the run of products
of quantities each within about 1e-12 (relative) of the oracle's; 1e-9
relative L2 per gradient field leaves three orders of magnitude for their
accumulation. FP32 storage: the adjoint recursion is linear in the forward
state, whose per-group FP32 bound is 1e-5 (tests/test_gpu_parity.py), and
the adjoint itself is computed in FP32 with the same rounding per step and
sums those products over the run; the gradient fields get 1e-4 relative L2
(measured: 7e-6 for mu, 6e-6 for v0)."""
import numpy as np
import pytest

from tests.cases import KIND, LAW_IDS

pytestmark = pytest.mark.gpu

F64, F32, BF16, F16 = 0, 1, 2, 3


@pytest.fixture(scope="module")
def lbm():
    import torch

    assert torch.cuda.is_available()
    from paper_2605_26677_gb300 import build

    build.build()
    from paper_2605_26677_gb300 import lbm as m

    return m


def small_workload(n=None, nx=133, ny=19, steps=120):
    """A ragged-size version of the differentiation workload. Three sensors
    sit midway (reached by the pulse early), three on the traction edge; the
    run is long enough for the pulse to reach the edge, so that the mu
    gradient is not a cancellation-level residue (with the wave still short of
    every sensor it is ~1e-10 of its natural scale and only rounding is
    compared)."""
    from synth.generators import adjoint_specimen

    w = adjoint_specimen(n=max(nx, ny), steps=steps, nsens=6, record_every=10, corr=4.0)
    # crop the square fields to nx x ny
    p = w.params
    w.nx, w.ny = nx, ny
    p["mu"] = p["mu"][:ny, :nx].copy()
    p["sensors"] = np.array([[nx // 2, (j * ny) // 3 + 1] for j in range(3)] +
                            [[nx - 1, (j * ny) // 3 + 2] for j in range(3)], dtype=np.int32)
    p["radius"] = nx / 8.0
    p["target"] = p["target"][:, :6, :].copy()
    return w


def gpu_ctx(lbm, w, storage):
    L = lbm.Lattice(w.nx, w.ny, dx=w.dx, c=w.c, omega=w.omega, storage=storage)
    lbm.lbm_set_material_field(L.ctx, LAW_IDS["NH"][0], w.params["mu"], w.params["lam_ratio"])
    for e, E in enumerate(w.edges):
        lbm.lbm_set_boundary(L.ctx, e, KIND[E.kind], E.value)
    return L


def oracle_lattice(w):
    from oracle import oracle as orc

    O = orc.Lattice(w.nx, w.ny, w.dx, w.c, w.omega)
    O.set_law(orc.NH, [1.0, 1.0])
    O.set_material_field(w.params["mu"], w.params["lam_ratio"])
    for e, E in enumerate(w.edges):
        O.set_edge(e, KIND[E.kind], E.value)
    return O


def gpu_gradients(lbm, w, storage, checkpoint_every=0, U0=None):
    import torch

    L = gpu_ctx(lbm, w, storage)
    A = lbm.lbm_adjoint_create(L.ctx, w.steps, checkpoint_every)
    try:
        p = w.params
        lbm.lbm_adjoint_set_loss(A, p["sensors"], p["records"], p["target"])
        if U0 is None:
            U0, _ = w.fields()
        U0d = torch.from_numpy(np.ascontiguousarray(U0)).cuda()
        loss = lbm.lbm_adjoint_forward(A, U0d)
        gmu = torch.zeros((w.ny, w.nx), dtype=torch.float64, device="cuda")
        gv0 = torch.zeros((2, w.ny, w.nx), dtype=torch.float64, device="cuda")
        lbm.lbm_adjoint_backward(A, gmu, gv0)
        info = lbm.lbm_adjoint_info(A)
    finally:
        lbm.lbm_adjoint_destroy(A)
        L.close()
    return loss, gmu.cpu().numpy(), gv0.cpu().numpy(), info


def oracle_gradients(w):
    O = oracle_lattice(w)
    p = w.params
    U0, _ = w.fields()
    sens = p["sensors"][:, 1].astype(np.int64) * w.nx + p["sensors"][:, 0]
    return O.adjoint(U0, w.steps, sens, p["records"], p["target"])


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("storage", [F64, F32, BF16, F16])
def test_material_field_forward_matches_oracle(lbm, storage):
    from tests.cases import group_errors
    from tests.test_gpu_parity import tol_for

    w = small_workload(steps=120)
    U0, _ = w.fields()
    L = gpu_ctx(lbm, w, storage)
    lbm.lbm_init(L.ctx, U0)
    lbm.lbm_step(L.ctx, w.steps)
    U, P, _ = lbm.lbm_read_state(L.ctx)
    u = lbm.lbm_read_displacement(L.ctx)
    L.close()
    O = oracle_lattice(w)
    O.init(U0)
    O.step(w.steps)
    Uo, Po, So = O.state()
    errs = group_errors({"U": U, "P": P, "u": u, "sigma": So}, {"U": Uo, "P": Po, "u": O.displacement(), "sigma": So})
    print("ADJFWD storage=%d" % storage, {k: "%.2e" % v for k, v in errs.items()})
    tol = tol_for(storage, w.steps, {"U": Uo, "P": Po}, w.c,
                  (w.params["lam_ratio"] + 2.0) * float(np.max(w.params["mu"])))
    for k in ("v", "F-I", "P", "u", "U"):
        assert errs[k] <= tol[k], (k, errs)


@pytest.mark.parametrize("storage", [F64, F32])
def test_adjoint_matches_oracle(lbm, storage):
    w = small_workload()
    loss, gmu, gv0, _ = gpu_gradients(lbm, w, storage)
    Lo, gmu_o, gv0_o = oracle_gradients(w)
    tol = 1e-9 if storage == F64 else 1e-4
    e_mu, e_v = rel(gmu, gmu_o), rel(gv0, gv0_o)
    print("adjoint vs oracle storage", storage, "loss %.3e" % abs(loss - Lo), "mu %.2e v0 %.2e" % (e_mu, e_v))
    assert abs(loss - Lo) <= (1e-12 if storage == F64 else 1e-5) * abs(Lo)
    assert e_mu <= tol and e_v <= tol


@pytest.mark.parametrize("storage", [F64, F32])
def test_checkpoint_interval_does_not_change_the_gradient(lbm, storage):
    w = small_workload(steps=45)
    ref = gpu_gradients(lbm, w, storage, checkpoint_every=1)
    for K in (7, 0, 45, 100):
        got = gpu_gradients(lbm, w, storage, checkpoint_every=K)
        assert got[0] == ref[0]
        assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2]), K


@pytest.mark.parametrize("order", ["1", "4"])
def test_dynamic_task_order_does_not_change_the_gradient(lbm, monkeypatch, order):
    """The FP32 adjoint kernel in dynamic task order (LBM_ADJ_DYN: one
    counter or four stripes) gives the gradient of the static order bit for
    bit, with and without checkpointing (the side stream's recomputation in
    between the adjoint launches)."""
    w = small_workload(nx=300, ny=37, steps=45)
    for K in (1, 0):
        monkeypatch.setenv("LBM_ADJ_DYN", "0")
        ref = gpu_gradients(lbm, w, F32, checkpoint_every=K)
        monkeypatch.setenv("LBM_ADJ_DYN", order)
        got = gpu_gradients(lbm, w, F32, checkpoint_every=K)
        assert got[0] == ref[0]
        assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2]), K


def test_gradient_matches_central_differences_of_the_gpu_forward(lbm):
    import torch

    w = small_workload(nx=200, ny=90, steps=300)
    loss, gmu, gv0, _ = gpu_gradients(lbm, w, F64)
    U0, _ = w.fields()
    L = gpu_ctx(lbm, w, F64)
    A = lbm.lbm_adjoint_create(L.ctx, w.steps)
    p = w.params
    lbm.lbm_adjoint_set_loss(A, p["sensors"], p["records"], p["target"])
    rng = np.random.default_rng(4)
    mu0 = p["mu"].copy()
    try:
        for _ in range(4):
            dmu = rng.standard_normal(mu0.shape) * mu0
            dv = rng.standard_normal((2, w.ny, w.nx)) * 0.01
            h = 1e-5

            def f(s):
                lbm.lbm_set_material_field(L.ctx, 1, mu0 + s * h * dmu, 2.0)
                U = U0.copy()
                U[:2] += s * h * dv
                return lbm.lbm_adjoint_forward(A, torch.from_numpy(U).cuda())

            fd = (f(1) - f(-1)) / (2 * h)
            ad = float((gmu * dmu).sum() + (gv0 * dv).sum())
            assert abs(ad - fd) <= 1e-6 * abs(fd), (ad, fd)
    finally:
        lbm.lbm_adjoint_destroy(A)
        L.close()


def test_autograd_function(lbm):
    import torch

    from paper_2605_26677_gb300.autograd import SensorMisfit

    w = small_workload(steps=40)
    loss, gmu, gv0, _ = gpu_gradients(lbm, w, F64)
    U0, _ = w.fields()
    mu = torch.from_numpy(w.params["mu"]).cuda().requires_grad_(True)
    v0 = torch.from_numpy(np.ascontiguousarray(U0[:2])).cuda().requires_grad_(True)
    fn = SensorMisfit.from_workload(w, storage=F64)
    try:
        L = fn(mu, v0)
        L.backward()
    finally:
        fn.close()
    assert float(L) == loss
    assert np.array_equal(mu.grad.cpu().numpy(), gmu)
    assert np.array_equal(v0.grad.cpu().numpy(), gv0)


def test_material_field_from_device_equals_host(lbm):
    import torch

    w = small_workload(steps=30)
    U0, _ = w.fields()
    out = []
    for dev in (False, True):
        L = gpu_ctx(lbm, w, F32)
        if dev:
            lbm.lbm_set_material_field_device(L.ctx, 1, torch.from_numpy(w.params["mu"]).cuda(), 2.0)
        lbm.lbm_init(L.ctx, U0)
        lbm.lbm_step(L.ctx, w.steps)
        out.append(lbm.lbm_read_state(L.ctx, want_P=False)[0])
        L.close()
    assert np.array_equal(out[0], out[1])
    L = gpu_ctx(lbm, w, F32)
    for bad in (-1.0, np.nan, 0.0):
        mu = w.params["mu"].copy()
        mu[3, 5] = bad
        with pytest.raises(lbm.LbmError, match="LBM_ERR_ARG"):
            lbm.lbm_set_material_field_device(L.ctx, 1, torch.from_numpy(mu).cuda(), 2.0)
    L.close()


def test_adjoint_argument_errors(lbm):
    w = small_workload(steps=10)
    L = lbm.Lattice(w.nx, w.ny, c=w.c, storage=F32)
    lbm.lbm_set_material(L.ctx, 1, [2.0, 1.0])
    with pytest.raises(lbm.LbmError, match="LBM_ERR_STATE"):
        lbm.lbm_adjoint_create(L.ctx, 10)  # no material field
    L.close()
    L = lbm.Lattice(w.nx, w.ny, c=w.c, storage=lbm.LBM_STORE_BF16)
    lbm.lbm_set_material_field(L.ctx, 1, w.params["mu"], 2.0)  # a field steps in every storage
    with pytest.raises(lbm.LbmError, match="LBM_ERR_UNSUPPORTED"):
        lbm.lbm_adjoint_create(L.ctx, 10)  # the adjoint needs FP64 or FP32
    L.close()
    L = gpu_ctx(lbm, w, F32)
    A = lbm.lbm_adjoint_create(L.ctx, 10)
    import torch

    g1 = torch.zeros((w.ny, w.nx), dtype=torch.float64, device="cuda")
    g2 = torch.zeros((2, w.ny, w.nx), dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LbmError, match="LBM_ERR_STATE"):
        lbm.lbm_adjoint_backward(A, g1, g2)  # no forward
    with pytest.raises(lbm.LbmError, match="LBM_ERR_ARG"):
        lbm.lbm_adjoint_set_loss(A, [[w.nx, 0]], [5], np.zeros((1, 1, 2)))  # sensor outside
    with pytest.raises(lbm.LbmError, match="LBM_ERR_ARG"):
        lbm.lbm_adjoint_set_loss(A, [[0, 0]], [11], np.zeros((1, 1, 2)))  # step beyond nsteps
    with pytest.raises(lbm.LbmError, match="LBM_ERR_ARG"):
        lbm.lbm_adjoint_set_loss(A, [[0, 0], [0, 0]], [5], np.zeros((1, 2, 2)))  # sensor twice
    lbm.lbm_adjoint_set_loss(A, [[w.nx - 1, 3]], [5, 10], np.zeros((2, 1, 2)))
    U0, _ = w.fields()
    lbm.lbm_adjoint_forward(A, torch.from_numpy(U0).cuda())
    lbm.lbm_step(L.ctx, 1)  # the context moved on
    with pytest.raises(lbm.LbmError, match="LBM_ERR_STATE"):
        lbm.lbm_adjoint_backward(A, g1, g2)
    lbm.lbm_adjoint_destroy(A)
    L.close()


# ---------------------------------------------------------------- full size
@pytest.mark.slow
def test_full_size_gradient_against_central_differences(lbm):
    """1024^2, 2000 steps, FP32 adjoint with sqrt(N) checkpoints, against
    central differences (h = 1e-3, relative to mu and to the pulse amplitude)
    of the FP64 forward loss along 16 random directions: agreement within
    1e-4 of the directional derivative's scale (the largest |FD| of the 16)."""
    import torch

    from synth.generators import adjoint_specimen

    w = adjoint_specimen()
    loss32, gmu, gv0, info = gpu_gradients(lbm, w, F32)
    print("full size: loss", loss32, info)
    U0, _ = w.fields()
    L = gpu_ctx(lbm, w, F64)
    A = lbm.lbm_adjoint_create(L.ctx, w.steps)  # only its forward (the loss) is used
    p = w.params
    lbm.lbm_adjoint_set_loss(A, p["sensors"], p["records"], p["target"])
    rng = np.random.default_rng(16)
    mu0 = p["mu"]
    h = 1e-3
    fds, ads = [], []
    try:
        for _ in range(16):
            dmu = rng.standard_normal(mu0.shape) * mu0
            dv = rng.standard_normal((2, w.ny, w.nx)) * 0.01

            def f(s):
                lbm.lbm_set_material_field(L.ctx, 1, mu0 + s * h * dmu, 2.0)
                U = U0.copy()
                U[:2] += s * h * dv
                return lbm.lbm_adjoint_forward(A, torch.from_numpy(U).cuda())

            fds.append((f(1) - f(-1)) / (2 * h))
            ads.append(float((gmu * dmu).sum() + (gv0 * dv).sum()))
    finally:
        lbm.lbm_adjoint_destroy(A)
        L.close()
    fds, ads = np.array(fds), np.array(ads)
    scale = np.abs(fds).max()
    print("FD vs adjoint: max |diff| / scale = %.2e" % (np.abs(fds - ads).max() / scale))
    assert np.abs(fds - ads).max() <= 1e-4 * scale

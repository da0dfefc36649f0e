"""C-ABI behaviour on the GPU: call order, argument and capacity errors, the
latched device status (J <= 0, Newton failure, non-finite state) with the
state still readable afterwards, device-pointer entry points, checkpoints,
profiling counters."""
import numpy as np
import pytest

from tests.cases import Case, run_oracle, smooth_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch

    assert torch.cuda.is_available()
    from paper_2605_26677_gb300 import build

    build.build()
    from paper_2605_26677_gb300 import lbm as m

    return m


def make(lbm, nx=24, ny=16, storage=1, **kw):
    L = lbm.Lattice(nx, ny, storage=storage, **kw)
    lbm.lbm_set_material(L.ctx, lbm.LBM_LAW_NH, [1.0, 0.5])
    return L


def rest(nx, ny):
    U0 = np.zeros((6, ny, nx))
    U0[2] = U0[5] = 1.0
    return U0


def test_call_order(lbm):
    L = make(lbm)
    with pytest.raises(lbm.LbmError, match="LBM_ERR_STATE"):
        lbm.lbm_step(L.ctx, 1)
    with pytest.raises(lbm.LbmError, match="LBM_ERR_STATE"):
        lbm.lbm_read_state(L.ctx)
    lbm.lbm_init(L.ctx, rest(24, 16))
    lbm.lbm_set_material(L.ctx, lbm.LBM_LAW_NH, [1.0, 0.5])  # allowed: applies from the next step
    with pytest.raises(lbm.LbmError, match="LBM_ERR_STATE"):
        lbm.lbm_set_body_force(L.ctx, 0.0, 1.0)
    with pytest.raises(lbm.LbmError, match="LBM_ERR_ARG"):
        lbm.lbm_step(L.ctx, -1)
    lbm.lbm_step(L.ctx, 0)
    L.close()
    L = lbm.Lattice(8, 8)
    with pytest.raises(lbm.LbmError, match="LBM_ERR_STATE"):
        lbm.lbm_init(L.ctx, rest(8, 8))  # no material
    L.close()


def test_argument_checks(lbm):
    L = make(lbm)
    for law, bad in ((lbm.LBM_LAW_GENT, [1.0, 0.5]), (lbm.LBM_LAW_GENT, [1.0, 0.5, -1.0]),
                     (lbm.LBM_LAW_MR, [1.0, -0.1, 0.2]), (lbm.LBM_LAW_YEOH, [1.0, 0.5, 0.1]),
                     (lbm.LBM_LAW_NH, [1.0, -0.5]), (7, [1.0, 0.5])):
        with pytest.raises(lbm.LbmError, match="LBM_ERR_ARG"):
            lbm.lbm_set_material(L.ctx, law, bad)
    lbm.lbm_set_material(L.ctx, lbm.LBM_LAW_GENT, [1.0, 0.5, 10.0])
    lbm.lbm_set_material(L.ctx, lbm.LBM_LAW_NH, [1.0, 0.5])
    with pytest.raises(lbm.LbmError, match="LBM_ERR_ARG"):
        lbm.lbm_set_boundary(L.ctx, 4, lbm.LBM_BC_VELOCITY)
    with pytest.raises(lbm.LbmError, match="LBM_ERR_ARG"):
        lbm.lbm_set_boundary(L.ctx, 0, lbm.LBM_BC_VELOCITY, (np.nan, 0.0))
    with pytest.raises(lbm.LbmError, match="LBM_ERR_ARG"):
        lbm.lbm_set_boundary(L.ctx, 0, lbm.LBM_BC_VELOCITY, (0.0, 0.0), lbm.LBM_T_SIN2_RAMP, (0.0,))
    # unpaired periodic edge
    lbm.lbm_set_boundary(L.ctx, lbm.LBM_EDGE_LEFT, lbm.LBM_BC_VELOCITY)
    with pytest.raises(lbm.LbmError, match="LBM_ERR_ARG"):
        lbm.lbm_init(L.ctx, rest(24, 16))
    lbm.lbm_set_boundary(L.ctx, lbm.LBM_EDGE_RIGHT, lbm.LBM_BC_TRACTION)
    lbm.lbm_init(L.ctx, rest(24, 16))
    L.close()
    # lattice slower than the P wave: c <= sqrt(lambda + 2 mu)
    L = lbm.Lattice(8, 8, c=1.0)
    lbm.lbm_set_material(L.ctx, lbm.LBM_LAW_NH, [1.0, 0.5])
    with pytest.raises(lbm.LbmError, match="LBM_ERR_ARG"):
        lbm.lbm_init(L.ctx, rest(8, 8))
    L.close()
    # a non-periodic direction needs three nodes
    L = make(lbm, 2, 8)
    lbm.lbm_set_boundary(L.ctx, 0, lbm.LBM_BC_VELOCITY)
    lbm.lbm_set_boundary(L.ctx, 1, lbm.LBM_BC_VELOCITY)
    with pytest.raises(lbm.LbmError, match="LBM_ERR_ARG"):
        lbm.lbm_init(L.ctx, rest(2, 8))
    L.close()


def test_out_of_memory_is_reported(lbm):
    # 46000^2 nodes in FP64: two buffers of 24 planes need about 0.8 TB
    with pytest.raises(lbm.LbmError, match="LBM_ERR_OOM"):
        lbm.lbm_create(46000, 46000, storage=lbm.LBM_STORE_F64)
    # the device is still usable afterwards
    L = make(lbm)
    lbm.lbm_init(L.ctx, rest(24, 16))
    lbm.lbm_step(L.ctx, 3)
    L.close()


def test_nonpositive_J_at_init(lbm):
    L = make(lbm, 12, 10)
    U0 = rest(12, 10)
    U0[2, 4, 5] = -0.5  # det F < 0 at one node
    with pytest.raises(lbm.LbmError, match="LBM_ERR_NONPOSITIVE_J"):
        lbm.lbm_init(L.ctx, U0)
    # the state is readable after the error (and the latch persists)
    with pytest.raises(lbm.LbmError, match="LBM_ERR_NONPOSITIVE_J"):
        lbm.lbm_read_state(L.ctx)
    lbm.lbm_init(L.ctx, rest(12, 10))  # init clears the latch
    lbm.lbm_step(L.ctx, 2)
    L.close()


def test_nonfinite_state(lbm):
    L = make(lbm, 12, 10)
    U0 = rest(12, 10)
    U0[0, 3, 3] = np.nan
    lbm.lbm_init(L.ctx, U0, order=0)
    with pytest.raises(lbm.LbmError, match="LBM_ERR_NONFINITE"):
        lbm.lbm_step(L.ctx, 1)
    U = np.empty((6, 10, 12))
    with pytest.raises(lbm.LbmError, match="LBM_ERR_NONFINITE"):
        lbm.lbm_read_state(L.ctx, U)
    assert np.isnan(U).any() and np.isfinite(U).any()
    L.close()


def test_newton_failure_on_unreachable_traction(lbm):
    # a traction of 1e12 cannot be met within 20 damped Newton steps from F = I
    from oracle import oracle as orc

    nx, ny = 12, 10
    L = make(lbm, nx, ny, storage=0)
    lbm.lbm_set_boundary(L.ctx, 0, lbm.LBM_BC_TRACTION, (1e12, 0.0))
    lbm.lbm_set_boundary(L.ctx, 1, lbm.LBM_BC_TRACTION, (1e12, 0.0))
    lbm.lbm_init(L.ctx, rest(nx, ny))
    with pytest.raises(lbm.LbmError, match="LBM_ERR_NEWTON"):
        lbm.lbm_step(L.ctx, 1)
    L.close()
    O = orc.Lattice(nx, ny, 1.0, 5.0, 2.0)
    O.set_law(orc.NH, [1.0, 0.5])
    O.set_edge(0, orc.TRACTION, (1e12, 0.0))
    O.set_edge(1, orc.TRACTION, (1e12, 0.0))
    O.init(rest(nx, ny))
    O.step(1)
    assert O.status & orc.NEWTON_FAIL


def test_device_pointer_entry_points(lbm):
    import torch

    nx, ny = 37, 21
    U0 = smooth_field(nx, ny, seed=2)
    u0 = 0.1 * smooth_field(nx, ny, seed=9)[:2]
    A = make(lbm, nx, ny, storage=0)
    lbm.lbm_init(A.ctx, U0, u0)
    lbm.lbm_step(A.ctx, 25)
    U, P, _ = lbm.lbm_read_state(A.ctx)
    u = lbm.lbm_read_displacement(A.ctx)
    B = make(lbm, nx, ny, storage=0)
    lbm.lbm_init_device(B.ctx, torch.from_numpy(U0).cuda(), torch.from_numpy(u0).cuda())
    lbm.lbm_step_async(B.ctx, 25)
    Ud = torch.empty((6, ny, nx), dtype=torch.float64, device="cuda")
    Pd = torch.empty((4, ny, nx), dtype=torch.float64, device="cuda")
    ud = torch.empty((2, ny, nx), dtype=torch.float64, device="cuda")
    lbm.lbm_read_state_device(B.ctx, Ud, Pd)
    lbm.lbm_read_displacement_device(B.ctx, ud)
    lbm.lbm_sync(B.ctx)
    assert np.array_equal(Ud.cpu().numpy(), U)
    assert np.array_equal(Pd.cpu().numpy(), P)
    assert np.array_equal(ud.cpu().numpy(), u)
    A.close()
    B.close()


@pytest.mark.parametrize("storage", [0, 1])
def test_checkpoint_roundtrip_is_exact(lbm, storage):
    nx, ny = 40, 22
    L = make(lbm, nx, ny, storage=storage)
    lbm.lbm_set_boundary(L.ctx, 0, lbm.LBM_BC_VELOCITY)
    lbm.lbm_set_boundary(L.ctx, 1, lbm.LBM_BC_TRACTION, (0.02, 0.0), lbm.LBM_T_SIN2_RAMP, (30.0,))
    lbm.lbm_init(L.ctx, smooth_field(nx, ny, seed=6, periodic=False))
    lbm.lbm_step(L.ctx, 17)
    blob = lbm.lbm_save(L.ctx)
    lbm.lbm_step(L.ctx, 23)
    Ua, _, ta = lbm.lbm_read_state(L.ctx)
    ua = lbm.lbm_read_displacement(L.ctx)
    lbm.lbm_load(L.ctx, blob)
    assert lbm.lbm_info(L.ctx)[0] == 17
    lbm.lbm_step(L.ctx, 23)
    Ub, _, tb = lbm.lbm_read_state(L.ctx)
    ub = lbm.lbm_read_displacement(L.ctx)
    assert ta == tb and np.array_equal(Ua, Ub) and np.array_equal(ua, ub)
    with pytest.raises(lbm.LbmError, match="LBM_ERR_ARG"):
        lbm.lbm_load(L.ctx, blob[:100])
    L.close()


@pytest.mark.parametrize("fb_mode", [0, 1])
def test_profile_counts_launches(lbm, fb_mode):
    """Node form: the step kernel writes the next step's ghost cells, so the
    ghost kernel runs once after initialization and again only after new edge
    data. Extrapolated form: the edge kernel runs before every step."""
    L = make(lbm, 300, 200, fb_mode=fb_mode)
    lbm.lbm_set_boundary(L.ctx, 0, lbm.LBM_BC_VELOCITY)
    lbm.lbm_set_boundary(L.ctx, 1, lbm.LBM_BC_TRACTION, (0.01, 0.0))
    lbm.lbm_init(L.ctx, rest(300, 200))
    lbm.lbm_profile(L.ctx, True)
    lbm.lbm_step(L.ctx, 7)
    lbm.lbm_set_boundary(L.ctx, 1, lbm.LBM_BC_TRACTION, (0.02, 0.0))
    lbm.lbm_step(L.ctx, 5)
    p = lbm.lbm_profile_read(L.ctx)
    assert p["step"][0] == 12 and p["edges"][0] == (2 if fb_mode == 0 else 12)
    assert p["step"][1] > 0 and p["edges"][1] > 0
    lbm.lbm_profile(L.ctx, False)
    assert lbm.lbm_bytes_per_node_update(L.ctx) == 224.0
    L.close()


def test_rest_state_is_exact_on_gpu(lbm):
    for storage in (0, 1):
        nx, ny = 77, 41
        L = make(lbm, nx, ny, storage=storage)
        for e, k in enumerate((1, 2, 2, 2)):
            lbm.lbm_set_boundary(L.ctx, e, k)
        lbm.lbm_init(L.ctx, rest(nx, ny))
        lbm.lbm_step(L.ctx, 100)
        U, P, _ = lbm.lbm_read_state(L.ctx)
        assert np.array_equal(U, rest(nx, ny)) and not P.any()
        L.close()


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_page_locked_host_arrays_give_the_same_results(lbm, storage):
    """Page-locked host arrays are written in place by the read-out kernels;
    pageable ones go through a device copy. Both routes give the same bits
    (and page-locked inputs to lbm_init the same state as pageable ones)."""
    import torch

    nx, ny = 150, 37
    U0 = smooth_field(nx, ny, seed=9, amp=0.04, periodic=False)
    u0 = 0.01 * smooth_field(nx, ny, seed=10)[:2]
    res = []
    for pinned in (False, True):
        L = make(lbm, nx, ny, storage=storage, omega=1.9)
        lbm.lbm_set_boundary(L.ctx, 0, lbm.LBM_BC_VELOCITY)
        lbm.lbm_set_boundary(L.ctx, 1, lbm.LBM_BC_TRACTION, (0.02, 0.01))
        if pinned:
            a = torch.from_numpy(U0).pin_memory().numpy()
            b = torch.from_numpy(u0).pin_memory().numpy()
            Uo = torch.full((6, ny, nx), np.nan, dtype=torch.float64).pin_memory().numpy()
            Po = torch.full((4, ny, nx), np.nan, dtype=torch.float64).pin_memory().numpy()
            uo = torch.full((2, ny, nx), np.nan, dtype=torch.float64).pin_memory().numpy()
            so = torch.full((4, ny, nx), np.nan, dtype=torch.float64).pin_memory().numpy()
        else:
            a, b = U0.copy(), u0.copy()
            Uo, Po, uo, so = (np.full((m, ny, nx), np.nan) for m in (6, 4, 2, 4))
        lbm.lbm_init(L.ctx, a, b, 2)
        lbm.lbm_step(L.ctx, 25)
        lbm.lbm_read_state(L.ctx, Uo, Po)
        lbm.lbm_read_displacement(L.ctx, uo)
        lbm.lbm_read_cauchy(L.ctx, so)
        res.append([np.array(x, copy=True) for x in (Uo, Po, uo, so)])
        L.close()
    for x, y in zip(*res):
        assert np.all(np.isfinite(x))
        assert np.array_equal(x.view(np.uint64), y.view(np.uint64))


@pytest.mark.parametrize("yper", [False, True])
def test_banded_host_init_equals_device_init(lbm, yper):
    """lbm_init copies a large host state in row bands, each band's
    initialization starting once the rows its stencils reach have arrived
    (periodic rows: the first band last). The state equals, bit for bit, that
    of lbm_init_device on the whole state already on the device, with and
    without u0, on a lattice above the banding threshold whose row count is
    not a multiple of the band count."""
    import torch

    nx, ny = 1100, 1203  # 6 x 8 B x 1.32 M nodes = 64 MB and more
    U0 = smooth_field(nx, ny, seed=21, amp=0.04, periodic=yper)
    u0 = 0.01 * smooth_field(nx, ny, seed=22)[:2]
    out = []
    for route in ("host", "device"):
        for with_u0 in (False, True):
            L = make(lbm, nx, ny, storage=1, omega=1.9)
            if not yper:
                lbm.lbm_set_boundary(L.ctx, lbm.LBM_EDGE_BOTTOM, lbm.LBM_BC_VELOCITY)
                lbm.lbm_set_boundary(L.ctx, lbm.LBM_EDGE_TOP, lbm.LBM_BC_TRACTION, (0.02, 0.01))
            uu = u0 if with_u0 else None
            if route == "host":
                lbm.lbm_init(L.ctx, torch.from_numpy(U0).pin_memory().numpy(), uu, 2)
            else:
                lbm.lbm_init_device(L.ctx, torch.from_numpy(U0).cuda(),
                                    None if uu is None else torch.from_numpy(uu).cuda(), 2)
            lbm.lbm_step(L.ctx, 2)
            U, P, _ = lbm.lbm_read_state(L.ctx)
            out.append((U, P, lbm.lbm_read_displacement(L.ctx)))
            L.close()
    for x, y in zip(out[:2], out[2:]):
        for a, b in zip(x, y):
            assert np.all(np.isfinite(a))
            assert np.array_equal(a.view(np.uint64), b.view(np.uint64))


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_dynamic_and_static_task_order_give_the_same_bits(lbm, storage, monkeypatch):
    """The step kernels take their tasks in static grid-stride order or
    claim them dynamically from device counters (LBM_DYN=0 / 1 force one,
    LBM_DYN_STRIPES=1 / 4 the number of counters; otherwise the first
    lbm_step times the variants); a node's update does not depend on which
    warp runs it, so every order gives the same bits, over several steps
    (each dynamic launch uses the counter set the previous one zeroed) and
    with the variant choice's trial launches in between."""
    nx, ny = 300, 41
    U0 = smooth_field(nx, ny, seed=12, amp=0.04, periodic=False)
    runs = [("0", None), ("1", "4")] + ([("1", "1")] if storage >= 2 else [])
    res = []
    for dyn, ns in runs:
        monkeypatch.setenv("LBM_DYN", dyn)
        if ns is None:
            monkeypatch.delenv("LBM_DYN_STRIPES", raising=False)
        else:
            monkeypatch.setenv("LBM_DYN_STRIPES", ns)
        L = make(lbm, nx, ny, storage=storage, omega=1.9)
        lbm.lbm_set_boundary(L.ctx, 0, lbm.LBM_BC_VELOCITY)
        lbm.lbm_set_boundary(L.ctx, 1, lbm.LBM_BC_TRACTION, (0.02, 0.01))
        lbm.lbm_init(L.ctx, U0)
        for n in (1, 2, 7):
            lbm.lbm_step(L.ctx, n)
        v = lbm.lbm_step_variant(L.ctx)
        assert v["dynamic"] == (0 if ns is None else int(ns))
        assert v["staged"] in ((0, 1) if dyn == "0" and storage >= 2 else (0,))
        U, P, _ = lbm.lbm_read_state(L.ctx)
        res.append((U, P, lbm.lbm_read_displacement(L.ctx)))
        L.close()
    for other in res[1:]:
        for x, y in zip(res[0], other):
            assert np.array_equal(x.view(np.uint64), y.view(np.uint64))


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_task_order_with_a_material_field(lbm, storage, monkeypatch):
    """Per-node material (the adjoint's forward): static and dynamic task
    order give the same bits, over several lbm_step calls and after the
    variant choice's trial launches."""
    nx, ny = 260, 33
    U0 = smooth_field(nx, ny, seed=31, amp=0.03, periodic=False)
    rng = np.random.default_rng(5)
    mu = 0.5 * np.exp(0.2 * rng.standard_normal((ny, nx)))
    res = []
    for dyn in ("0", "1"):
        monkeypatch.setenv("LBM_DYN", dyn)
        monkeypatch.delenv("LBM_DYN_STRIPES", raising=False)
        L = make(lbm, nx, ny, storage=storage, omega=1.9, c=6.0)
        lbm.lbm_set_material_field(L.ctx, lbm.LBM_LAW_NH, mu, 2.0)
        lbm.lbm_set_boundary(L.ctx, 0, lbm.LBM_BC_VELOCITY)
        lbm.lbm_set_boundary(L.ctx, 1, lbm.LBM_BC_TRACTION, (0.01, 0.0))
        lbm.lbm_init(L.ctx, U0)
        for n in (1, 4, 6):
            lbm.lbm_step(L.ctx, n)
        v = lbm.lbm_step_variant(L.ctx)
        assert (v["dynamic"] > 0) == (dyn == "1") and v["staged"] == 0
        U, P, _ = lbm.lbm_read_state(L.ctx)
        res.append((U, P, lbm.lbm_read_displacement(L.ctx)))
        L.close()
    for x, y in zip(*res):
        assert np.all(np.isfinite(x))
        assert np.array_equal(x.view(np.uint64), y.view(np.uint64))

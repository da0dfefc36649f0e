"""Python binding of the C ABI in include/lbm.h (argument marshalling only).

Every function has the name of the C entry point it calls. Host arrays are
numpy float64 arrays of shape (m, ny, nx); device arrays are torch CUDA
float64 tensors of the same shape. A non-OK status raises LbmError carrying
the status code and lbm_last_error(). All computation happens in the CUDA
library; if it is missing, importing this module fails.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblbm_gb300.so")

LBM_OK, LBM_ERR_ARG, LBM_ERR_STATE, LBM_ERR_OOM, LBM_ERR_CUDA, LBM_ERR_NONPOSITIVE_J, LBM_ERR_NEWTON, \
    LBM_ERR_NONFINITE, LBM_ERR_UNSUPPORTED = range(9)
STATUS_NAMES = ["LBM_OK", "LBM_ERR_ARG", "LBM_ERR_STATE", "LBM_ERR_OOM", "LBM_ERR_CUDA", "LBM_ERR_NONPOSITIVE_J",
                "LBM_ERR_NEWTON", "LBM_ERR_NONFINITE", "LBM_ERR_UNSUPPORTED"]
LBM_STORE_F64, LBM_STORE_F32, LBM_STORE_BF16, LBM_STORE_F16 = range(4)
LBM_EDGE_LEFT, LBM_EDGE_RIGHT, LBM_EDGE_BOTTOM, LBM_EDGE_TOP = range(4)
LBM_BC_PERIODIC, LBM_BC_VELOCITY, LBM_BC_TRACTION = range(3)
LBM_LAW_SVK, LBM_LAW_NH, LBM_LAW_LOGNH, LBM_LAW_MR, LBM_LAW_YEOH, LBM_LAW_GENT = range(6)
LBM_T_CONST, LBM_T_LINEAR_RAMP, LBM_T_SIN2_RAMP, LBM_T_SIN_PULSE, LBM_T_RICKER, LBM_T_TABLE = range(6)
LBM_FB_NODE, LBM_FB_EXTRAP2 = range(2)

# every symbol include/lbm.h declares
EXPORTS = ["lbm_create", "lbm_destroy", "lbm_last_error", "lbm_set_material", "lbm_set_material_field",
           "lbm_set_material_field_device",
           "lbm_set_body_force",
           "lbm_set_boundary", "lbm_set_boundary_table", "lbm_init", "lbm_init_device", "lbm_step", "lbm_step_async", "lbm_step_variant", "lbm_sync",
           "lbm_read_state", "lbm_read_state_device", "lbm_read_displacement", "lbm_read_displacement_device",
           "lbm_read_cauchy", "lbm_diagnostics", "lbm_save", "lbm_load", "lbm_info", "lbm_profile",
           "lbm_profile_read", "lbm_bytes_per_node_update", "lbm_diagnostics_state_noalloc",
           "lbm_batch_create", "lbm_batch_destroy", "lbm_batch_last_error", "lbm_batch_size_class",
           "lbm_batch_get_tiles", "lbm_batch_set_tile", "lbm_batch_get_task_orders",
           "lbm_batch_set_task_order", "lbm_batch_tune", "lbm_batch_step", "lbm_batch_info",
           "lbm_adjoint_create", "lbm_adjoint_destroy", "lbm_adjoint_last_error", "lbm_adjoint_set_loss",
           "lbm_adjoint_forward", "lbm_adjoint_backward", "lbm_adjoint_info"]
LBM_BATCH_MAX_MEMBERS = 4096
LBM_BATCH_CLASSES = 5


class lbm_config(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("dx", C.c_double), ("c", C.c_double),
                ("omega", C.c_double), ("storage", C.c_int32), ("fb_mode", C.c_int32),
                ("device", C.c_int32), ("stream", C.c_void_p)]


class Context:
    """Opaque context handle returned by lbm_create (passed to ctypes as the
    C pointer), with the lattice size for marshalling."""

    def __init__(self, handle, nx, ny):
        self._as_parameter_ = handle
        self.nx, self.ny = nx, ny


class LbmError(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__("%s: %s" % (name, message))


if not os.path.exists(LIB_PATH):
    raise ImportError("CUDA library %s is missing; build it with paper_2605_26677_gb300.build.build()" % LIB_PATH)

_lib = C.CDLL(LIB_PATH)
_dp = C.POINTER(C.c_double)
_ctx = C.c_void_p

_lib.lbm_create.argtypes = [C.POINTER(lbm_config), C.POINTER(C.c_void_p)]
_lib.lbm_destroy.argtypes = [_ctx]
_lib.lbm_destroy.restype = None
_lib.lbm_last_error.argtypes = [_ctx]
_lib.lbm_last_error.restype = C.c_char_p
_lib.lbm_set_material.argtypes = [_ctx, C.c_int32, _dp, C.c_int32]
_lib.lbm_set_material_field.argtypes = [_ctx, C.c_int32, _dp, C.c_double]
_lib.lbm_set_material_field_device.argtypes = [_ctx, C.c_int32, C.c_void_p, C.c_double]
_lib.lbm_set_body_force.argtypes = [_ctx, C.c_double, C.c_double]
_lib.lbm_set_boundary.argtypes = [_ctx, C.c_int32, C.c_int32, _dp, C.c_int32, _dp, _dp]
_lib.lbm_set_boundary_table.argtypes = [_ctx, C.c_int32, C.c_int32, _dp, _dp]
_lib.lbm_init.argtypes = [_ctx, C.c_void_p, C.c_void_p, C.c_int32]
_lib.lbm_init_device.argtypes = [_ctx, C.c_void_p, C.c_void_p, C.c_int32]
_lib.lbm_step.argtypes = [_ctx, C.c_int64]
_lib.lbm_step_async.argtypes = [_ctx, C.c_int64]
_lib.lbm_step_variant.argtypes = [_ctx, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
_lib.lbm_sync.argtypes = [_ctx]
_lib.lbm_read_state.argtypes = [_ctx, C.c_void_p, C.c_void_p, _dp]
_lib.lbm_read_state_device.argtypes = [_ctx, C.c_void_p, C.c_void_p]
_lib.lbm_read_displacement.argtypes = [_ctx, C.c_void_p]
_lib.lbm_read_displacement_device.argtypes = [_ctx, C.c_void_p]
_lib.lbm_read_cauchy.argtypes = [_ctx, C.c_void_p]
_lib.lbm_diagnostics.argtypes = [_ctx, _dp]
_lib.lbm_save.argtypes = [_ctx, C.c_void_p, C.POINTER(C.c_size_t)]
_lib.lbm_load.argtypes = [_ctx, C.c_void_p, C.c_size_t]
_lib.lbm_info.argtypes = [_ctx, C.POINTER(C.c_int64), _dp, _dp]
_lib.lbm_profile.argtypes = [_ctx, C.c_int32]
_lib.lbm_profile_read.argtypes = [_ctx, _dp]
_lib.lbm_bytes_per_node_update.argtypes = [_ctx]
_lib.lbm_bytes_per_node_update.restype = C.c_double
_lib.lbm_diagnostics_state_noalloc.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, _dp, C.c_int32,
                                               C.c_double, C.c_void_p, C.c_int32, C.c_void_p]


_ip = C.POINTER(C.c_int32)
_lib.lbm_batch_create.argtypes = [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_void_p)]
_lib.lbm_batch_destroy.argtypes = [C.c_void_p]
_lib.lbm_batch_destroy.restype = None
_lib.lbm_batch_last_error.argtypes = [C.c_void_p]
_lib.lbm_batch_last_error.restype = C.c_char_p
_lib.lbm_batch_size_class.argtypes = [C.c_int32]
_lib.lbm_batch_size_class.restype = C.c_int32
_lib.lbm_batch_get_tiles.argtypes = [C.c_void_p, _ip]
_lib.lbm_batch_set_tile.argtypes = [C.c_void_p, C.c_int32, C.c_int32]
_lib.lbm_batch_get_task_orders.argtypes = [C.c_void_p, _ip]
_lib.lbm_batch_set_task_order.argtypes = [C.c_void_p, C.c_int32, C.c_int32]
_lib.lbm_batch_tune.argtypes = [C.c_void_p, C.c_int32, _dp]
_lib.lbm_batch_step.argtypes = [C.c_void_p, C.c_int64, C.c_int32, _ip]
_lib.lbm_batch_info.argtypes = [C.c_void_p, C.POINTER(C.c_int64), _ip, _ip]


_lib.lbm_adjoint_create.argtypes = [_ctx, C.c_int64, C.c_int32, C.POINTER(C.c_void_p)]
_lib.lbm_adjoint_destroy.argtypes = [C.c_void_p]
_lib.lbm_adjoint_destroy.restype = None
_lib.lbm_adjoint_last_error.argtypes = [C.c_void_p]
_lib.lbm_adjoint_last_error.restype = C.c_char_p
_lib.lbm_adjoint_set_loss.argtypes = [C.c_void_p, C.c_int32, _ip, C.c_int32, _ip, _dp]
_lib.lbm_adjoint_forward.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, _dp]
_lib.lbm_adjoint_backward.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
_lib.lbm_adjoint_info.argtypes = [C.c_void_p, _ip, C.POINTER(C.c_int64), _dp, _dp]


def library():
    """The loaded ctypes library (for symbol checks)."""
    return _lib


def _check(ctx, status):
    if status != LBM_OK:
        msg = _lib.lbm_last_error(ctx)
        raise LbmError(status, msg.decode() if msg else "")
    return status


def _host(a, shape=None):
    """Pointer to a C-contiguous float64 numpy array (checked, not copied)."""
    if a is None:
        return None
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags.c_contiguous:
        raise TypeError("expected a C-contiguous float64 numpy array")
    if shape is not None and a.size != int(np.prod(shape)):
        raise ValueError("expected %s elements, got %s" % (int(np.prod(shape)), a.size))
    return a.ctypes.data


def _dev(t, numel=None):
    """Device pointer of a contiguous float64 CUDA tensor."""
    if t is None:
        return None
    import torch

    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError("expected %d elements, got %d" % (numel, t.numel()))
    return t.data_ptr()


def _arr(v, n):
    if v is None:
        return None
    a = np.zeros(n, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64).ravel()
    a[: len(v)] = v
    return a


# ---------------------------------------------------------------- the ABI
def lbm_create(nx, ny, dx=1.0, c=5.0, omega=2.0, storage=LBM_STORE_F32, fb_mode=LBM_FB_NODE, device=0,
               stream=None):
    """Returns an opaque context handle. stream: a torch.cuda.Stream, an int
    handle, or None for the current torch stream of `device` if torch is
    initialised, else the default stream."""
    if stream is None:
        try:
            import torch

            stream = torch.cuda.current_stream(device).cuda_stream if torch.cuda.is_available() else 0
        except Exception:
            stream = 0
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    cfg = lbm_config(nx, ny, dx, c, omega, storage, fb_mode, device, C.c_void_p(stream or None))
    h = C.c_void_p()
    _check(None, _lib.lbm_create(C.byref(cfg), C.byref(h)))
    return Context(h, nx, ny)


def lbm_destroy(ctx):
    if ctx is not None and ctx._as_parameter_ is not None:
        _lib.lbm_destroy(ctx)
        ctx._as_parameter_ = None


def lbm_last_error(ctx=None):
    m = _lib.lbm_last_error(ctx)
    return m.decode() if m else ""


def lbm_set_material(ctx, law, params):
    p = np.asarray(params, dtype=np.float64)
    _check(ctx, _lib.lbm_set_material(ctx, law, p.ctypes.data_as(_dp), len(p)))


def lbm_set_material_field(ctx, law, mu, lam_ratio):
    """mu: (ny, nx) float64 host array; lambda = lam_ratio * mu per node."""
    m = np.ascontiguousarray(mu, dtype=np.float64)
    if m.size != ctx.nx * ctx.ny:
        raise ValueError("mu needs one value per node")
    _check(ctx, _lib.lbm_set_material_field(ctx, law, m.ctypes.data_as(_dp), float(lam_ratio)))


def lbm_set_material_field_device(ctx, law, mu_dev, lam_ratio):
    """mu_dev: (ny, nx) float64 CUDA tensor."""
    _check(ctx, _lib.lbm_set_material_field_device(ctx, law, _dev(mu_dev, ctx.nx * ctx.ny), float(lam_ratio)))


def lbm_set_body_force(ctx, b1, b2):
    _check(ctx, _lib.lbm_set_body_force(ctx, b1, b2))


def lbm_set_boundary(ctx, edge, bc, value=(0.0, 0.0), timefn=LBM_T_CONST, tparams=None, profile=None):
    v = _arr(value, 2)
    tp = _arr(tparams, 4)
    pr = None if profile is None else np.ascontiguousarray(profile, dtype=np.float64)
    if pr is not None and pr.size != (ctx.ny if edge in (LBM_EDGE_LEFT, LBM_EDGE_RIGHT) else ctx.nx):
        raise ValueError("profile needs one value per edge node")
    _check(ctx, _lib.lbm_set_boundary(ctx, edge, bc, v.ctypes.data_as(_dp), timefn,
                                      None if tp is None else tp.ctypes.data_as(_dp),
                                      None if pr is None else pr.ctypes.data_as(_dp)))


def lbm_set_boundary_table(ctx, edge, t, g):
    """Piecewise-linear g(t) through (t[i], g[i]) for an edge with LBM_T_TABLE."""
    t = np.ascontiguousarray(t, dtype=np.float64).ravel()
    g = np.ascontiguousarray(g, dtype=np.float64).ravel()
    if t.size != g.size:
        raise ValueError("t and g need the same length")
    _check(ctx, _lib.lbm_set_boundary_table(ctx, edge, t.size, t.ctypes.data_as(_dp), g.ctypes.data_as(_dp)))


def lbm_init(ctx, U0, u0=None, order=2):
    """U0: (6, ny, nx) float64 host array; u0: (2, ny, nx) or None."""
    U0 = np.ascontiguousarray(U0, dtype=np.float64)
    u0 = None if u0 is None else np.ascontiguousarray(u0, dtype=np.float64)
    _check(ctx, _lib.lbm_init(ctx, _host(U0), _host(u0), order))


def lbm_init_device(ctx, U0_dev, u0_dev=None, order=2):
    _check(ctx, _lib.lbm_init_device(ctx, _dev(U0_dev), _dev(u0_dev), order))


def lbm_step(ctx, nsteps):
    _check(ctx, _lib.lbm_step(ctx, int(nsteps)))


def lbm_step_async(ctx, nsteps):
    _check(ctx, _lib.lbm_step_async(ctx, int(nsteps)))


def lbm_step_variant(ctx):
    """{"staged": 0/1, "dynamic": 0/1}: the step-launch variant the context runs now."""
    st, dy = C.c_int32(), C.c_int32()
    _check(ctx, _lib.lbm_step_variant(ctx, C.byref(st), C.byref(dy)))
    return {"staged": st.value, "dynamic": dy.value}


def lbm_sync(ctx):
    _check(ctx, _lib.lbm_sync(ctx))


def _shape(ctx):
    return ctx.nx, ctx.ny


def lbm_read_state(ctx, U=None, P=None, want_P=True):
    """Returns (U (6,ny,nx), P (4,ny,nx) or None, t). Output arrays may be
    passed in (pinned host memory works)."""
    nx, ny = _shape(ctx)
    U = np.empty((6, ny, nx)) if U is None else U
    if want_P and P is None:
        P = np.empty((4, ny, nx))
    t = C.c_double()
    _check(ctx, _lib.lbm_read_state(ctx, _host(U, (6, ny, nx)), _host(P, (4, ny, nx)), C.byref(t)))
    return U, P, t.value


def lbm_read_state_device(ctx, U_dev, P_dev=None):
    nx, ny = _shape(ctx)
    _check(ctx, _lib.lbm_read_state_device(ctx, _dev(U_dev, 6 * nx * ny), _dev(P_dev, 4 * nx * ny)))


def lbm_read_displacement(ctx, u=None):
    nx, ny = _shape(ctx)
    u = np.empty((2, ny, nx)) if u is None else u
    _check(ctx, _lib.lbm_read_displacement(ctx, _host(u, (2, ny, nx))))
    return u


def lbm_read_displacement_device(ctx, u_dev):
    nx, ny = _shape(ctx)
    _check(ctx, _lib.lbm_read_displacement_device(ctx, _dev(u_dev, 2 * nx * ny)))


def lbm_read_cauchy(ctx, sigma=None):
    nx, ny = _shape(ctx)
    sigma = np.empty((4, ny, nx)) if sigma is None else sigma
    _check(ctx, _lib.lbm_read_cauchy(ctx, _host(sigma, (4, ny, nx))))
    return sigma


def lbm_diagnostics(ctx):
    out = np.zeros(10)
    _check(ctx, _lib.lbm_diagnostics(ctx, out.ctypes.data_as(_dp)))
    return out


def lbm_save(ctx):
    n = C.c_size_t(0)
    _check(ctx, _lib.lbm_save(ctx, None, C.byref(n)))
    buf = np.empty(n.value, dtype=np.uint8)
    _check(ctx, _lib.lbm_save(ctx, buf.ctypes.data, C.byref(n)))
    return buf


def lbm_load(ctx, buf):
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(ctx, _lib.lbm_load(ctx, buf.ctypes.data, buf.size))


def lbm_info(ctx):
    s, t, dt = C.c_int64(), C.c_double(), C.c_double()
    _check(ctx, _lib.lbm_info(ctx, C.byref(s), C.byref(t), C.byref(dt)))
    return s.value, t.value, dt.value


def lbm_profile(ctx, enable):
    _check(ctx, _lib.lbm_profile(ctx, 1 if enable else 0))


def lbm_profile_read(ctx):
    out = np.zeros(4)
    _check(ctx, _lib.lbm_profile_read(ctx, out.ctypes.data_as(_dp)))
    return {"step": (int(out[0]), out[1]), "edges": (int(out[2]), out[3])}


def lbm_bytes_per_node_update(ctx):
    return _lib.lbm_bytes_per_node_update(ctx)


def lbm_diagnostics_state_noalloc(U_dev, nx, ny, law, params, dx, out_dev, device=0, stream=None):
    """U_dev: (6, ny, nx) float64 CUDA tensor; out_dev: 10-element float64 CUDA
    tensor. Enqueued on `stream` (default: torch's current stream)."""
    if stream is None:
        import torch

        stream = torch.cuda.current_stream(device).cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    p = np.asarray(params, dtype=np.float64)
    st = _lib.lbm_diagnostics_state_noalloc(_dev(U_dev, 6 * nx * ny), nx, ny, law, p.ctypes.data_as(_dp), len(p),
                                            dx, _dev(out_dev, 10), device, C.c_void_p(stream or None))
    _check(None, st)


# ---------------------------------------------------------------- batches
class Batch:
    """Opaque batch handle returned by lbm_batch_create; keeps its members
    (Context objects) referenced."""

    def __init__(self, handle, members):
        self._as_parameter_ = handle
        self.members = list(members)


def _bcheck(b, status):
    if status != LBM_OK:
        msg = _lib.lbm_batch_last_error(b)
        raise LbmError(status, msg.decode() if msg else "")
    return status


def lbm_batch_create(members):
    """members: sequence of contexts (lbm_create handles)."""
    arr = (C.c_void_p * len(members))(*[m._as_parameter_ for m in members])
    h = C.c_void_p()
    _bcheck(None, _lib.lbm_batch_create(arr, len(members), C.byref(h)))
    return Batch(h, members)


def lbm_batch_destroy(b):
    if b is not None and b._as_parameter_ is not None:
        _lib.lbm_batch_destroy(b)
        b._as_parameter_ = None


def lbm_batch_last_error(b=None):
    m = _lib.lbm_batch_last_error(b)
    return m.decode() if m else ""


def lbm_batch_size_class(nx):
    return _lib.lbm_batch_size_class(int(nx))


def lbm_batch_get_tiles(b):
    v = (C.c_int32 * LBM_BATCH_CLASSES)()
    _bcheck(b, _lib.lbm_batch_get_tiles(b, v))
    return list(v)


def lbm_batch_set_tile(b, size_class, vec):
    _bcheck(b, _lib.lbm_batch_set_tile(b, int(size_class), int(vec)))


def lbm_batch_get_task_orders(b):
    v = (C.c_int32 * LBM_BATCH_CLASSES)()
    _bcheck(b, _lib.lbm_batch_get_task_orders(b, v))
    return list(v)


def lbm_batch_set_task_order(b, size_class, dynamic):
    _bcheck(b, _lib.lbm_batch_set_task_order(b, int(size_class), int(dynamic)))


def lbm_batch_tune(b, reps=20):
    """Returns (tiles per class, microseconds per launch [class][tile index])."""
    us = np.zeros(LBM_BATCH_CLASSES * 3)
    _bcheck(b, _lib.lbm_batch_tune(b, int(reps), us.ctypes.data_as(_dp)))
    return lbm_batch_get_tiles(b), us.reshape(LBM_BATCH_CLASSES, 3)


def lbm_batch_step(b, nsteps, graph_steps=0, raise_on_error=True):
    """Returns the per-member status list."""
    st = (C.c_int32 * len(b.members))()
    s = _lib.lbm_batch_step(b, int(nsteps), int(graph_steps), st)
    if raise_on_error:
        _bcheck(b, s)
    return list(st)


def lbm_batch_info(b):
    n, l, g = C.c_int64(), C.c_int32(), C.c_int32()
    _bcheck(b, _lib.lbm_batch_info(b, C.byref(n), C.byref(l), C.byref(g)))
    return {"nodes": n.value, "launches_per_step": l.value, "graphs": g.value}


# ---------------------------------------------------------------- adjoint
class Adjoint:
    """Opaque adjoint handle returned by lbm_adjoint_create; keeps its
    context referenced."""

    def __init__(self, handle, ctx, nsteps):
        self._as_parameter_ = handle
        self.ctx = ctx
        self.nsteps = nsteps


def _acheck(a, status):
    if status != LBM_OK:
        msg = _lib.lbm_adjoint_last_error(a)
        raise LbmError(status, msg.decode() if msg else "")
    return status


def lbm_adjoint_create(ctx, nsteps, checkpoint_every=0):
    h = C.c_void_p()
    _acheck(None, _lib.lbm_adjoint_create(ctx, int(nsteps), int(checkpoint_every), C.byref(h)))
    return Adjoint(h, ctx, nsteps)


def lbm_adjoint_destroy(a):
    if a is not None and a._as_parameter_ is not None:
        _lib.lbm_adjoint_destroy(a)
        a._as_parameter_ = None


def lbm_adjoint_last_error(a=None):
    m = _lib.lbm_adjoint_last_error(a)
    return m.decode() if m else ""


def lbm_adjoint_set_loss(a, sens_xy, rec_steps, target):
    """sens_xy: (nsens, 2) node (x, y); rec_steps: (nrec,); target: (nrec, nsens, 2)."""
    s = np.ascontiguousarray(sens_xy, dtype=np.int32).reshape(-1, 2)
    r = np.ascontiguousarray(rec_steps, dtype=np.int32).ravel()
    t = np.ascontiguousarray(target, dtype=np.float64)
    if t.size != len(r) * len(s) * 2:
        raise ValueError("target needs (nrec, nsens, 2) values")
    _acheck(a, _lib.lbm_adjoint_set_loss(a, len(s), s.ctypes.data_as(_ip), len(r), r.ctypes.data_as(_ip),
                                         t.ctypes.data_as(_dp)))


def lbm_adjoint_forward(a, U0_dev, order=2):
    """U0_dev: (6, ny, nx) float64 CUDA tensor. Returns the loss."""
    L = C.c_double()
    _acheck(a, _lib.lbm_adjoint_forward(a, _dev(U0_dev, 6 * a.ctx.nx * a.ctx.ny), int(order), C.byref(L)))
    return L.value


def lbm_adjoint_backward(a, g_mu_dev, g_v0_dev):
    """g_mu_dev: (ny, nx), g_v0_dev: (2, ny, nx) float64 CUDA tensors (written)."""
    N = a.ctx.nx * a.ctx.ny
    _acheck(a, _lib.lbm_adjoint_backward(a, _dev(g_mu_dev, N), _dev(g_v0_dev, 2 * N)))


def lbm_adjoint_info(a):
    k, n, f, b = C.c_int32(), C.c_int64(), C.c_double(), C.c_double()
    _acheck(a, _lib.lbm_adjoint_info(a, C.byref(k), C.byref(n), C.byref(f), C.byref(b)))
    return {"checkpoint_every": k.value, "stored_states": n.value, "forward_ms": f.value, "backward_ms": b.value}


# ---------------------------------------------------------------- helper
class Lattice:
    """Owning wrapper: creates a context and destroys it when collected."""

    def __init__(self, nx, ny, **cfg):
        self.ctx = lbm_create(nx, ny, **cfg)
        self.nx, self.ny = nx, ny

    def close(self):
        if getattr(self, "ctx", None) is not None:
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

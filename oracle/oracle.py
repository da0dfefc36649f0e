"""ctypes wrapper around the FP64 CPU oracle (``tlv_oracle.c``).

TEST INFRASTRUCTURE. The oracle is the parity reference for the CUDA library;
only the tests, the package smoke check and the benchmark's CPU-baseline leg
import this module. It never imports the product package and the product
package never imports it.

Array conventions follow ``tlv_oracle.h``: fields are ``(m, ny, nx)`` float64
arrays (component-major, x fastest); F is ``(F11, F12, F21, F22)``.
"""
import ctypes as C

import numpy as np

from . import build as _build

SVK, NH, LOGNH, MR, YEOH, GENT = range(6)
LEFT, RIGHT, BOTTOM, TOP = range(4)
PERIODIC, VELOCITY, TRACTION = range(3)
T_CONST, T_LINEAR_RAMP, T_SIN2_RAMP, T_SIN_PULSE, T_RICKER = range(5)
BAD_J, NEWTON_FAIL, NONFINITE = 1, 2, 4
FB_NODE, FB_EXTRAP2 = 0, 1

_lib = None
_dp = C.POINTER(C.c_double)


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = C.CDLL(path)
        lib.orc_set_threads.argtypes = [C.c_int]
        lib.orc_threads.restype = C.c_int
        lib.orc_new.restype = C.c_void_p
        lib.orc_new.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double]
        lib.orc_free.argtypes = [C.c_void_p]
        lib.orc_set_law.argtypes = [C.c_void_p, C.c_int, _dp, C.c_int]
        lib.orc_set_body_force.argtypes = [C.c_void_p, C.c_double, C.c_double]
        lib.orc_set_fb_mode.argtypes = [C.c_void_p, C.c_int]
        lib.orc_set_body_force_field.argtypes = [C.c_void_p, _dp]
        lib.orc_set_material_field.argtypes = [C.c_void_p, _dp, C.c_double]
        lib.orc_adjoint.argtypes = [C.c_void_p, _dp, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_long), C.c_int,
                                    C.POINTER(C.c_int), _dp, _dp, _dp, _dp]
        lib.orc_set_edge.argtypes = [C.c_void_p, C.c_int, C.c_int, _dp, C.c_int, _dp, _dp]
        lib.orc_set_edge_data.argtypes = [C.c_void_p, C.c_int, _dp]
        lib.orc_init.argtypes = [C.c_void_p, _dp, _dp, C.c_int, _dp, _dp]
        lib.orc_step.argtypes = [C.c_void_p, C.c_int]
        lib.orc_state.argtypes = [C.c_void_p, _dp, _dp, _dp]
        lib.orc_displacement.argtypes = [C.c_void_p, _dp]
        lib.orc_populations.argtypes = [C.c_void_p, _dp]
        lib.orc_set_populations.argtypes = [C.c_void_p, _dp]
        lib.orc_status.argtypes = [C.c_void_p]
        lib.orc_step_count.argtypes = [C.c_void_p]
        lib.orc_step_count.restype = C.c_long
        lib.orc_time.argtypes = [C.c_void_p]
        lib.orc_time.restype = C.c_double
        lib.orc_dt.argtypes = [C.c_void_p]
        lib.orc_dt.restype = C.c_double
        lib.orc_piola.argtypes = [C.c_int, _dp, _dp, _dp]
        lib.orc_piola_cplx.argtypes = [C.c_int, _dp, _dp, _dp, _dp, _dp]
        lib.orc_energy.argtypes = [C.c_int, _dp, _dp]
        lib.orc_energy.restype = C.c_double
        lib.orc_tangent.argtypes = [C.c_int, _dp, _dp, _dp]
        lib.orc_flux.argtypes = [_dp, _dp, _dp, _dp]
        lib.orc_feq.argtypes = [_dp, _dp, C.c_double, _dp]
        lib.orc_timefn.argtypes = [C.c_int, _dp, C.c_double]
        lib.orc_timefn.restype = C.c_double
        _lib = lib
    return _lib


def _p(a):
    """float64 C-contiguous array -> (pointer, keep-alive array); None -> NULL."""
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.ctypes.data_as(_dp), a


def _params(prm):
    a = np.zeros(8)
    a[: len(prm)] = prm
    return a


def set_threads(n):
    """OpenMP threads of the oracle's per-node loops (bit-identical results
    for any count)."""
    _load().orc_set_threads(int(n))


def threads():
    return _load().orc_threads()


# ---------------------------------------------------------------- pointwise
def piola(law, prm, F):
    lib = _load()
    P = np.zeros(4)
    pp, _k1 = _p(_params(prm))
    fp, _k2 = _p(F)
    rc = lib.orc_piola(law, pp, fp, P.ctypes.data_as(_dp))
    return P, rc


def piola_cplx(law, prm, Fre, Fim):
    lib = _load()
    Pre, Pim = np.zeros(4), np.zeros(4)
    pp, _k1 = _p(_params(prm))
    a, _k2 = _p(Fre)
    b, _k3 = _p(Fim)
    lib.orc_piola_cplx(law, pp, a, b, Pre.ctypes.data_as(_dp), Pim.ctypes.data_as(_dp))
    return Pre, Pim


def energy(law, prm, F):
    lib = _load()
    pp, _k1 = _p(_params(prm))
    fp, _k2 = _p(F)
    return lib.orc_energy(law, pp, fp)


def tangent(law, prm, F):
    """C[iA, kB] as a (4, 4) array, rows iA = 2i+A, columns kB = 2k+B."""
    lib = _load()
    Ct = np.zeros(16)
    pp, _k1 = _p(_params(prm))
    fp, _k2 = _p(F)
    lib.orc_tangent(law, pp, fp, Ct.ctypes.data_as(_dp))
    return Ct.reshape(4, 4)


def flux(U, P):
    lib = _load()
    X, Y = np.zeros(6), np.zeros(6)
    up, _k1 = _p(U)
    pp, _k2 = _p(P)
    lib.orc_flux(up, pp, X.ctypes.data_as(_dp), Y.ctypes.data_as(_dp))
    return X, Y


def feq(U, P, c):
    """(4, 6) equilibrium populations f^eq_q for q = (1,0),(0,1),(-1,0),(0,-1)."""
    lib = _load()
    out = np.zeros(24)
    up, _k1 = _p(U)
    pp, _k2 = _p(P)
    lib.orc_feq(up, pp, c, out.ctypes.data_as(_dp))
    return out.reshape(4, 6)


def timefn(kind, tp, t):
    lib = _load()
    a = np.zeros(4)
    a[: len(tp)] = tp
    tpp, _k = _p(a)
    return lib.orc_timefn(kind, tpp, t)


# ---------------------------------------------------------------- lattice
class Lattice:
    """One D2Q4x6 lattice on nx x ny cell-centred nodes (Sec. 3)."""

    def __init__(self, nx, ny, dx=1.0, c=5.0, omega=2.0):
        self._lib = _load()
        self.nx, self.ny, self.N = nx, ny, nx * ny
        self._h = self._lib.orc_new(nx, ny, dx, c, omega)
        if not self._h:
            raise ValueError("orc_new rejected nx=%d ny=%d dx=%g c=%g omega=%g" % (nx, ny, dx, c, omega))
        self.dx, self.c, self.omega = dx, c, omega
        self.dt = self._lib.orc_dt(self._h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_free(h)
            self._h = None

    def set_law(self, law, prm):
        a = _params(prm)
        if self._lib.orc_set_law(self._h, law, a.ctypes.data_as(_dp), len(prm)) != 0:
            raise ValueError("bad law")

    def set_fb_mode(self, mode):
        if self._lib.orc_set_fb_mode(self._h, mode) != 0:
            raise ValueError("bad F^b mode")

    def set_body_force(self, b1, b2):
        self._lib.orc_set_body_force(self._h, b1, b2)

    def set_body_force_field(self, b):
        p, _k = _p(None if b is None else np.asarray(b).reshape(2, self.ny, self.nx))
        self._lib.orc_set_body_force_field(self._h, p)

    def set_material_field(self, mu, lam_ratio):
        """Per-node shear modulus (ny, nx) with lambda = lam_ratio * mu (SVK, NH,
        LOGNH; after set_law); None reverts to the uniform parameters."""
        p, _k = _p(None if mu is None else np.asarray(mu).reshape(self.ny, self.nx))
        if self._lib.orc_set_material_field(self._h, p, lam_ratio) != 0:
            raise ValueError("bad material field")

    def adjoint(self, U0, nsteps, sens, rec_steps, target, order=2):
        """Reference adjoint of L = 1/2 sum_k sum_s |u(X_s, t^{n_k}) - d_{k,s}|^2.
        sens: node indices iy * nx + ix; rec_steps: recorded steps; target:
        (len(rec_steps), len(sens), 2). Returns (L, dL/dmu (ny, nx), dL/dv0
        (2, ny, nx))."""
        a, _k1 = _p(np.asarray(U0).reshape(6, self.ny, self.nx))
        sens = np.ascontiguousarray(sens, dtype=np.int64)
        rec = np.ascontiguousarray(rec_steps, dtype=np.int32)
        tg, _k2 = _p(np.asarray(target).reshape(len(rec), len(sens), 2))
        loss = np.zeros(1)
        gmu = np.zeros((self.ny, self.nx))
        gv0 = np.zeros((2, self.ny, self.nx))
        rc = self._lib.orc_adjoint(self._h, a, order, int(nsteps), len(sens),
                                   sens.ctypes.data_as(C.POINTER(C.c_long)), len(rec),
                                   rec.ctypes.data_as(C.POINTER(C.c_int)), tg, loss.ctypes.data_as(_dp),
                                   gmu.ctypes.data_as(_dp), gv0.ctypes.data_as(_dp))
        if rc != 0:
            raise RuntimeError("orc_adjoint failed with %d" % rc)
        return float(loss[0]), gmu, gv0

    def edge_len(self, e):
        return self.ny if e in (LEFT, RIGHT) else self.nx

    def set_edge(self, e, kind, value=(0.0, 0.0), timefn=T_CONST, tp=(0, 0, 0, 0), profile=None):
        v, _k1 = _p(np.asarray(value, dtype=np.float64))
        t4 = np.zeros(4)
        t4[: len(tp)] = tp
        tpp, _k2 = _p(t4)
        pr, _k3 = _p(None if profile is None else np.asarray(profile).reshape(self.edge_len(e)))
        if self._lib.orc_set_edge(self._h, e, kind, v, timefn, tpp, pr) != 0:
            raise ValueError("bad edge")

    def set_edge_data(self, e, vals):
        p, _k = _p(None if vals is None else np.asarray(vals).reshape(2, self.edge_len(e)))
        self._lib.orc_set_edge_data(self._h, e, p)

    def init(self, U0, u0=None, order=2, dUdX=None, dUdY=None):
        sh6 = (6, self.ny, self.nx)
        a, _k1 = _p(np.asarray(U0).reshape(sh6))
        b, _k2 = _p(None if u0 is None else np.asarray(u0).reshape(2, self.ny, self.nx))
        gx, _k3 = _p(None if dUdX is None else np.asarray(dUdX).reshape(sh6))
        gy, _k4 = _p(None if dUdY is None else np.asarray(dUdY).reshape(sh6))
        rc = self._lib.orc_init(self._h, a, b, order, gx, gy)
        if rc != 0:
            raise ValueError("orc_init failed with %d" % rc)

    def step(self, n=1):
        if self._lib.orc_step(self._h, int(n)) != 0:
            raise RuntimeError("orc_step before init")

    def state(self):
        """(U (6,ny,nx), P (4,ny,nx), sigma (4,ny,nx)) at the current time level."""
        U = np.zeros((6, self.ny, self.nx))
        P = np.zeros((4, self.ny, self.nx))
        S = np.zeros((4, self.ny, self.nx))
        self._lib.orc_state(self._h, U.ctypes.data_as(_dp), P.ctypes.data_as(_dp), S.ctypes.data_as(_dp))
        return U, P, S

    def displacement(self):
        u = np.zeros((2, self.ny, self.nx))
        self._lib.orc_displacement(self._h, u.ctypes.data_as(_dp))
        return u

    def populations(self):
        f = np.zeros((4, 6, self.ny, self.nx))
        self._lib.orc_populations(self._h, f.ctypes.data_as(_dp))
        return f

    def set_populations(self, f):
        p, _k = _p(np.asarray(f).reshape(4, 6, self.ny, self.nx))
        self._lib.orc_set_populations(self._h, p)

    @property
    def status(self):
        return self._lib.orc_status(self._h)

    @property
    def step_count(self):
        return self._lib.orc_step_count(self._h)

    @property
    def time(self):
        return self._lib.orc_time(self._h)


def node_coords(nx, ny, dx):
    """Cell-centred material coordinates X, Y of shape (ny, nx)."""
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dx
    return np.meshgrid(x, y, indexing="xy")

"""torch.autograd binding of the library's adjoint (argument marshalling only).

SensorMisfit(...)(mu, v0) returns the sensor-displacement misfit
L = 1/2 sum_k sum_s |u(X_s, t^{n_k}) - d_{k,s}|^2 of a run started from
U0 = (v0, F = I) on a lattice whose shear modulus is the field mu (lambda =
lam_ratio * mu), as a 0-d CUDA float64 tensor; L.backward() fills mu.grad and
v0.grad from lbm_adjoint_backward. The forward, the checkpoints and the
backward all run in the CUDA library.
"""
import numpy as np
import torch

from . import lbm

_KIND = {"periodic": lbm.LBM_BC_PERIODIC, "velocity": lbm.LBM_BC_VELOCITY, "traction": lbm.LBM_BC_TRACTION}


class _Misfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mu, v0, owner):
        o = owner
        lbm.lbm_set_material_field_device(o.lattice.ctx, o.law, mu.detach().contiguous(), o.lam_ratio)
        U0 = torch.zeros((6, o.ny, o.nx), dtype=torch.float64, device=mu.device)
        U0[2] = 1.0
        U0[5] = 1.0
        U0[:2] = v0.detach()
        loss = lbm.lbm_adjoint_forward(o.adjoint, U0, o.order)
        ctx.owner = o
        return torch.tensor(loss, dtype=torch.float64, device=mu.device)

    @staticmethod
    def backward(ctx, gL):
        o = ctx.owner
        gmu = torch.empty((o.ny, o.nx), dtype=torch.float64, device=gL.device)
        gv0 = torch.empty((2, o.ny, o.nx), dtype=torch.float64, device=gL.device)
        lbm.lbm_adjoint_backward(o.adjoint, gmu, gv0)
        return gL * gmu, gL * gv0, None


class SensorMisfit:
    """nx, ny, dx, c, omega: the lattice; edges: four (kind, value) pairs
    (left, right, bottom, top; kind 'periodic', 'velocity' or 'traction');
    sensors: (nsens, 2) node (x, y); records: recorded steps; target:
    (records, sensors, 2); steps: the run length; storage: LBM_STORE_F64 or
    LBM_STORE_F32; law: SVK, NH or LOGNH."""

    def __init__(self, nx, ny, c, omega, edges, sensors, records, target, steps, lam_ratio=2.0, dx=1.0,
                 storage=lbm.LBM_STORE_F32, law=lbm.LBM_LAW_NH, checkpoint_every=0, order=2, device=0):
        self.nx, self.ny, self.law, self.lam_ratio, self.order = nx, ny, law, lam_ratio, order
        self.lattice = lbm.Lattice(nx, ny, dx=dx, c=c, omega=omega, storage=storage, device=device)
        # a placeholder field so that the adjoint can be created; each call sets the real one
        lbm.lbm_set_material_field(self.lattice.ctx, law, np.ones((ny, nx)), lam_ratio)
        for e, (kind, value) in enumerate(edges):
            lbm.lbm_set_boundary(self.lattice.ctx, e, _KIND[kind], value)
        self.adjoint = lbm.lbm_adjoint_create(self.lattice.ctx, steps, checkpoint_every)
        lbm.lbm_adjoint_set_loss(self.adjoint, sensors, records, target)

    @classmethod
    def from_workload(cls, w, **kw):
        p = w.params
        return cls(w.nx, w.ny, w.c, w.omega, [(E.kind, E.value) for E in w.edges], p["sensors"], p["records"],
                   p["target"], w.steps, lam_ratio=p["lam_ratio"], dx=w.dx, **kw)

    def __call__(self, mu, v0):
        return _Misfit.apply(mu, v0, self)

    def close(self):
        if getattr(self, "adjoint", None) is not None:
            lbm.lbm_adjoint_destroy(self.adjoint)
            self.adjoint = None
        if getattr(self, "lattice", None) is not None:
            self.lattice.close()
            self.lattice = None

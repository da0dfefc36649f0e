"""Exact fields of the manufactured solution of Sec. 4.1 (Eq. 28) for the tests.

The Piola stress is obtained here by symbolic differentiation of the log-NH
strain energy of Appendix A (P = dW/dF), and the body force by Eq. (29),
b = d2u/dt2 - Div P(I + Grad u), so nothing here reuses the oracle's closure
code. Needs sympy (available on the development host only).
"""
import numpy as np
import sympy as sp

A_AMP, K_WAVE, LAM, MU = sp.Rational(8, 100), 2 * sp.pi, sp.Rational(2, 3), 1


class MMS:
    def __init__(self):
        X, Y, t = sp.symbols("X Y t", real=True)
        A, k = A_AMP, K_WAVE
        ux = A * sp.sin(k * (X - sp.Rational(23, 100) * t)) * sp.cos(k * (Y - sp.Rational(17, 100) * t)) \
            * sp.sin(k * (t - sp.Rational(11, 100)))
        uy = A * sp.cos(k * (X + sp.Rational(19, 100) * t)) * sp.sin(k * (Y - sp.Rational(29, 100) * t)) \
            * sp.cos(k * (t + sp.Rational(7, 100)))
        f = sp.symbols("f11 f12 f21 f22")
        Fm = sp.Matrix([[f[0], f[1]], [f[2], f[3]]])
        J = Fm.det()
        C = Fm.T * Fm
        W = MU / 2 * (C.trace() - 2 - 2 * sp.log(J)) + LAM / 2 * sp.log(J) ** 2
        Psym = [sp.diff(W, s) for s in f]
        Fex = [1 + sp.diff(ux, X), sp.diff(ux, Y), sp.diff(uy, X), 1 + sp.diff(uy, Y)]
        Pex = [p.subs(dict(zip(f, Fex))) for p in Psym]
        divP = [sp.diff(Pex[0], X) + sp.diff(Pex[1], Y), sp.diff(Pex[2], X) + sp.diff(Pex[3], Y)]
        b = [sp.diff(ux, t, 2) - divP[0], sp.diff(uy, t, 2) - divP[1]]
        U = [sp.diff(ux, t), sp.diff(uy, t)] + Fex
        lam = lambda e: sp.lambdify((X, Y, t), e, "numpy", cse=True)
        self._U = lam(U)
        self._UX = lam([sp.diff(e, X) for e in U])
        self._UY = lam([sp.diff(e, Y) for e in U])
        self._b = lam(b)
        self._u = lam([ux, uy])
        self._P = lam(Pex)

    @staticmethod
    def _arr(vals, shape):
        return np.array([np.broadcast_to(np.asarray(v, dtype=float), shape) for v in vals])

    def U(self, X, Y, t):
        return self._arr(self._U(X, Y, t), np.shape(X))

    def dUdX(self, X, Y, t):
        return self._arr(self._UX(X, Y, t), np.shape(X))

    def dUdY(self, X, Y, t):
        return self._arr(self._UY(X, Y, t), np.shape(X))

    def b(self, X, Y, t):
        return self._arr(self._b(X, Y, t), np.shape(X))

    def u(self, X, Y, t):
        return self._arr(self._u(X, Y, t), np.shape(X))

    def P(self, X, Y, t):
        return self._arr(self._P(X, Y, t), np.shape(X))

    def sigma(self, X, Y, t):
        P = self.P(X, Y, t)
        F = self.U(X, Y, t)[2:]
        J = F[0] * F[3] - F[1] * F[2]
        return np.array([(P[0] * F[0] + P[1] * F[1]) / J, (P[0] * F[2] + P[1] * F[3]) / J,
                         (P[2] * F[0] + P[3] * F[1]) / J, (P[2] * F[2] + P[3] * F[3]) / J])

"""The 2D sixth-order GPU path (``csrc/fch2d.cpp``) does not apply the iteration's terms one by one
as the oracle does (26 line sweeps per iteration); by linearity it applies H_x, H_y to a few
combinations (14 sweeps).  This restates that call sequence in numpy, with the oracle's line
inverse in place of the sweeps, and checks that it reaches the oracle's iterates: the same
iteration counts and the same fields to rounding, over two steps (W carried), periodic and
Neumann, on a non-square domain.
"""
import numpy as np
import pytest

from oracle.fch import fch2d_be_step
from oracle.helmholtz import helmholtz_inverse
from oracle.solver import Problem
from paper_1611_04214_gb300.inputs import paper_ic_2d


def _regrouped_step(prob, u, dt, eta, state):
    eps = prob.eps
    a = np.cbrt(dt * eps ** 4)
    c_eta, c_f, c_p = dt * eta * eps ** 4 / a ** 2, dt * eps ** 2 / a ** 2, dt / a

    def Hx(g):
        return helmholtz_inverse(g, a, prob.hx, prob.bc, prob.M, axis=1)

    def Hy(g):
        return helmholtz_inverse(g, a, prob.hy, prob.bc, prob.M, axis=0)

    def from_w(w):
        hx, hy = Hx(w), Hy(w)
        v = Hx(hy)
        return v, (2 * v - hx - hy) / a, v - hx - hy + w

    vn = u + 1.0
    m2vn = Hx(Hy(Hx(Hy(vn))))
    W = state.get("W", vn)
    v, lap, xw = from_w(W)
    for k in range(1, prob.max_iter + 1):
        f = v * (v * (v - 3) + 2)
        fp = v * (3 * v - 6) + 2
        p = f * fp - (eps ** 2 * fp * lap + eta * eps ** 2 * f)
        s1 = (3 + 2 * c_eta) * v - 2 * c_f * f + c_p * p           # 2A + B
        A = (3 + c_eta) * v - c_f * f
        C = Hx(Hy(s1)) - Hx(A) - Hy(A)                             # K A + M^{-1} B
        E = xw - 3 * W
        t1 = Hy(E)
        D = Hx(t1) - Hx(E) - t1 + xw                               # 3W - 3XW + X^2 W
        s2, s3 = 2 * C + D, C + D
        W_new = m2vn + Hx(Hy(s2)) - Hx(s3) - Hy(s3) + D           # M^{-2} v^n + K C + X D
        v_new, lap, xw = from_w(W_new)
        res = np.abs(v_new - v).max()
        v, W = v_new, W_new
        if res < prob.tol:
            break
    state["W"] = W
    return v - 1.0, k


@pytest.mark.parametrize("bc,shape", [("periodic", (24, 32)), ("neumann", (20, 28))])
def test_regrouped_sequence_reaches_the_oracle_iterates(bc, shape):
    ny, nx = shape
    prob = Problem(nx=nx, ny=ny, Lx=2 * np.pi, Ly=1.5 * np.pi, bc=bc, eps=0.18, M=6, tol=1e-12, max_iter=3000)
    u = paper_ic_2d(nx, ny, bc == "periodic")
    state, got, ref, w = {}, u.copy(), u.copy(), None
    for _ in range(2):
        got, k = _regrouped_step(prob, got, 0.05, 1.0, state)
        r = fch2d_be_step(prob, ref + 1.0, 0.05, 1.0, w)
        w, ref = r.w, r.v - 1.0
        assert k == r.iters
        assert np.abs(got - ref).max() < 1e-12

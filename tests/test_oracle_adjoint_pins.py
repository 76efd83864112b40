"""Pins of the oracle adjoint (no counterpart in the paper: the reverse of the
section 2.2 update with dt frozen).  The taped reverse sweep is checked
against an independent forward-mode (dual-number) evaluation of the same
step by the dot-product identity <J v, w> = <v, J^T w>, and both against
central finite differences of the step and of a multi-step loss."""
import numpy as np

import oracle
from oracle import adjoint as OD
from paper_1712_07070_b300 import ics

G53 = 5.0 / 3.0


def spun_up(n, seed, steps=2, **kw):
    """The turbulence state after a few forward steps: its initial density and
    pressure are uniform, which puts every density/pressure limiter exactly on
    its kink (a = b = 0), where the step has no derivative; finite-difference
    checks are made away from kinks."""
    U = ics.turbulence(n, seed=seed, **kw)
    U, _ = oracle.run_periodic(U, 1.0 / n, G53, 0.5, steps)
    return U


def test_dot_product_identity_one_step():
    U = ics.sod_noise(8, seed=3)
    dt = oracle.dt_cfl2(U, G53, 0.5, 1 / 8)
    rng = np.random.default_rng(0)
    for _ in range(3):
        v = rng.normal(size=U.shape)
        w = rng.normal(size=U.shape)
        Jv = OD.jvp_step(U, v, 1 / 8, dt, G53)
        JTw = OD.adj_step(U, w, 1 / 8, dt, G53)
        a, b = float((Jv * w).sum()), float((v * JTw).sum())
        assert abs(a - b) <= 1e-12 * max(abs(a), abs(b)), (a, b)


def test_tangent_matches_central_differences():
    U = spun_up(8, 2)
    dt = oracle.dt_cfl2(U, G53, 0.5, 1 / 8)
    v = ics.smooth_directions(U.shape, 1, seed=7)[0]
    h = 1e-6
    Jv = OD.jvp_step(U, v, 1 / 8, dt, G53)
    Sp, _ = oracle.step_periodic(U + h * v, 1 / 8, dt, G53)
    Sm, _ = oracle.step_periodic(U - h * v, 1 / 8, dt, G53)
    fd = (Sp - Sm) / (2 * h)
    assert np.abs(fd - Jv).sum() <= 1e-5 * np.abs(Jv).sum()


def test_adjoint_gradient_matches_finite_differences_multistep():
    n = 16
    dh = 1 / n
    U0 = spun_up(n, 5)
    target = spun_up(n, 5, density_seed=6)[0]
    dts = []
    U = U0
    for _ in range(5):
        dt = oracle.dt_cfl2(U, G53, 0.5, dh)
        dts.append(dt)
        U, _ = oracle.step_periodic(U, dh, dt, G53)
    grad, _ = OD.gradient(U0, dts, dh, G53, target)
    dirs = ics.smooth_directions(U0.shape, 3, seed=11)
    h = 1e-6
    for v in dirs:
        Lp = OD.loss(OD.run_frozen(U0 + h * v, dts, dh, G53)[-1], target, dh ** 3)
        Lm = OD.loss(OD.run_frozen(U0 - h * v, dts, dh, G53)[-1], target, dh ** 3)
        fd = (Lp - Lm) / (2 * h)
        g = float((grad * v).sum())
        assert abs(fd - g) <= 1e-5 * abs(g), (fd, g)

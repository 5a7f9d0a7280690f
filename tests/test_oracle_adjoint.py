"""Pins of the oracle's reference gradients: complex-step directional derivatives of the
run loss against FP64 central finite differences (the two agree to the finite-difference
truncation error)."""

import numpy as np
import pytest

from oracle import adjoint
from paper_2002_05265_gb300 import flows


@pytest.mark.parametrize("model,loss", [("bgk", "misfit"), ("chm", "misfit"), ("k", "ke"), ("rr", "misfit")])
def test_complex_step_matches_central_differences(model, loss):
    rho, ux, uy = flows.vortex(10, 8, Ma=0.3, noise=1e-3, seed=3)
    tx, ty = ux + 0.01, uy - 0.02
    rates = (1.7, 1.2, 0.9)
    g = np.random.default_rng(5)
    dx, dy = g.standard_normal(ux.shape), g.standard_normal(uy.shape)
    cs = adjoint.directional_derivative(rho, ux, uy, model, rates, 6, loss, tx, ty, dux=dx, duy=dy)
    h = 1e-6
    lp = adjoint.run_loss(rho, ux + h * dx, uy + h * dy, model, rates, 6, loss, tx, ty)
    lm = adjoint.run_loss(rho, ux - h * dx, uy - h * dy, model, rates, 6, loss, tx, ty)
    assert cs == pytest.approx((lp - lm) / (2 * h), rel=1e-6)
    for k in range(3):
        d = [0.0, 0.0, 0.0]
        d[k] = 1.0
        cs = adjoint.directional_derivative(rho, ux, uy, model, rates, 6, loss, tx, ty, drates=d)
        rp = list(rates); rp[k] += h
        rm = list(rates); rm[k] -= h
        fd = (adjoint.run_loss(rho, ux, uy, model, tuple(rp), 6, loss, tx, ty)
              - adjoint.run_loss(rho, ux, uy, model, tuple(rm), 6, loss, tx, ty)) / (2 * h)
        # central differences carry ~eps * L / h ~ 1e-10 of rounding noise (L ~ 1)
        assert cs == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_bgk_loss_does_not_depend_on_high_order_rates():
    rho, ux, uy = flows.vortex(8, Ma=0.2, noise=1e-3, seed=4)
    for k in (1, 2):
        d = [0.0, 0.0, 0.0]
        d[k] = 1.0
        assert adjoint.directional_derivative(rho, ux, uy, "bgk", (1.5, 1.2, 1.1), 4, "ke", drates=d) == 0.0

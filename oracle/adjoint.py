"""Reference gradients of a final-state loss of the stream-and-collide run (test
infrastructure only, like the rest of this package).

The loss of an N-step run started from the equilibrium f^eq(rho0, u0) (Sec. 5a) is an
analytic function of the initial velocity and of the relaxation rates, so its directional
derivatives follow exactly (to rounding) from the complex-step method: perturb the inputs by
i h d with a tiny h and read Im(L) / h.  This is independent of any adjoint derivation: it
runs the plain oracle forward in complex arithmetic.

Losses: "misfit" L = 1/2 sum_x |u^N(x) - u*(x)|^2, "ke" L = 1/2 sum_x rho |u|^2.
"""

import numpy as np

from .collision import macroscopic
from .lbm import init_equilibrium, run

H_CS = 1e-30


def run_loss(rho0, ux0, uy0, model, rates, nsteps, loss="misfit", ux_t=None, uy_t=None):
    f = init_equilibrium(rho0, ux0, uy0)
    f = run(f, model, rates, nsteps)
    rho, ux, uy = macroscopic(f)
    if loss == "misfit":
        return 0.5 * ((ux - ux_t) ** 2 + (uy - uy_t) ** 2).sum()
    if loss == "ke":
        return 0.5 * (rho * (ux * ux + uy * uy)).sum()
    raise ValueError(loss)


def directional_derivative(rho0, ux0, uy0, model, rates, nsteps, loss="misfit", ux_t=None, uy_t=None,
                           dux=None, duy=None, drates=(0.0, 0.0, 0.0)):
    """dL/dh of L(u0 + h du, rates + h drates) at h = 0, by the complex step."""
    zx = np.zeros_like(ux0) if dux is None else dux
    zy = np.zeros_like(uy0) if duy is None else duy
    cr = tuple(complex(r, H_CS * d) for r, d in zip(rates, drates))
    val = run_loss(rho0.astype(complex), ux0 + 1j * H_CS * zx, uy0 + 1j * H_CS * zy, model, cr, nsteps, loss,
                   ux_t, uy_t)
    return float(np.imag(val) / H_CS)

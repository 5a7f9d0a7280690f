"""Stream-and-collide time stepping (Eq. StreamCollide) on a periodic nx x ny lattice.

State: pre-collision populations f[i, y, x] at time t.  One step collides every node with
the chosen model and then pushes each post-collision population to its downstream
neighbour, f_i(x + xi_i, t + 1) = f*_i(x, t), with periodic wrap (Eq. StreamCollide; the
paper's domains are periodic, Sec. 5a).
"""

import numpy as np

from .d2q9 import XI, CS2, Q
from .collision import collide, macroscopic
from .equilibrium import feq

PRESETS = ("srt", "reg")


def omega_from_nu(nu):
    """omega_nu = 1 / (nu / c_s^2 + 1/2)  (Sec. 4c)."""
    return 1.0 / (nu / CS2 + 0.5)


def rates_from_nu(nu, preset="srt"):
    """Relaxation-rate presets of Sec. 4c: SRT omega3 = omega4 = omega_nu;
    REG omega3 = omega4 = 1."""
    w = omega_from_nu(nu)
    if preset == "srt":
        return (w, w, w)
    if preset == "reg":
        return (w, 1.0, 1.0)
    raise ValueError(preset)


def init_equilibrium(rho, ux, uy, eq_order=4):
    """f(x, 0) = f^eq(rho(x), u(x))  (initial state of Sec. 5a)."""
    return feq(rho, ux, uy, eq_order)


def stream(fs):
    """Periodic push streaming: f_i(x + xi_i) = f*_i(x)  (Eq. StreamCollide, left side)."""
    out = np.empty_like(fs)
    for i in range(Q):
        out[i] = np.roll(fs[i], shift=(int(XI[i, 1]), int(XI[i, 0])), axis=(0, 1))
    return out


def step(f, model, rates, eq_order=4):
    """One time step: collide every node, then stream (Eq. StreamCollide)."""
    w_nu, w3, w4 = rates
    return stream(collide(model, f, w_nu, w3, w4, eq_order))


def run(f, model, rates, nsteps, eq_order=4):
    for _ in range(nsteps):
        f = step(f, model, rates, eq_order)
    return f


def moments_output(f):
    """rho, u_x, u_y and the second-order raw moments Pi_ab = sum_i xi_a xi_b f_i of the
    pre-collision state (Sec. 1; App. B)."""
    rho, ux, uy = macroscopic(f)
    pxx = sum(float(XI[i, 0] * XI[i, 0]) * f[i] for i in range(Q))
    pxy = sum(float(XI[i, 0] * XI[i, 1]) * f[i] for i in range(Q))
    pyy = sum(float(XI[i, 1] * XI[i, 1]) * f[i] for i in range(Q))
    return rho, ux, uy, pxx, pxy, pyy


def reductions(f, uref=(0.0, 0.0)):
    """Global diagnostics of the pre-collision state, in FP64:
    [sum rho, sum rho u_x, sum rho u_y, sum rho |u|^2 / 2, <|u|^2>, <|u - uref|^2>,
     min rho, number of nodes with a non-finite rho or u].
    <.> is the mean over nodes; <|u|^2> / u_0^2 is the blow-up criterion of Sec. 5b."""
    rho, ux, uy = macroscopic(f)
    finite = np.isfinite(rho) & np.isfinite(ux) & np.isfinite(uy)
    r, x, y = rho[finite], ux[finite], uy[finite]
    n = rho.size
    return np.array([
        r.sum(), (r * x).sum(), (r * y).sum(), 0.5 * (r * (x * x + y * y)).sum(),
        (x * x + y * y).sum() / n, ((x - uref[0]) ** 2 + (y - uref[1]) ** 2).sum() / n,
        r.min() if r.size else np.nan, float(n - finite.sum())])

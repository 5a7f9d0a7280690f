"""Linear stability analysis of the stream-and-collide scheme (App. A).

The perturbed discrete equation (Eq. DiscretePerturbedEq) is
    f'_i(x + xi_i, t + 1) = [delta_ij + J_ij] f'_j(x, t),
with J_ij = dOmega_i / df_j at the uniform equilibrium state (Eq. Perturbed_Collision), so
delta + J is the Jacobian of the collision map f -> f*.  Plane waves
f' = A exp(i(k.x - omega t)) give the eigenproblem (Eq. EigenvaluePbDiscrete)
    E^D [delta + J] A = exp(-i omega) A,   E^D_ij = exp(-i xi_i.k) delta_ij,
so the growth rate of a mode is Im(omega) = ln |exp(-i omega)|.

The Jacobian is taken numerically, as in the paper (App. A says it used a dedicated
library), here by the complex-step method: d f*_i / d f_j = Im(C(f + i h e_j))_i / h,
which is exact to rounding for the rational collision maps of App. B.
"""

import numpy as np

from .d2q9 import XI, Q
from .collision import collide
from .equilibrium import feq

H_CS = 1e-30


def collision_map_jacobian(model, rho, ux, uy, rates, eq_order=4):
    """delta_ij + J_ij = d f*_i / d f_j at f = f^eq(rho, u)  (App. A)."""
    w_nu, w3, w4 = rates
    base = feq(np.array([rho], dtype=complex), np.array([ux], dtype=complex),
               np.array([uy], dtype=complex), eq_order)
    G = np.zeros((Q, Q))
    for j in range(Q):
        fp = base.copy()
        fp[j] += 1j * H_CS
        G[:, j] = collide(model, fp, w_nu, w3, w4, eq_order)[:, 0].imag / H_CS
    return G


def discrete_matrix(G, kx, ky):
    """M^D = E^D [delta + J] for the wavenumber k = (kx, ky)  (App. A)."""
    E = np.exp(-1j * (XI[:, 0] * kx + XI[:, 1] * ky))
    return E[:, None] * G


def eigenvalues(G, kx, ky):
    """Eigenvalues exp(-i omega) of M^D(k)."""
    return np.linalg.eigvals(discrete_matrix(G, kx, ky))


def omegas(G, kx, ky):
    """omega = i ln(lambda) for each eigenvalue lambda; Im(omega) = ln|lambda| is the growth
    rate and Re(omega) = -arg(lambda) the frequency (Eq. MonochromPlaneWaves)."""
    lam = eigenvalues(G, kx, ky)
    return 1j * np.log(lam)


def max_growth_rate(G, kxs, kys):
    """max over the k grid and the nine modes of Im(omega) = ln|lambda|."""
    best = -np.inf
    for kx in kxs:
        for ky in kys:
            best = max(best, float(np.max(np.log(np.abs(eigenvalues(G, kx, ky))))))
    return best

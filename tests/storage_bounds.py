"""Rounding model behind the reduced-precision tolerances of the GPU tests (test code, not
part of the library): every step rounds each stored population g_i = f_i - s_i once to the
storage type, an error uniform on +-ulp/2 and independent between populations, nodes and
steps.  The collision conserves mass and momentum exactly, so the rounding that lands in the
conserved moments is never relaxed and adds up as a random walk."""

import numpy as np

XI = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
# the velocity error of reduced storage is held to this multiple of storage_walk_error: it
# covers the spread of a sum of random kicks over ~10^4 nodes and the FP32 collision
# arithmetic, whose rounding is ~2^-13 of the 16-bit storage's
WALK_FACTOR = 2.0

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def _ulp(g, storage):
    """Spacing of the storage type's numbers around each FP64 value g (FP16: 11 significant
    bits, subnormal spacing 2^-24; BF16: 8 significant bits; FP32: 24)."""
    a = np.abs(g)
    if storage == "f16":
        return np.spacing(a.astype(np.float16)).astype(np.float64)
    if storage == "f32":
        return np.spacing(a.astype(np.float32)).astype(np.float64)
    bits = {"bf16": 8}[storage]
    e = np.frexp(np.where(a > 0, a, 1.0))[1]
    return np.ldexp(1.0, e - bits)


def storage_walk_error(f0, storage, steps):
    """Expected normalised L2 velocity error of storing g_i = f_i - w_i rho0 in a reduced
    type for `steps` steps (the rounding model behind the storage tolerances).

    Every step rounds each stored population once, an error uniform on +-ulp/2 (variance
    ulp^2/12) and independent between populations, nodes and steps.  The collision conserves
    mass and momentum exactly, so the part of the rounding that lands in the conserved moments
    is never relaxed: the velocity of a node receives the kick du_a = sum_i (xi_ia - u_a) dg_i
    / rho each step and the kicks add up as a random walk (viscous damping at the lattice
    scale, nu k^2 per step, is neglected, which over-estimates).  After N steps the error
    variance per node is N sum_i |xi_i - u|^2 ulp_i^2 / 12 / rho^2, so the normalised L2 error
    is sqrt(N <that sum>) / sqrt(<|u|^2>), with the ulps of the initial state's stored values."""
    rho = f0.sum(axis=0)
    ux = sum(float(XI[i][0]) * f0[i] for i in range(9)) / rho
    uy = sum(float(XI[i][1]) * f0[i] for i in range(9)) / rho
    ulp = _ulp(f0 - W[:, None, None], storage)
    var = sum(((XI[i][0] - ux) ** 2 + (XI[i][1] - uy) ** 2) * ulp[i] ** 2 / 12 for i in range(9)) / rho ** 2
    return float(np.sqrt(steps * var.mean() / (ux * ux + uy * uy).mean()))


def conservation_walk_bound(f0, storage, steps, sigmas=6.0):
    """Bound on the drift of the FP64 totals of mass and x / y momentum after `steps` steps
    of a state stored as g = f - w rho0: the collision conserves them exactly, so only the
    per-step rounding of the nine stored populations moves them; those errors (uniform on
    +-ulp/2, independent) add up as a random walk with per-step variance
    sum_x sum_i c_i^2 ulp_i^2 / 12 (c_i = 1 for mass, xi_ia for momentum).  Returns
    `sigmas` standard deviations after `steps` steps for (mass, jx, jy)."""
    ulp2 = _ulp(f0 - W[:, None, None], storage) ** 2 / 12
    var_m = ulp2.sum()
    var_x = sum(XI[i][0] ** 2 * ulp2[i].sum() for i in range(9))
    var_y = sum(XI[i][1] ** 2 * ulp2[i].sum() for i in range(9))
    return sigmas * np.sqrt(steps * np.array([var_m, var_x, var_y]))

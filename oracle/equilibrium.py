"""Discrete equilibria of Sec. 2.

extended (default, "order 4"): Eq. extendedFeq.  The equilibrium raw moments are the closed
forms listed after Eq. RMcoll (App. B):
    M00 = rho, M10 = rho u_x, M01 = rho u_y,
    M20 = rho (u_x^2 + c_s^2), M02 = rho (u_y^2 + c_s^2), M11 = rho u_x u_y,
    M21 = M20 u_y, M12 = u_x M02, M22 = M20 M02 / rho,
and the populations follow from the second equality of Eq. extendedFeq.

second order ("order 2"): Sec. 2 obtains it "by imposing M^eq_pq = 0 for p+q >= 3" in
Eq. extendedFeq.  Read literally with raw moments this breaks the second-order matching
conditions (M20 = sum xi_x^2 f would no longer be recovered by the populations formula),
so the reading taken is the Hermite one: the equilibrium Hermite moments of order >= 3
vanish, A^eq_21 = A^eq_12 = A^eq_22 = 0, which is the textbook second-order polynomial
equilibrium.  Converted to raw moments with Eq. HM2RM_Q9 this gives
    M21 = rho c_s^2 u_y,  M12 = rho c_s^2 u_x,  M22 = c_s^2 rho (u_x^2 + u_y^2) + rho c_s^4.

partial third order ("order 3"): the middle truncation of Fig. 4, which Sec. 2 motivates by
the third-order terms M^eq_21, M^eq_12 that correct the off-diagonal viscous stress.  Same
Hermite reading: the equilibrium keeps A^eq_21 = rho u_x^2 u_y and A^eq_12 = rho u_x u_y^2 of
the extended equilibrium and drops the fourth-order one, A^eq_22 = 0.  In raw moments M21
and M12 are those of the extended equilibrium and
    M22 = c_s^2 (M20 + M02) - c_s^4 rho = c_s^2 rho (u_x^2 + u_y^2) + rho c_s^4,
i.e. the extended M22 minus rho u_x^2 u_y^2.
"""

import numpy as np

from .d2q9 import CS2, XI, Q
from .moments import populations_from_raw


def raw_equilibrium_moments(rho, ux, uy, order=4):
    """Equilibrium raw moments M^eq_pq, p, q <= 2 (App. B after Eq. RMcoll; orders 2 and 3
    per the readings in the module docstring)."""
    M = {}
    M[0, 0] = rho
    M[1, 0] = rho * ux
    M[0, 1] = rho * uy
    M[2, 0] = rho * (ux * ux + CS2)
    M[0, 2] = rho * (uy * uy + CS2)
    M[1, 1] = rho * ux * uy
    if order == 4:
        M[2, 1] = M[2, 0] * uy
        M[1, 2] = ux * M[0, 2]
        M[2, 2] = M[2, 0] * M[0, 2] / rho
    elif order == 3:
        M[2, 1] = M[2, 0] * uy
        M[1, 2] = ux * M[0, 2]
        M[2, 2] = CS2 * (M[2, 0] + M[0, 2]) - CS2 * CS2 * rho
    elif order == 2:
        M[2, 1] = rho * CS2 * uy
        M[1, 2] = rho * CS2 * ux
        M[2, 2] = CS2 * rho * (ux * ux + uy * uy) + rho * CS2 * CS2
    else:
        raise ValueError("equilibrium order must be 2, 3 or 4")
    return M


def feq(rho, ux, uy, order=4):
    """Equilibrium populations f^eq_i, shape (9, ...) (Eq. extendedFeq, second equality,
    i.e. Eq. Q9postCollVDF_RM applied to the equilibrium moments)."""
    return np.array(populations_from_raw(raw_equilibrium_moments(rho, ux, uy, order)))


def feq_product_form(rho, ux, uy):
    """Extended equilibrium in its product form (Eq. extendedFeq, first equality):
    f^eq_(sx,sy) = (1/rho) * [factor in x] * [factor in y] with
    factor_0(x) = M00 - M20, factor_s(x) = (s M10 + M20)/2 and likewise in y."""
    M = raw_equilibrium_moments(rho, ux, uy, 4)
    fx = {0: M[0, 0] - M[2, 0], 1: 0.5 * (M[1, 0] + M[2, 0]), -1: 0.5 * (-M[1, 0] + M[2, 0])}
    fy = {0: M[0, 0] - M[0, 2], 1: 0.5 * (M[0, 1] + M[0, 2]), -1: 0.5 * (-M[0, 1] + M[0, 2])}
    return np.array([fx[int(XI[i, 0])] * fy[int(XI[i, 1])] / rho for i in range(Q)])

"""Moment spaces of App. B, written as plain sums over the nine populations.

Every moment set is a dict {(p, q): array} for p, q <= 2.  Arrays hold one value per node
(any shape, FP64 or complex128).

Readings of the paper taken here:
  * the raw-moment definition after Eq. RMcoll prints xi_{i,x}^q for the second factor;
    the second factor is xi_{i,y}^q (otherwise M_pq would not depend on y at all);
  * Eq. CHpoly prints H~_12 = (xi_y - u_y)[(xi_y - u_y)^2 - c_s^2]; its own definition
    H~_12 = H~_10 H~_02 gives (xi_x - u_x)[(xi_y - u_y)^2 - c_s^2], which is used;
  * the central-moment to raw-moment back-transform is deferred by the paper to an
    external appendix; the binomial identity that defines central moments is used.
"""

from math import comb

from .d2q9 import XI, CS2, PQ, Q


def raw_moments(f):
    """M_pq = sum_i xi_{i,x}^p xi_{i,y}^q f_i  (App. B, definition after Eq. RMcoll)."""
    M = {}
    for (p, q) in PQ:
        M[p, q] = sum(float(XI[i, 0] ** p * XI[i, 1] ** q) * f[i] for i in range(Q))
    return M


def populations_from_raw(M):
    """f_i from raw moments M_pq, p,q <= 2  (Eq. Q9postCollVDF_RM; the same map is the
    second equality of Eq. extendedFeq).  Returns the list of nine populations in the
    lattice index order."""
    f = [None] * Q
    for i in range(Q):
        s, l = int(XI[i, 0]), int(XI[i, 1])
        if s == 0 and l == 0:
            f[i] = M[0, 0] - (M[2, 0] + M[0, 2]) + M[2, 2]
        elif l == 0:
            f[i] = 0.5 * (s * M[1, 0] + M[2, 0] - s * M[1, 2] - M[2, 2])
        elif s == 0:
            f[i] = 0.5 * (l * M[0, 1] + M[0, 2] - l * M[2, 1] - M[2, 2])
        else:
            f[i] = 0.25 * (s * l * M[1, 1] + s * M[1, 2] + l * M[2, 1] + M[2, 2])
    return f


def _hermite_1d(n, c):
    """One-dimensional (central) Hermite polynomial of Eq. CHpoly for order n in the
    peculiar velocity c: 1, c, c^2 - c_s^2."""
    if n == 0:
        return 1.0 + 0.0 * c
    if n == 1:
        return c
    return c * c - CS2


def central_hermite_moments(f, ux, uy):
    """A~_pq = sum_i H~_{i,pq} f_i with the central Hermite polynomials of Eq. CHpoly,
    H~_{i,pq} = H~_{i,p0} H~_{i,0q} (peculiar velocity xi_i - u)."""
    A = {}
    for (p, q) in PQ:
        A[p, q] = sum(_hermite_1d(p, float(XI[i, 0]) - ux) * _hermite_1d(q, float(XI[i, 1]) - uy) * f[i]
                      for i in range(Q))
    return A


def hermite_moments(f):
    """A_pq = sum_i H_{i,pq} f_i: the non-central Hermite moments, i.e. Eq. CHpoly with
    the peculiar velocity replaced by xi_i itself (App. B, text after Eq. CHpoly)."""
    A = {}
    for (p, q) in PQ:
        A[p, q] = sum(_hermite_1d(p, float(XI[i, 0])) * _hermite_1d(q, float(XI[i, 1])) * f[i]
                      for i in range(Q))
    return A


def raw_from_hermite(A):
    """Post-collision RMs from HMs (Eq. HM2RM_Q9), written with rho = A_00,
    rho u_x = A_10, rho u_y = A_01 as in that equation."""
    M = {}
    M[0, 0] = A[0, 0]
    M[1, 0] = A[1, 0]
    M[0, 1] = A[0, 1]
    M[1, 1] = A[1, 1]
    M[2, 0] = A[2, 0] + A[0, 0] * CS2
    M[0, 2] = A[0, 2] + A[0, 0] * CS2
    M[2, 1] = A[2, 1] + CS2 * A[0, 1]          # rho c_s^2 u_y
    M[1, 2] = A[1, 2] + CS2 * A[1, 0]          # rho c_s^2 u_x
    M[2, 2] = A[2, 2] + CS2 * (A[2, 0] + A[0, 2]) + A[0, 0] * CS2 * CS2
    return M


def hermite_from_central_hermite(At, rho, ux, uy):
    """Post-collision HMs from CHMs (Eq. CHM2HM_Q9).  The equation assumes the conserved
    central moments A~_00 = rho, A~_10 = A~_01 = 0, which hold after collision."""
    A = {}
    A[0, 0] = At[0, 0]
    A[1, 0] = At[1, 0] + rho * ux
    A[0, 1] = At[0, 1] + rho * uy
    A[2, 0] = At[2, 0] + rho * ux * ux
    A[0, 2] = At[0, 2] + rho * uy * uy
    A[1, 1] = At[1, 1] + rho * ux * uy
    A[2, 1] = At[2, 1] + uy * At[2, 0] + 2.0 * ux * At[1, 1] + rho * ux * ux * uy
    A[1, 2] = At[1, 2] + ux * At[0, 2] + 2.0 * uy * At[1, 1] + rho * ux * uy * uy
    A[2, 2] = (At[2, 2] + 2.0 * uy * At[2, 1] + 2.0 * ux * At[1, 2] + uy * uy * At[2, 0]
               + ux * ux * At[0, 2] + 4.0 * ux * uy * At[1, 1] + rho * ux * ux * uy * uy)
    return A


def central_moments(f, ux, uy):
    """K~_pq = sum_i (xi_{i,x} - u_x)^p (xi_{i,y} - u_y)^q f_i: central moments, i.e. raw
    moments in the co-moving velocity xi~ = xi - u (App. B, text after Eq. CHpoly)."""
    K = {}
    for (p, q) in PQ:
        K[p, q] = sum((float(XI[i, 0]) - ux) ** p * (float(XI[i, 1]) - uy) ** q * f[i] for i in range(Q))
    return K


def raw_from_central(K, ux, uy):
    """Raw moments from central moments by the binomial expansion of
    xi^p = (xi~ + u)^p:  M_pq = sum_{a<=p, b<=q} C(p,a) C(q,b) u_x^(p-a) u_y^(q-b) K~_ab.
    (The paper defers this back-transform to an external appendix; this is the identity
    that defines central moments, closed on p, q <= 2.)"""
    M = {}
    for (p, q) in PQ:
        M[p, q] = sum(comb(p, a) * comb(q, b) * ux ** (p - a) * uy ** (q - b) * K[a, b]
                      for a in range(p + 1) for b in range(q + 1))
    return M


def cumulants_from_central(K):
    """D2Q9 cumulants C_pq (p, q <= 2) from central moments (reading of the cumulant model
    named in Sec. 1 and Sec. 4c; its definition is deferred by the paper to an external
    reference).  Cumulants are rho times the derivatives of the log of the moment
    generating function; up to third order they equal the central moments, and
      C_22 = K~_22 - (K~_20 K~_02 + 2 K~_11^2) / rho.
    C_00 = rho and C_10 = C_01 = K~_10 = K~_01 are carried unchanged."""
    C = dict(K)
    rho = K[0, 0]
    C[2, 2] = K[2, 2] - (K[2, 0] * K[0, 2] + 2.0 * K[1, 1] * K[1, 1]) / rho
    return C


def central_from_cumulants(C):
    """Inverse of cumulants_from_central: K~_22 = C_22 + (K~_20 K~_02 + 2 K~_11^2) / rho,
    with the second-order central moments equal to the second-order cumulants passed in
    (after collision these are the post-collision values)."""
    K = dict(C)
    rho = C[0, 0]
    K[2, 2] = C[2, 2] + (C[2, 0] * C[0, 2] + 2.0 * C[1, 1] * C[1, 1]) / rho
    return K

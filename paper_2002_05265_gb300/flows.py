"""Seeded synthetic inputs: initial macroscopic fields (rho, u_x, u_y) of the flows the
paper simulates.  This module holds no lattice-Boltzmann arithmetic (no equilibrium, no
collision, no streaming): it only produces FP64 numpy arrays [ny][nx] that both the CUDA
path and the FP64 oracle start from.

Random numbers come from numpy's Philox counter-based generator with the seed recorded.
Node coordinates are x = 0..nx-1, y = 0..ny-1 (lattice units); the lattice sound speed is
c_s = 1/sqrt(3).
"""

import numpy as np

CS = 1.0 / np.sqrt(3.0)


def _rng(seed):
    return np.random.Generator(np.random.Philox(seed))


def vortex(nx, ny=None, Ma=0.1, beta=0.5, radius_frac=0.1, rho0=1.0, noise=0.0, seed=1,
           center=None, rows=None):
    """Isothermal convected vortex of Sec. 5a (first-order Taylor form of the isentropic
    vortex about T_0 = c_s^2):
        rho = rho0 [1 - eps^2/(2 c_s^2) exp(-r^2)],
        u_x = u0 - eps (y - y_c)/R exp(-r^2/2),  u_y = eps (x - x_c)/R exp(-r^2/2),
    eps = beta u0, u0 = Ma c_s, r = |x - x_c| / R.  R = radius_frac * nx (the workloads use
    R = 0.1 L; the paper's figure uses R = L/20).  The vortex sits at the domain centre
    unless `center` is given.  `noise` adds independent U(-noise, noise) to u_x and u_y.
    `rows` = (y0, y1) returns only rows y0 <= y < y1 of the same field (without noise), so
    that very large lattices can be generated in slabs."""
    ny = nx if ny is None else ny
    u0 = Ma * CS
    eps = beta * u0
    R = radius_frac * nx
    xc, yc = (nx / 2.0, ny / 2.0) if center is None else center
    y0, y1 = (0, ny) if rows is None else rows
    if rows is not None and noise:
        raise ValueError("row slabs are generated without noise")
    y, x = np.meshgrid(np.arange(y0, y1, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    r2 = ((x - xc) ** 2 + (y - yc) ** 2) / (R * R)
    rho = rho0 * (1.0 - eps * eps / (2.0 * CS * CS) * np.exp(-r2))
    ux = u0 - eps * (y - yc) / R * np.exp(-r2 / 2.0)
    uy = eps * (x - xc) / R * np.exp(-r2 / 2.0)
    if noise:
        g = _rng(seed)
        ux = ux + g.uniform(-noise, noise, size=ux.shape)
        uy = uy + g.uniform(-noise, noise, size=uy.shape)
    return rho, ux, uy


def double_shear_layer(nx, ny=None, Ma=0.1, width_frac=1.0 / 80.0, delta=0.05, rho0=1.0):
    """Periodic double shear layer (App. C):
        u_x = u0 tanh(kappa (y - L/4)) for y <= L/2,  u0 tanh(kappa (3L/4 - y)) above,
        u_y = delta u0 sin(2 pi (x/L + 1/4)),  rho = rho0,  kappa = 1 / (width_frac L),
    u0 = Ma c_s.  (The paper initialises it as in an external reference; this is the
    standard form of that test.)"""
    ny = nx if ny is None else ny
    u0 = Ma * CS
    kappa = 1.0 / (width_frac * ny)
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    ux = np.where(y <= ny / 2.0, u0 * np.tanh(kappa * (y - ny / 4.0)), u0 * np.tanh(kappa * (3.0 * ny / 4.0 - y)))
    uy = delta * u0 * np.sin(2.0 * np.pi * (x / nx + 0.25))
    rho = np.full_like(ux, rho0)
    return rho, ux, uy


def uniform_noise(nx, ny=None, Ma=0.0, phi=0.0, amp=1e-6, rho0=1.0, seed=0):
    """Uniform flow u = Ma c_s (cos phi, sin phi) plus independent U(-amp, amp) noise on
    u_x and u_y (perturbed uniform flow of the stability study, Sec. 5b)."""
    ny = nx if ny is None else ny
    g = _rng(seed)
    u0 = Ma * CS
    ux = u0 * np.cos(phi) + g.uniform(-amp, amp, size=(ny, nx))
    uy = u0 * np.sin(phi) + g.uniform(-amp, amp, size=(ny, nx))
    rho = np.full((ny, nx), rho0)
    return rho, ux, uy


def shear_wave(nx, ny=None, amp=1e-4, mode=1, u0=0.0, rho0=1.0):
    """Transverse shear wave u_y = amp sin(2 pi mode x / nx) on a uniform flow u_x = u0
    (its amplitude decays as exp(-nu k^2 t), Sec. 3b)."""
    ny = nx if ny is None else ny
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    uy = amp * np.sin(2.0 * np.pi * mode * x / nx)
    ux = np.full_like(uy, u0)
    rho = np.full_like(uy, rho0)
    return rho, ux, uy


def smooth_random_field(nx, ny, kmax, seed):
    """Random smooth periodic field: Fourier modes with |k_x|, |k_y| <= kmax and N(0, 1)
    amplitudes, normalised to unit root-mean-square (seeded Philox)."""
    g = _rng(seed)
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    out = np.zeros((ny, nx))
    for kx in range(-kmax, kmax + 1):
        for ky in range(0, kmax + 1):
            a, b = g.normal(size=2)
            ph = 2.0 * np.pi * (kx * x / nx + ky * y / ny)
            out += a * np.cos(ph) + b * np.sin(ph)
    return out / np.sqrt((out ** 2).mean())


def gaussian_noise(shape, sigma, seed):
    """N(0, sigma^2) array of the given shape (seeded Philox)."""
    return _rng(seed).normal(0.0, sigma, size=shape)


def random_populations_perturbation(shape, amp, seed):
    """U(-amp, amp) array of the given shape (used to perturb a state off equilibrium)."""
    return _rng(seed).uniform(-amp, amp, size=shape)

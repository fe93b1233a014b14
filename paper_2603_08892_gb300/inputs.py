"""Seeded synthetic inputs shared by the tests, the bench, the oracle checks and the library users.

This module holds input data only -- initial velocity fields and random seeds -- and none
of the solver's arithmetic (no truncation, projection, phase shift or time stepping): both
the CUDA library and the CPU oracle receive the same physical fields and truncate and
project them themselves.

Workloads (the paper measures on flows defined by equations, so these *are* the
workloads, generated at the paper's shapes and sizes):

* Taylor-Green vortex, Section 3.4, Eq. (T-G-init): u = (sin x cos y cos z,
  -cos x sin y cos z, 0) on [0, 2 pi)^3;
* 2D Taylor-Green cells u = (sin x cos y, -cos x sin y, 0): a steady solution of the Euler
  equations (its nonlinear term is a pure gradient) used as an exact-solution check;
* homogeneous isotropic turbulence initial field (Section 6.2 starts from a stationary
  state we do not have): a random solenoidal field u = curl A of a Gaussian vector
  potential, shell-rescaled to E(k) ~ k^4 exp(-2 (k/k_p)^2), k_p = 4, total energy 1.5
  (u_rms = 1 per component);
* small random solenoidal perturbations (ensembles): the same generator band-limited to
  |k| <= 4 and scaled to a fraction of the Taylor-Green rms velocity.

All generators return float64 arrays u[c, z, y, x] (x fastest).
"""
import math

import numpy as np


def grid(N):
    x = 2.0 * math.pi * np.arange(N) / N
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return X, Y, Z


def taylor_green(N):
    """Taylor-Green initial velocity (Section 3.4, Eq. T-G-init) on an N^3 grid."""
    X, Y, Z = grid(N)
    u = np.empty((3, N, N, N))
    u[0] = np.sin(X) * np.cos(Y) * np.cos(Z)
    u[1] = -np.cos(X) * np.sin(Y) * np.cos(Z)
    u[2] = 0.0
    return u


def taylor_green_2d(N, amplitude=1.0):
    """2D Taylor-Green cells embedded in 3D (steady for the Euler equations)."""
    X, Y, _ = grid(N)
    u = np.zeros((3, N, N, N))
    u[0] = amplitude * np.sin(X) * np.cos(Y)
    u[1] = -amplitude * np.cos(X) * np.sin(Y)
    return u


def _kgrid(N):
    k = np.fft.fftfreq(N, 1.0 / N)
    KZ, KY, KX = np.meshgrid(k, k, k, indexing="ij")
    return KX, KY, KZ


def random_solenoidal(N, seed, kcut, energy_total=None, spectrum=None):
    """Random real solenoidal field u = curl A, band-limited to |k| <= kcut.

    ``spectrum(k)`` (vectorised over integer shells) gives the target shell energies, or
    None for the curl of white noise; ``energy_total`` rescales the whole field to that
    kinetic energy <|u|^2>/2.  Modes with any |k_i| = N/2 are zero.
    """
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((3, N, N, N))
    Ah = np.fft.fftn(A, axes=(1, 2, 3)) / float(N) ** 3
    KX, KY, KZ = _kgrid(N)
    uh = np.empty_like(Ah)
    uh[0] = 1j * (KY * Ah[2] - KZ * Ah[1])
    uh[1] = 1j * (KZ * Ah[0] - KX * Ah[2])
    uh[2] = 1j * (KX * Ah[1] - KY * Ah[0])
    K = np.sqrt(KX * KX + KY * KY + KZ * KZ)
    keep = (K <= kcut) & (np.abs(KX) < N // 2) & (np.abs(KY) < N // 2) & (np.abs(KZ) < N // 2)
    uh *= keep
    if spectrum is not None:
        shell = np.floor(K + 0.5).astype(int)
        e_mode = 0.5 * np.sum(np.abs(uh) ** 2, axis=0)
        e_shell = np.bincount(shell.ravel(), weights=e_mode.ravel())
        target = spectrum(np.arange(len(e_shell), dtype=float))
        scale = np.where(e_shell > 0, np.sqrt(target / np.where(e_shell > 0, e_shell, 1.0)), 0.0)
        uh *= scale[shell]
    u = np.real(np.fft.ifftn(uh * float(N) ** 3, axes=(1, 2, 3)))
    if energy_total is not None:
        e = 0.5 * np.mean(np.sum(u * u, axis=0))
        if e > 0:
            u *= math.sqrt(energy_total / e)
    return u


def hit_initial(N, seed, kp=4.0, energy_total=1.5, kcut=None):
    """Random-phase solenoidal field with E(k) ~ k^4 exp(-2 (k/kp)^2) and total energy 1.5."""
    kcut = (N // 2 - 1) if kcut is None else kcut
    return random_solenoidal(
        N, seed, kcut, energy_total=energy_total,
        spectrum=lambda k: k ** 4 * np.exp(-2.0 * (k / kp) ** 2))


def taylor_green_perturbed(N, seed, fraction=0.01, kcut=4):
    """Taylor-Green field plus a random solenoidal perturbation on |k| <= kcut with rms
    velocity ``fraction`` times the Taylor-Green rms velocity."""
    u = taylor_green(N)
    p = random_solenoidal(N, seed, kcut)
    rms_tg = math.sqrt(np.mean(np.sum(u * u, axis=0)))
    rms_p = math.sqrt(np.mean(np.sum(p * p, axis=0)))
    if rms_p > 0:
        u = u + p * (fraction * rms_tg / rms_p)
    return u


def cfl_dt(N, cfl, umax, t_end=None):
    """dt = cfl * dx / umax, rounded down so that t_end (if given) lands on a step."""
    dt = cfl * (2.0 * math.pi / N) / umax
    if t_end is not None:
        dt = t_end / math.ceil(t_end / dt)
    return dt

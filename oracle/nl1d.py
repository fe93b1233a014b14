"""The one-dimensional quadratic model of Section 3.3 (Eq. model-1d, the "nl1d" solver).

TEST INFRASTRUCTURE ONLY (see :mod:`oracle`).

Paper passages followed:

* Model -- Section 3.3, Eq. (model-1d): dS/dt = -sign(S) S^2 on [0, 2 pi), so wavenumbers are
  integers; for S > 0 it is dS/dt = -S^2 (Eq. model-1d-2) with the exact solution
  S0 / (1 + S0 t) (Eq. 1d_exact).
* Pseudo-spectral evaluation with truncation -- Section 3.2: the product is formed on the N
  grid points (so it aliases), transformed, and modes with |k| >= kmax = C_t k_N are zeroed;
  the DFT convention of the supplementary material (1/N on the forward transform).
* Time stepping -- Section 3.3 (one RK2 step keeps the dt^2 term S^3 of the Taylor
  expansion) with the RK2 of Section 4.1 without viscosity: the midpoint form
  S_half = S + dt/2 N(S), S_new = S + dt N(S_half).
* Real fields store k >= 0 only (the end of Section 3.3): an alias that would land at a
  negative wavenumber appears at its mirror 2 k_N - k_nl.

The state is the half spectrum S^(k), k = 0 .. N/2 (the Nyquist entry is zero whenever
kmax <= N/2).  numpy.fft serves as the transform.
"""
import numpy as np


def truncate(Sh, kmax):
    """Zero the modes with k >= kmax (Section 3.2)."""
    out = np.array(Sh, dtype=complex)
    out[np.arange(out.shape[-1]) >= kmax] = 0.0
    return out


def to_spectral(s):
    """Half spectrum with the 1/N forward normalisation."""
    s = np.asarray(s, dtype=float)
    return np.fft.rfft(s) / s.shape[-1]


def to_physical(Sh, N):
    return np.fft.irfft(np.asarray(Sh) * N, n=N)


def nonlinear(Sh, N, kmax):
    """T FFT[-sign(S) S^2] with the product taken on the N grid points (Eq. model-1d)."""
    s = to_physical(Sh, N)
    return truncate(to_spectral(-np.sign(s) * s * s), kmax)


def rk2_step(Sh, dt, N, kmax):
    half = Sh + 0.5 * dt * nonlinear(Sh, N, kmax)
    return Sh + dt * nonlinear(half, N, kmax)


def run(s0, dt, nsteps, kmax):
    """Half spectrum after nsteps RK2 steps from the physical field s0 (truncated first)."""
    N = len(s0)
    Sh = truncate(to_spectral(s0), kmax)
    for _ in range(nsteps):
        Sh = rk2_step(Sh, dt, N, kmax)
    return Sh


def initial(N, k0=10, amplitude=0.7):
    """S(x, 0) = 1 + 0.7 cos(k0 x) on the N grid points (Eq. 1d_initial, k0 = 10)."""
    x = 2 * np.pi * np.arange(N) / N
    return 1.0 + amplitude * np.cos(k0 * x)

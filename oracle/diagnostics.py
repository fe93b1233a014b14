"""Diagnostics of the oracle: energy, dissipation, spectra and the spectral error index.

TEST INFRASTRUCTURE ONLY (see :mod:`oracle`).

Paper passages followed:

* total kinetic energy E and dissipation rate eps as spatial means (Section 3.4,
  Fig. spatialmeans:192): E = <|u|^2>/2 = (1/2) sum_k |uh|^2 (Parseval with the 1/N
  convention of supplementary Eq. dft_def), eps = nu <|omega|^2> = nu sum_k k^2 |uh|^2;
* one-dimensional spectra E(k_x), E(k_y), E(k_z) and their use in the error index
  (Section 3.4, Eq. quality; Appendix A, Eq. quality-i-disc);
* shell spectrum E(k) on integer bins;
* nonlinear energy flux and cumulative dissipation (Section 3.4, Fig. spectra:192): the running
  sums over shells of the nonlinear transfer T(k) = sum_shell Re(uh* . Nh) and of the
  dissipation spectrum 2 nu k^2 E(k); flux Pi(k) = -sum_{k' <= k} T(k') (positive for a
  transfer towards small scales), cumulative dissipation D(k) = sum_{k' <= k} 2 nu k'^2 E(k');
* windowed error metrics (Section 6, Table tab:960): Err_early and Err_late are the error index
  over the first and second half of the output times, Err(Ebar) the relative error of the
  time-averaged spectra with the same weights.

Readings: half-spectrum sums use the Hermitian weights w (1 at kx = 0, 2 elsewhere);
shell bin = floor(|k| + 1/2); 1D spectra fold +/-k_i onto |k_i|; the discrete error index
sums k = 1 .. ceil(kmax) - 1 (the printed sum starts at k = 0 where its weight 1/k is
singular) and averages the three directions.
"""
import math

import numpy as np

from . import spectral as sp


def energy(S):
    N = S.shape[-2]
    w = sp.hermitian_weights(N)
    return 0.5 * float(np.sum(w * np.sum(np.abs(S) ** 2, axis=0)))


def dissipation(S, nu):
    N = S.shape[-2]
    KX, KY, KZ = sp.wavenumbers(N)
    w = sp.hermitian_weights(N)
    K2 = KX * KX + KY * KY + KZ * KZ
    return nu * float(np.sum(w * K2 * np.sum(np.abs(S) ** 2, axis=0)))


def enstrophy(S):
    """Z = <|omega|^2>/2 = (1/2) sum_k k^2 |uh|^2."""
    return dissipation(S, 1.0) * 0.5


def shell_bin(K2):
    """floor(|k| + 1/2) for integer k^2 (float64 square root)."""
    return np.floor(np.sqrt(K2) + 0.5).astype(int)


SPEC_SHELL = 0
SPEC_X = 1
SPEC_Y = 2
SPEC_Z = 3


def spectrum(S, kind, nbins):
    """Energy spectrum with ``nbins`` bins k = 0..nbins-1 (modes beyond are dropped)."""
    N = S.shape[-2]
    KX, KY, KZ = sp.wavenumbers(N)
    w = sp.hermitian_weights(N)
    e = 0.5 * w * np.sum(np.abs(S) ** 2, axis=0)
    if kind == SPEC_SHELL:
        b = shell_bin(KX * KX + KY * KY + KZ * KZ)
    elif kind == SPEC_X:
        b = np.abs(KX).astype(int)
    elif kind == SPEC_Y:
        b = np.abs(KY).astype(int)
    elif kind == SPEC_Z:
        b = np.abs(KZ).astype(int)
    else:
        raise ValueError("unknown spectrum kind")
    out = np.zeros(nbins)
    ok = b < nbins
    np.add.at(out, b[ok], e[ok])
    return out


def error_index(spectra, spectra_ref, kmax):
    """Discrete spectral error index (Appendix A, Eq. quality-i-disc), averaged over x, y, z.

    spectra, spectra_ref: sequences over output times of (E_x, E_y, E_z) 1D spectra.
    Reading: k = 1 .. ceil(kmax) - 1, weights 1/k.
    """
    kend = int(math.ceil(kmax)) - 1
    ks = np.arange(1, kend + 1, dtype=float)
    wk = 1.0 / ks
    Nt = len(spectra)
    errs = []
    for d in range(3):
        tot = 0.0
        for j in range(Nt):
            E = np.asarray(spectra[j][d])[1 : kend + 1]
            Er = np.asarray(spectra_ref[j][d])[1 : kend + 1]
            tot += float(np.sum(wk * 100.0 * np.abs(Er - E) / Er))
        errs.append(tot / (Nt * float(np.sum(wk))))
    return float(np.mean(errs))


def _shell_sum(N, values, nbins):
    """Sum of half-spectrum values (already weighted) over shell bins 0..nbins-1."""
    KX, KY, KZ = sp.wavenumbers(N)
    b = shell_bin(KX * KX + KY * KY + KZ * KZ)
    out = np.zeros(nbins)
    ok = b < nbins
    np.add.at(out, b[ok], values[ok])
    return out


def transfer_spectrum(S, Nl, nbins):
    """T(k): energy change rate of shell k due to the nonlinear term Nl (both [3][N][N][N/2]).

    d/dt (1/2)|uh|^2 = Re(uh* . duh/dt) over the full spectrum, Hermitian weights w on the
    half spectrum.
    """
    N = S.shape[-2]
    w = sp.hermitian_weights(N)
    t = w * np.sum(np.real(np.conj(S) * Nl), axis=0)
    return _shell_sum(N, t, nbins)


def energy_flux(S, Nl, nbins):
    """Pi(k) = -sum_{k' <= k} T(k')."""
    return -np.cumsum(transfer_spectrum(S, Nl, nbins))


def dissipation_spectrum(S, nu, nbins):
    N = S.shape[-2]
    KX, KY, KZ = sp.wavenumbers(N)
    w = sp.hermitian_weights(N)
    K2 = KX * KX + KY * KY + KZ * KZ
    return _shell_sum(N, nu * w * K2 * np.sum(np.abs(S) ** 2, axis=0), nbins)


def cumulative_dissipation(S, nu, nbins):
    """D(k) = sum_{k' <= k} 2 nu k'^2 E(k') (tends to eps at the last shell)."""
    return np.cumsum(dissipation_spectrum(S, nu, nbins))


def error_index_windows(spectra, spectra_ref, kmax):
    """(Err_early, Err_late, Err(Ebar)) over a sequence of output times (Table tab:960).

    The first half of the samples is the early window, the second half the late one (an odd
    count puts the middle sample in both); Err(Ebar) compares the spectra averaged over all
    samples with the error index's weights.
    """
    Nt = len(spectra)
    h = (Nt + 1) // 2
    early = error_index(spectra[:h], spectra_ref[:h], kmax)
    late = error_index(spectra[Nt - h:], spectra_ref[Nt - h:], kmax)
    mean = [tuple(np.mean([np.asarray(s[d]) for s in spectra], axis=0) for d in range(3))]
    mean_ref = [tuple(np.mean([np.asarray(s[d]) for s in spectra_ref], axis=0) for d in range(3))]
    return early, late, error_index(mean, mean_ref, kmax)

"""Host-side analysis of the library's outputs (measurement, not the compute path).

error_index: the spectral error index of the paper (Sec. 3.4, Eq. quality; Appendix A,
Eq. quality-i-disc) computed from 1D energy spectra returned by ns_energy_spectrum.
error_index_windows: Err_early, Err_late and Err(Ebar) of Sec. 6 (Table tab:960): the index
over the first and second half of the samples and on the time-averaged spectra.
Reading of the discrete formula: the sum runs over k = 1 .. ceil(kmax) - 1 (the printed sum
starts at k = 0, where its weight 1/k is singular), with weights 1/k, averaged over time
samples and over the x, y, z spectra.
"""
import math

import numpy as np


def error_index(spectra, spectra_ref, kmax):
    """Mean over x, y, z of the log-k-weighted relative error (%) of 1D spectra.

    spectra, spectra_ref: sequences over time samples of (E_x, E_y, E_z) arrays indexed by k.
    """
    kend = int(math.ceil(kmax)) - 1
    k = np.arange(1, kend + 1, dtype=float)
    wk = 1.0 / k
    out = []
    for d in range(3):
        acc = 0.0
        for s, r in zip(spectra, spectra_ref):
            E = np.asarray(s[d], dtype=float)[1:kend + 1]
            Er = np.asarray(r[d], dtype=float)[1:kend + 1]
            acc += float(np.sum(wk * 100.0 * np.abs(Er - E) / Er))
        out.append(acc / (len(spectra) * float(np.sum(wk))))
    return float(np.mean(out))


def error_index_windows(spectra, spectra_ref, kmax):
    """(Err_early, Err_late, Err(Ebar)): the first / second half of the samples (the middle
    one in both when their count is odd) and the spectra averaged over every sample."""
    n = len(spectra)
    h = (n + 1) // 2
    early = error_index(spectra[:h], spectra_ref[:h], kmax)
    late = error_index(spectra[n - h:], spectra_ref[n - h:], kmax)

    def avg(seq):
        return [tuple(np.mean([np.asarray(s[d], dtype=float) for s in seq], axis=0) for d in range(3))]

    return early, late, error_index(avg(spectra), avg(spectra_ref), kmax)

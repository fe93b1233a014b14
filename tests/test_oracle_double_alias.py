"""Pins of the "no double aliases" truncation (Section 4.2, Fig.
truncation:spherical:double:aliases(b); supplementary classification of alias classes).

The mask is checked against things other than its own formula: the brute-force alias-class
convolution (no double-alias class may land on a retained mode), the 3/2-padded alias-free
product (with it, the isotropic phase-shift average is alias-free at any C_t), the
Patterson-Orszag threshold 2 sqrt(2)/3, and the symmetries of the lattice.
"""
import math

import numpy as np
import pytest

from oracle import nonlinear as nl
from oracle import spectral as sp
from paper_2603_08892_gb300 import inputs


def full_from_half(N, mask_half):
    """Full-spectrum [N, N, N] boolean mask from the half spectrum (Hermitian mirror)."""
    full = np.zeros((N, N, N), dtype=bool)
    full[:, :, : N // 2] = mask_half
    k = np.fft.fftfreq(N, 1.0 / N).astype(int)
    for ix in range(N // 2 + 1, N):  # kx < 0: mirror of -k
        mx = (-k[ix]) % N
        full[:, :, ix] = mask_half[np.ix_((-k) % N, (-k) % N, [mx])][:, :, 0]
    return full


def random_truncated_full(N, mask_full, seed):
    rng = np.random.default_rng(seed)
    uf = np.fft.fftn(rng.standard_normal((N, N, N))) / N ** 3
    return uf * mask_full


@pytest.mark.parametrize("N", [8, 12])
def test_no_double_alias_class_lands_on_a_retained_mode(N):
    kmax = N / 2.0  # C_t = 1: double aliases exist
    sph = full_from_half(N, sp.truncation_mask(N, kmax))
    nda = full_from_half(N, sp.truncation_mask(N, kmax, sp.TRUNC_NO_DOUBLE_ALIAS))
    # products of spherically retained modes, split by alias class (brute force)
    W = nl.classified_convolution(random_truncated_full(N, sph, 1), random_truncated_full(N, sph, 2))
    doubles = [e for e in W if sum(c != 0 for c in e) == 2]
    assert len(doubles) == 12
    landed_sph = max(np.abs(W[e][sph]).max() for e in doubles)
    landed_nda = max(np.abs(W[e][nda]).max() for e in doubles)
    if N >= 12:
        assert landed_sph > 1e-4  # the spherical truncation keeps modes double aliases reach
    assert landed_nda == 0.0      # none of them survives the no-double-alias truncation


@pytest.mark.parametrize("N,ct", [(12, 1.0), (16, 1.0), (24, 0.97)])
def test_phase_shift_exact_is_alias_free_with_no_double_aliases(N, ct):
    # single and triple aliases cancel in the isotropic average, double aliases are masked:
    # the nonlinear term equals the 3/2-padded (alias-free) one with the same truncation
    kmax = ct * N / 2.0
    kind = sp.TRUNC_NO_DOUBLE_ALIAS
    S = sp.set_velocity(inputs.random_solenoidal(N, 5, kcut=N / 2), kmax, kind)
    dx = 2 * math.pi / N
    avg = 0.5 * (nl.nonlinear(S, [0, 0, 0], kmax, kind) + nl.nonlinear(S, [dx / 2] * 3, kmax, kind))
    pad = nl.nonlinear_padded(S, kmax, kind)
    scale = np.abs(pad).max()
    assert np.abs(avg - pad).max() < 1e-14 * scale
    # with the purely spherical truncation the same average keeps the double aliases
    Ss = sp.set_velocity(inputs.random_solenoidal(N, 5, kcut=N / 2), kmax)
    avg_s = 0.5 * (nl.nonlinear(Ss, [0, 0, 0], kmax) + nl.nonlinear(Ss, [dx / 2] * 3, kmax))
    assert np.abs(avg_s - nl.nonlinear_padded(Ss, kmax)).max() > 1e-6 * scale


@pytest.mark.parametrize("N", [12, 16, 24, 48])
def test_nothing_removed_up_to_the_patterson_orszag_threshold(N):
    # a spherical truncation at (2 sqrt 2 / 3) k_N already excludes every double alias
    for ct in (2.0 / 3.0, 0.9, 2 * math.sqrt(2) / 3 * (1 - 1e-9)):
        kmax = ct * N / 2
        assert np.array_equal(sp.truncation_mask(N, kmax, sp.TRUNC_NO_DOUBLE_ALIAS),
                              sp.truncation_mask(N, kmax))
    # above it modes near the edges of the cube (two large components) are removed
    kmax = N / 2
    removed = sp.truncation_mask(N, kmax) & ~sp.truncation_mask(N, kmax, sp.TRUNC_NO_DOUBLE_ALIAS)
    KX, KY, KZ = sp.wavenumbers(N)
    big = [np.abs(K[removed]) for K in (KX, KY, KZ)]
    # the removed region lies near the edges of the cube: no removed mode is on an axis
    assert removed.sum() > 0
    assert np.all((big[0] > 0).astype(int) + (big[1] > 0).astype(int) + (big[2] > 0).astype(int) >= 2)


def test_mask_symmetries():
    N, kmax = 16, 8.0
    m = full_from_half(N, sp.truncation_mask(N, kmax, sp.TRUNC_NO_DOUBLE_ALIAS))
    # invariant under permutations of the axes and under k -> -k of any component
    assert np.array_equal(m, np.transpose(m, (1, 0, 2)))
    assert np.array_equal(m, np.transpose(m, (2, 1, 0)))
    k = np.fft.fftfreq(N, 1.0 / N).astype(int)
    flip = (-k) % N
    assert np.array_equal(m, m[flip, :, :]) and np.array_equal(m, m[:, flip, :])

"""Pins of the oracle's spectral basics against definitions, closed forms and brute force."""
import math

import numpy as np
import pytest

from oracle import diagnostics as dg
from oracle import spectral as sp
from paper_2603_08892_gb300 import inputs


def direct_dft(u):
    """Triple sum of supplementary Eq. (dft_def) applied in x, y, z (O(N^6))."""
    N = u.shape[-1]
    j = np.arange(N)
    x = 2.0 * math.pi * j / N
    k = np.fft.fftfreq(N, 1.0 / N)
    out = np.zeros((N, N, N // 2), dtype=complex)
    for iz in range(N):
        for iy in range(N):
            for ix in range(N // 2):
                ph = np.exp(-1j * (k[iz] * x[:, None, None] + k[iy] * x[None, :, None]
                                   + ix * x[None, None, :]))
                out[iz, iy, ix] = np.sum(u * ph) / N ** 3
    return out


@pytest.mark.parametrize("N", [6, 8])
def test_forward_matches_direct_dft(N):
    rng = np.random.default_rng(1)
    u = rng.standard_normal((N, N, N))
    np.testing.assert_allclose(sp.forward(u[None])[0], direct_dft(u), atol=1e-14)


def test_single_mode_layout_and_roundtrip():
    N = 8
    X, Y, Z = inputs.grid(N)
    u = np.cos(2 * X + 3 * Y - Z)
    uh = sp.forward(u[None])[0]
    # cos(k.x) = (e^{ik.x} + e^{-ik.x})/2 -> 1/2 at k = (2, 3, -1), index [kz, ky, kx]
    expect = np.zeros_like(uh)
    expect[-1 % N, 3, 2] = 0.5
    np.testing.assert_allclose(uh, expect, atol=1e-15)
    np.testing.assert_allclose(sp.inverse(uh[None])[0], u, atol=1e-14)


def test_parseval_energy():
    N = 12
    u = inputs.random_solenoidal(N, 3, kcut=5)
    S = sp.forward(u)
    e_phys = 0.5 * np.mean(np.sum(u * u, axis=0))
    assert abs(dg.energy(S) - e_phys) < 1e-14


def test_projection_closed_form():
    # A = (sin2x cos2z, 0, 0); grad phi with lap phi = div A gives
    # P A = (1/2 sin2x cos2z, 0, -1/2 cos2x sin2z)
    N = 8
    X, Y, Z = inputs.grid(N)
    A = np.zeros((3, N, N, N))
    A[0] = np.sin(2 * X) * np.cos(2 * Z)
    expect = np.zeros_like(A)
    expect[0] = 0.5 * np.sin(2 * X) * np.cos(2 * Z)
    expect[2] = -0.5 * np.cos(2 * X) * np.sin(2 * Z)
    got = sp.inverse(sp.project(sp.forward(A)))
    np.testing.assert_allclose(got, expect, atol=1e-14)


def test_projection_idempotent_kills_gradients():
    N = 12
    rng = np.random.default_rng(2)
    v = sp.forward(rng.standard_normal((3, N, N, N)))
    Pv = sp.project(v)
    assert sp.divergence_ratio(Pv) < 1e-15
    np.testing.assert_allclose(sp.project(Pv), Pv, atol=1e-16)
    KX, KY, KZ = sp.wavenumbers(N)
    phi = sp.forward(rng.standard_normal((1, N, N, N)))[0]
    grad = np.stack([1j * KX * phi, 1j * KY * phi, 1j * KZ * phi])
    assert np.abs(sp.project(grad)).max() < 1e-16


def lattice_count(kmax, cubic=False):
    K = int(math.ceil(kmax)) + 1
    n = 0
    for a in range(-K, K + 1):
        for b in range(-K, K + 1):
            for c in range(-K, K + 1):
                if cubic:
                    n += max(abs(a), abs(b), abs(c)) < kmax
                else:
                    n += a * a + b * b + c * c < kmax * kmax
    return n


def test_truncation_counts():
    # k^2 < 4 keeps exactly {-1,0,1}^3 (27 points); "<=" would add (+-2,0,0) etc.
    N = 8
    m = sp.truncation_mask(N, 2.0)
    assert int(np.sum(sp.hermitian_weights(N) * m)) == 27
    for N, kmax in [(12, 4.0), (12, 2 * math.sqrt(2) / 3 * 6), (16, 16 / 3.0), (16, 8.0)]:
        w = sp.hermitian_weights(N)
        assert int(np.sum(w * sp.truncation_mask(N, kmax))) == lattice_count(kmax)
        assert int(np.sum(w * sp.truncation_mask(N, kmax, sp.TRUNC_CUBIC))) == \
            lattice_count(kmax, cubic=True)


def test_kmax_thresholds_exact_integers():
    assert sp.kmax2_threshold(128.0) == 16383
    assert sp.kmax2_threshold(2 * math.sqrt(2) / 3 * 16) == 227
    assert sp.kmax_int_threshold(4.0) == 3
    assert sp.kmax_int_threshold(4.5) == 4


def test_spectra_sum_and_bins():
    N = 12
    S = sp.forward(inputs.random_solenoidal(N, 5, kcut=5))
    E = dg.energy(S)
    for kind in (dg.SPEC_SHELL, dg.SPEC_X, dg.SPEC_Y, dg.SPEC_Z):
        assert abs(dg.spectrum(S, kind, 2 * N).sum() - E) < 1e-14
    X, Y, Z = inputs.grid(N)
    u = np.zeros((3, N, N, N))
    u[0] = np.cos(3 * Y + 4 * Z)  # |k| = 5, energy 1/4
    S = sp.forward(u)
    sh = dg.spectrum(S, dg.SPEC_SHELL, 8)
    assert abs(sh[5] - 0.25) < 1e-15 and abs(sh.sum() - 0.25) < 1e-15
    ey = dg.spectrum(S, dg.SPEC_Y, 8)
    assert abs(ey[3] - 0.25) < 1e-15
    ex = dg.spectrum(S, dg.SPEC_X, 8)
    assert abs(ex[0] - 0.25) < 1e-15


def test_error_index_special_cases():
    ref = [(np.linspace(1, 2, 10), np.linspace(1, 3, 10), np.linspace(2, 3, 10))] * 3
    assert dg.error_index(ref, ref, 9.0) == 0.0
    scaled = [tuple(1.1 * a for a in r) for r in ref]
    assert abs(dg.error_index(scaled, ref, 9.0) - 10.0) < 1e-12
    # a 20% error at k = 1 only: weight (1/1) / sum_{k=1}^{8} 1/k
    one = [tuple(np.where(np.arange(10) == 1, 1.2, 1.0) * a for a in r) for r in ref]
    H8 = sum(1.0 / k for k in range(1, 9))
    assert abs(dg.error_index(one, ref, 9.0) - 20.0 / H8) < 1e-12


def test_package_error_index_agrees_with_oracle():
    from paper_2603_08892_gb300 import analysis

    rs = np.random.default_rng(4)
    a = [tuple(rs.random(20) + 0.5 for _ in range(3)) for _ in range(4)]
    b = [tuple(rs.random(20) + 0.5 for _ in range(3)) for _ in range(4)]
    assert abs(analysis.error_index(a, b, 15.5) - dg.error_index(a, b, 15.5)) < 1e-12


def test_package_windowed_error_metrics_agree_with_oracle():
    from paper_2603_08892_gb300 import analysis

    rs = np.random.default_rng(6)
    a = [tuple(rs.random(20) + 0.5 for _ in range(3)) for _ in range(5)]
    b = [tuple(rs.random(20) + 0.5 for _ in range(3)) for _ in range(5)]
    got = analysis.error_index_windows(a, b, 15.5)
    ref = dg.error_index_windows(a, b, 15.5)
    assert max(abs(x - y) for x, y in zip(got, ref)) < 1e-12

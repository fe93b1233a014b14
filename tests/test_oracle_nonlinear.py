"""Pins of the oracle's nonlinear term: brute-force alias classes, closed forms, invariants."""
import math

import numpy as np
import pytest

from oracle import nonlinear as nl
from oracle import spectral as sp
from oracle import diagnostics as dg
from paper_2603_08892_gb300 import inputs


def band_limited_real(N, seed):
    """Random real field whose spectrum has every |k_i| < N/2 (no Nyquist content)."""
    rng = np.random.default_rng(seed)
    uf = np.fft.fftn(rng.standard_normal((N, N, N))) / N ** 3
    k = np.fft.fftfreq(N, 1.0 / N)
    bad = np.abs(k) >= N // 2
    uf[bad, :, :] = 0
    uf[:, bad, :] = 0
    uf[:, :, bad] = 0
    return np.real(np.fft.ifftn(uf * N ** 3))


def shifted_product_hat(u, v, delta):
    """De-shifted product exp(-ik.D) FFT[u_D v_D] through the oracle's transforms."""
    N = u.shape[-1]
    sh = sp.shift_factor(N, delta)
    uh = sp.forward(u[None])[0] * sh
    vh = sp.forward(v[None])[0] * sh
    prod = sp.inverse(uh[None])[0] * sp.inverse(vh[None])[0]
    return sp.forward(prod[None])[0] * np.conj(sh)


@pytest.mark.parametrize("N", [6, 8])
def test_alias_classes_brute_force(N):
    u = band_limited_real(N, 10)
    v = band_limited_real(N, 11)
    W = nl.classified_convolution(np.fft.fftn(u) / N ** 3, np.fft.fftn(v) / N ** 3)
    half = (slice(None), slice(None), slice(0, N // 2))
    rng = np.random.default_rng(3)
    dx = 2 * math.pi / N
    for U in ([0.0, 0.0, 0.0], [0.5, 0.5, 0.5], list(rng.random(3)), [0.5, 0.0, 0.25]):
        got = shifted_product_hat(u, v, [dx * c for c in U])
        # each aliased direction i carries exp(i 2 k_N e_i Delta_i) = exp(i 2 pi e_i U_i)
        expect = sum(np.exp(2j * math.pi * (e[0] * U[0] + e[1] * U[1] + e[2] * U[2])) * W[e]
                     for e in W)
        np.testing.assert_allclose(got, expect[half], atol=1e-13)
    # the isotropic half-cell shift flips single and triple aliases, keeps double aliases
    avg = 0.5 * (shifted_product_hat(u, v, [0, 0, 0]) + shifted_product_hat(u, v, [dx / 2] * 3))
    even = sum(W[e] for e in W if sum(abs(c) for c in e) in (0, 2))
    np.testing.assert_allclose(avg, even[half], atol=1e-13)
    # there is aliasing to cancel in this test at all
    assert np.abs(W[(1, 0, 0)]).max() > 1e-3 and np.abs(W[(1, 1, 0)]).max() > 1e-4


@pytest.mark.parametrize("N", [12, 16])
def test_ps_exact_is_alias_free_at_2sqrt2_over_3(N):
    kmax = 2 * math.sqrt(2) / 3 * (N / 2)
    S = sp.set_velocity(inputs.random_solenoidal(N, 4, kcut=N / 2), kmax)
    dx = 2 * math.pi / N
    avg = 0.5 * (nl.nonlinear(S, [0, 0, 0], kmax) + nl.nonlinear(S, [dx / 2] * 3, kmax))
    pad = nl.nonlinear_padded(S, kmax)
    scale = np.abs(pad).max()
    assert np.abs(avg - pad).max() < 1e-14 * max(scale, 1.0)
    # and the unshifted term alone is aliased
    assert np.abs(nl.nonlinear(S, [0, 0, 0], kmax) - pad).max() > 1e-6 * scale


@pytest.mark.parametrize("N", [8, 12, 16])
def test_taylor_green_first_evaluation_closed_form(N):
    X, Y, Z = inputs.grid(N)
    S = sp.set_velocity(inputs.taylor_green(N), N / 2)
    expect = np.stack([-np.sin(2 * X) * np.cos(2 * Z) / 8,
                       -np.sin(2 * Y) * np.cos(2 * Z) / 8,
                       (np.cos(2 * X) + np.cos(2 * Y)) * np.sin(2 * Z) / 8])
    dx = 2 * math.pi / N
    for delta in ([0, 0, 0], [dx / 2] * 3, [0.1 * dx, 0.7 * dx, 0.33 * dx]):
        got = sp.inverse(nl.nonlinear(S, delta, N / 2))
        np.testing.assert_allclose(got, expect, atol=1e-15)
        got = sp.inverse(nl.nonlinear_advective(S, delta, N / 2))
        np.testing.assert_allclose(got, expect, atol=1e-15)


def test_taylor_green_invariants():
    N = 16
    nu = 1.0 / 1600
    S = sp.set_velocity(inputs.taylor_green(N), N / 2)
    assert abs(dg.energy(S) - 1 / 8) < 1e-15
    assert abs(dg.dissipation(S, nu) - 3 * nu / 4) < 1e-17


def test_2d_taylor_green_has_no_nonlinear_term():
    N = 12
    S = sp.set_velocity(inputs.taylor_green_2d(N), N / 2)
    dx = 2 * math.pi / N
    for delta in ([0, 0, 0], [0.3 * dx, 0.9 * dx, 0.5 * dx]):
        assert np.abs(nl.nonlinear(S, delta, N / 2)).max() < 1e-16


@pytest.mark.parametrize("kmax_frac", [1.0, 2.0 / 3.0])
def test_energy_conservation_and_solenoidal(kmax_frac):
    N = 12
    kmax = kmax_frac * N / 2
    S = sp.set_velocity(inputs.random_solenoidal(N, 7, kcut=N / 2), kmax)
    w = sp.hermitian_weights(N)
    dx = 2 * math.pi / N
    for delta in ([0, 0, 0], [dx / 2] * 3, [0.37 * dx, 0.11 * dx, 0.93 * dx]):
        Nh = nl.nonlinear(S, delta, kmax)
        transfer = np.sum(w * np.real(np.sum(np.conj(S) * Nh, axis=0)))
        assert abs(transfer) < 1e-15 * np.abs(Nh).max() * max(1.0, np.abs(S).max()) * N ** 3
        assert sp.divergence_ratio(Nh) < 1e-14
        KX, KY, KZ = sp.wavenumbers(N)
        assert np.abs(Nh[:, ~sp.truncation_mask(N, kmax)]).max() == 0.0


def test_rotational_equals_advective_without_aliasing():
    N = 12
    kmax = 2.0 / 3.0 * N / 2
    S = sp.set_velocity(inputs.random_solenoidal(N, 8, kcut=N / 2), kmax)
    a = nl.nonlinear(S, [0, 0, 0], kmax)
    b = nl.nonlinear_advective(S, [0, 0, 0], kmax)
    np.testing.assert_allclose(a, b, atol=1e-14)
    # with aliasing (C_t = 1) the two forms differ
    kmax = N / 2
    S = sp.set_velocity(inputs.random_solenoidal(N, 8, kcut=N / 2), kmax)
    assert np.abs(nl.nonlinear(S, [0, 0, 0], kmax) - nl.nonlinear_advective(S, [0, 0, 0], kmax)).max() > 1e-6

"""Nonlinear term of the oracle, with phase shifting, plus the alias-analysis references.

TEST INFRASTRUCTURE ONLY (see :mod:`oracle`).

Paper passages followed:

* Pseudo-spectral product: two inverse FFTs, a pointwise product, one forward FFT --
  Section 3.1, Eq. (w_product_convo) and the paragraph after it.
* Discrete convolution with aliases, 3D classes e in {-1,0,1}^3 -- supplementary
  Eqs. (orthogonality_3D), (alias_full): w(k) = sum_e sum_{kn+km-k = 2 k_N e} u(kn) v(km).
* Shifted and de-shifted product -- Section 4.1, Eqs. (rogallo_ps_1)-(rogallo_ps_3) and
  Section 4.2: each aliased direction i picks up exp(i 2 k_N e_i Delta_i).
* Nonlinear operator N(S) = projection of the quadratic term onto divergence-free fields --
  Section 4.1 below Eq. (base-eq).  The oracle evaluates it in rotational form
  P(u x omega); the advective form -P(u . grad u) is provided as well and equals it when
  no aliasing occurs (u x omega and -u.grad u differ by the gradient grad(|u|^2/2)).
"""
import numpy as np

from . import spectral as sp


def shifted_fields(uh, delta):
    """Velocity and vorticity on the grid shifted by delta: IFFT(exp(ik.delta) uh), IFFT(ik x ...)."""
    N = uh.shape[-2]
    us = uh * sp.shift_factor(N, delta)
    return sp.inverse(us), sp.inverse(sp.curl(us))


def cross(a, b):
    """Pointwise cross product of two 3-component physical fields."""
    return np.stack(
        [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]
    )


def nonlinear(uh, delta, kmax, kind=sp.TRUNC_SPHERICAL):
    """Shifted-and-de-shifted nonlinear term  N~_Delta(S) = T P exp(-ik.Delta) FFT[u_Delta x w_Delta].

    Section 4.1 (definition of N~ after Eq. sum_ps_non_ps) with the 3D shift operator of
    Section 4.2; T is the truncation mask (Section 3.2), P the Leray projection; the mean
    mode is set to zero.  delta = (0, 0, 0) gives the plain (aliased) nonlinear term.
    """
    N = uh.shape[-2]
    u, w = shifted_fields(uh, delta)
    Fh = sp.forward(cross(u, w)) * np.conj(sp.shift_factor(N, delta))
    Fh = Fh * sp.truncation_mask(N, kmax, kind)
    return sp.project(Fh)


def nonlinear_advective(uh, delta, kmax, kind=sp.TRUNC_SPHERICAL):
    """Same as :func:`nonlinear` with the advective form -u . grad u (Section 2, Eq. N-S-incompr-qdm)."""
    N = uh.shape[-2]
    KX, KY, KZ = sp.wavenumbers(N)
    sh = sp.shift_factor(N, delta)
    us = uh * sh
    u = sp.inverse(us)
    adv = np.zeros_like(u)
    for j, K in enumerate((KX, KY, KZ)):
        # d/dx_j of every component, then contract with u_j
        du = sp.inverse(1j * K * us)
        adv += u[j] * du
    Fh = sp.forward(-adv) * np.conj(sh)
    Fh = Fh * sp.truncation_mask(N, kmax, kind)
    return sp.project(Fh)


# --------------------------------------------------------------------------------------
# References used to pin the phase-shift mechanics (not used by the schemes themselves)
# --------------------------------------------------------------------------------------


def full_spectrum(uh):
    """Half spectrum [N, N, N/2] -> full spectrum [N, N, N] of a real field (Hermitian mirror).

    The kx = -N/2 plane is zero (the half spectrum has no Nyquist plane).
    """
    N = uh.shape[-2]
    return np.fft.fftn(np.real(sp.inverse(uh[None])[0]), axes=(0, 1, 2)) / float(N) ** 3


def classified_convolution(uf, vf):
    """Brute-force discrete convolution split by alias class (supplementary Eq. alias_full).

    uf, vf: full spectra [N, N, N] in FFT index order (k in [-N/2, N/2)).  Returns a dict
    e -> W_e (full spectrum [N, N, N]) with
        W_e(k) = sum_{kn, km in K, kn + km - k = N e} uf(kn) vf(km),
    for e in {-1, 0, 1}^3 (2 k_N = N since L = 2*pi).  The plain pseudo-spectral product is
    sum_e W_e (supplementary Eq. rogallo_double_sum).  O(27 N^6): only for N <= 12.
    """
    N = uf.shape[0]
    k = np.fft.fftfreq(N, 1.0 / N).astype(int)  # wavenumber of each index
    # index of a wavenumber, valid only for wavenumbers in [-N/2, N/2)
    def idx(kk):
        return np.mod(kk, N)

    KZ, KY, KX = np.meshgrid(k, k, k, indexing="ij")  # output wavenumbers
    out = {}
    for ez in (-1, 0, 1):
        for ey in (-1, 0, 1):
            for ex in (-1, 0, 1):
                W = np.zeros((N, N, N), dtype=complex)
                for iz in range(N):
                    for iy in range(N):
                        for ix in range(N):
                            a = uf[iz, iy, ix]
                            if a == 0:
                                continue
                            # km = k + N e - kn, must lie in [-N/2, N/2)
                            mz = KZ + N * ez - k[iz]
                            my = KY + N * ey - k[iy]
                            mx = KX + N * ex - k[ix]
                            ok = (
                                (mz >= -N // 2) & (mz < N // 2)
                                & (my >= -N // 2) & (my < N // 2)
                                & (mx >= -N // 2) & (mx < N // 2)
                            )
                            W[ok] += a * vf[idx(mz[ok]), idx(my[ok]), idx(mx[ok])]
                out[(ex, ey, ez)] = W
    return out


def padded_product_hat(uh, vh):
    """Alias-free product of two real fields by the 3/2 zero-padding rule (Section 1).

    uh, vh: half spectra [N, N, N/2] with every |k_i| < N/2.  The spectra are zero-padded
    to M = 3N/2 points per direction, multiplied on the M grid and truncated back to N;
    the result is the clean (e = 0) part of the convolution for |k_i| < N/2.
    """
    N = uh.shape[-2]
    if (3 * N) % 4:
        raise ValueError("need 3N/2 even")
    M = 3 * N // 2

    def pad(h):
        big = np.zeros((M, M, M // 2), dtype=complex)
        k = np.fft.fftfreq(N, 1.0 / N).astype(int)
        iz = np.mod(k, M)
        big[np.ix_(iz, iz, np.arange(N // 2))] = h
        return big

    def unpad(H):
        k = np.fft.fftfreq(N, 1.0 / N).astype(int)
        iz = np.mod(k, M)
        return H[np.ix_(iz, iz, np.arange(N // 2))]

    pu = sp.inverse(pad(uh)[None])[0]
    pv = sp.inverse(pad(vh)[None])[0]
    return unpad(sp.forward((pu * pv)[None])[0])


def nonlinear_padded(uh, kmax, kind=sp.TRUNC_SPHERICAL):
    """Alias-free nonlinear term T P FFT[u x w] with the 3/2-padded product (textbook dealiasing)."""
    N = uh.shape[-2]
    w = sp.curl(uh)
    Fh = np.empty_like(uh)
    for c, (a, b) in enumerate(((1, 2), (2, 0), (0, 1))):
        Fh[c] = padded_product_hat(uh[a], w[b]) - padded_product_hat(uh[b], w[a])
    Fh = Fh * sp.truncation_mask(N, kmax, kind)
    return sp.project(Fh)

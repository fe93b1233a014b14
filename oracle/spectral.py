"""Spectral basics of the oracle: DFT convention, wavenumbers, truncation, projection, shifts.

TEST INFRASTRUCTURE ONLY (see :mod:`oracle`).

Paper passages followed:

* DFT convention -- supplementary material, Eq. (dft_def): the forward transform carries
  the 1/N factor per direction, the inverse none; wavenumbers k in [-N/2, N/2-1].
* Domain size 2*pi so that wavenumbers are integers -- Section 2 (numerical methods).
* Truncations -- Section 3.2, Fig. truncation:common: "cubic" zeroes modes with any
  |k_i| >= kmax, "spherical" zeroes modes with |k| >= kmax, kmax = C_t k_N.  "No double
  aliases" (Section 4.2, Fig. truncation:spherical:double:aliases(b); supplementary alias
  classes): the spherical truncation minus every mode that a double alias can reach.
* Leray projection onto divergence-free fields -- Section 4.1 below Eq. (base-eq): the
  nonlinear term is the projection of the advective term onto the divergence-free space.
* Phase-shift operator -- Section 4.2, Eq. (shift_operator_3d): P_Delta(X) = exp(i k.Delta) X,
  inverse exp(-i k.Delta) X.
"""
import numpy as np

TRUNC_SPHERICAL = 0

# Threads of the 3D transforms.  None: numpy.fft (single thread).  An integer n: scipy.fft
# with n workers -- the same pocketfft algorithm, split across threads, for the full-size
# (256^3 and larger) oracle runs of the tests and of the timed CPU baseline.
_FFT_WORKERS = None


def set_fft_workers(n):
    """Use ``n`` threads for the 3D transforms (None: numpy.fft, one thread); returns the old value."""
    global _FFT_WORKERS
    old, _FFT_WORKERS = _FFT_WORKERS, (None if n is None else max(1, int(n)))
    return old


def _rfftn(u):
    if _FFT_WORKERS is None:
        return np.fft.rfftn(u, axes=(-3, -2, -1))
    import scipy.fft

    return scipy.fft.rfftn(u, axes=(-3, -2, -1), workers=_FFT_WORKERS)


def _irfftn(full, N):
    if _FFT_WORKERS is None:
        return np.fft.irfftn(full, s=(N, N, N), axes=(-3, -2, -1))
    import scipy.fft

    return scipy.fft.irfftn(full, s=(N, N, N), axes=(-3, -2, -1), workers=_FFT_WORKERS)
TRUNC_CUBIC = 1
TRUNC_NO_DOUBLE_ALIAS = 2


def wavenumbers(N):
    """Integer wavenumber grids (KX, KY, KZ), each of shape (N, N, N//2), index order [kz, ky, kx].

    kz, ky follow FFT order 0..N/2-1, -N/2..-1; kx = 0..N/2-1 (half spectrum, Nyquist
    plane dropped).  L = 2*pi so k is an integer (Section 2).
    """
    if N % 2:
        raise ValueError("N must be even")
    k = np.fft.fftfreq(N, 1.0 / N)
    kx = np.arange(N // 2, dtype=float)
    KZ, KY, KX = np.meshgrid(k, k, kx, indexing="ij")
    return KX, KY, KZ


def hermitian_weights(N):
    """Weights w of the half spectrum for sums over the full spectrum: 1 at kx = 0, else 2.

    A real field has uh(-k) = conj(uh(k)) (Section 3.3, last paragraph), so a sum over all
    k of a real-valued quadratic form equals the half-spectrum sum weighted by w.
    """
    w = np.full((N, N, N // 2), 2.0)
    w[:, :, 0] = 1.0
    return w


def forward(u):
    """Physical real fields [..., N, N, N] -> half spectrum [..., N, N, N//2].

    uh(k) = N^-3 sum_x u(x) exp(-i k.x)  (supplementary Eq. dft_def, applied per direction),
    with the kx = N/2 plane dropped.
    """
    N = u.shape[-1]
    uh = _rfftn(u) / float(N) ** 3
    return uh[..., : N // 2]


def inverse(uh):
    """Half spectrum [..., N, N, N//2] -> physical real fields [..., N, N, N].

    u(x) = sum_k uh(k) exp(i k.x) over the full spectrum (Section 3.1, Eq. u_expansion_1d in
    3D), the missing half being the Hermitian mirror and the kx = N/2 plane zero.
    """
    N = uh.shape[-2]
    full = np.zeros(uh.shape[:-1] + (N // 2 + 1,), dtype=complex)
    full[..., : N // 2] = uh
    return _irfftn(full, N) * float(N) ** 3


def kmax2_threshold(kmax):
    """Largest integer m with m < kmax**2, computed in float64.

    The strict test |k|^2 < kmax^2 of Section 3.2 ("|k| >= kmax are zeroed") on integer k^2
    is the same as k^2 <= m.
    """
    q = float(kmax) * float(kmax)
    m = int(np.floor(q))
    if float(m) == q:
        m -= 1
    return m


def kmax_int_threshold(kmax):
    """Largest integer m with m < kmax (cubic truncation: keep |k_i| <= m)."""
    q = float(kmax)
    m = int(np.floor(q))
    if float(m) == q:
        m -= 1
    return m


def double_alias_shifts():
    """The 12 vectors e in {-1, 0, 1}^3 with exactly one zero component: the alias classes
    called double aliases (supplementary material, classification of e)."""
    out = []
    for ez in (-1, 0, 1):
        for ey in (-1, 0, 1):
            for ex in (-1, 0, 1):
                if (ex == 0) + (ey == 0) + (ez == 0) == 1:
                    out.append((ex, ey, ez))
    return out


def double_alias_reach(N, kmax):
    """Modes k that a double alias can reach from the spherically retained modes.

    A product of retained modes kn + km with |kn|^2, |km|^2 <= m (m = kmax2_threshold) lands on
    k = kn + km - N e (2 k_N = N); for a double-alias class e this needs
    |k + N e| <= |kn| + |km| <= 2 sqrt(m), i.e. |k + N e|^2 <= 4 m.  The set returned is every k
    meeting that bound for some double-alias e: it contains every mode a double alias reaches
    (reading of the paper: the removed region is this bound, not the exact lattice set).
    """
    KX, KY, KZ = wavenumbers(N)
    m4 = 4 * kmax2_threshold(kmax)
    reach = np.zeros(KX.shape, dtype=bool)
    for ex, ey, ez in double_alias_shifts():
        d2 = (KX + N * ex) ** 2 + (KY + N * ey) ** 2 + (KZ + N * ez) ** 2
        reach |= d2 <= m4
    return reach


def truncation_mask(N, kmax, kind=TRUNC_SPHERICAL):
    """Boolean mask of retained modes (Section 3.2, Fig. truncation:common).

    spherical: keep |k| < kmax; cubic: keep max_i |k_i| < kmax; no double aliases: the
    spherical mask without double_alias_reach (which is empty when 3 sqrt(m) < sqrt(2) N,
    the discrete form of kmax <= (2 sqrt 2 / 3) k_N).
    Every admissible kmax (<= N/2) zeroes the Nyquist rows ky = -N/2, kz = -N/2.
    """
    KX, KY, KZ = wavenumbers(N)
    if kind not in (TRUNC_SPHERICAL, TRUNC_CUBIC, TRUNC_NO_DOUBLE_ALIAS):
        raise ValueError("unknown truncation kind")
    if kind == TRUNC_CUBIC:
        m = kmax_int_threshold(kmax)
        keep = (np.abs(KX) <= m) & (np.abs(KY) <= m) & (np.abs(KZ) <= m)
    else:
        K2 = KX * KX + KY * KY + KZ * KZ
        keep = K2 <= kmax2_threshold(kmax)
        if kind == TRUNC_NO_DOUBLE_ALIAS:
            keep &= ~double_alias_reach(N, kmax)
    return keep


def project(vh, N=None):
    """Leray projection P(k) = I - k k / |k|^2 applied to a 3-component half spectrum.

    The k = 0 mode, where P is undefined, is set to zero.
    """
    N = vh.shape[-2] if N is None else N
    KX, KY, KZ = wavenumbers(N)
    K2 = KX * KX + KY * KY + KZ * KZ
    K2s = np.where(K2 == 0, 1.0, K2)
    kdotv = KX * vh[0] + KY * vh[1] + KZ * vh[2]
    out = np.empty_like(vh)
    out[0] = vh[0] - KX * kdotv / K2s
    out[1] = vh[1] - KY * kdotv / K2s
    out[2] = vh[2] - KZ * kdotv / K2s
    out[:, 0, 0, 0] = 0.0
    return out


def shift_factor(N, delta):
    """exp(i k.Delta) on the half spectrum (Section 4.2, Eq. shift_operator_3d)."""
    KX, KY, KZ = wavenumbers(N)
    d = np.asarray(delta, dtype=float)
    return np.exp(1j * (KX * d[0] + KY * d[1] + KZ * d[2]))


def curl(uh):
    """Spectral curl i k x uh of a 3-component half spectrum."""
    N = uh.shape[-2]
    KX, KY, KZ = wavenumbers(N)
    w = np.empty_like(uh)
    w[0] = 1j * (KY * uh[2] - KZ * uh[1])
    w[1] = 1j * (KZ * uh[0] - KX * uh[2])
    w[2] = 1j * (KX * uh[1] - KY * uh[0])
    return w


def divergence_ratio(uh):
    """max |k.uh| / max(|k| |uh|): 0 for a solenoidal field."""
    N = uh.shape[-2]
    KX, KY, KZ = wavenumbers(N)
    kd = np.abs(KX * uh[0] + KY * uh[1] + KZ * uh[2])
    kk = np.sqrt(KX * KX + KY * KY + KZ * KZ) * np.sqrt(np.sum(np.abs(uh) ** 2, axis=0))
    den = kk.max()
    return 0.0 if den == 0 else kd.max() / den


def integrating_factor(N, nu, tau):
    """E_tau(k) = exp(sigma tau) with sigma = -nu |k|^2 (Section 4.1, Eq. base-eq)."""
    KX, KY, KZ = wavenumbers(N)
    return np.exp(-nu * (KX * KX + KY * KY + KZ * KZ) * tau)


def set_velocity(u, kmax, kind=TRUNC_SPHERICAL):
    """Physical velocity -> truncated, projected spectral state (the state S of Eq. base-eq)."""
    N = u.shape[-1]
    uh = forward(u)
    uh = uh * truncation_mask(N, kmax, kind)
    return project(uh)

"""Large-scale, time-correlated random forcing at a constant injection rate.

TEST INFRASTRUCTURE ONLY (see :mod:`oracle`).

PARITY UNPINNED against the paper: the paper only says that a random, time-correlated
forcing injects energy at large scales at a constant rate equal to one (Section 2) and
that the forcing depends on the instantaneous flow state (Section 6.2).  Its mechanics
are not given.  The reading implemented here (and, independently, by the CUDA library):

* forced modes: integer k of the stored half spectrum with kf_min^2 <= |k|^2 <= kf_max^2;
* random pattern g_j(k) for redraw j: a complex normal (:func:`oracle.rng.normal_complex`)
  per canonical mode and component, canonical = kx > 0, or kx = 0 and (kz > 0, or kz = 0
  and ky > 0); the kx = 0 modes outside the canonical half are the complex conjugates of
  their mirrors so the forcing is a real field.  Counter of (j, m, c) is (j*M + m)*3 + c,
  m the index of the canonical mode in the loop order kz = -K..K, ky = -K..K, kx = 0..K
  (K = floor(kf_max)), M the number of canonical modes;
* pattern f_j = P(k) g_j (Leray projection), redrawn every t_corr and linearly
  interpolated in time: f(t) = (1 - th) f_j + th f_{j+1}, j = floor(t / t_corr),
  th = t / t_corr - j;
* amplitude: O = a f with a the root of smaller modulus of
      a^2 (dt/2) <f, f> + a Re<S, f> - eps = 0,
  <.,.> the full-spectrum inner product, i.e. an Euler step dt of the forcing alone
  injects exactly eps*dt of kinetic energy, whatever the state S (the invariant that
  pins this module).
"""
import math

import numpy as np

from . import rng
from . import spectral as sp


def shell_modes(N, kf_min, kf_max):
    """Canonical forced modes as a list of (kx, ky, kz) in counter order."""
    K = int(math.floor(kf_max))
    out = []
    for kz in range(-K, K + 1):
        for ky in range(-K, K + 1):
            for kx in range(0, K + 1):
                k2 = kx * kx + ky * ky + kz * kz
                if not (kf_min * kf_min <= k2 <= kf_max * kf_max):
                    continue
                canonical = kx > 0 or (kz > 0 or (kz == 0 and ky > 0))
                if kx < N // 2 and canonical:
                    out.append((kx, ky, kz))
    return out


def pattern(N, kf_min, kf_max, seed, j):
    """Projected random pattern f_j on the half spectrum [3, N, N, N/2]."""
    modes = shell_modes(N, kf_min, kf_max)
    M = len(modes)
    g = np.zeros((3, N, N, N // 2), dtype=complex)
    for m, (kx, ky, kz) in enumerate(modes):
        for c in range(3):
            v = rng.normal_complex(seed, (j * M + m) * 3 + c)
            g[c, kz % N, ky % N, kx] = v
            if kx == 0:
                g[c, (-kz) % N, (-ky) % N, 0] = np.conj(v)
    return sp.project(g)


class Forcing:
    """Constant-rate forcing O(S, t) (reading documented in the module doc)."""

    def __init__(self, N, kf_min, kf_max, eps, t_corr, seed):
        self.N, self.kf_min, self.kf_max = N, kf_min, kf_max
        self.eps, self.t_corr, self.seed = eps, t_corr, seed
        self._cache = {}
        self.w = sp.hermitian_weights(N)

    def _pat(self, j):
        if j not in self._cache:
            self._cache[j] = pattern(self.N, self.kf_min, self.kf_max, self.seed, j)
        return self._cache[j]

    def pattern_at(self, t):
        x = t / self.t_corr
        j = int(math.floor(x))
        th = x - j
        return (1.0 - th) * self._pat(j) + th * self._pat(j + 1)

    def amplitude(self, S, f, dt):
        """Root of smaller modulus of a^2 (dt/2)<f,f> + a Re<S,f> - eps = 0."""
        b = float(np.sum(self.w * np.real(np.conj(S) * f)))
        c = 0.5 * dt * float(np.sum(self.w * np.abs(f) ** 2))
        s = math.sqrt(b * b + 4.0 * c * self.eps)
        return 2.0 * self.eps / (b + s) if b >= 0.0 else 2.0 * self.eps / (b - s)

    def term(self, S, t, dt):
        """Forcing term O(S) at time t for a step of size dt."""
        f = self.pattern_at(t)
        return self.amplitude(S, f, dt) * f

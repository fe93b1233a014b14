"""Counter-based random numbers of the oracle: splitmix64 and the random phase shifts.

TEST INFRASTRUCTURE ONLY (see :mod:`oracle`).

The paper draws the components of the shift delta_alpha "at each time step from [0, dx]
at uniform probability" (Section 4.2, paragraph after the second-stage formula of "RK2
phase-shift random") without naming a generator.  Reading used here and, independently,
by the CUDA library's host code:

* generator: splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014; the 64-bit finaliser as published by S. Vigna).  The n-th
  output (n = 0, 1, ...) of the generator seeded with s is mix(s + (n + 1) * gamma),
  gamma = 0x9E3779B97F4A7C15, which makes it counter based;
* uniform double in [0, 1): the top 53 bits times 2^-53;
* delta_alpha(step)_i = dx * U(seed, 3 * step + i), i = 0, 1, 2 (x, y, z), dx = 2*pi/N;
* delta_beta = delta_alpha + (dx/2)(1, 1, 1), so |delta_alpha_i - delta_beta_i| = dx/2.
"""
import math

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def splitmix64(seed, n):
    """n-th output of splitmix64 seeded with ``seed`` (both unsigned 64-bit integers)."""
    z = (int(seed) + (int(n) + 1) * GAMMA) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def uniform01(seed, n):
    """Uniform double in [0, 1) from the n-th splitmix64 output (top 53 bits)."""
    return (splitmix64(seed, n) >> 11) * (1.0 / 9007199254740992.0)


def shift_alpha(seed, step, N):
    """delta_alpha of time step ``step`` for grid size N (reading stated in the module doc)."""
    dx = 2.0 * math.pi / N
    return [dx * uniform01(seed, 3 * step + i) for i in range(3)]


def shift_beta(delta_alpha, N):
    """delta_beta = delta_alpha + dx/2 in each direction (Section 4.2: |da_i - db_i| = dx/2)."""
    dx = 2.0 * math.pi / N
    return [d + 0.5 * dx for d in delta_alpha]


def normal_complex(seed, n):
    """Complex normal r exp(i theta) from outputs 2n and 2n+1 (Box-Muller, 1958); E|g|^2 = 2."""
    u1 = uniform01(seed, 2 * n)
    u2 = uniform01(seed, 2 * n + 1)
    r = math.sqrt(-2.0 * math.log(1.0 - u1))
    th = 2.0 * math.pi * u2
    return complex(r * math.cos(th), r * math.sin(th))

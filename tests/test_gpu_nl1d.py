"""GPU parity of the 1D quadratic model (ns_nl1d, Sec. 3.3) with the oracle: the paper's
aliased and 2/3-truncated examples, a batch of random positive and sign-changing fields,
grids that are not 2^a 3^b, the largest size, and the argument checks."""
import numpy as np
import pytest

from oracle import nl1d as o1

pytestmark = pytest.mark.gpu


def _fields(N, nb, seed):
    rng = np.random.default_rng(seed)
    x = 2 * np.pi * np.arange(N) / N
    out = [o1.initial(N)]
    for i in range(nb - 1):
        k = rng.integers(1, max(2, N // 4), size=3)
        a = rng.standard_normal(3) * 0.3
        base = 1.0 if i % 2 == 0 else 0.0  # positive fields, then fields that change sign
        out.append(base + sum(a[j] * np.cos(k[j] * x + j) for j in range(3)))
    return np.array(out)


@pytest.mark.parametrize("N,kmax,steps", [(22, 11.0, 1), (32, 32 / 3, 1), (22, 11.0, 25),
                                          (30, 10.0, 7), (64, 32.0, 40), (2048, 1024.0, 2)])
def test_matches_oracle(ns, N, kmax, steps):
    s0 = _fields(N, 5, seed=N)
    dt = 0.05
    got = ns.nl1d(s0, kmax, dt, steps)
    for b in range(len(s0)):
        ref = o1.run(s0[b], dt, steps, kmax)
        assert np.max(np.abs(got[b] - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_paper_aliases_on_the_gpu(ns):
    S22 = ns.nl1d(o1.initial(22), 11.0, 0.1, 1)
    S32 = ns.nl1d(o1.initial(32), 32 / 3, 0.1, 1)
    assert abs(S22[2]) > 1e-3 and abs(S22[8]) > 1e-4          # aliases of 20 and 30
    assert set(np.nonzero(np.abs(S32) > 1e-14)[0]) == {0, 10}  # the 2/3 rule removes them
    # no steps: the truncated initial spectrum, 1 and 0.7 / 2
    S0 = ns.nl1d(o1.initial(22), 11.0, 0.1, 0)
    assert abs(S0[0] - 1.0) < 1e-15 and abs(S0[10] - 0.35) < 1e-15


def test_arguments(ns):
    s = np.ones(16)
    for N, kmax, dt, n in [(16, 0.0, 0.1, 1), (16, 9.0, 0.1, 1), (16, 4.0, 0.0, 1), (16, 4.0, 0.1, -1)]:
        with pytest.raises(ns.NSError) as e:
            ns.nl1d(np.ones(N), kmax, dt, n)
        assert e.value.code == 1
    for bad in (np.ones(15), np.ones(2), np.ones(4096)):
        with pytest.raises(ns.NSError) as e:
            ns.nl1d(bad, 1.0, 0.1, 1)
        assert e.value.code == 1
    assert ns.nl1d(s, 4.0, 0.1, 3).shape == (9,)

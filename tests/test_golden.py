"""The oracle against values the paper prints for its worked examples (tests/golden/*.txt,
each file citing the passage it transcribes)."""
import os

import numpy as np

from oracle import nl1d

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = (t.strip() for t in line.split("=", 1))
                vals[k] = float(v)
    return vals


def test_nl1d_worked_example_sec3_3():
    g = load("nl1d_aliases_sec3_3.txt")
    k0, amp = int(g["k0"]), g["amplitude"]
    assert g["k_nl1"] == 2 * k0 and g["k_nl2"] == 3 * k0
    dt = 0.1
    # N = 22, C_t = 1: after one RK2 step the two largest modes besides k = 0 and k0 are the
    # printed aliases of k_nl1 and k_nl2 (the products of aliases with one another, O(dt^2)
    # smaller, reach further modes such as 2 + 2 = 4)
    N = int(g["N_aliased"])
    assert g["kN_aliased"] == N // 2
    S1 = nl1d.run(nl1d.initial(N, k0, amp), dt, 1, N / 2)
    other = [k for k in np.argsort(-np.abs(S1)) if k not in (0, k0)]
    assert sorted(other[:2]) == sorted([int(g["alias_1"]), int(g["alias_2"])])
    assert abs(S1[other[2]]) < 0.05 * abs(S1[int(g["alias_2"])])
    for knl, ka in ((g["k_nl1"], g["alias_1"]), (g["k_nl2"], g["alias_2"])):
        assert abs(knl - 2 * g["kN_aliased"]) == ka
    # N = 32, C_t = 2/3: the largest kept wavenumber is 10 and the alias of k_nl1 (12) is cut
    N = int(g["N_dealiased"])
    assert g["kN_dealiased"] == N // 2
    kmax = g["Ct_dealiased_num"] / g["Ct_dealiased_den"] * (N // 2)
    kept = np.nonzero(np.abs(nl1d.truncate(np.ones(N // 2 + 1, complex), kmax)) > 0)[0]
    assert kept.max() == g["kmax_kept_dealiased"]
    assert 2 * g["kN_dealiased"] - g["k_nl1"] == g["alias_1_dealiased"] > g["kmax_kept_dealiased"]
    S1 = nl1d.run(nl1d.initial(N, k0, amp), dt, 1, kmax)
    assert abs(S1[int(g["alias_1_dealiased"])]) == 0.0
    assert set(np.nonzero(np.abs(S1) > 1e-14)[0].tolist()) == {0, k0}

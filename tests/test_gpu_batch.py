"""Batched ensembles: one persistent launch advances members of uneven N.

Parity against the FP64 oracle (each member with its own seed), agreement with single
contexts running the same kernels, and the bounded-wait failure path (a wait that can never
be satisfied must end the launch with NS_ERR_TIMEOUT, leaving the GPU usable)."""
import numpy as np
import pytest

from oracle import schemes as sc
from oracle import spectral as osp
from paper_2603_08892_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def members(Ns, seed0=30):
    return [inputs.random_solenoidal(N, seed0 + i, kcut=N / 2, energy_total=1.0) for i, N in enumerate(Ns)]


@pytest.mark.parametrize("scheme,oscheme", [(4, sc.SCHEME_PS_RANDOM), (3, sc.SCHEME_PS_APPROX)])
def test_batch_fp64_matches_oracle(ns, scheme, oscheme):
    Ns = [16, 32, 16, 48, 32]
    nus = [0.01, 0.005, 0.02, 0.01, 0.003]
    seeds = [3, 4, 5, 6, 7]
    dts = [0.01, 0.008, 0.012, 0.01, 0.005]
    us = members(Ns)
    with ns.Batch(Ns, nus, [N / 2 for N in Ns], seeds=seeds, scheme=scheme, precision=ns.FP64) as b:
        for i, u in enumerate(us):
            b.set_velocity(i, u)
        b.step(dts, 3)
        b.step(dts, 2)  # two launches: the sequence must not depend on call boundaries
        got = [b.get_state(i) for i in range(len(Ns))]
        E, eps = b.energy()
    for i, N in enumerate(Ns):
        prob = sc.Problem(N, nus[i], N / 2)
        ref, _ = sc.run(osp.set_velocity(us[i], N / 2), dts[i], 5, prob, oscheme, seed=seeds[i])
        assert rel(got[i], ref) < 1e-12, i
    assert np.all(np.isfinite(E)) and np.all(E > 0)


def test_batch_fp32_equals_single_contexts(ns):
    Ns = [32, 64, 96, 128, 32]
    nus = [1 / 1600] * len(Ns)
    dts = [0.5 * 2 * np.pi / N / 2 for N in Ns]
    us = [inputs.taylor_green_perturbed(N, i) for i, N in enumerate(Ns)]
    with ns.Batch(Ns, nus, [N / 2 for N in Ns], seeds=list(range(len(Ns))), precision=ns.FP32) as b:
        for i, u in enumerate(us):
            b.set_velocity(i, u)
        b.step(dts, 4)
        got = [b.get_state(i) for i in range(len(Ns))]
    for i, N in enumerate(Ns):
        with ns.Solver(N, nus[i], N / 2, scheme=ns.RK2_PS_RANDOM, precision=ns.FP32, seed=i) as s:
            s.set_velocity(us[i])
            s.step(dts[i], 4)
            ref = s.get_state()
        assert rel(got[i], ref) < 1e-6, i
    # and the FP32 members stay within the per-step tolerance of the FP64 oracle
    prob = sc.Problem(32, nus[0], 16.0)
    ref, _ = sc.run(osp.set_velocity(us[0], 16.0), dts[0], 4, prob, sc.SCHEME_PS_RANDOM, seed=0)
    assert rel(got[0], ref) < 4 * 2e-5


def test_batch_bounded_wait_times_out_and_recovers(ns):
    Ns = [16, 32, 16]
    us = members(Ns)
    with ns.Batch(Ns, [0.01] * 3, [N / 2 for N in Ns]) as b:
        for i, u in enumerate(us):
            b.set_velocity(i, u)
        b.set_spin_limit(2000)
        b.test_stall(True)  # every per-step wait now needs a count nothing will reach
        with pytest.raises(ns.NSError) as e:
            b.step([0.01] * 3, 2)
        assert e.value.code == 7  # NS_ERR_TIMEOUT
        b.test_stall(False)
        b.set_spin_limit(2000000)
        for i, u in enumerate(us):
            b.set_velocity(i, u)
        b.step([0.01] * 3, 2)
        E, _ = b.energy()
        assert np.all(np.isfinite(E))


def test_batch_rejects_unsupported_sizes(ns):
    with pytest.raises(ns.NSError) as e:
        ns.Batch([16, 24], [0.01, 0.01], [8.0, 12.0])
    assert e.value.code == 2
    with pytest.raises(ns.NSError) as e:
        ns.Batch([16], [0.01], [8.0], scheme=ns.RK4)
    assert e.value.code == 1


def test_batch_graph_reuse_matches_oracle(ns):
    # two calls with the same nsteps: the second replays the captured CUDA graph; every
    # member must still follow its oracle trajectory (FP64)
    Ns = [16, 32, 16]
    nus = [0.01, 0.005, 0.02]
    seeds = [11, 12, 13]
    dts = [0.01, 0.008, 0.012]
    us = members(Ns, seed0=60)
    with ns.Batch(Ns, nus, [N / 2 for N in Ns], seeds=seeds, precision=ns.FP64) as b:
        for i, u in enumerate(us):
            b.set_velocity(i, u)
        b.step(dts, 3)
        b.step(dts, 3)  # same nsteps: graph replay
        b.step(dts, 3)
        got = [b.get_state(i) for i in range(len(Ns))]
    for i, N in enumerate(Ns):
        prob = sc.Problem(N, nus[i], N / 2)
        ref, _ = sc.run(osp.set_velocity(us[i], N / 2), dts[i], 9, prob, sc.SCHEME_PS_RANDOM,
                        seed=seeds[i])
        assert rel(got[i], ref) < 1e-12, i


def test_batch_fp32_members_match_oracle(ns, report):
    # FP32 members of every size of the ensemble workload against the FP64 oracle
    Ns = [32, 64, 96, 128]
    nus = [1 / 1600] * len(Ns)
    dts = [0.5 * 2 * np.pi / N / 2 for N in Ns]
    us = [inputs.taylor_green_perturbed(N, 40 + i) for i, N in enumerate(Ns)]
    with ns.Batch(Ns, nus, [N / 2 for N in Ns], seeds=[20 + i for i in range(len(Ns))],
                  precision=ns.FP32) as b:
        for i, u in enumerate(us):
            b.set_velocity(i, u)
        b.step(dts, 2)
        b.step(dts, 2)  # graph replay
        got = [b.get_state(i) for i in range(len(Ns))]
    for i, N in enumerate(Ns):
        prob = sc.Problem(N, nus[i], N / 2)
        ref, _ = sc.run(osp.set_velocity(us[i], N / 2), dts[i], 4, prob, sc.SCHEME_PS_RANDOM,
                        seed=20 + i)
        err = rel(got[i], ref)
        report("batch_member_N%d_4_steps_fp32" % N, err, 4 * 2e-5)
        assert err < 4 * 2e-5, i  # four FP32 steps


@pytest.mark.parametrize("sched", [(1, 0), (4, 0), (8, 1), (0, 0)])
def test_batch_schedules_give_identical_results(ns, sched):
    # the work-list granularity and CTAs per SM change the order of the work, not the result;
    # the grid schedule (0, 0) runs the same tile bodies as ordinary launches per pass
    Ns = [32, 64, 16]
    us = members(Ns, seed0=70)
    out = []
    for s in ((1, 0), sched):
        with ns.Batch(Ns, [0.01] * 3, [N / 2 for N in Ns], seeds=[1, 2, 3], precision=ns.FP32) as b:
            b.set_schedule(*s)
            for i, u in enumerate(us):
                b.set_velocity(i, u)
            b.step([0.01] * 3, 3)
            out.append([b.get_state(i) for i in range(3)])
    for a, c in zip(*out):
        assert np.array_equal(a, c)


def test_batch_tuner_leaves_the_states_unchanged(ns):
    # the first step tunes the schedule on the ensemble and restores the states it touched
    Ns = [32, 64]
    us = members(Ns, seed0=80)
    ref = []
    with ns.Batch(Ns, [0.01] * 2, [N / 2 for N in Ns], seeds=[5, 6], precision=ns.FP64) as b:
        b.set_schedule(1, 0)
        for i, u in enumerate(us):
            b.set_velocity(i, u)
        b.step([0.01] * 2, 2)
        ref = [b.get_state(i) for i in range(2)]
    with ns.Batch(Ns, [0.01] * 2, [N / 2 for N in Ns], seeds=[5, 6], precision=ns.FP64) as b:
        for i, u in enumerate(us):
            b.set_velocity(i, u)
        b.step([0.01] * 2, 2)  # tunes first
        got = [b.get_state(i) for i in range(2)]
        g, q = b.schedule()
        assert g in (0, 1, 2, 4, 8) and q in (0, 1)
    for a, c in zip(ref, got):
        assert np.array_equal(a, c)

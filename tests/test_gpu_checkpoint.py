"""Checkpoint files (ns_checkpoint_save / ns_checkpoint_load): a run resumed from a file gives
the same bits as the uninterrupted run, for the random scheme with forcing (shifts drawn from
the seed and step count, forcing patterns from the seed and time) and in FP32 and FP64."""
import numpy as np
import pytest

from paper_2603_08892_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("forced", [False, True])
def test_resume_from_file_is_bitwise(ns, tmp_path, prec, forced):
    N, nu, dt = 32, 0.005, 0.01
    u = inputs.random_solenoidal(N, 8, kcut=8, energy_total=1.0)
    path = str(tmp_path / "run.ckpt")

    def make():
        s = ns.Solver(N, nu, N / 2, scheme=ns.RK2_PS_RANDOM, precision=prec, seed=77)
        if forced:
            s.set_forcing(2.0, 3.0, 0.1, 0.5, seed=5)
        return s

    with make() as a:
        a.set_velocity(u)
        a.step(dt, 7)
        a.checkpoint_save(path)
        a.step(dt, 9)
        ref = a.get_state()
        tref = a.time()
    with ns.Solver(N, nu, N / 2, scheme=ns.RK2_PS_RANDOM, precision=prec, seed=1) as b:
        b.checkpoint_load(path)  # restores the seed 77, the time, the step count and forcing
        assert b.time()[1] == 7
        b.step(dt, 9)
        got = b.get_state()
        assert b.time() == tref
    assert np.array_equal(got, ref)


def test_checkpoint_errors(ns, tmp_path):
    path = str(tmp_path / "x.ckpt")
    with ns.Solver(16, 0.01, 8.0) as s:
        with pytest.raises(ns.NSError) as e:
            s.checkpoint_save(path)  # no state yet
        assert e.value.code == 8
        s.set_velocity(inputs.taylor_green(16))
        s.checkpoint_save(path)
    with ns.Solver(16, 0.02, 8.0) as s:  # another viscosity
        with pytest.raises(ns.NSError) as e:
            s.checkpoint_load(path)
        assert e.value.code == 1
    with open(path, "r+b") as f:  # truncated file
        f.truncate(100)
    with ns.Solver(16, 0.01, 8.0) as s:
        with pytest.raises(ns.NSError) as e:
            s.checkpoint_load(path)
        assert e.value.code == 10
        with pytest.raises(ns.NSError) as e:
            s.checkpoint_load(str(tmp_path / "missing.ckpt"))
        assert e.value.code == 10

"""The single-field decomposition's GPU side: a nonlinear evaluation split over two ranks (two
processes on one GPU, gloo exchanging host copies between the rank-range passes), against the
FP64 oracle and one context's whole-field evaluation.  The ranks' kernels never wait on one
another: every exchange happens on the host between launches."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for p in (HERE, ROOT):
    if p not in sys.path:
        sys.path.insert(0, p)

import _dist_worker  # noqa: E402

pytestmark = pytest.mark.gpu


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("prec", [1, 0])
def test_decomposed_nonlinear_two_ranks_on_gpu(ns, prec):
    mp.spawn(_dist_worker.decomposed_nonlinear_gpu, args=(2, free_port(), prec), nprocs=2, join=True)


def test_rank_calls_reject_bad_ranges(ns):
    with ns.Solver(16, 0.0, 8.0) as s:
        with pytest.raises(ns.NSError) as e:
            s.rank_slab(4, 4)
        assert e.value.code == 1
        with pytest.raises(ns.NSError) as e:
            s.rank_pencil(ns.RANK_INIT, [0.0, 0.0, 0.0], 0, 17)
        assert e.value.code == 1
        with pytest.raises(ns.NSError) as e:
            s.rank_get(ns.BUF_STATE, 2, 0, 4)
        assert e.value.code == 1

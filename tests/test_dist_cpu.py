"""CPU multi-process tests (gloo, world size 2) of the multi-rank code paths: the single-field
decomposition's all-to-all exchanges and a whole decomposed nonlinear evaluation against the
single-process oracle, and the bench's replica timing helpers."""
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


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("fn", [_dist_worker.exchange_roundtrip, _dist_worker.decomposed_nonlinear,
                                _dist_worker.replica_timing])
def test_two_cpu_ranks(fn):
    mp.spawn(fn, args=(2, free_port()), nprocs=2, join=True)

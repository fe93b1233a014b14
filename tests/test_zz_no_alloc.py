"""The allocation-free nonlinear-term entry point against the context-based one.

ns_nonlinear_noalloc exists for callers that cannot allocate device memory (their device
memory is held by their own allocator, or their loop must not allocate once running).  It
works in one fixed array inside the library, so this test checks that two calls in a row
reuse it correctly: each must match ns_nonlinear on the same FP32 state.  The file is named
to be collected last.
"""
import math

import numpy as np
import pytest

from paper_2603_08892_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("N,trunc", [(32, 0), (48, 1), (64, 0)])
def test_noalloc_matches_context_entry_point_twice(ns, N, trunc):
    import torch

    kmax = N / 2 if trunc == 0 else 0.9 * N / 2
    u = inputs.random_solenoidal(N, 40 + N, kcut=N / 2, energy_total=1.0)
    dx = 2 * math.pi / N
    deltas = [[0.3 * dx, 0.7 * dx, 0.1 * dx], [0.5 * dx] * 3]
    with ns.Solver(N, 0.0, kmax, truncation=trunc, precision=ns.FP32) as s:
        s.set_velocity(u)
        S = s.get_state()  # FP32 values widened to complex128
        refs = [s.nonlinear(d, S) for d in deltas]
    state = torch.from_numpy(S.astype(np.complex64)).cuda()
    out = torch.empty_like(state)
    stream = torch.cuda.current_stream()
    for d, ref in zip(deltas, refs):
        out.fill_(complex(float("nan"), float("nan")))  # every element must be written
        ns.nonlinear_noalloc(state.data_ptr(), out.data_ptr(), N, kmax, d, truncation=trunc,
                             stream=stream.cuda_stream)
        got = out.cpu().numpy().astype(np.complex128)
        assert np.isfinite(got).all()
        assert rel(got, ref) < 1e-5


def test_noalloc_rejects_sizes_beyond_its_array(ns):
    with pytest.raises(ns.NSError) as e:
        ns.nonlinear_noalloc(1, 1, 96, 48.0, [0.0, 0.0, 0.0])
    assert e.value.code == 2
    with pytest.raises(ns.NSError) as e:
        ns.nonlinear_noalloc(1, 1, 32, 17.0, [0.0, 0.0, 0.0])
    assert e.value.code == 3

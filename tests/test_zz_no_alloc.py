"""The allocation-free nonlinear-term entry point against the context-based one.

ns_nonlinear_noalloc exists for callers that cannot allocate device memory (their device
memory is held by their own allocator, or their loop must not allocate once running).  It
works in one fixed array inside the library, so this test checks that two calls in a row
reuse it correctly: each must match ns_nonlinear on the same FP32 state, and the FP64 oracle
within the FP32 tolerance of the nonlinear term.  A second test runs in a fresh process, where
the entry point is the first use of the library, and checks that once that first call has
placed the library on the device, later calls leave the free device memory unchanged.  The
file is named to be collected last.
"""
import math
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from oracle import nonlinear as onl
from oracle import spectral as osp
from paper_2603_08892_gb300 import inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("N,trunc,side_stream", [(32, 0, False), (48, 1, False), (64, 0, False),
                                                 (16, 2, False), (8, 0, False), (32, 0, True)])
def test_noalloc_matches_context_entry_point_twice(ns, N, trunc, side_stream):
    import torch

    kmax = N / 2 if trunc != 1 else 0.9 * N / 2
    u = inputs.random_solenoidal(N, 40 + N, kcut=N / 2, energy_total=1.0)
    dx = 2 * math.pi / N
    deltas = [[0.3 * dx, 0.7 * dx, 0.1 * dx], [0.5 * dx] * 3]
    with ns.Solver(N, 0.0, kmax, truncation=trunc, precision=ns.FP32) as s:
        s.set_velocity(u)
        S = s.get_state()  # FP32 values widened to complex128
        refs = [s.nonlinear(d, S) for d in deltas]
    state = torch.from_numpy(S.astype(np.complex64)).cuda()
    out = torch.empty_like(state)
    stream = torch.cuda.Stream() if side_stream else torch.cuda.current_stream()
    if side_stream:
        stream.wait_stream(torch.cuda.current_stream())  # state and out are ready
    for d, ref in zip(deltas, refs):
        with torch.cuda.stream(stream):
            out.fill_(complex(float("nan"), float("nan")))  # every element must be written
        ns.nonlinear_noalloc(state.data_ptr(), out.data_ptr(), N, kmax, d, truncation=trunc,
                             stream=stream.cuda_stream)
        got = out.cpu().numpy().astype(np.complex128)
        assert np.isfinite(got).all()
        assert rel(got, ref) < 1e-5
        assert rel(got, onl.nonlinear(S, d, kmax, trunc)) < 2e-5


def test_noalloc_first_use_then_no_device_memory(ns):
    # fresh process: the entry point is the library's first use on the device
    code = textwrap.dedent("""
        import math, sys
        import numpy as np, torch
        sys.path.insert(0, %r)
        from paper_2603_08892_gb300 import binding as ns
        N = 32
        rng = np.random.default_rng(1)
        S = (rng.standard_normal((3, N, N, N // 2)) + 1j * rng.standard_normal((3, N, N, N // 2)))
        state = torch.from_numpy(S.astype(np.complex64)).cuda()
        out = torch.empty_like(state)
        d = [0.1, 0.2, 0.3]
        st = torch.cuda.current_stream().cuda_stream
        ns.nonlinear_noalloc(state.data_ptr(), out.data_ptr(), N, N / 2, d, stream=st)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        a = out.clone()
        for _ in range(3):
            ns.nonlinear_noalloc(state.data_ptr(), out.data_ptr(), N, N / 2, d, stream=st)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert torch.equal(a, out)
        # the clone above is torch's (its caching allocator), made before free0 was read
        print("FREE", free0, free1)
        assert free1 == free0, (free0, free1)
    """ % ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr


def test_noalloc_rejects_sizes_beyond_its_array(ns):
    with pytest.raises(ns.NSError) as e:
        ns.nonlinear_noalloc(1, 1, 96, 48.0, [0.0, 0.0, 0.0])
    assert e.value.code == 2
    with pytest.raises(ns.NSError) as e:
        ns.nonlinear_noalloc(1, 1, 32, 17.0, [0.0, 0.0, 0.0])
    assert e.value.code == 3

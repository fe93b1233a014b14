"""Host-side checks (no GPU): the C-ABI library builds, loads, and exports every symbol
that include/ns.h declares; argument validation paths that need no device."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    hdrs = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
            if f.endswith(".h")]
    names = []
    for h in hdrs:
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(ns_[a-z_0-9]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import ctypes

    from paper_2603_08892_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["ns_init", "ns_init_ex", "ns_destroy", "ns_set_velocity", "ns_step",
              "ns_set_forcing", "ns_energy_spectrum", "ns_energy", "ns_nonlinear"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_the_exports(lib):
    from paper_2603_08892_gb300 import binding

    assert set(binding.EXPORTED) <= set(declared_functions())
    assert set(declared_functions()) <= set(binding.EXPORTED)


def test_init_rejects_bad_arguments_before_touching_a_device(lib):
    from paper_2603_08892_gb300 import binding as ns

    cases = [(7, 3.0, ns.ERRORS and 2), (10, 4.0, 2), (6, 2.0, 2), (16, 8.5, 3), (16, 0.0, 3)]
    for N, kmax, code in cases:
        with pytest.raises(ns.NSError) as e:
            ns.Solver(N, 0.01, kmax)
        assert e.value.code == code
    with pytest.raises(ns.NSError) as e:
        ns.Solver(16, 0.01, 8.0, L=1.0)
    assert e.value.code == 1
    with pytest.raises(ns.NSError) as e:
        ns.Solver(16, -1.0, 8.0)
    assert e.value.code == 1
    with pytest.raises(ns.NSError) as e:
        ns.Solver(16, 0.01, 8.0, scheme=9)
    assert e.value.code == 1


def test_fma_peak_argument_checks():
    # rejected before any CUDA call, so this runs without a GPU
    import ctypes

    from paper_2603_08892_gb300 import binding as b

    out = ctypes.c_double()
    assert b._fma_peak(0, 7, ctypes.byref(out)) == 1  # NS_ERR_INVALID_ARG
    assert b._fma_peak(0, b.FP32, None) == 1

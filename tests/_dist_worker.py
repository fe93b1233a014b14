"""Rank bodies of the CPU multi-process tests (spawned with torch.multiprocessing, gloo)."""
import os

import numpy as np
import torch
import torch.distributed as dist


def _init(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def exchange_roundtrip(rank, world, port):
    from paper_2603_08892_gb300 import decomp

    _init(rank, world, port)
    try:
        N, M, F = 12, 6, 5
        rng = np.random.default_rng(7)
        g = rng.standard_normal((F, N, N, M)) + 1j * rng.standard_normal((F, N, N, M))  # same on all
        lo, hi = decomp.blocks(N, world)[rank]
        pen = torch.from_numpy(np.ascontiguousarray(g[:, :, lo:hi, :]))
        slab = decomp.pencil_to_slab(pen)
        assert np.array_equal(slab.numpy(), g[:, lo:hi, :, :])
        back = decomp.slab_to_pencil(slab)
        assert np.array_equal(back.numpy(), g[:, :, lo:hi, :])
    finally:
        dist.destroy_process_group()


def decomposed_nonlinear(rank, world, port):
    """One nonlinear evaluation split over the ranks: pencil pass on the own ky block,
    all-to-all, slab pass on the own z block, all-to-all back, spectral stage; compared with
    the single-process oracle."""
    import math

    from oracle import nonlinear as onl
    from oracle import spectral as osp
    from paper_2603_08892_gb300 import decomp, inputs

    _init(rank, world, port)
    try:
        N, M = 16, 8
        kmax = N / 2
        dx = 2 * math.pi / N
        delta = [0.3 * dx, 0.55 * dx, 0.8 * dx]
        S = osp.set_velocity(inputs.random_solenoidal(N, 3, kcut=N / 2), kmax)
        ref = onl.nonlinear(S, delta, kmax)
        lo, hi = decomp.blocks(N, world)[rank]
        KX, KY, KZ = osp.wavenumbers(N)
        kx, ky, kz = KX[:, lo:hi], KY[:, lo:hi], KZ[:, lo:hi]
        sh = osp.shift_factor(N, delta)
        Ss = (S * sh)[:, :, lo:hi, :]
        w = np.stack([1j * (ky * Ss[2] - kz * Ss[1]), 1j * (kz * Ss[0] - kx * Ss[2]),
                      1j * (kx * Ss[1] - ky * Ss[0])])
        # pencil pass: inverse z transform of u and omega (no 1/N on inverse transforms)
        mixed = np.fft.ifft(np.concatenate([Ss, w]), axis=1) * N
        slab = decomp.pencil_to_slab(torch.from_numpy(np.ascontiguousarray(mixed))).numpy()
        # slab pass: inverse y, inverse real x, u x omega, forward x and y (1/N each)
        a = np.fft.ifft(slab, axis=2) * N
        full = np.zeros(a.shape[:-1] + (M + 1,), dtype=complex)
        full[..., :M] = a
        phys = np.fft.irfft(full, n=N, axis=3) * N
        cr = np.cross(phys[:3], phys[3:], axis=0)
        fy = np.fft.fft(np.fft.rfft(cr, axis=3)[..., :M] / N, axis=2) / N
        back = decomp.slab_to_pencil(torch.from_numpy(np.ascontiguousarray(fy))).numpy()
        # spectral stage (pointwise in k): forward z, de-shift, truncation, projection
        Nl = np.fft.fft(back, axis=1) / N * np.conj(sh[:, lo:hi, :])
        Nl = Nl * osp.truncation_mask(N, kmax)[:, lo:hi, :]
        whole = np.zeros((3, N, N, M), dtype=complex)
        whole[:, :, lo:hi, :] = Nl
        Nl = osp.project(whole)[:, :, lo:hi, :]
        assert np.abs(Nl - ref[:, :, lo:hi, :]).max() < 1e-13 * np.abs(ref).max()
    finally:
        dist.destroy_process_group()


def replica_timing(rank, world, port):
    """The bench's N > 1 helpers: barrier and the max over ranks of the timed interval."""
    import bench

    _init(rank, world, port)
    try:
        bench.barrier(world)
        assert bench.reduce_max(1.5 + rank, world) == 1.5 + (world - 1)
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def decomposed_nonlinear_gpu(rank, world, port, prec):
    """The same decomposed evaluation on the GPU: every rank runs the library's kernels on its
    ranges (pencil pass on its ky rows, slab pass on its z planes) on one shared device, the
    two all-to-all exchanges of the mixed fields and of the transformed products go through
    gloo on host copies.  Compared with the single-process oracle and with one context's
    whole-field evaluation."""
    import math

    import torch

    from oracle import nonlinear as onl
    from oracle import spectral as osp
    from paper_2603_08892_gb300 import binding as ns
    from paper_2603_08892_gb300 import decomp, inputs

    _init(rank, world, port)
    try:
        torch.cuda.set_device(0)
        N = 32
        kmax = N / 2
        dx = 2 * math.pi / N
        delta = [0.3 * dx, 0.55 * dx, 0.8 * dx]
        S = osp.set_velocity(inputs.random_solenoidal(N, 3, kcut=N / 2), kmax)
        lo, hi = decomp.blocks(N, world)[rank]
        with ns.Solver(N, 0.0, kmax, precision=prec) as s:
            s.rank_set(ns.BUF_STATE, 1, lo, hi, S[:, :, lo:hi, :])  # own ky rows only
            s.rank_pencil(ns.RANK_INIT, delta, lo, hi)
            mixed = s.rank_get(ns.BUF_MIXED, 1, lo, hi)
            slab = decomp.pencil_to_slab(torch.from_numpy(mixed)).numpy()
            s.rank_set(ns.BUF_MIXED, 0, lo, hi, slab)
            s.rank_slab(lo, hi)
            ft = s.rank_get(ns.BUF_FT, 0, lo, hi)
            back = decomp.slab_to_pencil(torch.from_numpy(ft)).numpy()
            s.rank_set(ns.BUF_FT, 1, lo, hi, back)
            s.rank_pencil(ns.RANK_NL, delta, lo, hi)
            got = s.rank_get(ns.BUF_NL, 1, lo, hi)
        with ns.Solver(N, 0.0, kmax, precision=prec) as s1:
            whole = s1.nonlinear(delta, S)[:, :, lo:hi, :]
        ref = onl.nonlinear(S, delta, kmax)[:, :, lo:hi, :]
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < (1e-12 if prec == 1 else 2e-5), err
        assert np.linalg.norm(got - whole) <= (1e-14 if prec == 1 else 1e-6) * np.linalg.norm(whole)
    finally:
        dist.destroy_process_group()

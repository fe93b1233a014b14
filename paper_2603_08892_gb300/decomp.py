"""Single-field domain decomposition of the two-pass step over P ranks (one GPU each).

The pencil pass needs complete z columns, the slab pass complete (y, x) planes, so a field
split over P ranks changes owner at every pass boundary (the transposes of a distributed 3D
FFT, as with the slab decompositions of the paper's FFTW-MPI runs, Sec. 2):

* pencil layout: rank r holds the ky index block Y_r = [r N/P, (r+1) N/P) of every column,
  arrays [F][N (z or kz)][N/P (ky)][N/2 (kx)];
* slab layout: rank r holds the z block Z_r = [r N/P, (r+1) N/P), arrays
  [F][N/P (z)][N (y or ky)][N/2 (kx)].

Per nonlinear evaluation the 5 mixed fields go pencil -> slab after the pencil pass and the 3
transformed products slab -> pencil after the slab pass: one all-to-all each, every rank
sending an equal block of F (N/P)^2 N/2 values to every other rank.  The state stays in the
pencil layout.  The functions work on torch tensors of any device through
torch.distributed.all_to_all_single (NCCL between GPUs; gloo on CPU ranks in the tests).
"""
import torch
import torch.distributed as dist


def blocks(N, world):
    """Index range of every rank's block (ky in the pencil layout, z in the slab layout)."""
    if N % world:
        raise ValueError("N must be a multiple of the number of ranks")
    n = N // world
    return [(r * n, (r + 1) * n) for r in range(world)]


def pencil_to_slab(x, group=None):
    """[F][N][N/P][M] (all z, own ky block) -> [F][N/P][N][M] (own z block, all ky)."""
    world = dist.get_world_size(group)
    F, N, nl, M = x.shape
    if nl * world != N:
        raise ValueError("pencil block shape does not match the number of ranks")
    # send block q: this rank's ky block on rank q's z block
    send = x.reshape(F, world, nl, nl, M).permute(1, 0, 2, 3, 4).contiguous()
    recv = torch.empty_like(send)
    dist.all_to_all_single(recv, send, group=group)
    # recv[q]: [F][own z block][ky block of q][M]
    return recv.permute(1, 2, 0, 3, 4).reshape(F, nl, world * nl, M)


def slab_to_pencil(y, group=None):
    """[F][N/P][N][M] (own z block, all ky) -> [F][N][N/P][M] (all z, own ky block)."""
    world = dist.get_world_size(group)
    F, nl, N, M = y.shape
    if nl * world != N:
        raise ValueError("slab block shape does not match the number of ranks")
    # send block q: this rank's z block on rank q's ky block
    send = y.reshape(F, nl, world, nl, M).permute(2, 0, 1, 3, 4).contiguous()
    recv = torch.empty_like(send)
    dist.all_to_all_single(recv, send, group=group)
    # recv[q]: [F][z block of q][own ky block][M]
    return recv.permute(1, 0, 2, 3, 4).reshape(F, world * nl, nl, M)


def exchange_bytes(N, world, fields, itemsize):
    """Bytes one rank sends to the others in one exchange of `fields` fields."""
    nl = N // world
    return fields * nl * nl * (N // 2) * itemsize * (world - 1)

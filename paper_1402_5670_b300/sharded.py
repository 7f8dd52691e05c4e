"""One transform split over ranks by filter ranges (torch.distributed plumbing).

The inverse of eq. reconstruction is a sum over filters j (Algorithm 2): each rank
turns the coefficients of its filter range into one partial spectrum
(sl_inverse_partial), the partials are added by one all-reduce, and every rank
finishes with the division by Psi and the inverse FFT (sl_inverse_finish). The
forward transform (Algorithm 1) needs the signal's spectrum on every rank: rank
`root` computes it (sl_spectrum) and broadcasts it, then each rank produces its own
range (sl_forward_range). These are the two exchange steps of the split; all
arithmetic runs in the library's kernels.

With the NCCL backend the collectives act on the device buffers directly; with gloo
(CPU ranks, tests) they go through host copies.
"""
from __future__ import annotations

from typing import List, Tuple


def filter_ranges(R: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous filter ranges [j0, j1) for `world` ranks, sizes differing by at most
    one (every filter costs the same: one FFT each way)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    base, extra = divmod(R, world)
    out, j = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((j, j + n))
        j += n
    return out


def _collective(t, fn, group):
    import torch.distributed as dist
    if dist.get_backend(group) == "nccl":
        fn(t)
        return t
    h = t.cpu()
    fn(h)
    t.copy_(h)
    return t


def sharded_forward(bank, x, group=None, root: int = 0):
    """This rank's filter range and its coefficients [j1 - j0][dims]. x (a CUDA tensor
    of the bank's shape) is read on rank `root` only."""
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    j0, j1 = filter_ranges(bank.R, world)[rank]
    xhat = bank._empty((2 * bank.spectrum_points,))
    if rank == root:
        bank.spectrum(x, out=xhat)
    _collective(xhat, lambda t: dist.broadcast(t, src=root, group=group), group)
    return (j0, j1), bank.forward_range(xhat, j0, j1)


def sharded_inverse(bank, coeffs, j_range, dual: bool = True, group=None):
    """The dual-frame inverse (dual=True) or the adjoint of the whole coefficient set,
    from this rank's range coeffs [j1 - j0][dims]; every rank gets the result."""
    import torch.distributed as dist
    j0, j1 = j_range
    part = bank.inverse_partial(coeffs, j0, j1)
    _collective(part, lambda t: dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group), group)
    return bank.inverse_finish(part, dual)

"""One transform split by filter ranges over ranks (the multi-GPU form of the path).

The inverse of eq. reconstruction is a sum over filters (Algorithm 2): each rank
forms the partial spectrum of its range, one all-reduce adds them, and the division
by Psi and the inverse FFT finish it. CPU tests run the oracle's split on two gloo
ranks; GPU tests check the library's range calls against the unsharded calls and the
oracle, on one GPU (ranks as separate processes that never wait on each other's
kernels: they meet only in gloo collectives on host copies).
"""
import json
import os
import socket
import sys

import numpy as np
import pytest

from oracle import shearlet_oracle as O
from paper_1402_5670_b300 import synth
from paper_1402_5670_b300.sharded import filter_ranges
from tests.conftest import oracle_system

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("R,world", [(49, 2), (49, 3), (17, 4), (292, 8), (3, 5), (1, 1)])
def test_filter_ranges_cover_all_filters_once(R, world):
    rs = filter_ranges(R, world)
    assert len(rs) == world and rs[0][0] == 0 and rs[-1][1] == R
    for (a0, a1), (b0, _) in zip(rs, rs[1:]):
        assert a1 == b0
    sizes = [j1 - j0 for j0, j1 in rs]
    assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 0


# ------------------------------------------------------- oracle, CPU ranks ---

CASES = [((32, 32), 2, (1, 1)), ((16, 16, 16), 2, (0, 1))]


def _oracle_rank(rank, ws, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    from oracle import shearlet_oracle as Orc
    from paper_1402_5670_b300 import synth as sy
    from paper_1402_5670_b300.sharded import filter_ranges as fr
    res = {}
    for i, (dims, J, sl) in enumerate(CASES):
        s = Orc.build_system(dims, J, sl)
        x = sy.gaussian_field(dims, 40 + i).astype(np.float64)
        C = Orc.forward(x, s)                      # every rank could; each uses its range
        j0, j1 = fr(s.R, ws)[rank]
        acc = Orc.inverse_partial(C, s, range(j0, j1))
        t = torch.from_numpy(np.stack([acc.real, acc.imag]))
        dist.all_reduce(t, op=dist.ReduceOp.SUM)   # the one exchange step of the inverse
        summed = t[0].numpy() + 1j * t[1].numpy()
        y = Orc.inverse_finish(summed, s, dual=True)
        ya = Orc.inverse_finish(summed, s, dual=False)
        res[str(i)] = {"inv": rel(y, Orc.inverse(C, s)), "adj": rel(ya, Orc.adjoint(C, s)),
                       "pr": rel(y, x)}
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)
    dist.destroy_process_group()


def test_oracle_partial_sums_over_two_ranks_equal_unsharded_inverse(tmp_path):
    """Two gloo ranks each sum FFT(C_j) psi_hat_j over their filter range; the
    all-reduced sum, divided by Psi (or not) and transformed back, equals the oracle's
    unsharded inverse (adjoint) to 1e-12 and reconstructs x (eq. reconstruction)."""
    import torch.multiprocessing as mp
    ws = 2
    mp.start_processes(_oracle_rank, args=(ws, _free_port(), str(tmp_path)), nprocs=ws,
                       start_method="spawn", join=True)
    for r in range(ws):
        res = json.load(open(tmp_path / f"rank{r}.json"))
        for case in res.values():
            assert case["inv"] < 1e-12 and case["adj"] < 1e-12 and case["pr"] < 1e-12


def test_pin_catches_a_rank_that_skips_its_last_filter():
    """Planted mistake: ranges that drop one filter at a boundary. The split sum must
    then miss perfect reconstruction."""
    dims, J, sl = (32, 32), 2, (1, 1)
    s = oracle_system(dims, J, sl)
    x = synth.gaussian_field(dims, 41).astype(np.float64)
    C = O.forward(x, s)
    (a0, a1), (b0, b1) = filter_ranges(s.R, 2)
    acc = O.inverse_partial(C, s, range(a0, a1 - 1)) + O.inverse_partial(C, s, range(b0, b1))
    assert rel(O.inverse_finish(acc, s), x) > 1e-3


# ---------------------------------------------------------- library, GPU ---

GPU_CASES = [((256, 256), 4, (1, 1, 2, 2)), ((64, 32), 2, (1, 1)), ((32, 16, 8), 2, (1, 1))]


@pytest.mark.gpu
@pytest.mark.parametrize("case", GPU_CASES, ids=str)
def test_ranges_match_unsharded_calls_and_oracle(case):
    """sl_forward_range over 3 ranges concatenates to sl_forward bit for bit; the sum of
    the 3 sl_inverse_partial spectra, finished by sl_inverse_finish, matches sl_inverse
    / sl_adjoint and the oracle to 1e-5; an empty range gives a zero partial."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_5670_b300.build import build
    from paper_1402_5670_b300.shearlet import Bank
    build()
    dims, J, sl = case
    b = Bank(dims, J, sl, device=0)
    s = oracle_system(dims, J, sl)
    x = synth.add_noise(synth.piecewise_smooth_image(dims, 3) if len(dims) == 2
                        else synth.moving_ellipses_volume(dims, 3), 20.0, 4)
    xg = torch.from_numpy(x).cuda()
    C = b.forward(xg)
    xhat = b.spectrum(xg)
    parts = []
    pieces = []
    for j0, j1 in filter_ranges(b.R, 3):
        Cr = b.forward_range(xhat, j0, j1)
        pieces.append(Cr)
        parts.append(b.inverse_partial(Cr, j0, j1))
    assert torch.equal(torch.cat(pieces), C)
    summed = parts[0] + parts[1] + parts[2]
    y = b.inverse_finish(summed, dual=True)
    ya = b.inverse_finish(summed, dual=False)
    Cn = C.cpu().numpy().astype(np.float64)
    assert rel(y.cpu().numpy(), b.inverse(C).cpu().numpy()) < 1e-5
    assert rel(ya.cpu().numpy(), b.adjoint(C).cpu().numpy()) < 1e-5
    assert rel(y.cpu().numpy(), O.inverse(Cn, s)) < 1e-5
    assert rel(ya.cpu().numpy(), O.adjoint(Cn, s)) < 1e-5
    z = b.inverse_partial(C[:0], 5, 5)
    assert float(z.abs().max()) == 0.0
    torch.cuda.synchronize()


def _gpu_rank(rank, ws, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    from paper_1402_5670_b300 import synth as sy
    from paper_1402_5670_b300.sharded import sharded_forward, sharded_inverse
    from paper_1402_5670_b300.shearlet import Bank
    torch.cuda.set_device(0)
    dims, J, sl = (256, 256), 4, (1, 1, 2, 2)
    b = Bank(dims, J, sl, device=0)
    x = torch.from_numpy(sy.add_noise(sy.piecewise_smooth_image(dims, 5), 20.0, 6)).cuda()
    (j0, j1), Cr = sharded_forward(b, x)
    y = sharded_inverse(b, Cr, (j0, j1), dual=True)
    ya = sharded_inverse(b, Cr, (j0, j1), dual=False)
    torch.cuda.synchronize()
    np.save(os.path.join(out_dir, f"C{rank}.npy"), Cr.cpu().numpy())
    np.save(os.path.join(out_dir, f"y{rank}.npy"), y.cpu().numpy())
    np.save(os.path.join(out_dir, f"ya{rank}.npy"), ya.cpu().numpy())
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump([j0, j1], f)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.gpu
def test_two_ranks_gloo_match_unsharded(tmp_path):
    """Two processes (ranks) on the one GPU: rank 0's spectrum is broadcast, each
    rank computes its filter range, the partial spectra are all-reduced (gloo, host
    copies) and finished. Coefficients concatenate to sl_forward's bit for bit; both
    ranks' inverse and adjoint match sl_inverse / sl_adjoint to 1e-5."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.multiprocessing as mp
    from paper_1402_5670_b300.build import build
    from paper_1402_5670_b300.shearlet import Bank
    build()
    ws = 2
    mp.start_processes(_gpu_rank, args=(ws, _free_port(), str(tmp_path)), nprocs=ws,
                       start_method="spawn", join=True)
    dims, J, sl = (256, 256), 4, (1, 1, 2, 2)
    b = Bank(dims, J, sl, device=0)
    x = torch.from_numpy(synth.add_noise(synth.piecewise_smooth_image(dims, 5), 20.0, 6)).cuda()
    C = b.forward(x)
    yi = b.inverse(C).cpu().numpy()
    ya = b.adjoint(C).cpu().numpy()
    Cn = C.cpu().numpy()
    for r in range(ws):
        j0, j1 = json.load(open(tmp_path / f"r{r}.json"))
        assert np.array_equal(np.load(tmp_path / f"C{r}.npy"), Cn[j0:j1])
        assert rel(np.load(tmp_path / f"y{r}.npy"), yi) < 1e-5
        assert rel(np.load(tmp_path / f"ya{r}.npy"), ya) < 1e-5

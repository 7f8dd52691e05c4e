"""The subsampled transform (sampling on per-scale lattices) and its inversion by
conjugate gradients.

CPU tests pin the oracle: the adjoint identity of the subsampled transform, exactness
of the preconditioned CG in one step when nothing is subsampled (the frame operator is
then the dual-frame weight itself, eq. frame_filter), convergence to the signal from
its own subsampled coefficients, and a planted lattice-phase mistake. GPU tests compare
the library with the oracle.
"""
import numpy as np
import pytest

from oracle import shearlet_oracle as O
from paper_1402_5670_b300 import synth
from tests.conftest import oracle_system

torch = pytest.importorskip("torch")


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def image(dims, seed):
    return synth.add_noise(synth.piecewise_smooth_image(dims, seed), 20.0, seed + 1)


@pytest.mark.parametrize("case", [((32, 32), 2, (1, 1)), ((64, 32), 3, (0, 1, 1))], ids=str)
def test_sub_adjoint_identity(case):
    """<T_sub x, c> = <x, T_sub* c> to 1e-12 for random x and c."""
    dims, J, sl = case
    s = oracle_system(dims, J, sl)
    x = synth.gaussian_field(dims, 50).astype(np.float64)
    steps = O.sub_steps(s)
    c = [synth.gaussian_field((dims[0] // st, dims[1] // st), 60 + j).astype(np.float64)
         for j, st in enumerate(steps)]
    lhs = sum(float(np.sum(a * b)) for a, b in zip(O.forward_sub(x, s), c))
    rhs = float(np.sum(x * O.adjoint_sub(c, s)))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0) * 10


def test_sub_steps_and_sizes():
    """Steps 2^(J-1-j) per scale (the finest keeps every point), 2^(J-1) for the
    lowpass; the compact sizes follow."""
    s = oracle_system((64, 64), 3, (0, 1, 1))
    steps = O.sub_steps(s)
    assert steps[0] == 4
    for j, m in enumerate(s.meta[1:], start=1):
        assert steps[j] == 2 ** (2 - m.scale)
    sizes = [a.size for a in O.forward_sub(np.zeros((64, 64)), s)]
    assert sizes == [64 * 64 // st ** 2 for st in steps]


def test_preconditioned_cg_is_exact_without_subsampling():
    """With every step 1, S = T*T is the multiplication by Psi in frequency, so the
    preconditioner inverts it exactly and one CG step returns x (to 1e-12)."""
    dims, J, sl = (32, 32), 2, (1, 1)
    s = oracle_system(dims, J, sl)
    x = image(dims, 3).astype(np.float64)
    ones = [1] * s.R
    c = O.forward_sub(x, s, ones)
    y, hist = O.cg_inverse_sub(c, s, 1, True, ones)
    assert rel(y, x) < 1e-12 and hist[-1] < 1e-12


@pytest.mark.parametrize("precondition,iters,tol", [(True, 25, 1e-10), (False, 80, 1e-6)])
def test_cg_recovers_the_signal_from_its_subsampled_coefficients(precondition, iters, tol):
    """The subsampled system is a frame (T_sub is injective): CG on S x = T_sub* T_sub x
    converges to x; with the preconditioner in far fewer steps."""
    dims, J, sl = (64, 64), 3, (1, 1, 2)
    s = oracle_system(dims, J, sl)
    x = image(dims, 5).astype(np.float64)
    y, hist = O.cg_inverse_sub(O.forward_sub(x, s), s, iters, precondition)
    assert rel(y, x) < tol
    assert hist[-1] < hist[0]


def test_pin_catches_lattice_phase_slip(monkeypatch):
    """Planted mistake: the adjoint puts the samples back one row off the lattice. The
    adjoint identity must fail."""
    dims, J, sl = (32, 32), 2, (1, 1)
    s = oracle_system(dims, J, sl)
    steps = O.sub_steps(s)

    def bad_adjoint_sub(c, sysm, st=None):
        st = O.sub_steps(sysm) if st is None else st
        full = np.zeros((sysm.R,) + tuple(sysm.dims))
        for j in range(sysm.R):
            full[j][1::st[j], ::st[j]] = c[j][: len(range(1, dims[0], st[j]))]
        return O.adjoint(full, sysm)
    x = synth.gaussian_field(dims, 51).astype(np.float64)
    c = [synth.gaussian_field((dims[0] // st, dims[1] // st), 70 + j).astype(np.float64)
         for j, st in enumerate(steps)]
    lhs = sum(float(np.sum(a * b)) for a, b in zip(O.forward_sub(x, s), c))
    rhs = float(np.sum(x * bad_adjoint_sub(c, s)))
    assert abs(lhs - rhs) > 1e-3 * abs(lhs)


def test_library_layout_matches_oracle():
    from paper_1402_5670_b300.build import build
    from paper_1402_5670_b300.shearlet import Bank
    build()
    b = Bank((128, 64), 4, (1, 1, 2, 2), device=-1)
    st, off = b.sub_layout()
    s_or = O.sub_steps(oracle_system((128, 64), 4, (1, 1, 2, 2)))
    assert list(st) == s_or
    assert list(np.diff(off)) == [128 * 64 // v ** 2 for v in s_or] and off[0] == 0
    b.close()


# ---------------------------------------------------------------------- GPU ---

GPU_CASES = [((256, 256), 4, (1, 1, 2, 2)), ((64, 128), 3, (1, 1, 2))]


@pytest.fixture(scope="module")
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_5670_b300.build import build
    build()


@pytest.mark.gpu
@pytest.mark.parametrize("case", GPU_CASES, ids=str)
def test_gpu_forward_and_adjoint_sub_match_oracle(_gpu, case):
    from paper_1402_5670_b300.shearlet import Bank
    dims, J, sl = case
    b = Bank(dims, J, sl, device=0)
    s = oracle_system(dims, J, sl)
    x = image(dims, 7)
    c = b.forward_sub(torch.from_numpy(x).cuda())
    st, off = b.sub_layout()
    ref = O.forward_sub(x.astype(np.float64), s)
    cn = c.cpu().numpy()
    for j in range(b.R):
        got = cn[off[j]:off[j + 1]].reshape(ref[j].shape)
        assert rel(got, ref[j]) < 1e-5, j
    cr = synth.gaussian_field((int(off[-1]),), 8)
    parts = [cr[off[j]:off[j + 1]].reshape(ref[j].shape).astype(np.float64) for j in range(b.R)]
    xa = b.adjoint_sub(torch.from_numpy(cr).cuda()).cpu().numpy()
    assert rel(xa, O.adjoint_sub(parts, s)) < 1e-5
    b.close()


@pytest.mark.gpu
def test_gpu_cg_inverse_matches_oracle_and_reconstructs(_gpu):
    """Preconditioned CG, 12 steps at 256^2: the GPU reconstructs x from its subsampled
    coefficients to 2e-5 (FP32) and matches the oracle's 12-step iterate from the same
    coefficients, both residuals below 1e-4. Plain CG (30 steps) decreases the
    residual like the oracle's (within 30%)."""
    from paper_1402_5670_b300.shearlet import Bank
    dims, J, sl = (256, 256), 4, (1, 1, 2, 2)
    b = Bank(dims, J, sl, device=0)
    s = oracle_system(dims, J, sl)
    x = image(dims, 9)
    c = b.forward_sub(torch.from_numpy(x).cuda())
    y, res = b.inverse_sub(c, 12, True)
    st, off = b.sub_layout()
    cn = c.cpu().numpy().astype(np.float64)
    parts = [cn[off[j]:off[j + 1]].reshape(dims[0] // st[j], dims[1] // st[j]) for j in range(b.R)]
    yr, hist = O.cg_inverse_sub(parts, s, 12, True)
    assert rel(y.cpu().numpy(), x) < 2e-5
    assert rel(y.cpu().numpy(), yr) < 2e-5
    assert res < 1e-4 and hist[-1] < 1e-4
    y2, res2 = b.inverse_sub(c, 30, False)
    _, hist2 = O.cg_inverse_sub(parts, s, 30, False)
    assert abs(res2 - hist2[-1]) <= 0.3 * hist2[-1]
    assert res2 < 0.05
    b.close()

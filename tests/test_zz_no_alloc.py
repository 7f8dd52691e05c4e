"""sl_forward_noalloc: the forward transform for callers that cannot allocate device
memory at transform time (fixed budgets, host callbacks, memory owned by another
component). Its scratch is a static device array; the caller passes the filter
spectra, the input and the output. Checked against sl_forward on two calls in a row,
within the tolerance of the parity tests. This file runs last (test_zz_*)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel(a, b):
    a = a.double()
    b = b.double()
    return float((a - b).abs().max() / b.abs().max().clamp_min(1e-300))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_5670_b300.build import build
    build()


@pytest.mark.parametrize("case", [((512, 512), 4, (1, 1, 2, 2)), ((64, 32), 2, (1, 1)),
                                  ((32, 16, 8), 2, (1, 1)), ((64, 64, 64), 3, (0, 0, 1))],
                         ids=str)
def test_noalloc_forward_matches_forward_twice(case):
    from paper_1402_5670_b300 import shearlet as S
    from paper_1402_5670_b300 import synth
    dims, J, sl = case
    with S.Bank(dims, J, sl, device=0) as b:
        psi = torch.from_numpy(b.filters_f32()).cuda().contiguous()
        x = synth.add_noise(synth.gaussian_field(dims, 3, 40.0) + 100.0, 5.0, 4)
        xg = torch.from_numpy(x).cuda()
        ref = b.forward(xg)
        for _ in range(2):  # the static scratch keeps the last call's contents
            out = torch.full((b.R,) + dims, float("nan"), device="cuda")
            S.sl_forward_noalloc(b.handle, psi.data_ptr(), xg.data_ptr(), out.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            assert rel(out, ref) < TOL


def test_noalloc_on_tensor_core_bank_matches_fp32_forward():
    """On a bank built in the BF16 tensor-core mode the allocation-free call still runs
    the FP32 kernels: its result matches the FP32 bank's sl_forward to 1e-5, twice."""
    from paper_1402_5670_b300 import shearlet as S
    from paper_1402_5670_b300 import synth
    dims, J, sl = (256, 256), 3, (1, 1, 2)
    x = torch.from_numpy(synth.add_noise(synth.piecewise_smooth_image(dims, 6), 20.0, 7)).cuda()
    with S.Bank(dims, J, sl, device=0) as bf:
        ref = bf.forward(x)
    with S.Bank(dims, J, sl, device=0, precision="tc_bf16") as bt:
        assert bt.precision == "tc_bf16"
        psi = torch.from_numpy(bt.filters_f32()).cuda().contiguous()
        for _ in range(2):
            out = torch.full((bt.R,) + dims, float("nan"), device="cuda")
            S.sl_forward_noalloc(bt.handle, psi.data_ptr(), x.data_ptr(), out.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            assert rel(out, ref) < TOL


def test_noalloc_with_host_only_bank():
    """A host-only bank allocates no device memory; the caller supplies the filters
    (here evaluated in FP64 on the host and rounded to FP32)."""
    from paper_1402_5670_b300 import shearlet as S
    from paper_1402_5670_b300 import synth
    dims, J, sl = (128, 256), 3, (1, 1, 2)
    hb = S.Bank(dims, J, sl, device=-1)
    psi = torch.from_numpy(np.stack([hb.eval_f64(j) for j in range(hb.R)]).astype(np.float32)).cuda()
    x = torch.from_numpy(synth.gaussian_field(dims, 5, 30.0)).cuda()
    with S.Bank(dims, J, sl, device=0) as db:
        ref = db.forward(x)
    for _ in range(2):
        out = torch.empty((hb.R,) + dims, device="cuda")
        S.sl_forward_noalloc(hb.handle, psi.data_ptr(), x.data_ptr(), out.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert rel(out, ref) < TOL
    hb.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1402_5670_b300 import shearlet as S
    hb = S.Bank((128, 128, 128), 1, (0,), device=-1)
    t = torch.zeros(8, device="cuda")
    with pytest.raises(S.ShearletError) as ei:
        S.sl_forward_noalloc(hb.handle, t.data_ptr(), t.data_ptr(), t.data_ptr(), None)
    assert "SL_ENOTSUP" in str(ei.value) and "16 MiB" in str(ei.value)
    hb.close()

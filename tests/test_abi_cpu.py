"""CPU checks of the C ABI: the library loads, exports every symbol the header
declares, validates arguments, and its host-side filter construction (closed-form
frequency responses, FP64) matches the oracle's spatial construction."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1402_5670_b300 import shearlet as S
from paper_1402_5670_b300.build import build
from tests.conftest import ROOT, oracle_system

HEADER = os.path.join(ROOT, "include", "shearlet.h")


@pytest.fixture(scope="module")
def L():
    build()
    return S.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sl_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["sl_build_filters", "sl_forward", "sl_adjoint", "sl_inverse", "sl_threshold",
                 "sl_denoise", "sl_free_filters", "sl_status_str"]:
        assert must in names


def test_library_exports_every_declared_symbol(L):
    for name in declared_functions():
        assert hasattr(L, name), name
    assert set(declared_functions()) == set(S.SIGNATURES)


def test_status_strings(L):
    for code, name in S.STATUS.items():
        assert L.sl_status_str(code).decode() == name


@pytest.mark.parametrize("dims,J,sl,err", [
    ((12, 16), 2, (1, 1), S.STATUS[5]),        # not a power of two
    ((4, 16), 1, (1,), "SL_EINVAL"),           # too small
    ((2048, 16), 1, (1,), "SL_ENOTSUP"),       # too large
    ((16, 16), 0, (), "SL_EINVAL"),            # no scales
    ((16, 16), 1, (-1,), "SL_EINVAL"),         # negative level
    ((16, 16, 256), 1, (0,), "SL_ENOTSUP"),    # 3D plane larger than one CTA holds
    ((768, 64), 1, (1,), "SL_ENOTSUP"),        # 3 * 2^8: only 384 has a mixed-radix plan
    ((384, 16, 16), 1, (0,), "SL_ENOTSUP"),    # 384 is a 2D size only
    ((192, 64), 1, (0,), "SL_ENOTSUP"),        # 192 is a 3D size only
    ((16, 192, 64), 1, (0,), "SL_ENOTSUP"),    # a 192 plane must be 192 x 192
])
def test_invalid_arguments_are_rejected(L, dims, J, sl, err):
    with pytest.raises(S.ShearletError) as ei:
        S.sl_build_filters(dims, J, sl, False, -1)
    assert err in str(ei.value)


def test_transform_on_host_only_bank_is_an_error(L):
    b = S.Bank((16, 16), 1, (1,), device=-1)
    st = L.sl_forward(b.handle, None, None, None)
    assert S.STATUS[st] == "SL_EINVAL"
    assert L.sl_forward(None, None, None, None) == 1
    b.close()


CASES = [((64, 64), 3, (0, 1, 1), False), ((64, 32), 2, (1, 1), False),
         ((256, 256), 2, (1, 1), False), ((32, 32), 2, (1, 2), True),
         ((16, 16, 16), 2, (0, 1), False), ((32, 16, 8), 2, (1, 1), False),
         ((16, 16, 16), 1, (1,), True), ((384, 64), 2, (1, 1), False),
         ((64, 384), 3, (0, 1, 1), False), ((16, 192, 192), 2, (0, 1), False),
         ((192, 16, 8), 1, (1,), False),
         # shear level 3 in 2D (refinement by 8, R = 49) and level 2 in 3D (R = 243)
         ((64, 64), 2, (2, 3), False), ((32, 32, 32), 2, (1, 2), False)]


@pytest.mark.parametrize("case", CASES, ids=str)
def test_library_bank_matches_oracle(L, case):
    """The library evaluates each filter from the closed form of its frequency response;
    the oracle convolves, shears and folds finite filters in space and then takes a DFT.
    Both must give the same normalised real spectra, frame weight, norms and order."""
    dims, J, sl, full = case
    b = S.Bank(dims, J, sl, full, device=-1)
    s = oracle_system(dims, J, sl, full)
    assert b.R == s.R
    nh = dims[-1] // 2 + 1
    for j in range(b.R):
        m = s.meta[j]
        assert b.scale_of[j] == m.scale and b.cone_of[j] == m.cone
        assert tuple(b.k_of[j][:len(m.k)]) == m.k
        ref = s.psi_hat(j)[..., :nh]
        assert np.max(np.abs(b.eval_f64(j) - ref)) <= 1e-12
    assert np.max(np.abs(b.eval_f64(-1) - s.Psi[..., :nh])) <= 1e-12
    assert np.max(np.abs(b.norms - s.norms)) <= 1e-12
    assert abs(b.A - s.A) <= 1e-12 and abs(b.B - 1.0) <= 1e-15
    b.close()


def test_library_bank_matches_oracle_at_512():
    """Full size of the 2D benchmark system (512^2, four scales, levels 1,1,2,2)."""
    b = S.Bank((512, 512), 4, (1, 1, 2, 2), device=-1)
    s = oracle_system((512, 512), 4, (1, 1, 2, 2))
    for j in range(0, b.R, 6):
        assert np.max(np.abs(b.eval_f64(j) - s.psi_hat(j)[:, :257])) <= 1e-12
    assert abs(b.A - s.A) <= 1e-12
    b.close()


def test_library_bank_matches_oracle_at_384():
    """A 384^2 grid (3 * 2^7, one of the batch sizes) with the 49-filter system."""
    b = S.Bank((384, 384), 4, (1, 1, 2, 2), device=-1)
    s = oracle_system((384, 384), 4, (1, 1, 2, 2))
    assert b.R == 49
    for j in list(range(0, b.R, 8)) + [b.R - 1]:
        assert np.max(np.abs(b.eval_f64(j) - s.psi_hat(j)[:, :193])) <= 1e-12
    assert abs(b.A - s.A) <= 1e-12
    b.close()



def test_library_bank_matches_oracle_at_shear_level_4():
    """The maximum shear level (refinement by 16, R = 65 on 64 x 64): the library's
    closed-form bank against values the oracle's spatial construction wrote to
    tests/golden/shear4_bank_64x64.json (make_shear4_bank.py; the oracle build takes
    minutes): order, norms, frame bound A and 12 sampled spectrum values per filter,
    each to 1e-12."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "shear4_bank_64x64.json")) as f:
        g = json.load(f)
    b = S.Bank(tuple(g["dims"]), g["nScales"], tuple(g["shearLevels"]), device=-1)
    assert b.R == g["R"] == len(g["filters"])
    assert abs(b.A - g["A"]) <= 1e-12
    for j, fl in enumerate(g["filters"]):
        assert b.scale_of[j] == fl["scale"] and b.cone_of[j] == fl["cone"]
        assert tuple(b.k_of[j][:len(fl["k"])]) == tuple(fl["k"])
        assert abs(b.norms[j] - fl["norm"]) <= 1e-12
        ph = b.eval_f64(j)
        for k0, k1, v in fl["samples"]:
            assert abs(ph[k0, k1] - v) <= 1e-12, (j, k0, k1)
    b.close()

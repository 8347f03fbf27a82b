"""The integer-pipe binary32 <-> binary64 conversions that the FP32
refinement loops of the local solves use, against the GPU's own conversions,
bit for bit: every float bit pattern to double, and doubles that round to
ties, near-ties, subnormals, zero and overflow to float (IEEE 754 encodings,
round to nearest, ties to even)."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_04653_gb300 import build
    build.build()


def _hook():
    from paper_2104_04653_gb300 import mrcm
    L = mrcm.lib()
    L.mrcm_test_fp_convert.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p,
                                       ctypes.c_void_p]
    L.mrcm_test_fp_convert.restype = ctypes.c_int32
    return L, mrcm


def test_conversions_match_the_hardware_on_every_float_pattern():
    import torch
    L, mrcm = _hook()
    bad = torch.zeros(2, dtype=torch.int64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.mrcm_test_fp_convert(0, 1 << 32, bad.data_ptr(), stream) == mrcm.MRCM_OK
    assert bad.tolist() == [0, 0]


def test_conversion_hook_rejects_bad_arguments():
    import torch
    L, mrcm = _hook()
    bad = torch.zeros(2, dtype=torch.int64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.mrcm_test_fp_convert(0, (1 << 32) + 1, bad.data_ptr(), stream) == mrcm.MRCM_EINVAL
    assert L.mrcm_test_fp_convert(0, 16, None, stream) == mrcm.MRCM_EINVAL
    assert L.mrcm_test_fp_convert(0, 0, bad.data_ptr(), stream) == mrcm.MRCM_OK

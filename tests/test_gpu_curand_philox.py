"""The oracle's Philox-4x32-10 (Salmon et al., SC'11), and the library's,
against cuRAND's implementation of the same generator, word for word.

The walks draw every random number from Philox-4x32-10 blocks with key =
the seed and counter = (g lo, g hi, step, tag) (reading R11 of the
estimator's draws).  cuRAND's curand_init(seed, subsequence, offset) +
curand4() yields exactly the block of counter (offset/4 lo, offset/4 hi,
subsequence lo, subsequence hi) under key = seed, so a helper kernel built
from tests/cuda/curand_philox.cu produces reference words for any counter.
A swapped multiplier, a crossed hi/lo wiring or a missing key bump in the
oracle changes every word."""
import ctypes
import os
import subprocess

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_05581_b300 as mcs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_lib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("curand") / "libcurand_philox.so")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler",
                           "-fPIC", "-o", out, os.path.join(HERE, "cuda", "curand_philox.cu")])
    lib = ctypes.CDLL(out)
    lib.curand_philox_words.argtypes = [ctypes.c_ulonglong, ctypes.c_ulonglong, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_ulonglong, ctypes.c_void_p]
    lib.curand_philox_words.restype = ctypes.c_int
    return lib


def _curand(lib, start, n, c2, c3, key):
    out = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    assert lib.curand_philox_words(start, n, c2, c3, key, out.data_ptr()) == 0
    return out.cpu().numpy().view(np.uint32)


# (start, c2, c3, key): walk start draws (step 0, radial tag and rejection
# tags), walk steps, killing-walk keys, counters across the 32-bit carry and
# nearly all-ones words (cuRAND's offset is 4 g in 64 bits, so g < 2^62)
CASES = [(0, 0, 0xFFFFFFFF, 0), (5, 0, 3, 0x0123456789ABCDEF), (1 << 20, 17, 0, 7),
         ((1 << 32) - 1000, 1023, 31, 0x4B494C4C00000001),
         ((1 << 62) - (1 << 16), 0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFFFFFFFFFF)]


@pytest.mark.parametrize("start,c2,c3,key", CASES)
def test_oracle_philox_equals_curand(oracle, curand_lib, start, c2, c3, key):
    n = 1 << 16
    ref = _curand(curand_lib, start, n, c2, c3, key)
    assert np.array_equal(oracle.philox(start, n, c2, c3, key), ref)


@pytest.mark.parametrize("start,c2,c3,key", CASES)
def test_library_philox_equals_curand(curand_lib, start, c2, c3, key):
    n = 1 << 16
    ref = _curand(curand_lib, start, n, c2, c3, key)
    got = mcs.philox_words(start, n, c2, c3, key).cpu().numpy().view(np.uint32)
    assert np.array_equal(got, ref)

"""Philox4x32-10 against cuRAND's device Philox4_32_10 (a library that is run,
not copied).

cuRAND keys the generator with the 64-bit seed and starts its 128-bit counter
at (0, 0, subsequence); an offset that is a multiple of 4 advances the low 64
bits of the counter by offset / 4, and every curand4() returns one block and
increments the counter.  So draw k after curand_init(seed, S, 4n) is
Philox(counter = (n + k, 0, S_lo, S_hi), key = (seed_lo, seed_hi)), which
the oracle's implementation must reproduce; the CUDA library's own Philox is
tied to the oracle by the bit-exact parity tests.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    out_dir = os.path.join(HERE, "cuda", "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "libcurand_philox_test.so")
    src = os.path.join(HERE, "cuda", "curand_philox.cu")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                           "-Xcompiler", "-fPIC", "-o", so, src])
    lib = ctypes.CDLL(so)
    lib.curand_philox_draw.argtypes = [ctypes.c_ulonglong, ctypes.c_ulonglong, ctypes.c_ulonglong,
                                       ctypes.POINTER(ctypes.c_uint32), ctypes.c_int]
    return lib


@pytest.mark.parametrize("seed,subseq,n", [(0, 0, 0), (1, 0, 0), (0x1234567890ABCDEF, 7, 3),
                                            (42, (1 << 40) + 5, 1000), (2 ** 64 - 1, 2 ** 63, 17)])
def test_oracle_philox_equals_curand(curand_lib, seed, subseq, n):
    k = 6
    buf = (ctypes.c_uint32 * (4 * k))()
    assert curand_lib.curand_philox_draw(seed, subseq, 4 * n, buf, k) == 0
    got = np.frombuffer(buf, dtype=np.uint32).reshape(k, 4)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for d in range(k):
        ctr = [(n + d) & 0xFFFFFFFF, (n + d) >> 32, subseq & 0xFFFFFFFF, subseq >> 32]
        assert oracle.philox4x32_10(ctr, key) == [int(x) for x in got[d]], (seed, subseq, n, d)

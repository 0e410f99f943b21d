"""The oracle's Philox4x32-10 against cuRAND's device Philox4_32_10, bit for bit.

The paper only asks for i.i.d. standard Gaussians (Sec. 2.1); the noise of both sides is drawn
from Philox4x32-10 (Salmon et al., SC'11) keyed by (seed, n, l, atom).  This test pins the
oracle's raw bit stream to an independent implementation of the published generator, cuRAND's
curand_kernel.h, on a grid of keys and counters that exercises every word: a wrong multiplier,
Weyl constant, round count or word order fails it.  (The GPU kernels are pinned to the oracle
through the trajectory parity tests, which use the same draws.)"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
from gpu_util import dev, torch

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_lib(tmp_path_factory):
    dev()
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = str(tmp_path_factory.mktemp("curand") / "libphilox_curand.so")
    cmd = [nvcc, "-shared", "-Xcompiler", "-fPIC", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
           "-cudart", "static", os.path.join(HERE, "philox_curand.cu"), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    L = ctypes.CDLL(out)
    L.curand_philox_blocks.argtypes = [ctypes.c_int] + [ctypes.c_void_p] * 4
    return L


def test_oracle_philox_equals_curand_philox(curand_lib):
    rng = np.random.default_rng(20221220)
    seeds = [0, 1, 0xFFFFFFFF, 0x100000000, 0xDEADBEEFCAFEF00D] + [int(x) for x in rng.integers(0, 2**63, 11)]
    subs = [0, 1, 7, 0xFFFFFFFF, 0x100000001] + [int(x) for x in rng.integers(0, 2**40, 3)]
    blocks = [0, 1, 2, 255, 0xFFFFFFFF, 0x123456789] + [int(x) for x in rng.integers(0, 2**33, 2)]
    grid = np.array([(s, q, b) for s in seeds for q in subs for b in blocks], dtype=np.uint64)
    n = len(grid)
    d = dev()
    cols = [torch.from_numpy(grid[:, i].astype(np.int64, casting="unsafe").copy()).to(d) for i in range(3)]
    out = torch.zeros(4 * n, dtype=torch.int32, device=d)
    rc = curand_lib.curand_philox_blocks(n, cols[0].data_ptr(), cols[1].data_ptr(), cols[2].data_ptr(),
                                         out.data_ptr())
    assert rc == 0
    got = out.cpu().numpy().view(np.uint32).reshape(n, 4)
    mask = 0xFFFFFFFF
    for i, (s, q, b) in enumerate(grid.tolist()):
        ctr = [b & mask, b >> 32, q & mask, q >> 32]
        key = [s & mask, s >> 32]
        want = O.philox4x32_10(ctr, key)
        assert np.array_equal(got[i], want), (s, q, b, got[i], want)

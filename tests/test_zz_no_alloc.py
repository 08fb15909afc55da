"""The allocation-free entry point muffin_spectral_l1_noalloc.

It serves callers that cannot allocate device memory (a framework that owns
every device byte, a plugin handed fixed buffers, a memory-capped service):
its scratch lives in a static device array inside the library.  This file is
collected last so that a failure here comes after every other test has run.

Each result is checked twice: against the existing entry point
(muffin_objective's spectral term, which uses a caller workspace) and against
the FP64 oracle's spectral transform, whose l1 norm is summed on the host.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import muffin_oracle as mo
from gpu_helpers import small_cube, problem, gpu_solver

pytestmark = pytest.mark.gpu
TOL = 1e-6   # relative, as for the objective terms in test_gpu_parity.py


def _entry(lib):
    fn = lib.lib.muffin_spectral_l1_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    err = lib.lib.muffin_noalloc_last_error
    err.restype = ctypes.c_char_p
    err.argtypes = []
    return fn, err


def _existing_entry_l1(n, L, seed, x):
    """The existing entry point: muffin_objective's spectral term with mu_lambda = 1."""
    cube = small_cube(n, L, 1, seed=seed)
    p = problem(cube, 1, 1, 0.25, 1.0, tau=1e-3)
    m = gpu_solver(cube, p)
    m.set_cube(torch.from_numpy(x).cuda())
    _, terms = m.objective()
    m.close()
    return terms[2]


def _oracle_l1(x):
    """sum over pixels of ||W_lambda x^n||_1 in FP64 (Eq. 6, third term)."""
    return float(np.sum(np.abs(mo.spectral_analysis(x.reshape(x.shape[0], -1).astype(np.float64)))))


def _call(fn, err, x, out_slot):
    L = x.shape[0]
    xd = torch.from_numpy(np.ascontiguousarray(x.reshape(L, -1))).cuda()
    r = fn(xd.data_ptr(), xd.shape[1], L, out_slot.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert r == 0, err()
    torch.cuda.synchronize()
    return float(out_slot.item())


def test_noalloc_matches_existing_entry_point_twice(lib):
    """Two calls in a row (FFT-DCT path, then dense-DCT path), each equal to the
    spectral term of muffin_objective and to the oracle."""
    fn, err = _entry(lib)
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    cases = [(64, 64, 101), (32, 15, 102)]
    for i, (n, L, seed) in enumerate(cases):
        x = np.abs(np.random.Generator(np.random.PCG64(seed)).standard_normal((L, n, n))).astype(np.float32)
        got = _call(fn, err, x, out[i:i + 1])
        ref = _existing_entry_l1(n, L, seed, x)
        assert abs(got - ref) <= TOL * abs(ref), (got, ref)
        orc = _oracle_l1(x)
        assert abs(got - orc) <= TOL * abs(orc), (got, orc)


@pytest.mark.parametrize("n_pix,L", [(33 * 33, 15), (1000, 16), (1, 1), (31, 256)])
def test_noalloc_ragged_pixel_counts_match_oracle(lib, n_pix, L):
    """Pixel counts that are not a multiple of the kernel's 32 pixels per block
    (the last block is partly empty), on both DCT paths, against the oracle."""
    fn, err = _entry(lib)
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    x = np.random.Generator(np.random.PCG64(n_pix + L)).standard_normal((L, n_pix)).astype(np.float32)
    for _ in range(2):   # the second call reuses the partial sums the first one left behind
        got = _call(fn, err, x, out)
        orc = _oracle_l1(x)
        assert abs(got - orc) <= TOL * abs(orc), (got, orc)


def test_noalloc_rejects_sizes_beyond_its_array(lib):
    fn, err = _entry(lib)
    x = torch.zeros(4, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert fn(x.data_ptr(), (1 << 20) + 1, 1, out.data_ptr(), s) == -1 and b"n_pix" in err()
    assert fn(x.data_ptr(), 16, 257, out.data_ptr(), s) == -1 and b"nchan" in err()

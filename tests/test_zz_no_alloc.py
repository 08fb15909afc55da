"""The allocation-free entry point muffin_spectral_l1_noalloc.

It serves callers that cannot allocate device memory (a framework that owns
every device byte, a plugin handed fixed buffers, a memory-capped service):
its scratch lives in a static device array inside the library.  This file is
collected last so that a failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

from gpu_helpers import small_cube, problem, gpu_solver

pytestmark = pytest.mark.gpu


def _entry(lib):
    fn = lib.lib.muffin_spectral_l1_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    err = lib.lib.muffin_noalloc_last_error
    err.restype = ctypes.c_char_p
    err.argtypes = []
    return fn, err


def _reference_l1(n, L, seed, x):
    """The existing entry point: muffin_objective's spectral term with mu_lambda = 1."""
    cube = small_cube(n, L, 1, seed=seed)
    p = problem(cube, 1, 1, 0.25, 1.0, tau=1e-3)
    m = gpu_solver(cube, p)
    m.set_cube(torch.from_numpy(x).cuda())
    _, terms = m.objective()
    m.close()
    return terms[2]


def test_noalloc_matches_objective_term_twice(lib):
    fn, err = _entry(lib)
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    cases = [(64, 64, 101), (32, 15, 102)]      # FFT-DCT path, then dense-DCT path
    for i, (n, L, seed) in enumerate(cases):
        x = np.abs(np.random.Generator(np.random.PCG64(seed)).standard_normal((L, n, n))).astype(np.float32)
        xd = torch.from_numpy(x).cuda()
        r = fn(xd.data_ptr(), n * n, L, out[i:i + 1].data_ptr(), stream)
        assert r == 0, err()
        torch.cuda.synchronize()
        ref = _reference_l1(n, L, seed, x)
        got = float(out[i].item())
        assert abs(got - ref) <= 1e-6 * abs(ref), (got, ref)


def test_noalloc_rejects_sizes_beyond_its_array(lib):
    fn, err = _entry(lib)
    x = torch.zeros(4, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert fn(x.data_ptr(), (1 << 20) + 1, 1, out.data_ptr(), s) == -1 and b"n_pix" in err()
    assert fn(x.data_ptr(), 16, 257, out.data_ptr(), s) == -1 and b"nchan" in err()

"""The C ABI without a GPU: the library loads, exports every entry point that
a header under include/ declares, and its host-side checks behave (no compute
calls)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


def declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(muffin_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def so():
    from paper_1602_08847_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    return ctypes.CDLL(build.LIB)


def test_every_declared_symbol_is_exported(so):
    names = declared_functions()
    assert len(HEADERS) >= 2 and len(names) >= 30
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing


def test_check_params_and_workspace():
    from paper_1602_08847_gb300.muffin import make_params, muffin_check_params, muffin_workspace_bytes, stage_names
    ok = make_params(512, 256, 5)
    assert muffin_check_params(ok) == (0, "ok")
    nb = muffin_workspace_bytes(ok)
    vox = 512 * 512 * 256
    # state (X, 6 planes of U, V) + y, b, K, FFT / wavelet / spectral scratch, FP64 spectra
    assert 4 * vox * 12 < nb < 4 * vox * 32
    for bad, why in [(make_parms := make_params(500, 4, 2), "power of two"),
                     (make_params(64, 4, 6), "2^J < N"),
                     (make_params(64, 0, 2), "nchan"),
                     (make_params(64, 4, 2, gen=3), "iuwt_gen"),
                     (make_params(64, 4, 2, mu_s=-1.0), "mu_s"),
                     (make_params(64, 4, 3, fine_levels=4), "fine_levels"),
                     (make_params(32, 4, 3, fine_levels=1), "N >= 64"),
                     (make_params(1024, 4, 5, fine_levels=1), "shared memory"),
                     (make_params(64, 2, 2, weights=[1.0, 0.0]), "weights")]:
        code, msg = muffin_check_params(bad)
        assert code == -1 and why in msg, (why, msg)
        assert muffin_workspace_bytes(bad) == 0
    assert make_parms.nx == 500
    assert stage_names() == ["iuwt_fine_adjoint", "fft_rows_fwd", "fft_cols_filter", "fft_rows_inv_primal",
                             "iuwt_fine_analysis", "iuwt_coarse", "spectral_dct"]


def test_init_rejects_bad_arguments_before_any_cuda_call():
    from paper_1602_08847_gb300.muffin import lib, make_params
    ctx = ctypes.c_void_p()
    p = make_params(64, 4, 2)
    r = lib.muffin_init(ctypes.byref(ctx), ctypes.byref(p), None, None, 0, None)
    assert r == -1 and b"NULL" in lib.muffin_last_error(None)
    r = lib.muffin_init(ctypes.byref(ctx), ctypes.byref(p), 256, 0x1001, 1 << 30, None)
    assert r == -1 and b"aligned" in lib.muffin_last_error(None)
    r = lib.muffin_init(ctypes.byref(ctx), ctypes.byref(p), 256, 0x1000, 16, None)
    assert r == -3
    assert lib.muffin_iterate(None, 1) == -1


def test_net_sizes_and_create_argument_checks(so):
    so.muffin_net_workspace_bytes.restype = ctypes.c_size_t
    so.muffin_net_workspace_bytes.argtypes = [ctypes.c_int] * 5
    so.muffin_conv3d_scratch_bytes.restype = ctypes.c_size_t
    so.muffin_conv3d_scratch_bytes.argtypes = [ctypes.c_int] * 3
    so.muffin_net_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.POINTER(ctypes.c_float), ctypes.c_int, ctypes.c_void_p,
                                     ctypes.c_size_t, ctypes.c_void_p]
    so.muffin_net_num_params.argtypes = [ctypes.c_int]
    assert so.muffin_net_num_params(1) == 112481
    assert so.muffin_net_num_params(6) == 112481 + 5 * 865
    assert so.muffin_net_num_params(0) == 0 and so.muffin_net_num_params(9) == 0
    infer = so.muffin_net_workspace_bytes(64, 256, 256, 1, 0)
    train = so.muffin_net_workspace_bytes(64, 256, 256, 6, 1)
    V = 64 * 256 * 256
    assert infer >= V * 2 + 2 * V * 64               # input map + two feature maps
    assert train >= V * 2 + 7 * V * 64 + 6 * V * 4   # five kept maps, two gradient maps, loss gradients
    assert so.muffin_net_workspace_bytes(0, 4, 4, 1, 0) == 0
    assert so.muffin_net_workspace_bytes(4, 4, 4, 9, 0) == 0
    assert so.muffin_net_workspace_bytes(1 << 20, 1 << 10, 1 << 10, 1, 0) == 0
    assert so.muffin_conv3d_scratch_bytes(3, 5, 7) > 27648 * 2
    net = ctypes.c_void_p()
    assert so.muffin_net_create(ctypes.byref(net), 0, 8, 8, 1, None, 0, None, 0, None) == -1
    assert so.muffin_net_create(ctypes.byref(net), 4, 8, 8, 1, None, 0, None, 1 << 20, None) == -1
    neg = (ctypes.c_float * 2)(1.0, -1.0)
    assert so.muffin_net_create(ctypes.byref(net), 4, 8, 8, 2, neg, 0, ctypes.c_void_p(256), 1 << 30, None) == -1
    assert so.muffin_net_create(ctypes.byref(net), 4, 8, 8, 1, None, 0, ctypes.c_void_p(256), 16, None) == -3
    assert not net.value


def test_daubechies_filters_match_the_oracle(so):
    """The library's own filters (host C++, Durand-Kerner roots) equal the
    oracle's (numpy roots) for every basis of the union."""
    import numpy as np
    from oracle import muffin_oracle as mo
    so.muffin_daubechies_filter.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    for p in range(1, 9):
        buf = (ctypes.c_double * 16)()
        assert so.muffin_daubechies_filter(p, buf) == 0
        assert np.allclose(np.array(buf[:2 * p]), mo.daubechies_lowpass(p), rtol=0, atol=1e-12), p
    assert so.muffin_daubechies_filter(0, (ctypes.c_double * 16)()) == -1
    assert so.muffin_daubechies_filter(9, (ctypes.c_double * 16)()) == -1

"""The C ABI without a GPU: the library loads, exports every entry point that
include/muffin.h declares, and its host-side checks behave (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "muffin.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(muffin_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def so():
    from paper_1602_08847_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    return ctypes.CDLL(build.LIB)


def test_every_declared_symbol_is_exported(so):
    names = declared_functions()
    assert len(names) >= 19
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

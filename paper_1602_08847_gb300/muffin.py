"""Python binding of libmuffin (include/muffin.h): argument marshalling only.

Every step of the MUFFIN iteration runs in the CUDA library; this module only
passes device pointers, sizes and the current torch stream through ctypes.
PyTorch provides device memory (the workspace and the cubes) and streams.
There is no CPU fallback: importing this module on a machine where the
library was not built raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libmuffin.so")

MUFFIN_OK = 0
ERRORS = {-1: "MUFFIN_ERR_ARG", -2: "MUFFIN_ERR_CUDA", -3: "MUFFIN_ERR_NOMEM", -4: "MUFFIN_ERR_STATE",
          -5: "MUFFIN_ERR_NONFINITE", -6: "MUFFIN_ERR_TIMEOUT"}


class MuffinError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class muffin_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nchan", ctypes.c_int), ("nscales", ctypes.c_int),
        ("iuwt_gen", ctypes.c_int), ("mu_s", ctypes.c_double), ("mu_l", ctypes.c_double),
        ("tau", ctypes.c_double), ("sigma", ctypes.c_double), ("rho", ctypes.c_double),
        ("h_chan_weight", ctypes.POINTER(ctypes.c_double)), ("fine_levels", ctypes.c_int),
        ("power_iters", ctypes.c_int), ("dictionary", ctypes.c_int),
    ]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libmuffin.so not built ({_LIB_PATH}); run python -m paper_1602_08847_gb300.build")
    lib = ctypes.CDLL(_LIB_PATH)
    P, I, D, S, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t, None
    pd = ctypes.POINTER(ctypes.c_double)
    sig = {
        "muffin_workspace_bytes": (S, [ctypes.POINTER(muffin_params)]),
        "muffin_check_params": (I, [ctypes.POINTER(muffin_params), ctypes.c_char_p, S]),
        "muffin_init": (I, [ctypes.POINTER(P), ctypes.POINTER(muffin_params), P, P, S, P]),
        "muffin_set_psf": (I, [P, P]),
        "muffin_iterate": (I, [P, I]),
        "muffin_objective": (I, [P, pd, pd]),
        "muffin_get_cube": (I, [P, P]),
        "muffin_set_cube": (I, [P, P]),
        "muffin_get_state": (I, [P, P, P, P, ctypes.POINTER(ctypes.c_longlong)]),
        "muffin_set_state": (I, [P, P, P, P, ctypes.c_longlong]),
        "muffin_set_mu": (I, [P, D, D]),
        "muffin_step_sizes": (I, [P, pd, pd, pd, pd, pd, pd, pd]),
        "muffin_iterate_timed": (I, [P, I, pd, I]),
        "muffin_set_plan": (I, [P, I, I]),
        "muffin_block_threads": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "muffin_plan": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "muffin_num_stages": (I, []),
        "muffin_stage_name": (ctypes.c_char_p, [I]),
        "muffin_stage_bytes": (D, [P, I]),
        "muffin_kernels_per_iteration": (I, [P]),
        "muffin_tiling": (I, [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
        "muffin_daubechies_filter": (I, [I, ctypes.POINTER(ctypes.c_double)]),
        "muffin_last_error": (ctypes.c_char_p, [P]),
        "muffin_batch_create": (I, [ctypes.POINTER(P), ctypes.POINTER(P), I, P]),
        "muffin_batch_iterate": (I, [P, I]),
        "muffin_batch_last_error": (ctypes.c_char_p, [P]),
        "muffin_batch_set_mode": (I, [P, I]),
        "muffin_batch_mode": (I, [P]),
        "muffin_batch_set_wait_limit": (I, [P, ctypes.c_longlong]),
        "muffin_batch_check": (I, [P]),
        "muffin_batch_destroy": (V, [P]),
        "muffin_destroy": (V, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()
lib = _lib


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


DICTIONARIES = {"iuwt": 0, "union": 1}


def make_params(n, nchan, nscales, gen=1, mu_s=0.25, mu_l=3.0, tau=0.0, sigma=0.0, rho=0.0, weights=None,
                fine_levels=-1, power_iters=0, dictionary="iuwt"):
    p = muffin_params()
    p.nx = p.ny = int(n)
    p.nchan, p.nscales, p.iuwt_gen = int(nchan), int(nscales), int(gen)
    p.mu_s, p.mu_l, p.tau, p.sigma, p.rho = float(mu_s), float(mu_l), float(tau), float(sigma), float(rho)
    p._w = None
    if weights is not None:
        arr = (ctypes.c_double * len(weights))(*[float(v) for v in weights])
        p._w = arr
        p.h_chan_weight = ctypes.cast(arr, ctypes.POINTER(ctypes.c_double))
    p.fine_levels, p.power_iters = int(fine_levels), int(power_iters)
    p.dictionary = DICTIONARIES[dictionary]
    return p


def muffin_workspace_bytes(p: muffin_params) -> int:
    return int(_lib.muffin_workspace_bytes(ctypes.byref(p)))


def muffin_check_params(p: muffin_params) -> tuple[int, str]:
    buf = ctypes.create_string_buffer(256)
    r = _lib.muffin_check_params(ctypes.byref(p), buf, 256)
    return r, buf.value.decode()


def stage_names() -> list[str]:
    return [_lib.muffin_stage_name(k).decode() for k in range(_lib.muffin_num_stages())]


class Muffin:
    """One MUFFIN problem on the current CUDA device (a context of libmuffin).

    ``dirty`` and ``psf`` are [L][N][N] float32 tensors (device or host; host
    tensors are copied to the device first).
    """

    def __init__(self, dirty: torch.Tensor, psf: torch.Tensor | None = None, *, nscales: int, gen: int = 1,
                 mu_s: float = 0.25, mu_l: float = 3.0, tau: float = 0.0, sigma: float = 0.0, rho: float = 0.0,
                 weights=None, fine_levels: int = -1, power_iters: int = 0, dictionary: str = "iuwt", device="cuda"):
        L, n, n2 = dirty.shape
        self.shape = (L, n, n2)
        self.nscales = nscales
        self.dictionary = dictionary
        self.u_planes = 8 if dictionary == "union" else nscales + 1   # planes of the dual U per channel
        self.params = make_params(n, L, nscales, gen, mu_s, mu_l, tau, sigma, rho, weights, fine_levels, power_iters,
                                  dictionary)
        code, msg = muffin_check_params(self.params)
        if code != MUFFIN_OK:
            raise MuffinError(code, msg)
        nbytes = muffin_workspace_bytes(self.params)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
        d = dirty.to(device=device, dtype=torch.float32).contiguous()
        self._ctx = ctypes.c_void_p()
        r = _lib.muffin_init(ctypes.byref(self._ctx), ctypes.byref(self.params), _ptr(d), _ptr(self.workspace),
                             nbytes, _stream())
        if r != MUFFIN_OK:
            raise MuffinError(r, _lib.muffin_last_error(None).decode())
        if psf is not None:
            self.set_psf(psf)

    def _check(self, r: int):
        if r != MUFFIN_OK:
            raise MuffinError(r, _lib.muffin_last_error(self._ctx).decode())

    @property
    def ctx(self):
        return self._ctx

    def set_psf(self, psf: torch.Tensor):
        p = psf.to(device=self.workspace.device, dtype=torch.float32).contiguous()
        self._check(_lib.muffin_set_psf(self._ctx, _ptr(p)))

    def iterate(self, n: int = 1):
        self._check(_lib.muffin_iterate(self._ctx, int(n)))

    def iterate_timed(self, n: int) -> list[float]:
        k = _lib.muffin_num_stages()
        ms = (ctypes.c_double * k)()
        self._check(_lib.muffin_iterate_timed(self._ctx, int(n), ms, k))
        return list(ms)

    def objective(self) -> tuple[float, tuple[float, float, float]]:
        tot = ctypes.c_double()
        terms = (ctypes.c_double * 3)()
        self._check(_lib.muffin_objective(self._ctx, ctypes.byref(tot), terms))
        return tot.value, tuple(terms)

    def get_cube(self) -> torch.Tensor:
        x = torch.empty(self.shape, dtype=torch.float32, device=self.workspace.device)
        self._check(_lib.muffin_get_cube(self._ctx, _ptr(x)))
        return x

    def set_cube(self, x: torch.Tensor):
        x = x.to(device=self.workspace.device, dtype=torch.float32).contiguous()
        self._check(_lib.muffin_set_cube(self._ctx, _ptr(x)))

    def get_state(self):
        L, n, _ = self.shape
        dev = self.workspace.device
        x = torch.empty((L, n, n), dtype=torch.float32, device=dev)
        u = torch.empty((L, self.u_planes, n, n), dtype=torch.float32, device=dev)
        v = torch.empty((L, n, n), dtype=torch.float32, device=dev)
        it = ctypes.c_longlong()
        self._check(_lib.muffin_get_state(self._ctx, _ptr(x), _ptr(u), _ptr(v), ctypes.byref(it)))
        return x, u, v, it.value

    def set_state(self, x, u, v, it: int = 0):
        dev = self.workspace.device
        x = x.to(device=dev, dtype=torch.float32).contiguous()
        u = u.to(device=dev, dtype=torch.float32).contiguous()
        v = v.to(device=dev, dtype=torch.float32).contiguous()
        self._check(_lib.muffin_set_state(self._ctx, _ptr(x), _ptr(u), _ptr(v), int(it)))
        torch.cuda.current_stream().synchronize()

    def set_mu(self, mu_s: float, mu_l: float):
        self._check(_lib.muffin_set_mu(self._ctx, float(mu_s), float(mu_l)))

    def step_sizes(self) -> dict:
        vals = [ctypes.c_double() for _ in range(7)]
        self._check(_lib.muffin_step_sizes(self._ctx, *[ctypes.byref(v) for v in vals]))
        keys = ["tau", "sigma", "rho", "beta", "l_norm2", "beta_closed", "ws_norm2"]
        return {k: v.value for k, v in zip(keys, vals)}

    def stage_bytes(self) -> list[float]:
        return [_lib.muffin_stage_bytes(self._ctx, k) for k in range(_lib.muffin_num_stages())]

    def kernels_per_iteration(self) -> int:
        return int(_lib.muffin_kernels_per_iteration(self._ctx))

    def set_plan(self, channels_per_group: int, branches: int = 1):
        """Channels per group of the pass (0: whole cube) and graph branches (1..3)."""
        self._check(_lib.muffin_set_plan(self._ctx, int(channels_per_group), int(branches)))

    def plan(self) -> tuple[int, int]:
        g, b = ctypes.c_int(), ctypes.c_int()
        self._check(_lib.muffin_plan(self._ctx, ctypes.byref(g), ctypes.byref(b)))
        return g.value, b.value

    def block_threads(self) -> tuple[int, int]:
        """Threads per block of the vectorised fine and coarse wavelet kernels."""
        f, c = ctypes.c_int(), ctypes.c_int()
        self._check(_lib.muffin_block_threads(self._ctx, ctypes.byref(f), ctypes.byref(c)))
        return f.value, c.value

    def tiling(self) -> tuple[int, int]:
        j1, cs = ctypes.c_int(), ctypes.c_int()
        self._check(_lib.muffin_tiling(self._ctx, ctypes.byref(j1), ctypes.byref(cs)))
        return j1.value, cs.value

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            torch.cuda.current_stream().synchronize()
            _lib.muffin_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several Muffin problems (cubes of any sizes) advanced together: one CUDA
    graph launch per pass runs every cube's kernels as parallel branches."""

    def __init__(self, problems: list):
        self.problems = list(problems)
        arr = (ctypes.c_void_p * len(self.problems))(*[m.ctx.value for m in self.problems])
        self._b = ctypes.c_void_p()
        r = _lib.muffin_batch_create(ctypes.byref(self._b), arr, len(self.problems), _stream())
        if r != MUFFIN_OK:
            raise MuffinError(r, _lib.muffin_batch_last_error(None).decode())

    def iterate(self, n: int = 1):
        r = _lib.muffin_batch_iterate(self._b, int(n))
        if r != MUFFIN_OK:
            raise MuffinError(r, _lib.muffin_batch_last_error(self._b).decode())

    def set_mode(self, mode: str):
        """"graph": parallel graph branches per cube; "persistent": one persistent launch per pass."""
        m = {"graph": 0, "persistent": 1}[mode]
        r = _lib.muffin_batch_set_mode(self._b, m)
        if r != MUFFIN_OK:
            raise MuffinError(r, _lib.muffin_batch_last_error(self._b).decode())

    @property
    def mode(self) -> str:
        return {0: "graph", 1: "persistent"}[int(_lib.muffin_batch_mode(self._b))]

    def set_wait_limit(self, polls: int | None):
        """Poll bound of the persistent kernel's barrier waits (None: the default)."""
        r = _lib.muffin_batch_set_wait_limit(self._b, -1 if polls is None else int(polls))
        if r != MUFFIN_OK:
            raise MuffinError(r, _lib.muffin_batch_last_error(self._b).decode())

    def check(self):
        """Wait for the batch; raise MuffinError(TIMEOUT) if a barrier wait gave up."""
        r = _lib.muffin_batch_check(self._b)
        if r != MUFFIN_OK:
            raise MuffinError(r, _lib.muffin_batch_last_error(self._b).decode())

    def close(self):
        if getattr(self, "_b", None) and self._b.value:
            torch.cuda.current_stream().synchronize()
            _lib.muffin_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(dirty, psf, n_iter: int, **kw) -> torch.Tensor:
    """Whole call from host or device cubes: set up, run n_iter passes, return X (on the input's device)."""
    m = Muffin(dirty, psf, **kw)
    m.iterate(n_iter)
    x = m.get_cube()
    out = x.to(dirty.device) if dirty.device.type == "cpu" else x
    m.close()
    return out

"""Python binding of the warm-start network (include/muffin_net.h).

Argument marshalling only: the forward pass, the loss, the gradients and Adam
all run in libmuffin's CUDA kernels.  PyTorch provides the device memory
(workspaces, cubes, parameter vectors) and the stream.  Like the rest of the
package there is no CPU fallback: this module raises at import when the
library is missing.
"""
from __future__ import annotations

import ctypes

import torch

from . import muffin as _m

_lib = _m.lib
_P, _I, _S, _F = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_float
_SIG = {
    "muffin_net_num_params": (_I, [_I]),
    "muffin_net_workspace_bytes": (_S, [_I, _I, _I, _I, _I]),
    "muffin_net_create": (_I, [ctypes.POINTER(_P), _I, _I, _I, _I, ctypes.POINTER(_F), _I, _P, _S, _P]),
    "muffin_net_set_params": (_I, [_P, _P]),
    "muffin_net_get_params": (_I, [_P, _P]),
    "muffin_net_predict": (_I, [_P, _P, _P, _P]),
    "muffin_net_loss_grad": (_I, [_P, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_double)]),
    "muffin_net_train_step": (_I, [_P, _P, _P, _P, _F, _P]),
    "muffin_net_last_error": (ctypes.c_char_p, [_P]),
    "muffin_net_wait_timeouts": (_I, []),
    "muffin_net_check": (_I, [_P]),
    "muffin_net_set_wait_limit": (_I, [ctypes.c_longlong]),
    "muffin_net_destroy": (None, [_P]),
    "muffin_conv3d_scratch_bytes": (_S, [_I, _I, _I]),
    "muffin_conv3d_forward": (_I, [_P, _P, _P, _I, _P, _I, _I, _I, _P, _S, _P]),
    "muffin_conv3d_backward_data": (_I, [_P, _P, _P, _P, _I, _I, _I, _P, _S, _P]),
    "muffin_conv3d_backward_weights": (_I, [_P, _P, _P, _P, _I, _I, _I, _P, _S, _P]),
    "muffin_conv3d_last_error": (ctypes.c_char_p, []),
}
for _name, (_res, _args) in _SIG.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args

FEATURES = 32


def n_params(n_out: int = 1) -> int:
    """Packed parameter count of the network with n_out output maps."""
    n = int(_lib.muffin_net_num_params(int(n_out)))
    if n == 0:
        raise ValueError(f"n_out must be in [1, 8], got {n_out}")
    return n


N_PARAMS = n_params(1)


def wait_timeouts() -> int:
    """Tensor-core waits that gave up since the last call (0 in a healthy run)."""
    return int(_lib.muffin_net_wait_timeouts())


def set_wait_limit(polls: int | None) -> None:
    """Poll bound of the tensor-core pipeline waits (None: the default 2^20)."""
    r = int(_lib.muffin_net_set_wait_limit(-1 if polls is None else int(polls)))
    if r != 0:
        raise _m.MuffinError(r, "muffin_net_set_wait_limit failed")


def _ptr(t):
    return None if t is None else t.data_ptr()


def _dev_f32(t: torch.Tensor, name: str) -> torch.Tensor:
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    return t


def _map(t: torch.Tensor, shape, name: str) -> torch.Tensor:
    if not (t.is_cuda and t.dtype == torch.bfloat16 and t.is_contiguous()) or tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must be a contiguous bfloat16 CUDA tensor of shape {tuple(shape)}")
    return t


class WarmStartNet:
    """The network on nz x ny x nx cubes (a libmuffin network context).

    n_out output maps: map 0 predicts the cube, maps 1 .. n_out-1 further
    fields of the state (the planes of the wavelet dual U when n_out = J + 2);
    out_weight gives the n_out loss weights (default all 1)."""

    def __init__(self, shape, training: bool = False, theta: torch.Tensor | None = None, n_out: int = 1,
                 out_weight=None):
        self.shape = tuple(int(s) for s in shape)
        nz, ny, nx = self.shape
        self.training = bool(training)
        self.n_out = int(n_out)
        self.n_params = n_params(self.n_out)
        nbytes = int(_lib.muffin_net_workspace_bytes(nz, ny, nx, self.n_out, int(self.training)))
        if nbytes == 0:
            raise ValueError(f"invalid cube shape {self.shape}")
        lam = None
        if out_weight is not None:
            if len(out_weight) != self.n_out:
                raise ValueError("out_weight needs one value per output map")
            lam = (_F * self.n_out)(*[float(v) for v in out_weight])
        self._ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self._net = _P()
        r = _lib.muffin_net_create(ctypes.byref(self._net), nz, ny, nx, self.n_out, lam, int(self.training),
                                   self._ws.data_ptr(), nbytes, torch.cuda.current_stream().cuda_stream)
        if r != 0:
            raise _m.MuffinError(r, _lib.muffin_net_last_error(None).decode())
        if theta is not None:
            self.set_params(theta)

    def _check(self, r: int):
        if r != 0:
            raise _m.MuffinError(r, _lib.muffin_net_last_error(self._net).decode())

    def _cube(self, t: torch.Tensor, name: str) -> torch.Tensor:
        _dev_f32(t, name)
        if tuple(t.shape) != self.shape:
            raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {self.shape}")
        return t

    def set_params(self, theta: torch.Tensor):
        theta = _dev_f32(theta.reshape(-1), "theta")
        if theta.numel() != self.n_params:
            raise ValueError(f"theta has {theta.numel()} values, expected {self.n_params}")
        self._check(_lib.muffin_net_set_params(self._net, theta.data_ptr()))

    def get_params(self) -> torch.Tensor:
        out = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        self._check(_lib.muffin_net_get_params(self._net, out.data_ptr()))
        return out

    def _aux_shape(self):
        nz, ny, nx = self.shape
        return (nz, self.n_out - 1, ny, nx)

    def _aux_target(self, t):
        if self.n_out == 1:
            return None
        if t is None or not (t.is_cuda and t.dtype == torch.bfloat16 and t.is_contiguous()) \
                or tuple(t.shape) != self._aux_shape():
            raise ValueError(f"target_aux must be a contiguous bfloat16 CUDA tensor of shape {self._aux_shape()}")
        return t

    def predict(self, dirty: torch.Tensor):
        """(cube [nz][ny][nx], fields [nz][n_out-1][ny][nx] or None)."""
        self._cube(dirty, "dirty")
        x = torch.empty_like(dirty)
        aux = torch.empty(self._aux_shape(), dtype=torch.float32, device="cuda") if self.n_out > 1 else None
        self._check(_lib.muffin_net_predict(self._net, dirty.data_ptr(), x.data_ptr(), _ptr(aux)))
        return x, aux

    def loss_grad(self, dirty: torch.Tensor, target_x: torch.Tensor,
                  target_aux: torch.Tensor | None = None) -> tuple[float, torch.Tensor]:
        self._cube(dirty, "dirty")
        self._cube(target_x, "target_x")
        ta = self._aux_target(target_aux)
        g = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        loss = ctypes.c_double()
        self._check(_lib.muffin_net_loss_grad(self._net, dirty.data_ptr(), target_x.data_ptr(), _ptr(ta),
                                              g.data_ptr(), ctypes.byref(loss)))
        return loss.value, g

    def train_step(self, dirty: torch.Tensor, target_x: torch.Tensor, target_aux: torch.Tensor | None, lr: float,
                   loss_out: torch.Tensor | None = None):
        """One Adam step; loss_out (a float64 CUDA scalar) receives the loss."""
        self._cube(dirty, "dirty")
        self._cube(target_x, "target_x")
        ta = self._aux_target(target_aux)
        if loss_out is not None and not (loss_out.is_cuda and loss_out.dtype == torch.float64):
            raise ValueError("loss_out must be a float64 CUDA tensor")
        self._check(_lib.muffin_net_train_step(self._net, dirty.data_ptr(), target_x.data_ptr(), _ptr(ta),
                                               float(lr), _ptr(loss_out)))

    def check(self):
        """Wait for the stream; raise MuffinError(TIMEOUT) if a tensor-core wait gave up
        since the last check (the parameter updates queued after it were dropped)."""
        self._check(_lib.muffin_net_check(self._net))

    def close(self):
        if getattr(self, "_net", None) is not None and self._net.value:
            _lib.muffin_net_destroy(self._net)
            self._net = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


# ---------------------------------------------------------------- single 32 -> 32 layers

def _scratch(nz, ny, nx) -> torch.Tensor:
    return torch.empty(int(_lib.muffin_conv3d_scratch_bytes(nz, ny, nx)), dtype=torch.uint8, device="cuda")


def _layer_check(r: int):
    if r != 0:
        raise _m.MuffinError(r, _lib.muffin_conv3d_last_error().decode())


def conv3d_forward(a: torch.Tensor, w: torch.Tensor, b: torch.Tensor | None, relu: bool) -> torch.Tensor:
    """z = act(conv(a, w) + b); a bfloat16 [nz][ny][nx][32], w float32 [32][32][3][3][3]."""
    nz, ny, nx = a.shape[:3]
    _map(a, (nz, ny, nx, FEATURES), "a")
    w = _dev_f32(w.contiguous(), "w")
    if b is not None:
        b = _dev_f32(b.contiguous(), "b")
    z = torch.empty_like(a)
    s = _scratch(nz, ny, nx)
    _layer_check(_lib.muffin_conv3d_forward(a.data_ptr(), w.data_ptr(), _ptr(b), int(relu), z.data_ptr(), nz, ny,
                                            nx, s.data_ptr(), s.numel(), torch.cuda.current_stream().cuda_stream))
    return z


def conv3d_backward_data(dz: torch.Tensor, w: torch.Tensor, mask: torch.Tensor | None) -> torch.Tensor:
    """da = (mask > 0) * conv^T(dz, w)."""
    nz, ny, nx = dz.shape[:3]
    _map(dz, (nz, ny, nx, FEATURES), "dz")
    if mask is not None:
        _map(mask, (nz, ny, nx, FEATURES), "mask")
    w = _dev_f32(w.contiguous(), "w")
    da = torch.empty_like(dz)
    s = _scratch(nz, ny, nx)
    _layer_check(_lib.muffin_conv3d_backward_data(dz.data_ptr(), w.data_ptr(), _ptr(mask), da.data_ptr(), nz, ny,
                                                  nx, s.data_ptr(), s.numel(),
                                                  torch.cuda.current_stream().cuda_stream))
    return da


def conv3d_backward_weights(a: torch.Tensor, dz: torch.Tensor) -> tuple[torch.Tensor, torch.Tensor]:
    """(dw float32 [32][32][3][3][3], db float32 [32])."""
    nz, ny, nx = a.shape[:3]
    _map(a, (nz, ny, nx, FEATURES), "a")
    _map(dz, (nz, ny, nx, FEATURES), "dz")
    dw = torch.empty((FEATURES, FEATURES, 3, 3, 3), dtype=torch.float32, device="cuda")
    db = torch.empty(FEATURES, dtype=torch.float32, device="cuda")
    s = _scratch(nz, ny, nx)
    _layer_check(_lib.muffin_conv3d_backward_weights(a.data_ptr(), dz.data_ptr(), dw.data_ptr(), db.data_ptr(), nz,
                                                     ny, nx, s.data_ptr(), s.numel(),
                                                     torch.cuda.current_stream().cuda_stream))
    return dw, db


# ---------------------------------------------------------------- warm start of Algorithm 1

def warm_start(problem, net: WarmStartNet, net_input: torch.Tensor, keep_state: bool = False) -> dict:
    """Move ``problem`` (a muffin.Muffin) to the network's state.

    The network maps ``net_input`` (the dirty cube, or the cube after a few
    passes) to the cube X and, when it has J + 2 output maps, the wavelet
    dual U.  V is kept when ``keep_state`` (else 0), and so is U when the
    network does not give it.  The method's own state stays the fallback, and
    the objective decides: the prediction is kept only if the objective of
    Eqs. 5-6 is lower at the predicted X than at the current one.  Returns what was
    decided and both objectives."""
    f0, _ = problem.objective()
    x0, u0, v0, it = problem.get_state()
    if not keep_state:
        x0, u0, v0, it = torch.zeros_like(x0), torch.zeros_like(u0), torch.zeros_like(v0), 0
    x, aux = net.predict(net_input)
    u = u0
    if aux is not None:
        if aux.shape[1] != problem.u_planes:
            raise ValueError(f"network gives {aux.shape[1]} fields, the problem has {problem.u_planes} planes of U")
        u = aux
    problem.set_state(x, u, v0, it)
    f1, _ = problem.objective()
    used = f1 < f0
    if not used:
        problem.set_state(x0, u0, v0, it)
    return {"used": bool(used), "f_start": f0, "f_net": f1}


# ---------------------------------------------------------------- timing

def _time_main(argv=None) -> None:
    """Times training steps and predictions of the network on a seeded
    synthetic cube (uniform input and targets, U targets in [-1, 1]) with CUDA
    events on the current stream after warm-up, and prints one JSON line."""
    import argparse
    import json

    from . import synth

    ap = argparse.ArgumentParser(prog="python -m paper_1602_08847_gb300.net")
    ap.add_argument("--shape", type=int, nargs=3, default=[64, 256, 256], metavar=("NZ", "NY", "NX"))
    ap.add_argument("--n-out", type=int, default=6)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    args = ap.parse_args(argv)
    shape, k = tuple(args.shape), args.n_out
    g = torch.Generator(device="cuda").manual_seed(0)
    y = torch.rand(shape, device="cuda", generator=g)
    tx = torch.rand(shape, device="cuda", generator=g)
    tu = None
    if k > 1:
        tu = (torch.rand((shape[0], k - 1) + shape[1:], device="cuda", generator=g) * 2 - 1).to(torch.bfloat16)
    theta = torch.from_numpy(synth.net_init(0, k)).cuda()
    weights = [1000.0] + [4.0] + [1.0] * (k - 2) if k > 1 else [1.0]
    tr = WarmStartNet(shape, training=True, theta=theta, n_out=k, out_weight=weights)
    inf = WarmStartNet(shape, theta=theta, n_out=k)
    for _ in range(args.warmup):
        tr.train_step(y, tx, tu, 1e-3)
        inf.predict(y)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    for _ in range(args.reps):
        tr.train_step(y, tx, tu, 1e-3)
    ev[1].record()
    for _ in range(args.reps):
        inf.predict(y)
    ev[2].record()
    torch.cuda.synchronize()
    print(json.dumps({"shape": list(shape), "n_out": k, "reps": args.reps,
                      "train_step_ms": ev[0].elapsed_time(ev[1]) / max(args.reps, 1),
                      "predict_ms": ev[1].elapsed_time(ev[2]) / max(args.reps, 1),
                      "wait_timeouts": wait_timeouts()}))


if __name__ == "__main__":
    _time_main()

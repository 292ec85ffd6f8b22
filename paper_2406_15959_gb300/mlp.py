"""Python binding of the learned interface warm start (include/elm_mlp.h): argument
marshalling only; forward, backward and Adam run in the library's CUDA kernels (the layers'
products on the tensor cores at FP32 accuracy)."""
from __future__ import annotations

import ctypes

from . import elm_ddm as _E

SYMBOLS = ("elm_mlp_create", "elm_mlp_param_count", "elm_mlp_get_params", "elm_mlp_set_params",
           "elm_mlp_forward", "elm_mlp_gradient", "elm_mlp_train_step", "elm_mlp_check",
           "elm_mlp_destroy", "elm_mlp_last_error")

_bound = False


def _lib():
    global _bound
    lib = _E.load()
    if not _bound:
        P, I = ctypes.c_void_p, ctypes.c_int
        lib.elm_mlp_create.argtypes = [I, I, I, I, ctypes.c_uint64, P, ctypes.POINTER(P)]
        lib.elm_mlp_param_count.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
        lib.elm_mlp_get_params.argtypes = [P, P]
        lib.elm_mlp_set_params.argtypes = [P, P]
        lib.elm_mlp_forward.argtypes = [P, P, I, P]
        lib.elm_mlp_gradient.argtypes = [P, P, P, I, P, P]
        lib.elm_mlp_train_step.argtypes = [P, P, P, I, ctypes.c_float, P]
        lib.elm_mlp_check.argtypes = [P]
        lib.elm_mlp_destroy.argtypes = [P]
        lib.elm_mlp_last_error.argtypes = [P]
        lib.elm_mlp_last_error.restype = ctypes.c_char_p
        for name in SYMBOLS[:-1]:
            getattr(lib, name).restype = ctypes.c_int
        _bound = True
    return lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class MLP:
    """d_in -> d_hidden -> d_hidden -> d_out with GELU, FP32 (products at FP32 accuracy on the
    tensor cores), on one CUDA stream."""

    def __init__(self, d_in: int, d_hidden: int, d_out: int, max_batch: int, seed: int = 0, stream=None):
        import torch
        self.lib = _lib()
        self.d_in, self.d_hidden, self.d_out, self.max_batch = d_in, d_hidden, d_out, max_batch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        rc = self.lib.elm_mlp_create(d_in, d_hidden, d_out, max_batch, seed,
                                     ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if rc != _E.OK:
            raise _E.ElmDdmError(rc, self.lib.elm_mlp_last_error(None).decode())
        self.h = h
        n = ctypes.c_int64()
        self._rc(self.lib.elm_mlp_param_count(self.h, ctypes.byref(n)))
        self.n_params = n.value
        self._loss = torch.zeros(1, dtype=torch.float32, device="cuda")

    def _rc(self, rc):
        if rc != _E.OK:
            raise _E.ElmDdmError(rc, self.lib.elm_mlp_last_error(self.h).decode())

    def params(self):
        import torch
        out = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        self._rc(self.lib.elm_mlp_get_params(self.h, _ptr(out)))
        return out

    def set_params(self, p):
        self._rc(self.lib.elm_mlp_set_params(self.h, _ptr(p.contiguous())))

    def forward(self, x):
        import torch
        y = torch.empty((x.shape[0], self.d_out), dtype=torch.float32, device=x.device)
        self._rc(self.lib.elm_mlp_forward(self.h, _ptr(x.contiguous()), x.shape[0], _ptr(y)))
        return y

    def gradient(self, x, target):
        """(loss, gradient in the parameter layout) without an update."""
        import torch
        g = torch.empty(self.n_params, dtype=torch.float32, device=x.device)
        self._rc(self.lib.elm_mlp_gradient(self.h, _ptr(x.contiguous()), _ptr(target.contiguous()),
                                           x.shape[0], _ptr(self._loss), _ptr(g)))
        return self._loss.clone(), g

    def train_step(self, x, target, lr: float):
        """One Adam step; returns the batch loss (device tensor) before the update."""
        self._rc(self.lib.elm_mlp_train_step(self.h, _ptr(x), _ptr(target), x.shape[0], float(lr),
                                             _ptr(self._loss)))
        return self._loss

    def check(self):
        """Synchronise; raise if a bounded wait of a GEMM kernel gave up since the last check."""
        self._rc(self.lib.elm_mlp_check(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.elm_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

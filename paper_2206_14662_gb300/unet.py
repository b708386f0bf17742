"""Binding of the learned field-solve warm start (pic_unet_* in
include/pic.h): argument marshalling only; every step runs in libpic's
kernels.  Device arrays are torch CUDA tensors (float32, contiguous)."""
from __future__ import annotations

import ctypes

import numpy as np

from ._capi import PicAllocator, _check, _torch_allocator, lib

c_i64 = ctypes.c_int64
vp = ctypes.c_void_p


def _sig():
    L = lib()
    if getattr(L, "_unet_sig", False):
        return L
    P = ctypes.POINTER
    L.pic_unet_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, vp, P(PicAllocator), P(vp)]
    L.pic_unet_free.argtypes = [vp]
    L.pic_unet_free.restype = None
    L.pic_unet_param_count.argtypes = [vp]
    L.pic_unet_param_count.restype = c_i64
    for name in ("pic_unet_set_params", "pic_unet_get_params", "pic_unet_get_grads"):
        getattr(L, name).argtypes = [vp, vp]
    L.pic_unet_forward.argtypes = [vp, vp, vp]
    L.pic_unet_backward.argtypes = [vp, vp, vp]
    L.pic_unet_train_step.argtypes = [vp, vp, vp, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                      ctypes.c_float, c_i64, vp]
    L._unet_sig = True
    return L


def _dev(t):
    import torch
    assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
    return vp(t.data_ptr())


class UNet:
    """One pic_unet: ``precision`` 16 (BF16 tensor cores) or 32 (FP32 test
    mode)."""

    def __init__(self, base_channels: int, H: int, W: int, batch: int, precision: int = 16,
                 stream=None):
        import torch
        L = _sig()
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = int(stream)
        self.shape = (batch, H, W)
        al, self._keep = _torch_allocator()
        self._alloc = al
        h = vp()
        _check(L.pic_unet_create(base_channels, H, W, batch, precision, vp(self.stream),
                                 ctypes.byref(self._alloc), ctypes.byref(h)), "pic_unet_create")
        self.h = h
        self.n_params = int(L.pic_unet_param_count(h))
        self.t = 0

    def close(self):
        if getattr(self, "h", None):
            lib().pic_unet_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.size == self.n_params
        _check(_sig().pic_unet_set_params(self.h, a.ctypes.data_as(vp)), "pic_unet_set_params")
        self.t = 0

    def set_tensor_path(self, mode: int):
        """pic_unet_set_tensor_path: -1 automatic, 0 mma.sync only, 1 the
        tcgen05 kernel wherever the shape allows."""
        L = lib()
        L.pic_unet_set_tensor_path.argtypes = [vp, ctypes.c_int]
        _check(L.pic_unet_set_tensor_path(self.h, int(mode)), "pic_unet_set_tensor_path")

    def get_params(self) -> np.ndarray:
        a = np.zeros(self.n_params, dtype=np.float32)
        _check(_sig().pic_unet_get_params(self.h, a.ctypes.data_as(vp)), "pic_unet_get_params")
        return a

    def get_grads(self) -> np.ndarray:
        a = np.zeros(self.n_params, dtype=np.float32)
        _check(_sig().pic_unet_get_grads(self.h, a.ctypes.data_as(vp)), "pic_unet_get_grads")
        return a

    def forward(self, x, y=None):
        import torch
        if y is None:
            y = torch.empty(self.shape, dtype=torch.float32, device=x.device)
        _check(_sig().pic_unet_forward(self.h, _dev(x), _dev(y)), "pic_unet_forward")
        return y

    def backward(self, gy, gx=None):
        _check(_sig().pic_unet_backward(self.h, _dev(gy), _dev(gx) if gx is not None else None),
               "pic_unet_backward")
        return gx

    def train_step(self, x, target, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, loss=None):
        self.t += 1
        _check(_sig().pic_unet_train_step(self.h, _dev(x), _dev(target), lr, beta1, beta2, eps,
                                          self.t, _dev(loss) if loss is not None else None),
               "pic_unet_train_step")

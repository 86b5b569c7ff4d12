"""Python binding of libkct_conv (include/kct_conv.h): tensor-core 3x3x3 convolutions for the
learned CGLS warm start, and a torch.autograd.Function built on them.

Activations are channels-last bf16 tensors [n, d, h, w, c]; weights are kept as float32
master copies [cout, 27, cin] and cast to bf16 for each call. Every convolution (forward,
input gradient, weight gradient) runs in libkct_conv; torch only provides memory, the
layout copies the weight gradient needs and the elementwise glue.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkct_conv.so")

_lib = None
_err = {}


class ConvDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("d", ctypes.c_int32), ("h", ctypes.c_int32), ("w", ctypes.c_int32),
                ("cin", ctypes.c_int32), ("cout", ctypes.c_int32)]


def load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libkct_conv.so not built ({LIB_PATH}); run `python -m paper_2110_09841_b300.build`")
        lib = ctypes.CDLL(LIB_PATH)
        V, I32 = ctypes.c_void_p, ctypes.c_int32
        lib.kct_conv3d_fwd.argtypes = [ctypes.POINTER(ConvDesc), V, V, V, V, I32, V, V]
        lib.kct_conv3d_fwd.restype = ctypes.c_int
        lib.kct_conv3d_wgrad.argtypes = [ctypes.POINTER(ConvDesc), V, V, V, V, V, V, V]
        lib.kct_conv3d_wgrad.restype = ctypes.c_int
        lib.kct_conv_last_error.argtypes = []
        lib.kct_conv_last_error.restype = ctypes.c_char_p
        _lib = lib
    return _lib


def err_word(device) -> torch.Tensor:
    """The device error word the convolution kernels set when a bounded wait runs out."""
    key = torch.device(device).index or 0
    if key not in _err:
        _err[key] = torch.zeros(1, dtype=torch.int32, device=device)
    return _err[key]


def _check(rc):
    if rc != 0:
        raise RuntimeError(f"libkct_conv status {rc}: {load().kct_conv_last_error().decode()}")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def conv3d_fwd(x: torch.Tensor, w: torch.Tensor, bias: torch.Tensor | None = None, relu: bool = False):
    """y = conv(x, w) + bias (then ReLU). x [n, d, h, w, cin] bf16, w [cout, 27, cin] bf16."""
    n, d, h, wd, cin = x.shape
    cout = w.shape[0]
    assert x.dtype == torch.bfloat16 and w.dtype == torch.bfloat16 and x.is_contiguous() and w.is_contiguous()
    assert w.shape == (cout, 27, cin)
    y = torch.empty((n, d, h, wd, cout), dtype=torch.bfloat16, device=x.device)
    desc = ConvDesc(n, d, h, wd, cin, cout)
    b = None if bias is None else bias.contiguous().float()
    _check(load().kct_conv3d_fwd(ctypes.byref(desc), _ptr(x), _ptr(w), _ptr(b), _ptr(y), int(relu),
                                 _ptr(err_word(x.device)), _stream()))
    return y


def flip_transpose(w: torch.Tensor) -> torch.Tensor:
    """Weights of the input gradient: w'[ci][26 - t][co] = w[co][t][ci]."""
    return w.flip(1).transpose(0, 2).contiguous()


def conv3d_dgrad(gy: torch.Tensor, w: torch.Tensor):
    """Gradient with respect to the input of y = conv(x, w): a convolution of gy."""
    return conv3d_fwd(gy.contiguous(), flip_transpose(w))


def conv3d_wgrad(x: torch.Tensor, gy: torch.Tensor) -> torch.Tensor:
    """gw[co][t][ci] = sum_v gy[v][co] x[v + offset(t)][ci] (float32)."""
    n, d, h, wd, cin = x.shape
    cout = gy.shape[-1]
    gt = gy.permute(0, 4, 1, 2, 3).contiguous()
    xp = torch.nn.functional.pad(x, (0, 0, 1, 1))                      # zero column on both sides of x
    xt = [xp[:, :, :, k:k + wd, :].permute(0, 4, 1, 2, 3).contiguous() for k in range(3)]
    gw = torch.empty((cout, 27, cin), dtype=torch.float32, device=x.device)
    desc = ConvDesc(n, d, h, wd, cin, cout)
    _check(load().kct_conv3d_wgrad(ctypes.byref(desc), _ptr(gt), _ptr(xt[0]), _ptr(xt[1]), _ptr(xt[2]), _ptr(gw),
                                   _ptr(err_word(x.device)), _stream()))
    return gw


class Conv3dFn(torch.autograd.Function):
    """relu(conv(x, w) + b) (or without ReLU) with x channels-last bf16 and float32 master
    weights w [cout, 27, cin], b [cout]; gradients by the tensor-core kernels."""

    @staticmethod
    def forward(ctx, x, w, b, relu):
        wb = w.to(torch.bfloat16).contiguous()
        y = conv3d_fwd(x.contiguous(), wb, b, relu)
        ctx.save_for_backward(x, wb, y if relu else None)
        ctx.relu = relu
        return y

    @staticmethod
    def backward(ctx, gy):
        x, wb, y = ctx.saved_tensors
        g = gy.to(torch.bfloat16)
        if ctx.relu:
            g = g * (y > 0).to(g.dtype)
        g = g.contiguous()
        gx = conv3d_dgrad(g, wb) if ctx.needs_input_grad[0] else None
        gw = conv3d_wgrad(x.contiguous(), g) if ctx.needs_input_grad[1] else None
        gb = g.float().sum(dim=(0, 1, 2, 3)) if ctx.needs_input_grad[2] else None
        return gx, gw, gb, None


def conv3d(x, w, b, relu=True):
    return Conv3dFn.apply(x, w, b, relu)

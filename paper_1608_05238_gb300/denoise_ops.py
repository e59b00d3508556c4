"""Binding of the denoiser kernels (include/mcr_denoise.h): argument marshalling only.

Tensors are torch CUDA tensors; activations NHWC bf16 with a channel stride padded to a multiple
of 64, weights [n_pad][taps][cin_pad] bf16.  No CPU fallback: missing library or GPU raises.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import mcr

_bound = False


class _ConvDesc(C.Structure):
    _fields_ = [("B", C.c_int32), ("H", C.c_int32), ("W", C.c_int32), ("cin_pad", C.c_int32), ("x", C.c_void_p),
                ("taps", C.c_int32), ("cout", C.c_int32), ("n_pad", C.c_int32), ("w", C.c_void_p),
                ("bias", C.c_void_p), ("relu", C.c_int32), ("mask", C.c_void_p), ("mask_stride", C.c_int32),
                ("mask_off", C.c_int32), ("out", C.c_void_p), ("out_f32", C.c_int32), ("out_stride", C.c_int32),
                ("out_off", C.c_int32)]


EXPORTS = ("dn_conv", "dn_check")


def lib():
    global _bound
    L = mcr.load()
    if not _bound:
        L.dn_conv.argtypes = [C.POINTER(_ConvDesc), C.c_void_p]
        L.dn_conv.restype = C.c_int
        L.dn_check.argtypes = [C.c_void_p]
        L.dn_check.restype = C.c_int
        _bound = True
    return L


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def conv(x: torch.Tensor, w: torch.Tensor, cout: int, out: torch.Tensor, *, taps: int = 9, bias=None,
         relu: bool = False, mask: torch.Tensor | None = None, mask_off: int = 0, out_off: int = 0, stream=None):
    """out[..., out_off:out_off+cout] = epilogue(conv(x, w)) on the tensor cores (``dn_conv``).

    x: [B, H, W, cin_pad] bf16; w: [n_pad, taps, cin_pad] bf16; out: [B, H, W, out_stride] bf16 or
    fp32; mask (optional, bf16 NHWC): zero the outputs where mask[..., mask_off + n] <= 0.
    """
    assert x.is_cuda and x.dtype == torch.bfloat16 and x.is_contiguous() and x.dim() == 4
    assert w.is_cuda and w.dtype == torch.bfloat16 and w.is_contiguous() and w.shape[1] == taps
    assert out.is_cuda and out.is_contiguous() and out.dtype in (torch.bfloat16, torch.float32)
    B, H, W, cin_pad = x.shape
    assert w.shape[2] == cin_pad and out.shape[:3] == x.shape[:3]
    if bias is not None:
        assert bias.is_cuda and bias.dtype == torch.float32 and bias.is_contiguous()
    if mask is not None:
        assert mask.is_cuda and mask.dtype == torch.bfloat16 and mask.shape[:3] == x.shape[:3]
    d = _ConvDesc(B, H, W, cin_pad, x.data_ptr(), taps, cout, w.shape[0], w.data_ptr(),
                  bias.data_ptr() if bias is not None else None, 1 if relu else 0,
                  mask.data_ptr() if mask is not None else None, mask.shape[3] if mask is not None else 0, mask_off,
                  out.data_ptr(), 1 if out.dtype == torch.float32 else 0, out.shape[3], out_off)
    rc = lib().dn_conv(C.byref(d), _stream(stream))
    if rc != 0:
        raise mcr.McrError(rc, "dn_conv")
    return out


def check(stream=None):
    rc = lib().dn_check(_stream(stream))
    if rc != 0:
        raise mcr.McrError(rc, "dn_check (a tensor-core kernel gave up waiting)")

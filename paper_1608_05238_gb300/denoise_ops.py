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
                ("out_off", C.c_int32), ("cin", C.c_int32)]


class _HeadDesc(C.Structure):
    _fields_ = [("mode", C.c_int32), ("res", C.c_void_p), ("res_stride", C.c_int32), ("scale", C.c_void_p),
                ("pred", C.c_void_p), ("target", C.c_void_p), ("dout", C.c_void_p), ("dout_stride", C.c_int32),
                ("loss", C.c_void_p)]


HEAD_PREDICT, HEAD_LOSS = 1, 2


class _AdamLayer(C.Structure):
    _fields_ = [("w", C.c_void_p), ("m", C.c_void_p), ("v", C.c_void_p), ("g", C.c_void_p), ("wf", C.c_void_p),
                ("cin_pad", C.c_int32), ("wd", C.c_void_p), ("cout_pad", C.c_int32), ("cout", C.c_int32),
                ("taps", C.c_int32), ("cin", C.c_int32), ("b", C.c_void_p), ("mb", C.c_void_p), ("vb", C.c_void_p),
                ("gb", C.c_void_p)]


class _Slice(C.Structure):
    _fields_ = [("data", C.c_void_p), ("stride", C.c_int32), ("off", C.c_int32)]


EXPORTS = ("dn_conv", "dn_conv_head", "dn_wgrad", "dn_wgrad_nhwc", "dn_wgrad_bias_nhwc", "dn_to_ct", "dn_pool2", "dn_pool2_bwd", "dn_up2", "dn_up2_bwd", "dn_bias_grad",
           "dn_mse", "dn_residual", "dn_adam", "dn_adam_bias", "dn_adam_multi", "dn_pack_input", "dn_sample_scale", "dn_pack_target", "dn_predict_output",
           "dn_unpack_output", "dn_check")


def lib():
    global _bound
    L = mcr.load()
    if not _bound:
        vp, i32, i64, f32 = C.c_void_p, C.c_int32, C.c_int64, C.c_float
        S = _Slice
        sig = {
            "dn_conv": [C.POINTER(_ConvDesc), vp],
            "dn_conv_head": [C.POINTER(_ConvDesc), C.POINTER(_HeadDesc), vp],
            "dn_wgrad": [i32, i32, i32, i32, i32, i32, vp, vp, vp, vp],
            "dn_wgrad_nhwc": [S, S, i32, i32, i32, i32, i32, i32, vp, vp],
            "dn_wgrad_bias_nhwc": [S, S, i32, i32, i32, i32, i32, i32, vp, vp, vp],
            "dn_to_ct": [S, i32, i32, i32, i32, i32, vp, vp],
            "dn_pool2": [S, i32, i32, i32, i32, S, vp],
            "dn_pool2_bwd": [S, S, S, i32, i32, i32, i32, S, vp],
            "dn_up2": [S, i32, i32, i32, i32, S, vp],
            "dn_up2_bwd": [S, S, i32, i32, i32, i32, S, vp],
            "dn_bias_grad": [S, i64, i32, vp, vp],
            "dn_mse": [vp, i32, vp, i32, vp, i64, i32, vp, i32, vp, vp],
            "dn_residual": [vp, i32, vp, i32, i64, i32, vp, vp],
            "dn_adam": [vp, vp, vp, vp, i32, i32, i32, f32, f32, f32, f32, i32, vp, i32, vp, i32, vp],
            "dn_adam_bias": [vp, vp, vp, vp, i32, f32, f32, f32, f32, i32, vp],
            "dn_adam_multi": [C.POINTER(_AdamLayer), i32, f32, f32, f32, f32, i32, vp],
            "dn_pack_input": [vp, vp, i32, i64, i32, vp, i32, vp],
            "dn_sample_scale": [vp, i32, i64, i32, vp, vp],
            "dn_pack_target": [vp, vp, i32, i64, i32, vp, vp],
            "dn_unpack_output": [vp, vp, i32, i64, i32, vp, vp],
            "dn_predict_output": [vp, i32, vp, i32, vp, i32, i64, i32, vp, vp],
            "dn_check": [vp],
        }
        for name, args in sig.items():
            getattr(L, name).argtypes = args
            getattr(L, name).restype = C.c_int
        _bound = True
    return L


def _call(name, *args):
    rc = getattr(lib(), name)(*args)
    if rc != 0:
        raise mcr.McrError(rc, name)


class Act:
    """An NHWC bf16 activation slice: channels [off, off + C) of ``t`` ([B, H, W, stride])."""

    def __init__(self, t: torch.Tensor, C: int, off: int = 0):
        assert t.is_cuda and t.dtype == torch.bfloat16 and t.is_contiguous() and t.dim() == 4
        assert 0 <= off and off + C <= t.shape[3]
        self.t, self.C, self.off = t, C, off

    @property
    def B(self):
        return self.t.shape[0]

    @property
    def H(self):
        return self.t.shape[1]

    @property
    def W(self):
        return self.t.shape[2]

    def s(self) -> _Slice:
        return _Slice(self.t.data_ptr(), self.t.shape[3], self.off)


def _null_slice() -> _Slice:
    return _Slice(None, 1, 0)


def wgrad(dzT: torch.Tensor, xT: torch.Tensor, B, H, W, taps, cout, cin, dw: torch.Tensor, stream=None):
    """dw [cout][taps][cin] += weight gradient from dz^T [cout][B][HW] and x^T copies [3][cin][B][HW]."""
    assert dzT.dtype == torch.bfloat16 and xT.dtype == torch.bfloat16 and dw.dtype == torch.float32
    assert dzT.numel() >= cout * B * H * W and xT.numel() >= 3 * cin * B * H * W and dw.numel() >= cout * taps * cin
    _call("dn_wgrad", B, H, W, taps, cout, cin, _p(dzT), _p(xT), _p(dw), _stream(stream))


def wgrad_nhwc(dz: Act, x: Act, taps: int, dw: torch.Tensor, db: torch.Tensor | None = None, stream=None):
    """dw[n][tap][c] += sum over pixels of dz[p][n] x[p + tap][c], read from the NHWC slices; with
    ``db`` also the bias gradient db[n] += sum over pixels of dz[p][n] (``dn_wgrad_bias_nhwc``)."""
    if db is None:
        _call("dn_wgrad_nhwc", dz.s(), x.s(), x.B, x.H, x.W, taps, dz.C, x.C, _p(dw), _stream(stream))
    else:
        assert db.is_cuda and db.dtype == torch.float32 and db.numel() >= dz.C
        _call("dn_wgrad_bias_nhwc", dz.s(), x.s(), x.B, x.H, x.W, taps, dz.C, x.C, _p(dw), _p(db), _stream(stream))


def to_ct(src: Act, shifted: bool, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    n = (3 if shifted else 1) * src.C * src.B * src.H * src.W
    if out is None:
        out = torch.empty(n, dtype=torch.bfloat16, device=src.t.device)
    assert out.numel() >= n and out.dtype == torch.bfloat16
    _call("dn_to_ct", src.s(), src.B, src.H, src.W, src.C, 1 if shifted else 0, _p(out), _stream(stream))
    return out


def pool2(src: Act, dst: Act, stream=None):
    _call("dn_pool2", src.s(), src.B, src.H, src.W, src.C, dst.s(), _stream(stream))


def pool2_bwd(dp: Act, skip: Act | None, act: Act, dz: Act, stream=None):
    _call("dn_pool2_bwd", dp.s(), skip.s() if skip is not None else _null_slice(), act.s(), act.B, act.H, act.W,
          act.C, dz.s(), _stream(stream))


def up2(src: Act, dst: Act, stream=None):
    _call("dn_up2", src.s(), src.B, src.H, src.W, src.C, dst.s(), _stream(stream))


def up2_bwd(du: Act, act: Act, dz: Act, stream=None):
    _call("dn_up2_bwd", du.s(), act.s(), act.B, act.H, act.W, act.C, dz.s(), _stream(stream))


def bias_grad(dz: Act, db: torch.Tensor, stream=None):
    _call("dn_bias_grad", dz.s(), dz.B * dz.H * dz.W, dz.C, _p(db), _stream(stream))


def mse(out: torch.Tensor, x: torch.Tensor, t: torch.Tensor, C: int, dout: torch.Tensor, loss: torch.Tensor,
        stream=None):
    P = out.shape[0] * out.shape[1] * out.shape[2]
    _call("dn_mse", _p(out), out.shape[3], _p(x), x.shape[3], _p(t), P, C, _p(dout), dout.shape[3], _p(loss),
          _stream(stream))


def residual(out: torch.Tensor, x: torch.Tensor, C: int, y: torch.Tensor, stream=None):
    P = out.shape[0] * out.shape[1] * out.shape[2]
    _call("dn_residual", _p(out), out.shape[3], _p(x), x.shape[3], P, C, _p(y), _stream(stream))


def adam(w, m, v, g, cout, taps, cin, lr, b1, b2, eps, step, wf, cin_pad, wd=None, cout_pad=0, stream=None):
    _call("dn_adam", _p(w), _p(m), _p(v), _p(g), cout, taps, cin, lr, b1, b2, eps, step, _p(wf), cin_pad, _p(wd),
          cout_pad, _stream(stream))


def adam_bias(b, m, v, g, lr, b1, b2, eps, step, stream=None):
    _call("dn_adam_bias", _p(b), _p(m), _p(v), _p(g), b.numel(), lr, b1, b2, eps, step, _stream(stream))


def adam_table(layers):
    """Descriptors of dn_adam_multi from tuples (w, m, v, g, wf, cin_pad, wd, cout_pad, cout, taps, cin,
    b, mb, vb, gb) of tensors / ints (wd, b may be None).  The tensors must outlive the table."""
    arr = (_AdamLayer * len(layers))()
    for i, (w, m, v, g, wf, cin_pad, wd, cout_pad, cout, taps, cin, b, mb, vb, gb) in enumerate(layers):
        arr[i] = _AdamLayer(w.data_ptr(), m.data_ptr(), v.data_ptr(), g.data_ptr(), wf.data_ptr(), cin_pad,
                            None if wd is None else wd.data_ptr(), cout_pad, cout, taps, cin,
                            None if b is None else b.data_ptr(), None if mb is None else mb.data_ptr(),
                            None if vb is None else vb.data_ptr(), None if gb is None else gb.data_ptr())
    return arr


def adam_multi(table, lr, b1, b2, eps, step, stream=None):
    """Every layer of ``table`` (``adam_table``) stepped in one launch (``dn_adam_multi``)."""
    _call("dn_adam_multi", table, len(table), lr, b1, b2, eps, step, _stream(stream))


def pack_input(src: torch.Tensor, scale: torch.Tensor, dst: torch.Tensor, stream=None):
    B, Cc = src.shape[0], src.shape[1]
    _call("dn_pack_input", _p(src), _p(scale), B, src.shape[2] * src.shape[3], Cc, _p(dst), dst.shape[3],
          _stream(stream))


def sample_scale(src: torch.Tensor, scale: torch.Tensor, stream=None):
    """scale[b] = 1 / mean |channel 0| of the channel-major fp32 maps src [B][C][H][W] (the mean
    fluence of forward maps; for the signed adjoint maps the mean magnitude of a_0*)."""
    _call("dn_sample_scale", _p(src), src.shape[0], src.shape[2] * src.shape[3], src.shape[1], _p(scale),
          _stream(stream))


def predict_output(out: torch.Tensor, x: torch.Tensor, C: int, scale: torch.Tensor, dst: torch.Tensor, stream=None):
    """dst [B][C][H][W] = (x[..., :C] + out[..., :C]) / scale[b] from the NHWC network output and input."""
    B, H, W = x.shape[:3]
    _call("dn_predict_output", _p(out), out.shape[3], _p(x), x.shape[3], _p(scale), B, H * W, C, _p(dst),
          _stream(stream))


def pack_target(src: torch.Tensor, scale: torch.Tensor, dst: torch.Tensor, stream=None):
    B, Cc = src.shape[0], src.shape[1]
    _call("dn_pack_target", _p(src), _p(scale), B, src.shape[2] * src.shape[3], Cc, _p(dst), _stream(stream))


def unpack_output(src: torch.Tensor, scale: torch.Tensor, dst: torch.Tensor, stream=None):
    B, Cc = dst.shape[0], dst.shape[1]
    _call("dn_unpack_output", _p(src), _p(scale), B, dst.shape[2] * dst.shape[3], Cc, _p(dst), _stream(stream))


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def conv(x: torch.Tensor, w: torch.Tensor, cout: int, out: torch.Tensor, *, taps: int = 9, bias=None,
         relu: bool = False, mask: torch.Tensor | None = None, mask_off: int = 0, out_off: int = 0,
         cin: int = 0, stream=None):
    """out[..., out_off:out_off+cout] = epilogue(conv(x, w)) on the tensor cores (``dn_conv``).

    x: [B, H, W, cin_pad] bf16; w: [n_pad, taps, cin_pad] bf16; out: [B, H, W, out_stride] bf16 or
    fp32; mask (optional, bf16 NHWC): zero the outputs where mask[..., mask_off + n] <= 0; cin: the
    input channels that hold data (0: all), the rest taken as zero.
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
                  out.data_ptr(), 1 if out.dtype == torch.float32 else 0, out.shape[3], out_off, cin)
    rc = lib().dn_conv(C.byref(d), _stream(stream))
    if rc != 0:
        raise mcr.McrError(rc, "dn_conv")
    return out


def conv_head(x: torch.Tensor, w: torch.Tensor, cout: int, bias, res: torch.Tensor, scale: torch.Tensor, *,
              pred: torch.Tensor | None = None, target: torch.Tensor | None = None, dout: torch.Tensor | None = None,
              loss: torch.Tensor | None = None, stream=None):
    """The 1x1 output layer with the residual head fused into its epilogue (``dn_conv_head``).

    With ``pred`` ([B][cout][H][W] fp32): pred = (res + conv(x, w) + bias) / scale.  With ``target``
    ([B][cout][H][W] fp32, unscaled), ``dout`` (bf16 NHWC) and ``loss`` (FP64 scalar): the residual MSE
    against scale * target and its gradient seed.
    """
    assert x.is_cuda and x.dtype == torch.bfloat16 and x.is_contiguous() and x.dim() == 4
    assert w.is_cuda and w.dtype == torch.bfloat16 and w.is_contiguous() and w.shape[1] == 1
    assert res.is_cuda and res.dtype == torch.bfloat16 and res.is_contiguous() and res.shape[:3] == x.shape[:3]
    assert scale.is_cuda and scale.dtype == torch.float32 and scale.numel() == x.shape[0]
    B, H, W, cin_pad = x.shape
    assert w.shape[2] == cin_pad
    if bias is not None:
        assert bias.is_cuda and bias.dtype == torch.float32 and bias.is_contiguous()
    if pred is not None:
        assert pred.is_cuda and pred.dtype == torch.float32 and pred.is_contiguous()
        assert tuple(pred.shape) == (B, cout, H, W)
        h = _HeadDesc(HEAD_PREDICT, res.data_ptr(), res.shape[3], scale.data_ptr(), pred.data_ptr(), None, None, 0, None)
    else:
        assert target is not None and dout is not None and loss is not None
        assert target.is_cuda and target.dtype == torch.float32 and target.is_contiguous()
        assert tuple(target.shape) == (B, cout, H, W)
        assert dout.is_cuda and dout.dtype == torch.bfloat16 and dout.is_contiguous() and dout.shape[:3] == x.shape[:3]
        assert loss.is_cuda and loss.dtype == torch.float64
        h = _HeadDesc(HEAD_LOSS, res.data_ptr(), res.shape[3], scale.data_ptr(), None, target.data_ptr(),
                      dout.data_ptr(), dout.shape[3], loss.data_ptr())
    d = _ConvDesc(B, H, W, cin_pad, x.data_ptr(), 1, cout, w.shape[0], w.data_ptr(),
                  bias.data_ptr() if bias is not None else None, 0, None, 0, 0, None, 0, 0, 0)
    rc = lib().dn_conv_head(C.byref(d), C.byref(h), _stream(stream))
    if rc != 0:
        raise mcr.McrError(rc, "dn_conv_head")


def wait_probe(spins: int, stream=None) -> bool:
    """``dn_wait_probe``: the tensor-core kernels' bounded mbarrier wait, limited to ``spins`` polls, on
    a barrier nothing arrives at; True when it gave up (and latched the error dn_check reports)."""
    out = C.c_int32(-1)
    L = lib()
    L.dn_wait_probe.argtypes = [C.c_uint32, C.POINTER(C.c_int32), C.c_void_p]
    L.dn_wait_probe.restype = C.c_int
    rc = L.dn_wait_probe(int(spins), C.byref(out), _stream(stream))
    if rc != 0:
        raise mcr.McrError(rc, "dn_wait_probe")
    return out.value == 1


def check(stream=None):
    rc = lib().dn_check(_stream(stream))
    if rc != 0:
        raise mcr.McrError(rc, "dn_check (a tensor-core kernel gave up waiting)")

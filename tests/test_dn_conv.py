"""Tensor-core convolution (dn_conv) against a plain PyTorch CPU convolution of the same bf16 data."""
import numpy as np
import pytest
import torch
import torch.nn.functional as Fnn

from paper_1608_05238_gb300 import _build, denoise_ops as ops, mcr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    ops.lib()


def _ref(x, w, cin, cout, taps, bias=None, relu=False, mask=None, mask_off=0):
    """CPU fp64 reference: NHWC bf16 input / [n_pad][taps][cin_pad] weights -> NHWC fp64."""
    xc = x.double().cpu()[..., :cin].permute(0, 3, 1, 2)
    k = 3 if taps == 9 else 1
    wc = w.double().cpu()[:cout, :, :cin].reshape(cout, k, k, cin).permute(0, 3, 1, 2)
    y = Fnn.conv2d(xc, wc, padding=k // 2).permute(0, 2, 3, 1)
    if bias is not None:
        y = y + bias.double().cpu()
    if relu:
        y = y.clamp_min(0)
    if mask is not None:
        y = y * (mask.double().cpu()[..., mask_off:mask_off + cout] > 0)
    return y


def _case(B, H, W, cin, cout, taps, seed, cin_pad=None, n_pad=None):
    g = torch.Generator().manual_seed(seed)
    cin_pad = cin_pad or ((cin + 63) // 64) * 64
    n_pad = n_pad or ((cout + 15) // 16) * 16
    x = torch.zeros(B, H, W, cin_pad)
    x[..., :cin] = torch.randn(B, H, W, cin, generator=g)
    w = torch.zeros(n_pad, taps, cin_pad)
    w[:cout, :, :cin] = torch.randn(cout, taps, cin, generator=g) / np.sqrt(taps * cin)
    return x.bfloat16().cuda(), w.bfloat16().cuda(), cin_pad, n_pad


@pytest.mark.parametrize("B,H,W,cin,cout,taps", [
    (1, 4, 32, 64, 16, 1),     # one tile, plain GEMM
    (2, 16, 32, 64, 32, 9),    # 3x3, several tiles of 4 rows
    (1, 2, 256, 128, 64, 9),   # rows of 256 pixels: two tiles per row, two channel blocks
    (1, 8, 64, 64, 256, 9),    # N = 256
    (3, 8, 128, 33, 48, 9),    # padded input channels
    (1, 12, 32, 64, 128, 9),   # three 128-pixel tiles: no 256-pixel pairing
    (2, 4, 32, 64, 96, 9),     # a 256-pixel pair spanning two images
    (2, 5, 128, 64, 32, 9),    # odd image height, 256-pixel pairs over rows of 128
    (1, 3, 512, 192, 16, 9),   # rows of 512 pixels, three channel blocks, N = 16
])
def test_conv_fp32_output_matches_reference(B, H, W, cin, cout, taps):
    x, w, cin_pad, n_pad = _case(B, H, W, cin, cout, taps, seed=B * 100 + H + W + cout)
    out = torch.full((B, H, W, ((cout + 7) // 8) * 8), float("nan"), device="cuda")
    ops.conv(x, w, cout, out, taps=taps)
    ops.check()
    ref = _ref(x, w, cin, cout, taps)
    got = out[..., :cout].double().cpu()
    assert torch.allclose(got, ref, rtol=1e-4, atol=1e-4 * ref.abs().max().item())


def test_conv_bias_relu_bf16_slice_and_mask():
    B, H, W, cin, cout = 2, 8, 64, 96, 40
    x, w, cin_pad, n_pad = _case(B, H, W, cin, cout, 9, seed=7)
    bias = torch.randn(cout).cuda()
    out = torch.zeros(B, H, W, 128, dtype=torch.bfloat16, device="cuda")
    ops.conv(x, w, cout, out, bias=bias, relu=True, out_off=64)
    ref = _ref(x, w, cin, cout, 9, bias=bias, relu=True)
    got = out[..., 64:64 + cout].double().cpu()
    assert torch.allclose(got, ref, rtol=2 ** -7, atol=1e-3)
    assert torch.count_nonzero(out[..., :64]) == 0 and torch.count_nonzero(out[..., 64 + cout:]) == 0
    mask = torch.randn(B, H, W, 64).bfloat16().cuda()
    out2 = torch.zeros(B, H, W, cout + (8 - cout % 8) % 8, device="cuda")
    ops.conv(x, w, cout, out2, mask=mask, mask_off=8)
    ops.check()
    ref2 = _ref(x, w, cin, cout, 9, mask=mask, mask_off=8)
    assert torch.allclose(out2[..., :cout].double().cpu(), ref2, rtol=1e-4, atol=1e-4 * ref2.abs().max().item())


def test_wide_row_conv_bias_relu_slice_and_mask():
    """Paired 256-pixel tiles of 256-pixel rows (N <= 64) through every epilogue option."""
    B, H, W, cin, cout = 2, 6, 256, 72, 40
    x, w, cin_pad, n_pad = _case(B, H, W, cin, cout, 9, seed=17)
    bias = torch.randn(cout).cuda()
    out = torch.zeros(B, H, W, 128, dtype=torch.bfloat16, device="cuda")
    ops.conv(x, w, cout, out, bias=bias, relu=True, out_off=64)
    ref = _ref(x, w, cin, cout, 9, bias=bias, relu=True)
    assert torch.allclose(out[..., 64:64 + cout].double().cpu(), ref, rtol=2 ** -7, atol=1e-3)
    assert torch.count_nonzero(out[..., :64]) == 0 and torch.count_nonzero(out[..., 64 + cout:]) == 0
    mask = torch.randn(B, H, W, 64).bfloat16().cuda()
    out2 = torch.zeros(B, H, W, 40, device="cuda")
    ops.conv(x, w, cout, out2, mask=mask, mask_off=16)
    ops.check()
    ref2 = _ref(x, w, cin, cout, 9, mask=mask, mask_off=16)
    assert torch.allclose(out2.double().cpu(), ref2, rtol=1e-4, atol=1e-4 * ref2.abs().max().item())


def test_haloed_conv_epilogue_options():
    """Few output channels (N <= 32) on rows of 256 pixels take the haloed kernel: bias, ReLU,
    bf16 slice output and the ReLU-mask path against the reference."""
    B, H, W, cin, cout = 2, 6, 256, 72, 30
    x, w, cin_pad, n_pad = _case(B, H, W, cin, cout, 9, seed=19)
    bias = torch.randn(cout).cuda()
    out = torch.zeros(B, H, W, 128, dtype=torch.bfloat16, device="cuda")
    ops.conv(x, w, cout, out, bias=bias, relu=True, out_off=64)
    ref = _ref(x, w, cin, cout, 9, bias=bias, relu=True)
    assert torch.allclose(out[..., 64:64 + cout].double().cpu(), ref, rtol=2 ** -7, atol=1e-3)
    assert torch.count_nonzero(out[..., :64]) == 0 and torch.count_nonzero(out[..., 64 + cout:]) == 0
    mask = torch.randn(B, H, W, 64).bfloat16().cuda()
    out2 = torch.zeros(B, H, W, 32, device="cuda")
    ops.conv(x, w, cout, out2, mask=mask, mask_off=16)
    ops.check()
    ref2 = _ref(x, w, cin, cout, 9, mask=mask, mask_off=16)
    assert torch.allclose(out2[..., :cout].double().cpu(), ref2, rtol=1e-4, atol=1e-4 * ref2.abs().max().item())


@pytest.mark.parametrize("B,H,W,cin,cout,relu_mask", [(2, 5, 256, 32, 32, False), (1, 7, 128, 20, 16, True),
                                                      (3, 2, 512, 32, 30, True)])
def test_haloed_conv_on_32_channel_inputs(B, H, W, cin, cout, relu_mask):
    """An input with at most 32 channels in use (rows of 64, the rest garbage under zero weights)
    takes the 32-channel haloed kernel (64-byte rows and swizzle, two K steps per tap): same
    products as the reference on the used channels, with bias/ReLU or the mask epilogue."""
    x, w, cin_pad, n_pad = _case(B, H, W, cin, cout, 9, seed=31 + cin)
    g = torch.Generator().manual_seed(77)
    garbage = torch.randn(B, H, W, cin_pad - cin, generator=g).bfloat16().cuda()
    x = torch.cat([x[..., :cin], garbage], dim=3).contiguous()  # padded channels hold data; their weights are 0
    out = torch.zeros(B, H, W, 32, device="cuda")
    if relu_mask:
        mask = torch.randn(B, H, W, 64, generator=g).bfloat16().cuda()
        ops.conv(x, w, cout, out, mask=mask, mask_off=8, cin=cin)
        ref = _ref(x, w, cin, cout, 9, mask=mask, mask_off=8)
    else:
        bias = torch.randn(cout, generator=g).cuda()
        ops.conv(x, w, cout, out, bias=bias, relu=True, cin=cin)
        ref = _ref(x, w, cin, cout, 9, bias=bias, relu=True)
    ops.check()
    assert torch.allclose(out[..., :cout].double().cpu(), ref, rtol=1e-4, atol=1e-4 * ref.abs().max().item())
    # the full-width path on the same data (cin not given) agrees
    out64 = torch.zeros_like(out)
    if relu_mask:
        ops.conv(x, w, cout, out64, mask=mask, mask_off=8)
    else:
        ops.conv(x, w, cout, out64, bias=bias, relu=True)
    assert torch.allclose(out, out64, rtol=1e-5, atol=1e-5 * out64.abs().max().item())


def test_conv_rejects_bad_shapes():
    x, w, _, _ = _case(1, 4, 32, 64, 16, 9, seed=1)
    out = torch.zeros(1, 4, 32, 16, device="cuda")
    with pytest.raises(Exception):
        ops.conv(x[:, :, :16].contiguous(), w, 16, out[:, :, :16].contiguous())  # W < 32
    with pytest.raises(Exception):
        ops.conv(x, w, 16, torch.zeros(1, 4, 32, 12, device="cuda"))  # out stride not a multiple of 8


def test_bounded_wait_runs_out_and_the_context_stays_usable():
    """A tensor-core kernel's mbarrier wait gives up after its poll limit instead of hanging: the
    same wait, limited to 2000 polls on a barrier nothing arrives at, reports the timeout, latches
    the error that dn_check returns (once: it is cleared), and a convolution afterwards still
    computes what it should."""
    ops.check()  # a clean latch to start from
    assert ops.wait_probe(2000) is True
    with pytest.raises(mcr.McrError):
        ops.check()
    ops.check()
    x, w, cin_pad, n_pad = _case(1, 8, 64, 64, 32, 9, seed=5)
    out = torch.full((1, 8, 64, 32), float("nan"), device="cuda")
    ops.conv(x, w, 32, out, taps=9)
    ops.check()
    ref = _ref(x, w, 64, 32, 9)
    assert torch.allclose(out.double().cpu(), ref, rtol=1e-4, atol=1e-4 * ref.abs().max().item())

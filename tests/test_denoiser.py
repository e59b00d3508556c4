"""The tensor-core U-Net denoiser and its kernels against plain PyTorch CPU references."""
import numpy as np
import pytest
import torch
import torch.nn.functional as Fnn

from oracle import denoiser_ref as ref
from paper_1608_05238_gb300 import _build
from paper_1608_05238_gb300 import denoise_ops as ops
from paper_1608_05238_gb300.denoise_ops import Act
from paper_1608_05238_gb300.denoiser import UNet, r64, sample_scale

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    ops.lib()


def _nhwc(B, H, W, C, stride, seed, positive=False):
    g = torch.Generator().manual_seed(seed)
    t = torch.zeros(B, H, W, stride)
    v = torch.randn(B, H, W, C, generator=g)
    t[..., :C] = v.abs() if positive else v
    return t.bfloat16().cuda()


@pytest.mark.parametrize("B,H,W,cin,cout,taps", [(2, 16, 32, 64, 32, 9), (1, 32, 64, 96, 128, 9),
                                                 (2, 16, 16, 33, 48, 1), (1, 8, 128, 200, 256, 9)])
def test_wgrad_matches_autograd(B, H, W, cin, cout, taps):
    x = _nhwc(B, H, W, cin, r64(cin), 1)
    dz = _nhwc(B, H, W, cout, r64(cout), 2)
    dw = torch.zeros(cout, taps, cin, device="cuda")
    dzT = ops.to_ct(Act(dz, cout), False)
    xT = ops.to_ct(Act(x, cin), True)
    ops.wgrad(dzT, xT, B, H, W, taps, cout, cin, dw)
    ops.check()
    k = 3 if taps == 9 else 1
    xc = x.double().cpu()[..., :cin].permute(0, 3, 1, 2)
    w = torch.zeros(cout, cin, k, k, dtype=torch.float64, requires_grad=True)
    y = Fnn.conv2d(xc, w, padding=k // 2)
    y.backward(dz.double().cpu()[..., :cout].permute(0, 3, 1, 2))
    ref_dw = w.grad.permute(0, 2, 3, 1).reshape(cout, taps, cin)
    got = dw.double().cpu()
    assert torch.allclose(got, ref_dw, rtol=1e-4, atol=1e-4 * ref_dw.abs().max().item())


@pytest.mark.parametrize("B,H,W,cin,cout,taps,xoff,zoff", [(2, 16, 32, 64, 32, 9, 0, 0), (1, 32, 64, 96, 128, 9, 64, 0),
                                                            (2, 16, 16, 33, 48, 1, 0, 64), (1, 8, 128, 200, 256, 9, 0, 0),
                                                            (3, 4, 16, 40, 33, 9, 24, 8), (1, 64, 256, 32, 32, 9, 32, 0),
                                                            # haloed nine-tap kernel (cout <= 64, W % 64 == 0)
                                                            (2, 8, 64, 33, 32, 9, 0, 0), (1, 16, 128, 96, 64, 9, 0, 0),
                                                            (2, 4, 128, 192, 33, 9, 8, 0), (1, 3, 64, 64, 16, 9, 0, 64)])
def test_wgrad_nhwc_matches_autograd(B, H, W, cin, cout, taps, xoff, zoff):
    """The weight gradient read straight from NHWC slices (MN-major operands, tap shifts as TMA
    coordinates) equals FP64 autograd of the convolution, also for slices at channel offsets; the
    bias gradient that comes with it is the pixel sum of dz."""
    x = _nhwc(B, H, W, cin + xoff, r64(cin + xoff), 11)
    dz = _nhwc(B, H, W, cout + zoff, r64(cout + zoff), 12)
    dw = torch.zeros(cout, taps, cin, device="cuda")
    db = torch.full((cout,), 0.25, device="cuda")
    ops.wgrad_nhwc(Act(dz, cout, zoff), Act(x, cin, xoff), taps, dw, db=db)
    ops.check()
    ref_db = dz.double().cpu()[..., zoff:zoff + cout].sum(dim=(0, 1, 2)) + 0.25
    assert torch.allclose(db.cpu().double(), ref_db, rtol=1e-5, atol=1e-3), (db.cpu()[:4], ref_db[:4])
    k = 3 if taps == 9 else 1
    xc = x.double().cpu()[..., xoff:xoff + cin].permute(0, 3, 1, 2)
    w = torch.zeros(cout, cin, k, k, dtype=torch.float64, requires_grad=True)
    y = Fnn.conv2d(xc, w, padding=k // 2)
    y.backward(dz.double().cpu()[..., zoff:zoff + cout].permute(0, 3, 1, 2))
    ref_dw = w.grad.permute(0, 2, 3, 1).reshape(cout, taps, cin)
    got = dw.double().cpu()
    assert torch.allclose(got, ref_dw, rtol=1e-4, atol=1e-4 * ref_dw.abs().max().item())


@pytest.mark.parametrize("C", [40, 33])  # 16-byte vector path (C, strides, offsets multiples of 8) / scalar path
def test_layout_pool_upsample_and_backward_kernels(C):
    B, H, W = 2, 16, 32
    x = _nhwc(B, H, W, C + 48, 128, 3)
    src = Act(x, C, 48)  # a slice at channel offset 48 of rows of 128
    t = ops.to_ct(src, True)
    xs = x.float().cpu()[..., 48:48 + C]
    ct = xs.permute(3, 0, 1, 2).reshape(C, B, H * W)
    plane = C * B * H * W
    assert torch.equal(t[plane:2 * plane].float().cpu().view(C, B, H * W), ct)
    left = torch.zeros_like(xs)
    left[:, :, 1:] = xs[:, :, :-1]  # copy 0: x shifted by -1
    assert torch.equal(t[:plane].float().cpu().view(C, B, H * W), left.permute(3, 0, 1, 2).reshape(C, B, H * W))
    p = torch.zeros(B, H // 2, W // 2, 64, dtype=torch.bfloat16, device="cuda")
    ops.pool2(src, Act(p, C))
    rp = Fnn.avg_pool2d(xs.permute(0, 3, 1, 2), 2).permute(0, 2, 3, 1)
    assert torch.allclose(p[..., :C].float().cpu(), rp, rtol=2 ** -8, atol=1e-2)
    u = torch.zeros(B, H, W, 64, dtype=torch.bfloat16, device="cuda")
    ops.up2(Act(p, C), Act(u, C, 8))
    assert torch.equal(u[..., 8:8 + C].float().cpu(), Fnn.interpolate(p[..., :C].float().cpu().permute(0, 3, 1, 2),
                                                                      scale_factor=2).permute(0, 2, 3, 1))
    # backward kernels with masks
    act = _nhwc(B, H // 2, W // 2, C, 64, 4)
    du = _nhwc(B, H, W, C, 64, 5)
    dz = torch.zeros(B, H // 2, W // 2, 64, dtype=torch.bfloat16, device="cuda")
    ops.up2_bwd(Act(du, C), Act(act, C), Act(dz, C))
    r = du.float().cpu()[..., :C].reshape(B, H // 2, 2, W // 2, 2, C).sum(dim=(2, 4)) * (act.float().cpu()[..., :C] > 0)
    assert torch.allclose(dz[..., :C].float().cpu(), r, rtol=2 ** -7, atol=1e-2)
    dp = _nhwc(B, H // 2, W // 2, C, 64, 6)
    skip = _nhwc(B, H, W, C, 64, 7)
    act2 = _nhwc(B, H, W, C, 64, 8)
    dz2 = torch.zeros(B, H, W, 64, dtype=torch.bfloat16, device="cuda")
    ops.pool2_bwd(Act(dp, C), Act(skip, C), Act(act2, C), Act(dz2, C))
    r2 = (skip.float().cpu()[..., :C] + 0.25 * dp.float().cpu()[..., :C].repeat_interleave(2, 1).repeat_interleave(2, 2))
    r2 = r2 * (act2.float().cpu()[..., :C] > 0)
    assert torch.allclose(dz2[..., :C].float().cpu(), r2, rtol=2 ** -7, atol=1e-2)
    db = torch.zeros(C, device="cuda")
    ops.bias_grad(Act(skip, C), db)
    assert torch.allclose(db.cpu(), skip.float().cpu()[..., :C].sum(dim=(0, 1, 2)), rtol=1e-4, atol=1e-3)


@pytest.mark.parametrize("C,stride,off", [(32, 64, 0), (64, 192, 128), (256, 256, 0), (24, 64, 40), (33, 64, 0),
                                          (36, 40, 0), (5, 64, 58)])
def test_bias_grad_sums_every_pixel_of_the_slice(C, stride, off):
    B, H, W = 2, 64, 128
    dz = _nhwc(B, H, W, stride, stride, 30 + C)
    db = torch.full((C,), 0.5, device="cuda")
    ops.bias_grad(Act(dz, C, off), db)
    ops.check()
    ref = dz.double().cpu()[..., off:off + C].sum(dim=(0, 1, 2)) + 0.5
    assert torch.allclose(db.cpu().double(), ref, rtol=1e-5, atol=2e-3)


@pytest.mark.parametrize("B,C,H,W", [(3, 33, 32, 64), (2, 64, 16, 16), (2, 70, 8, 24), (2, 5, 6, 10)])
def test_pack_input_writes_scaled_bf16_rows(B, C, H, W):
    """NHWC bf16 rows of x * scale[b] (round to nearest even), channels >= C untouched."""
    g = torch.Generator().manual_seed(C)
    x = torch.rand(B, C, H, W, generator=g) * 3
    scale = torch.rand(B, generator=g) + 0.5
    dst = torch.full((B, H, W, r64(C)), 7.0, dtype=torch.bfloat16, device="cuda")
    ops.pack_input(x.cuda(), scale.cuda(), dst)
    ops.check()
    ref = (x * scale.view(B, 1, 1, 1)).permute(0, 2, 3, 1).bfloat16()
    assert torch.equal(dst[..., :C].cpu(), ref)
    assert bool((dst[..., C:].float() == 7.0).all())


@pytest.mark.parametrize("cout,taps,cin", [(32, 9, 33), (128, 9, 96), (33, 1, 32), (70, 9, 45)])
def test_adam_step_and_weight_copies(cout, taps, cin):
    """One Adam step (bias-corrected, step 5) on the FP32 master weights, their BF16 forward copy and
    the transposed, tap-flipped copy of the input-gradient pass: the tiled kernel (with the copy)
    and the flat one (without) update identically, and both follow the formula in FP32."""
    g = torch.Generator().manual_seed(cout * 100 + cin)
    shp = (cout, taps, cin)
    w0, m0 = torch.randn(*shp, generator=g), 0.01 * torch.randn(*shp, generator=g)
    v0, g0 = 1e-3 * torch.rand(*shp, generator=g), torch.randn(*shp, generator=g)
    cin_pad, cout_pad = r64(cin), r64(cout)
    lr, b1, b2, eps, step = 1e-3, 0.9, 0.999, 1e-8, 5
    outs = []
    for with_wd in (False, True):
        w, m, v, gr = (t.clone().cuda() for t in (w0, m0, v0, g0))
        wf = torch.zeros((cout + 15) // 16 * 16, taps, cin_pad, dtype=torch.bfloat16, device="cuda")
        wd = torch.zeros(cin, taps, cout_pad, dtype=torch.bfloat16, device="cuda") if with_wd else None
        ops.adam(w, m, v, gr, cout, taps, cin, lr, b1, b2, eps, step, wf, cin_pad, wd, cout_pad if with_wd else 0)
        outs.append((w, m, v, gr, wf, wd))
    ops.check()
    (w1, m1, v1, g1, wf1, _), (w2, m2, v2, g2, wf2, wd2) = outs
    for a, b in ((w1, w2), (m1, m2), (v1, v2), (wf1, wf2)):
        assert torch.equal(a, b)
    assert not g1.any() and not g2.any()  # the gradient is consumed
    assert torch.equal(wd2.permute(2, 1, 0).flip(1)[:cout].cpu(), wf2[:cout, :, :cin].cpu())
    assert torch.equal(wf2[:cout, :, :cin].cpu(), w2.cpu().bfloat16())
    f = lambda z: torch.tensor(z, dtype=torch.float32)  # the kernel's FP32 hyper-parameters
    one, B1, B2 = f(1.0), f(b1), f(b2)
    mi = B1 * m0 + (one - B1) * g0
    vi = B2 * v0 + (one - B2) * g0 * g0
    ref = w0 - f(lr) * (mi / (one - B1 ** step)) / (torch.sqrt(vi / (one - B2 ** step)) + f(eps))
    assert torch.allclose(w2.cpu(), ref, rtol=1e-6, atol=1e-7)
    assert torch.allclose(m2.cpu(), mi, rtol=1e-6, atol=1e-8) and torch.allclose(v2.cpu(), vi, rtol=1e-6, atol=0)


def test_multi_tensor_adam_equals_per_layer_steps():
    """dn_adam_multi over several layers (3x3 and 1x1, with and without the transposed copy and the
    bias) leaves every buffer bit-identical to per-layer dn_adam + dn_adam_bias."""
    g = torch.Generator().manual_seed(17)
    shapes = [(32, 9, 33, True, True), (256, 9, 256, True, True), (33, 1, 32, True, False), (70, 9, 45, False, True)]

    def make():
        g.manual_seed(17)
        out = []
        for cout, taps, cin, bias, with_wd in shapes:
            t = lambda *sh, s=1.0: (s * torch.randn(*sh, generator=g)).cuda()
            w, m, v, gr = t(cout, taps, cin), t(cout, taps, cin, s=0.01), t(cout, taps, cin, s=0.03).abs(), t(cout, taps, cin)
            wf = torch.zeros((cout + 15) // 16 * 16, taps, r64(cin), dtype=torch.bfloat16, device="cuda")
            wd = torch.zeros(cin, taps, r64(cout), dtype=torch.bfloat16, device="cuda") if with_wd else None
            b = (t(cout), t(cout, s=0.01), t(cout, s=0.03).abs(), t(cout)) if bias else (None,) * 4
            out.append([w, m, v, gr, wf, r64(cin), wd, r64(cout) if with_wd else 0, cout, taps, cin, *b])
        return out

    lr, b1, b2, eps, step = 2e-3, 0.9, 0.999, 1e-8, 3
    ref = make()
    for w, m, v, gr, wf, cin_pad, wd, cout_pad, cout, taps, cin, b, mb, vb, gb in ref:
        ops.adam(w, m, v, gr, cout, taps, cin, lr, b1, b2, eps, step, wf, cin_pad, wd, cout_pad)
        if b is not None:
            ops.adam_bias(b, mb, vb, gb, lr, b1, b2, eps, step)
    got = make()
    table = ops.adam_table([tuple(e) for e in got])
    ops.adam_multi(table, lr, b1, b2, eps, step)
    ops.check()
    for r, q in zip(ref, got):
        for x, y in zip(r, q):
            if isinstance(x, torch.Tensor):
                assert torch.equal(x, y)


def test_sample_scale_is_inverse_mean_fluence():
    g = torch.Generator().manual_seed(5)
    x = torch.rand(3, 5, 64, 32, generator=g) * torch.tensor([1.0, 1e-3, 7.0]).view(3, 1, 1, 1)
    x[2, 0] = 0.0  # an all-dark sample: clamped at 1e-30
    got = sample_scale(x.cuda()).cpu().double()
    m = x[:, 0].double().mean(dim=(1, 2)).clamp_min(1e-30)
    assert torch.allclose(got, (1.0 / m).float().double(), rtol=1e-6, atol=0)


def test_predict_output_is_residual_then_unpack():
    B, H, W, C = 2, 16, 32, 33
    g = torch.Generator().manual_seed(9)
    x = _nhwc(B, H, W, C, 64, 21)
    out = torch.randn(B, H, W, 40, generator=g).cuda()
    scale = (torch.rand(B, generator=g) + 0.5).cuda()
    y = torch.empty(B, H, W, C, device="cuda")
    ops.residual(out, x, C, y)
    ref = torch.empty(B, C, H, W, device="cuda")
    ops.unpack_output(y, scale, ref)
    got = torch.empty(B, C, H, W, device="cuda")
    ops.predict_output(out, x, C, scale, got)
    assert torch.allclose(got, ref, rtol=2e-7, atol=0)


def _head_inputs(B, H, W, cout, seed):
    g = torch.Generator().manual_seed(seed)
    n_pad = (cout + 15) // 16 * 16
    x = _nhwc(B, H, W, 32, 64, seed)                  # the head's input (d0b activations)
    x0 = _nhwc(B, H, W, cout, 64, seed + 1, positive=True)  # the packed network input
    w = torch.zeros(n_pad, 1, 64)
    w[:cout, 0, :32] = 0.1 * torch.randn(cout, 32, generator=g)
    bias = (0.01 * torch.randn(cout, generator=g)).cuda()
    scale = (torch.rand(B, generator=g) + 0.5).cuda()
    t = (torch.rand(B, cout, H, W, generator=g) + 0.5).cuda()
    return x, w.bfloat16().cuda(), bias, x0, scale, t


@pytest.mark.parametrize("B,H,W,cout", [(2, 16, 128, 33), (3, 16, 32, 20), (1, 8, 256, 48)])
def test_fused_head_is_bit_identical_to_conv_then_output_kernels(B, H, W, cout):
    """dn_conv_head against dn_conv (fp32 NHWC output) followed by dn_predict_output, and by
    dn_pack_target + dn_mse: the prediction and the gradient seed are bit-identical, the loss equal
    up to the FP32 partial sums over 16 channels the fused head takes before its FP64 sum."""
    x, w, bias, x0, scale, t = _head_inputs(B, H, W, cout, 40 + cout)
    out = torch.zeros(B, H, W, (cout + 7) // 8 * 8, device="cuda")
    ops.conv(x, w, cout, out, taps=1, bias=bias)
    ref_pred = torch.empty(B, cout, H, W, device="cuda")
    ops.predict_output(out, x0, cout, scale, ref_pred)
    pred = torch.full((B, cout, H, W), float("nan"), device="cuda")
    ops.conv_head(x, w, cout, bias, x0, scale, pred=pred)
    ops.check()
    assert torch.equal(pred, ref_pred)

    tpk = torch.zeros(B, H, W, cout, device="cuda")
    ops.pack_target(t, scale, tpk)
    ref_dout = torch.zeros(B, H, W, 64, dtype=torch.bfloat16, device="cuda")
    ref_loss = torch.zeros((), dtype=torch.float64, device="cuda")
    ops.mse(out, x0, tpk, cout, ref_dout, ref_loss)
    dout = torch.zeros_like(ref_dout)
    loss = torch.zeros_like(ref_loss)
    ops.conv_head(x, w, cout, bias, x0, scale, target=t, dout=dout, loss=loss)
    ops.check()
    assert torch.equal(dout, ref_dout)
    # FP32 partial sums over 16 channels (then FP64) against FP64 throughout: a few FP32 ulps
    assert abs(loss.item() - ref_loss.item()) <= 1e-6 * ref_loss.item()
    # and against the definition in FP64 on the CPU
    y = x0[..., :cout].double().cpu() + out[..., :cout].double().cpu()
    r = y - (t.cpu().permute(0, 2, 3, 1).double() * scale.cpu().double().view(B, 1, 1, 1))
    assert abs(loss.item() - (r ** 2).mean().item()) <= 1e-5 * loss.item()


def _data(B, H, W, C, seed):
    g = torch.Generator().manual_seed(seed)
    base = torch.rand(B, 1, H, W, generator=g) + 0.5
    x = base * (1 + 0.3 * torch.randn(B, C, H, W, generator=g)) / torch.arange(1, C + 1).view(1, C, 1, 1)
    t = base / torch.arange(1, C + 1).view(1, C, 1, 1)
    return x.float(), t.float()


def test_unet_forward_and_gradients_match_reference():
    B, C, H, W = 2, 33, 128, 128
    x, t = _data(B, H, W, C, 1)
    net = UNet(in_ch=C, seed=3)
    # perturb the output head so that every layer receives a gradient
    net.layers["out"].w.normal_(0, 0.05)
    net.layers["out"].refresh()
    xs, ts = x.cuda(), t.cuda()
    scale = sample_scale(xs)
    net.load(xs, scale, ts)
    net.forward()
    loss = net.loss_and_grad_seed().item()
    net.backward()
    ops.check()
    s = scale.cpu().view(B, 1, 1, 1)
    rl, ry, rg = ref.loss_and_grads(net.state(), x * s, t * s, bf16=True)
    assert abs(loss - rl) <= 2e-3 * rl
    # Element by element, per layer: the GPU keeps activations in BF16 (8-bit mantissa, rounding
    # 2^-9 relative) and accumulates in another order than the reference, so the two sides round
    # slightly different FP32 values to BF16 and about one activation in 1e3 differs by one BF16
    # unit (2^-8); propagated through up to 14 layers of the backward chain, a weight-gradient
    # element then moves by a few percent of its layer's RMS gradient (measured: at most 0.070 of
    # the RMS for weights, 0.017 for biases, over two inputs).  Bound: 0.15 x RMS for weight
    # elements, 0.05 x RMS for bias elements, plus the norm and direction of the whole layer.
    for name, lay in net.layers.items():
        gw, gb = lay.gw.cpu().double(), lay.gb.cpu().double()
        rw, rb = (v.double() for v in rg[name])
        err = (gw - rw).norm() / rw.norm()
        cos = torch.nn.functional.cosine_similarity(gw.flatten(), rw.flatten(), dim=0)
        assert err < 5e-2 and cos > 0.998, (name, err.item(), cos.item())
        rms_w = rw.pow(2).mean().sqrt()
        assert float((gw - rw).abs().max()) <= 0.15 * float(rms_w), (name, float((gw - rw).abs().max() / rms_w))
        rms_b = rb.pow(2).mean().sqrt()
        assert float((gb - rb).abs().max()) <= 0.05 * float(rms_b) + 1e-30, name


def test_unet_training_reduces_loss():
    B, C, H, W = 2, 33, 128, 128
    x, t = _data(B, H, W, C, 2)
    net = UNet(in_ch=C, seed=4)
    xs, ts = x.cuda(), t.cuda()
    scale = sample_scale(xs)
    losses = [net.train_step(xs, scale, ts, lr=1e-3).item() for _ in range(60)]
    ops.check()
    assert losses[-1] < 0.7 * losses[0], losses[::10]
    pred = net.predict(xs, scale)
    assert pred.shape == xs.shape and torch.isfinite(pred).all()


def test_denoiser_trained_on_mc_pairs_beats_low_count_mc():
    """Trained on pairs the MC generates, the denoiser moves low-count maps closer to the
    high-count MC (the yardstick of its error) than the low-count MC itself is, on held-out phantoms."""
    from paper_1608_05238_gb300 import denoise_train as dt
    K, n = 8, 128
    x, t = dt.make_pairs(72, n=n, dx=0.1, K=K, n_low=20_000, n_high=2_000_000, seed0=20_000)
    net = UNet(in_ch=2 * K + 1, seed=1)
    dt.train(net, x[:64], t[:64], steps=300, batch=8, lr=2e-3)
    ops.check()
    ev = dt.evaluate(net, x[64:], t[64:])
    # measured after 300 steps: overall 0.163 -> 0.116, fluence a_0 0.063 -> 0.033
    assert ev["err_denoised"] < 0.8 * ev["err_input"], ev
    assert ev["err_a0_denoised"] < 0.7 * ev["err_a0_input"], ev

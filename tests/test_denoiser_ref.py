"""CPU pins of the plain PyTorch denoiser reference (oracle/denoiser_ref.py), which the GPU U-Net
is compared against: the weight layout is the convolution it claims to be, the residual output
is exact, and its gradients are those of its own loss (central finite differences in FP64)."""
import torch
import torch.nn.functional as F

from oracle import denoiser_ref as ref

CH = {"e0a": (None, 32), "e0b": (32, 32), "e1a": (32, 64), "e1b": (64, 64), "e2a": (64, 128),
      "e2b": (128, 128), "ma": (128, 256), "mb": (256, 256), "d2a": (256 + 128, 128), "d2b": (128, 128),
      "d1a": (128 + 64, 64), "d1b": (64, 64), "d0a": (64 + 32, 32), "d0b": (32, 32), "out": (32, None)}


def _params(cin, seed, dtype=torch.float64, scale=1.0):
    g = torch.Generator().manual_seed(seed)
    P = {}
    for n in ref.NAMES:
        ci, co = CH[n]
        ci = cin if ci is None else ci
        co = cin if co is None else co
        taps = 1 if n == "out" else 9
        w = torch.randn(co, taps, ci, generator=g, dtype=dtype) * scale * (2.0 / (taps * ci)) ** 0.5
        b = torch.randn(co, generator=g, dtype=dtype) * 0.01
        P[n] = (w, b)
    return P


def test_weight_layout_is_cross_correlation_with_tap_ky_kx():
    """w[cout][taps][cin] with tap = 3 ky + kx reads x[y + ky - 1][x + kx - 1] (zero padding): the
    same tap order and offsets as the tensor-core kernel's shifted tiles."""
    x = torch.arange(1.0, 1 + 5 * 6, dtype=torch.float64).reshape(1, 1, 5, 6)
    for tap in range(9):
        ky, kx = divmod(tap, 3)
        w = torch.zeros(1, 9, 1, dtype=torch.float64)
        w[0, tap, 0] = 1.0
        y = ref._conv(x, w, None, False, False)
        want = torch.zeros_like(x)
        for i in range(5):
            for j in range(6):
                si, sj = i + ky - 1, j + kx - 1
                if 0 <= si < 5 and 0 <= sj < 6:
                    want[0, 0, i, j] = x[0, 0, si, sj]
        assert torch.equal(y, want), tap


def test_residual_output_is_exact_with_a_zero_head():
    P = _params(5, 1)
    P["out"] = (torch.zeros_like(P["out"][0]), torch.zeros_like(P["out"][1]))
    x = torch.rand(2, 5, 16, 16, dtype=torch.float64, generator=torch.Generator().manual_seed(2))
    y, out = ref.forward(P, x, bf16=False)
    assert torch.equal(out, torch.zeros_like(out)) and torch.equal(y, x)


def test_reference_gradients_match_central_differences():
    torch.manual_seed(0)
    cin = 3
    P = _params(cin, 3, scale=0.7)
    g = torch.Generator().manual_seed(4)
    x = torch.rand(1, cin, 16, 16, dtype=torch.float64, generator=g) + 0.5
    t = torch.rand(1, cin, 16, 16, dtype=torch.float64, generator=g) + 0.5
    leaves = {n: (w.clone().requires_grad_(True), b.clone().requires_grad_(True)) for n, (w, b) in P.items()}
    loss = ((ref.forward(leaves, x, bf16=False)[0] - t) ** 2).mean()
    loss.backward()

    def loss_at(Q):
        with torch.no_grad():
            return ((ref.forward(Q, x, bf16=False)[0] - t) ** 2).mean().item()

    for k in range(4):
        d = {n: (torch.randn(w.shape, dtype=torch.float64, generator=g), torch.randn(b.shape, dtype=torch.float64, generator=g))
             for n, (w, b) in P.items()}
        analytic = sum((leaves[n][0].grad * d[n][0]).sum() + (leaves[n][1].grad * d[n][1]).sum() for n in P).item()
        h = 1e-7  # small enough that no ReLU of the network changes side
        plus = {n: (w + h * d[n][0], b + h * d[n][1]) for n, (w, b) in P.items()}
        minus = {n: (w - h * d[n][0], b - h * d[n][1]) for n, (w, b) in P.items()}
        fd = (loss_at(plus) - loss_at(minus)) / (2 * h)
        assert abs(fd - analytic) <= 1e-6 * abs(analytic) + 1e-10, (k, fd, analytic)


def test_pool_and_upsample_are_the_textbook_operators():
    x = torch.rand(1, 2, 8, 8, dtype=torch.float64, generator=torch.Generator().manual_seed(6))
    p = F.avg_pool2d(x, 2)
    assert torch.allclose(p[0, 1, 2, 3], x[0, 1, 4:6, 6:8].mean())
    u = F.interpolate(p, scale_factor=2, mode="nearest")
    assert torch.equal(u[0, :, 5, 7], p[0, :, 2, 3])

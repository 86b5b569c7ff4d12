"""Pins of the oracle U-Net: the zero head is the identity correction, and the network's
wiring equals an explicit re-construction from loop convolutions, loop pooling and index
upsampling (two levels, tiny volume)."""
import torch

import oracle.unet as ounet
from oracle import conv as oconv


def params(levels=2, base=2, seed=0):
    g = torch.Generator().manual_seed(seed)
    ch = [base * 2 ** i for i in range(levels)]
    p = {}

    def add(name, co, ci):
        p[name + "_w"] = torch.randn((co, 27, ci), generator=g, dtype=torch.float64) * 0.3
        p[name + "_b"] = torch.randn(co, generator=g, dtype=torch.float64) * 0.1

    cin = base
    for i in range(levels):
        add(f"enc{i}a", ch[i], cin)
        add(f"enc{i}b", ch[i], ch[i])
        cin = ch[i]
    for i in range(levels - 2, -1, -1):
        add(f"up{i}", ch[i], ch[i + 1])
        add(f"dec{i}a", ch[i], 2 * ch[i])
        add(f"dec{i}b", ch[i], ch[i])
    add("head", base, base)
    return p


def test_zero_head_is_identity():
    p = params()
    p["head_w"].zero_()
    p["head_b"].zero_()
    inp = torch.rand((1, 4, 4, 4), dtype=torch.float64)
    torch.testing.assert_close(ounet.forward(p, inp, levels=2, base=2), inp, rtol=0, atol=0)


def test_wiring_equals_explicit_construction():
    p = params()
    inp = torch.rand((1, 4, 4, 4), generator=torch.Generator().manual_seed(1), dtype=torch.float64)

    def c(name, x, relu=True):
        w = p[name + "_w"]
        co, _, ci = w.shape
        y = oconv.conv3d_loops(x, w.permute(0, 2, 1).reshape(co, ci, 3, 3, 3), p[name + "_b"])
        return y.clamp(min=0) if relu else y

    def pool(x):
        n, ch, d, h, w = x.shape
        out = torch.full((n, ch, d // 2, h // 2, w // 2), -torch.inf, dtype=torch.float64)
        for a in range(2):
            for b in range(2):
                for e in range(2):
                    out = torch.maximum(out, x[:, :, a::2, b::2, e::2])
        return out

    def up(x):
        n, ch, d, h, w = x.shape
        zi = torch.arange(2 * d) // 2
        yi = torch.arange(2 * h) // 2
        xi = torch.arange(2 * w) // 2
        return x[:, :, zi][:, :, :, yi][:, :, :, :, xi]

    x = torch.zeros((1, 2, 4, 4, 4), dtype=torch.float64)
    x[:, 0] = inp
    s0 = c("enc0b", c("enc0a", x))
    x1 = c("enc1b", c("enc1a", pool(s0)))
    u = c("up0", up(x1))
    x = c("dec0b", c("dec0a", torch.cat([u, s0], dim=1)))
    ref = inp + c("head", x, relu=False)[:, 0]
    torch.testing.assert_close(ounet.forward(p, inp, levels=2, base=2), ref, rtol=1e-12, atol=1e-12)

"""The warm-start U-Net on the tensor-core convolutions against the FP64 oracle network.

The GPU network keeps activations in bf16 (each layer's output rounded to 2^-9 relative),
so its output and gradients differ from the FP64 network by the accumulated bf16 rounding of
about 20 layers: a few 1e-3 relative. The checks allow 3e-2 relative (L2) and a cosine
similarity of at least 0.999; a wrong kernel, layout or flipped tap gives O(1) errors.
"""
import pytest
import torch

import oracle.unet as ounet
from paper_2110_09841_b300.unet import UNet3D

pytestmark = pytest.mark.gpu

SHAPE = (1, 8, 64, 128)     # n, d, h, w: the smallest volume whose coarsest level (1 x 8 x 16) the kernels take


def rel(a, b):
    return float((a - b).norm() / b.norm())


def cos(a, b):
    return float((a * b).sum() / (a.norm() * b.norm()))


def test_forward_and_gradients_match_oracle():
    model = UNet3D(seed=3).cuda()
    model.scale.fill_(4.0)
    with torch.no_grad():                          # give the head nonzero weights so every layer gets gradient
        model.head_w.normal_(0.0, 0.05, generator=torch.Generator(device="cuda").manual_seed(1))
    g = torch.Generator().manual_seed(7)
    inp = torch.rand(SHAPE, generator=g)
    target = torch.rand(SHAPE, generator=g)
    out = model(inp.cuda())
    loss = torch.mean((out - target.cuda()) ** 2)
    loss.backward()

    # the oracle gets the bf16-rounded weights the GPU network used
    p = {name: t.detach().cpu().double() for name, t in model.named_parameters()}
    scale = float(model.scale)
    for n in model.names:
        p[n + "_w"] = model.get_parameter(n + "_w").detach().to(torch.bfloat16).cpu().double().requires_grad_(True)
        p[n + "_b"] = p[n + "_b"].requires_grad_(True)
    ref = ounet.forward(p, inp.double(), scale=scale)
    rloss = torch.mean((ref - target.double()) ** 2)
    rloss.backward()
    assert rel(out.detach().cpu().double(), ref.detach()) < 3e-2
    for n in model.names:
        for suffix in ("_w", "_b"):
            gg = model.get_parameter(n + suffix).grad.cpu().double()
            rg = p[n + suffix].grad
            if rg.norm() == 0:
                continue
            assert rel(gg, rg) < 3e-2, (n + suffix, rel(gg, rg))
            assert cos(gg, rg) > 0.999, (n + suffix, cos(gg, rg))


def _torch_fp32_net(model):
    """The same network in torch FP32 (channels-first convolutions) with the model's FP32
    master weights."""
    import torch.nn.functional as F

    p = {n: torch.nn.Parameter(v.detach().clone().float()) for n, v in model.named_parameters()}
    scale = float(model.scale)

    def c(name, x, relu=True):
        w = p[name + "_w"]
        co, _, ci = w.shape
        y = F.conv3d(x, w.permute(0, 2, 1).reshape(co, ci, 3, 3, 3), p[name + "_b"], padding=1)
        return torch.relu(y) if relu else y

    def forward(inp):
        n, d, h, w = inp.shape
        x = torch.zeros((n, 16, d, h, w), device=inp.device)
        x[:, 0] = inp * scale
        skips = []
        for i in range(4):
            if i > 0:
                x = F.max_pool3d(x, 2)
            x = c(f"enc{i}a", x)
            x = c(f"enc{i}b", x)
            skips.append(x)
        for i in range(2, -1, -1):
            x = c(f"up{i}", F.interpolate(x, scale_factor=2, mode="nearest"))
            x = torch.cat([x, skips[i]], dim=1)
            x = c(f"dec{i}a", x)
            x = c(f"dec{i}b", x)
        return inp + c("head", x, relu=False)[:, 0] / scale

    return p, forward


def test_full_size_gradients_match_torch_fp32():
    """At the 128^3 training size the oracle network is too slow; the reference is the same
    network in torch FP32 on the GPU with the FP32 master weights, so the differences are the
    bf16 weights and activations of the tensor-core network (measured: output 2.4e-3,
    gradients 3e-3 to 2.1e-2 relative)."""
    prev = torch.backends.cudnn.allow_tf32
    torch.backends.cudnn.allow_tf32 = False
    try:
        shape = (1, 128, 128, 128)
        model = UNet3D(seed=3).cuda()
        model.scale.fill_(150.0)
        with torch.no_grad():
            model.head_w.normal_(0.0, 0.05, generator=torch.Generator(device="cuda").manual_seed(1))
        g = torch.Generator(device="cuda").manual_seed(7)
        inp = 0.01 * torch.rand(shape, device="cuda", generator=g)
        target = 0.01 * torch.rand(shape, device="cuda", generator=g)
        p, forward = _torch_fp32_net(model)
        out = model(inp)
        torch.mean((out - target) ** 2).backward()
        ref = forward(inp)
        torch.mean((ref - target) ** 2).backward()
        assert rel(out.detach(), ref.detach()) < 1e-2
        for name, v in model.named_parameters():
            assert rel(v.grad, p[name].grad) < 3e-2, name
            assert cos(v.grad, p[name].grad) > 0.999, name
    finally:
        torch.backends.cudnn.allow_tf32 = prev

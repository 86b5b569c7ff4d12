"""Tensor-core 3x3x3 convolutions (libkct_conv) against the FP64 oracle convolution.

Inputs are drawn in float32 and rounded to bf16 once; the oracle gets the same bf16 values in
float64. Products of bf16 values are exact in FP32, so the GPU result differs from the
oracle by the FP32 accumulation (bounded by K * 2^-24 * sum |x||w| for K terms, far less in
practice; 1e-4 of that absolute sum is allowed) and, for bf16 outputs, by the final rounding
(at most half a bf16 unit, 2^-9 relative; 2^-8 is allowed).
"""
import pytest
import torch

from oracle import conv as oconv
from paper_2110_09841_b300 import conv

pytestmark = pytest.mark.gpu

CASES = [  # n, d, h, w, cin, cout
    (1, 4, 8, 16, 16, 16),
    (1, 3, 4, 32, 32, 64),
    (2, 2, 2, 64, 64, 32),
    (1, 2, 1, 128, 128, 128),
    (1, 2, 8, 16, 48, 96),
    (1, 3, 8, 16, 128, 16),
]


def rand(shape, seed, scale=1.0):
    g = torch.Generator().manual_seed(seed)
    return (torch.randn(shape, generator=g) * scale).to(torch.bfloat16)


def to_cf(t):        # [n, d, h, w, c] -> [n, c, d, h, w]
    return t.permute(0, 4, 1, 2, 3)


def w_cf(w):         # [cout, 27, cin] -> [cout, cin, 3, 3, 3]
    co, _, ci = w.shape
    return w.permute(0, 2, 1).reshape(co, ci, 3, 3, 3)


def check(got, ref, absref, rel_out):
    got = got.double().cpu()
    bound = rel_out * ref.abs() + 1e-4 * absref + 1e-30
    excess = ((got - ref).abs() - bound).max()
    assert excess <= 0, float(excess)


@pytest.mark.parametrize("case", CASES)
def test_forward_matches_oracle(case):
    n, d, h, w, ci, co = case
    x = rand((n, d, h, w, ci), 1)
    wt = rand((co, 27, ci), 2, 0.1)
    b = torch.randn(co, generator=torch.Generator().manual_seed(3))
    err = conv.err_word("cuda")
    y = conv.conv3d_fwd(x.cuda(), wt.cuda(), b.cuda())
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref = to_cf_inv(oconv.conv3d(to_cf(x.double()), w_cf(wt.double()), b.double()))
    absref = to_cf_inv(oconv.conv3d(to_cf(x.double()).abs(), w_cf(wt.double()).abs()))
    check(y, ref, absref, 2.0 ** -8)


def to_cf_inv(t):    # [n, c, d, h, w] -> [n, d, h, w, c]
    return t.permute(0, 2, 3, 4, 1)


@pytest.mark.parametrize("case", CASES[:4])
def test_relu_epilogue(case):
    n, d, h, w, ci, co = case
    x = rand((n, d, h, w, ci), 4)
    wt = rand((co, 27, ci), 5, 0.1)
    y = conv.conv3d_fwd(x.cuda(), wt.cuda(), None, relu=True)
    y0 = conv.conv3d_fwd(x.cuda(), wt.cuda(), None, relu=False)
    torch.testing.assert_close(y, torch.clamp(y0, min=0), rtol=0, atol=0)


@pytest.mark.parametrize("case", CASES)
def test_input_gradient_matches_oracle(case):
    n, d, h, w, ci, co = case
    x = rand((n, d, h, w, ci), 6)
    wt = rand((co, 27, ci), 7, 0.1)
    gy = rand((n, d, h, w, co), 8)
    gx = conv.conv3d_dgrad(gy.cuda(), wt.cuda())
    torch.cuda.synchronize()
    rx, _ = oconv.conv3d_grads(to_cf(x.double()), w_cf(wt.double()), to_cf(gy.double()))
    ax, _ = oconv.conv3d_grads(to_cf(x.double()), w_cf(wt.double()).abs(), to_cf(gy.double()).abs())
    check(gx, to_cf_inv(rx), to_cf_inv(ax), 2.0 ** -8)


@pytest.mark.parametrize("case", CASES)
def test_weight_gradient_matches_oracle(case):
    n, d, h, w, ci, co = case
    x = rand((n, d, h, w, ci), 9)
    wt = rand((co, 27, ci), 10, 0.1)
    gy = rand((n, d, h, w, co), 11)
    gw = conv.conv3d_wgrad(x.cuda(), gy.cuda())
    torch.cuda.synchronize()
    assert int(conv.err_word("cuda").item()) == 0
    _, rw = oconv.conv3d_grads(to_cf(x.double()), w_cf(wt.double()), to_cf(gy.double()))
    _, aw = oconv.conv3d_grads(to_cf(x.double()).abs(), w_cf(wt.double()), to_cf(gy.double()).abs())
    # oracle [cout, cin, 3, 3, 3] -> [cout, 27, cin]
    rw = rw.reshape(co, ci, 27).permute(0, 2, 1)
    aw = aw.reshape(co, ci, 27).permute(0, 2, 1)
    check(gw, rw, aw, 0.0)


def test_autograd_function_gradients():
    n, d, h, w, ci, co = 1, 4, 8, 16, 16, 32
    x = rand((n, d, h, w, ci), 12).cuda().requires_grad_(True)
    wt = (torch.randn((co, 27, ci), generator=torch.Generator().manual_seed(13)) * 0.1).cuda().requires_grad_(True)
    b = torch.zeros(co, device="cuda", requires_grad=True)
    y = conv.conv3d(x, wt, b, relu=False)
    gy = rand((n, d, h, w, co), 14).cuda()
    (y.float() * gy.float()).sum().backward()
    wb = wt.detach().to(torch.bfloat16).double().cpu()
    rx, rw = oconv.conv3d_grads(to_cf(x.detach().double().cpu()), w_cf(wb), to_cf(gy.double().cpu()))
    ax, _ = oconv.conv3d_grads(to_cf(x.detach().double().cpu()), w_cf(wb).abs(), to_cf(gy.double().cpu()).abs())
    _, aw = oconv.conv3d_grads(to_cf(x.detach().double().cpu()).abs(), w_cf(wb), to_cf(gy.double().cpu()).abs())
    check(x.grad, to_cf_inv(rx), to_cf_inv(ax), 2.0 ** -8)
    check(wt.grad, rw.reshape(co, ci, 27).permute(0, 2, 1), aw.reshape(co, ci, 27).permute(0, 2, 1), 0.0)
    torch.testing.assert_close(b.grad.cpu().double(), gy.double().cpu().sum(dim=(0, 1, 2, 3)), rtol=1e-5, atol=1e-3)


@pytest.fixture
def no_tf32():
    prev = torch.backends.cudnn.allow_tf32
    torch.backends.cudnn.allow_tf32 = False
    yield
    torch.backends.cudnn.allow_tf32 = prev


def test_unet_layer_shapes_at_full_size_match_torch_fp32(no_tf32):
    """The U-Net's layer shapes at the 128^3 training size (and one 8 x 64 x 128 case), against
    torch's FP32 convolution of the same bf16 operands on the GPU (the oracle is too slow at
    this size). Forward and input gradient differ by the bf16 rounding of their outputs
    (about 2^-9 relative per element, 1.7e-3 in L2); the FP32 weight gradient agrees to 1e-5."""
    import torch.nn.functional as F

    def rel(a, b):
        return float((a.double() - b.double()).norm() / b.double().norm())

    g = torch.Generator(device="cuda").manual_seed(0)
    for (d, h, w), ci, co in [((128, 128, 128), 16, 16), ((128, 128, 128), 32, 16), ((64, 64, 64), 16, 32),
                              ((16, 16, 16), 128, 128), ((8, 64, 128), 16, 16)]:
        x = torch.randn((1, d, h, w, ci), device="cuda", generator=g).to(torch.bfloat16)
        wt = (0.1 * torch.randn((co, 27, ci), device="cuda", generator=g)).to(torch.bfloat16)
        gy = (1e-9 * torch.randn((1, d, h, w, co), device="cuda", generator=g)).to(torch.bfloat16)
        conv.err_word("cuda").zero_()
        y = conv.conv3d_fwd(x, wt)
        gx = conv.conv3d_dgrad(gy, wt)
        gw = conv.conv3d_wgrad(x, gy)
        torch.cuda.synchronize()
        assert int(conv.err_word("cuda").item()) == 0
        xc, gyc, wc = to_cf(x.float()), to_cf(gy.float()), w_cf(wt.float())
        ry = to_cf_inv(F.conv3d(xc, wc, padding=1))
        rgx = to_cf_inv(torch.nn.grad.conv3d_input(xc.shape, wc, gyc, padding=1))
        rgw = torch.nn.grad.conv3d_weight(xc, (co, ci, 3, 3, 3), gyc, padding=1).reshape(co, ci, 27).permute(0, 2, 1)
        case = ((d, h, w), ci, co)
        assert rel(y, ry) < 3e-3, case
        assert rel(gx, rgx) < 3e-3, case
        assert rel(gw, rgw) < 1e-4, case

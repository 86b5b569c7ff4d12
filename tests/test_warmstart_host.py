"""Host logic of the warm-start training that needs no GPU: the learning-rate schedule, the
training loop (on a tiny CPU model with the U-Net's interface) and the summary."""
import math

import pytest
import torch

from paper_2110_09841_b300 import warmstart


def test_lr_factor_warmup_then_cosine():
    assert warmstart.lr_factor(0, 100) == pytest.approx(1.0)
    assert warmstart.lr_factor(50, 100) == pytest.approx(0.05 + 0.95 * 0.5)
    assert warmstart.lr_factor(100, 100) == pytest.approx(0.05)
    assert warmstart.lr_factor(250, 100) == pytest.approx(0.05)          # held after the last step
    f = [warmstart.lr_factor(k, 100, warmup=10) for k in range(101)]
    assert f[0] == pytest.approx(0.1) and f[9] == pytest.approx(1.0)     # linear ramp over 10 steps
    assert f[10] == pytest.approx(1.0) and f[100] == pytest.approx(0.05)
    assert all(a >= b for a, b in zip(f[10:], f[11:]))                  # non-increasing after the ramp
    assert f[55] == pytest.approx(0.05 + 0.95 * 0.5 * (1 + math.cos(math.pi * 45 / 90)))


class _Scale(torch.nn.Module):
    """out = inp + (a * inp * scale + b) / scale: the U-Net's interface (a scale buffer set by
    train, a correction added to the input) with two parameters."""

    def __init__(self):
        super().__init__()
        self.a = torch.nn.Parameter(torch.zeros(()))
        self.b = torch.nn.Parameter(torch.zeros(()))
        self.register_buffer("scale", torch.ones(()))

    def forward(self, inp):
        return inp + (self.a * inp * self.scale + self.b) / self.scale


@pytest.mark.parametrize("warmup,clip", [(0, 0.0), (20, 0.0), (0, 1e-3)])
def test_train_fits_a_learnable_map(warmup, clip):
    g = torch.Generator().manual_seed(0)
    xs = 0.01 * torch.rand((16, 4, 4, 4), generator=g)
    ts = 3.0 * xs + 0.002                       # reachable: a = 2, b = 0.002 * scale
    model = _Scale()
    logs = []
    hist = warmstart.train(model, xs, ts, epochs=30, lr=5e-2, log=logs.append, warmup=warmup, clip=clip,
                           log_every=40)
    assert float(model.scale) == pytest.approx(1.0 / float(ts.abs().mean()))
    assert len(hist) == 30 and hist[-1] < 1e-3 * hist[0]
    assert sum(line.startswith("step ") for line in logs) == 30 * 16 // 40
    assert sum(line.startswith("epoch ") for line in logs) == 30


def test_summarise_counts_and_means():
    rows = [{"seed": s, "iters_zero": 20 + s, "iters_warm": 10, "time_zero_s": 1.0, "time_warm_s": 0.5 + s,
             "inference_s": 0.1, "normal0_warm": 0.01, "rel_err_x0": 0.2, "rel_err_cgls_zero": 0.1,
             "rel_err_cgls_warm": 0.1, "converged": True} for s in range(2)]
    s = warmstart.summarise(rows)
    assert s["iters_zero"] == 20.5 and s["iters_warm"] == 10 and s["seeds"] == 2
    assert s["warm_faster"] == 1 and s["all_converged"] is True


def test_loss_value_closed_form():
    t = torch.zeros((1, 3, 4, 5))
    ramp = 0.5 * torch.arange(5.0)                        # error grows by 0.5 per step along x
    out = t + ramp
    mse = float((ramp ** 2).mean())
    assert float(warmstart.loss_value(out, t)) == pytest.approx(mse)
    # differences: 0.5 along x, 0 along y and z
    assert float(warmstart.loss_value(out, t, edge_weight=2.0)) == pytest.approx(mse + 2.0 * 0.25)
    # a constant error has no differences
    assert float(warmstart.loss_value(t + 1.0, t, edge_weight=3.0)) == pytest.approx(1.0)
    # a checkerboard error along z: differences of 2 everywhere along z
    chk = (-1.0) ** torch.arange(3.0)
    assert float(warmstart.loss_value(t + chk[None, :, None, None], t, edge_weight=1.0)) == pytest.approx(1.0 + 4.0)


def test_train_with_edge_term_fits():
    g = torch.Generator().manual_seed(1)
    xs = 0.01 * torch.rand((8, 4, 4, 4), generator=g)
    ts = 3.0 * xs + 0.002
    model = _Scale()
    hist = warmstart.train(model, xs, ts, epochs=40, lr=5e-2, edge_weight=1.0)
    assert hist[-1] < 1e-3 * hist[0]


def test_save_and_load_round_trip(tmp_path):
    from paper_2110_09841_b300.unet import UNet3D

    a = UNet3D(seed=1)
    with torch.no_grad():
        a.scale.fill_(123.0)
        a.head_w.normal_(0.0, 0.1, generator=torch.Generator().manual_seed(2))
    path = str(tmp_path / "unet.pt")
    warmstart.save_model(a, path)
    b = warmstart.load_model(UNet3D(seed=9), path)
    assert float(b.scale) == 123.0
    for (na, ta), (nb, tb) in zip(a.state_dict().items(), b.state_dict().items()):
        assert na == nb and torch.equal(ta, tb), na

"""The projector as a differentiable, batched operator on the GPU: autograd gradients against
central finite differences and against the FP64 oracle's adjoint, batched launches against
single ones, and replay of a captured CUDA graph."""
import numpy as np
import pytest
import torch

import oracle
from paper_2110_09841_b300 import autograd, inputs
from paper_2110_09841_b300.kct import Projector

pytestmark = pytest.mark.gpu

TOL = 1e-4


def sub16():
    return inputs.make_geometry((16, 16, 16), (1.0, 1.0, 1.0), (40, 32), (0.8, 0.8), 9, 750.0, 1200.0, 360.0)


@pytest.mark.parametrize("vname", ["exact", "relaxed"])
def test_gradient_matches_central_differences(vname):
    """d/dx 0.5 |A x - y|^2 = A^T (A x - y); for a quadratic loss the central difference with
    h = 1e-3 differs from the directional derivative only by rounding. The projections are
    float32: each b_i carries a rounding error of about eps32 |b_i| of random sign, which moves
    the loss by sum_i r_i delta b_i, so the difference quotient carries about
    eps32 sqrt(sum (r_i b_i)^2) / h; the test allows 4 of those plus 2e-4 relative."""
    g = sub16()
    A = Projector(g, vname, "cos")
    x = inputs.uniform_volume(g.vol_shape, 1, device="cuda").requires_grad_(True)
    y = inputs.uniform_projections(g.proj_shape, 2, device="cuda")
    d = inputs.uniform_volume(g.vol_shape, 3, device="cuda") - 0.5

    def loss(v):
        r = (autograd.project(v, A) - y).double()
        return 0.5 * (r * r).sum()

    L = loss(x)
    L.backward()
    gd = float((x.grad.double() * d.double()).sum())
    h = 1e-3
    with torch.no_grad():
        fd = (float(loss(x + h * d)) - float(loss(x - h * d))) / (2 * h)
        b = A.project(x.detach()).double()
        noise = 2.0 ** -24 * float(((b - y.double()) * b).norm()) / h
    assert abs(gd - fd) <= 2e-4 * abs(fd) + 4.0 * noise


def test_gradient_matches_oracle_adjoint():
    g = sub16()
    A = Projector(g, "exact", "cos")
    x = inputs.uniform_volume(g.vol_shape, 4, device="cuda").requires_grad_(True)
    y = inputs.uniform_projections(g.proj_shape, 5, device="cuda")
    r = autograd.project(x, A) - y
    (0.5 * (r * r).sum()).backward()
    ref = oracle.backproject(g, r.detach().cpu().double().numpy(), 0, 0)
    got = x.grad.cpu().double().numpy()
    mx = np.abs(ref).max()
    assert np.abs(got - ref).max() <= TOL * mx
    big = np.abs(ref) >= 1e-3 * mx
    assert (np.abs(got - ref)[big] / np.abs(ref[big])).max() <= TOL


def test_backproject_function_gradient_is_projection():
    g = sub16()
    A = Projector(g, "relaxed", "cos")
    y = inputs.uniform_projections(g.proj_shape, 6, device="cuda").requires_grad_(True)
    w = inputs.uniform_volume(g.vol_shape, 7, device="cuda")
    (autograd.backproject(y, A) * w).sum().backward()
    ref = A.project(w)
    torch.testing.assert_close(y.grad, ref, rtol=1e-5, atol=1e-6 * float(ref.abs().max()))


@pytest.mark.parametrize("vname", ["exact", "relaxed"])
def test_batched_launch_equals_single_launches(vname):
    """A batch of perfusion-like frames through shared views in one launch."""
    g = inputs.make_geometry((24, 24, 20), (1.0, 1.0, 1.0), (48, 40), (0.8, 0.8), 20, 750.0, 1200.0, 360.0)
    frames = inputs.perfusion_frames(g, 31, frames=4, device="cuda")
    A = Projector(g, vname, "cos")
    b = A.project_batch(frames)
    for f in range(4):
        ref = A.project(frames[f].contiguous())
        torch.testing.assert_close(b[f], ref, rtol=1e-5, atol=1e-6 * float(ref.abs().max()))
    y = inputs.uniform_projections((4,) + g.proj_shape, 8, device="cuda")
    xb = A.backproject_batch(y)
    for f in range(4):
        torch.testing.assert_close(xb[f], A.backproject(y[f].contiguous()), rtol=0, atol=0)
    # autograd through the batched path
    fr = frames.clone().requires_grad_(True)
    (autograd.project(fr, A) * y).sum().backward()
    torch.testing.assert_close(fr.grad, xb, rtol=0, atol=0)


def test_captured_graph_replays():
    """Projection and adjoint enqueue work only (no allocation, no synchronisation), so they
    can be captured in a CUDA graph and replayed on new inputs."""
    g = inputs.workload_geometry("cvp32")
    A = Projector(g, "exact", "cos")
    x = torch.zeros(g.vol_shape, device="cuda")
    y = torch.zeros(g.proj_shape, device="cuda")
    b = torch.empty(g.proj_shape, device="cuda")
    xb = torch.empty(g.vol_shape, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        A.project(x, out=b)
        A.backproject(y, out=xb)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        A.project(x, out=b)
        A.backproject(y, out=xb)
    for seed in (1, 2):
        x.copy_(inputs.workload_phantom("cvp32").cuda() * seed)
        y.copy_(inputs.uniform_projections(g.proj_shape, seed, device="cuda"))
        graph.replay()
        torch.cuda.synchronize()
        rb, rx = A.project(x), A.backproject(y)
        torch.testing.assert_close(b, rb, rtol=1e-5, atol=1e-6 * float(rb.abs().max()))
        torch.testing.assert_close(xb, rx, rtol=0, atol=0)


@pytest.mark.parametrize("vname", ["exact", "relaxed"])
def test_batched_calls_captured_in_a_graph(vname):
    """A batch of perfusion-like frames projected and backprojected by one batched launch each,
    captured once in a CUDA graph and replayed on new frames (the configuration of the batched
    benchmark, at a small size): replays equal eager batched calls."""
    g = inputs.make_geometry((24, 24, 20), (1.0, 1.0, 1.0), (48, 40), (0.8, 0.8), 20, 750.0, 1200.0, 200.0)
    A = Projector(g, vname, "cos")
    A.autotune(inputs.perfusion_frames(g, 40, frames=1, device="cuda")[0].contiguous())
    frames = torch.zeros((4,) + g.vol_shape, device="cuda")
    proj = torch.empty((4,) + g.proj_shape, device="cuda")
    back = torch.empty((4,) + g.vol_shape, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        A.project_batch(frames, out=proj)
        A.backproject_batch(proj, out=back)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        A.project_batch(frames, out=proj)
        A.backproject_batch(proj, out=back)
    for seed in (41, 42):
        frames.copy_(inputs.perfusion_frames(g, seed, frames=4, device="cuda"))
        graph.replay()
        torch.cuda.synchronize()
        rp = A.project_batch(frames)
        torch.testing.assert_close(proj, rp, rtol=1e-5, atol=1e-6 * float(rp.abs().max()))
        torch.testing.assert_close(back, A.backproject_batch(proj), rtol=0, atol=0)
    assert A.device_error() == 0


@pytest.mark.parametrize("vname", ["exact", "relaxed"])
def test_autotuned_chunk_gives_the_same_projection(vname):
    g = inputs.workload_geometry("cvp32")
    x = inputs.workload_phantom("cvp32").cuda()
    A = Projector(g, vname, "cos")
    assert A.view_chunk == 16
    ref = A.project(x)
    chunk, ms = A.autotune(x)
    assert chunk in (1, 2, 4, 8, 16, 32, 64) and ms > 0 and A.view_chunk == chunk
    for c in (1, 5, 64):
        A.view_chunk = c
        torch.testing.assert_close(A.project(x), ref, rtol=1e-5, atol=1e-6 * float(ref.abs().max()))
    from paper_2110_09841_b300.kct import KctError
    with pytest.raises(KctError):
        A.view_chunk = 65

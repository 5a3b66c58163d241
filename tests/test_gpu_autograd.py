"""The compliance as a torch.autograd.Function: its gradient must be the
library's adjoint gradient (same kernels, bitwise), agree with the oracle's
adjoint gradient, follow the chain rule through torch, and match central
differences of the Function's own forward value."""
import numpy as np
import pytest

import lattice_inputs as LI
from oracle import grad as ograd

from romb_testutil import small_rom

pytestmark = pytest.mark.gpu
romb = pytest.importorskip("paper_2604_09113_gb300")
torch = pytest.importorskip("torch")
from paper_2604_09113_gb300.autograd import compliance  # noqa: E402


@pytest.fixture(scope="module")
def setup():
    p = 4
    R, path = small_rom(0, p, 0.18, 0.40, 20, 12, 1)
    lat = LI.lattice(4, 3, p, 2, seed=41, mu_mode="uniform", mu_range=(0.22, 0.36), rho=5e-4)
    ctx = romb.Context(0)
    romb.romb_train_load(ctx.h, path)
    yield dict(R=R, lat=lat, ctx=ctx)
    ctx.close()


@pytest.mark.parametrize("device", ["cuda", "cpu"])
def test_gradient_is_the_adjoint_gradient(setup, device):
    lat, ctx = setup["lat"], setup["ctx"]
    ctrl = torch.tensor(lat.ctrl, device=device, requires_grad=True)
    mu = torch.tensor(lat.mu, device=device, requires_grad=True)
    c = compliance(ctx, lat, ctrl, mu, rtol=1e-12)
    c.backward(retain_graph=True)
    g_ctrl, g_mu = ctrl.grad.clone(), mu.grad.clone()
    ctrl.grad, mu.grad = None, None
    (3.0 * c + c * c).backward()
    # the same calls through the C ABI directly
    romb.romb_assemble(ctx.h, lat, romb.ROMB_FP64)
    romb.romb_factor(ctx.h)
    nodes = (lat.p * lat.nx + 1) * (lat.p * lat.ny + 1)
    romb.romb_bddc_solve(ctx.h, nodes, rtol=1e-12, maxit=1000)
    c0, dx, _, dmu = romb.romb_compliance_grad(ctx.h, len(lat.ctrl), lat.ncells)
    assert c.item() == c0
    assert torch.equal(g_ctrl.cpu(), torch.from_numpy(dx)) and torch.equal(g_mu.cpu(), torch.from_numpy(dmu))
    w = 3.0 + 2.0 * c0    # chain rule through torch
    assert np.allclose(ctrl.grad.cpu().numpy(), w * dx, rtol=1e-14, atol=0)
    assert np.allclose(mu.grad.cpu().numpy(), w * dmu, rtol=1e-14, atol=0)
    co, dxo, dmuo, _ = ograd.compliance_gradient(lat, {0: setup["R"]})
    assert abs(c0 - co) <= 1e-10 * abs(co)
    assert np.abs(dx - dxo).max() <= 1e-8 * np.abs(dxo).max()
    assert np.abs(dmu - dmuo).max() <= 1e-8 * np.abs(dmuo).max()


def test_central_differences_of_the_forward(setup):
    lat, ctx = setup["lat"], setup["ctx"]
    ctrl = torch.tensor(lat.ctrl, device="cuda", requires_grad=True)
    mu = torch.tensor(lat.mu, device="cuda", requires_grad=True)
    compliance(ctx, lat, ctrl, mu, rtol=1e-13).backward()
    g = torch.Generator().manual_seed(5)
    h = 1e-5
    with torch.no_grad():
        for which in ("ctrl", "mu"):
            v = torch.randn(ctrl.shape if which == "ctrl" else mu.shape, generator=g, dtype=torch.float64).cuda()
            cs = []
            for s in (1.0, -1.0):
                a = ctrl + s * h * v if which == "ctrl" else ctrl
                b = mu + s * h * v if which == "mu" else mu
                cs.append(compliance(ctx, lat, a, b, rtol=1e-13).item())
            fd = (cs[0] - cs[1]) / (2 * h)
            an = ((ctrl.grad if which == "ctrl" else mu.grad) * v).sum().item()
            assert abs(fd - an) <= 1e-5 * abs(an), (which, fd, an)

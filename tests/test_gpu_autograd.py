"""Differentiable F(c), theta(c) through torch.autograd (needs a GB300).

g(x) = exp(i sum_a c_a(x) lambda_a).  The reference values come from the oracle's F and
theta (Eqs. (1)-(3)) of the field transformed on the CPU; gradients are checked against
central finite differences of that oracle forward (float64, h = 1e-6) and, at c = 0,
against the analytic gradient Tr[lambda_a Delta] / (2i nd Nc V).
"""
import numpy as np
import pytest

import oracle
from paper_1412_1498_gb300 import fields

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gf():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1412_1498_gb300 import build
    build.build()
    from paper_1412_1498_gb300 import gf as m
    return m


def oracle_F_theta(U, c, gauge):
    # g = exp(i c.lambda) by scipy's matrix exponential (batched over the sites)
    from scipy.linalg import expm
    Lt, Lz, Ly, Lx = U.shape[:4]
    X = np.einsum("...a,aij->...ij", c.reshape(Lt, Lz, Ly, Lx, 8), fields.gell_mann())
    W = fields.gauge_transform(U, expm(1j * X))
    F, th, _, _ = oracle.measure(W, gauge)
    return F, th


def make(gf, dims, gauge, U):
    fx = gf.GaugeFixer(dims, gauge, gf.GF_FP64_18, autograd=True)
    fx.upload(U)
    return fx


@pytest.mark.parametrize("gauge", [0, 1])
def test_forward_matches_oracle(gf, gauge):
    from paper_1412_1498_gb300.autograd import functional_theta
    dims = (4, 4, 4, 6)
    V = int(np.prod(dims))
    U = fields.random_gauge_config(dims, 0.5, 100)
    c = np.random.default_rng(1).normal(scale=0.3, size=(V, 8))
    fx = make(gf, dims, gauge, U)
    F, th = functional_theta(torch.from_numpy(c).cuda(), fx)
    rF, rth = oracle_F_theta(U, c, gauge)
    assert abs(F.item() - rF) < 1e-12 * abs(rF) and abs(th.item() - rth) < 1e-12 * rth
    fx.close()


@pytest.mark.parametrize("gauge", [0, 1])
def test_gradient_at_zero_is_delta(gf, gauge):
    from paper_1412_1498_gb300.autograd import functional_theta
    dims = (4, 4, 6, 4)
    V = int(np.prod(dims))
    nd = 4 if gauge == 0 else 3
    U = fields.random_gauge_config(dims, 0.5, 101)
    fx = make(gf, dims, gauge, U)
    c = torch.zeros((V, 8), dtype=torch.float64, device="cuda", requires_grad=True)
    F, th = functional_theta(c, fx)
    F.backward()
    D = oracle.delta(U, gauge).reshape(V, 3, 3)
    want = (np.einsum("aij,sji->sa", fields.gell_mann(), D) / (2j * nd * 3 * V)).real
    got = c.grad.cpu().numpy()
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()
    fx.close()


@pytest.mark.parametrize("gauge", [0, 1])
def test_gradients_match_central_differences(gf, gauge):
    from paper_1412_1498_gb300.autograd import functional_theta
    dims = (4, 4, 4, 4)
    V = int(np.prod(dims))
    U = fields.random_gauge_config(dims, 0.5, 102)
    rng = np.random.default_rng(2)
    c0 = rng.normal(scale=0.2, size=(V, 8))
    fx = make(gf, dims, gauge, U)
    grads = []
    for which in (0, 1):
        c = torch.from_numpy(c0.copy()).cuda().requires_grad_(True)
        out = functional_theta(c, fx)
        out[which].backward()
        grads.append(c.grad.cpu().numpy())
    h = 1e-6
    for _ in range(12):
        s, a = int(rng.integers(V)), int(rng.integers(8))
        cp, cm = c0.copy(), c0.copy()
        cp[s, a] += h
        cm[s, a] -= h
        fp, tp = oracle_F_theta(U, cp, gauge)
        fm, tm = oracle_F_theta(U, cm, gauge)
        for which, (vp, vm) in enumerate(((fp, fm), (tp, tm))):
            fd = (vp - vm) / (2 * h)
            scale = np.abs(grads[which]).max()
            assert abs(grads[which][s, a] - fd) < 1e-6 * scale, (which, s, a, grads[which][s, a], fd)
    fx.close()


def test_sgd_first_step_is_naive_descent_and_50_steps_ascend(gf):
    # loss = -F, lr = alpha nd Nc V / 2: the first SGD step from c = 0 is g = exp((alpha/2)
    # Delta), the naive steepest-descent step of Eq. (7) with the exact exponential
    from paper_1412_1498_gb300.autograd import functional_theta
    dims = (8, 8, 8, 8)
    V = int(np.prod(dims))
    alpha = 0.08
    U = fields.random_gauge_config(dims, 0.4, 1, 2)
    fx = make(gf, dims, 0, U)
    c = torch.zeros((V, 8), dtype=torch.float64, device="cuda", requires_grad=True)
    opt = torch.optim.SGD([c], lr=alpha * 4 * 3 * V / 2)
    hist = []
    for step in range(50):
        opt.zero_grad()
        F, th = functional_theta(c, fx)
        hist.append((F.item(), th.item()))
        (-F).backward()
        opt.step()
        if step == 0:
            D = oracle.delta(U).reshape(dims[::-1] + (3, 3))
            from scipy.linalg import expm
            W = fields.gauge_transform(U, expm(0.5 * alpha * D))     # Eq. (7): g = exp(alpha/2 Delta)
            F1, th1 = oracle_F_theta(U, c.detach().cpu().numpy(), 0)
            assert abs(F1 - oracle.measure(W)[0]) < 1e-12
    F, th = functional_theta(c, fx)
    hist.append((F.item(), th.item()))
    Fs = np.array([h[0] for h in hist])
    assert np.all(np.diff(Fs) > -1e-13) and Fs[-1] > Fs[0]
    assert hist[-1][1] < hist[0][1]
    fx.close()

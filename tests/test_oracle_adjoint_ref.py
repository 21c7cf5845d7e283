"""Pins for the differentiable torch restatement of the scheme (oracle side):
its forward equals the C oracle's frozen run, its autograd gradient equals
central finite differences of the C oracle, and its eps_2 equals the C one."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from oracle import torch_ref as T


def setup(n, scheme, seed, bc=(0, 0, 0)):
    if bc[0] == 1:
        g, w = W.smooth_periodic(n=n, seed=seed, scheme=scheme)
    else:
        g, w = W.lumpy(n=n, seed=seed, scheme=scheme)
        w[1] = 0.3 * np.tanh(w[0] - 1.0)
        w[2] = -0.2 * np.tanh(w[0] - 2.0)
    g.bc = bc
    c = oracle.make_cfg(g.n, g.dx, scheme=scheme, bc=bc)
    u0 = oracle.prim2con(w)
    return g, c, u0


@pytest.mark.parametrize("scheme,bc", [(5, (0, 0, 0)), (7, (0, 0, 0)), (5, (1, 1, 1))])
def test_torch_forward_equals_c_oracle(oracle_lib, scheme, bc):
    g, c, u0 = setup((7, 8, 9), scheme, 3, bc)
    ref, t, k, al, dts = oracle_lib.run(c, u0, 2, record=True)
    got = T.run_frozen(torch.from_numpy(u0), al, dts, g.n, g.dx, g.bc, (scheme + 1) // 2).numpy()
    for f in range(5):
        assert np.abs(got[f] - ref[f]).max() <= 1e-13 * np.abs(ref[f]).max()


@pytest.mark.parametrize("scheme", [5, 7])
def test_torch_gradient_equals_oracle_finite_differences(oracle_lib, scheme):
    g, c, u0 = setup((6, 7, 5), scheme, 5)
    _, _, _, al, dts = oracle_lib.run(c, u0, 2, record=True)
    rng = np.random.default_rng(1)
    lam = rng.standard_normal(u0.shape)
    ut = torch.from_numpy(u0.copy()).requires_grad_(True)
    J = (T.run_frozen(ut, al, dts, g.n, g.dx, g.bc, (scheme + 1) // 2) * torch.from_numpy(lam)).sum()
    J.backward()
    grad = ut.grad.numpy()
    for idx in [(0, 2, 3, 1), (1, 0, 0, 0), (3, 4, 6, 5), (4, 1, 1, 2), (2, 4, 2, 3), (0, 0, 6, 5)]:
        h = 1e-6 * max(abs(u0[idx]), u0[0][idx[1:]])
        up, um = u0.copy(), u0.copy()
        up[idx] += h
        um[idx] -= h
        fp = (oracle_lib.run(c, up, 2, alpha_in=al, dt_in=dts)[0] * lam).sum()
        fm = (oracle_lib.run(c, um, 2, alpha_in=al, dt_in=dts)[0] * lam).sum()
        fd = (fp - fm) / (2 * h)
        assert abs(fd - grad[idx]) <= 2e-6 * max(1.0, abs(grad[idx])), (idx, fd, grad[idx])


def test_torch_eps2_equals_c_oracle(oracle_lib):
    g, c, u0 = setup((9, 8, 7), 5, 8)
    a = oracle_lib.eps2(c, u0)
    b = float(T.eps2(torch.from_numpy(u0)))
    assert abs(a - b) <= 1e-14 * max(1.0, abs(a))
    assert abs(a) > 1e-3

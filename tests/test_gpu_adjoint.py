"""Hand-written adjoint kernels (hydro_forward_record / hydro_adjoint /
hydro_eps2) against the plain CPU torch-autograd restatement of the scheme
(tiny grids) and against central finite differences of the C oracle with the
Lax-Friedrichs speeds and time steps frozen (the 24^3 and 96^3 adjoint
configurations).  Tolerance: relative error 1e-7 (the stated bar) for the
autograd comparison; finite differences carry their own truncation error."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from oracle import torch_ref as T
from parity import field_errors, oracle_cfg

pytestmark = pytest.mark.gpu
ADJ_TOL = 1e-7


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_03360_gb300.build as B
    B.build()
    oracle.build()


def flow_state(n, seed, scheme, bc=(0, 0, 0)):
    if bc[0] == 1:
        g, w = W.smooth_periodic(n=n, seed=seed, scheme=scheme, vamp=0.4)
    else:
        g, w = W.lumpy(n=n, seed=seed, scheme=scheme)
        w[1] = 0.3 * np.tanh(w[0] - 1.0)
        w[2] = -0.2 * np.tanh(w[0] - 2.0)
        w[3] = 0.1 * np.tanh(w[0] - 1.5)
    g.bc = bc
    return g, oracle.prim2con(w)


def reference_vjp(g, u0, lam, nsteps):
    """Oracle-recorded speeds/dt, torch autograd of the frozen run."""
    _, _, _, al, dts = oracle.run(oracle_cfg(g), u0, nsteps, record=True)
    ut = torch.from_numpy(u0.copy()).requires_grad_(True)
    uN = T.run_frozen(ut, al, dts, g.n, g.dx, g.bc, (g.scheme + 1) // 2)
    (uN * torch.from_numpy(lam)).sum().backward()
    return ut.grad.numpy(), al, dts


@pytest.mark.parametrize("scheme,dims,bc,nsteps,ckpt", [
    (5, (10, 9, 8), (0, 0, 0), 3, 2),
    (7, (9, 10, 11), (0, 0, 0), 3, 1),
    (5, (12, 11, 10), (1, 1, 1), 4, 3),
    (7, (8, 12, 1), (0, 0, 0), 2, 5),
    (5, (1, 13, 9), (0, 0, 0), 3, 2),
    # pencils of at least 8r cells are swept in two segments whose shared
    # cells (the middle, and with periodic boundaries the ends) are summed
    (5, (27, 9, 8), (0, 0, 0), 3, 2),
    (5, (9, 26, 8), (1, 1, 1), 3, 2),
    (7, (8, 9, 35), (0, 0, 0), 2, 1),
    (7, (33, 8, 9), (1, 1, 1), 2, 1),
])
def test_adjoint_matches_torch_autograd(scheme, dims, bc, nsteps, ckpt):
    from paper_1604_03360_gb300 import Hydro
    g, u0 = flow_state(dims, 40 + sum(dims), scheme, bc)
    lam = np.random.default_rng(7).standard_normal(u0.shape)
    ref, al, dts = reference_vjp(g, u0, lam, nsteps)
    with Hydro.from_grid(g) as h:
        h.set_state(u0)
        h.forward_record(nsteps, ckpt)
        gal, gdt = h.recorded_steps()
        got = h.adjoint(lam)
    # the GPU's own forward speeds and steps agree with the oracle's
    assert np.abs(gal - al).max() <= 1e-13 * np.abs(al).max()
    assert np.abs(gdt - dts).max() <= 1e-13 * np.abs(dts).max()
    err = field_errors(got, ref)
    assert np.all(err <= ADJ_TOL), err


# pencil-kernel variants (HYDRO_ADJ_PENCIL): integer-pipe products and CTAs
# per SM; every one gives the same bits
ADJ_PENCIL_VARIANTS = 6


@pytest.mark.parametrize("scheme,dims,bc", [
    (5, (27, 9, 8), (0, 0, 0)),
    (5, (9, 26, 8), (1, 1, 1)),
    (7, (33, 8, 9), (1, 1, 1)),
    (7, (8, 9, 35), (0, 0, 0)),
])
def test_adjoint_pencil_variants_give_the_same_bits(scheme, dims, bc, monkeypatch):
    from paper_1604_03360_gb300 import Hydro
    g, u0 = flow_state(dims, 40 + sum(dims), scheme, bc)
    lam = np.random.default_rng(7).standard_normal(u0.shape)
    got = []
    with Hydro.from_grid(g) as h:
        for v in range(ADJ_PENCIL_VARIANTS):
            monkeypatch.setenv("HYDRO_ADJ_PENCIL", str(v))
            h.set_state(u0)
            h.forward_record(2, 1)
            got.append(h.adjoint(lam))
    for v in range(1, ADJ_PENCIL_VARIANTS):
        assert np.array_equal(got[v], got[0]), v


@pytest.mark.parametrize("nsteps,ckpt", [(5, 2), (3, 3), (4, 1)])
def test_adjoint_repeated_after_one_forward(nsteps, ckpt):
    """The first reverse sweep after a recorded forward takes the last
    segment's stage inputs from the forward, later ones recompute it: the same
    bits either way."""
    from paper_1604_03360_gb300 import Hydro
    g, u0 = flow_state((12, 11, 10), 77, 5, (0, 0, 0))
    lam = np.random.default_rng(3).standard_normal(u0.shape)
    with Hydro.from_grid(g) as h:
        h.set_state(u0)
        h.forward_record(nsteps, ckpt)
        first = h.adjoint(lam)
        second = h.adjoint(lam)
    assert np.array_equal(first, second)


def test_eps2_value_and_gradient():
    from paper_1604_03360_gb300 import Hydro
    g, u0 = flow_state((14, 12, 10), 3, 5)
    ut = torch.from_numpy(u0.copy()).requires_grad_(True)
    e_ref = T.eps2(ut)
    e_ref.backward()
    with Hydro.from_grid(g) as h:
        h.set_state(u0)
        grad = np.empty_like(u0)
        e = h.eps2(None, grad)
        e2 = h.eps2(torch.from_numpy(u0).cuda())
    assert abs(e - oracle.eps2(oracle_cfg(g), u0)) <= 1e-13 * abs(e)
    assert e == e2
    assert np.all(field_errors(grad, ut.grad.numpy()) <= 1e-12)


def test_autograd_chain_eps2_wrt_initial_energy():
    """e0 -> state at rest -> N steps -> eps_2, one backward pass through the
    torch.autograd.Function wrappers, against torch autograd of the reference."""
    from paper_1604_03360_gb300 import Hydro
    from paper_1604_03360_gb300 import autograd as HA
    g, w = W.lumpy(n=(11, 10, 9), seed=17)
    e0 = torch.from_numpy(w[0].copy()).cuda().requires_grad_(True)
    n0 = torch.from_numpy(w[4].copy()).cuda()
    with Hydro.from_grid(g) as h:
        eps = HA.eps2(HA.evolve(HA.state_at_rest(e0, n0), h, 3, 2), h)
        eps.backward()
        got = e0.grad.cpu().numpy()
    u0 = oracle.prim2con(w)
    _, _, _, al, dts = oracle.run(oracle_cfg(g), u0, 3, record=True)
    er = torch.from_numpy(w[0].copy()).requires_grad_(True)
    z = torch.zeros_like(er)
    ur = torch.stack([er, z, z, z, torch.from_numpy(w[4].copy())])
    T.eps2(T.run_frozen(ur, al, dts, g.n, g.dx, g.bc, 3)).backward()
    ref = er.grad.numpy()
    assert abs(float(eps.detach()) - oracle.eps2(oracle_cfg(g), oracle.run(oracle_cfg(g), u0, 3)[0])) <= 1e-13
    assert np.abs(got - ref).max() <= ADJ_TOL * np.abs(ref).max()


def _eps2_after(c, u0, al, dts):
    return oracle.eps2(c, oracle.run(c, u0, len(dts), alpha_in=al, dt_in=dts)[0])


def _richardson_fd(c, u0, al, dts, direction, h):
    """Central differences at h and h/2, Richardson-combined (error O(h^4))."""
    def cd(hh):
        return (_eps2_after(c, u0 + hh * direction, al, dts) - _eps2_after(c, u0 - hh * direction, al, dts)) / (2 * hh)
    a, b = cd(h), cd(h / 2)
    return (4 * b - a) / 3


def test_eps2_gradient_24cube_against_finite_differences():
    """Adjoint configuration at 24^3 (lumpy e, v = 0, seed 1604, WENO5, 50
    steps, checkpoint every 10).  The CFL number is scaled by 24/96 so that the
    50 steps cover the physical time of the 96^3 run (t ~ 2.2); at CFL 0.3 the
    coarse grid would run past t ~ 3, where the near-vacuum outflow turns
    unphysical.  d eps_2 / d e_0 at sampled cells (the hot-spot centres and two
    fixed cells) vs Richardson-extrapolated central differences of the oracle
    with the oracle's frozen speeds and steps."""
    from paper_1604_03360_gb300 import Hydro
    g, w = W.lumpy(n=(24, 24, 24), seed=1604)
    g.cfl = 0.3 * 24 / 96
    c = oracle_cfg(g)
    u0 = oracle.prim2con(w)
    _, _, _, al, dts = oracle.run(c, u0, 50, record=True)
    with Hydro.from_grid(g) as h:
        h.set_state(u0)
        h.forward_record(50, 10)
        uN = h.get_state()
        lam = np.empty_like(u0)
        h.eps2(uN, lam)
        grad = h.adjoint(lam)
    cent, _ = W.lumpy_params(1604)
    cells = [tuple(int((cc[d] + 6.0) / g.dx[d]) for d in (2, 1, 0)) for cc in cent[:4]] + [(12, 12, 12), (5, 18, 9)]
    fd = []
    for cell in cells:
        dirn = np.zeros_like(u0)
        dirn[(0,) + cell] = 1.0
        fd.append(_richardson_fd(c, u0, al, dts, dirn, 2e-5 * u0[(0,) + cell]))
    fd = np.array(fd)
    got = np.array([grad[(0,) + cell] for cell in cells])
    assert np.abs(got - fd).max() <= ADJ_TOL * np.abs(fd).max(), (got, fd)
    assert np.all(np.abs(got - fd) <= 1e-6 * np.abs(fd) + 1e-12)


def test_eps2_gradient_96cube_directional_derivative():
    """The adjoint configuration itself: 96^3, WENO5, 50 steps at CFL 0.3,
    checkpoint every 10.  <d eps_2/d e_0, delta> for a smooth bump delta vs a
    central difference of the oracle along delta (frozen speeds and steps)."""
    from paper_1604_03360_gb300 import Hydro
    g, w = W.lumpy(n=(96, 96, 96), seed=1604)
    c = oracle_cfg(g)
    u0 = oracle.prim2con(w)
    with Hydro.from_grid(g) as h:
        h.set_state(u0)
        h.forward_record(50, 10)
        uN = h.get_state()
        assert h.steps == 50 and 1.5 < h.t < 3.0, h.t
        lam = np.empty_like(u0)
        eps_gpu = h.eps2(uN, lam)
        grad = h.adjoint(lam)
    x, y, z = g.centres()
    bump = np.exp(-((x - 1.0) ** 2 + (y + 0.5) ** 2 + z ** 2) / 2.0)
    dirn = np.zeros_like(u0)
    dirn[0] = bump
    _, _, _, al, dts = oracle.run(c, u0, 50, record=True)
    hstep = 1e-5
    fd = (_eps2_after(c, u0 + hstep * dirn, al, dts) - _eps2_after(c, u0 - hstep * dirn, al, dts)) / (2 * hstep)
    got = float((grad[0] * bump).sum())
    assert abs(eps_gpu - _eps2_after(c, u0, al, dts)) <= 1e-12
    assert abs(got - fd) <= 1e-6 * abs(fd), (got, fd)

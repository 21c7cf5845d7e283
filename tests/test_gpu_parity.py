"""GPU (C-ABI) vs CPU oracle parity: element-wise, per field, within the
stated tolerance of 1e-11 (normwise relative error per field)."""
import numpy as np
import pytest

import oracle
import workloads as W
from parity import TOL, assert_parity, field_errors, oracle_cfg, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_03360_gb300.build as B
    B.build()
    oracle.build()


def with_flow(g, w, scale=0.3):
    """Add a smooth velocity field to data generated at rest."""
    x, y, z = g.centres()
    sh = w[0].shape
    w[1] = np.broadcast_to(scale * np.tanh(x / 3.0) * np.ones_like(y), sh)
    w[2] = np.broadcast_to(-0.5 * scale * np.tanh((y - 0.5) / 2.0) * np.ones_like(z), sh)
    w[3] = np.broadcast_to(0.4 * scale * np.sin(z / 2.0) * np.ones_like(x), sh)
    return w


@pytest.mark.parametrize("scheme", [5, 7])
def test_sod_full_config(scheme):
    """1+1D Sod tube, N = 400, CFL 0.4, to t = 0.4 (Sec. 3, Fig. 1 setup)."""
    g, w = W.sod(N=400, scheme=scheme)
    assert_parity(g, w, 100000, t0=0.0, t_end=0.4)


@pytest.mark.parametrize("scheme", [5, 7])
@pytest.mark.parametrize("dims", [(37, 29, 21), (16, 8, 40), (53, 11, 9)])
def test_ragged_lumpy_flow(scheme, dims):
    """Uneven grid spanning several 16 x 8 tiles and z chunks with ragged tails."""
    g, w = W.lumpy(n=dims, seed=sum(dims), scheme=scheme)
    w = with_flow(g, w)
    assert_parity(g, w, 6)


@pytest.mark.parametrize("scheme", [5, 7])
def test_periodic_smooth(scheme):
    g, w = W.smooth_periodic(n=(19, 13, 11), amp=0.3, vamp=0.5, seed=4, scheme=scheme)
    g.cfl = 0.4
    assert_parity(g, w, 8)


@pytest.mark.parametrize("dims", [(1, 1, 40), (1, 40, 1), (40, 1, 1), (23, 17, 1), (1, 19, 23), (21, 1, 18),
                                  (1, 1, 1), (2, 2, 2)])
def test_degenerate_dimensions(dims):
    g, w = W.lumpy(n=dims, seed=5, scheme=5)
    w = with_flow(g, w)
    assert_parity(g, w, 5)


def test_mixed_boundaries():
    g, w = W.smooth_periodic(n=(24, 17, 12), seed=8, scheme=7)
    g.bc = (1, 0, 1)
    assert_parity(g, w, 5)


@pytest.mark.parametrize("scheme", [5, 7])
def test_hubble_exact_init(scheme):
    g, w = W.hubble(N=40, scheme=scheme)
    assert_parity(g, w, 10, t0=g.t0)


@pytest.mark.parametrize("scheme", [7, 5])
def test_ellipsoidal_reduced_long_run(scheme):
    """Ellipsoidal flow (Sec. 3, Fig. 2 setup) at 48^3 for the full 200 steps.
    The CFL number is scaled by 48/256 so that the time step, and hence the
    physical time reached after 200 steps (t ~ 5.8), match the 256^3 run; at
    CFL 0.3 a coarse grid would run 5x longer, past the point where the
    near-vacuum corners (|v| -> 1) turn unphysical."""
    g, w = W.ellipsoidal(N=48, scheme=scheme)
    g.cfl = 0.3 * 48 / 256
    assert_parity(g, w, 200)


@pytest.mark.parametrize("scheme", [5, 7])
def test_hubble_full_size_128(scheme):
    """Hubble-like flow at the full 128^3 grid (exact-init, t0 = 10)."""
    g, w = W.hubble(N=128, scheme=scheme)
    assert_parity(g, w, 2, t0=g.t0)


def test_ellipsoidal_full_size_256_weno7():
    """The benchmark workload itself: 256^3 ellipsoidal flow, WENO7, two steps
    in the launch configuration the benchmark times."""
    g, w = W.ellipsoidal(N=256, scheme=7)
    assert_parity(g, w, 2)


def test_ellipsoidal_full_config_200_steps_stays_physical():
    """All 200 steps of the 256^3 WENO7 configuration: no unphysical state,
    the time reached matches the CFL rule, total energy only leaves through
    the outflow boundaries (it cannot grow)."""
    from paper_1604_03360_gb300 import Hydro
    g, w = W.ellipsoidal(N=256, scheme=7)
    with Hydro.from_grid(g) as h:
        h.set_primitive(w)
        e0 = h.get_state()[0].sum()
        h.step(200)
        u = h.get_state()
        assert h.steps == 200 and 5.0 < h.t < 6.5, (h.steps, h.t)
    assert np.isfinite(u).all()
    assert u[0].sum() <= e0 * (1 + 1e-12)
    M = np.sqrt(u[1] ** 2 + u[2] ** 2 + u[3] ** 2)
    assert (u[0] > M).all()


def test_t_end_stops_stepping():
    g, w = W.sod(N=120, scheme=5)
    ref, tr, kr = run_oracle(g, w, 100000, 0.0, 0.1)
    got, tg, kg = run_gpu(g, w, kr + 25, 0.0, 0.1)
    assert kg == kr and tg == pytest.approx(0.1, abs=1e-15)
    assert np.all(field_errors(got, ref) <= TOL)


def test_set_state_and_set_primitive_agree():
    g, w = W.lumpy(n=(20, 18, 16), seed=2)
    w = with_flow(g, w)
    u0 = oracle.prim2con(w)
    a, _, _ = run_gpu(g, w, 3, use_primitive=True)
    b, _, _ = run_gpu(g, w, 3, use_primitive=False, u0=u0)
    assert np.all(field_errors(a, b) <= 1e-13)


def test_bitwise_deterministic():
    g, w = W.ellipsoidal(N=36, scheme=7)
    a, _, _ = run_gpu(g, w, 5)
    b, _, _ = run_gpu(g, w, 5)
    assert np.array_equal(a, b)


def test_primitives_and_speeds():
    from paper_1604_03360_gb300 import Hydro
    g, w = W.lumpy(n=(17, 15, 13), seed=12)
    w = with_flow(g, w)
    u0 = oracle.prim2con(w)
    with Hydro.from_grid(g) as h:
        h.set_state(u0)
        p = h.get_primitive()
        a, _ = h.speeds()
    np.testing.assert_allclose(p, oracle.con2prim(u0), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(a, oracle.alpha(oracle_cfg(g), u0), rtol=1e-14)


def test_device_tensors_roundtrip():
    import torch
    from paper_1604_03360_gb300 import Hydro
    g, w = W.lumpy(n=(24, 20, 16), seed=13)
    u0 = oracle.prim2con(w)
    dev = torch.from_numpy(u0).cuda()
    with Hydro.from_grid(g) as h:
        h.set_state(dev)
        h.step(2)
        out = torch.empty_like(dev)
        h.get_state(out)
        host = h.get_state()
    assert np.array_equal(out.cpu().numpy(), host)
    ref = oracle.run(oracle_cfg(g), u0, 2)[0]
    assert np.all(field_errors(host, ref) <= TOL)


def test_unphysical_state_reported():
    from paper_1604_03360_gb300 import Hydro, HydroError
    g, w = W.lumpy(n=(10, 10, 10), seed=3)
    u0 = oracle.prim2con(w)
    u0[1, 4, 5, 6] = 3.0 * u0[0, 4, 5, 6]
    with Hydro.from_grid(g) as h:
        h.set_state(u0)
        with pytest.raises(HydroError) as ei:
            h.sync()
        assert ei.value.code == 4


# TMA-staged launches need an even nx (x rows a multiple of 16 bytes)
TMA_VARIANTS = {5: (10, 11), 7: (11, 12)}


@pytest.mark.parametrize("scheme,variant", [(5, 0), (5, 1), (5, 2), (5, 3), (5, 4), (5, 5), (5, 6), (5, 7), (5, 8),
                                            (5, 9), (5, 10), (5, 11), (5, 12), (5, 13), (5, 14),
                                            (7, 0), (7, 1), (7, 2), (7, 3), (7, 4), (7, 5), (7, 6), (7, 7),
                                            (7, 8), (7, 9), (7, 10), (7, 11), (7, 12), (7, 13), (7, 14),
                                            (7, 15), (7, 16), (7, 17)])
def test_every_launch_variant(scheme, variant):
    """Every compiled CTA tile shape, with a short z chunk so several chunks
    meet inside the grid, matches the oracle (ragged tiles in x and y)."""
    from paper_1604_03360_gb300 import Hydro
    nx = 38 if variant in TMA_VARIANTS[scheme] else 37
    g, w = W.lumpy(n=(nx, 29, 21), seed=77, scheme=scheme)
    w = with_flow(g, w)
    u0 = oracle.prim2con(w)
    ref = oracle.run(oracle_cfg(g), u0, 4)[0]
    with Hydro.from_grid(g) as h:
        h.set_launch(variant, 8)
        assert h.launch()[0] == variant and h.launch()[3] == 8
        h.set_state(u0)
        h.step(4)
        got = h.get_state()
    assert np.all(field_errors(got, ref) <= TOL)


# pairs of launch variants that must agree bit for bit: per-face tiles of
# other shapes and face orders, (per-face variant, pencil-sweep variant) with
# the same CTA tile, (pencil sweep on the FP64 unit only, pencil sweep with
# integer-pipe products) and (fused z faces, z faces from the z pass)
SWEEP_PAIRS = {5: ((0, 2), (0, 3), (0, 4), (1, 5), (4, 6), (6, 7), (7, 8), (8, 12), (12, 13), (13, 14)),
               7: ((0, 2), (0, 3), (1, 4), (3, 5), (5, 6), (6, 7), (7, 8), (8, 9), (7, 13), (13, 14), (14, 15), (15, 16), (16, 17))}


@pytest.mark.parametrize("scheme", [5, 7])
@pytest.mark.parametrize("n", [(37, 29, 21), (40, 1, 1), (1, 33, 9), (23, 1, 17), (18, 20, 1), (16, 16, 12)])
def test_pencil_sweep_matches_per_face_bitwise(scheme, n):
    """The pencil sweep carries stencil differences from face to face; it
    performs the same floating-point operations on the same operands as
    reconstructing every face afresh, so both give the same bits -- on full
    and ragged tiles and with one or two active in-plane axes.  The variant
    whose products run on the integer pipe must give the same bits too, and so
    must the variant whose z faces come from the separate z pass (z pencils
    swept with carried differences), and the three-pass variant (x, y and z
    faces from their own passes, then a per-cell combination)."""
    from paper_1604_03360_gb300 import Hydro
    g, w = W.lumpy(n=n, seed=91, scheme=scheme)
    w = with_flow(g, w)
    u0 = oracle.prim2con(w)
    for v_face, v_sweep in SWEEP_PAIRS[scheme]:
        out = []
        for v in (v_face, v_sweep):
            with Hydro.from_grid(g) as h:
                h.set_launch(v, 5)
                h.set_state(u0)
                h.step(3)
                out.append(h.get_state())
        assert np.array_equal(out[0], out[1]), (v_face, v_sweep)


# (variant without TMA, TMA-staged variant with the same arithmetic)
TMA_PAIRS = {5: ((9, 10), (8, 11), (6, 10)), 7: ((10, 11), (7, 12), (5, 11))}


@pytest.mark.parametrize("scheme", [5, 7])
@pytest.mark.parametrize("n,bc", [((38, 29, 21), (0, 0, 0)), ((40, 1, 1), (0, 0, 0)), ((2, 30, 9), (0, 0, 0)),
                                  ((16, 16, 12), (1, 1, 1)), ((34, 18, 1), (1, 0, 0)), ((50, 6, 7), (0, 1, 0))])
def test_tma_staged_variants_bitwise(scheme, n, bc):
    """The TMA-staged stage kernel reads in-grid cells from a tensor-map tile
    and out-of-grid cells (boundary rule) from global memory; it performs the
    same arithmetic as the kernel that loads every cell from global memory, so
    both give the same bits: ragged tiles, degenerate axes, periodic and
    outflow edges."""
    from paper_1604_03360_gb300 import Hydro
    g, w = W.lumpy(n=n, seed=93, scheme=scheme)
    w = with_flow(g, w)
    g.bc = bc
    u0 = oracle.prim2con(w)
    ref = oracle.run(oracle_cfg(g), u0, 3)[0]
    for v_plain, v_tma in TMA_PAIRS[scheme]:
        out = []
        for v in (v_plain, v_tma):
            with Hydro.from_grid(g) as h:
                h.set_launch(v, 5)
                h.set_state(u0)
                h.step(3)
                out.append(h.get_state())
        assert np.array_equal(out[0], out[1]), (v_plain, v_tma)
        assert np.all(field_errors(out[1], ref) <= TOL)


@pytest.mark.parametrize("scheme", [5, 7])
def test_tma_staged_variants_need_even_nx(scheme):
    from paper_1604_03360_gb300 import Hydro, HydroError
    g, w = W.lumpy(n=(37, 16, 12), seed=3, scheme=scheme)
    with Hydro.from_grid(g) as h:
        for v in TMA_VARIANTS[scheme]:
            with pytest.raises(HydroError) as ei:
                h.set_launch(v)
            assert ei.value.code == 1 and "even nx" in str(ei.value)
        h.set_primitive(w)
        h.autotune()                         # skips them
        assert h.launch()[0] not in TMA_VARIANTS[scheme]


def test_kernels_per_step_follows_the_launch():
    """A z-pass launch runs two kernels per RK3 stage when z is active, a fused
    one a single kernel, a three-pass one a pass per active axis and the
    combination; begin and end add two."""
    from paper_1604_03360_gb300 import Hydro
    for n, v, want in (((16, 16, 12), 7, 8), ((16, 16, 12), 5, 5), ((16, 16, 1), 7, 5), ((16, 16, 12), 13, 14),
                       ((16, 1, 12), 13, 11), ((16, 16, 1), 16, 11)):
        g, w = W.lumpy(n=n, seed=5, scheme=7)
        with Hydro.from_grid(g) as h:
            assert h.launch()[0] == 16         # the default launch (three-pass)
            h.set_launch(v)
            assert h.kernels_per_step() == want, (n, v)


def test_autotune_keeps_results(tmp_path, monkeypatch):
    from paper_1604_03360_gb300 import Hydro
    monkeypatch.setenv("HYDRO_TUNE_CACHE", str(tmp_path / "tune.txt"))
    g, w = W.ellipsoidal(N=40, scheme=7)
    u0 = oracle.prim2con(w)
    ref = oracle.run(oracle_cfg(g), u0, 3)[0]
    for attempt in range(2):          # second pass reads the cache
        with Hydro.from_grid(g) as h:
            h.set_state(u0)
            ms = h.autotune()
            assert (ms > 0) if attempt == 0 else (ms == -1.0)
            h.step(3)
            got = h.get_state()
        assert np.all(field_errors(got, ref) <= TOL)
    assert (tmp_path / "tune.txt").read_text().strip()


# ---------------------------------------------------------------- local Lax-Friedrichs
@pytest.mark.parametrize("scheme", [5, 7])
def test_local_lf_sod(scheme):
    g, w = W.sod(N=400, scheme=scheme)
    g.split = 1
    assert_parity(g, w, 100000, t0=0.0, t_end=0.4)


@pytest.mark.parametrize("scheme", [5, 7])
@pytest.mark.parametrize("dims", [(37, 29, 21), (23, 17, 1), (1, 19, 23)])
def test_local_lf_ragged(scheme, dims):
    g, w = W.lumpy(n=dims, seed=5 + sum(dims), scheme=scheme)
    w = with_flow(g, w)
    g.split = 1
    assert_parity(g, w, 6)


@pytest.mark.parametrize("scheme", [5, 7])
def test_local_lf_periodic_and_ellipsoidal(scheme):
    g, w = W.smooth_periodic(n=(19, 13, 11), amp=0.3, vamp=0.5, seed=4, scheme=scheme)
    g.split = 1
    assert_parity(g, w, 8)
    g, w = W.ellipsoidal(N=40, scheme=scheme)
    g.split = 1
    g.cfl = 0.3 * 40 / 256
    assert_parity(g, w, 40)


@pytest.mark.parametrize("scheme,variant", [(5, 0), (5, 1), (5, 2), (5, 3), (5, 4), (7, 0), (7, 1), (7, 2), (7, 3)])
def test_local_lf_every_launch_variant(scheme, variant):
    from paper_1604_03360_gb300 import Hydro
    g, w = W.lumpy(n=(37, 29, 21), seed=78, scheme=scheme)
    w = with_flow(g, w)
    g.split = 1
    u0 = oracle.prim2con(w)
    ref = oracle.run(oracle_cfg(g), u0, 4)[0]
    with Hydro.from_grid(g) as h:
        h.set_launch(variant, 8)
        h.set_state(u0)
        h.step(4)
        got = h.get_state()
    assert np.all(field_errors(got, ref) <= TOL)


# (ring variant, z-pass or three-pass variant) of the local-LF launches
LLF_PAIRS = {5: ((0, 2), (1, 3), (0, 4)), 7: ((0, 1), (0, 2), (0, 3))}


@pytest.mark.parametrize("scheme", [5, 7])
@pytest.mark.parametrize("n,bc", [((37, 29, 21), (0, 0, 0)), ((16, 16, 12), (1, 1, 1)), ((23, 17, 1), (0, 0, 0)),
                                  ((1, 19, 23), (0, 1, 0)), ((9, 8, 40), (0, 0, 1))])
def test_local_lf_zpass_matches_ring_bitwise(scheme, n, bc):
    """The local-LF z pass forms each z face from the same raw values with the
    same operations as the stage kernel's z ring, so both launches give the
    same bits (ragged tiles, several z chunks, periodic and outflow z); so do
    the local-LF three-pass launches (x, y and z passes, then the combination
    that also stores the speeds)."""
    from paper_1604_03360_gb300 import Hydro
    g, w = W.lumpy(n=n, seed=97, scheme=scheme)
    w = with_flow(g, w)
    g.bc, g.split = bc, 1
    u0 = oracle.prim2con(w)
    for v_ring, v_zp in LLF_PAIRS[scheme]:
        out = []
        for v in (v_ring, v_zp):
            with Hydro.from_grid(g) as h:
                h.set_launch(v, 6)
                h.set_state(u0)
                h.step(3)
                out.append(h.get_state())
        assert np.array_equal(out[0], out[1]), (v_ring, v_zp)


def test_local_lf_rejected_where_unsupported():
    from paper_1604_03360_gb300 import Hydro, HydroError
    g, w = W.lumpy(n=(12, 11, 10), seed=2)
    g.split = 1
    with Hydro.from_grid(g) as h:
        h.set_primitive(w)
        with pytest.raises(HydroError) as ei:
            h.forward_record(2, 1)
        assert ei.value.code == 1 and "global Lax-Friedrichs" in str(ei.value)


# ---------------------------------------------------------------- several charges
@pytest.mark.parametrize("scheme,split,nq", [(5, 0, 2), (7, 0, 3), (5, 1, 3), (7, 1, 2)])
def test_several_charges_match_oracle(scheme, split, nq):
    g, w = W.lumpy(n=(37, 29, 21), seed=90 + nq, scheme=scheme)
    w = with_flow(g, w)
    g.split, g.nq = split, nq
    assert_parity(g, W.with_charges(g, w, nq), 6)


@pytest.mark.parametrize("scheme,split,nq", [(5, 0, 2), (7, 0, 3), (5, 1, 3), (7, 1, 2)])
@pytest.mark.parametrize("n,bc", [((37, 29, 21), (0, 0, 0)), ((16, 16, 12), (1, 1, 1)), ((23, 17, 1), (0, 0, 0)),
                                  ((1, 19, 23), (0, 1, 0)), ((9, 8, 40), (0, 0, 1))])
def test_several_charges_three_pass_matches_stage_kernel_bitwise(scheme, split, nq, n, bc):
    """With several charges the three-pass launch (one warp per field in the
    x, y and z passes, then the combination) is the default; every face gets
    the same operations on the same operands as in the 16x8 stage kernel, so
    both give the same bits (ragged, degenerate, periodic and outflow axes)."""
    from paper_1604_03360_gb300 import Hydro
    g, w = W.lumpy(n=n, seed=71 + nq, scheme=scheme)
    w = with_flow(g, w)
    g.bc, g.split, g.nq = bc, split, nq
    wq = W.with_charges(g, w, nq)
    out = []
    for v in (0, 1):
        with Hydro.from_grid(g) as h:
            assert h.launch()[0] == 1          # the default for several charges
            h.set_launch(v, 6)
            h.set_primitive(wq)
            h.step(3)
            out.append(h.get_state())
            if v == 1:
                assert h.kernels_per_step() == 2 + 3 * (1 + sum(int(m > 1) for m in n))
    assert out[0].shape[0] == 4 + nq
    assert np.array_equal(out[0], out[1])


def test_extra_charges_evolve_like_the_single_charge():
    from paper_1604_03360_gb300 import Hydro
    g, w = W.lumpy(n=(30, 26, 22), seed=61, scheme=5)
    w = with_flow(g, w)
    w3 = W.with_charges(g, w, 3)
    g.nq = 3
    with Hydro.from_grid(g) as h:
        h.set_primitive(w3)
        h.step(5)
        u3 = h.get_state()
        p3 = h.get_primitive()
    assert u3.shape[0] == 7
    g.nq = 1
    for j in (4, 5, 6):
        wj = w3[:5].copy()
        wj[4] = w3[j]
        with Hydro.from_grid(g) as h:
            h.set_primitive(wj)
            h.step(5)
            u1 = h.get_state()
        assert np.abs(u1[4] - u3[j]).max() <= 1e-14 * np.abs(u1[4]).max()
        assert np.all(field_errors(u3[:4], u1[:4]) <= 1e-14)
    np.testing.assert_allclose(p3, oracle.con2prim(u3), rtol=1e-12, atol=1e-14)


def test_several_charges_rejected_where_unsupported():
    from paper_1604_03360_gb300 import Hydro, HydroBatch, HydroError
    g, w = W.lumpy(n=(12, 11, 10), seed=2)
    g.nq = 2
    with pytest.raises(HydroError):
        HydroBatch([g, g])
    with Hydro.from_grid(g) as h:
        h.set_primitive(W.with_charges(g, w, 2))
        with pytest.raises(HydroError):
            h.forward_record(2, 1)


# ---------------------------------------------------------------- MUSTA-FORCE + MUSCL
@pytest.mark.parametrize("limiter,stages", [(0, 2), (1, 1), (2, 3), (3, 2)])
def test_musta_sod(limiter, stages):
    g, w = W.sod(N=400, scheme=5)
    g.scheme, g.limiter, g.musta_stages = 2, limiter, stages
    assert_parity(g, w, 100000, t0=0.0, t_end=0.4)


@pytest.mark.parametrize("dims", [(37, 29, 21), (23, 17, 1), (1, 19, 23), (16, 16, 40)])
def test_musta_ragged_and_degenerate(dims):
    g, w = W.lumpy(n=dims, seed=7 + sum(dims), scheme=5)
    w = with_flow(g, w)
    g.scheme, g.limiter = 2, 1
    assert_parity(g, w, 6)


@pytest.mark.parametrize("variant", [0, 1])
def test_musta_periodic_and_variants(variant):
    from paper_1604_03360_gb300 import Hydro
    g, w = W.smooth_periodic(n=(19, 13, 11), amp=0.3, vamp=0.5, seed=4, scheme=5)
    g.scheme, g.limiter = 2, 2
    u0 = oracle.prim2con(w)
    ref = oracle.run(oracle_cfg(g), u0, 8)[0]
    with Hydro.from_grid(g) as h:
        h.set_launch(variant, 6)
        h.set_state(u0)
        h.step(8)
        got = h.get_state()
    assert np.all(field_errors(got, ref) <= TOL)


def test_musta_ellipsoidal():
    g, w = W.ellipsoidal(N=40, scheme=5)
    g.scheme, g.cfl = 2, 0.3 * 40 / 256
    assert_parity(g, w, 40)


def test_musta_rejected_where_unsupported():
    from paper_1604_03360_gb300 import Hydro, HydroBatch, HydroError
    g, w = W.lumpy(n=(12, 11, 10), seed=2)
    g.scheme = 2
    with pytest.raises(HydroError):
        HydroBatch([g])
    with Hydro.from_grid(g) as h:
        h.set_primitive(w)
        with pytest.raises(HydroError):
            h.forward_record(2, 1)
    g.split = 1
    with pytest.raises(HydroError):
        Hydro.from_grid(g)


# ---------------------------------------------------------------- characteristic-wise WENO
@pytest.mark.parametrize("scheme", [5, 7])
def test_charwise_sod(scheme):
    g, w = W.sod(N=400, scheme=scheme)
    g.charwise = 1
    assert_parity(g, w, 100000, t0=0.0, t_end=0.4)


@pytest.mark.parametrize("scheme", [5, 7])
@pytest.mark.parametrize("dims", [(37, 29, 21), (23, 17, 1), (1, 19, 23), (1, 1, 40)])
def test_charwise_ragged_and_degenerate(scheme, dims):
    g, w = W.lumpy(n=dims, seed=17 + sum(dims), scheme=scheme)
    w = with_flow(g, w)
    g.charwise = 1
    assert_parity(g, w, 6)


@pytest.mark.parametrize("scheme", [5, 7])
def test_charwise_periodic_and_ellipsoidal(scheme):
    g, w = W.smooth_periodic(n=(19, 13, 11), amp=0.3, vamp=0.5, seed=4, scheme=scheme)
    g.charwise = 1
    assert_parity(g, w, 8)
    g, w = W.ellipsoidal(N=40, scheme=scheme)
    g.charwise = 1
    g.cfl = 0.3 * 40 / 256
    assert_parity(g, w, 40)


@pytest.mark.parametrize("scheme,nq", [(5, 2), (7, 3)])
def test_charwise_several_charges(scheme, nq):
    g, w = W.lumpy(n=(37, 29, 21), seed=40 + nq, scheme=scheme)
    w = with_flow(g, w)
    g.charwise, g.nq = 1, nq
    assert_parity(g, W.with_charges(g, w, nq), 6)


@pytest.mark.parametrize("scheme,variant", [(5, 0), (5, 1), (5, 2), (5, 3), (5, 4), (7, 0), (7, 1), (7, 2), (7, 3)])
def test_charwise_every_launch_variant(scheme, variant):
    """Fused stage kernels (WENO5 0, 1; WENO7 0) and the face passes + the
    combination (the rest) against the oracle."""
    from paper_1604_03360_gb300 import Hydro
    g, w = W.lumpy(n=(37, 29, 21), seed=79, scheme=scheme)
    w = with_flow(g, w)
    g.charwise = 1
    u0 = oracle.prim2con(w)
    ref = oracle.run(oracle_cfg(g), u0, 4)[0]
    with Hydro.from_grid(g) as h:
        h.set_launch(variant, 8)
        h.set_state(u0)
        h.step(4)
        got = h.get_state()
    assert np.all(field_errors(got, ref) <= TOL)


@pytest.mark.parametrize("scheme,nq", [(5, 2), (7, 3)])
@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("n,bc", [((37, 29, 21), (0, 0, 0)), ((16, 15, 12), (1, 1, 1)), ((1, 19, 23), (0, 1, 0))])
def test_charwise_charges_every_launch_variant(scheme, nq, variant, n, bc):
    """Several charges, characteristic-wise: the 16x8 stage kernel (0) and the
    face passes (1-3) against the oracle, ragged, periodic and degenerate."""
    from paper_1604_03360_gb300 import Hydro
    g, w = W.lumpy(n=n, seed=83 + nq, scheme=scheme)
    w = with_flow(g, w)
    g.bc, g.charwise, g.nq = bc, 1, nq
    wq = W.with_charges(g, w, nq)
    u0 = oracle.prim2con(wq)
    ref = oracle.run(oracle_cfg(g), u0, 4)[0]
    with Hydro.from_grid(g) as h:
        h.set_launch(variant, 8)
        h.set_state(u0)
        h.step(4)
        got = h.get_state()
    assert np.all(field_errors(got, ref) <= TOL)


def test_charwise_rejected_where_unsupported():
    from paper_1604_03360_gb300 import Hydro, HydroBatch, HydroError
    g, w = W.lumpy(n=(12, 11, 10), seed=2)
    g.charwise = 1
    with pytest.raises(HydroError):
        HydroBatch([g])
    with Hydro.from_grid(g) as h:
        h.set_primitive(w)
        with pytest.raises(HydroError):
            h.forward_record(2, 1)


# ---------------------------------------------------------------- general EOS p = cs2 (e - m n)
@pytest.mark.parametrize("scheme,split", [(5, 0), (7, 0), (5, 1)])
def test_gas_shock_tube(scheme, split):
    g, w = W.gas_sod(N=400, scheme=scheme)
    g.split = split
    assert_parity(g, w, 100000, t0=0.0, t_end=0.4)


def _gas_lumpy(dims, seed, scheme, m=1.0):
    g, w = W.lumpy(n=dims, seed=seed, scheme=scheme)
    w = with_flow(g, w)
    w[0] = w[0] + m * w[4]            # internal energy e - m n stays positive
    g.cs2, g.mass = 2.0 / 3.0, m
    return g, w


@pytest.mark.parametrize("scheme", [5, 7])
@pytest.mark.parametrize("dims", [(37, 29, 21), (23, 17, 1), (1, 1, 40)])
def test_gas_ragged_and_degenerate(scheme, dims):
    g, w = _gas_lumpy(dims, 7 + sum(dims), scheme)
    assert_parity(g, w, 6)


def test_gas_periodic_local_lf_and_charges():
    g, w = W.smooth_periodic(n=(19, 13, 11), amp=0.3, vamp=0.5, seed=4, scheme=7)
    w[0] = w[0] + 0.5 * w[4]
    g.cs2, g.mass, g.split = 0.4, 0.5, 1
    assert_parity(g, w, 8)
    g, w = _gas_lumpy((30, 22, 18), 3, 5)
    g.nq = 3
    assert_parity(g, W.with_charges(g, w, 3), 5)


def test_gas_primitives_read_back():
    from paper_1604_03360_gb300 import Hydro
    g, w = _gas_lumpy((20, 18, 16), 12, 5)
    with Hydro.from_grid(g) as h:
        h.set_primitive(w)
        h.step(3)
        u = h.get_state()
        p = h.get_primitive()
    ref = oracle.con2prim(u, g.cs2, g.mass)
    assert np.abs(p - ref).max() <= 1e-13 * np.abs(ref).max()


def test_gas_rejected_where_unsupported():
    from paper_1604_03360_gb300 import Hydro, HydroBatch, HydroError
    g, w = _gas_lumpy((12, 11, 10), 2, 5)
    with pytest.raises(HydroError):
        HydroBatch([g])
    with Hydro.from_grid(g) as h:
        h.set_primitive(w)
        with pytest.raises(HydroError):
            h.forward_record(2, 1)
        with pytest.raises(HydroError):
            h.eps2()
    for kw in (dict(scheme=2), dict(charwise=1)):
        for k, v in kw.items():
            setattr(g, k, v)
        with pytest.raises(HydroError):
            Hydro.from_grid(g)
        g.scheme, g.charwise = 5, 0

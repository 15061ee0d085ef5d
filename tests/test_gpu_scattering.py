"""First-order diffuse scattering (rt_set_scattering, rt_scattering_gain;
Sec. II-B) against the FP64 oracle over the same lattice rays."""
import numpy as np
import pytest

from oracle import oracle as O
from oracle import scattering as SC
from paper_2303_11103_gb300 import rt
from paper_2303_11103_gb300 import scenes as S

from gpu_helpers import FC, setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tracer():
    tr = rt.Tracer(0, FC)
    yield tr
    tr.close()


def test_scattering_matches_oracle(tracer):
    sc = S.tiny_scene()
    tx = S.Devices(np.array([[-60.0, 0.0, 25.0]], np.float32), np.array([[0.2, 0.05, 0.0]], np.float32),
                   S.TR38901_VH)
    rx = S.Devices(np.array([[-75.0, 0.0, 1.5], [60.0, 10.0, 1.5], [30.0, 25.0, 1.5], [-20.0, -40.0, 6.0]],
                            np.float32), np.array([[0.5, 0.0, 0.0]] * 4, np.float32),
                   S.Antenna(S.ANT_DIPOLE, (np.pi / 4, -np.pi / 4)))
    setup(tracer, sc, tx, rx)
    N = 20000
    assert float(tracer.scattering_gain(N).abs().sum()) == 0.0      # no coefficients set: no scattering
    S_m = np.array([0.5], np.float32)
    tracer.set_scattering(S_m)
    g = tracer.scattering_gain(N).cpu().numpy()
    og = SC.scattering_gain(O.make_scene(sc), sc.mat_id, S_m.astype(np.float64), FC, tx, rx, N)
    assert g.shape == og.shape == (4, 2, 2)
    assert (og > 0).sum() >= 8
    # a lattice ray whose decision is near-degenerate may land on either side: 1e-3 of the total
    assert np.all(np.abs(g - og) <= 2e-3 * og + 1e-3 * og.sum(axis=(1, 2), keepdims=True)), (g, og)
    with pytest.raises(rt.RtError):
        tracer.set_scattering(np.zeros(3, np.float32))


@pytest.mark.parametrize("uneven", [False, True])
def test_scattering_several_transmitters(tracer, uneven):
    """Three transmitters, a ray count that is no multiple of the warp width
    (warps straddle two transmitters), all pairs or uneven receiver sets
    (one empty): every pair's gain equals the oracle's for its transmitter."""
    sc = S.tiny_scene()
    tx = S.Devices(np.array([[-60.0, 0.0, 25.0], [0.0, 50.0, 10.0], [45.0, -30.0, 3.0]], np.float32),
                   np.array([[0.2, 0.05, 0.0], [1.5, 0.0, 0.1], [-2.0, 0.0, 0.0]], np.float32), S.TR38901_VH)
    rx = S.Devices(np.array([[-75.0, 0.0, 1.5], [60.0, 10.0, 1.5], [30.0, 25.0, 1.5], [-20.0, -40.0, 6.0],
                             [10.0, 70.0, 2.0], [-40.0, 30.0, 1.5]], np.float32),
                   np.array([[0.5, 0.0, 0.0]] * 6, np.float32), S.Antenna(S.ANT_DIPOLE, (0.0,)))
    off = [0, 4, 4, 6] if uneven else None
    setup(tracer, sc, tx, rx, off)
    N = 4999
    S_m = np.array([0.7], np.float32)
    tracer.set_scattering(S_m)
    g = tracer.scattering_gain(N).cpu().numpy()
    osc = O.make_scene(sc)
    n_pairs = 6 if uneven else 18
    assert g.shape == (n_pairs, 1, 2)
    live = 0
    for t in range(3):
        rs = range(off[t], off[t + 1]) if uneven else range(6)
        if len(rs) == 0:
            continue
        sub = S.Devices(rx.pos[list(rs)], rx.ypr[list(rs)], rx.antenna)
        og = SC.scattering_gain(osc, sc.mat_id, S_m.astype(np.float64), FC, tx, sub, N, tx_index=t)
        got = g[list(rs)] if uneven else g[t * 6:(t + 1) * 6]
        assert np.all(np.abs(got - og) <= 2e-3 * og + 1e-3 * og.sum(axis=(1, 2), keepdims=True)), (t, got, og)
        live += int((og > 0).any(axis=(1, 2)).sum())
    assert live >= 4


def test_scattering_vjp_matches_oracle(tracer):
    """dL/dS of the scattered gain (three materials, random upstream
    gradient) against the oracle's derivative of the definition."""
    sc = S.tiny_scene_3mat()
    tx = S.Devices(np.array([[-50.0, -50.0, 20.0]], np.float32), np.zeros((1, 3), np.float32), S.TR38901_VH)
    rx = S.Devices(np.array([[-75.0, 0.0, 1.5], [60.0, 10.0, 1.5], [30.0, 25.0, 1.5], [-20.0, -40.0, 6.0]],
                            np.float32), np.zeros((4, 3), np.float32), S.Antenna(S.ANT_DIPOLE, (0.0,)))
    setup(tracer, sc, tx, rx)
    S_m = np.array([0.4, 0.7, 0.0], np.float32)
    tracer.set_scattering(S_m)
    N = 10000
    up = np.random.default_rng(1).normal(size=(4, 1, 2)).astype(np.float32)
    gs = tracer.scattering_gain_vjp(N, up).cpu().numpy()
    og = SC.scattering_gain_vjp(O.make_scene(sc), sc.mat_id, S_m.astype(np.float64), FC, tx, rx, N, up)
    assert gs.shape == (3,) and gs[2] == 0.0 and np.abs(og[:2]).min() > 0
    assert np.allclose(gs, og, rtol=3e-3, atol=2e-3 * np.abs(og).max()), (gs, og)
    with pytest.raises(rt.RtError):
        tracer.scattering_gain_vjp(N, np.zeros(5, np.float32))


def test_directive_pattern_matches_oracle(tracer):
    """Per-material patterns (Lambertian, directive alpha_R = 3 and 8) for
    the gain and its VJP; exponents out of range are rejected."""
    sc = S.tiny_scene_3mat()
    tx = S.Devices(np.array([[-50.0, -50.0, 20.0]], np.float32), np.array([[0.3, 0.1, 0.0]], np.float32),
                   S.TR38901_VH)
    rx = S.Devices(np.array([[-75.0, 0.0, 1.5], [60.0, 10.0, 1.5], [30.0, 25.0, 1.5], [-20.0, -40.0, 6.0]],
                            np.float32), np.zeros((4, 3), np.float32), S.Antenna(S.ANT_DIPOLE, (0.0, np.pi / 2)))
    setup(tracer, sc, tx, rx)
    S_m = np.array([0.5, 0.6, 0.7], np.float32)
    alpha = np.array([-1, 3, 8], np.int32)
    tracer.set_scattering(S_m)
    tracer.set_scattering_pattern(alpha)
    N = 20000
    osc = O.make_scene(sc)
    g = tracer.scattering_gain(N).cpu().numpy()
    og = SC.scattering_gain(osc, sc.mat_id, S_m.astype(np.float64), FC, tx, rx, N, alpha=alpha)
    assert (og > 0).sum() >= 12
    assert np.all(np.abs(g - og) <= 2e-3 * og + 1e-3 * og.sum(axis=(1, 2), keepdims=True)), (g, og)
    up = np.random.default_rng(2).normal(size=(4, 2, 2)).astype(np.float32)
    gs = tracer.scattering_gain_vjp(N, up).cpu().numpy()
    ogs = SC.scattering_gain_vjp(osc, sc.mat_id, S_m.astype(np.float64), FC, tx, rx, N, up, alpha=alpha)
    assert np.allclose(gs, ogs, rtol=3e-3, atol=2e-3 * np.abs(ogs).max()), (gs, ogs)
    for bad in ([-2, 0, 0], [0, 65, 0], [0, 0]):
        with pytest.raises(rt.RtError):
            tracer.set_scattering_pattern(bad)


def test_scattering_many_receivers():
    """200 receivers: each ray's receivers are split over several threads
    (three chunks, the last one shorter); the gain and its VJP equal the
    oracle's."""
    tr = rt.Tracer(0, FC)
    try:
        sc = S.tiny_scene()
        tx = S.Devices(np.array([[-60.0, -20.0, 25.0]], np.float32), np.zeros((1, 3), np.float32), S.TR38901_VH)
        rng = np.random.default_rng(7)
        xy = rng.uniform(-95.0, 95.0, size=(400, 2))
        xy = xy[(np.abs(xy[:, 0]) > 12.0) | (np.abs(xy[:, 1]) > 12.0)][:200]
        rx = S.Devices(np.concatenate([xy, np.full((200, 1), 1.5)], 1).astype(np.float32), np.zeros((200, 3), np.float32),
                       S.V_ISO)
        setup(tr, sc, tx, rx)
        S_m = np.array([0.6], np.float32)
        tr.set_scattering(S_m)
        N = 2000
        g = tr.scattering_gain(N).cpu().numpy()
        og = SC.scattering_gain(O.make_scene(sc), sc.mat_id, S_m.astype(np.float64), FC, tx, rx, N)
        assert (og > 0).sum() > 150
        assert np.all(np.abs(g - og) <= 2e-3 * og + 1e-3 * og.sum(axis=(1, 2), keepdims=True)), (g, og)
        up = rng.normal(size=(200, 1, 2)).astype(np.float32)
        gs = tr.scattering_gain_vjp(N, up).cpu().numpy()
        ogs = SC.scattering_gain_vjp(O.make_scene(sc), sc.mat_id, S_m.astype(np.float64), FC, tx, rx, N, up)
        scale = 2.0 / float(S_m[0]) * float(np.sum(np.abs(up) * og))   # bound of |dL/dS|
        assert np.allclose(gs, ogs, rtol=3e-3, atol=2e-3 * scale), (gs, ogs, scale)
    finally:
        tr.close()


def test_negative_coefficient_scatters_nothing(tracer):
    """A coefficient <= 0 scatters nothing, in the gain and in its VJP."""
    sc = S.tiny_scene_3mat()
    tx = S.Devices(np.array([[-50.0, -50.0, 20.0]], np.float32), np.zeros((1, 3), np.float32), S.TR38901_VH)
    rx = S.Devices(np.array([[-75.0, 0.0, 1.5], [-20.0, -40.0, 6.0]], np.float32), np.zeros((2, 3), np.float32),
                   S.V_ISO)
    setup(tracer, sc, tx, rx)
    S_m = np.array([-0.5, 0.6, 0.0], np.float32)
    tracer.set_scattering(S_m)
    N = 5000
    g = tracer.scattering_gain(N).cpu().numpy()
    og = SC.scattering_gain(O.make_scene(sc), sc.mat_id, S_m.astype(np.float64), FC, tx, rx, N)
    assert np.all(np.abs(g - og) <= 2e-3 * og + 1e-3 * og.sum(axis=(1, 2), keepdims=True)), (g, og)
    gs = tracer.scattering_gain_vjp(N, np.ones((2, 1, 2), np.float32)).cpu().numpy()
    assert gs[0] == 0.0 and gs[2] == 0.0 and gs[1] > 0.0

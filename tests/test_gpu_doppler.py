"""Time evolution of the CIR from the devices' motion (rt_apply_doppler,
Sec. II-A Listing 3) against the FP64 oracle on the same paths: with the
paper's example settings (1 MHz sampling, 14 time steps, a transmitter
moving at [3, 0, 0] m/s) and with moving receivers too."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2303_11103_gb300 import rt
from paper_2303_11103_gb300 import scenes as S

from gpu_helpers import A_ABS, A_REL, FC, compare_path_sets, gpu_paths, setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tracer():
    tr = rt.Tracer(0, FC)
    yield tr
    tr.close()


def _case(tracer, case):
    if case == "tiny_visible":
        sc = S.tiny_scene()
        tx, rx = S.tiny_devices(visible=True)
        N, D = 10000, 2
    else:
        sc = S.city_scene(n_side=6, size=150.0, seed=5)
        tx, rx = S.city_devices(sc, n_rx=24, half=70.0)
        N, D = 20000, 3
    setup(tracer, sc, tx, rx)
    tracer.compute_paths(D, N)
    gsets, p = gpu_paths(tracer)
    osc = O.make_scene(sc)
    ora_paths, ora_c = O.compute_paths(osc, tx.pos[0], rx.pos, D, N)
    common = compare_path_sets(osc, tx.pos[0], rx.pos, gsets, ora_paths, ora_c)
    sel = [q for q in ora_paths if q.valid]
    return osc, tx, rx, gsets, p["offsets"].cpu().numpy(), sel, common


@pytest.mark.parametrize("case", ["tiny_visible", "small_city"])
@pytest.mark.parametrize("moving_rx", [False, True])
def test_doppler_matches_oracle(tracer, case, moving_rx):
    osc, tx, rx, gsets, off, sel, common = _case(tracer, case)
    fs, T = 1e6, 14
    vt = np.array([[3.0, 0.0, 0.0]], np.float32)
    vr = (np.random.default_rng(7).normal(0.0, 2.0, (len(rx.pos), 3)).astype(np.float32) if moving_rx else None)
    a, _ = tracer.cir()
    at = tracer.apply_doppler(a, fs, T, vt, vr).cpu().numpy()
    a = a.cpu().numpy()
    assert at.shape == a.shape + (T,)
    # t = 0 is the CIR itself, and the modulus does not change
    assert np.array_equal(at[..., 0], a)
    assert np.allclose(np.abs(at), np.abs(a)[..., None], rtol=1e-5, atol=0)
    oa, _ = O.path_field(osc, FC, tx, rx, 0, sel)
    oat = O.doppler(oa, sel, tx.pos[0], rx.pos, FC, fs, T, vt[0], vr)
    idx = {(q.rx, q.seq): i for i, q in enumerate(sel)}
    n = 0
    for r in range(len(rx.pos)):
        amax = max([np.abs(oa[idx[(r, s)]]).max() for s in common[r]] + [0.0])
        for k, s in enumerate(gsets[r]):
            if s not in common[r]:
                continue
            i, j = off[r] + k, idx[(r, s)]
            # end to end against the oracle's coefficients
            err = np.abs(at[i] - oat[j])
            assert np.all(err <= A_REL * np.abs(oat[j]) + A_ABS * amax), (s, at[i], oat[j])
            # the time evolution alone: the oracle's Doppler on the GPU's own a
            ref = O.doppler(a[i:i + 1].astype(np.complex128), [sel[j]], tx.pos[0], rx.pos, FC, fs, T, vt[0], vr)[0]
            assert np.all(np.abs(at[i] - ref) <= 2e-5 * np.abs(a[i])[..., None] + 1e-30), (s, at[i], ref)
            n += 1
    assert n >= 4


def test_doppler_arguments(tracer):
    _case(tracer, "tiny_visible")
    a, _ = tracer.cir()
    with pytest.raises(rt.RtError):
        tracer.apply_doppler(a, 1e6, 0, [3.0, 0.0, 0.0])
    with pytest.raises(rt.RtError):
        tracer.apply_doppler(a, -1.0, 4, [3.0, 0.0, 0.0])
    # devices at rest: every time step is the CIR
    at = tracer.apply_doppler(a, 1e6, 5, [0.0, 0.0, 0.0]).cpu().numpy()
    assert np.array_equal(at, np.repeat(a.cpu().numpy()[..., None], 5, axis=-1))


def test_doppler_and_array_per_transmitter(tracer):
    """Two transmitters with their own velocities and orientations: each path
    takes its own transmitter's (Doppler against the oracle, array phases
    against the oracle on the GPU's own coefficients)."""
    sc = S.tiny_scene()
    _, rx = S.tiny_devices(visible=True)
    tx = S.Devices(np.array([[-60.0, 0.0, 25.0], [-50.0, 30.0, 20.0]], np.float32),
                   np.array([[0.3, 0.0, 0.0], [-1.2, 0.1, 0.2]], np.float32), S.TR38901_VH)
    setup(tracer, sc, tx, rx)
    tracer.compute_paths(2, 20000)
    gsets, p = gpu_paths(tracer)
    a, _ = tracer.cir()
    vt = np.array([[3.0, 0.0, 0.0], [0.0, -2.0, 1.0]], np.float32)
    at = tracer.apply_doppler(a, 1e6, 6, vt).cpu().numpy()
    el = rt.planar_array(2, 2, 0.5, 0.5, O.C0 / FC)
    ael = tracer.apply_array(a, el).cpu().numpy()
    a = a.cpu().numpy()
    off = p["offsets"].cpu().numpy()
    osc = O.make_scene(sc)
    n = 0
    for t in range(2):
        ora, _ = O.compute_paths(osc, tx.pos[t], rx.pos, 2, 20000)
        byseq = {q.seq: q for q in ora if q.valid}
        for k, s in enumerate(gsets[t]):   # pair t: transmitter t, receiver 0
            if s not in byseq:
                continue
            i = off[t] + k
            q = byseq[s]
            q0 = O.OPath(0, q.seq, q.valid, q.margin, q.points, q.length)
            ref = O.doppler(a[i:i + 1].astype(np.complex128), [q0], tx.pos[t], rx.pos, FC, 1e6, 6, vt[t])[0]
            assert np.all(np.abs(at[i] - ref) <= 2e-5 * np.abs(a[i])[..., None] + 1e-30)
            refa = O.array_response(a[i:i + 1].astype(np.complex128), [q0], tx.pos[t], tx.ypr[t], rx.pos, rx.ypr,
                                    FC, el, np.zeros((1, 3)))[0]
            assert np.all(np.abs(ael[i] - refa) <= 3e-5 * np.abs(refa) + 1e-12)
            n += 1
    assert n >= 4

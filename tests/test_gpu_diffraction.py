"""First-order edge diffraction (rt_compute_diffraction, rt_diffraction_cir;
Sec. II-B) against the FP64 UTD oracle on the same scenes: the wedge list,
the set of diffracted paths (decisions the oracle marks near-degenerate
excused) and their coefficients and delays."""
import numpy as np
import pytest

from oracle import diffraction as DF
from oracle import oracle as O
from paper_2303_11103_gb300 import rt
from paper_2303_11103_gb300 import scenes as S

from gpu_helpers import A_ABS, A_REL, FC, TAU_REL, setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tracer():
    tr = rt.Tracer(0, FC)
    yield tr
    tr.close()


def _case(case):
    if case == "tiny":
        sc = S.tiny_scene()
        tx, _ = S.tiny_devices()
        rx = S.Devices(np.array([[30.0, 25.0, 1.5], [40.0, -30.0, 1.5], [-75.0, 0.0, 1.5], [60.0, 10.0, 1.5]],
                                np.float32), np.zeros((4, 3), np.float32), S.V_ISO)
    else:
        sc = S.city_scene(n_side=6, size=150.0, seed=5)
        tx, rx = S.city_devices(sc, n_rx=16, half=70.0, tx_antenna=S.TR38901_VH)
        rx = S.Devices(rx.pos, rx.ypr + np.float32([0.3, 0.1, -0.2]), S.Antenna(S.ANT_DIPOLE, (np.pi / 4, -np.pi / 4)))
    return sc, tx, rx


@pytest.mark.parametrize("case", ["tiny", "small_city"])
def test_diffraction_matches_oracle(tracer, case):
    sc, tx, rx = _case(case)
    setup(tracer, sc, tx, rx)
    P = tracer.compute_diffraction()
    faces, ne = (x.cpu().numpy() for x in tracer.wedges())
    ws = DF.wedges(sc.verts)
    # the same wedges (keyed by their two faces) with the same exterior angles
    ora_w = {(w.f0, w.f1): i for i, w in enumerate(ws)}
    assert sorted(ora_w) == sorted(tuple(f) for f in faces)
    for k, f in enumerate(faces):
        assert abs(ne[k] - ws[ora_w[tuple(f)]].n) < 1e-6
    d = tracer.diffraction()
    off, wed, pts = (d[k].cpu().numpy() for k in ("offsets", "wedge", "points"))
    assert P == len(wed) and off[-1] == P
    gpu = {}
    for r in range(len(rx.pos)):
        for i in range(off[r], off[r + 1]):
            gpu[(r, ora_w[tuple(faces[wed[i]])])] = i
    osc = O.make_scene(sc)
    osel = []
    n_common = 0
    for r in range(len(rx.pos)):
        for wi, w in enumerate(ws):
            ok, D, m = DF.evaluate(osc, w, tx.pos[0], rx.pos[r])
            on_gpu = (r, wi) in gpu
            if ok != on_gpu:
                assert m < max(osc.eps, 1e-3), (r, wi, ok, m)   # near-degenerate decision
                continue
            if ok:
                i = gpu[(r, wi)]
                assert np.linalg.norm(pts[i] - D) < 1e-3
                osel.append((i, DF.DPath(r, wi, D, 0.0, m)))
                n_common += 1
    assert n_common >= (3 if case == "tiny" else 10)
    a, tau = (x.cpu().numpy() for x in tracer.diffraction_cir())
    oa, otau = DF.diffracted_field(ws, [p for _, p in osel], FC, tx, rx)
    for r in range(len(rx.pos)):
        js = [j for j, (i, p) in enumerate(osel) if p.rx == r]
        if not js:
            continue
        amax = max(np.abs(oa[j]).max() for j in js)
        for j in js:
            i = osel[j][0]
            assert abs(tau[i] - otau[j]) <= TAU_REL * otau[j]
            if osel[j][1].margin < 1e-3:
                continue   # on a shadow or reflection boundary: one term's sign is a rounding decision
            err = np.abs(a[i] - oa[j])
            assert np.all(err <= A_REL * np.abs(oa[j]) + A_ABS * amax), (r, osel[j][1].wedge, a[i], oa[j])


def test_diffraction_empty_and_rescene(tracer):
    """No wedges in a ground-only scene; a new scene rebuilds the wedges."""
    sc = S.ground_only_scene(100.0)
    tx, rx = S.tiny_devices()
    setup(tracer, sc, tx, rx)
    assert tracer.compute_diffraction() == 0
    assert tracer.wedges()[0].shape[0] == 0
    sc2, tx2, rx2 = _case("tiny")
    setup(tracer, sc2, tx2, rx2)
    assert tracer.wedges()[0].shape[0] == 12
    assert tracer.compute_diffraction() > 0


def test_diffraction_uneven_receiver_sets(tracer):
    """Several transmitters with uneven receiver sets (one empty): every
    pair's diffracted paths equal the oracle's for that transmitter."""
    sc = S.city_scene(n_side=6, size=150.0, seed=5)
    tx, rx = S.city_devices(sc, n_rx=12, half=70.0)
    tx3 = S.Devices(np.concatenate([tx.pos, tx.pos + np.float32([[-5.0, 3.0, 2.0]]), tx.pos + np.float32([[4.0, 4.0, 0.0]])]),
                    np.zeros((3, 3), np.float32), tx.antenna)
    off = [0, 5, 5, 12]
    setup(tracer, sc, tx3, rx, off)
    tracer.compute_diffraction()
    faces = [tuple(f) for f in tracer.wedges()[0].cpu().numpy()]
    d = tracer.diffraction()
    doff, wed = d["offsets"].cpu().numpy(), d["wedge"].cpu().numpy()
    ws = DF.wedges(sc.verts)
    osc = O.make_scene(sc)
    n = 0
    for t in range(3):
        for r in range(off[t], off[t + 1]):
            got = sorted(faces[k] for k in wed[doff[r]:doff[r + 1]])
            want, edge = [], []
            for w in ws:
                ok, _, m = DF.evaluate(osc, w, tx3.pos[t], rx.pos[r])
                if m < max(osc.eps, 1e-3):
                    edge.append((w.f0, w.f1))
                elif ok:
                    want.append((w.f0, w.f1))
            assert set(want) <= set(got) and set(got) - set(want) <= set(edge), (t, r)
            n += len(got)
    assert n > 0


def test_diffraction_coverage_map_matches_oracle(tracer):
    """The diffracted part of a coverage map (Listing 2's coverage map with
    diffraction) around the tiny scene's box, per cell against the oracle's
    sum over the diffracted paths to the cell centre."""
    sc = S.tiny_scene()
    tx = S.Devices(np.array([[-60.0, 0.0, 25.0]], np.float32), np.array([[0.2, 0.05, 0.0]], np.float32),
                   S.TR38901_VH)
    rx = S.Devices(np.zeros((1, 3), np.float32), np.zeros((1, 3), np.float32), S.V_ISO)
    setup(tracer, sc, tx, rx)
    grid = dict(x0=-64.0, y0=-64.0, cell=8.0, nx=16, ny=16, h=1.5)
    for port in (0, 1):
        g = tracer.coverage_map_diffraction(grid, port).cpu().numpy()
        og, om = DF.diffraction_map(O.make_scene(sc), sc.verts, tx, grid, port, rx.antenna, FC)
        sure = om > 1e-3
        assert np.count_nonzero(og[sure] > 0) >= 20
        bad = sure & ~(np.abs(g - og) <= 2e-3 * og + 1e-12 * og.max())
        assert not bad.any(), [(tuple(ix), g[tuple(ix)], og[tuple(ix)], om[tuple(ix)]) for ix in np.argwhere(bad)[:8]]

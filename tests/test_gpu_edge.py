"""Edge cases of the CUDA path: empty and one-triangle scenes, a scene whose
triangles all bypass the hierarchy (large ground quad), LOS only, more paths
than the initial path capacity (grow-and-retry), and argument errors."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2303_11103_gb300 import rt
from paper_2303_11103_gb300 import scenes as S

from gpu_helpers import A_ABS, A_REL, FC, gpu_paths, setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tracer():
    tr = rt.Tracer(0, FC)
    yield tr
    tr.close()


def _devices(n_rx, seed=0, z_tx=20.0, half=80.0):
    rng = np.random.default_rng(seed)
    tx = S.Devices(np.array([[0.0, 0.0, z_tx]], np.float32), np.zeros((1, 3), np.float32), S.V_ISO)
    rxp = np.concatenate([rng.uniform(-half, half, (n_rx, 2)), np.full((n_rx, 1), 1.5)], 1).astype(np.float32)
    return tx, S.Devices(rxp, np.zeros((n_rx, 3), np.float32), S.V_ISO)


def test_empty_scene_los_only(tracer):
    sc = S.Scene(np.zeros((0, 9), np.float32), np.zeros(0, np.int32), np.array([S.CONCRETE], np.float32))
    tx, rx = _devices(7)
    setup(tracer, sc, tx, rx)
    assert tracer.compute_paths(3, 5000) == 7
    a, tau = tracer.cir()
    d = np.linalg.norm(rx.pos - tx.pos, axis=1)
    lam = 299792458.0 / FC
    assert np.allclose(np.abs(a.cpu().numpy()[:, 0, 0]), lam / (4 * np.pi * d), rtol=1e-5)
    g, h = tracer.coverage_map(dict(x0=-10.0, y0=-10.0, cell=5.0, nx=4, ny=4, h=0.0), 2, 100000)
    assert int(h.sum()) > 0


@pytest.mark.parametrize("kind", ["one_triangle", "ground_only", "ground_plus_one_wall"])
def test_small_scenes_match_oracle(tracer, kind):
    if kind == "one_triangle":
        v = np.array([[-30, -30, 0, 40, -25, 0, -20, 50, 0]], np.float32)
        sc = S.Scene(v, np.zeros(1, np.int32), np.array([S.GROUND], np.float32))
    elif kind == "ground_only":
        sc = S.ground_only_scene(300.0)
    else:   # two large ground triangles outside the hierarchy + a one-leaf hierarchy
        g = S.ground_only_scene(300.0)
        wall = np.array([[25, -20, 0, 25, 20, 0, 25, 0, 30]], np.float32)
        sc = S.Scene(np.concatenate([g.verts, wall]), np.array([0, 0, 1], np.int32),
                     np.array([S.GROUND, S.CONCRETE], np.float32))
    tx, rx = _devices(12, seed=1)
    setup(tracer, sc, tx, rx)
    tracer.compute_paths(2, 20000)
    gsets, _ = gpu_paths(tracer)
    osc = O.make_scene(sc)
    paths, _ = O.compute_paths(osc, tx.pos[0], rx.pos, 2, 20000)
    for r in range(12):
        want = sorted(p.seq for p in paths if p.rx == r and p.valid)
        assert sorted(gsets[r]) == want
    a, tau = tracer.cir()
    sel = [p for p in paths if p.valid]
    oa, otau = O.path_field(osc, FC, tx, rx, 0, sel)
    assert np.allclose(a.cpu().numpy(), oa, rtol=A_REL, atol=A_ABS * np.abs(oa).max())


def test_more_paths_than_initial_capacity(tracer):
    sc = S.ground_only_scene(2000.0)
    tx, rx = _devices(40000, seed=2, half=900.0)
    setup(tracer, sc, tx, rx)
    P = tracer.compute_paths(1, 2000)
    assert P == 80000                      # LOS + one ground reflection per receiver (> 65536)
    off = tracer.paths()["offsets"].cpu().numpy()
    assert np.all(np.diff(off) == 2)


def test_argument_errors(tracer):
    sc = S.tiny_scene()
    tx, rx = S.tiny_devices(visible=True)
    setup(tracer, sc, tx, rx)
    with pytest.raises(rt.RtError) as e:
        tracer.compute_paths(7, 1000)
    assert e.value.code == -1
    with pytest.raises(rt.RtError):
        tracer.coverage_map(dict(x0=0.0, y0=0.0, cell=1.0, nx=4, ny=4, h=1.5), 2, 1000, tx_port=1)
    with pytest.raises(rt.RtError):
        tracer.coverage_map(dict(x0=0.0, y0=0.0, cell=0.0, nx=4, ny=4, h=1.5), 2, 1000)
    with pytest.raises(rt.RtError):
        tracer.set_rx(rx.pos, rx.ypr, rx.antenna, [0, 5])   # offsets must end at m
    with pytest.raises(rt.RtError):
        tracer.set_materials(np.ones((3, 2), np.float32))   # material count differs
    # the context stays usable after errors
    setup(tracer, sc, tx, rx)
    assert tracer.compute_paths(2, 10000) == 4


@pytest.mark.parametrize("n_side", [1, 2, 6, 20])
def test_builders_give_identical_hits(tracer, n_side):
    """The closest hit of every query does not depend on the hierarchy: the
    radix-tree builder and the clustering builder, each in the binary and
    the 8-wide node layout, give the same per-ray hit lists, the same path
    set and the same coverage map (one box, 2 x 2 boxes, a small city, and
    the full 4802-triangle city), and all keep every triangle reachable."""
    big = n_side == 20
    sc = S.city_scene(n_side=n_side, size=500.0 if big else 150.0, seed=1 if big else 5)
    tx, rx = S.city_devices(sc, n_rx=16, half=240.0 if big else 70.0)
    N, D = 50021, 3
    grid = dict(x0=-75.0, y0=-75.0, cell=2.0, nx=75, ny=75, h=1.5)
    hits, sets, maps = [], [], []
    try:
        for b in (rt.BVH_KARRAS, rt.BVH_PLOC):
            for w in (2, 8):
                tracer.set_bvh_builder(b)
                tracer.set_bvh_width(w)
                setup(tracer, sc, tx, rx)
                tracer.compute_paths(D, N, record_rays=True)
                hits.append(tracer.ray_hits()[0].cpu().numpy().copy())
                sets.append(gpu_paths(tracer)[0])
                maps.append([x.cpu().numpy() for x in tracer.coverage_map(grid, D, N)])
    finally:
        tracer.set_bvh_builder(rt.BVH_PLOC)
        tracer.set_bvh_width(2)
    for k in range(1, 4):
        assert np.array_equal(hits[0], hits[k]), k
        assert sets[0] == sets[k], k
        assert np.array_equal(maps[0][1], maps[k][1]), k
        assert np.allclose(maps[0][0], maps[k][0], rtol=1e-5, atol=0), k
    assert (hits[0] >= 0).sum() > (N if n_side >= 6 else N // 20)   # many rays bounce


def test_unknown_builder_rejected(tracer):
    with pytest.raises(rt.RtError):
        tracer.set_bvh_builder(7)
    with pytest.raises(rt.RtError):
        tracer.set_bvh_width(4)


@pytest.mark.parametrize("n_tx", [1, 24])
def test_dedup_modes_identical(tracer, n_tx):
    """Hash and sort duplicate removal give the same candidates (sequences,
    order and witness rays) and the same paths. With 24 rooftop transmitters
    over the 4802-triangle city the distinct candidates outnumber the
    8192-key one-launch sort, so the large-sort branch runs as well."""
    sc = S.city_scene(n_side=20, size=500.0, seed=1)
    _, rx = S.city_devices(sc, n_rx=16, half=240.0)
    tx = S.rooftop_transmitters(sc, n_tx=n_tx)
    N, D = 200003, 3
    cands, sets, arrays = [], [], []
    try:
        for mode in (rt.DEDUP_HASH, rt.DEDUP_SORT):
            tracer.set_dedup(mode)
            setup(tracer, sc, tx, rx)
            tracer.compute_paths(D, N)
            cands.append([x.cpu().numpy().copy() for x in tracer.candidates()])
            s, p = gpu_paths(tracer)
            sets.append(s)
            arrays.append({k: v.cpu().numpy().copy() for k, v in p.items() if torch.is_tensor(v)})
    finally:
        tracer.set_dedup(rt.DEDUP_HASH)
    for a, b in zip(cands[0], cands[1]):
        assert np.array_equal(a, b)
    assert sets[0] == sets[1]
    for k in arrays[0]:
        assert np.array_equal(arrays[0][k], arrays[1][k]), k
    if n_tx > 1:
        assert len(cands[0][0]) > 8192
    with pytest.raises(rt.RtError):
        tracer.set_dedup(5)


def test_extensions_with_no_paths(tracer):
    """Doppler, arrays and diffraction on a context without paths: empty
    outputs, no error; a ground-only scene has no wedges."""
    sc = S.ground_only_scene(100.0)
    tx, rx = _devices(3)
    setup(tracer, sc, tx, rx)
    tracer.compute_paths(0, 0, los=False)
    assert tracer.n_paths == 0
    a = torch.zeros((0, 1, 1), dtype=torch.complex64, device="cuda")
    assert tracer.apply_doppler(a, 1e6, 4, [1.0, 0.0, 0.0]).shape == (0, 1, 1, 4)
    assert tracer.apply_array(a, np.zeros((2, 3))).shape == (0, 1, 2)
    assert tracer.compute_diffraction() == 0
    ad, td = tracer.diffraction_cir()
    assert ad.shape[0] == 0 and td.shape[0] == 0
    assert tracer.diffraction()["offsets"].cpu().numpy().tolist() == [0, 0, 0, 0]
    g = tracer.coverage_map_diffraction(dict(x0=-50.0, y0=-50.0, cell=10.0, nx=10, ny=10, h=1.5))
    assert float(g.abs().sum()) == 0.0

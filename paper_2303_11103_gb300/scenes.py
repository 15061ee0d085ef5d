"""Seeded synthetic scene and radio-device generators.

This module only builds inputs: triangle meshes made of boxes and a ground
quad, material tables and transmitter/receiver placements. It holds none of
the propagation arithmetic, so the CUDA path and the CPU oracle can both take
their inputs from here.

The paper's own scenes (Munich and Etoile, built from OpenStreetMap, Sec. II
and Sec. III-A) are not available; these seeded box cities stand in for them.
Materials are described by relative permittivity and conductivity only, the
two properties the paper names for radio materials (Sec. II).

Seeds: 0 tiny, 1 city geometry, 2 transmitter/receiver placement,
3 materials of the differentiation workload, 4 surrogate training sites,
14 surrogate held-out sites, 6-10 dense path lists.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# (eps_r, sigma [S/m]) of the named materials of the workloads.
CONCRETE = (5.24, 0.123)
GLASS = (6.31, 0.0036)
GROUND = (5.13, 0.0047)

ANT_ISO, ANT_DIPOLE, ANT_TR38901 = 0, 1, 2


@dataclass
class Antenna:
    """Pattern kind and per-port polarization slant angles (radians)."""
    kind: int = ANT_ISO
    slants: tuple = (0.0,)

    @property
    def n_ports(self) -> int:
        return len(self.slants)


V_ISO = Antenna(ANT_ISO, (0.0,))
TR38901_VH = Antenna(ANT_TR38901, (0.0, np.pi / 2))
TR38901_V = Antenna(ANT_TR38901, (0.0,))


@dataclass
class Scene:
    verts: np.ndarray            # float32 [T, 9]: v0, v1, v2 of each triangle
    mat_id: np.ndarray           # int32 [T]
    materials: np.ndarray        # float32 [M, 2]: eps_r, sigma
    name: str = ""
    footprints: np.ndarray = field(default_factory=lambda: np.zeros((0, 5), np.float64))
    # footprints: [B, 5] = x0, x1, y0, y1, height of each box building

    @property
    def n_tris(self) -> int:
        return int(self.verts.shape[0])


@dataclass
class Devices:
    pos: np.ndarray              # float32 [n, 3]
    ypr: np.ndarray              # float32 [n, 3] yaw, pitch, roll (radians)
    antenna: Antenna = field(default_factory=lambda: V_ISO)


def box_triangles(x0, x1, y0, y1, z0, z1) -> np.ndarray:
    """12 triangles (6 faces x 2) of an axis-aligned box, float64 [12, 9]."""
    c = np.array([[x0, y0, z0], [x1, y0, z0], [x1, y1, z0], [x0, y1, z0],
                  [x0, y0, z1], [x1, y0, z1], [x1, y1, z1], [x0, y1, z1]], np.float64)
    faces = [(0, 1, 2, 3), (4, 5, 6, 7), (0, 1, 5, 4),
             (1, 2, 6, 5), (2, 3, 7, 6), (3, 0, 4, 7)]
    tris = []
    for a, b, cc, d in faces:
        tris.append(np.concatenate([c[a], c[b], c[cc]]))
        tris.append(np.concatenate([c[a], c[cc], c[d]]))
    return np.stack(tris)


def ground_triangles(half: float) -> np.ndarray:
    c = np.array([[-half, -half, 0.0], [half, -half, 0.0],
                  [half, half, 0.0], [-half, half, 0.0]])
    return np.stack([np.concatenate([c[0], c[1], c[2]]),
                     np.concatenate([c[0], c[2], c[3]])])


def tiny_scene() -> Scene:
    """200 x 200 m ground plus one 20 x 20 x 30 m box at the origin, all concrete."""
    tris = np.concatenate([ground_triangles(100.0),
                           box_triangles(-10, 10, -10, 10, 0, 30)])
    mats = np.array([CONCRETE], np.float32)
    return Scene(tris.astype(np.float32), np.zeros(len(tris), np.int32), mats, "tiny",
                 np.array([[-10, 10, -10, 10, 30.0]]))


def tiny_scene_3mat() -> Scene:
    """The tiny scene with three materials: the ground and the box's floor
    (0), the box's two x-facing walls (1), its other walls and roof (2)."""
    sc = tiny_scene()
    v = sc.verts.reshape(-1, 3, 3)
    x_wall = np.all(v[:, :, 0] == v[:, :1, 0], axis=1)
    on_ground = np.all(v[:, :, 2] == 0.0, axis=1)
    mat = np.where(on_ground, 0, np.where(x_wall, 1, 2)).astype(np.int32)
    return Scene(sc.verts, mat, np.array([CONCRETE, GLASS, CONCRETE], np.float32), "tiny3", sc.footprints)


def tiny_devices(visible: bool = False):
    """Tx (-60,0,25), Rx (60,10,1.5); the 'visible' variant moves Rx to (-75,0,1.5)."""
    tx = Devices(np.array([[-60.0, 0.0, 25.0]], np.float32), np.zeros((1, 3), np.float32), V_ISO)
    rxp = [-75.0, 0.0, 1.5] if visible else [60.0, 10.0, 1.5]
    rx = Devices(np.array([rxp], np.float32), np.zeros((1, 3), np.float32), V_ISO)
    return tx, rx


def ground_only_scene(half: float = 1000.0, mat=CONCRETE) -> Scene:
    tris = ground_triangles(half)
    return Scene(tris.astype(np.float32), np.zeros(2, np.int32),
                 np.array([mat], np.float32), "ground")


def city_scene(n_side: int = 20, size: float = 500.0, seed: int = 1,
               n_materials: int = 0, mat_seed: int = 3) -> Scene:
    """Box city on a jittered n_side x n_side grid over a size x size ground.

    Footprints are uniform in [10, 40] m, heights uniform in [10, 60] m, grid
    jitter uniform in [-5, 5] m. Overlapping boxes are kept. With the default
    three materials each building is concrete or glass (half each, by seed)
    and the ground is material 2. With n_materials > 0 the materials are
    drawn as eps_r ~ U(2, 8), sigma ~ logU(1e-3, 1) and assigned to the
    ground (material 0) and to buildings at random.
    """
    rng = np.random.default_rng(seed)
    pitch = size / n_side
    tris, mats, fps = [], [], []
    if n_materials > 0:
        mrng = np.random.default_rng(mat_seed)
        eps = mrng.uniform(2.0, 8.0, n_materials)
        sig = 10.0 ** mrng.uniform(-3.0, 0.0, n_materials)
        materials = np.stack([eps, sig], 1).astype(np.float32)
        ground_mat = 0
    else:
        materials = np.array([CONCRETE, GLASS, GROUND], np.float32)
        ground_mat = 2
    g = ground_triangles(size / 2)
    tris.append(g)
    mats += [ground_mat] * 2
    brng = np.random.default_rng(seed + 1000)
    for i in range(n_side):
        for j in range(n_side):
            cx = -size / 2 + pitch * (i + 0.5) + rng.uniform(-5, 5)
            cy = -size / 2 + pitch * (j + 0.5) + rng.uniform(-5, 5)
            w, d = rng.uniform(10, 40, 2)
            h = rng.uniform(10, 60)
            x0, x1, y0, y1 = cx - w / 2, cx + w / 2, cy - d / 2, cy + d / 2
            tris.append(box_triangles(x0, x1, y0, y1, 0.0, h))
            if n_materials > 0:
                m = int(brng.integers(0, n_materials))
            else:
                m = int(brng.integers(0, 2))
            mats += [m] * 12
            fps.append([x0, x1, y0, y1, h])
    verts = np.concatenate(tris).astype(np.float32)
    return Scene(verts, np.array(mats, np.int32), materials, f"city{n_side}",
                 np.array(fps, np.float64))


def _inside_any(fps: np.ndarray, x: float, y: float, margin: float = 0.0) -> bool:
    if len(fps) == 0:
        return False
    return bool(np.any((x > fps[:, 0] - margin) & (x < fps[:, 1] + margin) &
                       (y > fps[:, 2] - margin) & (y < fps[:, 3] + margin)))


def _height_at(fps: np.ndarray, x: float, y: float) -> float:
    if len(fps) == 0:
        return 0.0
    m = (x > fps[:, 0]) & (x < fps[:, 1]) & (y > fps[:, 2]) & (y < fps[:, 3])
    return float(fps[m, 4].max()) if m.any() else 0.0


class _FootprintRaster:
    """Exact point-in-(dilated)-footprint test accelerated by a 1 m raster:
    cells fully inside a footprint reject, cells touching none accept, the
    rest fall back to the exact test."""

    def __init__(self, fps, margin, cell=1.0):
        self.fps, self.margin, self.cell = fps, margin, cell
        lo = np.floor(min(fps[:, 0].min(), fps[:, 2].min()) - margin - 1)
        hi = np.ceil(max(fps[:, 1].max(), fps[:, 3].max()) + margin + 1)
        self.lo, self.n = lo, int((hi - lo) / cell) + 1
        self.touch = np.zeros((self.n, self.n), bool)
        self.full = np.zeros((self.n, self.n), bool)
        for x0, x1, y0, y1, _ in fps:
            a = (np.array([x0 - margin, x1 + margin, y0 - margin, y1 + margin]) - lo) / cell
            i0, i1, j0, j1 = int(np.floor(a[0])), int(np.floor(a[1])), int(np.floor(a[2])), int(np.floor(a[3]))
            self.touch[i0:i1 + 1, j0:j1 + 1] = True
            f0, f1, g0, g1 = int(np.ceil(a[0])), int(np.floor(a[1])) - 1, int(np.ceil(a[2])), int(np.floor(a[3])) - 1
            if f1 >= f0 and g1 >= g0:
                self.full[f0:f1 + 1, g0:g1 + 1] = True

    def inside(self, p):
        ij = np.floor((p - self.lo) / self.cell).astype(np.int64)
        ok = (ij >= 0).all(1) & (ij < self.n).all(1)
        res = np.zeros(len(p), bool)
        t = np.zeros(len(p), bool)
        f = np.zeros(len(p), bool)
        t[ok] = self.touch[ij[ok, 0], ij[ok, 1]]
        f[ok] = self.full[ij[ok, 0], ij[ok, 1]]
        res[f] = True
        amb = t & ~f
        if amb.any():
            q, m, fps = p[amb], self.margin, self.fps
            res[amb] = ((q[:, None, 0] > fps[None, :, 0] - m) & (q[:, None, 0] < fps[None, :, 1] + m) &
                        (q[:, None, 1] > fps[None, :, 2] - m) & (q[:, None, 1] < fps[None, :, 3] + m)).any(1)
        return res


def street_points(scene: Scene, n: int, rng, half: float, margin: float = 0.5, center=(0.0, 0.0)):
    """n points (x, y) by rejection from center + [-half, half]^2 outside every footprint."""
    fps = scene.footprints
    raster = None
    if len(fps):
        key = (id(fps), margin)
        raster = _RASTERS.get(key)
        if raster is None:
            raster = _RASTERS[key] = _FootprintRaster(fps, margin)
    out = np.zeros((0, 2))
    while len(out) < n:
        m = max(2 * (n - len(out)), 64)
        p = rng.uniform(-half, half, (m, 2)) + np.asarray(center, np.float64)
        if raster is not None:
            p = p[~raster.inside(p)]
        out = np.concatenate([out, p])
    return out[:n]


_RASTERS = {}


def city_devices(scene: Scene, n_rx: int = 1000, seed: int = 2,
                 tx_antenna: Antenna = TR38901_VH, rx_antenna: Antenna = V_ISO,
                 half: float = 240.0):
    """One Tx 30 m above a street point, n_rx receivers 1.5 m above streets."""
    rng = np.random.default_rng(seed)
    txy = street_points(scene, 1, rng, 0.6 * half)[0]
    tx = Devices(np.array([[txy[0], txy[1], 30.0]], np.float32),
                 np.array([[rng.uniform(-np.pi, np.pi), 0.1, 0.0]], np.float32), tx_antenna)
    rxy = street_points(scene, n_rx, rng, half)
    rx = Devices(np.concatenate([rxy, np.full((n_rx, 1), 1.5)], 1).astype(np.float32),
                 np.zeros((n_rx, 3), np.float32), rx_antenna)
    return tx, rx


def rooftop_transmitters(scene: Scene, n_tx: int = 64, seed: int = 2,
                         antenna: Antenna = TR38901_V, half: float = 240.0) -> Devices:
    """n_tx Tx with z ~ U(25, 60) at xy not inside a taller building, random azimuth."""
    rng = np.random.default_rng(seed + 100)
    pos, ypr = [], []
    while len(pos) < n_tx:
        x, y = rng.uniform(-half, half, 2)
        z = rng.uniform(25.0, 60.0)
        if _height_at(scene.footprints, x, y) >= z - 1.0:
            continue
        pos.append((x, y, z))
        ypr.append((rng.uniform(-np.pi, np.pi), 0.1, 0.0))
    return Devices(np.array(pos, np.float32), np.array(ypr, np.float32), antenna)


def surrogate_sites(scene: Scene, n_tx: int, n_rx_per_tx: int, seed: int = 4, half: float = 240.0,
                    mast=(1.0, 5.0), rx_radius: float = 100.0):
    """Transmitters over rooftops at continuous positions, with street receivers.

    Each transmitter stands 1 m outside a uniformly drawn point of the roof
    edge of a random building (a mast set back on the roof would see no
    street: the roof hides it), a uniform mast height above that roof, and
    not inside a taller building. Every draw is a new position, so two seeds
    give disjoint transmitter sets (transmitters never seen in training).
    Its receivers are street points within a square of half-side rx_radius
    around it (clipped to the city), 1.5 m high.
    Returns tx [n_tx, 3] and rx [n_tx, n_rx_per_tx, 3] (float32).
    """
    rng = np.random.default_rng(seed)
    fps = scene.footprints
    inner = fps[(np.abs(0.5 * (fps[:, 0] + fps[:, 1])) < half) &
                (np.abs(0.5 * (fps[:, 2] + fps[:, 3])) < half)]
    tx = []
    while len(tx) < n_tx:
        x0, x1, y0, y1, h = inner[rng.integers(0, len(inner))]
        w, dpt = x1 - x0, y1 - y0
        u = rng.uniform(0.0, 2.0 * (w + dpt))      # arc length along the roof edge
        if u < w:
            x, y = x0 + u, y0 - 1.0
        elif u < w + dpt:
            x, y = x1 + 1.0, y0 + (u - w)
        elif u < 2 * w + dpt:
            x, y = x1 - (u - w - dpt), y1 + 1.0
        else:
            x, y = x0 - 1.0, y1 - (u - 2 * w - dpt)
        z = h + rng.uniform(mast[0], mast[1])
        if _height_at(fps, x, y) >= z - 0.5:
            continue
        tx.append((x, y, z))
    rx = []
    for t in tx:
        r = min(rx_radius, half)
        c = np.clip([t[0], t[1]], -half + r, half - r)
        rx.append(np.concatenate([street_points(scene, n_rx_per_tx, rng, r, center=c),
                                  np.full((n_rx_per_tx, 1), 1.5)], 1))
    return np.array(tx, np.float32), np.stack(rx).astype(np.float32)


def dense_path_list(n_pairs: int = 1000, mean_paths: int = 64, n_port_pairs: int = 4, seed: int = 6,
                    tau_range=(2e-7, 3.3e-6)):
    """Seeded synthetic channel path list for the frequency response where it
    is compute-bound: many paths per (tx, rx) pair.

    Per pair a Poisson(mean_paths) number of paths (ragged), except pair 0
    with 3 * mean_paths + 5 (several shared-memory tiles) and pair 1 with
    none. Delays uniform over tau_range (60 m to 1 km of path length);
    coefficients of independent uniform phase and a magnitude uniform in dB
    over [-140, -70] dB, per port pair.
    Returns offsets int64 [n_pairs+1], a complex64 [P, n_port_pairs],
    tau float32 [P].
    """
    rng = np.random.default_rng(seed)
    cnt = rng.poisson(mean_paths, n_pairs).astype(np.int64)
    if n_pairs > 0:
        cnt[0] = 3 * mean_paths + 5
    if n_pairs > 1:
        cnt[1] = 0
    off = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
    P = int(off[-1])
    mag = 10.0 ** (rng.uniform(-140.0, -70.0, (P, n_port_pairs)) / 20.0)
    ph = rng.uniform(-np.pi, np.pi, (P, n_port_pairs))
    a = (mag * np.exp(1j * ph)).astype(np.complex64)
    tau = rng.uniform(tau_range[0], tau_range[1], P).astype(np.float32)
    return off, a, tau

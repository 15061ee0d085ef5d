"""Python wrapper of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py, never by the product path. It
shares no code with the CUDA library; inputs come from the seeded generators
in paper_2303_11103_gb300.scenes (geometry only).

What lives here rather than in C is plain bookkeeping that is obviously
correct in Python: duplicate removal of candidate paths with a set (Sec. II:
"duplicate paths are removed"), adding the line-of-sight candidate, canonical
ordering, and the frequency response as a direct FP64 sum (Sec. III-A: CIRs
transformed to OFDM frequency responses).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

C0 = 299792458.0
EPS0 = 8.8541878128e-12

# Scale factors of the geometric tolerances, relative to the scene extent.
TMIN_REL = 2e-6      # self-intersection offset t_min
EPS_REL = 4e-6       # near-degenerate decision margin


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (plain -O2, strict IEEE, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def nthreads() -> int:
    return int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1))


@dataclass
class OScene:
    V: np.ndarray          # float64 [T, 9]
    mat: np.ndarray        # int32 [T]
    mats: np.ndarray       # float64 [M, 2]
    tmin: float
    eps: float

    @property
    def T(self):
        return int(self.V.shape[0])

    @property
    def M(self):
        return int(self.mats.shape[0])


def make_scene(scene) -> OScene:
    V = _f64(scene.verts.astype(np.float64))
    pts = V.reshape(-1, 3)
    ext = float((pts.max(0) - pts.min(0)).max()) if len(pts) else 1.0
    return OScene(V, _i32(scene.mat_id), _f64(scene.materials.astype(np.float64)),
                  TMIN_REL * ext, EPS_REL * ext)


# --------------------------------------------------------------------------
# Rays
# --------------------------------------------------------------------------
def fibonacci(N: int, i0: int = 0, n: int | None = None) -> np.ndarray:
    """Fibonacci-lattice directions d_i, i in [i0, i0+n), FP64 [n, 3] (Sec. II)."""
    n = N - i0 if n is None else n
    out = np.empty((n, 3), np.float64)
    lib().ora_fibonacci(ctypes.c_longlong(N), ctypes.c_longlong(i0), ctypes.c_longlong(n), _p(out))
    return out


def closest_hit(osc: OScene, o, d, exclude=-1):
    t = ctypes.c_double()
    m = ctypes.c_double()
    o = _f64(o)
    d = _f64(d)
    i = lib().ora_closest_hit(osc.T, _p(osc.V), _p(o), _p(d), exclude, ctypes.c_double(osc.tmin),
                              ctypes.c_double(osc.eps), ctypes.byref(t), ctypes.byref(m))
    return i, t.value, m.value


def segment_clear(osc: OScene, p, q, ex0=-1, ex1=-1):
    """Is the segment p -> q free of occluders other than ex0 / ex1? (clear, margin)."""
    m = ctypes.c_double()
    c = lib().ora_segment_clear(osc.T, _p(osc.V), _p(_f64(p)), _p(_f64(q)), ex0, ex1, ctypes.c_double(osc.tmin),
                                ctypes.c_double(osc.eps), ctypes.byref(m))
    return bool(c), m.value


def trace_sbr(osc: OScene, tx, N: int, D: int, ray_ids=None):
    """Per-ray hit lists [n, D] (int32, -1 after a miss) and prefix margins [n, D]."""
    ray_ids = np.arange(N, dtype=np.int64) if ray_ids is None else _i64(ray_ids)
    n = len(ray_ids)
    hits = np.empty((n, D), np.int32)
    marg = np.empty((n, D), np.float64)
    lib().ora_trace_sbr(osc.T, _p(osc.V), _p(_f64(tx)), ctypes.c_longlong(N), _p(ray_ids),
                        ctypes.c_longlong(n), D, ctypes.c_double(osc.tmin),
                        ctypes.c_double(osc.eps), _p(hits), _p(marg), nthreads())
    return hits, marg


def candidates(hits: np.ndarray, marg: np.ndarray, ray_ids=None):
    """Candidate paths = every prefix of every ray's hit list, de-duplicated.

    Returns {seq tuple: (best discovery margin, lowest ray id)}.
    """
    n, D = hits.shape
    ray_ids = np.arange(n) if ray_ids is None else ray_ids
    out = {}
    for k in range(n):
        for b in range(D):
            if hits[k, b] < 0:
                break
            key = tuple(int(x) for x in hits[k, :b + 1])
            m = float(marg[k, b])
            r = int(ray_ids[k])
            if key in out:
                om, orr = out[key]
                out[key] = (max(om, m), min(orr, r))
            else:
                out[key] = (m, r)
    return out


def image_path(osc: OScene, tx, rx, seq):
    """(valid, reflection points [K,3], length, margin) of one candidate (Sec. II)."""
    K = len(seq)
    pts = np.zeros((max(K, 1), 3), np.float64)
    length = ctypes.c_double()
    m = ctypes.c_double()
    s = _i32(np.array(seq if K else [0]))
    ok = lib().ora_image_path(osc.T, _p(osc.V), _p(_f64(tx)), _p(_f64(rx)), _p(s), K,
                              ctypes.c_double(osc.tmin), ctypes.c_double(osc.eps), _p(pts),
                              ctypes.byref(length), ctypes.byref(m))
    return bool(ok), pts[:K], length.value, m.value


def _pack(seqs, D):
    n = len(seqs)
    arr = np.full((max(n, 1), max(D, 1)), -1, np.int32)
    dep = np.zeros(max(n, 1), np.int32)
    for i, s in enumerate(seqs):
        arr[i, :len(s)] = s
        dep[i] = len(s)
    return arr, dep


def validate(osc: OScene, tx, rxs, seqs, D):
    """Image method of every candidate against every receiver.

    Returns arrays (cand, rx, valid, margin) over the pairs that are valid or
    near-degenerate (margin < eps).
    """
    rxs = _f64(np.asarray(rxs).reshape(-1, 3))
    arr, dep = _pack(seqs, D)
    cap = max(1024, 4 * len(seqs) * 4)
    while True:
        oc = np.empty(cap, np.int64)
        orx = np.empty(cap, np.int32)
        ov = np.empty(cap, np.int32)
        om = np.empty(cap, np.float64)
        cnt = lib().ora_validate(osc.T, _p(osc.V), _p(_f64(tx)), len(rxs), _p(rxs),
                                 ctypes.c_longlong(len(seqs)), _p(arr), _p(dep), max(D, 1),
                                 ctypes.c_double(osc.tmin), ctypes.c_double(osc.eps),
                                 ctypes.c_longlong(cap), _p(oc), _p(orx), _p(ov), _p(om),
                                 nthreads())
        if cnt <= cap:
            return oc[:cnt], orx[:cnt], ov[:cnt].astype(bool), om[:cnt]
        cap = int(cnt) + 16


lib_restype_set = False


def _setup_restypes():
    global lib_restype_set
    if lib_restype_set:
        return
    L = lib()
    L.ora_validate.restype = ctypes.c_longlong
    L.ora_image_path.restype = ctypes.c_int
    L.ora_closest_hit.restype = ctypes.c_int
    lib_restype_set = True


@dataclass
class OPath:
    rx: int
    seq: tuple
    valid: bool
    margin: float
    points: np.ndarray
    length: float


def compute_paths(osc: OScene, tx, rxs, D: int, N: int, los: bool = True,
                  reflection: bool = True, ray_ids=None):
    """Specular paths from one Tx to every Rx (Sec. II heuristic method).

    Returns (paths, cands): paths = list of OPath, valid or near-degenerate,
    in canonical order (rx, depth, ids); cands = candidate dict of
    candidates(). Near-degenerate invalid pairs are kept with valid=False so
    that tests can excuse them.
    """
    _setup_restypes()
    rxs = np.asarray(rxs, np.float64).reshape(-1, 3)
    cands = {}
    if reflection and D > 0 and N > 0:
        hits, marg = trace_sbr(osc, tx, N, D, ray_ids)
        cands = candidates(hits, marg, ray_ids)
    seqs = sorted(cands.keys(), key=lambda s: (len(s), s))
    if los:
        seqs = [()] + seqs
    out = []
    if seqs:
        c, r, v, m = validate(osc, tx, rxs, seqs, max(D, 1))
        for ci, ri, vi, mi in zip(c, r, v, m):
            ok, pts, length, mm = image_path(osc, tx, rxs[ri], seqs[ci])
            out.append(OPath(int(ri), seqs[ci], bool(ok), float(mm), pts, length))
    out.sort(key=lambda p: (p.rx, len(p.seq), p.seq))
    return out, cands


def brute_force_paths(osc: OScene, tx, rx, D: int):
    """Exhaustive image method over every triangle sequence of length <= D.

    Sec. II: the exhaustive search the heuristic replaces; usable only on tiny
    scenes. Returns the list of (seq, margin) of valid paths (LOS included).
    """
    _setup_restypes()
    import itertools
    out = []
    for K in range(0, D + 1):
        for seq in itertools.product(range(osc.T), repeat=K):
            if any(seq[i] == seq[i + 1] for i in range(K - 1)):
                continue
            ok, pts, length, m = image_path(osc, tx, rx, seq)
            if ok:
                out.append((tuple(seq), m))
    return out


# --------------------------------------------------------------------------
# Field, CIR, frequency response
# --------------------------------------------------------------------------
def path_field(osc: OScene, fc: float, txdev, rxdev, tx_index: int, paths, grad: bool = False):
    """Channel coefficients a [P, nrp, ntp] complex128 and delays tau [P].

    With grad=True also da [P, nrp, ntp, ng] and dtau [P, ng], tangents w.r.t.
    (tx xyz, tx yaw/pitch/roll, eps_r[M], sigma[M]) by forward-mode dual
    numbers.
    """
    txa, rxa = txdev.antenna, rxdev.antenna
    P = len(paths)
    nrp, ntp = rxa.n_ports, txa.n_ports
    D = max([len(p.seq) for p in paths] + [1])
    seqs, dep = _pack([p.seq for p in paths], D)
    rx_of = _i32(np.array([p.rx for p in paths] if P else [0]))
    ng = 6 + 2 * osc.M if grad else 0
    if ng > 24:
        raise ValueError("at most 9 materials with gradients")
    a = np.zeros((max(P, 1), nrp, ntp, 2), np.float64)
    da = np.zeros((max(P, 1), nrp, ntp, max(ng, 1), 2), np.float64)
    tau = np.zeros(max(P, 1), np.float64)
    dtau = np.zeros((max(P, 1), max(ng, 1)), np.float64)
    if P:
        lib().ora_path_field(osc.T, _p(osc.V), _p(osc.mat), osc.M, _p(osc.mats),
                             ctypes.c_double(fc), _p(_f64(txdev.pos[tx_index])),
                             _p(_f64(txdev.ypr[tx_index])), txa.kind, ntp,
                             _p(_f64(np.array(txa.slants))), _p(_f64(rxdev.pos)),
                             _p(_f64(rxdev.ypr)), rxa.kind, nrp, _p(_f64(np.array(rxa.slants))),
                             ctypes.c_longlong(P), _p(rx_of), _p(seqs), _p(dep), D, ng,
                             _p(a), _p(da), _p(tau), _p(dtau), nthreads())
    a = (a[..., 0] + 1j * a[..., 1])[:P]
    tau = tau[:P]
    if not grad:
        return a, tau
    da = (da[..., 0] + 1j * da[..., 1])[:P, :, :, :ng]
    return a, tau, da, dtau[:P, :ng]


def doppler(a: np.ndarray, paths, tx, rxs, fc: float, fs: float, n_steps: int, v_tx, v_rx=None) -> np.ndarray:
    """Time evolution of the channel coefficients from the devices' motion
    (Sec. II-A, Listing 3: apply_doppler with a sampling frequency, a number
    of time steps and velocity vectors of the transmitters and receivers).

    Path i leaves the transmitter in the unit direction k_t (towards its
    first reflection point, or the receiver) and reaches the receiver in the
    unit direction k_r (from its last reflection point, or the transmitter).
    Its Doppler shift is f_D = (v_tx . k_t - v_rx . k_r) / lambda, the rate of
    change of -(path length) / lambda when the devices move, and
    a_i(t_n) = a_i exp(j 2 pi f_D t_n) at t_n = n / fs, n = 0..n_steps-1. The
    delays are kept.

    a [P, ...] complex, paths with .points [K, 3] and .rx, tx [3], rxs [R, 3],
    v_tx [3], v_rx [R, 3] or None -> [P, ..., n_steps] complex128.
    """
    lam = C0 / fc
    t = np.arange(n_steps, dtype=np.float64) / fs
    out = np.zeros(np.shape(a) + (n_steps,), np.complex128)
    txp = np.asarray(tx, np.float64)
    vt = np.asarray(v_tx, np.float64)
    for i, p in enumerate(paths):
        rxp = np.asarray(rxs[p.rx], np.float64)
        pts = [txp] + [np.asarray(q, np.float64) for q in p.points] + [rxp]
        kt = (pts[1] - pts[0]) / np.linalg.norm(pts[1] - pts[0])
        kr = (pts[-1] - pts[-2]) / np.linalg.norm(pts[-1] - pts[-2])
        fd = np.dot(vt, kt)
        if v_rx is not None:
            fd -= np.dot(np.asarray(v_rx[p.rx], np.float64), kr)
        fd /= lam
        out[i] = np.asarray(a[i])[..., None] * np.exp(2j * np.pi * fd * t)
    return out


def rotation_ypr(ypr) -> np.ndarray:
    """Device rotation R = Rz(yaw) Ry(pitch) Rx(roll) (3GPP TR 38.901 Sec. 7.1):
    the columns are the device's x, y, z axes in the global frame."""
    a, b, g = (float(v) for v in ypr)
    Rz = np.array([[np.cos(a), -np.sin(a), 0.0], [np.sin(a), np.cos(a), 0.0], [0.0, 0.0, 1.0]])
    Ry = np.array([[np.cos(b), 0.0, np.sin(b)], [0.0, 1.0, 0.0], [-np.sin(b), 0.0, np.cos(b)]])
    Rx = np.array([[1.0, 0.0, 0.0], [0.0, np.cos(g), -np.sin(g)], [0.0, np.sin(g), np.cos(g)]])
    return Rz @ Ry @ Rx


def array_response(a: np.ndarray, paths, tx, tx_ypr, rxs, rx_ypr, fc: float, tx_el, rx_el) -> np.ndarray:
    """Synthetic antenna arrays (Sec. II: arrays modelled after the ray
    tracing with a plane-wave assumption across the array).

    The paths are traced between the array centres. Element m of the
    transmit array sits at R_tx r_m from the centre (r_m in the device frame),
    element n of the receive array at R_rx s_n. Under the plane-wave
    assumption the path from element m to element n is shorter by
    k_t . R_tx r_m - k_r . R_rx s_n (k_t, k_r: unit departure and arrival
    directions of the path), so its coefficient is
    a[i][p][q] exp(j 2 pi (k_t . R_tx r_m - k_r . R_rx s_n) / lambda).

    a [P, nrp, ntp] complex, tx_el [Mt, 3], rx_el [Mr, 3] (metres, device
    frame), rx_ypr [R, 3] -> [P, Mr*nrp, Mt*ntp] with element-major, port-minor
    indices (n*nrp + p, m*ntp + q).
    """
    lam = C0 / fc
    a = np.asarray(a)
    P, nrp, ntp = a.shape
    tx_el = np.asarray(tx_el, np.float64).reshape(-1, 3)
    rx_el = np.asarray(rx_el, np.float64).reshape(-1, 3)
    Mt, Mr = len(tx_el), len(rx_el)
    out = np.zeros((P, Mr * nrp, Mt * ntp), np.complex128)
    txp = np.asarray(tx, np.float64)
    Rt = rotation_ypr(tx_ypr)
    for i, p in enumerate(paths):
        rxp = np.asarray(rxs[p.rx], np.float64)
        pts = [txp] + [np.asarray(q, np.float64) for q in p.points] + [rxp]
        kt = (pts[1] - pts[0]) / np.linalg.norm(pts[1] - pts[0])
        kr = (pts[-1] - pts[-2]) / np.linalg.norm(pts[-1] - pts[-2])
        Rr = rotation_ypr(rx_ypr[p.rx])
        ph_t = (tx_el @ Rt.T) @ kt / lam       # [Mt] cycles
        ph_r = -(rx_el @ Rr.T) @ kr / lam      # [Mr] cycles
        w = np.exp(2j * np.pi * (ph_r[:, None] + ph_t[None, :]))    # [Mr, Mt]
        out[i] = np.einsum("nm,pq->npmq", w, a[i]).reshape(Mr * nrp, Mt * ntp)
    return out


def subcarrier_freqs(K: int, spacing: float) -> np.ndarray:
    """Baseband subcarrier offsets f_k = (k - K/2) * spacing (k = 0..K-1)."""
    return (np.arange(K, dtype=np.float64) - K // 2) * spacing


def freq_response(a: np.ndarray, tau: np.ndarray, freqs: np.ndarray) -> np.ndarray:
    """H(f_k) = sum_i a_i exp(-j 2 pi f_k tau_i), direct FP64 summation.

    a [P, ...], tau [P] -> H [..., K].
    """
    ph = np.exp(-2j * np.pi * np.outer(tau, freqs))          # [P, K]
    return np.tensordot(a, ph, axes=([0], [0]))


def coverage(osc: OScene, fc, tx, txypr, txant, tx_port, rxant, N, D, grid,
             i0=0, i1=None):
    """Coverage map on the plane z = grid['h'] (see ora_coverage).

    grid = dict(x0, y0, cell, nx, ny, h). Returns gain, hits, marg [ny, nx].
    """
    i1 = N if i1 is None else i1
    nx, ny = int(grid["nx"]), int(grid["ny"])
    g = np.empty(nx * ny, np.float64)
    h = np.empty(nx * ny, np.float64)
    m = np.empty(nx * ny, np.float64)
    lib().ora_coverage(osc.T, _p(osc.V), _p(osc.mat), osc.M, _p(osc.mats), ctypes.c_double(fc),
                       _p(_f64(tx)), _p(_f64(txypr)), txant.kind,
                       ctypes.c_double(txant.slants[tx_port]), rxant.kind,
                       ctypes.c_double(rxant.slants[0]), ctypes.c_longlong(N),
                       ctypes.c_longlong(i0), ctypes.c_longlong(i1), D,
                       ctypes.c_double(grid["x0"]), ctypes.c_double(grid["y0"]),
                       ctypes.c_double(grid["cell"]), nx, ny, ctypes.c_double(grid["h"]),
                       ctypes.c_double(osc.tmin), ctypes.c_double(osc.eps),
                       _p(g), _p(h), _p(m), nthreads())
    return g.reshape(ny, nx), h.reshape(ny, nx), m.reshape(ny, nx)


def fresnel(eps_r, sigma, fc, cos1):
    rp = np.zeros(2)
    rl = np.zeros(2)
    lib().ora_fresnel(ctypes.c_double(eps_r), ctypes.c_double(sigma), ctypes.c_double(fc),
                      ctypes.c_double(cos1), _p(rp), _p(rl))
    return rp[0] + 1j * rp[1], rl[0] + 1j * rl[1]


def antenna(kind, slant, ypr, u):
    out = np.zeros(3)
    lib().ora_antenna(kind, ctypes.c_double(slant), _p(_f64(ypr)), _p(_f64(u)), _p(out))
    return out

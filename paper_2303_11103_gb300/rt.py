"""Python binding of the C ABI in include/rt.h (argument marshalling only).

Every step of the tracing path runs in librt_gb300.so; PyTorch only
provides device memory and the current CUDA stream. The low-level functions
carry the C names (rt_create, rt_load_scene, ...); `Tracer` bundles them
for convenience, and `CIR` / `FreqResponse` are autograd functions whose
backward passes call rt_cir_backward / rt_freq_response_backward.

There is no CPU fallback: if the library is missing or no GPU is present,
calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librt_gb300.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "rt.h")

RT_OK = 0
RT_LOS, RT_REFLECTION, RT_RECORD_RAYS = 1, 2, 0x100
ERRORS = {-1: "RT_ERR_INVALID_ARG", -2: "RT_ERR_CUDA", -3: "RT_ERR_OOM", -4: "RT_ERR_CAPACITY",
          -5: "RT_ERR_TIMEOUT", -6: "RT_ERR_NOT_READY"}

_lib = None


class RtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class rt_antenna(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n_ports", ctypes.c_int32), ("slant", ctypes.c_float * 2)]


class rt_grid(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_float), ("y0", ctypes.c_float), ("cell", ctypes.c_float),
                ("height", ctypes.c_float), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32)]


def header_symbols() -> list[str]:
    """Names of the functions include/rt.h declares."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^int\s+(rt_\w+)\s*\(", txt, re.M)))


def lib():
    """Load librt_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, u32, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double
        sig = {
            "rt_create": [ctypes.POINTER(vp), ctypes.c_int, vp],
            "rt_destroy": [vp],
            "rt_set_stream": [vp, vp],
            "rt_last_error": [vp, ctypes.c_char_p, ctypes.c_size_t],
            "rt_set_frequency": [vp, dbl],
            "rt_load_scene": [vp, vp, i64, vp, vp, i32],
            "rt_set_materials": [vp, vp, i32],
            "rt_set_bvh_builder": [vp, i32],
            "rt_set_bvh_width": [vp, i32],
            "rt_get_bvh": [vp, vp, i64, ctypes.POINTER(ctypes.c_int64)],
            "rt_set_dedup": [vp, i32],
            "rt_set_tx": [vp, vp, vp, i32, ctypes.POINTER(rt_antenna)],
            "rt_set_rx": [vp, vp, vp, i32, ctypes.POINTER(rt_antenna), vp],
            "rt_compute_paths": [vp, i32, i64, u32, ctypes.POINTER(i64)],
            "rt_ray_directions": [vp, i64, i64, i64, vp],
            "rt_num_pairs": [vp, ctypes.POINTER(i64)],
            "rt_get_paths": [vp, vp, vp, vp, vp, vp],
            "rt_get_candidates": [vp, ctypes.POINTER(i64), vp, vp, vp, vp],
            "rt_get_ray_hits": [vp, vp],
            "rt_cir": [vp, u32, vp, vp],
            "rt_apply_doppler": [vp, vp, vp, vp, dbl, i32, vp],
            "rt_apply_array": [vp, vp, vp, i32, vp, i32, vp],
            "rt_compute_diffraction": [vp, ctypes.POINTER(i64)],
            "rt_get_diffraction": [vp, vp, vp, vp],
            "rt_diffraction_cir": [vp, vp, vp],
            "rt_get_wedges": [vp, ctypes.POINTER(i64), vp, vp],
            "rt_coverage_map_diffraction": [vp, ctypes.POINTER(rt_grid), i32, vp],
            "rt_set_scattering": [vp, vp, i32],
            "rt_scattering_gain": [vp, i64, vp],
            "rt_set_scattering_pattern": [vp, vp, i32],
            "rt_scattering_gain_vjp": [vp, i64, vp, vp],
            "rt_freq_response": [vp, vp, vp, vp, i32, vp],
            "rt_freq_response_paths": [vp, vp, i64, i32, vp, vp, vp, i32, vp],
            "rt_probe_peak": [vp, i32, i32, i32, ctypes.POINTER(ctypes.c_double)],
            "rt_coverage_map": [vp, ctypes.POINTER(rt_grid), i32, i64, i32, vp, vp],
            "rt_coverage_map_accumulate": [vp, ctypes.POINTER(rt_grid), i32, i64, i64, i64, i32, vp, vp],
            "rt_coverage_map_noalloc": [vp, ctypes.POINTER(rt_grid), i32, i64, i32, vp, vp],
            "rt_coverage_map_async": [vp, ctypes.POINTER(rt_grid), i32, i64, i32, u32, i32, vp, vp],
            "rt_join": [vp],
            "rt_coverage_map_backward": [vp, ctypes.POINTER(rt_grid), i32, i64, i32, vp, vp],
            "rt_cir_backward": [vp, u32, vp, vp, vp, vp, vp, vp],
            "rt_freq_response_backward": [vp, vp, vp, vp, i32, vp, vp, vp],
            "rt_pair_gain": [vp, vp, ctypes.c_float, vp],
            "rt_graph_begin": [vp],
            "rt_graph_end": [vp],
            "rt_graph_launch": [vp],
            "rt_autotune": [vp, ctypes.POINTER(rt_grid), i32, i64, vp, vp, ctypes.c_char_p],
            "rt_get_tuning": [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)],
            "rt_set_tuning": [vp, i32, i32, i32],
            "rt_mlp_create": [ctypes.POINTER(vp), ctypes.c_int, vp, i32, i32, i32, ctypes.c_float,
                              ctypes.c_uint64, vp, vp],
            "rt_mlp_destroy": [vp],
            "rt_mlp_set_stream": [vp, vp],
            "rt_mlp_last_error": [vp, ctypes.c_char_p, ctypes.c_size_t],
            "rt_mlp_train_step": [vp, vp, vp, i32, ctypes.c_float, vp],
            "rt_mlp_set_baseline": [vp, ctypes.c_float],
            "rt_mlp_infer": [vp, vp, i64, vp],
            "rt_mlp_infer_layers": [vp, vp, i64, vp],
            "rt_mlp_num_params": [vp, ctypes.POINTER(i64)],
            "rt_mlp_get_params": [vp, vp],
            "rt_mlp_set_params": [vp, vp],
            "rt_mlp_get_grads": [vp, vp],
            "rt_mlp_save": [vp, vp, i64, ctypes.POINTER(i64)],
            "rt_mlp_load": [ctypes.POINTER(vp), ctypes.c_int, vp, vp, i64],
            "rt_mlp_status": [vp, ctypes.POINTER(u32)],
            "rt_gemm_bf16": [vp, vp, vp, i32, i32, i32, vp, i32, i32, vp, vp],
            "rt_profile": [vp, ctypes.c_int],
            "rt_profile_select": [vp, ctypes.c_char_p],
            "rt_profile_report": [vp, ctypes.c_char_p, ctypes.c_size_t, ctypes.c_int],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor expected")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _antenna(ant) -> rt_antenna:
    a = rt_antenna()
    a.kind = int(ant.kind)
    a.n_ports = len(ant.slants)
    for i, s in enumerate(ant.slants):
        a.slant[i] = float(s)
    return a


# ---------------------------------------------------------------- C-ABI names
def rt_create(device: int = 0):
    h = ctypes.c_void_p()
    code = lib().rt_create(ctypes.byref(h), int(device), _stream())
    if code:
        raise RtError(code, "rt_create failed")
    return h


def rt_destroy(ctx):
    lib().rt_destroy(ctx)


def rt_last_error(ctx) -> str:
    buf = ctypes.create_string_buffer(1024)
    lib().rt_last_error(ctx, buf, 1024)
    return buf.value.decode()


def _check(ctx, code):
    if code != RT_OK:
        raise RtError(code, rt_last_error(ctx))


def rt_set_stream(ctx):
    _check(ctx, lib().rt_set_stream(ctx, _stream()))


def rt_set_frequency(ctx, fc: float):
    _check(ctx, lib().rt_set_frequency(ctx, float(fc)))


def rt_load_scene(ctx, verts, mat_id, mat_params):
    _check(ctx, lib().rt_load_scene(ctx, _ptr(verts), int(verts.shape[0]), _ptr(mat_id), _ptr(mat_params),
                                    int(mat_params.shape[0])))


def rt_set_materials(ctx, mat_params):
    _check(ctx, lib().rt_set_materials(ctx, _ptr(mat_params), int(mat_params.shape[0])))


BVH_KARRAS, BVH_PLOC = 0, 1


def rt_set_bvh_builder(ctx, builder):
    _check(ctx, lib().rt_set_bvh_builder(ctx, int(builder)))


def rt_set_bvh_width(ctx, width):
    _check(ctx, lib().rt_set_bvh_width(ctx, int(width)))


def rt_get_bvh(ctx):
    """The binary hierarchy of the last load_scene: float32 [n_nodes, 16]
    (child boxes lo/hi, then the child references as int32 bit patterns)."""
    n = ctypes.c_int64()
    _check(ctx, lib().rt_get_bvh(ctx, None, 0, ctypes.byref(n)))
    out = np.zeros((max(n.value, 1), 16), np.float32)
    _check(ctx, lib().rt_get_bvh(ctx, out.ctypes.data_as(ctypes.c_void_p), n.value, ctypes.byref(n)))
    return out[:n.value]


DEDUP_HASH, DEDUP_SORT = 0, 1


def rt_set_dedup(ctx, mode):
    _check(ctx, lib().rt_set_dedup(ctx, int(mode)))


def rt_set_tx(ctx, pos, ypr, antenna):
    a = _antenna(antenna)
    _check(ctx, lib().rt_set_tx(ctx, _ptr(pos), _ptr(ypr), int(pos.shape[0]), ctypes.byref(a)))


def rt_set_rx(ctx, pos, ypr, antenna, rx_set_offsets=None):
    a = _antenna(antenna)
    off = None
    if rx_set_offsets is not None:
        arr = (ctypes.c_int32 * len(rx_set_offsets))(*[int(x) for x in rx_set_offsets])
        off = ctypes.cast(arr, ctypes.c_void_p)
    _check(ctx, lib().rt_set_rx(ctx, _ptr(pos), _ptr(ypr), int(pos.shape[0]), ctypes.byref(a), off))


def rt_compute_paths(ctx, max_depth: int, num_rays: int, flags: int) -> int:
    n = ctypes.c_int64()
    _check(ctx, lib().rt_compute_paths(ctx, int(max_depth), int(num_rays), int(flags), ctypes.byref(n)))
    return int(n.value)


def rt_ray_directions(ctx, num_rays, first, n, dirs):
    _check(ctx, lib().rt_ray_directions(ctx, int(num_rays), int(first), int(n), _ptr(dirs)))


def rt_num_pairs(ctx) -> int:
    n = ctypes.c_int64()
    _check(ctx, lib().rt_num_pairs(ctx, ctypes.byref(n)))
    return int(n.value)


def rt_get_paths(ctx, offsets=None, seq=None, points=None, depth=None, length=None):
    _check(ctx, lib().rt_get_paths(ctx, _ptr(offsets), _ptr(seq), _ptr(points), _ptr(depth), _ptr(length)))


def rt_get_candidates(ctx, tx=None, depth=None, seq=None, witness=None) -> int:
    n = ctypes.c_int64()
    _check(ctx, lib().rt_get_candidates(ctx, ctypes.byref(n), _ptr(tx), _ptr(depth), _ptr(seq), _ptr(witness)))
    return int(n.value)


def rt_get_ray_hits(ctx, hits):
    _check(ctx, lib().rt_get_ray_hits(ctx, _ptr(hits)))


def rt_cir(ctx, flags, a, tau):
    _check(ctx, lib().rt_cir(ctx, int(flags), _ptr(a), _ptr(tau)))


def rt_apply_doppler(ctx, a, tx_vel, rx_vel, fs, n_steps, a_t):
    _check(ctx, lib().rt_apply_doppler(ctx, _ptr(a), _ptr(tx_vel), _ptr(rx_vel) if rx_vel is not None else None,
                                       float(fs), int(n_steps), _ptr(a_t)))


def rt_apply_array(ctx, a, tx_el, rx_el, a_el):
    _check(ctx, lib().rt_apply_array(ctx, _ptr(a), _ptr(tx_el) if tx_el is not None else None,
                                     int(tx_el.shape[0]) if tx_el is not None else 0,
                                     _ptr(rx_el) if rx_el is not None else None,
                                     int(rx_el.shape[0]) if rx_el is not None else 0, _ptr(a_el)))


def planar_array(num_rows: int, num_cols: int, vertical_spacing: float, horizontal_spacing: float,
                 wavelength: float) -> np.ndarray:
    """Element positions [num_rows*num_cols, 3] (metres, device frame) of a
    planar array in the device's y-z plane, centred on the device: columns
    along y, rows along z, spacings in wavelengths; element r*num_cols + c."""
    r, c = np.meshgrid(np.arange(num_rows), np.arange(num_cols), indexing="ij")
    y = (c.ravel() - (num_cols - 1) / 2) * horizontal_spacing * wavelength
    z = (r.ravel() - (num_rows - 1) / 2) * vertical_spacing * wavelength
    return np.stack([np.zeros_like(y), y, z], 1).astype(np.float32)


def rt_freq_response(ctx, a, tau, freqs, H):
    _check(ctx, lib().rt_freq_response(ctx, _ptr(a), _ptr(tau), _ptr(freqs), int(freqs.shape[0]), _ptr(H)))


def rt_pair_gain(ctx, a, floor_db, out):
    _check(ctx, lib().rt_pair_gain(ctx, _ptr(a), float(floor_db), _ptr(out)))


def rt_coverage_map(ctx, grid: rt_grid, max_depth, num_rays, tx_port, gain, hits):
    _check(ctx, lib().rt_coverage_map(ctx, ctypes.byref(grid), int(max_depth), int(num_rays), int(tx_port),
                                      _ptr(gain), _ptr(hits)))


def rt_coverage_map_accumulate(ctx, grid: rt_grid, max_depth, num_rays, first_ray, ray_count, tx_port, gain,
                               hits):
    _check(ctx, lib().rt_coverage_map_accumulate(ctx, ctypes.byref(grid), int(max_depth), int(num_rays),
                                                 int(first_ray), int(ray_count), int(tx_port), _ptr(gain),
                                                 _ptr(hits)))


ASYNC_AFTER_TRACE = 1


def rt_coverage_map_async(ctx, grid: rt_grid, max_depth, num_rays, tx_port, gain, hits, flags=0, blocks_per_sm=0):
    """rt_coverage_map on the context's second stream, beside the calls that follow; rt_join before reading."""
    _check(ctx, lib().rt_coverage_map_async(ctx, ctypes.byref(grid), int(max_depth), int(num_rays), int(tx_port),
                                            int(flags), int(blocks_per_sm), _ptr(gain), _ptr(hits)))


def rt_join(ctx):
    _check(ctx, lib().rt_join(ctx))


def rt_coverage_map_noalloc(ctx, grid: rt_grid, max_depth, num_rays, tx_port, gain, hits):
    """rt_coverage_map without device allocation (static scratch, num_rays <= 2^20)."""
    _check(ctx, lib().rt_coverage_map_noalloc(ctx, ctypes.byref(grid), int(max_depth), int(num_rays),
                                              int(tx_port), _ptr(gain), _ptr(hits)))


def rt_cir_backward(ctx, flags, grad_a, grad_tau, g_eps, g_sigma, g_txpos, g_txypr):
    _check(ctx, lib().rt_cir_backward(ctx, int(flags), _ptr(grad_a), _ptr(grad_tau), _ptr(g_eps), _ptr(g_sigma),
                                      _ptr(g_txpos), _ptr(g_txypr)))


def rt_freq_response_paths(ctx, offsets, n_port_pairs, a, tau, freqs, H):
    """H(f) over a caller's CSR path list (offsets [n_pairs+1] int64)."""
    _check(ctx, lib().rt_freq_response_paths(ctx, _ptr(offsets), int(offsets.shape[0]) - 1, int(n_port_pairs),
                                             _ptr(a), _ptr(tau), _ptr(freqs), int(freqs.shape[0]), _ptr(H)))


PROBE_TRAVERSAL, PROBE_FFMA = 0, 1


def rt_probe_peak(ctx, kind, n_slab=8, n_tri=0) -> float:
    """Measured issue peak (operations/s) of the traversal arithmetic or FP32 FMA."""
    v = ctypes.c_double()
    _check(ctx, lib().rt_probe_peak(ctx, int(kind), int(n_slab), int(n_tri), ctypes.byref(v)))
    return float(v.value)


def rt_freq_response_backward(ctx, a, tau, freqs, grad_H, grad_a, grad_tau):
    _check(ctx, lib().rt_freq_response_backward(ctx, _ptr(a), _ptr(tau), _ptr(freqs), int(freqs.shape[0]),
                                                _ptr(grad_H), _ptr(grad_a), _ptr(grad_tau)))


def rt_graph_begin(ctx):
    _check(ctx, lib().rt_graph_begin(ctx))


def rt_graph_end(ctx):
    _check(ctx, lib().rt_graph_end(ctx))


def rt_graph_launch(ctx):
    _check(ctx, lib().rt_graph_launch(ctx))


def rt_autotune(ctx, grid: rt_grid, max_depth, num_rays, gain, hits, cache_path=None):
    _check(ctx, lib().rt_autotune(ctx, ctypes.byref(grid), int(max_depth), int(num_rays), _ptr(gain), _ptr(hits),
                                  cache_path.encode() if cache_path else None))


def rt_get_tuning(ctx):
    b, c, s = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(ctx, lib().rt_get_tuning(ctx, ctypes.byref(b), ctypes.byref(c), ctypes.byref(s)))
    return int(b.value), int(c.value), int(s.value)


def rt_set_tuning(ctx, block, chunk, smem_nodes):
    _check(ctx, lib().rt_set_tuning(ctx, int(block), int(chunk), int(smem_nodes)))


PROFILE_TIME, PROFILE_COUNT = 1, 2


def rt_profile(ctx, enable):
    """enable: bool (kernel timing) or flags PROFILE_TIME | PROFILE_COUNT."""
    flags = int(enable) if not isinstance(enable, bool) else (PROFILE_TIME if enable else 0)
    _check(ctx, lib().rt_profile(ctx, flags))


def rt_profile_select(ctx, names=None):
    """Time only the named kernels (iterable of names; None = all)."""
    arg = ",".join(names).encode() if names else None
    _check(ctx, lib().rt_profile_select(ctx, arg))


def rt_profile_report(ctx, reset: bool = False) -> dict:
    import json
    size = 1 << 16
    while True:
        buf = ctypes.create_string_buffer(size)
        code = lib().rt_profile_report(ctx, buf, size, 0)
        if code == -4 and size < (1 << 24):
            size *= 4
            continue
        _check(ctx, code)
        break
    if reset:
        _check(ctx, lib().rt_profile_report(ctx, buf, size, 1))
    return json.loads(buf.value.decode())


# --------------------------------------------------------------- convenience
class Tracer:
    """One rt_ctx on one device, with torch tensors in and out."""

    def __init__(self, device: int = 0, fc: float = 3.5e9):
        self.device = torch.device("cuda", device)
        self.ctx = rt_create(device)
        self.fc = fc
        rt_set_frequency(self.ctx, fc)
        self.n_tx = self.n_rx = 0
        self.ntp = self.nrp = 1
        self.max_depth = 0
        self.n_paths = 0
        self.n_dpaths = 0
        self.n_mat = 0

    def close(self):
        if self.ctx is not None:
            rt_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _t(self, x, dtype):
        return torch.as_tensor(x, dtype=dtype).to(self.device).contiguous()

    def sync_stream(self):
        rt_set_stream(self.ctx)

    def profile(self, enable: bool = True):
        rt_profile(self.ctx, enable)

    def report(self, reset: bool = False) -> dict:
        return rt_profile_report(self.ctx, reset)

    def load_scene(self, scene):
        self.sync_stream()
        self.n_dpaths = 0
        self._verts = self._t(scene.verts, torch.float32).reshape(-1, 9)
        self._mat = self._t(scene.mat_id, torch.int32)
        self._mats = self._t(scene.materials, torch.float32).reshape(-1, 2)
        self.n_mat = int(self._mats.shape[0])
        rt_load_scene(self.ctx, self._verts, self._mat, self._mats)

    def set_bvh_builder(self, builder):
        """Hierarchy for the next load_scene: BVH_KARRAS or BVH_PLOC."""
        rt_set_bvh_builder(self.ctx, builder)

    def set_bvh_width(self, width):
        """Traversal layout for the next load_scene: 2 (binary, default) or 8 (wide nodes)."""
        rt_set_bvh_width(self.ctx, width)

    def set_dedup(self, mode):
        """Candidate duplicate removal of compute_paths: DEDUP_HASH or DEDUP_SORT."""
        rt_set_dedup(self.ctx, mode)

    def set_materials(self, mats):
        self.sync_stream()
        self._mats = self._t(mats, torch.float32).reshape(-1, 2)
        rt_set_materials(self.ctx, self._mats)

    def set_tx(self, pos, ypr, antenna):
        self.sync_stream()
        self.n_dpaths = 0
        pos = self._t(pos, torch.float32).reshape(-1, 3)
        ypr = self._t(ypr, torch.float32).reshape(-1, 3)
        rt_set_tx(self.ctx, pos, ypr, antenna)
        self.n_tx, self.ntp, self.tx_antenna = int(pos.shape[0]), len(antenna.slants), antenna
        self._tx_pos, self._tx_ypr = pos, ypr

    def set_rx(self, pos, ypr, antenna, rx_set_offsets=None):
        self.sync_stream()
        self.n_dpaths = 0
        pos = self._t(pos, torch.float32).reshape(-1, 3)
        ypr = self._t(ypr, torch.float32).reshape(-1, 3)
        rt_set_rx(self.ctx, pos, ypr, antenna, rx_set_offsets)
        self.n_rx, self.nrp, self.rx_antenna = int(pos.shape[0]), len(antenna.slants), antenna

    def set_devices(self, tx, rx, rx_set_offsets=None):
        self.set_tx(tx.pos, tx.ypr, tx.antenna)
        self.set_rx(rx.pos, rx.ypr, rx.antenna, rx_set_offsets)

    def compute_paths(self, max_depth, num_rays, los=True, reflection=True, record_rays=False) -> int:
        self.sync_stream()
        flags = (RT_LOS if los else 0) | (RT_REFLECTION if reflection else 0) | (RT_RECORD_RAYS if record_rays else 0)
        self.n_paths = rt_compute_paths(self.ctx, max_depth, num_rays, flags)
        self.max_depth = max(int(max_depth), 1)
        self.num_rays = int(num_rays)
        return self.n_paths

    @property
    def n_pairs(self) -> int:
        return rt_num_pairs(self.ctx)

    def paths(self):
        """offsets [pairs+1], seq [P, D], points [P, D, 3], depth [P], length [P] (float64)."""
        P, D = self.n_paths, self.max_depth
        dev = self.device
        out = dict(offsets=torch.empty(self.n_pairs + 1, dtype=torch.int64, device=dev),
                   seq=torch.empty((max(P, 1), D), dtype=torch.int32, device=dev),
                   points=torch.empty((max(P, 1), D, 3), dtype=torch.float32, device=dev),
                   depth=torch.empty(max(P, 1), dtype=torch.int32, device=dev),
                   length=torch.empty(max(P, 1), dtype=torch.float64, device=dev))
        rt_get_paths(self.ctx, out["offsets"], out["seq"], out["points"], out["depth"], out["length"])
        for k in ("seq", "points", "depth", "length"):
            out[k] = out[k][:P]
        return out

    def path_pairs(self):
        """int64 [P]: the (tx, rx) pair index of every stored path."""
        off = self.paths()["offsets"]
        return torch.repeat_interleave(torch.arange(off.numel() - 1, device=self.device), off[1:] - off[:-1])

    def candidates(self):
        n = rt_get_candidates(self.ctx)
        D, dev = self.max_depth, self.device
        tx = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        dep = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        seq = torch.empty((max(n, 1), D), dtype=torch.int32, device=dev)
        wit = torch.empty(max(n, 1), dtype=torch.int64, device=dev)
        rt_get_candidates(self.ctx, tx, dep, seq, wit)
        return tx[:n], dep[:n], seq[:n], wit[:n]

    def ray_hits(self):
        h = torch.empty((self.n_tx, self.num_rays, self.max_depth), dtype=torch.int32, device=self.device)
        rt_get_ray_hits(self.ctx, h)
        return h

    def ray_directions(self, num_rays, first=0, n=None):
        n = num_rays - first if n is None else n
        d = torch.empty((n, 3), dtype=torch.float32, device=self.device)
        rt_ray_directions(self.ctx, num_rays, first, n, d)
        return d

    def cir_raw(self, los=True, reflection=True):
        """a as float32 [P, nrp, ntp, 2] (interleaved complex) and tau [P]."""
        self.sync_stream()
        P = self.n_paths
        a = torch.empty((max(P, 1), self.nrp, self.ntp, 2), dtype=torch.float32, device=self.device)
        tau = torch.empty(max(P, 1), dtype=torch.float32, device=self.device)
        rt_cir(self.ctx, (RT_LOS if los else 0) | (RT_REFLECTION if reflection else 0), a, tau)
        return a[:P], tau[:P]

    def cir(self, los=True, reflection=True):
        a, tau = self.cir_raw(los, reflection)
        return torch.view_as_complex(a), tau

    def apply_doppler(self, a, fs, n_steps, tx_velocities, rx_velocities=None):
        """Sec. II-A (Listing 3): a [P, nrp, ntp] complex -> [P, nrp, ntp, n_steps]
        with a_i(t_n) = a_i exp(j 2 pi f_D,i n / fs) from the devices' velocities
        (tx [n_tx, 3] or [3], rx [n_rx, 3] or None; m/s)."""
        self.sync_stream()
        dev = self.device
        vt = self._t(tx_velocities, torch.float32).reshape(-1, 3)
        if vt.shape[0] == 1 and self.n_tx > 1:
            vt = vt.expand(self.n_tx, 3)
        vt = vt.contiguous()
        vr = None
        if rx_velocities is not None:
            vr = self._t(rx_velocities, torch.float32).reshape(-1, 3)
            if vr.shape[0] == 1 and self.n_rx > 1:
                vr = vr.expand(self.n_rx, 3)
            vr = vr.contiguous()
        a_raw = torch.view_as_real(a.to(torch.complex64).contiguous()).contiguous()
        P = a_raw.shape[0]
        out = torch.empty((max(P, 1),) + tuple(a_raw.shape[1:-1]) + (int(n_steps), 2), dtype=torch.float32,
                          device=dev)
        if self.n_paths:
            rt_apply_doppler(self.ctx, a_raw, vt, vr, fs, n_steps, out)
        return torch.view_as_complex(out[:P])

    def apply_array(self, a, tx_elements=None, rx_elements=None):
        """Sec. II, synthetic arrays: a [P, nrp, ntp] complex -> [P, Mr*nrp, Mt*ntp]
        with every element pair's plane-wave phase (element positions [M, 3] in
        metres in the devices' frames; None: one element at the centre)."""
        self.sync_stream()
        te = self._t(tx_elements, torch.float32).reshape(-1, 3) if tx_elements is not None else None
        re = self._t(rx_elements, torch.float32).reshape(-1, 3) if rx_elements is not None else None
        Mt = te.shape[0] if te is not None else 1
        Mr = re.shape[0] if re is not None else 1
        a_raw = torch.view_as_real(a.to(torch.complex64).contiguous()).contiguous()
        P, nrp, ntp = a_raw.shape[0], a_raw.shape[1], a_raw.shape[2]
        out = torch.empty((max(P, 1), Mr * nrp, Mt * ntp, 2), dtype=torch.float32, device=self.device)
        if self.n_paths:
            rt_apply_array(self.ctx, a_raw, te, re, out)
        return torch.view_as_complex(out[:P])

    def compute_diffraction(self) -> int:
        """Sec. II-B: first-order diffracted paths of every (tx, rx) pair; returns their count."""
        self.sync_stream()
        n = ctypes.c_int64()
        _check(self.ctx, lib().rt_compute_diffraction(self.ctx, ctypes.byref(n)))
        self.n_dpaths = int(n.value)
        return self.n_dpaths

    def diffraction(self):
        """offsets [n_pairs+1], wedge [P], points [P, 3] of the diffracted paths."""
        self.sync_stream()
        P = self.n_dpaths
        off = torch.empty(self.n_pairs + 1, dtype=torch.int64, device=self.device)
        wedge = torch.empty(max(P, 1), dtype=torch.int32, device=self.device)
        pts = torch.empty((max(P, 1), 3), dtype=torch.float32, device=self.device)
        _check(self.ctx, lib().rt_get_diffraction(self.ctx, _ptr(off), _ptr(wedge), _ptr(pts)))
        return {"offsets": off, "wedge": wedge[:P], "points": pts[:P]}

    def wedges(self):
        """faces [n, 2] (original triangle ids) and exterior angle / pi [n] of the scene's wedges."""
        self.sync_stream()
        n = ctypes.c_int64()
        _check(self.ctx, lib().rt_get_wedges(self.ctx, ctypes.byref(n), None, None))
        faces = torch.empty((max(n.value, 1), 2), dtype=torch.int32, device=self.device)
        ne = torch.empty(max(n.value, 1), dtype=torch.float32, device=self.device)
        _check(self.ctx, lib().rt_get_wedges(self.ctx, ctypes.byref(n), _ptr(faces), _ptr(ne)))
        return faces[:n.value], ne[:n.value]

    def coverage_map_diffraction(self, grid: dict, tx_port: int = 0):
        """First-order diffracted part of the coverage map [n_tx, ny, nx]: the
        incoherent path gain of the diffracted paths to every cell centre."""
        self.sync_stream()
        g = rt_grid(float(grid["x0"]), float(grid["y0"]), float(grid["cell"]), float(grid["h"]),
                    int(grid["nx"]), int(grid["ny"]))
        gain = torch.empty((self.n_tx, g.ny, g.nx), dtype=torch.float32, device=self.device)
        _check(self.ctx, lib().rt_coverage_map_diffraction(self.ctx, ctypes.byref(g), int(tx_port), _ptr(gain)))
        return gain

    def set_scattering(self, coeff):
        """Scattering coefficients S [n_mat] of the scene's materials (0..1)."""
        self.sync_stream()
        c = self._t(coeff, torch.float32).reshape(-1)
        _check(self.ctx, lib().rt_set_scattering(self.ctx, _ptr(c), int(c.shape[0])))
        torch.cuda.current_stream().synchronize()

    def set_scattering_pattern(self, alpha_r):
        """Pattern per material: -1 Lambertian, 0..64 directive lobe exponent alpha_R."""
        self.sync_stream()
        a = np.ascontiguousarray(np.asarray(alpha_r, dtype=np.int32).reshape(-1))
        _check(self.ctx, lib().rt_set_scattering_pattern(self.ctx, a.ctypes.data, int(a.shape[0])))

    def scattering_gain(self, num_rays: int):
        """Incoherent first-order diffuse-scattering gain [n_pairs, nrp, ntp]."""
        self.sync_stream()
        g = torch.empty((self.n_pairs, self.nrp, self.ntp), dtype=torch.float32, device=self.device)
        _check(self.ctx, lib().rt_scattering_gain(self.ctx, int(num_rays), _ptr(g)))
        return g

    def scattering_gain_vjp(self, num_rays: int, grad_gain):
        """dL/dS [n_mat] from dL/dgain [n_pairs, nrp, ntp] of scattering_gain."""
        self.sync_stream()
        up = self._t(grad_gain, torch.float32).contiguous()
        if up.numel() != self.n_pairs * self.nrp * self.ntp:
            raise RtError(-1, "scattering_gain_vjp: grad_gain must have n_pairs * nrp * ntp elements")
        gs = torch.empty(self.n_mat, dtype=torch.float32, device=self.device)
        _check(self.ctx, lib().rt_scattering_gain_vjp(self.ctx, int(num_rays), _ptr(up), _ptr(gs)))
        return gs

    def diffraction_cir(self):
        """a [P, nrp, ntp] complex64 and tau [P] of the diffracted paths (UTD)."""
        self.sync_stream()
        P = self.n_dpaths
        a = torch.empty((max(P, 1), self.nrp, self.ntp, 2), dtype=torch.float32, device=self.device)
        tau = torch.empty(max(P, 1), dtype=torch.float32, device=self.device)
        _check(self.ctx, lib().rt_diffraction_cir(self.ctx, _ptr(a), _ptr(tau)))
        return torch.view_as_complex(a[:P]), tau[:P]

    def pair_gain(self, a_raw, floor_db=-400.0):
        """[pairs, 2] = (has path, incoherent path gain dB) from cir_raw's a."""
        self.sync_stream()
        out = torch.empty((self.n_pairs, 2), dtype=torch.float32, device=self.device)
        a_raw = a_raw.contiguous() if a_raw.numel() else torch.zeros((1, self.nrp, self.ntp, 2), device=self.device)
        rt_pair_gain(self.ctx, a_raw, floor_db, out)
        return out

    def freq_response_raw(self, a_raw, tau, freqs):
        self.sync_stream()
        freqs = self._t(freqs, torch.float64)
        K = int(freqs.shape[0])
        H = torch.empty((self.n_pairs, self.nrp, self.ntp, K, 2), dtype=torch.float32, device=self.device)
        a_raw = a_raw.contiguous() if a_raw.numel() else torch.zeros((1, self.nrp, self.ntp, 2), device=self.device)
        tau = tau.contiguous() if tau.numel() else torch.zeros(1, device=self.device)
        rt_freq_response(self.ctx, a_raw, tau, freqs, H)
        return H

    def freq_response(self, a, tau, freqs):
        a_raw = torch.view_as_real(a.contiguous()) if a.is_complex() else a
        return torch.view_as_complex(self.freq_response_raw(a_raw.contiguous(), tau, freqs))

    def coverage_map_backward(self, grid: dict, max_depth: int, num_rays: int, grad_gain, tx_port: int = 0):
        """d(sum grad_gain * gain)/d(tx yaw, pitch, roll) [n_tx, 3] (Sec. III-B)."""
        self.sync_stream()
        g = rt_grid(float(grid["x0"]), float(grid["y0"]), float(grid["cell"]), float(grid["h"]),
                    int(grid["nx"]), int(grid["ny"]))
        gg = self._t(grad_gain, torch.float32).contiguous()
        out = torch.empty((self.n_tx, 3), dtype=torch.float32, device=self.device)
        _check(self.ctx, lib().rt_coverage_map_backward(self.ctx, ctypes.byref(g), int(max_depth), int(num_rays),
                                                        int(tx_port), _ptr(gg), _ptr(out)))
        return out

    def coverage_map(self, grid: dict, max_depth: int, num_rays: int, tx_port: int = 0):
        self.sync_stream()
        g = rt_grid(float(grid["x0"]), float(grid["y0"]), float(grid["cell"]), float(grid["h"]),
                    int(grid["nx"]), int(grid["ny"]))
        gain = torch.empty((self.n_tx, g.ny, g.nx), dtype=torch.float32, device=self.device)
        hits = torch.empty((self.n_tx, g.ny, g.nx), dtype=torch.int32, device=self.device)
        rt_coverage_map(self.ctx, g, max_depth, num_rays, tx_port, gain, hits)
        return gain, hits

    def coverage_map_async(self, grid: dict, max_depth: int, num_rays: int, tx_port: int = 0,
                           after_trace: bool = False, blocks_per_sm: int = 0):
        """coverage_map traced beside the calls that follow (after_trace: from the
        next compute_paths' ray trace on); call join() before reading the tensors."""
        self.sync_stream()
        g = rt_grid(float(grid["x0"]), float(grid["y0"]), float(grid["cell"]), float(grid["h"]),
                    int(grid["nx"]), int(grid["ny"]))
        gain = torch.empty((self.n_tx, g.ny, g.nx), dtype=torch.float32, device=self.device)
        hits = torch.empty((self.n_tx, g.ny, g.nx), dtype=torch.int32, device=self.device)
        rt_coverage_map_async(self.ctx, g, max_depth, num_rays, tx_port, gain, hits,
                              ASYNC_AFTER_TRACE if after_trace else 0, blocks_per_sm)
        self._async_out = (gain, hits)   # kept alive while the second stream may write them
        return gain, hits

    def join(self):
        """Order the current stream after the last coverage_map_async."""
        self.sync_stream()
        rt_join(self.ctx)
        self._async_out = None

    def coverage_map_ranges(self, grid: dict, max_depth: int, num_rays: int, ranges, tx_port: int = 0):
        """Coverage map accumulated over lattice ray ranges [(first, count), ...]."""
        self.sync_stream()
        g = rt_grid(float(grid["x0"]), float(grid["y0"]), float(grid["cell"]), float(grid["h"]),
                    int(grid["nx"]), int(grid["ny"]))
        gain = torch.zeros((self.n_tx, g.ny, g.nx), dtype=torch.float32, device=self.device)
        hits = torch.zeros((self.n_tx, g.ny, g.nx), dtype=torch.int32, device=self.device)
        for first, count in ranges:
            rt_coverage_map_accumulate(self.ctx, g, max_depth, num_rays, first, count, tx_port, gain, hits)
        return gain, hits

    # gradients --------------------------------------------------------------
    def cir_backward(self, grad_a, grad_tau=None, los=True, reflection=True):
        """Returns (g_eps [M], g_sigma [M], g_txpos [n_tx, 3], g_txypr [n_tx, 3])."""
        self.sync_stream()
        dev = self.device
        ge = torch.zeros(self.n_mat, dtype=torch.float32, device=dev)
        gs = torch.zeros(self.n_mat, dtype=torch.float32, device=dev)
        gp = torch.zeros((self.n_tx, 3), dtype=torch.float32, device=dev)
        gy = torch.zeros((self.n_tx, 3), dtype=torch.float32, device=dev)
        ga = torch.view_as_real(grad_a.to(torch.complex64).contiguous()).contiguous()
        gt = grad_tau.to(torch.float32).contiguous() if grad_tau is not None else None
        if self.n_paths:
            rt_cir_backward(self.ctx, (RT_LOS if los else 0) | (RT_REFLECTION if reflection else 0), ga, gt,
                            ge, gs, gp, gy)
        return ge, gs, gp, gy

    def freq_response_backward(self, a, tau, freqs, grad_H):
        self.sync_stream()
        freqs = self._t(freqs, torch.float64)
        P = self.n_paths
        ga = torch.empty((max(P, 1), self.nrp, self.ntp, 2), dtype=torch.float32, device=self.device)
        gt = torch.empty(max(P, 1), dtype=torch.float32, device=self.device)
        if P:
            rt_freq_response_backward(self.ctx, torch.view_as_real(a.contiguous()).contiguous(), tau.contiguous(),
                                      freqs, torch.view_as_real(grad_H.to(torch.complex64).contiguous()).contiguous(),
                                      ga, gt)
        return torch.view_as_complex(ga[:P]), gt[:P]


class CIR(torch.autograd.Function):
    """(eps_r [M], sigma [M], tx_pos [n,3], tx_ypr [n,3]) -> (a [P,nrp,ntp], tau [P]).

    The forward uploads the parameters to the tracer and evaluates the stored
    paths (they must have been computed for this geometry); the backward
    replays them through rt_cir_backward.
    """

    @staticmethod
    def forward(ctx, tracer, eps_r, sigma, tx_pos, tx_ypr):
        tracer.set_materials(torch.stack([eps_r.detach(), sigma.detach()], 1).float())
        tracer.set_tx(tx_pos.detach().float(), tx_ypr.detach().float(), tracer.tx_antenna)
        a, tau = tracer.cir()
        ctx.tracer = tracer
        return a, tau

    @staticmethod
    def backward(ctx, grad_a, grad_tau):
        tr = ctx.tracer
        if grad_a is None:
            grad_a = torch.zeros((tr.n_paths, tr.nrp, tr.ntp), dtype=torch.complex64, device=tr.device)
        ge, gs, gp, gy = tr.cir_backward(grad_a, grad_tau)
        return None, ge, gs, gp, gy


class CoverageMap(torch.autograd.Function):
    """tx_ypr [n_tx, 3] -> gain map [n_tx, ny, nx]; backward through
    rt_coverage_map_backward (gradients with respect to the orientation)."""

    @staticmethod
    def forward(ctx, tracer, tx_ypr, grid, max_depth, num_rays, tx_port=0):
        tracer.set_tx(tracer._tx_pos, tx_ypr.detach().float(), tracer.tx_antenna)
        g, _ = tracer.coverage_map(grid, max_depth, num_rays, tx_port)
        ctx.args = (tracer, grid, max_depth, num_rays, tx_port)
        return g

    @staticmethod
    def backward(ctx, grad_gain):
        tracer, grid, max_depth, num_rays, tx_port = ctx.args
        return None, tracer.coverage_map_backward(grid, max_depth, num_rays, grad_gain, tx_port), None, None, None, None


class FreqResponse(torch.autograd.Function):
    """(a [P,nrp,ntp], tau [P]) -> H [pairs, nrp, ntp, K] with rt_freq_response(_backward)."""

    @staticmethod
    def forward(ctx, tracer, a, tau, freqs):
        ctx.tracer = tracer
        ctx.save_for_backward(a, tau, freqs)
        return tracer.freq_response(a, tau, freqs)

    @staticmethod
    def backward(ctx, grad_H):
        a, tau, freqs = ctx.saved_tensors
        ga, gt = ctx.tracer.freq_response_backward(a, tau, freqs, grad_H)
        return None, ga, gt, None


# ------------------------------------------------------------ surrogate MLP
def rt_gemm_bf16(A, B, bias=None, relu=False, out_bf16=False, status=None):
    """C = act(A B^T + bias) on tcgen05 (A [M, K], B [N, K] bfloat16 CUDA tensors)."""
    M, K = A.shape
    N = B.shape[0]
    C = torch.empty((M, N), dtype=torch.bfloat16 if out_bf16 else torch.float32, device=A.device)
    code = lib().rt_gemm_bf16(_stream(), _ptr(A), _ptr(B), int(M), int(N), int(K), _ptr(bias), int(bool(relu)),
                              int(bool(out_bf16)), _ptr(C), _ptr(status))
    if code:
        raise RtError(code, "rt_gemm_bf16 failed")
    return C


class Surrogate:
    """Fourier-feature MLP path-gain surrogate (rt_mlp_* C ABI)."""

    def __init__(self, lo, hi, n_freq=32, width=256, n_hidden=8, sigma=1.0, seed=0, device=0):
        self.F, self.W, self.L = n_freq, width, n_hidden
        self.device = torch.device("cuda", device)
        self.h = ctypes.c_void_p()
        lo = (ctypes.c_float * 6)(*[float(v) for v in lo])
        hi = (ctypes.c_float * 6)(*[float(v) for v in hi])
        code = lib().rt_mlp_create(ctypes.byref(self.h), device, _stream(), n_freq, width, n_hidden,
                                   float(sigma), int(seed), ctypes.cast(lo, ctypes.c_void_p),
                                   ctypes.cast(hi, ctypes.c_void_p))
        if code:
            raise RtError(code, "rt_mlp_create failed")
        n = ctypes.c_int64()
        lib().rt_mlp_num_params(self.h, ctypes.byref(n))
        self.n_params = int(n.value)

    def _check(self, code):
        if code:
            buf = ctypes.create_string_buffer(512)
            lib().rt_mlp_last_error(self.h, buf, 512)
            raise RtError(code, buf.value.decode())

    def close(self):
        if self.h:
            lib().rt_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _sync(self):
        lib().rt_mlp_set_stream(self.h, _stream())

    def set_baseline(self, wavelength):
        """Free-space (Friis) baseline: the gain head learns the residual."""
        self._check(lib().rt_mlp_set_baseline(self.h, float(wavelength)))

    def train_step(self, x, target, lr, loss_acc=None):
        self._sync()
        self._check(lib().rt_mlp_train_step(self.h, _ptr(x.contiguous()), _ptr(target.contiguous()),
                                            int(x.shape[0]), float(lr), _ptr(loss_acc)))

    def infer(self, x):
        self._sync()
        out = torch.empty((x.shape[0], 2), dtype=torch.float32, device=self.device)
        self._check(lib().rt_mlp_infer(self.h, _ptr(x.contiguous()), int(x.shape[0]), _ptr(out)))
        return out

    def infer_layers(self, x):
        """Layer-by-layer GEMM path (the reference of the fused inference kernel)."""
        self._sync()
        out = torch.empty((x.shape[0], 2), dtype=torch.float32, device=self.device)
        self._check(lib().rt_mlp_infer_layers(self.h, _ptr(x.contiguous()), int(x.shape[0]), _ptr(out)))
        return out

    def params(self):
        p = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        self._sync()
        self._check(lib().rt_mlp_get_params(self.h, _ptr(p)))
        return p

    def set_params(self, p):
        self._sync()
        self._check(lib().rt_mlp_set_params(self.h, _ptr(p.to(torch.float32).contiguous())))

    def save(self) -> bytes:
        """Serialised model (rt_mlp_save): shape, normalisation box, parameters."""
        self._sync()
        n = ctypes.c_int64()
        self._check(lib().rt_mlp_save(self.h, None, 0, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(int(n.value))
        self._check(lib().rt_mlp_save(self.h, ctypes.cast(buf, ctypes.c_void_p), int(n.value), ctypes.byref(n)))
        return buf.raw[:int(n.value)]

    @classmethod
    def load(cls, data: bytes, device: int = 0) -> "Surrogate":
        """A model from rt_mlp_save's bytes (rt_mlp_load)."""
        self = cls.__new__(cls)
        self.device = torch.device("cuda", device)
        self.h = ctypes.c_void_p()
        buf = ctypes.create_string_buffer(bytes(data), len(data))
        code = lib().rt_mlp_load(ctypes.byref(self.h), device, _stream(), ctypes.cast(buf, ctypes.c_void_p), len(data))
        if code:
            self.h = None
            raise RtError(code, "rt_mlp_load failed")
        self.F, self.W, self.L = (int(v) for v in np.frombuffer(bytes(data[8:20]), dtype="<i4"))
        n = ctypes.c_int64()
        lib().rt_mlp_num_params(self.h, ctypes.byref(n))
        self.n_params = int(n.value)
        return self

    def grads(self):
        g = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        self._sync()
        self._check(lib().rt_mlp_get_grads(self.h, _ptr(g)))
        return g

    def status(self) -> int:
        s = ctypes.c_uint32()
        self._check(lib().rt_mlp_status(self.h, ctypes.byref(s)))
        return int(s.value)

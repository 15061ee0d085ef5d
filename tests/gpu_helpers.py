"""Shared helpers of the GPU parity tests: run the CUDA path and the oracle
on the same seeded inputs and compare what is unique, excusing only
decisions the oracle marks near-degenerate (margin < eps)."""
from __future__ import annotations

import numpy as np
import torch

from oracle import oracle as O
from paper_2303_11103_gb300 import rt
from paper_2303_11103_gb300 import scenes as S

FC = 3.5e9

# Tolerances of the floating-point outputs (float32 path vs FP64 oracle).
TAU_REL = 1e-4          # path delays
A_REL, A_ABS = 1e-3, 1e-5   # |da| <= A_REL |a| + A_ABS max|a| (per receiver)
H_REL, H_ABS = 1e-3, 1e-5   # |dH| <= H_REL |H| + H_ABS sum_i |a_i| (per pair, port pair)
CM_DB = 0.05            # coverage cells with >= 16 hits
GRAD_REL = 1e-3


def gpu_paths(tr: rt.Tracer):
    """Per pair: list of (seq tuple) in GPU order, plus the raw tensors."""
    p = tr.paths()
    off = p["offsets"].cpu().numpy()
    seq = p["seq"].cpu().numpy()
    dep = p["depth"].cpu().numpy()
    out = []
    for q in range(len(off) - 1):
        out.append([tuple(int(x) for x in seq[i, :dep[i]]) for i in range(off[q], off[q + 1])])
    return out, p


def gpu_candidates(tr: rt.Tracer, tx_index: int = 0):
    tx, dep, seq, wit = (x.cpu().numpy() for x in tr.candidates())
    out = {}
    for i in range(len(tx)):
        if tx[i] != tx_index:
            continue
        out[tuple(int(x) for x in seq[i, :dep[i]])] = int(wit[i])
    return out


def compare_candidates(osc, tx, N, D, gpu_c, ora_c):
    """Candidate-set parity. Returns (n_common, n_excused)."""
    excused = 0
    for s, (m, r) in ora_c.items():
        if m >= osc.eps:
            assert s in gpu_c, f"oracle candidate {s} (margin {m}) missing on the GPU"
        elif s not in gpu_c:
            excused += 1
    extra = [s for s in gpu_c if s and s not in ora_c]
    for s in extra:
        w = gpu_c[s]
        hits, marg = O.trace_sbr(osc, tx, N, D, np.array([w]))
        K = len(s)
        assert marg[0, K - 1] < osc.eps, f"GPU candidate {s} from ray {w} is not near-degenerate in the oracle"
        excused += 1
    return len(set(gpu_c) & set(ora_c)), excused


def compare_path_sets(osc, tx, rxs, gpu_sets, ora_paths, ora_c):
    """Path-set parity per receiver. Returns dict rx -> set of common robust seqs."""
    common = {}
    for r in range(len(rxs)):
        ora_valid = {p.seq: p for p in ora_paths if p.rx == r and p.valid}
        ora_near = {p.seq for p in ora_paths if p.rx == r and p.margin < osc.eps}
        g = set(gpu_sets[r])
        assert len(g) == len(gpu_sets[r]), "duplicate path on the GPU"
        for s, p in ora_valid.items():
            disc_ok = (len(s) == 0) or (s in ora_c and ora_c[s][0] >= osc.eps)
            if p.margin >= osc.eps and disc_ok:
                assert s in g, f"rx {r}: oracle path {s} (margin {p.margin}) missing on the GPU"
        for s in g - set(ora_valid):
            if s in ora_near:
                continue
            ok, pts, length, m = O.image_path(osc, tx, rxs[r], s)
            assert ok or m < osc.eps, f"rx {r}: GPU path {s} is invalid in the oracle (margin {m})"
            # a valid path the oracle did not discover: discovery must be marginal
            assert (s not in ora_c) or ora_c[s][0] < osc.eps
        common[r] = {s for s in g & set(ora_valid) if ora_valid[s].margin >= osc.eps}
    return common


def setup(tr, scene, tx, rx, rx_sets=None):
    tr.load_scene(scene)
    tr.set_devices(tx, rx, rx_sets)

"""Helpers shared by the GPU tests (no method arithmetic here)."""

import numpy as np

import oracle
from synth import make_workload, normal_weights, random_structure


_models = {}


def get_model(spec):
    import paper_2402_03789_gb300 as sn
    key = repr(spec)
    if key not in _models:
        _models[key] = sn.SevenNet(spec, normal_weights(oracle.n_params(spec)), device=0)
    return _models[key]


def edge_set(dst, src, shift, pos, cell, rc, band=1e-6):
    """Edges as a set of tuples, dropping pairs within `band` of the cutoff."""
    d = pos[src] - pos[dst] + shift @ cell
    r = np.sqrt((d * d).sum(1))
    keep = np.abs(r - rc) > band
    return {(int(a), int(b), int(x), int(y), int(z))
            for a, b, (x, y, z) in zip(dst[keep], src[keep], shift[keep])}


def errors(E, F, W, Eo, Fo, Wo, n):
    f_rel = float(np.linalg.norm(F - Fo) / max(np.linalg.norm(Fo), 1e-300))
    e_pa = abs(E - Eo) / max(n, 1)
    w_rel = float(np.linalg.norm(W - Wo) / max(np.linalg.norm(Wo), 1e-300))
    return e_pa, f_rel, w_rel

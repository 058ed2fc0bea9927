"""Periodic neighbour lists (FP64), the graph of Sec. 2: nodes v, w joined when
|r_w - r_v| < r_c, every periodic image counted, self-images included.

Edges are directed: edge (v, w, S) has receiver v, sender w and displacement
    d = r_w - r_v + S @ cell     (S an integer 3-vector, cell rows = lattice vectors)
which is r_vw of Sec. 3.1.  Both directions of every pair are present.  The
returned arrays are sorted by (v, w, S) lexicographically.
"""

import math

import numpy as np


def _image_range(cell: np.ndarray, r_cut: float, pbc) -> list:
    vol = abs(np.linalg.det(cell))
    k = []
    for i in range(3):
        if not pbc[i]:
            k.append(0)
            continue
        a, b = cell[(i + 1) % 3], cell[(i + 2) % 3]
        width = vol / np.linalg.norm(np.cross(a, b))
        k.append(int(math.ceil(r_cut / width)) + 1)
    return k


def _sort_edges(dst, src, shift):
    order = np.lexsort((shift[:, 2], shift[:, 1], shift[:, 0], src, dst))
    return dst[order], src[order], shift[order]


def neighbor_list_bruteforce(pos, cell, r_cut, pbc=(True, True, True)):
    """All (v, w, S) with 0 < |r_w - r_v + S cell| < r_c.

    Positions are first wrapped into the cell along periodic directions
    (r = r~ + n cell, n integer); images S~ in [-k, k]^3 of the wrapped
    positions with k_i = ceil(r_c / perpendicular width_i) + 1 are searched,
    and S = S~ - n_w + n_v refers back to the given positions.
    O(N^2 * images); for small cells only.
    """
    pos = np.asarray(pos, np.float64)
    cell = np.asarray(cell, np.float64)
    frac = pos @ np.linalg.inv(cell)
    fl = np.where(np.asarray(pbc)[None, :], np.floor(frac), 0.0)
    wrapped = pos - fl @ cell
    k = _image_range(cell, r_cut, pbc)
    shifts = np.array([(a, b, c) for a in range(-k[0], k[0] + 1)
                       for b in range(-k[1], k[1] + 1)
                       for c in range(-k[2], k[2] + 1)], dtype=np.int64)
    n = pos.shape[0]
    D, S, W = [], [], []
    r2 = r_cut * r_cut
    for v in range(n):
        d = wrapped[None, :, :] - wrapped[v][None, None, :] + (shifts @ cell)[:, None, :]
        dd = (d * d).sum(-1)                       # [n_shift, n]
        keep = (dd < r2) & (dd > 0.0)
        si, wi = np.nonzero(keep)
        D.append(np.full(wi.shape[0], v, np.int64))
        W.append(wi)
        S.append(shifts[si] - fl[wi].astype(np.int64) + fl[v].astype(np.int64))
    dst = np.concatenate(D)
    src = np.concatenate(W)
    shift = np.concatenate(S).reshape(-1, 3)
    return _sort_edges(dst, src, shift)


def neighbor_list(pos, cell, r_cut, pbc=(True, True, True)):
    """Same edge set for large orthorhombic periodic cells (edge >= 2 r_c),
    via scipy's periodic k-d tree; other cells go to the brute force."""
    pos = np.asarray(pos, np.float64)
    cell = np.asarray(cell, np.float64)
    diag = np.diag(cell)
    ortho = np.allclose(cell, np.diag(diag)) and all(pbc)
    if not ortho or diag.min() < 2.0 * r_cut + 1e-9 or pos.shape[0] < 400:
        return neighbor_list_bruteforce(pos, cell, r_cut, pbc)
    from scipy.spatial import cKDTree
    frac_floor = np.floor(pos / diag)
    wrapped = pos - frac_floor * diag
    wrapped = np.where(wrapped >= diag, wrapped - diag, wrapped)
    tree = cKDTree(wrapped, boxsize=diag)
    pairs = tree.query_pairs(r_cut, output_type="ndarray")
    i, j = pairs[:, 0], pairs[:, 1]
    # minimum-image shift in the wrapped frame, then back to original positions
    dw = wrapped[j] - wrapped[i]
    s_w = -np.round(dw / diag)
    shift = s_w - frac_floor[j] + frac_floor[i]
    d = pos[j] - pos[i] + shift * diag
    dd = (d * d).sum(-1)
    keep = (dd < r_cut * r_cut) & (dd > 0)
    i, j, shift = i[keep], j[keep], shift[keep].astype(np.int64)
    dst = np.concatenate([i, j])
    src = np.concatenate([j, i])
    sh = np.concatenate([shift, -shift])
    return _sort_edges(dst, src, sh)

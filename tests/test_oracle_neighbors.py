"""Pins of the oracle neighbour lists against a literal triple loop."""

import itertools

import numpy as np

from oracle.neighbors import neighbor_list_bruteforce, neighbor_list
from synth import random_structure


def _literal(pos, cell, rc, kmax):
    out = set()
    n = len(pos)
    for v in range(n):
        for w in range(n):
            for S in itertools.product(range(-kmax, kmax + 1), repeat=3):
                d = pos[w] + np.array(S) @ cell - pos[v]
                r = float(np.sqrt((d * d).sum()))
                if 0 < r < rc:
                    out.add((v, w) + tuple(S))
    return out


def _as_set(edges):
    dst, src, sh = edges
    return {(int(a), int(b)) + tuple(int(x) for x in s) for a, b, s in zip(dst, src, sh)}


def test_bruteforce_matches_literal_loop_on_small_triclinic_cell():
    rng = np.random.default_rng(0)
    cell = np.array([[4.2, 0.0, 0.0], [1.1, 3.9, 0.0], [0.7, -0.6, 4.4]])
    pos = rng.uniform(0, 1, (6, 3)) @ cell + rng.normal(0, 2.0, (6, 3))  # some atoms outside
    e = neighbor_list_bruteforce(pos, cell, 5.0)
    lit = _literal(pos, cell, 5.0, 4)
    assert _as_set(e) == lit
    # self-images are present in a cell smaller than r_c
    assert any(a == b for a, b, *_ in lit)


def test_edges_come_in_reverse_pairs():
    s = random_structure({"Si": 10, "N": 6}, 3.1, 1.5, seed=3)
    dst, src, sh = neighbor_list_bruteforce(s.pos, s.cell, 5.0)
    fwd = _as_set((dst, src, sh))
    rev = _as_set((src, dst, -sh))
    assert fwd == rev


def test_kdtree_path_matches_bruteforce():
    s = random_structure({"Si": 200, "O": 400}, 2.2, 1.6, seed=9)
    pos = s.pos.copy()
    pos[:5] += s.cell[0] * 1.0      # unwrapped atoms
    pos[5:9] -= s.cell[2] * 2.0
    a = neighbor_list_bruteforce(pos, s.cell, 5.0)
    b = neighbor_list(pos, s.cell, 5.0)
    assert len(b[0]) > 0 and _as_set(a) == _as_set(b)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)

"""Full-size workloads (24,000-atom SiO2, 112,000-atom Si3N4) in the launch
configuration bench.py times: the edge set against the oracle's neighbour
list, and properties that hold at any size (zero net force, symmetric
virial, translation invariance, rotation equivariance, permutation invariance,
BF16 within the force tolerance of FP32)."""

import numpy as np
import pytest

import oracle
from synth import make_workload
from gpu_common import get_model

pytestmark = pytest.mark.gpu

_cache = {}


def _work(name):
    if name not in _cache:
        _cache[name] = make_workload(name)
    return _cache[name]


def _sorted_edges(dst, src, sh, pos, cell, rc, band=1e-6):
    d = pos[src] - pos[dst] + sh @ cell
    r = np.sqrt((d * d).sum(1))
    keep = np.abs(r - rc) > band
    dst, src, sh = dst[keep], src[keep], sh[keep]
    o = np.lexsort((sh[:, 2], sh[:, 1], sh[:, 0], src, dst))
    return np.stack([dst[o], src[o], sh[o, 0], sh[o, 1], sh[o, 2]], 1).astype(np.int64)


@pytest.mark.parametrize("name", ["sio2_24000", "si3n4_112000"])
def test_full_size_edge_set(name):
    s, spec = _work(name)
    model = get_model(spec)
    a = _sorted_edges(*model.neighbors(s.pos, s.cell), s.pos, s.cell, spec.r_cut)
    b = _sorted_edges(*oracle.neighbor_list(s.pos, s.cell, spec.r_cut), s.pos, s.cell, spec.r_cut)
    assert a.shape == b.shape and np.array_equal(a, b)


@pytest.mark.parametrize("name", ["sio2_24000", "si3n4_112000"])
def test_full_size_properties(name):
    s, spec = _work(name)
    model = get_model(spec)
    E32, F32, W32 = model.evaluate(s.pos, s.cell, s.species, "fp32")
    E16, F16, W16 = model.evaluate(s.pos, s.cell, s.species, "bf16")
    for E, F, W in ((E32, F32, W32), (E16, F16, W16)):
        assert np.isfinite(E) and np.all(np.isfinite(F))
        assert np.abs(F.sum(0)).max() <= 1e-9 * np.abs(F).sum()
        assert np.abs(W - W.T).max() <= 1e-4 * np.abs(W).max()
    f_rel = np.linalg.norm(F16 - F32) / np.linalg.norm(F32)
    print(f"{name}: bf16 vs fp32 force rel {f_rel:.2e}, dE/N {abs(E16 - E32) / s.n_atoms:.2e}")
    assert f_rel <= 5e-3
    Et, Ft, Wt = model.evaluate(s.pos + np.array([0.37, -1.21, 2.9]), s.cell, s.species, "fp32")
    assert abs(Et - E32) / s.n_atoms <= 1e-6
    assert np.linalg.norm(Ft - F32) / np.linalg.norm(F32) <= 1e-5


@pytest.mark.parametrize("name", ["sio2_24000", "si3n4_112000"])
def test_full_size_rotation_and_permutation(name):
    # E is invariant and F, W equivariant under a rotation of positions and cell
    # (r -> R r); a permutation of the input atoms permutes the forces.  Both
    # hold at any size, in the FP32 path's tolerances.
    from scipy.spatial.transform import Rotation
    s, spec = _work(name)
    model = get_model(spec)
    n = s.n_atoms
    E, F, W = model.evaluate(s.pos, s.cell, s.species, "fp32")
    R = Rotation.random(random_state=17).as_matrix()
    Er, Fr, Wr = model.evaluate(s.pos @ R.T, s.cell @ R.T, s.species, "fp32")
    assert abs(Er - E) / n <= 1e-6
    assert np.linalg.norm(Fr - F @ R.T) / np.linalg.norm(F) <= 1e-5
    assert np.linalg.norm(Wr - R @ W @ R.T) / np.linalg.norm(W) <= 1e-5
    p = np.random.default_rng(18).permutation(n)
    Ep, Fp, Wp = model.evaluate(s.pos[p], s.cell, np.asarray(s.species)[p], "fp32")
    assert abs(Ep - E) / n <= 1e-6
    assert np.linalg.norm(Fp - F[p]) / np.linalg.norm(F) <= 1e-5
    assert np.linalg.norm(Wp - W) / np.linalg.norm(W) <= 1e-5

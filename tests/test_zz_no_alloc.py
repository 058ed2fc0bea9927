"""sevennet_conv_forward_noalloc: the convolution forward for callers that may
not allocate device memory during the call.  Its scratch is a static device
array of the library, so this checks, through the C ABI, that two calls in a
row give the same messages as sevennet_conv_forward_dev (the allocating entry
point) within the FP32 tolerance used by the other convolution tests, and that
sizes beyond its fixed scratch are refused."""

import ctypes

import numpy as np
import pytest
import torch

import oracle
from oracle.model import layer_specs
from synth import MODEL_SEVENNET0, random_structure
from gpu_common import get_model

pytestmark = pytest.mark.gpu


def _inputs(spec, layer, seed):
    s = random_structure({"Si": 30, "O": 50}, 2.2, 1.6, seed=seed)
    dst, src, sh = oracle.neighbor_list(s.pos, s.cell, spec.r_cut)
    n = s.n_atoms
    d = s.pos[src] - s.pos[dst] + sh @ s.cell
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, dst + 1, 1)
    rp = np.cumsum(rp)
    L = layer_specs(spec)[layer]
    xdim = sum((2 * l + 1) * mu for l, mu in L.in_muls.items())
    x = np.random.default_rng(seed).normal(size=(n, xdim))
    dev = "cuda"
    return (n, len(src), torch.tensor(rp, dtype=torch.int32, device=dev),
            torch.tensor(src, dtype=torch.int32, device=dev),
            torch.tensor(d, dtype=torch.float32, device=dev),
            torch.tensor(x, dtype=torch.float32, device=dev))


def _call(lib, fn, model, layer, n, E, rp, src, d, x, mdim):
    m = torch.full((n, mdim), float("nan"), dtype=torch.float32, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = getattr(lib, fn)(model.handle, layer, n, E, ctypes.c_void_p(rp.data_ptr()),
                          ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                          ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(m.data_ptr()), 0, st)
    return rc, m


def test_noalloc_forward_matches_allocating_entry_point_twice():
    from paper_2402_03789_gb300 import _lib
    lib = _lib.load()
    spec = MODEL_SEVENNET0
    model = get_model(spec)
    for layer, seed in [(2, 61), (0, 62)]:          # two calls in a row
        n, E, rp, src, d, x = _inputs(spec, layer, seed)
        mdim = model.conv_dims(layer)[1]
        rc, m_ref = _call(lib, "sevennet_conv_forward_dev", model, layer, n, E, rp, src, d, x, mdim)
        assert rc == 0
        rc, m_new = _call(lib, "sevennet_conv_forward_noalloc", model, layer, n, E, rp, src, d, x, mdim)
        assert rc == 0
        torch.cuda.synchronize()
        a, b = m_new.cpu().numpy(), m_ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) / np.linalg.norm(b) <= 1e-5


def test_noalloc_refuses_sizes_beyond_its_scratch():
    from paper_2402_03789_gb300 import _lib
    lib = _lib.load()
    model = get_model(MODEL_SEVENNET0)
    n, E = 4, (1 << 18) + 1
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    rc = lib.sevennet_conv_forward_noalloc(model.handle, 0, n, E, ctypes.c_void_p(dummy.data_ptr()),
                                           ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()),
                                           ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()),
                                           0, None)
    assert rc == _lib.EINVAL
    assert b"exceed" in lib.sevennet_last_error()

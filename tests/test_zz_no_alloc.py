"""sevennet_conv_forward_noalloc: the convolution forward for callers that may
not allocate device memory during the call.  Its scratch is a static device
array of the library, so this checks, through the C ABI, that two calls in a
row give the same messages as sevennet_conv_forward_dev (the allocating entry
point; both run the same kernel, so bit for bit) in both precisions, that the
calls take nothing from the device's stream-ordered memory pool (which the
allocating entry point does use), and that sizes beyond its fixed scratch are
refused."""

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


def _call(lib, fn, model, layer, n, E, rp, src, d, x, mdim, prec):
    m = torch.full((n, mdim), float("nan"), dtype=torch.float32, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = getattr(lib, fn)(model.handle, layer, n, E, ctypes.c_void_p(rp.data_ptr()),
                          ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                          ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(m.data_ptr()), prec, st)
    return rc, m


class _Pool:
    """The device's default stream-ordered memory pool (driver API), whose
    used-memory high-water mark shows whether a call allocated from it."""
    USED_MEM_CURRENT, USED_MEM_HIGH = 7, 8      # CUmemPool_attribute

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        torch.cuda.synchronize()
        z = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH, ctypes.byref(z)) == 0
        return self.get(self.USED_MEM_CURRENT)

    def grew(self, base):
        torch.cuda.synchronize()
        return self.get(self.USED_MEM_HIGH) > base


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_forward_matches_allocating_entry_point_twice(prec):
    from paper_2402_03789_gb300 import _lib
    lib = _lib.load()
    spec = MODEL_SEVENNET0
    model = get_model(spec)
    pool = _Pool()
    for layer, seed in [(2, 61), (0, 62)]:          # two calls in a row
        n, E, rp, src, d, x = _inputs(spec, layer, seed)
        mdim = model.conv_dims(layer)[1]
        base = pool.reset_high()
        rc, m_ref = _call(lib, "sevennet_conv_forward_dev", model, layer, n, E, rp, src, d, x, mdim, prec)
        assert rc == 0
        assert pool.grew(base)                       # the allocating entry point takes pool memory
        base = pool.reset_high()
        rc, m_new = _call(lib, "sevennet_conv_forward_noalloc", model, layer, n, E, rp, src, d, x, mdim, prec)
        assert rc == 0
        assert not pool.grew(base)                   # this one does not
        a, b = m_new.cpu().numpy(), m_ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.array_equal(a, b)


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

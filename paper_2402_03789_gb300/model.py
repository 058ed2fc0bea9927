"""Python front end of the SevenNet GB300 library: models, MD, serving.

Thin wrappers over the C ABI in include/sevennet.h.  Host-buffer calls take
numpy arrays; device calls take CUDA torch tensors (PyTorch is used only for
device memory and streams).
"""

import ctypes

import numpy as np

from . import _lib as L


def make_config(spec, shift=None):
    """ModelConfig from any object with the hyper-parameter attributes
    (n_species, n_layers, mul, r_cut, n_basis, poly_p, mlp_hidden,
    avg_num_neigh, readout_hidden, scale, shift)."""
    g = (lambda k, d=None: spec.get(k, d)) if isinstance(spec, dict) else (lambda k, d=None: getattr(spec, k, d))
    mul = list(g("mul"))
    c = L.ModelConfig()
    c.n_species = int(g("n_species"))
    c.n_layers = int(g("n_layers"))
    c.lmax = len(mul) - 1
    for i in range(4):
        c.mul[i] = int(mul[i]) if i < len(mul) else 0
    c.r_cut = float(g("r_cut", 5.0))
    c.n_basis = int(g("n_basis", 8))
    c.poly_p = int(g("poly_p", 6))
    c.mlp_hidden = int(g("mlp_hidden", 64))
    c.avg_num_neigh = float(g("avg_num_neigh", 34.0))
    c.readout_hidden = int(g("readout_hidden", 64))
    c.scale = float(g("scale", 1.0))
    sh = shift if shift is not None else g("shift", None)
    keep = None
    if sh:
        keep = L.as_f64(sh)
        c.shift = L.dptr(keep)
    else:
        c.shift = None
    return c, keep


def n_params(spec) -> int:
    c, _keep = make_config(spec)
    n = L.load().sevennet_n_params(ctypes.byref(c))
    if n < 0:
        L.check(L.EINVAL)
    return int(n)


def padded_model(spec, weights):
    """(padded multiplicities, padded canonical weights) of the exact
    zero-padded model the library runs (sevennet_padded_weights; host only)."""
    lib = L.load()
    c, _keep = make_config(spec)
    w = L.as_f64(weights).reshape(-1)
    mul = (ctypes.c_int32 * 4)()
    L.check(lib.sevennet_padded_weights(ctypes.byref(c), L.dptr(w), w.size, mul, None, 0))
    cp, _kp = make_config(spec)
    for l in range(4):
        cp.mul[l] = mul[l]
    n = lib.sevennet_n_params(ctypes.byref(cp))
    if n < 0:
        L.check(L.EINVAL)
    out = np.zeros(int(n))
    L.check(lib.sevennet_padded_weights(ctypes.byref(c), L.dptr(w), w.size, mul, L.dptr(out), out.size))
    return tuple(int(mul[l]) for l in range(4) if mul[l]), out


def _prec(p):
    if isinstance(p, int):
        return p
    return L.PRECISION[p]


def _stream_ptr(stream, device=None):
    """cudaStream_t of `stream`; None means torch's current stream on `device`,
    so that kernels are ordered with the torch work that made and reads the
    tensors."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream(device)
    return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))


class SevenNet:
    """A model resident on one GPU."""

    def __init__(self, spec, weights, device: int = 0):
        self.lib = L.load()
        cfg, keep = make_config(spec)
        self._cfg = cfg
        self._keep = keep
        w = L.as_f64(weights).reshape(-1)
        h = ctypes.c_void_p()
        L.check(self.lib.sevennet_create_model(ctypes.byref(cfg), L.dptr(w), w.size, device, ctypes.byref(h)))
        self.handle = h
        self.device = device
        self.n_layers = cfg.n_layers

    def close(self):
        if getattr(self, "handle", None):
            self.lib.sevennet_destroy_model(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- host API
    def evaluate(self, pos, cell, species, precision="fp32", pbc=(1, 1, 1)):
        """(E, F [N,3], W [3,3]) of one periodic cell, host in / host out."""
        pos = L.as_f64(pos, (-1, 3))
        n = pos.shape[0]
        sp = L.as_i32(species)
        cell = L.as_f64(cell, (3, 3))
        pb = L.as_i32(pbc)
        e = np.zeros(1)
        f = np.zeros((n, 3))
        w = np.zeros((3, 3))
        L.check(self.lib.sevennet_eval_energy_forces_virial(
            self.handle, n, L.iptr(sp), L.dptr(pos), L.dptr(cell), L.iptr(pb), _prec(precision),
            L.dptr(e), L.dptr(f), L.dptr(w)))
        return float(e[0]), f, w

    def evaluate_decomposed(self, pos, cell, species, n_domains, precision="fp32"):
        """(E, F, W) through the single-process emulation of the spatial
        decomposition (n_domains slabs, ghost exchange per block)."""
        pos = L.as_f64(pos, (-1, 3))
        n = pos.shape[0]
        sp = L.as_i32(species)
        cell = L.as_f64(cell, (3, 3))
        e = np.zeros(1)
        f = np.zeros((n, 3))
        w = np.zeros((3, 3))
        L.check(self.lib.sevennet_eval_decomposed(self.handle, n, L.iptr(sp), L.dptr(pos), L.dptr(cell),
                                                  int(n_domains), _prec(precision), L.dptr(e), L.dptr(f),
                                                  L.dptr(w)))
        return float(e[0]), f, w

    def neighbors(self, pos, cell, pbc=(1, 1, 1)):
        """Edges (dst, src, shift) with input atom indices, library order."""
        pos = L.as_f64(pos, (-1, 3))
        cell = L.as_f64(cell, (3, 3))
        pb = L.as_i32(pbc)
        h = ctypes.c_void_p()
        ne = ctypes.c_int64()
        L.check(self.lib.sevennet_build_neighbors(self.handle, pos.shape[0], L.dptr(pos), L.dptr(cell),
                                                  L.iptr(pb), ctypes.byref(h), ctypes.byref(ne)))
        try:
            E = ne.value
            dst = np.zeros(E, np.int32)
            src = np.zeros(E, np.int32)
            sh = np.zeros((E, 3), np.int32)
            L.check(self.lib.sevennet_nlist_export(h, L.iptr(dst), L.iptr(src), L.iptr(sh)))
        finally:
            self.lib.sevennet_nlist_destroy(h)
        return dst, src, sh

    # -------------------------------------------------------------- diagnostics
    def profile(self, enable=True):
        L.check(self.lib.sevennet_profile(self.handle, 1 if enable else 0))

    def profile_read(self):
        """{family: (total_ms, launches)} since profile(True)."""
        n = 8
        names = ctypes.create_string_buffer(32 * n)
        ms = np.zeros(n)
        cnt = np.zeros(n, np.int64)
        nout = ctypes.c_int32()
        L.check(self.lib.sevennet_profile_read(self.handle, n, names, L.dptr(ms),
                                               cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                               ctypes.byref(nout)))
        out = {}
        for i in range(nout.value):
            nm = names.raw[32 * i:32 * (i + 1)].split(b"\0", 1)[0].decode()
            out[nm] = (float(ms[i]), int(cnt[i]))
        return out

    @staticmethod
    def launch_count():
        return int(L.load().sevennet_launch_count())

    @staticmethod
    def fp32_peak(device=0, packed=False, iters=20000):
        """Measured FP32 FMA throughput of the device: (TFLOP/s, flop, ms)."""
        flop, ms = ctypes.c_double(), ctypes.c_double()
        L.check(L.load().sevennet_fp32_peak(int(device), int(bool(packed)), int(iters),
                                            ctypes.byref(flop), ctypes.byref(ms)))
        return flop.value / (ms.value * 1e-3) / 1e12, flop.value, ms.value

    # -------------------------------------------------------------- device API
    def evaluate_batch_dev(self, atom_offsets, cells, species, pos, precision="fp32", pbc=None,
                           stream=None, out=None):
        """Batched evaluation; species/pos are CUDA tensors (int32, float64).

        Returns (energy [S], forces [N,3], virial [S,3,3]) as CUDA float64 tensors.
        """
        import torch
        off = np.ascontiguousarray(np.asarray(atom_offsets, dtype=np.int64))
        S = off.size - 1
        cells = L.as_f64(cells, (S, 3, 3))
        pb = None if pbc is None else L.as_i32(pbc).reshape(S, 3)
        assert species.is_cuda and species.dtype == torch.int32 and species.is_contiguous()
        assert pos.is_cuda and pos.dtype == torch.float64 and pos.is_contiguous()
        N = int(off[-1])
        if out is None:
            e = torch.empty(S, dtype=torch.float64, device=pos.device)
            f = torch.empty((N, 3), dtype=torch.float64, device=pos.device)
            w = torch.empty((S, 3, 3), dtype=torch.float64, device=pos.device)
        else:
            e, f, w = out
        L.check(self.lib.sevennet_eval_batch_dev(
            self.handle, S, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), L.dptr(cells),
            L.iptr(pb) if pb is not None else None, ctypes.c_void_p(species.data_ptr()),
            ctypes.c_void_p(pos.data_ptr()), _prec(precision), ctypes.c_void_p(e.data_ptr()),
            ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(w.data_ptr()), _stream_ptr(stream, pos.device)))
        return e, f, w

    def conv_dims(self, layer):
        xd = ctypes.c_int32()
        md = ctypes.c_int32()
        L.check(self.lib.sevennet_conv_dims(self.handle, layer, ctypes.byref(xd), ctypes.byref(md)))
        return xd.value, md.value

    def _check_conv_args(self, layer, row_ptr, src, d, x, g_m=None):
        import torch
        xdim, mdim = self.conv_dims(layer)
        dev = torch.device("cuda", self.device)
        for name, t, dt in (("row_ptr", row_ptr, torch.int32), ("src", src, torch.int32),
                            ("d", d, torch.float32), ("x", x, torch.float32), ("g_m", g_m, torch.float32)):
            if t is None:
                continue
            if t.dtype != dt or t.device != dev or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous {dt} tensor on {dev} "
                                 f"(got {t.dtype} on {t.device}, contiguous={t.is_contiguous()})")
        n = row_ptr.numel() - 1
        if d.shape != (src.numel(), 3) or x.shape != (n, xdim) or (g_m is not None and g_m.shape != (n, mdim)):
            raise ValueError("shapes: d [E, 3], x [n_atoms, x_dim] and g_m [n_atoms, m_dim] expected")
        return n, src.numel(), mdim

    def conv_forward(self, layer, row_ptr, src, d, x, precision="fp32", stream=None):
        import torch
        n, E, mdim = self._check_conv_args(layer, row_ptr, src, d, x)
        m = torch.empty((n, mdim), dtype=torch.float32, device=x.device)
        L.check(self.lib.sevennet_conv_forward_dev(
            self.handle, layer, n, E, ctypes.c_void_p(row_ptr.data_ptr()), ctypes.c_void_p(src.data_ptr()),
            ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(m.data_ptr()),
            _prec(precision), _stream_ptr(stream, x.device)))
        return m

    def conv_backward(self, layer, row_ptr, src, d, x, g_m, precision="fp32", stream=None):
        import torch
        n, E, _ = self._check_conv_args(layer, row_ptr, src, d, x, g_m)
        g_x = torch.empty_like(x)
        g_d = torch.zeros((E, 3), dtype=torch.float32, device=x.device)
        L.check(self.lib.sevennet_conv_backward_dev(
            self.handle, layer, n, E, ctypes.c_void_p(row_ptr.data_ptr()), ctypes.c_void_p(src.data_ptr()),
            ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(g_m.data_ptr()),
            ctypes.c_void_p(g_x.data_ptr()), ctypes.c_void_p(g_d.data_ptr()), _prec(precision),
            _stream_ptr(stream, x.device)))
        return g_x, g_d


class MD:
    """Velocity-Verlet MD on the device (NVE, or Nose-Hoover NVT), optional Verlet skin."""

    def __init__(self, model: SevenNet, pos, vel, species, masses, cell, precision="fp32"):
        self.model = model
        self.lib = model.lib
        pos = L.as_f64(pos, (-1, 3))
        self.n = pos.shape[0]
        vel = L.as_f64(vel, (-1, 3))
        sp = L.as_i32(species)
        ms = L.as_f64(masses)
        cell = L.as_f64(cell, (3, 3))
        h = ctypes.c_void_p()
        L.check(self.lib.sevennet_md_create(model.handle, self.n, L.iptr(sp), L.dptr(pos), L.dptr(vel),
                                            L.dptr(ms), L.dptr(cell), _prec(precision), ctypes.byref(h)))
        self.handle = h

    def step(self, n_steps, dt_fs=1.0):
        ep = np.zeros(n_steps)
        ek = np.zeros(n_steps)
        L.check(self.lib.sevennet_md_step(self.handle, n_steps, dt_fs, L.dptr(ep), L.dptr(ek)))
        return ep, ek

    def set_skin(self, skin_A: float):
        """Reuse a Verlet list of cutoff r_c + skin (0: rebuild every step)."""
        L.check(self.lib.sevennet_md_set_skin(self.handle, float(skin_A)))

    def set_nose_hoover(self, temperature_K: float, tau_fs: float):
        """Nose-Hoover NVT at temperature_K with time constant tau_fs (tau <= 0: NVE)."""
        L.check(self.lib.sevennet_md_set_nose_hoover(self.handle, float(temperature_K), float(tau_fs)))

    def set_nose_hoover_ramp(self, t_start_K: float, t_end_K: float, n_steps: int, tau_fs: float):
        """Nose-Hoover NVT whose target ramps linearly from t_start_K to t_end_K
        over the next n_steps steps (then stays at t_end_K)."""
        L.check(self.lib.sevennet_md_set_nose_hoover_ramp(self.handle, float(t_start_K), float(t_end_K),
                                                          int(n_steps), float(tau_fs)))

    def run_schedule(self, segments, dt_fs=1.0, tau_fs=100.0):
        """Run a temperature schedule under Nose-Hoover NVT, e.g. the melt-quench
        protocol of Sec. 5.2 (hold at 5000 K, hold at 3000 K, quench at -33 K/ps).

        segments: ("hold", T_K, n_steps) or ("ramp", T_start_K, T_end_K, n_steps).
        Returns the (E_pot, E_kin) logs of all steps."""
        eps, eks = [], []
        for seg in segments:
            if seg[0] == "hold":
                _, t, n = seg
                self.set_nose_hoover(t, tau_fs)
            elif seg[0] == "ramp":
                _, t0, t1, n = seg
                self.set_nose_hoover_ramp(t0, t1, n, tau_fs)
            else:
                raise ValueError(f"unknown schedule segment {seg[0]!r}")
            if n > 0:
                ep, ek = self.step(int(n), dt_fs)
                eps.append(ep)
                eks.append(ek)
        if not eps:
            return np.zeros(0), np.zeros(0)
        return np.concatenate(eps), np.concatenate(eks)

    def nose_hoover(self):
        """(xi, eta) of the thermostat."""
        xi = ctypes.c_double()
        eta = ctypes.c_double()
        L.check(self.lib.sevennet_md_get_nose_hoover(self.handle, ctypes.byref(xi), ctypes.byref(eta)))
        return xi.value, eta.value

    def stats(self):
        """(neighbour-list builds so far, edges of the last refreshed Verlet list)."""
        nb = ctypes.c_int64()
        ne = ctypes.c_int64()
        L.check(self.lib.sevennet_md_get_stats(self.handle, ctypes.byref(nb), ctypes.byref(ne)))
        return nb.value, ne.value

    def state(self):
        p = np.zeros((self.n, 3))
        v = np.zeros((self.n, 3))
        f = np.zeros((self.n, 3))
        L.check(self.lib.sevennet_md_get_state(self.handle, L.dptr(p), L.dptr(v), L.dptr(f)))
        return p, v, f

    def close(self):
        if getattr(self, "handle", None):
            self.lib.sevennet_md_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching evaluation server."""

    def __init__(self, model: SevenNet, hbm_budget_bytes: int, n_streams: int = 4,
                 max_batch_structs: int = 64, precision="fp32"):
        self.model = model
        self.lib = model.lib
        h = ctypes.c_void_p()
        L.check(self.lib.sevennet_server_create(model.handle, int(hbm_budget_bytes), n_streams,
                                                max_batch_structs, _prec(precision), ctypes.byref(h)))
        self.handle = h
        self._n = {}

    def submit(self, pos, cell, species):
        pos = L.as_f64(pos, (-1, 3))
        sp = L.as_i32(species)
        cell = L.as_f64(cell, (3, 3))
        req = L.Request(pos.shape[0], L.iptr(sp), L.dptr(pos), L.dptr(cell))
        t = ctypes.c_uint64()
        L.check(self.lib.sevennet_server_submit(self.handle, ctypes.byref(req), ctypes.byref(t)))
        self._n[t.value] = pos.shape[0]
        return t.value

    def poll(self, ticket):
        """None while running, else dict(energy, forces, virial, submit_s, done_s, batch_id, batch_structs)."""
        n = self._n[ticket]
        f = np.zeros((n, 3))
        res = L.Result()
        res.forces = L.dptr(f)
        done = ctypes.c_int()
        L.check(self.lib.sevennet_server_poll(self.handle, ticket, ctypes.byref(res), ctypes.byref(done)))
        if not done.value:
            return None
        del self._n[ticket]
        return dict(energy=res.energy, forces=f, virial=np.array(res.virial[:]).reshape(3, 3),
                    submit_s=res.submit_s, start_s=res.start_s, done_s=res.done_s, batch_id=res.batch_id,
                    batch_structs=res.batch_structs)

    def now(self):
        return self.lib.sevennet_server_now(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            self.lib.sevennet_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

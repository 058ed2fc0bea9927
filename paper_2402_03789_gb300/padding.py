"""Models with fewer than 32 channels of an irrep (the paper's 4-16 channel
benchmark models, Sec. 4) run as the same model with every multiplicity
rounded up to a multiple of 32 and the extra channels' weights set to zero.

The GPU kernels give a warp 32 channels of an irrep.  A zero channel stays zero
through every operation of the model: its linear rows and columns and its
radial-MLP output columns are zero, so its features, messages, gates (SiLU(0) =
0) and readout contributions vanish.  The energy, forces and virial of the
padded model therefore equal those of the original.  The library scales each
linear by 1 / sqrt(fan_in) of its own (padded) configuration, so the copied
weights are multiplied by sqrt(padded fan_in / true fan_in).

The canonical weight layout walked here is the library's (include/sevennet.h:
embedding; per block: self-connection and linear_1 per irrep, the radial MLP,
linear_2 per irrep; readout), with the block irreps of a NequIP interaction
block: the first block takes scalars only, the last keeps l3 = 0 paths only.
"""

from dataclasses import replace
from typing import List, Tuple

import numpy as np


def padded_mul(m: int) -> int:
    return 32 * ((int(m) + 31) // 32)


def needs_padding(spec) -> bool:
    return any(int(m) % 32 for m in spec.mul)


def _block(mul, lmax, t, n_layers):
    """(in_mul, paths [(l1, l2, l3)], y segments per l, msg segments per l, last)."""
    last = t == n_layers - 1
    in_mul = {0: mul[0]} if t == 0 else {l: mul[l] for l in range(lmax + 1)}
    paths = []
    for l1 in sorted(in_mul):
        for l2 in range(lmax + 1):
            for l3 in range(abs(l1 - l2), min(l1 + l2, lmax) + 1):
                if last and l3 != 0:
                    continue
                paths.append((l1, l2, l3))
    if last:
        y_seg = {0: [mul[0]]}
    else:
        y_seg = {0: [mul[l] for l in range(lmax + 1)]}           # scalars, then the gates of l >= 1
        y_seg.update({l: [mul[l]] for l in range(1, lmax + 1)})
    msg_seg = {}
    for (l1, _, l3) in paths:
        msg_seg.setdefault(l3, []).append(in_mul[l1])
    return in_mul, paths, y_seg, msg_seg, last


def _entries(spec) -> List[Tuple[str, List[int], List[int], str]]:
    """Canonical weight matrices: (name, row segments, col segments, fan_in kind)."""
    mul, lmax, T = list(spec.mul), len(spec.mul) - 1, spec.n_layers
    H, NB, RH = spec.mlp_hidden, spec.n_basis, spec.readout_hidden
    out = [("embed", [spec.n_species], [mul[0]], "none")]
    for t in range(T):
        in_mul, paths, y_seg, msg_seg, _ = _block(mul, lmax, t, T)
        for l in range(lmax + 1):
            if l in y_seg and l in in_mul:
                out.append((f"L{t}.sc.{l}", [in_mul[l]], y_seg[l], "rows"))
        for l in range(lmax + 1):
            if l in in_mul:
                out.append((f"L{t}.lin1.{l}", [in_mul[l]], [in_mul[l]], "rows"))
        out.append((f"L{t}.mlp0", [NB], [H], "none"))
        out.append((f"L{t}.mlp1", [H], [H], "none"))
        out.append((f"L{t}.mlp2", [H], [in_mul[l1] for (l1, _, _) in paths], "none"))
        for l in range(lmax + 1):
            if l in y_seg and l in msg_seg:
                out.append((f"L{t}.lin2.{l}", msg_seg[l], y_seg[l], "rows"))
    out.append(("readout0", [mul[0]], [RH], "rows"))
    out.append(("readout1", [RH], [1], "none"))
    return out


def n_params(spec) -> int:
    return sum(sum(r) * sum(c) for _, r, c, _ in _entries(spec))


def _index_map(segs: List[int]) -> np.ndarray:
    """Position of every true index in the padded concatenation of segments."""
    idx, base = [], 0
    for s in segs:
        idx.extend(range(base, base + s))
        base += padded_mul(s) if s else 0
    return np.asarray(idx, dtype=np.int64)


def pad_model(spec, weights):
    """(padded spec, padded canonical weight vector) of an exact equivalent model."""
    spec_p = replace(spec, mul=tuple(padded_mul(m) for m in spec.mul))
    w = np.asarray(weights, dtype=np.float64).reshape(-1)
    ents_t, ents_p = _entries(spec), _entries(spec_p)
    assert [e[0] for e in ents_t] == [e[0] for e in ents_p]
    out, o_t = [], 0
    pads_rows = {"embed", "readout1"} | {n for n, *_ in ents_t if n.endswith((".mlp0", ".mlp1"))}
    for (name, rt, ct, kind), (_, rp, cp, _) in zip(ents_t, ents_p):
        R, C = sum(rt), sum(ct)
        M = w[o_t:o_t + R * C].reshape(R, C)
        o_t += R * C
        rmap = np.arange(R) if name in pads_rows or name.endswith(".mlp2") else _index_map(rt)
        cmap = _index_map(ct) if not (name.endswith((".mlp0", ".mlp1")) or name == "readout1") else np.arange(C)
        P = np.zeros((sum(rp), sum(cp)))
        P[np.ix_(rmap, cmap)] = M
        if kind == "rows":
            P *= np.sqrt(sum(rp) / R)
        out.append(P.reshape(-1))
    assert o_t == w.size, "weight vector length does not match the model"
    return spec_p, np.concatenate(out)

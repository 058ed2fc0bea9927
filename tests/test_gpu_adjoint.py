"""The hand-written convolution adjoint behind torch.autograd.Function:
forward messages and gradients (dL/dx, dL/dd) against the FP64 oracle's
convolution and its autograd gradient, and against central finite differences
of the GPU function itself."""

import numpy as np
import pytest
import torch

import oracle
from oracle.model import ModelLayout, layer_specs, conv_layer, edge_features, radial_mlp
from synth import MODEL_SEVENNET0, MODEL_TINY, normal_weights, random_structure
from gpu_common import get_model

pytestmark = pytest.mark.gpu


def _setup(spec, layer, seed=41):
    s = random_structure({"Si": 30, "O": 50}, 2.2, 1.6, seed=seed)
    dst, src, sh = oracle.neighbor_list(s.pos, s.cell, spec.r_cut)
    n = s.n_atoms
    d = s.pos[src] - s.pos[dst] + sh @ s.cell
    row_ptr = np.zeros(n + 1, np.int64)
    np.add.at(row_ptr, dst + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    L = layer_specs(spec)[layer]
    rng = np.random.default_rng(seed)
    x = {l: rng.normal(size=(n, 2 * l + 1, mu)) for l, mu in L.in_muls.items()}
    return s, dst, src, d, row_ptr, L, x


def _pack(xd, n):
    return np.concatenate([xd[l].reshape(n, -1) for l in sorted(xd)], axis=1)


@pytest.mark.parametrize("spec,layer", [(MODEL_SEVENNET0, 0), (MODEL_SEVENNET0, 2), (MODEL_SEVENNET0, 4),
                                        (MODEL_TINY, 1)])
def test_conv_forward_and_adjoint_match_oracle(spec, layer):
    from paper_2402_03789_gb300.autograd import conv
    model = get_model(spec)
    s, dst, src, d, row_ptr, L, x = _setup(spec, layer)
    n = s.n_atoms
    Wd = ModelLayout(spec).unpack(normal_weights(oracle.n_params(spec)))
    xt = {l: torch.tensor(v, requires_grad=True) for l, v in x.items()}
    dt = torch.tensor(d, requires_grad=True)
    Y, B = edge_features(spec, dt)
    w = radial_mlp(spec, Wd, layer, B)
    m = conv_layer(spec, L, xt, Y, w, torch.as_tensor(dst), torch.as_tensor(src), n)
    mo = torch.cat([m[l].reshape(n, -1) for l in sorted(m)], dim=1)
    gm = np.random.default_rng(7).normal(size=tuple(mo.shape))
    loss = (mo * torch.as_tensor(gm)).sum()
    grads = torch.autograd.grad(loss, [xt[l] for l in sorted(xt)] + [dt])
    gxo = np.concatenate([g.detach().numpy().reshape(n, -1) for g in grads[:-1]], axis=1)
    gdo = grads[-1].detach().numpy()

    dev = "cuda"
    xg = torch.tensor(_pack(x, n), dtype=torch.float32, device=dev, requires_grad=True)
    dg = torch.tensor(d, dtype=torch.float32, device=dev, requires_grad=True)
    rp = torch.tensor(row_ptr, dtype=torch.int32, device=dev)
    sg = torch.tensor(src, dtype=torch.int32, device=dev)
    mg = conv(model, layer, xg, dg, rp, sg)
    rel = np.linalg.norm(mg.detach().cpu().numpy() - mo.detach().numpy()) / np.linalg.norm(mo.detach().numpy())
    assert rel <= 1e-5, rel
    (mg * torch.tensor(gm, dtype=torch.float32, device=dev)).sum().backward()
    rx = np.linalg.norm(xg.grad.cpu().numpy() - gxo) / np.linalg.norm(gxo)
    rd = np.linalg.norm(dg.grad.cpu().numpy() - gdo) / np.linalg.norm(gdo)
    print(f"layer {layer}: m {rel:.2e} dx {rx:.2e} dd {rd:.2e}")
    assert rx <= 1e-5 and rd <= 1e-5


def test_conv_adjoint_matches_finite_differences():
    from paper_2402_03789_gb300.autograd import conv
    spec, layer = MODEL_SEVENNET0, 1
    model = get_model(spec)
    s, dst, src, d, row_ptr, L, x = _setup(spec, layer, seed=43)
    n = s.n_atoms
    dev = "cuda"
    rp = torch.tensor(row_ptr, dtype=torch.int32, device=dev)
    sg = torch.tensor(src, dtype=torch.int32, device=dev)
    xg = torch.tensor(_pack(x, n), dtype=torch.float32, device=dev, requires_grad=True)
    gm = torch.tensor(np.random.default_rng(9).normal(size=(n, model.conv_dims(layer)[1])),
                      dtype=torch.float32, device=dev)
    d0 = torch.tensor(d, dtype=torch.float32, device=dev, requires_grad=True)
    (conv(model, layer, xg, d0, rp, sg) * gm).sum().backward()
    gd = d0.grad.cpu().numpy()
    gx = xg.grad.cpu().numpy()

    def loss(dd, xx):
        with torch.no_grad():
            return float((conv(model, layer, xx, dd, rp, sg) * gm).double().sum())

    h = 1e-2                      # displacement step (A); L is smooth on the scale of 1 A
    scale_d = np.abs(gd).max()
    for e, a in [(0, 0), (17, 1), (len(d) // 2, 2), (len(d) - 1, 0)]:
        dp = d0.detach().clone(); dp[e, a] += h
        dm = d0.detach().clone(); dm[e, a] -= h
        fd = (loss(dp, xg.detach()) - loss(dm, xg.detach())) / (2 * h)
        assert abs(fd - gd[e, a]) <= 2e-3 * scale_d, (e, a, fd, gd[e, a])
    scale_x = np.abs(gx).max()
    h = 0.1                       # L is linear in x
    for v, j in [(0, 0), (5, 100), (40, 300), (n - 1, 479)]:
        xp = xg.detach().clone(); xp[v, j] += h
        xm = xg.detach().clone(); xm[v, j] -= h
        fd = (loss(d0.detach(), xp) - loss(d0.detach(), xm)) / (2 * h)
        assert abs(fd - gx[v, j]) <= 2e-3 * scale_x, (v, j, fd, gx[v, j])


@pytest.mark.parametrize("spec,layer", [(MODEL_SEVENNET0, 0), (MODEL_SEVENNET0, 2), (MODEL_SEVENNET0, 4),
                                        (MODEL_TINY, 1)])
def test_bf16_conv_forward_matches_oracle(spec, layer):
    # BF16 path: w, x and the G matrices enter the tensor cores as BF16 with FP32
    # accumulation; the messages stay within a few BF16 roundings of the FP64 oracle
    model = get_model(spec)
    s, dst, src, d, row_ptr, L, x = _setup(spec, layer, seed=43)
    n = s.n_atoms
    Wd = ModelLayout(spec).unpack(normal_weights(oracle.n_params(spec)))
    dt = torch.tensor(d)
    Y, B = edge_features(spec, dt)
    w = radial_mlp(spec, Wd, layer, B)
    m = conv_layer(spec, L, {l: torch.tensor(v) for l, v in x.items()}, Y, w,
                   torch.as_tensor(dst), torch.as_tensor(src), n)
    mo = torch.cat([m[l].reshape(n, -1) for l in sorted(m)], dim=1).numpy()
    dev = "cuda"
    mg = model.conv_forward(layer, torch.tensor(row_ptr, dtype=torch.int32, device=dev),
                            torch.tensor(src, dtype=torch.int32, device=dev),
                            torch.tensor(d, dtype=torch.float32, device=dev),
                            torch.tensor(_pack(x, n), dtype=torch.float32, device=dev), "bf16")
    mg = mg.cpu().numpy()
    rel = np.linalg.norm(mg - mo) / np.linalg.norm(mo)
    worst = np.abs(mg - mo).max() / np.abs(mo).max()
    print(f"bf16 layer {layer}: messages rel {rel:.2e}, max {worst:.2e}")
    assert rel <= 1e-2 and worst <= 3e-2

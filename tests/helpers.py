"""Shared test helpers: one layer spec builds both the CUDA map and the oracle map, the
oracle's state can be uploaded into the CUDA map (so both start a step from identical
inputs), and states are compared element by element with the stated tolerances."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_2309_16818_gb300 import synth

# floating-point tolerance: |gpu - oracle| <= REL * max(|oracle|, scale of the layer)
REL = 1e-5


def specs_to(layers, which):
    """layers: list of dicts(channels, rule, dtype, w, var_meas, alpha0) -> oracle / mem layers."""
    from paper_2309_16818_gb300 import mem as M
    out = []
    for L in layers:
        kw = dict(w=L.get("w", 0.1), var_meas=L.get("var_meas", 1.0), alpha0=L.get("alpha0", 1.0))
        dt = L.get("dtype", O.F32)
        if which == "oracle":
            out.append(O.Layer(L["channels"], L["rule"], store=dt, **kw))
        else:
            out.append(M.Layer(L["channels"], L["rule"], dtype=dt, **kw))
    return out


def make_pair(W, res, layers, **kw):
    from paper_2309_16818_gb300 import mem as M
    g = M.Map(W, res, specs_to(layers, "mem"), **kw)
    kw.pop("max_points", None)
    kw.pop("n_maps", None)
    o = O.OracleMap(O.Params(W=W, res=res, layers=specs_to(layers, "oracle"), **kw))
    return g, o


def torch_dt(code):
    import torch
    return {O.F32: torch.float32, O.BF16: torch.bfloat16, O.F16: torch.float16}[code]


def upload_state(g, o, map_index=0):
    """Write the oracle's (storage-rounded) state into map `map_index` of the CUDA map."""
    import torch
    from paper_2309_16818_gb300 import mem as M
    dev = "cuda"
    g.set_layer(M.LAYER_HEIGHT, torch.tensor(o.h, dtype=torch.float32, device=dev), map_index=map_index)
    g.set_layer(M.LAYER_VARIANCE, torch.tensor(o.var, dtype=torch.float32, device=dev), map_index=map_index)
    g.set_layer(M.LAYER_VALID, torch.tensor(o.valid, device=dev), map_index=map_index)
    g.set_layer(M.LAYER_NACC, torch.tensor(o.n_acc.view(np.int32), device=dev), map_index=map_index)
    g.set_layer(M.LAYER_NREJ, torch.tensor(o.n_rej.view(np.int32), device=dev), map_index=map_index)
    for l, L in enumerate(o.p.layers):
        v = torch.tensor(o.layer_values(l), dtype=torch.float64, device=dev).to(torch_dt(L.store))
        g.set_layer(l, v.contiguous(), map_index=map_index)
        g.set_layer(l, torch.tensor(o.obs[l], device=dev), part=M.PART_OBSERVED, map_index=map_index)
        if L.rule == O.GAUSS:
            gv = o.gauss_var(l)
            assert np.all((gv == gv[:, :1]) | ~np.isfinite(gv)), "per-dimension variances differ"
            vv = np.where(np.isfinite(gv[:, 0]), gv[:, 0], 0.0)
            g.set_layer(l, torch.tensor(vv, dtype=torch.float32, device=dev), part=M.PART_VAR,
                        map_index=map_index)


def gpu_state(g, map_index=0):
    import torch
    from paper_2309_16818_gb300 import mem as M
    out = dict(
        h=g.get_layer(M.LAYER_HEIGHT, map_index=map_index).cpu().numpy().astype(np.float64),
        var=g.get_layer(M.LAYER_VARIANCE, map_index=map_index).cpu().numpy().astype(np.float64),
        valid=g.get_layer(M.LAYER_VALID, map_index=map_index).cpu().numpy(),
        n_acc=g.get_layer(M.LAYER_NACC, map_index=map_index).cpu().numpy().view(np.uint32),
        n_rej=g.get_layer(M.LAYER_NREJ, map_index=map_index).cpu().numpy().view(np.uint32),
        layers=[], obs=[], gvar=[])
    for l, L in enumerate(g.layers):
        out["layers"].append(g.get_layer(l, map_index=map_index).to(torch.float64).cpu().numpy())
        out["obs"].append(g.get_layer(l, part=M.PART_OBSERVED, map_index=map_index).cpu().numpy())
        out["gvar"].append(g.get_layer(l, part=M.PART_VAR, map_index=map_index).cpu().numpy()
                           .astype(np.float64) if L.rule == M.GAUSS else None)
    torch.cuda.synchronize()
    return out


def close(a, b, scale, rel=REL):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    tol = rel * np.maximum(np.abs(b), scale)
    bad = ~(np.abs(a - b) <= tol)
    return bad


def compare_states(gs, o, mask=None, what="", bf16_rel=2.0 ** -7):
    """Element-by-element comparison; `mask` (bool per cell) excludes cells whose
    decisions are not decided by the same inputs on both sides."""
    W2 = o.h.shape[0]
    m = np.ones(W2, bool) if mask is None else mask
    assert np.array_equal(gs["valid"][m], o.valid[m]), f"{what}: valid differs at {np.nonzero((gs['valid'] != o.valid) & m)[0][:10]}"
    assert np.array_equal(gs["n_acc"][m], o.n_acc[m]), f"{what}: n_acc differs at {np.nonzero((gs['n_acc'] != o.n_acc) & m)[0][:10]}"
    assert np.array_equal(gs["n_rej"][m], o.n_rej[m]), f"{what}: n_rej differs"
    v = m & (o.valid == 1)
    bad = close(gs["h"][v], o.h[v], 1.0)
    assert not bad.any(), f"{what}: h differs: gpu {gs['h'][v][bad][:5]} oracle {o.h[v][bad][:5]}"
    bad = close(gs["var"][v], o.var[v], 0.0)
    assert not bad.any(), f"{what}: var differs: gpu {gs['var'][v][bad][:5]} oracle {o.var[v][bad][:5]}"
    for l, L in enumerate(o.p.layers):
        assert np.array_equal(gs["obs"][l][m], o.obs[l][m]), f"{what}: observed flags of layer {l}"
        gv, ov = gs["layers"][l][m], o.layer_values(l)[m]
        if L.rule == O.CLASSMAX:
            assert np.array_equal(gv[:, 0], ov[:, 0]), f"{what}: class-max ids of layer {l}"
            assert np.array_equal(gv[:, 1], ov[:, 1]), f"{what}: class-max confidences of layer {l}"
            continue
        if L.store == O.F32:
            bad = close(gv, ov, 1.0)
        else:
            bad = ~(np.abs(gv - ov) <= bf16_rel * np.maximum(np.abs(ov), 1e-3))
        assert not bad.any(), f"{what}: layer {l} rule {L.rule}: gpu {gv[bad][:5]} oracle {ov[bad][:5]}"
        if L.rule == O.GAUSS:
            ob = m & (o.obs[l] == 1)
            bad = close(gs["gvar"][l][ob], o.gauss_var(l)[ob][:, 0], 0.0)
            assert not bad.any(), f"{what}: Gaussian variance of layer {l}"


def multimodal_layers():
    """The layers of the multi-modal point-cloud workload: colour average, Dirichlet class
    fusion, class max, exponential averaging of the class probabilities."""
    return [dict(channels=3, rule=O.LATEST), dict(channels=20, rule=O.DIRICHLET, alpha0=1.0),
            dict(channels=20, rule=O.CLASSMAX), dict(channels=20, rule=O.EXPAVG, w=0.1)]


def cloud_sources_np(cl):
    return [(cl.rgb, [0]), (cl.probs, [1, 2, 3])]


def cloud_sources_gpu(cl):
    import torch
    return [(torch.from_numpy(cl.rgb).cuda(), [0]), (torch.from_numpy(cl.probs).cuda(), [1, 2, 3])]


def cuda_xyz(cl):
    import torch
    return torch.from_numpy(np.ascontiguousarray(cl.xyz)).cuda()

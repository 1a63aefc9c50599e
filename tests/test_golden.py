"""Stored expected values (tests/golden/fusion_w12.json, written by tests/golden/make_golden.py
from the oracle alone): the oracle must still produce them (CPU), and the library must match
them element by element through the C ABI (GPU) -- point fusion with every rule, a move, a
second cloud with outliers, and a camera image with the visibility walk."""
import json
import os
import sys

import numpy as np
import pytest

import oracle as O

from helpers import compare_states, gpu_state, specs_to

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, GOLDEN)
import cases  # noqa: E402
import make_golden  # noqa: E402


def load():
    with open(os.path.join(GOLDEN, "fusion_w12.json")) as f:
        return json.load(f)


def _same(a, b, what):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    assert a.shape == b.shape, what
    fin = np.isfinite(a) & np.isfinite(b)
    af, bf = np.where(fin, a, 0.0), np.where(fin, b, 0.0)
    ok = (a == b) | (fin & (np.abs(af - bf) <= 1e-12 * np.maximum(np.abs(bf), 1.0)))
    assert ok.all(), f"{what}: {a[~ok][:5]} vs stored {b[~ok][:5]}"


def test_oracle_reproduces_stored_values():
    stored, now = load(), make_golden.run_oracle()
    assert stored["cite"] == now["cite"] and stored["layers"] == now["layers"]
    assert len(stored["steps"]) == len(now["steps"])
    for k, (s, n) in enumerate(zip(stored["steps"], now["steps"])):
        for key in ("kept", "n_visible", "vis", "pix", "near_cells"):
            assert s.get(key) == n.get(key), (k, key)
        for key in ("h", "var", "valid", "n_acc", "n_rej", "origin"):
            _same(n["state"][key], s["state"][key], f"step {k} {key}")
        for l in range(len(stored["layers"])):
            _same(n["state"]["layers"][l], s["state"]["layers"][l], f"step {k} layer {l}")
            _same(n["state"]["obs"][l], s["state"]["obs"][l], f"step {k} observed {l}")
            if s["state"]["gvar"][l] is not None:
                _same(n["state"]["gvar"][l], s["state"]["gvar"][l], f"step {k} gauss var {l}")


def test_fixture_exercises_every_rule_the_gate_and_visibility():
    d = load()
    last = d["steps"][-1]
    pts = [s for s in d["steps"] if s["kind"] == "points"]
    assert sum(pts[-1]["state"]["n_rej"]) > 0 and sum(last["state"]["valid"]) > 100
    assert 0 < last["n_visible"] < sum(last["state"]["valid"])
    assert {L["rule"] for L in d["layers"]} == {O.LATEST, O.DIRICHLET, O.CLASSMAX, O.EXPAVG, O.GAUSS}


class _Stored:
    """The stored state with the attributes compare_states reads from an oracle map."""

    def __init__(self, st, layers):
        self.h = np.asarray(st["h"])
        self.var = np.asarray(st["var"])
        self.valid = np.asarray(st["valid"], np.uint8)
        self.n_acc = np.asarray(st["n_acc"], np.uint32)
        self.n_rej = np.asarray(st["n_rej"], np.uint32)
        self.obs = [np.asarray(x, np.uint8) for x in st["obs"]]
        self._layers = [np.asarray(x) for x in st["layers"]]
        self._gvar = [None if x is None else np.asarray(x) for x in st["gvar"]]
        self.p = O.Params(W=0, res=0.0, layers=make_golden.oracle_layers())

    def layer_values(self, l):
        return self._layers[l]

    def gauss_var(self, l):
        return self._gvar[l]


@pytest.mark.gpu
def test_library_matches_stored_values():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_16818_gb300 import mem as M
    d = load()
    g = M.Map(d["W"], d["res"], specs_to(make_golden.LAYERS, "mem"))
    near = np.zeros(d["W"] ** 2, bool)
    for k, ((kind, kw), s) in enumerate(zip(cases.STEPS, d["steps"])):
        if kind == "points":
            xyz, rgb, probs, feat, T = cases.cloud(**kw)
            arrays = dict(rgb=rgb, probs=probs, feat=feat)
            src = [(torch.from_numpy(arrays[n]).cuda(), ls) for n, ls in make_golden.POINT_SOURCES]
            g.fuse_pointcloud(torch.from_numpy(xyz).cuda(), T, src)
            near[s["near_cells"]] = True
        elif kind == "move":
            g.move(kw["xy"])
            assert list(g.origin()) == s["state"]["origin"]
        else:
            H, Wi, K, T, feat, seg = cases.camera(**kw)
            arrays = dict(seg=seg, feat=feat)
            src = [(torch.from_numpy(arrays[n]).cuda(), ls) for n, ls in make_golden.IMAGE_SOURCES]
            vis = torch.empty(d["W"] ** 2, dtype=torch.uint8, device="cuda")
            pix = torch.empty(d["W"] ** 2, dtype=torch.int32, device="cuda")
            g.fuse_image(H, Wi, K, T, src, vis=vis, pix=pix)
            assert vis.cpu().numpy().tolist() == s["vis"], f"step {k}: visibility"
            assert pix.cpu().numpy().tolist() == s["pix"], f"step {k}: pixel indices"
        g.check()
        compare_states(gpu_state(g), _Stored(s["state"], d["layers"]), mask=~near, what=f"step {k} ({kind})")

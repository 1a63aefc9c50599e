"""Writes fusion_w12.json in this folder from the oracle alone (the CUDA path is never called):
`python tests/golden/make_golden.py` from the repository root.

The fixture follows the steps of cases.STEPS on a 12 x 12 map with a colour average (Sec. III-C1),
Dirichlet classes (Eq. 9-11), class max (Sec. III-C3), exponential averaging (Eq. 6) and a
Gaussian feature layer (Eq. 7-8) over the height update with its outlier gate (Sec. III-B); the
last step projects the map into a camera with the visibility walk (Sec. III-A). After every step
it stores the whole state, and for the image step the visibility and pixel index of every cell."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)

import cases  # noqa: E402
import oracle as O  # noqa: E402

LAYERS = [dict(channels=3, rule=O.LATEST), dict(channels=4, rule=O.DIRICHLET, alpha0=1.0),
          dict(channels=4, rule=O.CLASSMAX), dict(channels=4, rule=O.EXPAVG, w=0.3),
          dict(channels=3, rule=O.GAUSS, var_meas=0.5)]
POINT_SOURCES = [("rgb", [0]), ("probs", [1, 2, 3]), ("feat", [4])]
IMAGE_SOURCES = [("seg", [1, 2, 3]), ("feat", [4])]
CITE = ("Sec. III-B (height update, outlier gate), Sec. III-C (fusion rules: Eq. 6 exponential "
        "averaging, Eq. 7-8 Gaussian features, Eq. 9-11 Dirichlet classes, class max), Sec. III-A "
        "(projection into a camera, visibility against the height map)")


def oracle_layers():
    return [O.Layer(L["channels"], L["rule"], w=L.get("w", 0.1), var_meas=L.get("var_meas", 1.0),
                    alpha0=L.get("alpha0", 1.0)) for L in LAYERS]


def state(o):
    return dict(h=o.h.tolist(), var=o.var.tolist(), valid=o.valid.tolist(), n_acc=o.n_acc.tolist(),
                n_rej=o.n_rej.tolist(), origin=list(o.origin),
                layers=[o.layer_values(l).tolist() for l in range(len(LAYERS))],
                obs=[o.obs[l].tolist() for l in range(len(LAYERS))],
                gvar=[o.gauss_var(l).tolist() if L["rule"] == O.GAUSS else None for l, L in enumerate(LAYERS)])


def run_oracle():
    o = O.OracleMap(O.Params(W=cases.W, res=cases.RES, layers=oracle_layers()))
    out = []
    for kind, kw in cases.STEPS:
        rec = dict(kind=kind)
        if kind == "points":
            xyz, rgb, probs, feat, T = cases.cloud(**kw)
            arrays = dict(rgb=rgb, probs=probs, feat=feat)
            r = o.fuse_points(xyz, T, [(arrays[k], ls) for k, ls in POINT_SOURCES], want_cells=True, want_near=True)
            rec["kept"] = int(r["kept"])
            rec["near_cells"] = sorted(set(int(c) for c, nr in zip(r["cells"], r["near"]) if nr))
        elif kind == "move":
            o.move(kw["xy"])
        else:
            H, Wi, K, T, feat, seg = cases.camera(**kw)
            arrays = dict(seg=seg, feat=feat)
            r = o.fuse_image(H, Wi, [(arrays[k], ls) for k, ls in IMAGE_SOURCES], K, T)
            rec["n_visible"] = int(r["n_visible"])
            rec["vis"] = r["vis"].tolist()
            rec["pix"] = r["pix"].tolist()
        rec["state"] = state(o)
        out.append(rec)
    return dict(cite=CITE, W=cases.W, res=cases.RES, layers=LAYERS, steps=out)


if __name__ == "__main__":
    with open(os.path.join(HERE, "fusion_w12.json"), "w") as f:
        json.dump(run_oracle(), f, separators=(",", ":"))
        f.write("\n")
    print("wrote", os.path.join(HERE, "fusion_w12.json"))

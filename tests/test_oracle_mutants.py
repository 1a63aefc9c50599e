"""Planted mistakes: copies of the C oracle, each with one plausible error (a dropped term, a
wrong sign, a transposed index, swapped weights, an argmin for an argmax), must each fail the
oracle's pins in test_oracle_points.py and test_oracle_image_move.py -- so the pins would catch
that class of mistake in the oracle itself. The unaltered copy, built the same way, must pass.
CPU only; the altered copies live in a temporary folder."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
PINS = [os.path.join(ROOT, "tests", "test_oracle_points.py"),
        os.path.join(ROOT, "tests", "test_oracle_image_move.py"),
        os.path.join(ROOT, "tests", "test_oracle_raycast_drift.py"),
        os.path.join(ROOT, "tests", "test_oracle_topk.py"),
        os.path.join(ROOT, "tests", "test_oracle_plugins.py")]

# name -> [(exact source text, replacement)], each text occurring once in mem_oracle.c
MUTANTS = {
    "cell index transposed": [("*cell = iy * c->W + ix;", "*cell = ix * c->W + iy;")],
    "range term of the measurement noise dropped (Sec. III-B)":
        [("float sm = fmaf(c->sigma1, rs, c->sigma0);", "float sm = c->sigma0;")],
    "gate without the cell variance": [("float rhs = lam2 * (vj + vm);", "float rhs = lam2 * vm;")],
    "gate with lambda instead of lambda^2":
        [("float lam2 = c->gate_lambda * c->gate_lambda;", "float lam2 = c->gate_lambda;")],
    "Kalman mean: prior not weighted by its information":
        [("(s->h[j] / s->var[j] + Swz[j]) / P", "(s->h[j] + Swz[j]) / P")],
    "Kalman variance: prior information dropped":
        [("s->var[j] = store_round(c, ORC_F32, 1.0 / P);", "s->var[j] = store_round(c, ORC_F32, 1.0 / Sw[j]);")],
    "average rule returns the sum (Eq. 1)":
        [("th[j * C + k] = store_round(c, fmt, S[k] / N);", "th[j * C + k] = store_round(c, fmt, S[k]);")],
    "exponential averaging weights swapped (Eq. 2)":
        [("c->w[l] * a + (1.0 - c->w[l]) * th[j * C + k]", "(1.0 - c->w[l]) * a + c->w[l] * th[j * C + k]")],
    "Gaussian mean weights swapped (Eq. 6)":
        [("mu = sf2 / den * mu0 + N * s02 / den * mu_ml;", "mu = N * s02 / den * mu0 + sf2 / den * mu_ml;")],
    "Gaussian variance without the prior (Eq. 7)": [("s2 = sf2 * s02 / den;", "s2 = sf2 / den;")],
    "Dirichlet adds the mean instead of the sum (Eq. 12)":
        [("store_round(c, fmt, th[j * C + k] + S[k])", "store_round(c, fmt, th[j * C + k] + S[k] / N)")],
    "class max takes the minimum": [("double best = -INFINITY;", "double best = INFINITY;"),
                                    ("if (M[k] > best) {", "if (M[k] < best) {")],
    "pixel truncated instead of rounded": [("float fu = floorf(u + 0.5f), fv = floorf(v + 0.5f);",
                                            "float fu = floorf(u), fv = floorf(v);")],
    "ray height slope with the wrong sign": [("float ray = fmaf(tq, hz - hc, hc);", "float ray = fmaf(tq, hc - hz, hc);")],
    "pixel index transposed": [("int64_t p = (int64_t)py * Wi + px;", "int64_t p = (int64_t)px * H + py;")],
    "visibility test not strict": [("if ((float)h0[q] >= ray) {", "if ((float)h0[q] > ray + 1.0f) {")],
    "map move shifts the wrong way": [("long oy = iy + sy;", "long oy = iy - sy;")],
    "outlier variance without the rejected count":
        [("s->var[j] + (double)c->outlier_var * nr[j]", "s->var[j] + (double)c->outlier_var")],
    "time variance added to never-observed cells":
        [("if (s->valid[j]) s->var[j] = store_round(c, ORC_F32, s->var[j] + (double)c->time_var);",
          "s->var[j] = store_round(c, ORC_F32, s->var[j] + (double)c->time_var);")],
    "time variance only on cells touched by the call":
        [("if (s->valid[j]) s->var[j] = store_round(c, ORC_F32, s->var[j] + (double)c->time_var);",
          "if (s->valid[j] && np[j]) s->var[j] = store_round(c, ORC_F32, s->var[j] + (double)c->time_var);")],
    "exponential average blends a never-observed cell":
        [("double t = s->obs[l][j] ? c->w[l] * a + (1.0 - c->w[l]) * th[j * C + k] : a;",
          "double t = c->w[l] * a + (1.0 - c->w[l]) * th[j * C + k];")],
    "Gaussian first observation ignores the count": [("s2 = sf2 / N;", "s2 = sf2;")],
    "bf16 storage truncates": [("u = (u + 0x7fffu + ((u >> 16) & 1u)) & 0xffff0000u;", "u = u & 0xffff0000u;")],
    "Dirichlet prior fixed to 1":
        [("if (c->rule[l] == ORC_DIRICHLET) v = store_round(c, c->store[l], c->alpha0[l]);",
          "if (c->rule[l] == ORC_DIRICHLET) v = store_round(c, c->store[l], 1.0);")],
    "class max ties to the largest class": [("if (M[k] > best) {", "if (M[k] >= best) {")],
    "near plane not applied": [("if (!(Zc > c->z_near)) continue;", "if (!(Zc >= 0.0f)) continue;")],
    "range filter halves the maximum range":
        [("if (!(rs >= c->range_min && rs <= c->range_max)) return 0;",
          "if (!(rs >= c->range_min && rs < c->range_max * 0.5f)) return 0;")],
    "map edge off by one": [("if (!(qx >= -half && qx < half && qy >= -half && qy < half)) return 0;",
                             "if (!(qx >= -half && qx <= half && qy >= -half && qy < half)) return 0;")],
    "visibility walk includes the target cell": [("for (int32_t m = 1; m + 1 < n; ++m) {", "for (int32_t m = 1; m < n; ++m) {")],
    "ray parameter not normalised": [("        float tq = (float)num / (float)den;\n        float ray = fmaf(tq, hz - hc, hc);",
                                      "        float tq = (float)num;\n        float ray = fmaf(tq, hz - hc, hc);")],
    "image rule counts two observations per pixel":
        [("apply_rule(c, s, src[qs].layers[b], j, 1.0, S, S);", "apply_rule(c, s, src[qs].layers[b], j, 2.0, S, S);")],
    "invalid cells occlude": [("        if (!s->valid[q]) continue;\n        int32_t num", "        int32_t num")],
    "camera cell not clamped at the far edge": [("  if (!(qx <= half - 1.0f)) qx = half - 1.0f;", "")],
    "move truncates instead of rounding":
        [("long sx = lround((robot_xy[0] - s->origin[0]) / c->res);", "long sx = (long)((robot_xy[0] - s->origin[0]) / c->res);")],
    "move drops the accepted counts": [("      s->n_acc[jn] = a[jo];", "      s->n_acc[jn] = 0;")],
    "fill with a zero border instead of zero flux":
        [("        if (x > 0) s += h[j - 1], ++m;\n        if (x + 1 < W) s += h[j + 1], ++m;\n"
          "        if (y > 0) s += h[j - W], ++m;\n        if (y + 1 < H) s += h[j + W], ++m;\n        h[j] = s / m;",
          "        if (x > 0) s += h[j - 1];\n        if (x + 1 < W) s += h[j + 1];\n"
          "        if (y > 0) s += h[j - W];\n        if (y + 1 < H) s += h[j + W];\n        h[j] = s / 4;")],
    # drift compensation and ray-cast clean-up (Table I rows "drift compensation", "height
    # update & ray cast")
    "drift counts the gate's outliers":
        [("      if (d * d > lam2 * ((float)s->var[j] + vm)) continue;\n      esum", "      esum")],
    "drift counts points in invalid cells":
        [("      if (!s->valid[j]) continue;\n      float d = z - (float)s->h[j];", "      float d = z - (float)s->h[j];")],
    "drift moves the map the wrong way": [("s->h[j] = store_round(c, ORC_F32, s->h[j] + drift);",
                                           "s->h[j] = store_round(c, ORC_F32, s->h[j] - drift);")],
    "drift threshold off by one": [("drift_n >= c->drift_min_points", "drift_n > c->drift_min_points")],
    "drift error summed, not averaged": [("c->drift_alpha * (esum / (double)drift_n)", "c->drift_alpha * esum")],
    "drift ignores alpha": [("c->drift_alpha * (esum / (double)drift_n)", "(esum / (double)drift_n)")],
    "ray ends at the cell's stored height instead of the point":
        [("float ray = fmaf(tq, acc_z[a] - zs, zs);", "float ray = fmaf(tq, (float)h_gate[acc_cell[a]] - zs, zs);")],
    "ray slope with the wrong sign": [("float ray = fmaf(tq, acc_z[a] - zs, zs);", "float ray = fmaf(tq, zs - acc_z[a], zs);")],
    "clean-up clears cells that accepted a point":
        [("if (mark[q] && na[q] == 0 && s->valid[q]) {", "if (mark[q] && s->valid[q]) {")],
    "clean-up walk includes the sensor's cell":
        [("      for (int32_t m = 1; m + 1 < nl; ++m) {\n        int32_t qx", "      for (int32_t m = 0; m + 1 < nl; ++m) {\n        int32_t qx")],
    "clean-up margin ignored": [("if ((float)h_gate[q] - ray > c->ray_margin) mark[q] = 1;",
                                 "if ((float)h_gate[q] - ray > 0.0f) mark[q] = 1;")],
    "rejected points cast rays too":
        [("    if (rej) {\n      ++nr[j];\n", "    if (rej) {\n      ++nr[j];\n      if (c->ray_cleanup) {\n"
          "        acc_cell[n_accpt] = j;\n        acc_z[n_accpt] = z;\n        ++n_accpt;\n      }\n")],
    "clean-up ray parameter not normalised": [("        float tq = (float)num / (float)den;\n        float ray = fmaf(tq, acc_z[a] - zs, zs);",
                                               "        float tq = (float)num;\n        float ray = fmaf(tq, acc_z[a] - zs, zs);")],
    # surface normals (Table I "normal calculation")
    "normal central difference over one cell": [("*g = (hb - ha) / (2.0f * res);", "*g = (hb - ha) / res;")],
    "normal one-sided differences swapped": [("*g = (hb - hm) / res;", "*g = (hm - ha) / res;")],
    "normal not normalised": [("float inv = 1.0f / sqrtf(n2);", "float inv = 1.0f;")],
    "normal slope sign flipped": [("out[3 * j] = -gx * inv;", "out[3 * j] = gx * inv;")],
    "normal ignores invalid neighbours":
        [("int vl = ix > 0 && s->valid[j - 1], vr = ix + 1 < W && s->valid[j + 1];", "int vl = ix > 0, vr = ix + 1 < W;")],
    # top-k class input (Sec. III-C)
    "top-k id off by one": [("&& (int)id == k) v += r[2 * j + 1];", "&& (int)id == k + 1) v += r[2 * j + 1];")],
    "top-k repeated id overwrites": [("&& (int)id == k) v += r[2 * j + 1];", "&& (int)id == k) v = r[2 * j + 1];")],
    "top-k pair order swapped": [("float id = r[2 * j];", "float id = r[2 * j + 1];"),
                                 ("&& (int)id == k) v += r[2 * j + 1];", "&& (int)id == k) v += r[2 * j];")],
    "top-k accepts fractional ids": [("&& id == floorf(id) && (int)id == k)", "&& (int)id == k)")],
    "clean-up ray parameter along x only": [("int32_t num = (qx - sx) * dxs + (qy - sy) * dys;\n        float tq",
                                             "int32_t num = (qx - sx) * dxs;\n        float tq")],
}


def _build(tmp, name, subs):
    d = os.path.join(tmp, name.replace(" ", "_").replace("/", "_")[:40])
    os.makedirs(d, exist_ok=True)
    shutil.copy(os.path.join(ORACLE, "mem_oracle.h"), d)
    src = open(os.path.join(ORACLE, "mem_oracle.c")).read()
    for old, new in subs:
        assert src.count(old) == 1, (name, old)
        src = src.replace(old, new)
    with open(os.path.join(d, "mem_oracle.c"), "w") as f:
        f.write(src)
    lib = os.path.join(d, "liboracle.so")
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", lib,
                           os.path.join(d, "mem_oracle.c"), "-lm"])
    return lib


def _pins(lib):
    env = dict(os.environ, MEM_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] + PINS,
                       cwd=ROOT, env=env, capture_output=True, text=True)
    return r.returncode, r.stdout[-2000:]


def test_unaltered_copy_passes_the_pins(tmp_path):
    rc, out = _pins(_build(str(tmp_path), "unaltered", []))
    assert rc == 0, out


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(tmp_path, name):
    rc, out = _pins(_build(str(tmp_path), name, MUTANTS[name]))
    assert rc == 1, f"{name}: the pins did not fail (exit {rc})\n{out}"


# the float64 U-Net oracle (oracle/unet.py): name -> (exact source text, replacement)
UNET_MUTANTS = {
    "im2col tap order transposed": ("for ky in range(3) for kx in range(3)]", "for kx in range(3) for ky in range(3)]"),
    "col2im overwrites overlapping taps": ("xp[:, ky:ky + H, kx:kx + W, :] += cols[:, :, :, t, :]",
                                          "xp[:, ky:ky + H, kx:kx + W, :] = cols[:, :, :, t, :]"),
    "convolution bias dropped": ("y = im2col(x) @ w.reshape(-1, w.shape[3]) + b", "y = im2col(x) @ w.reshape(-1, w.shape[3])"),
    "upsample gradient averaged": ("return dy.reshape(N, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))",
                                   "return dy.reshape(N, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))"),
    "max-pool gradient to the minimum": ("am = v.argmax(axis=4)", "am = v.argmin(axis=4)"),
    "loss gradient without the factor 2": ("2.0 * diff / cnt", "diff / cnt"),
    "ReLU gradient mask dropped": ('dt = dt * (a[name + ".out"] > 0)', "dt = dt"),
    "skip concatenation order swapped in the forward pass": ("np.concatenate([upsample(e4), e3], axis=3)",
                                                             "np.concatenate([e3, upsample(e4)], axis=3)"),
    "head bias dropped": ('out = d1 @ p["out.w"] + p["out.b"]', 'out = d1 @ p["out.w"]'),
    "max pool takes the minimum": ("return v.max(axis=(2, 4))", "return v.min(axis=(2, 4))"),
    "upsample shifted by a row": ("return x.repeat(2, axis=1).repeat(2, axis=2)",
                                  "return np.roll(x.repeat(2, axis=1).repeat(2, axis=2), 1, axis=1)"),
    "weight gradient halved": ("dw = (im2col(x).T @ d).reshape(w.shape)", "dw = (im2col(x).T @ d).reshape(w.shape) * 0.5"),
    "bias gradient averaged": ("db = d.sum(axis=0)", "db = d.mean(axis=0)"),
    "loss not normalised by the hidden count": ("return float((diff ** 2).sum() / cnt), 2.0 * diff / cnt",
                                                "return float((diff ** 2).sum()), 2.0 * diff / cnt"),
    "hidden mask ignored in the loss": ("diff = (fill + res - target) * hidden", "diff = (fill + res - target)"),
    "decoder split at the skip width": ("du, de1 = split(dcat, c2)", "du, de1 = split(dcat, c1)"),
    "storage rounding skips the decoder input gradient": ('keep("up2", upsample_backward(du))', "upsample_backward(du)"),
    "storage rounding skips the activations": ("r = store(np.maximum(y, 0.0))", "r = np.maximum(y, 0.0)"),
    "storage rounding skips the skip sums": ('de2 = keep("skip2", de2 + maxpool_backward(a["e2"], de3))',
                                             'de2 = de2 + maxpool_backward(a["e2"], de3)'),
    "bf16 rounding truncates": ("u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000)", "u = ((u) & 0xFFFF0000)"),
}

_RUN_UNET = r'''
import sys, types
sys.path.insert(0, ROOT)
import oracle
src = open(ROOT + "/oracle/unet.py").read()
if OLD:
    assert src.count(OLD) == 1, OLD
    src = src.replace(OLD, NEW)
m = types.ModuleType("oracle.unet")
m.__file__ = ROOT + "/oracle/unet.py"
exec(compile(src, m.__file__, "exec"), m.__dict__)
sys.modules["oracle.unet"] = m
oracle.unet = m
import pytest
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", ROOT + "/tests/test_oracle_unet.py"]))
'''


def _unet_pins(old, new):
    code = f"ROOT = {ROOT!r}\nOLD = {old!r}\nNEW = {new!r}\n" + _RUN_UNET
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    return r.returncode, r.stdout[-2000:] + r.stderr[-2000:]


def test_unaltered_unet_oracle_passes_the_pins():
    rc, out = _unet_pins("", "")
    assert rc == 0, out


@pytest.mark.parametrize("name", sorted(UNET_MUTANTS))
def test_planted_unet_mistake_fails_a_pin(name):
    rc, out = _unet_pins(*UNET_MUTANTS[name])
    assert rc == 1, f"{name}: the pins did not fail (exit {rc})\n{out}"


# the PCA plugin oracle (oracle/plugins.py): name -> (exact source text, replacement)
PCA_MUTANTS = {
    "features not centred": ("    Xc = X - m\n", "    Xc = X\n"),
    "smallest eigenvalues taken": ("order = np.argsort(-w, kind=\"stable\")[:n_comp]", "order = np.argsort(w, kind=\"stable\")[:n_comp]"),
    "covariance normalised by n - 1": ("S = Xc.T @ Xc / n", "S = Xc.T @ Xc / (n - 1)"),
    "sign from the smallest component": ("i = int(np.argmax(np.abs(V[k])))", "i = int(np.argmin(np.abs(V[k])))"),
    "unobserved cells included": ("    X = f[obs]\n", "    X = f\n"),
}

_RUN_PCA = r'''
import sys, types
sys.path.insert(0, ROOT)
import oracle
src = open(ROOT + "/oracle/plugins.py").read()
if OLD:
    assert src.count(OLD) == 1, OLD
    src = src.replace(OLD, NEW)
m = types.ModuleType("oracle.plugins")
m.__file__ = ROOT + "/oracle/plugins.py"
exec(compile(src, m.__file__, "exec"), m.__dict__)
sys.modules["oracle.plugins"] = m
oracle.plugins = m
import pytest
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", ROOT + "/tests/test_oracle_plugins.py"]))
'''


def _pca_pins(old, new):
    code = f"ROOT = {ROOT!r}\nOLD = {old!r}\nNEW = {new!r}\n" + _RUN_PCA
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    return r.returncode, r.stdout[-2000:] + r.stderr[-2000:]


def test_unaltered_pca_oracle_passes_the_pins():
    rc, out = _pca_pins("", "")
    assert rc == 0, out


@pytest.mark.parametrize("name", sorted(PCA_MUTANTS))
def test_planted_pca_mistake_fails_a_pin(name):
    rc, out = _pca_pins(*PCA_MUTANTS[name])
    assert rc == 1, f"{name}: the pins did not fail (exit {rc})\n{out}"

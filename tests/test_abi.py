"""The C-ABI library loads and exports every entry point that include/mem.h declares; the
binding's structs match the header's layout. No device work (CPU only)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "mem.h")).read()
    return sorted(set(re.findall(r"^\s*(?:mem_status|const char \*)\s*(mem_\w+)\(", txt, re.M)))


def test_library_exports_every_declared_symbol():
    from paper_2309_16818_gb300 import build, mem
    build.build()
    L = C.CDLL(mem.LIB_PATH)
    names = declared()
    assert len(names) >= 13
    for n in names:
        assert hasattr(L, n), n
    assert sorted(mem.EXPORTS) == names


def test_struct_layout_matches_header():
    """Compile a tiny C program against mem.h and compare sizeof / offsetof with ctypes."""
    import subprocess
    import tempfile
    from paper_2309_16818_gb300 import mem
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "mem.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(mem_map_config), offsetof(mem_map_config, res),
         offsetof(mem_map_config, sigma0), offsetof(mem_map_config, max_points), sizeof(mem_source),
         sizeof(mem_layer_desc));
  return 0;
}'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        got = [int(x) for x in subprocess.check_output([exe]).split()]
    exp = [C.sizeof(mem.MapConfig), mem.MapConfig.res.offset, mem.MapConfig.sigma0.offset,
           mem.MapConfig.max_points.offset, C.sizeof(mem.Source), C.sizeof(mem.LayerDesc)]
    assert got == exp


def test_argument_errors_need_no_device():
    """Invalid configurations are rejected on the host before any CUDA call."""
    from paper_2309_16818_gb300 import mem
    cfg = mem.MapConfig()
    cfg.W, cfg.n_maps, cfg.res = 7, 1, 0.1   # odd W
    h = C.c_void_p()
    assert mem.lib().mem_create_map(C.byref(cfg), C.byref(h)) == mem.ERR_ARG
    assert b"even" in mem.lib().mem_last_error()
    cfg.W, cfg.res = 8, -1.0
    assert mem.lib().mem_create_map(C.byref(cfg), C.byref(h)) == mem.ERR_ARG
    assert mem.lib().mem_fuse_pointcloud(None, 0, None, 0, None, None, None) == mem.ERR_ARG


_NULL_PROBE = r'''
import ctypes as C, sys
sys.path.insert(0, ROOT)
from paper_2309_16818_gb300 import mem as M
L = M.lib()
for name in M.EXPORTS:
    if name == "mem_last_error":
        continue
    f = getattr(L, name)
    args = [None if t is C.c_void_p else (1.0 if t is C.c_float else 1) for t in f.argtypes]
    r = f(*args)
    print(name, r, bool(L.mem_last_error()))
w = (C.c_int32 * 4)(32, 64, 128, 128)
h = C.c_void_p()
print("unet_cin0", L.mem_unet_create(0, w, C.byref(h)))
w2 = (C.c_int32 * 4)(32, 48, 128, 128)
print("unet_width48", L.mem_unet_create(3, w2, C.byref(h)))
'''


def test_null_and_range_arguments_are_rejected_on_the_host():
    """Every entry point given NULL handles/pointers returns MEM_ERR_ARG with a message (the
    destroy calls accept NULL like free), and U-Net shape errors are caught before any device
    work -- all on a machine without a GPU, in a child process so a crash cannot hide."""
    import subprocess
    import sys
    from paper_2309_16818_gb300 import build
    build.build()
    r = subprocess.run([sys.executable, "-c", f"ROOT = {ROOT!r}\n" + _NULL_PROBE], capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    got = {}
    for line in r.stdout.split("\n"):
        parts = line.split()
        if len(parts) >= 2:
            got[parts[0]] = parts[1:]
    from paper_2309_16818_gb300 import mem
    for name in mem.EXPORTS:
        if name == "mem_last_error":
            continue
        status, has_msg = got[name]
        if name in ("mem_destroy_map", "mem_unet_destroy"):
            assert status == "0", name
        elif name == "mem_noalloc_check":
            # its only argument is a stream and NULL is the default stream: no argument error;
            # without a GPU it reports the failed CUDA call
            assert status in (str(mem.OK), str(mem.ERR_CUDA)), (name, status)
        else:
            assert status == str(mem.ERR_ARG) and has_msg == "True", (name, status)
    assert got["unet_cin0"] == [str(mem.ERR_ARG)]
    assert got["unet_width48"] == [str(mem.ERR_ARG)]


@pytest.mark.parametrize("field,value,msg", [
    ("W", 99, "W must be even"), ("W", 0, "W must be even"), ("res", -1.0, "res must be > 0"),
    ("n_maps", 0, "n_maps must be >= 1"), ("n_layers", 17, "n_layers out of range"),
    ("L0_channels", 0, "channels in"), ("L0_rule", 9, "bad rule"), ("L0_dtype", 7, "storage must be"),
    ("range_min", 60.0, "range_min > range_max"), ("L0_w", 1.5, "w in (0, 1]"),
    ("L0_dtype", 1, "CLASSMAX / DIRICHLET layers are F32")])
def test_map_config_is_validated_on_the_host(field, value, msg):
    """mem_create_map rejects an invalid configuration with MEM_ERR_ARG and a message before any
    device call (runs without a GPU)."""
    from paper_2309_16818_gb300 import build, mem
    build.build()
    L = mem.lib()
    c = mem.MapConfig()
    c.W, c.n_maps, c.res, c.n_layers = 100, 1, 0.05, 1
    c.layers[0].channels, c.layers[0].dtype = 3, 0
    c.layers[0].rule = 4 if msg.startswith("CLASSMAX") else (1 if field == "L0_w" else 0)
    c.layers[0].w, c.layers[0].var_meas, c.layers[0].alpha0 = 0.1, 1.0, 1.0
    c.sigma0, c.sigma1, c.gate_lambda = 0.01, 0.002, 2.0
    c.range_min, c.range_max, c.z_near, c.max_points = 0.1, 50.0, 0.05, 1000
    if field.startswith("L0_"):
        setattr(c.layers[0], field[3:], value)
    else:
        setattr(c, field, value)
    h = C.c_void_p()
    assert L.mem_create_map(C.byref(c), C.byref(h)) == mem.ERR_ARG
    assert msg in L.mem_last_error().decode()
    assert not h.value

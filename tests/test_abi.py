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

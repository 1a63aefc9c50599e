"""The benchmark reports a kernel's measured DRAM traffic only when the committed ncu summary
was taken from the current point-path kernel sources: the lookup matches the source hash, and
any change to those sources (even one byte) makes the figure unavailable (null) rather than
stale."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_source_hash_covers_the_point_sources_in_order():
    h = hashlib.sha256()
    for f in bench.POINT_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    assert bench.kernel_source_hash() == h.hexdigest()[:12]
    assert "paper_2309_16818_gb300/csrc/mem_points.cu" in bench.POINT_SOURCES


def test_traffic_row_matches_current_sources_or_is_null(tmp_path, monkeypatch):
    # a summary with one row for the current sources and one for other sources
    cur = bench.kernel_source_hash()
    other = "0" * 12 if cur != "0" * 12 else "1" * 12
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.md").write_text(
        "| kernel | sources | bytes | capture |\n|---|---|---|---|\n"
        f"| k_fuse_warps | {cur} | 55411712 | x |\n"
        f"| k_onesweep | {other} | 3747584 | y |\n")
    for f in bench.POINT_SOURCES:  # the hash reads the sources relative to the root
        d = tmp_path / os.path.dirname(f)
        d.mkdir(parents=True, exist_ok=True)
        (tmp_path / f).write_bytes(open(os.path.join(ROOT, f), "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("k_fuse_warps") == 55411712.0
    assert bench.ncu_traffic("k_onesweep") is None   # taken from other sources
    assert bench.ncu_traffic("k_points_key") is None  # no row
    # one changed byte in a kernel source: the counters no longer describe the kernel
    src = tmp_path / bench.POINT_SOURCES[0]
    src.write_bytes(src.read_bytes() + b"\n")
    assert bench.ncu_traffic("k_fuse_warps") is None


"""The benchmark's stored DRAM-traffic figure for the fused chunk kernel is
tied to that kernel's device code by a digest: an edit of the code before the
end markers of vx_star.cu and vx_star.cuh must drop the figure (the bench then
reports traffic as null), an edit after them must not."""
import os
import shutil

import bench


def _copy_tree(tmp_path):
    root = tmp_path / "repo"
    csrc = root / "paper_2502_09541_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("vx_star.cu", "vx_star.cuh", "vx_probe.cuh"):
        shutil.copy(os.path.join(bench.ROOT, "paper_2502_09541_gb300", "csrc", f), csrc / f)
    (root / "profiles").mkdir()
    shutil.copy(os.path.join(bench.ROOT, "profiles", "star_chunk_kernel_traffic.txt"),
                root / "profiles" / "star_chunk_kernel_traffic.txt")
    return root, csrc


def _edit(path, before_marker, marker):
    text = path.read_bytes()
    cut = text.index(marker)
    if before_marker:
        text = text[:cut] + b"// edited\n" + text[cut:]
    else:
        text = text + b"\n// edited\n"
    path.write_bytes(text)


def test_digest_follows_device_code_only(tmp_path, monkeypatch):
    root, csrc = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    base = bench.kernel_source_digest()
    kept = bench.traffic_ratio()  # the committed figure, or None if taken on other sources
    for f in ("vx_star.cu", "vx_star.cuh"):  # host code after the markers: figure kept
        _edit(csrc / f, False, bench.STAR_KERNEL_END[f])
        assert bench.kernel_source_digest() == base
    assert bench.traffic_ratio() == kept
    for f in ("vx_star.cu", "vx_star.cuh"):  # device code: figure dropped
        root2, csrc2 = _copy_tree(tmp_path / f.replace(".", "_"))
        monkeypatch.setattr(bench, "ROOT", str(root2))
        _edit(csrc2 / f, True, bench.STAR_KERNEL_END[f])
        assert bench.kernel_source_digest() != base
        assert bench.traffic_ratio() is None


def test_digest_covers_the_row_logic_header(tmp_path, monkeypatch):
    root, csrc = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    base = bench.kernel_source_digest()
    p = csrc / "vx_probe.cuh"
    p.write_bytes(p.read_bytes() + b"\n// edited\n")
    assert bench.kernel_source_digest() != base
    assert bench.traffic_ratio() is None

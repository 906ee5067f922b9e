"""Host-side logic of bench.py that needs no GPU."""
import os
import shutil

import bench


def test_code_only_drops_comments_and_layout():
    a = "int f(int x) { // add one\n  return x + 1; /* done */ }\n"
    b = "int f(int x)\n{\n    return x + 1;\n}\n// trailing note\n"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(a.replace("+ 1", "+ 2"))


def test_kernel_hash_ignores_comment_edits_only(tmp_path, monkeypatch):
    src = os.path.join(bench.ROOT, "paper_1203_5004_gb300", "csrc")
    dst = tmp_path / "paper_1203_5004_gb300" / "csrc"
    shutil.copytree(src, dst, ignore=shutil.ignore_patterns("*.o", "*.so"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    f = dst / "wg_fused.cuh"
    text = f.read_text()
    f.write_text("// an added comment line\n" + text)
    assert bench.kernel_source_hash() == h0
    f.write_text(text.replace("constexpr int kShearLanes = 3;", "constexpr int kShearLanes = 4;"))
    assert bench.kernel_source_hash() != h0

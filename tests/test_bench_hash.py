"""The key of the committed ncu figures (bench.kernel_source_hash): a hash of
the device-code sources that ignores comments and whitespace and changes
with any code change (CPU only)."""
import os
import shutil

import bench


def _copy_tree(tmp_path):
    src = os.path.join(bench.ROOT, "paper_1205_0359_gb300", "csrc")
    root = tmp_path / "root"
    shutil.copytree(src, root / "paper_1205_0359_gb300" / "csrc")
    return root


def test_strip_comments():
    src = "int a; // one\n/* two\n three */ int  b;\n\tint c;"
    assert bench.strip_comments(src) == "int a; int b; int c;"


def test_hash_ignores_comments_and_follows_code(tmp_path, monkeypatch):
    root = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    h0 = bench.kernel_source_hash()
    f = root / "paper_1205_0359_gb300" / "csrc" / "blas_impl.cuh"
    text = f.read_text()
    f.write_text("// a new comment line\n" + text.replace("\n", "\n   ", 3))
    assert bench.kernel_source_hash() == h0
    f.write_text(text + "\nconstexpr int a_new_constant = 1;\n")
    assert bench.kernel_source_hash() != h0
    # the host orchestration is not part of the key
    f.write_text(text)
    s = root / "paper_1205_0359_gb300" / "csrc" / "solver.cu"
    s.write_text(s.read_text() + "\nint host_only_change = 0;\n")
    assert bench.kernel_source_hash() == h0

"""The bench's capture keys: the code hash ignores comments and blank lines
and nothing else (CPU only)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_hash_ignores_comments_only(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2201_07408_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text("int f(int a)\n{\n    return a + 1;   // one\n}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.source_code_sha(["k.cu"])
    (csrc / "k.cu").write_text("/* a kernel\n   of one line */\nint f(int a)\n{\n\n    return a + 1;\n}\n")
    assert bench.source_code_sha(["k.cu"]) == h0
    (csrc / "k.cu").write_text("int f(int a)\n{\n    return a + 2;   // one\n}\n")
    assert bench.source_code_sha(["k.cu"]) != h0


def test_table_entries_name_existing_sources():
    for table in (bench.NCU_TRAFFIC, bench.NCU_L1):
        for (_, _, _), (_, src, sha) in table.items():
            assert os.path.exists(os.path.join(ROOT, "paper_2201_07408_gb300", "csrc", src))
            assert len(sha) == 64

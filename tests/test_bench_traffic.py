"""bench.py's traffic record is keyed on a digest of the kernel source that
ignores comments and blank lines: a comment edit keeps the recorded DRAM
bytes, a code edit drops them (the counters no longer describe the kernel)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

SRC = """// kernel
__global__ void k(float *x) {  // one store
  x[threadIdx.x] = 1.f;
}
"""


def test_digest_ignores_comments_only(tmp_path):
    a, b, c = tmp_path / "a.cu", tmp_path / "b.cu", tmp_path / "c.cu"
    a.write_text(SRC)
    b.write_text("/* a block\n   comment */\n" + SRC.replace("// one store", "// a different remark") + "\n\n")
    c.write_text(SRC.replace("1.f", "2.f"))
    assert bench.kernel_source_digest(str(a)) == bench.kernel_source_digest(str(b))
    assert bench.kernel_source_digest(str(a)) != bench.kernel_source_digest(str(c))


def test_record_is_consistent():
    rec = json.load(open(os.path.join(ROOT, "profiles", "cell_pass_lognormal128_traffic.json")))
    assert rec["bytes_per_launch"] == rec["dram_read_bytes"] + rec["dram_write_bytes"]
    assert len(rec["kernel_source_digest"]) == 64


def test_digest_covers_every_listed_source(tmp_path):
    a, h, h2 = tmp_path / "a.cu", tmp_path / "a.h", tmp_path / "a2.h"
    a.write_text(SRC)
    h.write_text("constexpr float kC = 0.5f;  // a constant\n")
    h2.write_text("constexpr float kC = 0.25f;\n")
    assert bench.kernel_source_digest([str(a), str(h)]) != bench.kernel_source_digest([str(a), str(h2)])
    assert bench.kernel_source_digest([str(a)]) == bench.kernel_source_digest(str(a))

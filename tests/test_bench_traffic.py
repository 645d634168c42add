"""bench.py reports an ncu DRAM figure as roofline.traffic only while the
measured kernel's definition is the one the counters were taken on."""
import hashlib
import os

import bench


def test_kernel_text_is_the_whole_definition(tmp_path):
    src = tmp_path / "k.cu"
    src.write_text("// x\ntemplate <int A>\n__global__ void foo_kernel(int *p)\n{\n    if (p) { p[0] = A; }\n}\n"
                   "__global__ void bar_kernel(int *p) { }\n")
    text = bench.kernel_text(str(src), "foo_kernel")
    assert text.startswith("template <int A>") and text.endswith("}")
    assert "bar_kernel" not in text and "p[0] = A;" in text
    assert bench.kernel_text(str(src), "missing_kernel") is None


def test_traffic_follows_the_kernel_hash(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("template <int A>\n__global__ void foo_kernel(int *p)\n{\n    p[0] = A;\n}\n")
    digest = hashlib.sha256(bench.kernel_text(str(src), "foo_kernel").encode()).hexdigest()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "TRAFFIC", {("k", "w"): {"bytes": 123.0, "source": "k.cu", "kernel": "foo_kernel",
                                                        "sha256": digest}})
    assert bench.traffic_bytes("k", "w") == 123.0
    assert bench.traffic_bytes("k", "other") is None
    # any edit of the definition voids the figure; text outside it does not
    src.write_text("// note\n" + src.read_text())
    assert bench.traffic_bytes("k", "w") == 123.0
    src.write_text(src.read_text().replace("p[0] = A;", "p[0] = A + 1;"))
    assert bench.traffic_bytes("k", "w") is None


def test_recorded_traffic_matches_the_current_kernels():
    """Every recorded figure names an existing kernel; a stale hash reads as null."""
    for (kern, wl), t in bench.TRAFFIC.items():
        path = os.path.join(bench.ROOT, t["source"])
        assert os.path.exists(path)
        assert bench.kernel_text(path, t["kernel"]) is not None
        got = bench.traffic_bytes(kern, wl)
        assert got is None or got == t["bytes"]

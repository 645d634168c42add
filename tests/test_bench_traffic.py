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


def test_alu_bound_takes_the_slower_pipe():
    """Issue lanes against the MUFU pipe at its ex2 and rcp rates: the
    self-energy pair (20 FP32 + 1 ex2 + 3 rcp) is MUFU bound at GB300's measured
    rates (ex2 32, rcp 16 per SM per clock) and at the nominal 16 and 16; the
    loop-kernel evaluation (14 + 1 + 1) is issue bound at both."""
    measured, nominal = {"ex2": 32.0, "rcp": 16.0}, {"ex2": 16.0, "rcp": 16.0}
    assert bench.alu_clk_per_unit(20, 1, 3, measured) == 1 / 32 + 3 / 16
    assert bench.alu_clk_per_unit(20, 1, 3, nominal) == 4 / 16
    assert bench.alu_clk_per_unit(14, 1, 1, measured) == 16 / 128
    assert bench.alu_clk_per_unit(14, 1, 1, nominal) == 16 / 128


def test_bench_functions_bind_their_arguments():
    """Every function of bench.py that reads `args` receives or binds it (the
    default bench line runs helpers that take no command-line arguments)."""
    import ast
    tree = ast.parse(open(os.path.join(bench.ROOT, "bench.py")).read())
    for fn in (n for n in ast.walk(tree) if isinstance(n, ast.FunctionDef)):
        params = {a.arg for a in fn.args.args}
        uses = any(isinstance(n, ast.Name) and n.id == "args" for n in ast.walk(fn))
        bound = any(isinstance(t, ast.Name) and t.id == "args"
                    for n in ast.walk(fn) if isinstance(n, ast.Assign) for t in n.targets)
        assert not uses or "args" in params or bound, fn.name

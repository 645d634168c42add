"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/qpfrg.h (no compute calls: these run without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "qpfrg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qpfrg_[a-z_0-9]+)\s*\(", src)))


def test_header_declarations_match_binding():
    from paper_2005_00827_gb300 import api
    assert declared_functions() == sorted(api.EXPORTS)


def test_library_exports_every_declared_symbol():
    from paper_2005_00827_gb300 import api
    lib = api.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_library_targets_sm103a():
    from paper_2005_00827_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.NVCC_FLAGS)
    assert os.path.exists(build.build())


def test_default_options():
    import math

    from paper_2005_00827_gb300 import api
    o = api.qpfrg_default_options()
    assert o.channel_mask == api.QPFRG_CH_ALL
    assert o.step == pytest.approx(math.log(0.98))
    assert o.stop_abs_v == 20.0 and o.eta == 0.02 and o.precision == api.QPFRG_FP64


def test_no_cpu_fallback_without_device():
    import torch

    from paper_2005_00827_gb300 import api
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(api.QpfrgError) as ei:
        api.Context(16, 4, 4, stream=0)
    assert ei.value.status == api.QPFRG_ERR_CUDA


def test_product_path_never_imports_oracle():
    pkg = os.path.join(ROOT, "paper_2005_00827_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.replace("Oracle", "").lower() or f == "inputs.py", f

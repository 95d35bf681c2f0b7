"""Host-side checks of the C ABI (no GPU needed): the library builds, loads
and exports every function that include/fvgb.h declares, and the binding
reports errors instead of falling back to anything."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fvgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fv_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("fv_create_blocks", "fv_set_state", "fv_residual", "fv_rk_stage", "fv_exchange_ghosts",
              "fv_adjoint_vjp", "fv_destroy", "fv_last_error", "fv_residual_norms"):
        assert f in names


def test_library_exports_every_declared_symbol():
    import paper_2012_02925_gb300 as fv
    from paper_2012_02925_gb300 import build
    build.build()
    L = fv.load_library()
    for name in declared_functions():
        assert hasattr(L, name), name
    assert set(fv.EXPORTS) <= set(declared_functions())


def test_no_gpu_means_a_clean_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import cases
    import paper_2012_02925_gb300 as fv
    with pytest.raises(fv.FvError) as e:
        fv.Solver.from_problem(cases.vortex_2d(8))
    assert e.value.code == fv.FV_ERR_CUDA


def test_product_code_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2012_02925_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text and "fv_oracle" not in text, f

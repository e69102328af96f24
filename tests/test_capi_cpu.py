"""Host-side checks of the C ABI (no GPU needed, no compute calls).

* libgbi.so builds and exports every function declared in include/gbi.h;
* the pure host calls (sizes, tables, status strings) answer;
* the generated tables (derived independently of the oracle, by exact rational
  arithmetic in gen_tables.py) agree with the oracle's quadrature and embeddings;
* the committed generated header is what the generator produces.
"""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbi.h")


@pytest.fixture(scope="module")
def gbi():
    import paper_1411_0278_gb300 as g
    from paper_1411_0278_gb300 import _native
    if not os.path.exists(_native.LIB_PATH):
        from paper_1411_0278_gb300 import build
        build.build()
    g.lib()
    return g


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gbi_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(gbi):
    names = declared_functions()
    assert len(names) >= 15
    L = gbi.lib()
    for n in names:
        assert hasattr(L, n), n


def test_host_calls(gbi):
    assert [gbi.h(t) for t in (2, 3, 4, 5, 40)] == [8, 25, 48, 77, 41]
    assert [gbi.d(t) for t in (2, 3, 4, 5, 40)] == [14, 31, 54, 83, 47]
    assert gbi.h(6) == -1 and gbi.h(1) == -1
    assert gbi.status_string(gbi.GBI_ERR_OVERLAP).startswith("spheres overlap")
    with pytest.raises(gbi.GbiError):
        gbi.component_scales(7)


def test_tuning_calls_validate_without_a_device(gbi):
    """The tuning entry points reject a missing context before touching the GPU."""
    import ctypes
    L = gbi.lib()
    offs = (ctypes.c_int * 2)(0, 10)
    assert L.gbi_tune(None, 2, 1, offs, 1, None) == gbi.GBI_ERR_ARG
    assert L.gbi_set_wpt(None, 4) == gbi.GBI_ERR_ARG
    assert L.gbi_pass_wpt(None, 2, 2, 2, 1, 100, 0) == -1
    assert L.gbi_solve_graph_replays(None) == -1
    assert L.gbi_kernel_launches(None) == -1


def test_nearfield_calls_validate_without_a_device(gbi):
    import ctypes
    import numpy as np
    from paper_1411_0278_gb300 import nearfield
    L = gbi.lib()
    th = nearfield.init_theta(0)
    assert th.size == gbi._native.MLP_NPARAM and th.dtype == np.float32
    assert L.gbi_mlp_set(None, th.ctypes.data, 1.0) == gbi.GBI_ERR_ARG
    assert L.gbi_mlp_forward(None, 1, None, None, None) == gbi.GBI_ERR_ARG
    n = ctypes.c_int()
    assert L.gbi_pairs(None, 10, None, 1.0, 4.0, 0, None, ctypes.byref(n)) == gbi.GBI_ERR_ARG
    assert L.gbi_mlp_train(None, 10, None, None, 1.0, 1, None, None, 1, 1, 1e-3, 1e-4, None) == gbi.GBI_ERR_ARG


def test_generated_tables_agree_with_oracle(gbi):
    from oracle import galerkin, tensors
    for trunc in (2, 3, 4, 5, tensors.MINIMAL):
        MB = tensors.ModeBasis(trunc)
        np.testing.assert_allclose(gbi.component_scales(trunc), MB.scale, rtol=1e-13)
        np.testing.assert_allclose(gbi.self_scalars(trunc), galerkin.self_scalars(trunc, 1.0), rtol=1e-11)


def test_generated_header_is_current(tmp_path):
    import sys
    sys.path.insert(0, os.path.join(ROOT, "paper_1411_0278_gb300"))
    try:
        import gen_tables
    finally:
        sys.path.pop(0)
    out = tmp_path / "g.cuh"
    gen_tables.emit(str(out))
    committed = open(os.path.join(ROOT, "paper_1411_0278_gb300", "csrc", "gbi_generated.cuh")).read()
    assert out.read_text() == committed


def test_product_package_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1411_0278_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f

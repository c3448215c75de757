"""The C-ABI library loads without a GPU and exports every entry point declared in include/*.h."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(toeplitz_ols_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    path = __graft_entry__._build_module().build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    for must in ("toeplitz_ols_create", "toeplitz_ols_solve", "toeplitz_ols_solve_batched",
                 "toeplitz_ols_solve_device", "toeplitz_ols_stream_open", "toeplitz_ols_gk_pass"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib):
    import paper_2112_12994_gb300 as t
    assert set(_declared()) <= set(t.SIGNATURES), set(_declared()) - set(t.SIGNATURES)


def test_host_side_contract_without_gpu(lib):
    import paper_2112_12994_gb300 as t
    assert t.strerror(t.TOLS_ERR_ARG) == "invalid argument"
    assert t.strerror(t.TOLS_NOT_CONVERGED).startswith("not converged")
    cfg = t.tols_config()
    t.lib.toeplitz_ols_config_default(ctypes.byref(cfg))
    assert cfg.precision == t.TOLS_FP64 and cfg.precond == t.TOLS_PRECOND_GRAM_CHOL
    # null output pointer is an argument error before any CUDA call
    assert t.lib.toeplitz_ols_create(None, ctypes.byref(cfg)) == t.TOLS_ERR_ARG
    # with no sm_103 device here, create reports NO_DEVICE rather than crashing
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if not has_gpu:
        h = ctypes.c_void_p()
        assert t.lib.toeplitz_ols_create(ctypes.byref(h), ctypes.byref(cfg)) == t.TOLS_ERR_NO_DEVICE


def test_binding_checks_device_buffers(lib):
    # the binding refuses a tensor that is too small, of the wrong element size or not contiguous before any
    # address reaches the library (CPU tensors stand in: the check needs no device)
    torch = pytest.importorskip("torch")
    import paper_2112_12994_gb300 as t
    y = torch.zeros(100, dtype=torch.float64)
    with pytest.raises(t.TolsError, match="d_unif"):
        t.toeplitz_ols_lsar(None, y, 100, 10, 20, torch.zeros(150, dtype=torch.float64))
    with pytest.raises(t.TolsError, match="d_unif"):
        t.toeplitz_ols_lsar(None, y, 100, 10, 20, torch.zeros(200, dtype=torch.float32))
    with pytest.raises(t.TolsError, match="d_rows"):
        t.toeplitz_ols_lsar(None, y, 100, 10, 20, torch.zeros(200, dtype=torch.float64),
                            torch.zeros(200, dtype=torch.int32))
    with pytest.raises(t.TolsError, match="d_y"):
        t.toeplitz_ols_gk_pass(None, t.TOLS_MIXED, y, 100, 5, torch.zeros(5, dtype=torch.float64), None, 0.0,
                               torch.zeros(95, dtype=torch.float32), torch.zeros(5, dtype=torch.float64))
    with pytest.raises(t.TolsError, match="d_u_new"):
        t.toeplitz_ols_gk_pass(None, t.TOLS_FP64, y, 100, 5, torch.zeros(5, dtype=torch.float64), None, 0.0,
                               torch.zeros(190, dtype=torch.float64)[::2], torch.zeros(5, dtype=torch.float64))
    with pytest.raises(t.TolsError, match="d_phi"):
        t.toeplitz_ols_solve_device(None, y, 100, 20, torch.zeros(19, dtype=torch.float64))


def test_binding_checks_sketch_buffers(lib):
    torch = pytest.importorskip("torch")
    import paper_2112_12994_gb300 as t
    y = torch.zeros(3000, dtype=torch.float64)
    with pytest.raises(t.TolsError, match="d_signs"):          # m2 = 4096 signs needed for m = 2997
        t.toeplitz_ols_srht(None, y, 3000, 3, torch.zeros(2997, dtype=torch.float64),
                            torch.zeros(10, dtype=torch.int64), torch.zeros(3, dtype=torch.float64))
    with pytest.raises(t.TolsError, match="d_rows"):
        t.toeplitz_ols_srht(None, y, 3000, 3, torch.zeros(4096, dtype=torch.float64),
                            torch.zeros(10, dtype=torch.int32), torch.zeros(3, dtype=torch.float64))
    keep = [np.arange(1498), np.arange(749)]
    with pytest.raises(t.TolsError, match="d_rh_unif"):
        t.toeplitz_ols_rh_lsar(None, y, 3000, 4, 100, 4, keep, torch.zeros(4 * (100 + 749), dtype=torch.float64),
                               torch.zeros(100, dtype=torch.float64), torch.zeros(400, dtype=torch.float64))


def _header_structs():
    """Field names and C types of the header's `typedef struct { ... } name;` blocks, comments stripped."""
    import re
    text = open(os.path.join(ROOT, "include", "toeplitz_ols.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct \{(.*?)\}\s*(\w+);", text, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            m = re.match(r"^(long long|\w+)\s*(\*?)\s*(.+)$", decl)     # one type, one or more names
            for nm in m.group(3).split(","):
                fields.append((nm.strip(), (m.group(1) + m.group(2)).replace(" ", "")))
        out[name] = fields
    return out


def test_binding_structs_mirror_the_header():
    """Every struct the C ABI passes by pointer has its ctypes mirror in the binding with the same fields in the
    same order and of the same size, so the two sides agree on the layout."""
    import ctypes
    import paper_2112_12994_gb300 as t
    sizes = {"int": 4, "double": 8, "longlong": 8, "size_t": 8, "void*": 8}
    for name, fields in _header_structs().items():
        mirror = getattr(t, name)
        assert [f for f, _ in mirror._fields_] == [f for f, _ in fields], name
        for (f, ctype), (_, py) in zip(fields, mirror._fields_):
            want = sizes.get(ctype, None)
            got = ctypes.sizeof(py)
            if want is None:            # a nested struct: compare with its own mirror
                want = ctypes.sizeof(getattr(t, ctype))
            assert got == want, (name, f, ctype, got)

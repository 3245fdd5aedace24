"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point include/lbm.h declares, and the binding's marshalling
matches the header's struct layouts."""
import ctypes
import os
import re

import pytest

from paper_1810_09299_gb300 import lbm, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(lbm.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return lbm.lib()


def test_library_exports_every_declared_symbol(L):
    declared = _header_functions()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(L, name), name
    assert sorted(lbm.EXPORTS) == declared


def test_struct_layouts_match_header():
    # lbm_params: 6 int32 + 8 doubles + 18 doubles + 1 double
    assert ctypes.sizeof(lbm.LbmParams) == 6 * 4 + 27 * 8
    assert lbm.LbmParams.rho_l.offset == 24
    assert ctypes.sizeof(lbm.LbmDiag) == 11 * 8


def _header_struct_fields(name):
    """Field names of `typedef struct { ... } name;` in include/lbm.h, in order."""
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "lbm.h")).read(), flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + ";", src).group(1)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        for part in decl.split(","):
            tok = part.strip().split()[-1]
            names.append(re.sub(r"\[.*\]", "", tok))
    return names


def test_binding_fields_follow_the_header():
    """The ctypes mirrors of lbm_params and lbm_diag name the header's fields in its order."""
    assert [f[0] for f in lbm.LbmParams._fields_] == _header_struct_fields("lbm_params")
    assert [f[0] for f in lbm.LbmDiag._fields_] == _header_struct_fields("lbm_diag")
    assert [f[0] for f in lbm.LbmDrop._fields_] == _header_struct_fields("lbm_drop")
    assert ctypes.sizeof(lbm.LbmDrop) == 4 * 8


def test_strerror_and_static_queries(L):
    assert lbm.strerror(0) == "ok"
    assert "invalid" in lbm.strerror(lbm.LBM_ERR_INVALID_ARG)
    assert lbm.num_variants() >= 1
    assert L.lbm_destroy(None) == 0
    assert L.lbm_kernel_launches(None) == 0


def test_invalid_arguments_rejected_before_device_work(L):
    """Validation happens on the host before any CUDA call."""
    h = ctypes.c_void_p()
    bad = []
    # nz * pitch (pitch = nr rounded up to 32) must stay below 2^31 node indices
    for kw in ({"nr": 1}, {"nz": 0}, {"rho_g": 0.0}, {"nu_l": -1.0}, {"W": 0.0}, {"mobility": 0.0},
               {"sigma": -0.1}, {"precision": 7}, {"p_coupling": 3}, {"collision": 2}, {"collision": -1},
               {"nz": 1 << 16, "nr": (1 << 15) + 1},
               # 16-bit storage: the column scales must be FP16 numbers (nr <= 65536)
               {"nz": 16, "nr": 65537, "precision": "mix_fp16"},
               {"nz": 16, "nr": 65537, "precision": "mix_bf16"}):
        c = workloads.static_drop(nr=16, nz=16, R=4.0)
        c.update(kw)
        bad.append(c)
    c = workloads.static_drop(nr=16, nz=16, R=4.0)
    c["sg"] = [2.5] * 9
    bad.append(c)
    for c in bad:
        p = lbm.make_params(c)
        assert L.lbm_create(ctypes.byref(p), None, ctypes.byref(h)) == lbm.LBM_ERR_INVALID_ARG
    assert L.lbm_create(None, None, ctypes.byref(h)) == lbm.LBM_ERR_INVALID_ARG
    p = lbm.make_params(workloads.static_drop(nr=16, nz=16, R=4.0))
    assert L.lbm_batch_create(ctypes.byref(p), 0, None, ctypes.byref(h)) == lbm.LBM_ERR_INVALID_ARG
    # mixed precisions in one batch
    arr = (lbm.LbmParams * 2)(lbm.make_params(dict(workloads.static_drop(nr=16, nz=16, R=4.0), precision="fp32")),
                              lbm.make_params(workloads.static_drop(nr=16, nz=16, R=4.0)))
    assert L.lbm_batch_create(arr, 2, None, ctypes.byref(h)) == lbm.LBM_ERR_INVALID_ARG


def test_oracle_binding_fields_follow_its_header():
    """The same check for the oracle's parameter and diagnostics blocks."""
    import oracle

    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "oracle", "axilbm_oracle.h")).read(), flags=re.S)

    def fields(name):
        body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + ";", src).group(1)
        out = []
        for decl in filter(None, (d.strip() for d in body.split(";"))):
            for part in decl.split(","):
                out.append(re.sub(r"\[.*\]", "", part.strip().split()[-1]))
        return out

    assert [f[0] for f in oracle.OrcParams._fields_] == fields("orc_params")
    assert [f[0] for f in oracle.OrcDiag._fields_] == fields("orc_diag")

"""The C library loads without a GPU and exports every symbol include/nnmg.h declares."""
import os
import re

from paper_2412_10910_gb300 import _abi

HEADER = os.path.join(os.path.dirname(__file__), "..", "include", "nnmg.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nnmg_[a-z_0-9]+)\s*\(", text)))


def test_header_declarations_are_exported_and_bound():
    lib = _abi.load()
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
        assert n in _abi.PROTOTYPES, n


def test_default_options_host_only():
    import ctypes as C
    lib = _abi.load()
    o = _abi.Options()
    lib.nnmg_default_options(C.byref(o))
    assert (o.degree, o.cheb_degree, o.lanczos_steps, o.max_nrhs) == (1, 3, 12, 16)
    assert o.smoothing_range == 20.0 and o.eig_safety == 1.2 and o.deterministic == 0


def test_options_struct_matches_header():
    """The ctypes mirror of nnmg_options has the header's fields in order."""
    text = open(HEADER).read()
    body = re.search(r"typedef struct \{([^}]*)\} nnmg_options;", text).group(1)
    fields = re.findall(r"(int|double)\s+(\w+);", body)
    names = [n if n != "lambda" else "lam" for _, n in fields]
    assert names == [f[0] for f in _abi.Options._fields_]


def test_invalid_arguments_rejected_without_gpu_work():
    import ctypes as C
    lib = _abi.load()
    h = C.c_void_p()
    o = _abi.Options()
    lib.nnmg_default_options(C.byref(o))
    assert lib.nnmg_setup_hierarchy(None, 0, C.byref(o), None, C.byref(h)) == _abi.INVALID_ARG
    assert b"n_levels" in lib.nnmg_last_error()
    o.degree = 7
    d = (_abi.LevelDesc * 1)()
    assert lib.nnmg_setup_hierarchy(d, 1, C.byref(o), None, C.byref(h)) == _abi.INVALID_ARG
    o.degree, o.deterministic = 1, 2
    assert lib.nnmg_setup_hierarchy(d, 1, C.byref(o), None, C.byref(h)) == _abi.INVALID_ARG
    assert b"invalid options" in lib.nnmg_last_error()
    assert lib.nnmg_n_levels(None) == 0 and lib.nnmg_hierarchy_bytes(None) == 0


def test_profile_columns_match_header():
    """The Python names of nnmg_vcycle_profile's columns follow the header's
    NNMG_PROF_* indices (the paper's six V-cycle components, then the two
    kernel classes)."""
    text = open(HEADER).read()
    idx = {m.group(1): int(m.group(2))
           for m in re.finditer(r"#define NNMG_PROF_([A-Z]+)\s+(\d+)", text)}
    assert idx.pop("COLS") == len(_abi.PROF_COLUMNS)
    names = {"PRE": "pre_smoother", "RESIDUAL": "residual", "RESTRICT": "restrictor",
             "COARSE": "coarse_solver", "PROLONG": "prolongator", "POST": "post_smoother",
             "OPERATOR": "operator", "VECTOR": "vector"}
    assert sorted(idx) == sorted(names)
    for k, i in idx.items():
        assert _abi.PROF_COLUMNS[i] == names[k], k


def test_size_estimate_runs_on_the_host():
    """nnmg_estimate_bytes needs no GPU (it numbers the meshes on the host):
    its solve bytes follow from the node counts of the oracle's independent
    numbering, and bad arguments are rejected."""
    import numpy as np
    from oracle import dofs
    from paper_2412_10910_gb300 import nnmg
    from synthetic import config_levels
    levels = config_levels("c1_2d_q1")
    k, nrhs = 2, 4
    hb, sb = nnmg.nnmg_estimate_bytes(levels, k, 1, nrhs=nrhs)
    counts = []
    for lv in levels:
        node_of, nn, _, _ = dofs.number_dofs(lv.cells, k, 2)
        counts.append((nn, lv.cells.shape[0]))
    # V-cycle vectors (f, x on every level; t, d and the cell buffer above the
    # coarsest) in FP32 and FP64, plus six PCG vectors (five FP64, one FP32)
    expect = 0
    for l, (nn, nc) in enumerate(counts):
        per = nn * nrhs * (4 if l else 2) + (counts[l - 1][1] * (k + 1) ** 2 * nrhs if l else 0)
        expect += per * 12
    expect += counts[-1][0] * nrhs * (5 * 8 + 4)
    assert sb == expect
    nc_top = counts[-1][1]
    assert hb > nc_top * 3 * (k + 1) ** 2 * 12          # FP64 + FP32 metric terms of the top level
    with np.testing.assert_raises(nnmg.NNMGError):
        nnmg.nnmg_estimate_bytes(levels, 7, 1)

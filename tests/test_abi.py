"""The C-ABI library loads without a GPU and exports every symbol include/dupin.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2504_09311_gb300", "libdupin.so")


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dupin.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dupin_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libdupin():
    if not os.path.exists(LIB):
        import __graft_entry__

        __graft_entry__.build()
    return ctypes.CDLL(LIB)


def test_header_declares_expected_api():
    names = declared_functions()
    for must in ("dupin_graph_load", "dupin_peel", "dupin_peel_batch", "dupin_serve_create", "dupin_serve_submit"):
        assert must in names


def test_every_declared_symbol_is_exported(libdupin):
    for name in declared_functions():
        assert hasattr(libdupin, name), name


def test_binding_covers_every_symbol():
    from paper_2504_09311_gb300 import dupin

    assert sorted(dupin.EXPORTS) == declared_functions()


def test_version_and_errors_without_gpu(libdupin):
    libdupin.dupin_version.restype = ctypes.c_char_p
    assert libdupin.dupin_version().decode().count(".") == 2
    # argument validation happens before any device work
    from paper_2504_09311_gb300 import dupin

    h = ctypes.c_void_p()
    rc = dupin.lib().dupin_graph_load(None, None, ctypes.byref(h))
    assert rc == dupin.ERR_INVALID_ARG
    assert "NULL" in dupin.last_error()


def test_batch_shape_arguments_without_gpu():
    """The launch-shape entry points reject bad arguments before any device call."""
    from paper_2504_09311_gb300 import dupin

    L = dupin.lib()
    assert L.dupin_batch_set_threads(64) == dupin.ERR_INVALID_ARG
    assert L.dupin_batch_get_threads(None) == dupin.ERR_INVALID_ARG
    assert L.dupin_batch_tune(None, None, -1, None, None) == dupin.ERR_INVALID_ARG
    assert L.dupin_batch_tune(None, None, 2, None, None) == dupin.ERR_INVALID_ARG


def test_struct_layouts_match_header():
    from paper_2504_09311_gb300 import dupin

    # 2 int64 + 7 pointers + uint32 (+ padding)
    assert ctypes.sizeof(dupin.GraphDesc) == 2 * 8 + 7 * 8 + 8
    assert ctypes.sizeof(dupin.Params) == 4 + 4 + 8 + 8 + 8 + 4 + 4 + 8 + 8  # ... + clique_q (+ padding)
    assert ctypes.sizeof(dupin.Result) == 6 * 8 + 10 * 8 + 4 * 4 + 8  # ... + phase_ms[4] + tail_ctas
    # and the library's own sizeof() of every public struct agrees
    L = dupin.lib()
    for st, nm in ((dupin.GraphDesc, b"dupin_graph_desc"), (dupin.Params, b"dupin_params"),
                   (dupin.Result, b"dupin_result"), (dupin.ServeConfig, b"dupin_serve_config"),
                   (dupin.ServeStats, b"dupin_serve_stats_t")):
        assert L.dupin_struct_size(nm) == ctypes.sizeof(st), nm
    assert L.dupin_struct_size(b"no_such_struct") == -1


def test_product_path_does_not_import_oracle():
    """The package and bench's timed path never reach the oracle."""
    import glob

    for path in glob.glob(os.path.join(ROOT, "paper_2504_09311_gb300", "**", "*.py"), recursive=True):
        src = open(path).read()
        assert "import oracle" not in src and "from oracle" not in src, path
    for path in glob.glob(os.path.join(ROOT, "paper_2504_09311_gb300", "csrc", "*")):
        src = open(path).read()
        assert "dupin_oracle" not in src and "liboracle" not in src, path


def test_binding_constants_match_header():
    """Every integer #define of include/dupin.h that the binding mirrors has the same value there."""
    from paper_2504_09311_gb300 import dupin

    src = open(os.path.join(ROOT, "include", "dupin.h")).read()
    defs = {m.group(1): int(m.group(2)) for m in re.finditer(r"^#define DUPIN_([A-Z0-9_]+)\s+(-?\d+)u?\b", src, re.M)}
    mirrored = {k: v for k, v in defs.items() if hasattr(dupin, k)}
    assert len(mirrored) >= 25, sorted(defs)
    for k, v in mirrored.items():
        assert getattr(dupin, k) == v, k
    assert set(dupin.METRICS.values()) == {defs[k] for k in ("DG", "DW", "FD", "TDS", "KCLIDS")}


def test_params_field_offsets():
    """dupin_params as the header lays it out: clique_q after tail_arc_cap."""
    from paper_2504_09311_gb300 import dupin

    offs = {name: getattr(dupin.Params, name).offset for name, _ in dupin.Params._fields_}
    assert offs == {"metric": 0, "k_mult": 4, "eps_num": 8, "eps_den": 16, "max_rounds": 24, "flags": 32,
                    "tail_cap": 36, "tail_arc_cap": 40, "clique_q": 48}
    p = dupin.make_params("kclids", 5, (1, 10), clique_q=6)
    assert (p.metric, p.k_mult, p.clique_q) == (dupin.KCLIDS, 5, 6)
    assert dupin.make_params("fd").clique_q == 0

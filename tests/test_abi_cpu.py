"""CPU-side checks of the C-ABI library: it builds, loads, exports every
declared entry point, and rejects invalid arguments before touching a GPU."""

import ctypes

import pytest

import oracle
from tests._util import ensure_built, header_functions


@pytest.fixture(scope="module")
def lib():
    return ensure_built()


def test_library_exports_every_declared_function(lib):
    declared = header_functions()
    assert "nncp_create" in declared and "nncp_mttkrp" in declared
    for name in declared:
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_function(lib):
    from paper_1806_07985_gb300 import nncp
    bound = set(nncp.exported_symbols())
    missing = [n for n in header_functions() if n not in bound]
    assert not missing, missing


@pytest.mark.parametrize("dims", [(512, 512, 512), (512, 512, 32, 16), (100, 512, 32, 16),
                                  (64,) * 5, (10, 20), (3, 1, 7), (7, 300, 2, 2, 5)])
def test_default_split_matches_oracle(lib, dims):
    from paper_1806_07985_gb300 import nncp
    assert nncp.nncp_default_split(dims) == oracle.default_root_split(dims)


@pytest.mark.parametrize("N,dims,R", [(1, (5,), 3), (9, (2,) * 9, 3), (3, (4, 0, 4), 2),
                                      (3, (4, 4, 4), 0), (3, (4, 4, 4), 129)])
def test_create_rejects_invalid_shapes(lib, N, dims, R):
    arr = (ctypes.c_int64 * len(dims))(*dims)
    ctx = ctypes.c_void_p()
    status = lib.nncp_create(N, arr, R, ctypes.byref(ctx))
    assert status == 1  # NNCP_ERR_INVALID_ARG
    assert not ctx.value
    assert len(lib.nncp_global_error()) > 0


def test_null_arguments_are_rejected(lib):
    assert lib.nncp_create(3, None, 4, None) == 1
    assert lib.nncp_set_options(None, 0, 0, None) == 1
    assert lib.nncp_mttkrp(None, 1, 0, None) == 1
    assert lib.nncp_solve(None, None, None, None, 1, 0.0, None, None) == 1
    assert lib.nncp_solve_bound(None, 1, 0.0, None, None, None) == 1
    assert lib.nncp_batch_solve(0, None, None, None, None, None, None, 1, 0.0, None, None,
                                None) == 1
    assert lib.nncp_batch_run(None, 1, 0.0, None, None, None, None) == 1
    assert lib.nncp_set_leaf_fusion(None, 1) == 1
    assert lib.nncp_set_nls(None, 1) == 1
    assert lib.nncp_set_nls_iters(None, 5) == 1
    lib.nncp_destroy(None)  # no-op


def test_version_string(lib):
    assert b"nncp-gb300" in lib.nncp_version()


def test_binding_refuses_unknown_nls_name():
    from paper_1806_07985_gb300 import nncp
    with pytest.raises(ValueError):
        nncp.nncp_set_nls(None, "bogus")
    assert set(nncp.NLS) == {"hals", "bpp", "admm", "apg"}


def test_nls_codes_match_the_header():
    import re
    from paper_1806_07985_gb300 import nncp
    import pathlib
    hdr = (pathlib.Path(__file__).resolve().parents[1] / "include" / "nncp.h").read_text()
    codes = {m.group(1).lower(): int(m.group(2))
             for m in re.finditer(r"#define NNCP_NLS_(\w+)\s+(\d+)", hdr)}
    assert codes == nncp.NLS

"""Host-side checks of the C ABI library (no GPU needed, no compute calls)."""
import ctypes
import os

import numpy as np
import pytest


@pytest.fixture(scope="module")
def ps():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2004_05188_gb300 as ps

    return ps


def test_library_exports_every_declared_symbol(ps):
    names = ps.header_functions()
    assert len(names) >= 10
    L = ps.lib()
    for n in names:
        assert hasattr(L, n), n
    out = os.popen(f"nm -D --defined-only {ps.LIB_PATH}").read()
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert set(names) <= exported
    # nothing but the declared API is exported from the library's own code
    assert {e for e in exported if e.startswith("ps_")} == set(names)


def test_version_and_error_string(ps):
    assert ps.lib().ps_version() >= 100
    assert isinstance(ps.lib().ps_last_error(), bytes)


def test_edge_table_matches_oracle_byte_for_byte(ps, orc):
    for spec in [(0.0, 0.01, 2.0), (0.0, 0.02, 2.0), (0.0, 0.001, 5.0), (0.0, 0.05, 2.5), (0.3, 0.007, 1.9)]:
        r0, dr, nb = ps.bins_from_spec(*spec)
        a = ps.edges(r0, dr, nb)
        b = orc.edges(r0, dr, nb)
        assert a.tobytes() == b.tobytes(), spec


def test_edge_table_argument_errors(ps):
    E = np.empty(10, np.float32)
    L = ps.lib()
    assert L.ps_bin_edges(ps.Bins(0.0, 0.0, 5), E.ctypes.data_as(ctypes.c_void_p)) == 1
    assert L.ps_bin_edges(ps.Bins(-1.0, 0.1, 5), E.ctypes.data_as(ctypes.c_void_p)) == 1
    assert L.ps_bin_edges(ps.Bins(0.0, 0.1, 0), E.ctypes.data_as(ctypes.c_void_p)) == 6
    assert L.ps_bin_edges(ps.Bins(0.0, 0.1, 5), None) == 1
    assert b"NULL" in L.ps_last_error()


def test_binding_host_helpers(ps):
    assert ps.bins_from_spec(0.0, 0.01, 2.0) == (0.0, 0.01, 200)
    m = ps.type_mask([0, 1, 65, 255])
    assert m[0] == 3 and m[1] == 2 and m[3] == np.uint64(1) << np.uint64(63)
    assert np.all(ps.type_mask("all") == np.uint64(0xFFFFFFFFFFFFFFFF))
    with pytest.raises(ValueError):
        ps.type_mask([256])
    with pytest.raises(ValueError):
        ps.bins_from_spec(0.0, 0.0, 1.0)

"""Host-side argument checks of the C ABI (no GPU): every entry point rejects NULL handles,
out-of-range sizes and bad parameters with a status code and a message, before any CUDA call
and with nothing enqueued (the library's convention for errors found on the host)."""
import ctypes

import pytest

import paper_2004_05188_gb300 as ps

OK, INVALID_ARG, UNSUPPORTED, CAPACITY = 0, 1, 6, 7


@pytest.fixture(scope="module")
def L():
    from paper_2004_05188_gb300 import _build

    _build.build()
    return ps.lib()


def _mask(*types):
    m = (ctypes.c_uint64 * 4)()
    for t in types:
        m[t >> 6] |= 1 << (t & 63)
    return m


def _check(L, rc, code, words):
    assert rc == code
    msg = L.ps_last_error().decode()
    assert all(w in msg for w in words), msg


def test_grid_create_arguments(L):
    h = ctypes.c_void_p()
    opts = ps.GridOpts(ctypes.sizeof(ps.GridOpts), 1.0, 0, 0)
    _check(L, L.ps_grid_create(-1, ctypes.byref(opts), ctypes.byref(h)), INVALID_ARG, ["n_max"])
    _check(L, L.ps_grid_create(10, ctypes.byref(opts), None), INVALID_ARG, ["out is NULL"])
    bad = ps.GridOpts(ctypes.sizeof(ps.GridOpts), 0.3, 0, 0)
    _check(L, L.ps_grid_create(10, ctypes.byref(bad), ctypes.byref(h)), INVALID_ARG, ["cell_scale"])
    assert not h.value


def test_null_grid_everywhere(L):
    m = _mask(1)
    b = ps.Bins(0.0, 0.01, 200)
    _check(L, L.ps_grid_build(None, None, None, 0, None, 1.0, None), INVALID_ARG, ["grid is NULL"])
    _check(L, L.ps_grid_get_info(None, None, None), INVALID_ARG, ["NULL"])
    _check(L, L.ps_spatstat(None, None, m, 0.0, b, None, 0, None, None, None, None, None, None), INVALID_ARG,
           ["grid is NULL"])
    _check(L, L.ps_sdm(None, None, m, 0.0, ps.SdmSpec(), None, None, None), INVALID_ARG, ["grid is NULL"])
    _check(L, L.ps_cluster(None, None, ps.ClusterSpec(), None, None, None, None, None), INVALID_ARG,
           ["grid is NULL"])
    _check(L, L.ps_rdf_soft_fwd(None, None, m, 0.0, 0.05, 1.0, b, None, None), INVALID_ARG, ["grid is NULL"])
    _check(L, L.ps_rdf_soft_bwd(None, None, m, 0.0, 0.05, 1.0, b, None, None, None, None), INVALID_ARG,
           ["grid is NULL"])
    # NULL output histograms are refused before the grid is looked at
    _check(L, L.ps_knn_hist(None, None, m, 0.0, 1, b, None, None, None, None), INVALID_ARG, ["d_hist is NULL"])
    _check(L, L.ps_rdf_hist(None, None, m, 0.0, b, None, None, None), INVALID_ARG, ["d_hist is NULL"])
    # destroying nothing is allowed
    assert L.ps_grid_destroy(None) == OK


def test_other_entry_points(L):
    h = ctypes.c_void_p()
    _check(L, L.ps_batch_create(None, 0, None, ctypes.byref(h)), INVALID_ARG, ["ps_batch_create"])
    _check(L, L.ps_shuffle_labels(None, None, 10, 1, None, None), INVALID_ARG, ["NULL"])
    e = (ctypes.c_float * 8194)()  # room for every edge, should a check ever let the call through
    _check(L, L.ps_bin_edges(ps.Bins(0.0, 0.01, 0), e), UNSUPPORTED, ["n_bins"])
    _check(L, L.ps_bin_edges(ps.Bins(0.0, 0.01, 8193), e), UNSUPPORTED, ["n_bins"])


def test_static_entry_point_sizes(L):
    m = _mask(1)
    b = ps.Bins(0.0, 0.01, 200)
    args = (m, 2.0, m, 0.0, b, None, 0, None, None, None, None, None, None)
    _check(L, L.ps_spatstat_static(None, None, None, 262145, *args), CAPACITY, ["PS_STATIC_MAX_IONS"])
    _check(L, L.ps_spatstat_static(None, None, None, -1, *args), INVALID_ARG, ["n < 0"])


def test_static_entry_point_checks_before_any_work(L):
    """Every argument check of the allocation-free call comes before it enqueues anything (it
    shares one scratch array, which a refused call must leave untouched): these fail here, on a
    machine without a GPU, with the statistics' own messages."""
    m = _mask(1)
    meta = (ctypes.c_uint64 * 6)()
    ks = (ctypes.c_uint32 * 1)(1)
    good = ps.Bins(0.0, 0.01, 200)
    _check(L, L.ps_spatstat_static(None, None, None, 0, m, 2.0, m, 0.0, ps.Bins(0.0, 0.01, 0), None, 0, None, None,
                                   meta, None, None, None), UNSUPPORTED, ["n_bins"])
    _check(L, L.ps_spatstat_static(None, None, None, 0, m, 2.0, m, 0.0, good, None, 0, None, None, None, None, None,
                                   None), INVALID_ARG, ["ps_spatstat_static", "d_meta"])
    _check(L, L.ps_spatstat_static(None, None, None, 0, m, 1.5, m, 0.0, good, None, 0, None, None, meta, None, None,
                                   None), INVALID_ARG, ["r_cut is below the histogram stop"])
    _check(L, L.ps_spatstat_static(None, None, None, 0, m, 2.0, m, 0.0, good, ks, 1, None, None, meta, None, None,
                                   None), INVALID_ARG, ["ks/d_knn"])
    _check(L, L.ps_spatstat_static(None, None, None, 0, m, 2.0, m, float("nan"), good, None, 0, None, None, meta, None,
                                   None, None), INVALID_ARG, ["dsrf_min is NaN"])
    _check(L, L.ps_spatstat_static(None, None, None, 5, m, 2.0, m, 0.0, good, None, 0, None, None, meta, None, None,
                                   None), INVALID_ARG, ["xyz/type is NULL"])
    _check(L, L.ps_spatstat_static(None, None, None, 0, None, 2.0, m, 0.0, good, None, 0, None, None, meta, None, None,
                                   None), INVALID_ARG, ["nbr_mask is NULL"])


def test_rdf_normalise_arguments(L):
    b = ps.Bins(0.0, 0.01, 200)
    _check(L, L.ps_rdf_normalise(None, None, None, 1.0, b, None, None, None), INVALID_ARG, ["grid is NULL"])

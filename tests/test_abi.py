"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/gconn.h declares, and validates variants."""
import ctypes

import pytest

import paper_2008_11839_gb300 as g
from paper_2008_11839_gb300 import _binding as b


@pytest.fixture(scope="module")
def lib():
    g.build()
    return g.lib()


def test_exports_every_declared_symbol(lib):
    names = b.declared_symbols()
    assert len(names) >= 17
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    for s in range(7):
        assert g.gconn_status_str(s)
    assert g.gconn_status_str(0) == "ok"


def test_variant_default_and_check(lib):
    v = g.gconn_variant_default()
    assert v.link == b.GCONN_LINK_REMCAS and v.find == b.GCONN_FIND_NAIVE and v.splice == b.GCONN_SPLICE_SPLIT_ONE
    assert v.sample == b.GCONN_SAMPLE_KOUT and v.k == 2 and v.hb_n == 4
    for purpose in (0, 1, 2):   # components, forest and incremental handle all accept it
        assert g.gconn_variant_check(v, 1, purpose) == b.GCONN_OK
    assert g.gconn_variant_check(v, 1, 0) == b.GCONN_OK
    # sampling needs CSR (Section 3.3)
    assert g.gconn_variant_check(v, 0, 0) == b.GCONN_E_UNSUPPORTED


BAD = [
    dict(link="remcas", find="compress"),          # Rem-CAS has no full compression
    dict(link="async", splice="splice"),           # splicing is Rem only
    dict(link="async", find="twotrysplit"),        # two-try splitting is JTB only
    dict(link="jtb", find="split"),
    dict(link="sv", find="halve"),
]


@pytest.mark.parametrize("kw", BAD)
def test_invalid_combinations(lib, kw):
    v = g.make_variant(**kw)
    assert g.gconn_variant_check(v, 0, 0) == b.GCONN_E_UNSUPPORTED


def test_forest_needs_root_based_lt(lib):
    for name in ["CUSA", "PUSA", "PUS", "EUSA", "EUS", "CUFA", "PUFA", "PUF", "EUFA", "EUF"]:
        v = g.make_variant(link="lt", lt=name)
        assert g.gconn_variant_check(v, 0, 0) == 0
        assert g.gconn_variant_check(v, 0, 1) == b.GCONN_E_UNSUPPORTED
        assert g.gconn_variant_check(v, 0, 2) == b.GCONN_E_UNSUPPORTED
    for name in ["CRSA", "PRSA", "PRS", "CRFA", "PRFA", "PRF"]:
        assert g.gconn_variant_check(g.make_variant(link="lt", lt=name), 0, 1) == 0
    v = g.make_variant(link="lt", lt="PRF")
    v.lt_rules = b.GCONN_LT_CONNECT          # Connect without Alter is not a listed rule set
    assert g.gconn_variant_check(v, 0, 0) == b.GCONN_E_UNSUPPORTED


def test_out_of_range_fields(lib):
    v = g.make_variant()
    v.ablation = 4                            # only the two documented ablation bits exist
    assert g.gconn_variant_check(v, 0, 0) == b.GCONN_E_INVAL
    v.ablation = b.GCONN_ABL_PLAIN_SAMPLE | b.GCONN_ABL_NO_VG
    assert g.gconn_variant_check(v, 1, 0) == 0
    v = g.make_variant(block=100)
    assert g.gconn_variant_check(v, 0, 0) == b.GCONN_E_INVAL
    v = g.make_variant()
    v.link = 12
    assert g.gconn_variant_check(v, 0, 0) == b.GCONN_E_INVAL


def test_all_valid_uf_combinations_accepted(lib):
    for link in ["async", "hooks", "early"]:
        for f in ["naive", "compress", "split", "halve", "fullshortcut"]:
            assert g.gconn_variant_check(g.make_variant(link=link, find=f), 0, 1) == 0
    for f in ["naive", "split", "halve"]:
        for sp in ["none", "split_one", "halve_one", "splice"]:
            v = g.make_variant(link="remcas", find=f, splice=sp)
            assert g.gconn_variant_check(v, 0, 0) == 0
            assert g.gconn_variant_check(v, 0, 2) == 0           # incremental
            want = b.GCONN_E_UNSUPPORTED if sp in ("none", "splice") else 0
            assert g.gconn_variant_check(v, 0, 1) == want        # forest: splice is not root-based
    for f in ["naive", "twotrysplit"]:
        assert g.gconn_variant_check(g.make_variant(link="jtb", find=f), 1, 1) == 0
    for sp in ["split_one", "halve_one"]:
        assert g.gconn_variant_check(g.make_variant(link="remlock", find="halve", splice=sp), 0, 1) == 0
    assert g.gconn_variant_check(g.make_variant(link="remlock", splice="splice"), 0, 1) == b.GCONN_E_UNSUPPORTED
    for link in ["afforest", "eclcc"]:
        assert g.gconn_variant_check(g.make_variant(link=link), 0, 1) == 0
        assert g.gconn_variant_check(g.make_variant(link=link, find="halve"), 0, 0) == b.GCONN_E_UNSUPPORTED
    for link in ["lp", "stergiou"]:
        assert g.gconn_variant_check(g.make_variant(link=link), 1, 0) == 0
        assert g.gconn_variant_check(g.make_variant(link=link), 0, 1) == b.GCONN_E_UNSUPPORTED
        assert g.gconn_variant_check(g.make_variant(link=link), 0, 2) == b.GCONN_E_UNSUPPORTED


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(b, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(b, "_lib", None)
    with pytest.raises(b.GconnUnavailable):
        b.lib()


def test_argument_checks_precede_device_work(lib):
    """Malformed arguments are rejected on the host before any CUDA call, so
    these run without a GPU: counts above 2^60, the reserved n, unaligned
    edge arrays and null outputs all give E_INVAL."""
    import numpy as np
    e = np.zeros((4, 2), np.uint32)
    lab = np.zeros(10, np.uint32)
    cases = [
        lambda: g.gconn_cc(10, (1 << 60) + 1, e, lab),                     # count limit
        lambda: g.gconn_cc(0xFFFFFFFF, 0, None, lab),                      # reserved vertex count
        lambda: g.gconn_cc(10, 3, e.reshape(-1)[1:7], lab),                # edges not 8-byte aligned
        lambda: g.gconn_cc(10, 4, e, None),                                # no output
        lambda: g.gconn_spanning_forest(10, 1 << 32, e, lab, lab, None),   # forest ids above 32 bits
    ]
    for call in cases:
        with pytest.raises(g.GconnError) as ex:
            call()
        assert ex.value.status == g.GCONN_E_INVAL

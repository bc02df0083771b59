"""The C-ABI library loads and exports every symbol include/tg.h declares;
its pure host functions agree with the oracle's layout (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tg_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2010_14058_gb300 import build, tg
    build.build()
    return tg.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2010_14058_gb300 import tg
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
        assert name in tg.SIGNATURES, name
    assert set(tg.SIGNATURES) == set(names)


def test_abi_version(lib):
    from paper_2010_14058_gb300 import tg
    assert tg.tg_abi_version() == 1


@pytest.mark.parametrize("L", range(1, 9))
@pytest.mark.parametrize("k", [3, 4])
def test_layout_matches_oracle(L, k, lib):
    from paper_2010_14058_gb300 import tg
    lay = tg.tg_layout(L, k)
    assert lay["per_edge_slots"] == oracle.per_edge_slots(L, k)
    assert lay["global_slots"] == oracle.global_slots(L, k)
    assert lay["pairs"] == L * (L + 1) // 2
    assert lay["orbit_offset"][2] == L
    assert sum(lay["global_block_size"]) == lay["global_slots"]
    assert lay["graphlet_edges"] == [1, 2, 3, 3, 3, 4, 4, 5, 6]


def test_layout_rejects_bad_arguments(lib):
    from paper_2010_14058_gb300 import tg
    with pytest.raises(tg.TGError) as e:
        tg.tg_layout(9, 4)
    assert e.value.name == "TG_ERR_TOO_MANY_TYPES"
    assert tg.tg_status_string(3) in e.value.detail == tg.tg_last_error()   # thread's last failure text
    with pytest.raises(tg.TGError) as e:
        tg.tg_layout(3, 5)
    assert e.value.name == "TG_ERR_INVALID_ARG"


def test_finalize_global_divides_and_checks(lib):
    from paper_2010_14058_gb300 import tg
    L, k = 2, 4
    lay = tg.tg_layout(L, k)
    raw = np.zeros(lay["global_slots"], dtype=np.int64)
    for b in range(9):
        off, sz = lay["global_block_offset"][b], lay["global_block_size"][b]
        raw[off:off + sz] = lay["graphlet_edges"][b] * np.arange(1, sz + 1)
    out = tg.tg_finalize_global(L, k, 1, raw)
    for b in range(9):
        off, sz = lay["global_block_offset"][b], lay["global_block_size"][b]
        np.testing.assert_array_equal(out[off:off + sz], np.arange(1, sz + 1))
    raw[lay["global_block_offset"][8]] += 1
    with pytest.raises(tg.TGError) as e:
        tg.tg_finalize_global(L, k, 1, raw)
    assert e.value.name == "TG_ERR_INTERNAL"


def test_status_strings(lib):
    from paper_2010_14058_gb300 import tg
    for code in tg.STATUS:
        assert tg.tg_status_string(code) not in ("", "unknown status")


def test_missing_library_fails_loudly(tmp_path):
    from paper_2010_14058_gb300 import tg
    with pytest.raises(tg.LibraryMissing):
        tg.load(str(tmp_path / "libtg.so"))


# ------------------------------------------- position-aware host functions

@pytest.mark.parametrize("L", range(1, 9))
def test_pa_layout_matches_oracle(L, lib):
    from paper_2010_14058_gb300 import tg
    lay = tg.tg_pa_layout(L)
    assert lay["per_edge_slots"] == oracle.pa_per_edge_slots(L)
    assert lay["global_block_size"] == oracle.pa_block_sizes(L)
    assert lay["global_slots"] == sum(oracle.pa_block_sizes(L))
    assert lay["global_block_offset"] == list(np.concatenate([[0], np.cumsum(oracle.pa_block_sizes(L))[:-1]]))
    from oracle_pins import pa_offsets
    assert lay["block_offset"][1:] == list(pa_offsets(L)[:12])


@pytest.mark.parametrize("L", [1, 2, 3, 5])
def test_pa_labelling_is_each_class_smallest_member(L, lib):
    """tg_pa_labelling(b, r) lies in the oracle's class r and is its
    lexicographically smallest labelling."""
    import itertools
    from paper_2010_14058_gb300 import tg
    for b in range(9):
        K = 2 if b == 0 else (3 if b <= 2 else 4)
        first = {}
        for lab in itertools.product(range(L), repeat=K):
            first.setdefault(oracle.pa_class(L, b, lab), list(lab))
        for r in range(oracle.pa_block_sizes(L)[b]):
            assert tg.tg_pa_labelling(L, b, r) == first[r]


@pytest.mark.parametrize("L", [1, 2, 3])
def test_pa_slot_class_matches_pins(L, lib):
    """The library's slot -> class table against the test's own decoding of
    every slot and the oracle's class of the decoded labelling."""
    from oracle_pins import slot_instance
    from paper_2010_14058_gb300 import tg
    lay = tg.tg_pa_layout(L)
    for pl in range(L):
        for ph in range(L):
            assert tg.tg_pa_slot_class(L, pl, ph, lay["per_edge_slots"]) == oracle.pa_class(L, 0, (pl, ph))
            for slot in range(lay["per_edge_slots"]):
                b, lab = slot_instance(L, slot, pl, ph)
                want = lay["global_block_offset"][b] + oracle.pa_class(L, b, lab)
                assert tg.tg_pa_slot_class(L, pl, ph, slot) == want, (pl, ph, slot)


def test_pa_host_functions_reject_bad_arguments(lib):
    from paper_2010_14058_gb300 import tg
    for call in (lambda: tg.tg_pa_layout(0), lambda: tg.tg_pa_labelling(9, 0, 0),
                 lambda: tg.tg_pa_labelling(3, 9, 0), lambda: tg.tg_pa_labelling(3, 3, 45),
                 lambda: tg.tg_pa_slot_class(3, 3, 0, 0), lambda: tg.tg_pa_slot_class(3, 0, 0, 127)):
        with pytest.raises(tg.TGError):
            call()


@pytest.mark.parametrize("L", [1, 2, 3, 5, 8])
def test_directed_layout_and_class_codes_match_oracle(L, lib):
    import paper_2010_14058_gb300 as tg
    lay = tg.tg_directed_layout(L)
    assert lay["per_edge_slots"] == 8 * L
    assert lay["classes"] == oracle.directed_classes(L)
    assert lay["global_slots"] == oracle.directed_global_slots(L)
    for r in range(lay["classes"]):
        t, a = tg.tg_directed_class_code(L, r)
        assert oracle.directed_class(L, t, a) == r          # each representative is in its class
    with pytest.raises(tg.TGError):
        tg.tg_directed_class_code(L, lay["classes"])


@pytest.mark.parametrize("L,X", [(1, 1), (2, 3), (5, 4), (8, 4)])
def test_edge_typed_layout_matches_oracle(L, X, lib):
    import paper_2010_14058_gb300 as tg
    lay = tg.tg_edge_typed_layout(L, X)
    assert lay["per_edge_slots"] == oracle.edge_typed_per_edge_slots(L, X)
    assert lay["triangle_offset"] == L * X
    assert lay["global_slots"] == oracle.edge_typed_global_slots(L, X)
    assert lay["global_block_offset"] == [0, lay["global_block_size"][0], sum(lay["global_block_size"][:2])]
    with pytest.raises(tg.TGError):
        tg.tg_edge_typed_layout(L, 5)                  # more edge types than TG_MAX_EDGE_TYPES

"""CPU checks of the C ABI: the library builds for sm_103a, loads without a GPU, exports every
symbol include/fewsum.h declares, and its host-only planning calls (segment ranges, harmonic
slot layout, validation) behave as documented.  No GPU call is made here.
"""
import os
import re

import numpy as np
import pytest

from paper_2104_04582_gb300 import _build
from paper_2104_04582_gb300 import fewsum as F
from paper_2104_04582_gb300 import workloads as W

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "fewsum.h")


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return F.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(few_[a-z_]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert declared_functions() == sorted(F.EXPORTED)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_abi_version_and_strerror(lib):
    assert F.few_abi_version() == 4
    assert F.few_strerror(F.FEW_OK) == "FEW_OK"
    assert F.few_strerror(F.FEW_ERR_LIMIT) == "FEW_ERR_LIMIT"
    assert F.few_strerror(999) == "FEW_ERR_UNKNOWN"


def test_mode_slots_full_grid(lib):
    # l = 2..10, m = 0..l, n = -30..30: rows m = 10..0 and m = -10..-1, 61 slots each
    assert F.few_mode_slots(W.mode_grid(10, 30)) == (21 * 61, 21)
    # l = 2..4, n = -5..5
    assert F.few_mode_slots(W.mode_grid(4, 5)) == (9 * 11, 9)


def test_mode_slots_partner_rows_and_zero_fill(lib):
    # (2,2,3): row m=2 holds n = 3 only, its partner row m=-2 holds n = -3; rows m = 1, 0, -1
    # exist (empty) for the Horner step in z_phi
    assert F.few_mode_slots([(2, 2, 3)]) == (1 + 1, 5)
    # m = 0 only: no partner rows; one row spanning n = -2..1 (zero-filled at n = -1, 0)
    assert F.few_mode_slots([(2, 0, 1), (3, 0, -2)]) == (4, 1)
    # rows span each one's own n range: m=1 holds n = 5..7 (3 slots), m=-1 holds n = -7..-5
    assert F.few_mode_slots([(2, 1, 5), (3, 1, 7)]) == (3 + 0 + 3, 3)


@pytest.mark.parametrize("modes", [
    [(1, 0, 0)], [(2, 3, 0)], [(2, -1, 0)], [(33, 0, 0)], [(2, 0, 1025)],
    [(2, 1, 1), (2, 1, 1)]])
def test_mode_validation(lib, modes):
    with pytest.raises(F.FewError) as e:
        F.few_mode_slots(modes)
    assert e.value.status == F.FEW_ERR_MODES


def test_plan_segments_rule(lib):
    t = W.knot_times(1000.0, 7)
    seg = F.few_plan_segments(t, 0.0, 3.0, 334)
    assert seg[0] == 0 and seg[-1] == 334
    for k in range(1, len(t) - 1):
        assert seg[k] == int(np.ceil(t[k] / 3.0))
    # every sample belongs to the segment whose knot interval holds it
    ts = np.arange(334) * 3.0
    for k in range(len(t) - 1):
        s = ts[seg[k]:seg[k + 1]]
        assert np.all(s >= t[k]) and np.all(s <= t[k + 1])


def test_plan_segments_sample_on_knot(lib):
    t = np.array([0.0, 10.0, 20.0, 30.0, 40.0])
    seg = F.few_plan_segments(t, 0.0, 5.0, 9)  # samples 0,5,...,40 (last on the last knot)
    assert list(seg) == [0, 2, 4, 6, 9]


@pytest.mark.parametrize("args,status", [
    ((np.array([0.0, 1.0, 2.0]), 0.0, 0.1, 5), F.FEW_ERR_KNOTS),
    ((np.array([0.0, 1.0, 1.0, 2.0, 3.0]), 0.0, 0.1, 5), F.FEW_ERR_KNOTS),
    ((np.array([0.0, 1.0, np.nan, 2.0, 3.0]), 0.0, 0.1, 5), F.FEW_ERR_KNOTS),
    ((np.array([0.0, 1.0, 2.0, 3.0]), -0.1, 0.1, 5), F.FEW_ERR_RANGE),
    ((np.array([0.0, 1.0, 2.0, 3.0]), 0.0, 0.1, 32), F.FEW_ERR_RANGE),
    ((np.array([0.0, 1.0, 2.0, 3.0]), 0.0, 0.0, 5), F.FEW_ERR_RANGE),
    ((np.array([0.0, 1.0, 2.0, 3.0]), 0.0, -1.0, 5), F.FEW_ERR_RANGE),
])
def test_plan_segments_validation(lib, args, status):
    with pytest.raises(F.FewError) as e:
        F.few_plan_segments(*args)
    assert e.value.status == status


def test_plan_segments_edge_counts(lib):
    t = np.array([0.0, 1.0, 2.0, 3.0])
    assert list(F.few_plan_segments(t, 0.0, 0.1, 0)) == [0, 0, 0, 0]
    assert list(F.few_plan_segments(t, 3.0, 0.1, 1)) == [0, 0, 0, 1]
    assert list(F.few_plan_segments(t, 0.0, 0.1, 31)) == [0, 10, 20, 31]

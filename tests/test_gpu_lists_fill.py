"""The one-pass list construction and its fallback (Sec. 4.3.2, Definitions
1-8): lists built from capped scratch rows must equal the oracle's, and when
a row overflows, the second enumeration pass must give the same lists, the
same CSR layout and the same potentials."""
import numpy as np
import pytest

import oracle
import workloads
from test_gpu_parity import _make, canonical_pairs, check_build

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", ["c1", "grid"])
def test_row_overflow_falls_back_to_second_pass(which):
    g = workloads.starfish_c1() if which == "c1" else workloads.small_grid(3, 2, 24, 5000, seed=11)
    geo, orc = _make(g)
    assert geo.lists_check() == 1              # default capacities: one enumeration
    check_build(geo, orc)
    L1 = geo.lists()
    v1 = geo.eval("S", g["density"])

    geo.lists_check(row_cap=1)                # every row too short: second pass
    geo.build()
    assert geo.lists_check() == 2
    check_build(geo, orc)
    L2 = geo.lists()
    for name in oracle.LISTS:
        assert np.array_equal(L1[name][0], L2[name][0]), name    # same offsets
        assert np.array_equal(L1[name][1], L2[name][1]), name    # same entries in the same order
    v2 = geo.eval("S", g["density"])
    assert np.array_equal(v1, v2)

    geo.lists_check(row_cap=0)                # defaults again
    geo.build()
    assert geo.lists_check() == 1
    L3 = geo.lists()
    for name in oracle.LISTS:
        assert np.array_equal(canonical_pairs(*L1[name]), canonical_pairs(*L3[name])), name
    geo.close()

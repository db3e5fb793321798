"""Host logic of bench.py's GAS leg (no GPU): the map from a GAS context's
determinant order to the full-CI oracle's.

A context from iscsi_init_gas sorts each spin's strings by their level under
its inner/outer split (electrons outside the first `nocc` orbitals), then by
colex rank, and takes for each alpha string the prefix of beta strings whose
levels fit.  The strings are built here that way, independently of the
library, and every mapped index must name the same orbitals in the oracle.
"""
import itertools
from math import comb

import numpy as np
import pytest

import bench
from oracle import Oracle
from paper_1609_07757_gb300.synthetic import make_integrals


def _split_strings(n, ne, nocc):
    subs = [tuple(c) for c in itertools.combinations(range(n), ne)]
    colex = lambda o: sum(comb(x, i + 1) for i, x in enumerate(o))
    level = lambda o: sum(1 for x in o if x >= nocc)
    subs.sort(key=lambda o: (level(o), colex(o)))
    orbs = np.array(subs, dtype=np.int32).reshape(len(subs), ne)
    return orbs, np.array([level(o) for o in subs], dtype=np.int32)


@pytest.mark.parametrize("n,na,nb,nocc,kmax", [(7, 2, 2, 3, 1), (8, 2, 1, 4, 2), (6, 3, 2, 2, 2), (6, 2, 0, 3, 1)])
def test_index_map_names_the_same_determinants(n, na, nb, nocc, kmax):
    h1, eri = make_integrals(n, 3, ell=3.0, nchol=4)
    o = Oracle(n, na, nb, 99, 0.0, h1, eri)
    ga, la = _split_strings(n, na, nocc)
    gb, lb = _split_strings(n, nb, nocc)
    idx = bench.index_map_to_oracle(o, (ga, la, gb, lb, kmax))
    expect = []
    for a in range(len(ga)):
        for b in range(len(gb)):
            if la[a] + lb[b] <= kmax:
                expect.append(o.det_index(ga[a], gb[b]))
    assert idx.tolist() == expect
    assert len(set(expect)) == len(expect)

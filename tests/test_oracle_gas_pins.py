"""Pins of the oracle's GAS restriction (Sec. "Generalized Active Space").

The oracle keeps a determinant iff its accumulated subspace occupations lie
within the limits, and restricts its Hamiltonian to the kept set.  It is
pinned against what does not use that code:
  - the dimension of the space counted in closed form (products of binomials
    over the allowed occupation distributions);
  - the Jordan-Wigner Fock-space Hamiltonian on a determinant list enumerated
    here by brute force with the occupation test written out again;
  - the excitation-level truncation of Eq. ci_hierarchy, which is itself a
    two-subspace GAS (reference orbitals, the rest): same determinants, same
    eigenvalues as the oracle truncated at that level;
  - the CAS special case: all electrons held in the first m orbitals gives
    the full CI of the m-orbital problem.
No GPU.
"""
import itertools
from math import comb

import numpy as np
import pytest

from oracle import Oracle
from oracle import gas
from oracle import jordan_wigner as jw
from paper_1609_07757_gb300.synthetic import make_integrals


def _rand_ints(n, seed):
    rng = np.random.default_rng(seed)
    h1 = rng.standard_normal((n, n))
    h1 = 0.5 * (h1 + h1.T)
    npair = n * (n + 1) // 2
    e = rng.standard_normal((npair, npair))
    return h1, 0.5 * (e + e.T)


def _distributions(ne, sizes):
    """All (e_0, ..., e_{S-1}) with sum ne and 0 <= e_j <= sizes[j]."""
    return [d for d in itertools.product(*[range(min(ne, s) + 1) for s in sizes]) if sum(d) == ne]


def _closed_form_count(na, nb, sizes, cmin, cmax):
    tot = 0
    for da in _distributions(na, sizes):
        for db in _distributions(nb, sizes):
            acc = np.cumsum(np.add(da, db))
            if np.all(acc >= cmin) and np.all(acc <= cmax):
                w = 1
                for j, s in enumerate(sizes):
                    w *= comb(s, da[j]) * comb(s, db[j])
                tot += w
    return tot


GAS_CASES = [  # n, na, nb, sizes, cmin, cmax
    (8, 2, 2, (2, 3, 3), (0, 3, 4), (4, 4, 4)),      # at most one electron in the last subspace
    (8, 2, 2, (2, 3, 3), (0, 2, 4), (4, 4, 4)),      # at most two
    (7, 3, 1, (3, 2, 2), (2, 3, 4), (4, 4, 4)),
    (9, 2, 1, (1, 4, 4), (1, 2, 3), (2, 3, 3)),      # upper limits active too
    (6, 2, 2, (2, 2, 1, 1), (1, 2, 3, 4), (4, 4, 4, 4)),
    (6, 3, 0, (3, 3), (2, 3), (3, 3)),
    (6, 2, 2, (6,), (4,), (4,)),                      # one subspace: no restriction
]


@pytest.mark.parametrize("n,na,nb,sizes,cmin,cmax", GAS_CASES)
def test_dimension_matches_closed_form(n, na, nb, sizes, cmin, cmax):
    h1, e = _rand_ints(n, 1)
    o = Oracle(n, na, nb, 99, 0.0, h1, e)  # full CI
    keep = gas.mask(o, sizes, cmin, cmax)
    assert int(keep.sum()) == _closed_form_count(na, nb, sizes, cmin, cmax)


def _brute_force_dets(n, na, nb, kmax, sizes, cmin, cmax):
    """GAS determinants by enumeration of all orbital subsets (independent of the oracle)."""
    edges = np.cumsum((0,) + tuple(sizes))
    out = []
    for A in itertools.combinations(range(n), na):
        for B in itertools.combinations(range(n), nb):
            level = sum(1 for p in A if p >= na) + sum(1 for p in B if p >= nb)
            if level > kmax:
                continue
            ok = True
            run = 0
            for j in range(len(sizes)):
                run += sum(1 for p in A + B if edges[j] <= p < edges[j + 1])
                if run < cmin[j] or run > cmax[j]:
                    ok = False
            if ok:
                out.append((A, B))
    return out


@pytest.mark.parametrize("n,na,nb,kmax,sizes,cmin,cmax", [
    (5, 2, 2, 9, (2, 2, 1), (0, 3, 4), (4, 4, 4)),
    (5, 2, 2, 2, (2, 1, 2), (1, 3, 4), (4, 4, 4)),
    (5, 2, 1, 9, (1, 2, 2), (0, 2, 3), (1, 3, 3)),
    (4, 2, 2, 9, (1, 1, 2), (1, 2, 4), (2, 4, 4)),
])
def test_restricted_hamiltonian_matches_jordan_wigner(n, na, nb, kmax, sizes, cmin, cmax):
    h1, eri = make_integrals(n, 7 * n + na, ell=3.0, nchol=6)
    o = Oracle(n, na, nb, kmax, 0.0, h1, eri)
    keep = gas.mask(o, sizes, cmin, cmax)
    dets = _brute_force_dets(n, na, nb, kmax, sizes, cmin, cmax)
    idx = np.array([o.det_index(A, B) for A, B in dets])
    assert sorted(idx.tolist()) == np.flatnonzero(keep).tolist()
    Hj = jw.projected(h1, jw.unpack_eri(eri, n), n, dets)
    Ho = o.dense_h()[np.ix_(idx, idx)]
    assert np.abs(Ho - Hj).max() <= 1e-12 * max(1.0, np.abs(Hj).max())
    # the oracle's restricted matrix in its own order has the same spectrum
    assert np.allclose(np.linalg.eigvalsh(gas.dense(o, keep)), np.linalg.eigvalsh(Hj), atol=1e-11, rtol=0)


@pytest.mark.parametrize("n,ne,k", [(7, 2, 2), (8, 2, 3), (6, 3, 2), (6, 3, 4)])
def test_level_truncation_is_a_two_subspace_gas(n, ne, k):
    h1, eri = make_integrals(n, 11 * n + k, ell=3.0, nchol=8)
    N = 2 * ne
    full = Oracle(n, ne, ne, 99, 0.0, h1, eri)
    keep = gas.mask(full, (ne, n - ne), (N - k, N), (N, N))
    _, la = full.strings(0)
    _, lb = full.strings(1)
    off = full.offsets()
    lev = np.concatenate([la[ia] + lb[:off[ia + 1] - off[ia]] for ia in range(len(la))])
    assert np.array_equal(keep, lev <= k)
    trunc = Oracle(n, ne, ne, k, 0.0, h1, eri)
    assert int(keep.sum()) == trunc.ndet
    e_gas = np.linalg.eigvalsh(gas.dense(full, keep))
    e_trunc = np.linalg.eigvalsh(trunc.dense_h())
    assert np.abs(e_gas - e_trunc).max() <= 1e-11 * max(1.0, np.abs(e_trunc).max())


@pytest.mark.parametrize("n,m,na,nb", [(7, 4, 2, 2), (8, 5, 2, 1), (6, 4, 3, 2)])
def test_cas_limit_is_full_ci_of_the_active_orbitals(n, m, na, nb):
    h1, eri = make_integrals(n, 13 * n + m, ell=3.0, nchol=8)
    N = na + nb
    big = Oracle(n, na, nb, 99, 0.0, h1, eri)
    keep = gas.mask(big, (m, n - m), (N, N), (N, N))
    mp = m * (m + 1) // 2
    small = Oracle(m, na, nb, 99, 0.0, h1[:m, :m], eri[:mp, :mp])
    assert int(keep.sum()) == small.ndet
    e_gas = np.linalg.eigvalsh(gas.dense(big, keep))
    e_small = np.linalg.eigvalsh(small.dense_h())
    assert np.abs(e_gas - e_small).max() <= 1e-11 * max(1.0, np.abs(e_small).max())


def test_sigma_is_the_projected_product():
    n, na, nb = 8, 2, 2
    h1, eri = make_integrals(n, 5, ell=3.0, nchol=8)
    o = Oracle(n, na, nb, 3, 0.0, h1, eri)
    keep = gas.mask(o, (2, 3, 3), (0, 3, 4), (4, 4, 4))
    assert 0 < keep.sum() < o.ndet
    c = np.random.default_rng(3).standard_normal(o.ndet)
    s = gas.sigma(o, c, keep)
    assert not np.any(s[~keep])
    ref = gas.dense(o, keep) @ c[keep]
    assert np.abs(s[keep] - ref).max() <= 1e-12 * np.abs(ref).max()


def test_limits_validated():
    h1, e = _rand_ints(5, 2)
    o = Oracle(5, 2, 2, 9, 0.0, h1, e)
    with pytest.raises(ValueError):
        gas.mask(o, (2, 2), (0, 4), (4, 4))
    assert gas.mask(o, (2, 3), (0, 0), (4, 4)).all()


def test_random_specs_match_brute_force():
    """60 seeded random subspace splits and limits (2-4 subspaces, any electron
    counts, level truncations included; half of them with limits within one of
    a random determinant's accumulated counts, so that the kept set is rarely
    empty or everything): the oracle's kept set equals the brute-force
    enumeration, and its size the closed-form count at full CI."""
    rng = np.random.default_rng(2024)
    for trial in range(60):
        n = int(rng.integers(4, 8))
        na, nb = int(rng.integers(0, 4)), int(rng.integers(0, 4))
        na, nb = min(na, n), min(nb, n)
        if na + nb == 0:
            na = 1
        N = na + nb
        ns = int(rng.integers(2, 5))
        cuts = np.sort(rng.choice(np.arange(1, n), size=min(ns - 1, n - 1), replace=False))
        sizes = tuple(int(x) for x in np.diff(np.concatenate([[0], cuts, [n]])))
        cmin, cmax = [], []
        if trial % 2:
            occ = np.zeros(n, dtype=int)
            occ[rng.choice(n, size=na, replace=False)] += 1
            occ[rng.choice(n, size=nb, replace=False)] += 1
            acc = np.cumsum([occ[a:b].sum() for a, b in zip(np.cumsum((0,) + sizes[:-1]), np.cumsum(sizes))])
            for j in range(len(sizes)):
                cmin.append(max(0, int(acc[j]) - int(rng.integers(0, 2))))
                cmax.append(min(N, int(acc[j]) + int(rng.integers(0, 2))))
        else:
            for j in range(len(sizes)):
                lo, hi = sorted(int(x) for x in rng.integers(0, N + 1, size=2))
                cmin.append(lo)
                cmax.append(hi)
        cmin[-1] = min(cmin[-1], N)
        cmax[-1] = N  # the last accumulated count is N: keep the space non-trivially reachable
        kmax = int(rng.integers(0, N + 1))
        h1, e = _rand_ints(n, 1)
        o = Oracle(n, na, nb, kmax, 0.0, h1, e)
        keep = gas.mask(o, sizes, cmin, cmax)
        dets = _brute_force_dets(n, na, nb, kmax, sizes, cmin, cmax)
        idx = sorted(o.det_index(A, B) for A, B in dets)
        assert idx == np.flatnonzero(keep).tolist(), (n, na, nb, kmax, sizes, cmin, cmax)
        if kmax >= N:
            assert int(keep.sum()) == _closed_form_count(na, nb, sizes, cmin, cmax)

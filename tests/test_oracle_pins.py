"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own arithmetic: the paper's
printed table and worked sign examples, closed forms, a Jordan-Wigner
Fock-space brute force of Eq. ham, library eigen-solvers on special cases,
and invariants.  No GPU.
"""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import ALL_CLASSES, Oracle, apply_operators
from oracle import jordan_wigner as jw
from paper_1609_07757_gb300.synthetic import make_integrals


def _eri_from_full(g, n):
    npair = n * (n + 1) // 2
    e = np.zeros((npair, npair))
    for p in range(n):
        for q in range(p + 1):
            for r in range(n):
                for s in range(r + 1):
                    e[p * (p + 1) // 2 + q, r * (r + 1) // 2 + s] = g[p, q, r, s]
    return e


def _det_list(o):
    ao, _ = o.strings(0)
    bo, _ = o.strings(1)
    off = o.offsets()
    dets = []
    for ia in range(len(ao)):
        for ib in range(off[ia + 1] - off[ia]):
            dets.append((tuple(int(x) for x in ao[ia]), tuple(int(x) for x in bo[ib])))
    return dets


def _levels(o):
    ne_a, ne_b = o.na, o.nb
    return [(sum(x >= ne_a for x in A), sum(x >= ne_b for x in B)) for A, B in _det_list(o)]


def _closed_ndet(n, na, nb, k):
    tot = 0
    for a in range(na + 1):
        for b in range(nb + 1):
            if a + b <= k:
                tot += math.comb(na, a) * math.comb(n - na, a) * math.comb(nb, b) * math.comb(n - nb, b)
    return tot


# ----------------------------------------------------------------------------
# paper: Table norb (determinant counts, CISD / CISDT / CISDTQ)


def _read_table(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "table_norb.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            parts = line.split()
            rows.append([int(parts[1])] + [None if x == "-" else int(x) for x in parts[2:5]])
    return rows


def test_table_norb_counts(golden_dir):
    rows = _read_table(golden_dir)
    assert len(rows) == 15
    for n, cisd, cisdt, cisdtq in rows:
        o = Oracle(n, 2, 2, 2, 0.0, np.zeros((n, n)), None) if n <= 2698 else None
        for k, ref in ((2, cisd), (3, cisdt), (4, cisdtq)):
            if ref is None:
                continue
            if k != 2:
                o2 = Oracle(n, 2, 2, k, 0.0, np.zeros((n, n)), None)
                assert o2.ndet == ref, (n, k)
            else:
                assert o.ndet == ref, (n, k)


def test_baseline_workload_counts():
    # full CI for 2 alpha / 2 beta electrons is C(n,2)^2
    for n in (10, 60, 100):
        o = Oracle(n, 2, 2, 4, 0.0, np.zeros((n, n)), None)
        assert o.ndet == math.comb(n, 2) ** 2
    for n, k in ((50, 2), (100, 2), (50, 3), (100, 3), (120, 3)):
        o = Oracle(n, 2, 2, k, 0.0, np.zeros((n, n)), None)
        assert o.ndet == _closed_ndet(n, 2, 2, k)
    for n, na, nb, k in ((9, 3, 2, 2), (8, 4, 1, 3), (7, 1, 3, 1), (6, 0, 2, 4)):
        o = Oracle(n, na, nb, k, 0.0, np.zeros((n, n)), None)
        assert o.ndet == _closed_ndet(n, na, nb, k)


# ----------------------------------------------------------------------------
# paper: worked sign examples, Eqs. contract and add


_LABEL = {"a": 0, "b": 1, "c": 2, "d": 3}


def _parse_ops(text):
    ops = []
    for tok in text.split():
        if tok.startswith("a+_"):
            ops.append((1, _LABEL[tok[3:]]))
        elif tok.startswith("a_"):
            ops.append((0, _LABEL[tok[2:]]))
        else:
            raise ValueError(tok)
    return ops


def _state(text):
    """(sign, occupied) of a product of creators acting on the vacuum; '-(...)' negates."""
    neg = text.startswith("-(")
    if neg:
        text = text[2:-1]
    sg, occ = apply_operators(_parse_ops(text), [])
    return (-sg if neg else sg), occ


def test_paper_sign_examples(golden_dir):
    seen = 0
    with open(os.path.join(golden_dir, "paper_sign_examples.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            name, rest = line.split(None, 1)
            cols = [c.strip() for c in rest.split("  ") if c.strip()]
            op, on, sign, result = cols
            s_in, occ_in = _state(on)
            s_op, occ_out = apply_operators(_parse_ops(op), occ_in)
            s_ref, occ_ref = _state(result)
            assert occ_out == occ_ref, name
            assert s_in * s_op == int(sign) * s_ref, name
            seen += 1
    assert seen == 2


def test_sign_rule_transpositions():
    # a+_p a+_q = - a+_q a+_p and a_p a+_p + a+_p a_p = 1 on every basis state of 3 modes
    for occ in itertools.chain.from_iterable(itertools.combinations(range(3), k) for k in range(4)):
        occ = list(occ)
        for p, q in itertools.permutations(range(3), 2):
            s1, o1 = apply_operators([(1, p), (1, q)], occ)
            s2, o2 = apply_operators([(1, q), (1, p)], occ)
            assert s1 == -s2 and (s1 == 0 or o1 == o2)
        for p in range(3):
            s1, o1 = apply_operators([(0, p), (1, p)], occ)
            s2, o2 = apply_operators([(1, p), (0, p)], occ)
            assert abs(s1) + abs(s2) == 1
            assert (o1 if s1 else o2) == occ


# ----------------------------------------------------------------------------
# independent brute force: Jordan-Wigner Fock-space matrix of Eq. ham


@pytest.mark.parametrize("n,na,nb,k", [(2, 1, 1, 2), (3, 1, 1, 2), (4, 2, 2, 4), (4, 2, 2, 2), (4, 2, 2, 1),
                                       (4, 2, 1, 3), (4, 1, 2, 2), (4, 3, 2, 2), (4, 3, 1, 9), (4, 0, 2, 2),
                                       (5, 2, 2, 2)])
def test_jordan_wigner_matches_dense_h(n, na, nb, k):
    h1, eri = make_integrals(n, 11 + n + na, ell=2.5, nchol=6)
    o = Oracle(n, na, nb, k, 0.0, h1, eri)
    H = o.dense_h()
    Hj = jw.projected(h1, jw.unpack_eri(eri, n), n, _det_list(o))
    assert np.max(np.abs(H - Hj)) < 1e-12


# ----------------------------------------------------------------------------
# closed forms


def test_h2_like_closed_form():
    # 2 orbitals, 1 alpha + 1 beta, h12 = 0, (11|12) = (22|12) = 0
    h11, h22, J11, J22, J12, K = -1.3, -0.4, 0.7, 0.5, 0.45, 0.18
    h1 = np.diag([h11, h22])
    g = np.zeros((2, 2, 2, 2))
    g[0, 0, 0, 0], g[1, 1, 1, 1] = J11, J22
    g[0, 0, 1, 1] = g[1, 1, 0, 0] = J12
    for p, q, r, s in itertools.product(range(2), repeat=4):
        if (p != q) and (r != s):
            g[p, q, r, s] = K
    o = Oracle(2, 1, 1, 2, 0.0, h1, _eri_from_full(g, 2))
    w = np.linalg.eigvalsh(o.dense_h())
    A, B = 2 * h11 + J11, 2 * h22 + J22
    root = math.sqrt(0.25 * (A - B) ** 2 + K * K)
    ref = sorted([0.5 * (A + B) - root, 0.5 * (A + B) + root, h11 + h22 + J12 - K, h11 + h22 + J12 + K])
    assert np.allclose(w, ref, atol=1e-13, rtol=0)


@pytest.mark.parametrize("n,na,nb", [(6, 2, 2), (6, 3, 1), (5, 1, 0), (7, 2, 3)])
def test_no_two_electron_part_closed_form(n, na, nb):
    h1, _ = make_integrals(n, 5, ell=2.0, nchol=1)
    o = Oracle(n, na, nb, 99, 0.0, h1, None)
    w = np.linalg.eigvalsh(o.dense_h())
    eps = np.linalg.eigvalsh(h1)
    sums = sorted(sum(eps[list(a)]) + sum(eps[list(b)])
                  for a in itertools.combinations(range(n), na) for b in itertools.combinations(range(n), nb))
    assert np.allclose(w, sums, atol=1e-12, rtol=0)


@pytest.mark.parametrize("n,m,k", [(6, 2, 2), (7, 3, 4), (5, 1, 2)])
def test_reference_energy_closed_form(n, m, k):
    h1, eri = make_integrals(n, 3, ell=3.0, nchol=7)
    g = jw.unpack_eri(eri, n)
    o = Oracle(n, m, m, k, 0.0, h1, eri)
    ref = 2 * sum(h1[i, i] for i in range(m)) + sum(2 * g[i, i, j, j] - g[i, j, j, i]
                                                    for i in range(m) for j in range(m))
    assert abs(o.hij(0, 0) - ref) < 1e-13


# ----------------------------------------------------------------------------
# screening


def test_screening_hermitian_and_limits():
    n = 6
    h1, eri = make_integrals(n, 9, ell=1.5, nchol=8)
    for tau in (0.0, 1e-6, 1e-3, 2e-2, 0.1):
        H = Oracle(n, 2, 2, 4, tau, h1, eri).dense_h()
        assert np.array_equal(H, H.T)
    big = 10 * max(np.abs(h1).max(), np.abs(eri).max())
    assert not Oracle(n, 2, 2, 4, big, h1, eri).dense_h().any()


def test_screen_drops_antisymmetrised_unit_as_one():
    # two alpha electrons in two orbitals: E = h11 + h22 - A_{21,21},
    # A_{21,21} = (21|12) - (22|11) = K - J is one unit (Eq. int_share).
    J, dA = 0.5, 1e-9
    g = np.zeros((2, 2, 2, 2))
    g[0, 0, 1, 1] = g[1, 1, 0, 0] = J
    for p, q, r, s in itertools.product(range(2), repeat=4):
        if p != q and r != s:
            g[p, q, r, s] = J - dA
    h1 = np.diag([-1.0, -0.25])
    e = _eri_from_full(g, 2)
    kept = Oracle(2, 2, 0, 2, 1e-10, h1, e).hij(0, 0)
    dropped = Oracle(2, 2, 0, 2, 1e-8, h1, e).hij(0, 0)
    assert dropped == -1.25
    assert abs(kept - (-1.25 + dA)) < 1e-15


def test_screen_threshold_is_strict():
    # a unit exactly equal to tau is dropped (keep iff |u| > tau)
    h1 = np.array([[-1.0, 0.25], [0.25, -0.5]])
    H = Oracle(2, 1, 0, 1, 0.25, h1, None).dense_h()
    assert H[0, 1] == 0.0 and H[0, 0] == -1.0


# ----------------------------------------------------------------------------
# truncation, invariances


def test_truncation_nesting_and_fci():
    n = 6
    h1, eri = make_integrals(n, 21, ell=3.0, nchol=10)
    e = [np.linalg.eigvalsh(Oracle(n, 2, 2, k, 0.0, h1, eri).dense_h())[0] for k in (1, 2, 3, 4, 7)]
    assert e[0] >= e[1] - 1e-12 and e[1] >= e[2] - 1e-12 and e[2] >= e[3] - 1e-12
    assert abs(e[3] - e[4]) < 1e-12


def _permute(h1, eri, n, perm):
    g = jw.unpack_eri(eri, n)
    P = np.array(perm)
    return h1[np.ix_(P, P)], _eri_from_full(g[np.ix_(P, P, P, P)], n)


def test_orbital_permutation_invariance_fci():
    n = 6
    h1, eri = make_integrals(n, 31, ell=2.0, nchol=9)
    w0 = np.linalg.eigvalsh(Oracle(n, 2, 2, 4, 1e-3, h1, eri).dense_h())
    perm = [3, 0, 5, 1, 4, 2]
    h2, e2 = _permute(h1, eri, n, perm)
    w1 = np.linalg.eigvalsh(Oracle(n, 2, 2, 4, 1e-3, h2, e2).dense_h())
    assert np.allclose(w0, w1, atol=1e-12, rtol=0)


def test_permutation_within_o_and_v_truncated():
    n = 7
    h1, eri = make_integrals(n, 41, ell=2.0, nchol=9)
    w0 = np.linalg.eigvalsh(Oracle(n, 2, 2, 2, 0.0, h1, eri).dense_h())
    h2, e2 = _permute(h1, eri, n, [1, 0, 6, 4, 2, 5, 3])
    w1 = np.linalg.eigvalsh(Oracle(n, 2, 2, 2, 0.0, h2, e2).dense_h())
    assert np.allclose(w0, w1, atol=1e-12, rtol=0)


def test_alpha_beta_swap():
    n = 6
    h1, eri = make_integrals(n, 51, ell=2.0, nchol=9)
    for na, nb, k in ((2, 1, 2), (3, 2, 3), (2, 2, 2)):
        w0 = np.linalg.eigvalsh(Oracle(n, na, nb, k, 1e-4, h1, eri).dense_h())
        w1 = np.linalg.eigvalsh(Oracle(n, nb, na, k, 1e-4, h1, eri).dense_h())
        assert np.allclose(w0, w1, atol=1e-12, rtol=0)


# ----------------------------------------------------------------------------
# the two sigma traversals, class structure, update counts


@pytest.mark.parametrize("n,na,nb,k,tau", [(6, 2, 2, 4, 0.0), (7, 2, 2, 2, 1e-3), (7, 2, 2, 3, 1e-2),
                                           (6, 3, 2, 3, 1e-4), (6, 1, 1, 2, 0.0), (6, 2, 0, 2, 0.0)])
def test_sigma_routes_agree(n, na, nb, k, tau):
    h1, eri = make_integrals(n, 61 + n, ell=2.0, nchol=8)
    o = Oracle(n, na, nb, k, tau, h1, eri)
    c = np.random.default_rng(3).normal(size=o.ndet)
    s_terms, _ = o.sigma_terms(c)
    s_rows = o.sigma(c)
    s_dense = o.dense_h() @ c
    scale = np.abs(s_dense).max()
    assert np.max(np.abs(s_terms - s_dense)) < 1e-13 * scale
    assert np.max(np.abs(s_rows - s_dense)) < 1e-13 * scale


def _class_delta():
    """(d level alpha, d level beta) of each class, from the paper's P,H labels (Eqs. class_to_ex_dx..the_end)."""
    out = {}
    # one-body H^{P,H}_{1,0,+-1} in the order H^{1,1}, H^{1,0}, H^{0,1}, H^{0,0}: d = (1 - H) - P
    for spin in range(2):
        for i, (P, H) in enumerate([(1, 1), (1, 0), (0, 1), (0, 0)]):
            d = (1 - H) - P
            out[4 * spin + i] = (d, 0) if spin == 0 else (0, d)
    # opposite-spin terms: per spin, creator ex (in V) raises, annihilator dx (in V) lowers
    kinds = {"OO": 0, "-1": -1, "+1": 1, "VV": 0}
    terms = [("-1", "-1"), ("VV", "-1"), ("-1", "VV"), ("OO", "-1"), ("-1", "OO"), ("VV", "VV"), ("-1", "+1"),
             ("OO", "VV"), ("VV", "OO"), ("+1", "-1"), ("OO", "OO"), ("+1", "VV"), ("VV", "+1"), ("+1", "OO"),
             ("OO", "+1"), ("+1", "+1")]
    for t, (a, b) in enumerate(terms):
        out[8 + t] = (kinds[a], kinds[b])
    for spin in range(2):
        for i, (P, H) in enumerate([(2, 2), (2, 1), (1, 2), (2, 0), (1, 1), (0, 2), (1, 0), (0, 1), (0, 0)]):
            d = 2 - H - P
            out[24 + 9 * spin + i] = (d, 0) if spin == 0 else (0, d)
    return out


def test_each_class_changes_levels_as_labelled():
    n = 6
    h1, eri = make_integrals(n, 71, ell=2.0, nchol=8)
    o = Oracle(n, 2, 2, 4, 0.0, h1, eri)
    lev = _levels(o)
    delta = _class_delta()
    Hsum = np.zeros((o.ndet, o.ndet))
    for cls in range(42):
        Hc = o.dense_h(1 << cls)
        I, J = np.nonzero(Hc)
        assert len(I) > 0, cls  # every class contributes in full CI
        for i, j in zip(I, J):
            assert (lev[i][0] - lev[j][0], lev[i][1] - lev[j][1]) == delta[cls], cls
        Hsum += Hc
    assert np.max(np.abs(Hsum - o.dense_h())) < 1e-13


def test_reference_block_uses_listed_classes():
    # <0|H|0> only involves H^{0,1}_{1,0,+-1} and H^{0,2}_{2,0,-2/0/2}
    n = 6
    h1, eri = make_integrals(n, 81, ell=2.0, nchol=8)
    o = Oracle(n, 2, 2, 2, 0.0, h1, eri)
    listed = [2, 6, 18, 29, 38]
    mask = sum(1 << c for c in listed)
    assert o.hij(0, 0, mask) == o.hij(0, 0)
    for cls in range(42):
        if cls not in listed:
            assert o.hij(0, 0, 1 << cls) == 0.0


def test_triple_single_blocks_pure_excitation_classes():
    # <X_{3,0,3}|H|X_{1,0,1}> only through H^{0,0}_{2,0,2}; the adjoint only through H^{2,2}_{2,0,2}
    n = 7
    h1, eri = make_integrals(n, 91, ell=2.0, nchol=8)
    o = Oracle(n, 3, 1, 3, 0.0, h1, eri)
    lev = _levels(o)
    I = [i for i, l in enumerate(lev) if l == (3, 0)]
    J = [j for j, l in enumerate(lev) if l == (1, 0)]
    H = o.dense_h()
    Hx = o.dense_h(1 << 32)
    Hd = o.dense_h(1 << 24)
    blk = H[np.ix_(I, J)]
    assert np.abs(blk).max() > 0
    assert np.array_equal(blk, Hx[np.ix_(I, J)])
    assert np.array_equal(H[np.ix_(J, I)], Hd[np.ix_(J, I)])


def test_update_count_closed_form_fci():
    n, ne = 6, 2
    h1, eri = make_integrals(n, 101, ell=3.0, nchol=8)
    o = Oracle(n, ne, ne, 4, 0.0, h1, eri)
    c = np.ones(o.ndet)
    _, nup = o.sigma_terms(c)
    N = math.comb(n, ne)

    def one(p, q):  # strings connected by a+_p a_q
        return math.comb(n - 1, ne - 1) if p == q else math.comb(n - 2, ne - 1)

    ob = sum(one(p, q) for p in range(n) for q in range(n)) * N * 2
    ss = sum(math.comb(n - len({p, q, r, s}), ne - 2)
             for p in range(n) for r in range(p) for q in range(n) for s in range(q)) * N * 2
    os_ = sum(one(p, q) * one(r, s) for p, q, r, s in itertools.product(range(n), repeat=4))
    assert nup == ob + ss + os_


def test_string_order_and_addressing():
    n = 8
    o = Oracle(n, 3, 2, 3, 0.0, np.zeros((n, n)), None)
    for spin, ne in ((0, 3), (1, 2)):
        orbs, lev = o.strings(spin)
        assert len(orbs) == math.comb(n, ne)
        keys = [(int(l), sum(math.comb(int(x), i + 1) for i, x in enumerate(s))) for s, l in zip(orbs, lev)]
        assert keys == sorted(keys)
        assert all(int(l) == sum(int(x) >= ne for x in s) for s, l in zip(orbs, lev))
    for idx, (A, B) in enumerate(_det_list(o)):
        assert o.det_index(A, B) == idx
    # a determinant above the truncation is outside the space
    assert o.det_index([5, 6, 7], [6, 7]) == -1


@pytest.mark.parametrize("n,na,nb,k,tau", [(6, 2, 2, 4, 0.0), (8, 2, 2, 2, 1e-6), (9, 2, 2, 3, 1e-3), (7, 3, 2, 3, 1e-5),
                                           (7, 1, 1, 2, 0.0), (8, 2, 1, 9, 1e-4), (6, 2, 0, 2, 0.0), (5, 0, 3, 9, 0.0),
                                           (6, 3, 3, 2, 0.0), (8, 2, 2, 0, 0.0)])
def test_update_count_from_string_levels(n, na, nb, k, tau):
    # the count from binomials over string levels (oracle/counts.py) equals the
    # number of updates the oracle performs applying every surviving term to
    # every determinant
    from oracle.counts import updates_per_sigma
    h1, eri = make_integrals(n, 300 + n, ell=3.0, nchol=8)
    o = Oracle(n, na, nb, k, tau, h1, eri)
    _, nup = o.sigma_terms(np.ones(o.ndet))
    assert updates_per_sigma(n, na, nb, k, tau, h1, eri) == nup


# ----------------------------------------------------------------------------
# operators other than the Hamiltonian (Sec. "Second part": any one- or
# two-electron operator through the same terms with its own integrals)


@pytest.mark.parametrize("n,na,nb,k", [(4, 2, 2, 4), (4, 2, 1, 3), (5, 2, 2, 2), (4, 3, 2, 9)])
def test_nonsymmetric_one_body_operator_against_jordan_wigner(n, na, nb, k):
    # a general one-body operator sum h_pq a+_p a_q (h not symmetric): the
    # oracle's dense matrix and its term-by-term sigma against the Fock-space
    # brute force; a transposed h must give the transposed matrix
    rng = np.random.default_rng(50 + n + na + k)
    h = rng.normal(0.0, 0.5, size=(n, n))
    _, eri = make_integrals(n, 60 + n, ell=2.5, nchol=6)
    o = Oracle(n, na, nb, k, 0.0, h, eri)
    H = o.dense_h()
    Hj = jw.projected(h, jw.unpack_eri(eri, n), n, _det_list(o))
    assert np.max(np.abs(H - Hj)) < 1e-12
    assert np.max(np.abs(H - H.T)) > 1e-3  # really not symmetric
    c = np.random.default_rng(1).normal(size=o.ndet)
    assert np.max(np.abs(o.sigma_terms(c)[0] - H @ c)) < 1e-12
    Ht = Oracle(n, na, nb, k, 0.0, np.ascontiguousarray(h.T), eri).dense_h()
    assert np.max(np.abs(Ht - H.T)) < 1e-12


def _square_operator(d):
    n = d.shape[0]
    npair = n * (n + 1) // 2
    eri = np.zeros((npair, npair))
    for p in range(n):
        for q in range(p + 1):
            for r in range(n):
                for s in range(r + 1):
                    eri[p * (p + 1) // 2 + q, r * (r + 1) // 2 + s] = 2.0 * d[p, q] * d[r, s]
    return np.ascontiguousarray(d @ d), eri


@pytest.mark.parametrize("n,na,nb", [(4, 2, 2), (5, 2, 1), (5, 3, 2), (6, 2, 2)])
def test_two_body_property_operator_is_the_square(n, na, nb):
    # D^2 for D = sum d_pq E_pq as a two-body operator (Eq. ham with
    # (pq|rs) = 2 d_pq d_rs, h1 = d d) equals D applied twice on full CI,
    # and matches the Fock-space brute force
    rng = np.random.default_rng(70 + n + na)
    d = rng.normal(0.0, 0.4, size=(n, n))
    d = 0.5 * (d + d.T)
    h2, eri2 = _square_operator(d)
    kfull = na + nb
    od = Oracle(n, na, nb, kfull, 0.0, d, None)
    od2 = Oracle(n, na, nb, kfull, 0.0, h2, eri2)
    Hd, Hd2 = od.dense_h(), od2.dense_h()
    assert np.max(np.abs(Hd2 - Hd @ Hd)) < 1e-12
    c = np.random.default_rng(2).normal(size=od.ndet)
    assert np.max(np.abs(od2.sigma_terms(c)[0] - od.sigma_terms(od.sigma_terms(c)[0])[0])) < 1e-11
    Hj = jw.projected(h2, jw.unpack_eri(eri2, n), n, _det_list(od2))
    assert np.max(np.abs(Hd2 - Hj)) < 1e-12

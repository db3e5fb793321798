"""Pins of the oracle's density matrices (Sec. "Density matrices", Eqs. d1, d2).

The oracle applies the operator strings of Eqs. d1 and d2 to every
determinant.  It is pinned here against what does not depend on that code:
the Jordan-Wigner Fock-space route, closed forms for single determinants,
the energy <c|H|c> from the oracle's Slater-Condon Hamiltonian (a different
traversal), particle-number traces and the operator algebra's symmetries.
No GPU.
"""
import numpy as np
import pytest

from oracle import Oracle
from oracle import jordan_wigner as jw
from paper_1609_07757_gb300.synthetic import make_integrals


def _rand_ints(n, seed):
    rng = np.random.default_rng(seed)
    h1 = rng.standard_normal((n, n))
    h1 = 0.5 * (h1 + h1.T)
    npair = n * (n + 1) // 2
    e = rng.standard_normal((npair, npair))
    return h1, 0.5 * (e + e.T)


def _det_list(o):
    ao, _ = o.strings(0)
    bo, _ = o.strings(1)
    off = o.offsets()
    return [(tuple(int(x) for x in ao[ia]), tuple(int(x) for x in bo[ib]))
            for ia in range(len(ao)) for ib in range(off[ia + 1] - off[ia])]


@pytest.mark.parametrize("n,na,nb,k", [(3, 1, 1, 9), (4, 2, 2, 9), (4, 2, 2, 2), (4, 2, 2, 1), (4, 2, 1, 2),
                                       (4, 1, 2, 1), (3, 2, 2, 9), (4, 3, 1, 9), (4, 1, 0, 9)])
def test_density_matches_jordan_wigner(n, na, nb, k):
    h1, e = _rand_ints(n, 11)
    o = Oracle(n, na, nb, k, 0.0, h1, e)
    rng = np.random.default_rng(n * 100 + na * 10 + nb + k)
    bra = rng.standard_normal(o.ndet)
    ket = rng.standard_normal(o.ndet)
    d1, d2 = o.density(bra, ket)
    j1, j2 = jw.density(n, _det_list(o), bra, ket)
    scale = max(1.0, np.abs(j2).max())
    assert np.abs(d1 - j1).max() <= 1e-13 * scale
    assert np.abs(d2 - j2).max() <= 1e-13 * scale


@pytest.mark.parametrize("n,na,nb,k", [(6, 2, 2, 2), (5, 3, 2, 9), (6, 1, 2, 3)])
def test_single_determinant_closed_form(n, na, nb, k):
    """c = one determinant: d1 = occupations, d2 = products of occupations
    minus exchange for equal spins (Wick's theorem for a single determinant)."""
    h1, e = _rand_ints(n, 3)
    o = Oracle(n, na, nb, k, 0.0, h1, e)
    dets = _det_list(o)
    d = np.eye(n)
    for I in (0, o.ndet // 2, o.ndet - 1):
        A, B = dets[I]
        c = np.zeros(o.ndet)
        c[I] = 1.0
        d1, d2 = o.density(c)
        na_ = np.zeros(n)
        nb_ = np.zeros(n)
        na_[list(A)] = 1
        nb_[list(B)] = 1
        assert np.array_equal(d1[0], np.diag(na_))
        assert np.array_equal(d1[1], np.diag(nb_))
        for blk, (x, y) in enumerate(((na_, na_), (na_, nb_), (nb_, nb_))):
            ref = np.einsum("p,r,pq,rt->pqrt", x, y, d, d)
            if blk != 1:
                ref -= np.einsum("p,r,pt,rq->pqrt", x, y, d, d)
            assert np.array_equal(d2[blk], ref), blk


def _energy_from_density(h1, g, d1, d2):
    """<c|H|c> of Eq. ham from the spin-resolved densities."""
    return (np.einsum("pq,pq", h1, d1[0] + d1[1]) + 0.5 * np.einsum("pqrt,pqrt", g, d2[0] + d2[2])
            + np.einsum("pqrt,pqrt", g, d2[1]))


@pytest.mark.parametrize("n,na,nb,k", [(6, 2, 2, 9), (6, 2, 2, 2), (7, 2, 2, 3), (5, 3, 2, 9), (6, 2, 1, 2)])
def test_energy_from_density_equals_expectation(n, na, nb, k):
    h1, eri = make_integrals(n, seed=n * 7 + k, ell=3.0, nchol=10)
    o = Oracle(n, na, nb, k, 0.0, h1, eri)
    rng = np.random.default_rng(5)
    c = rng.standard_normal(o.ndet)
    d1, d2 = o.density(c)
    H = o.dense_h()
    e_ref = c @ H @ c
    e_dm = _energy_from_density(h1, jw.unpack_eri(eri, n), d1, d2)
    assert abs(e_dm - e_ref) <= 1e-12 * max(1.0, abs(e_ref)) * o.ndet ** 0.5
    # transition form: <bra|H|ket> from the transition densities
    ket = rng.standard_normal(o.ndet)
    t1, t2 = o.density(c, ket)
    assert abs(_energy_from_density(h1, jw.unpack_eri(eri, n), t1, t2) - c @ H @ ket) <= 1e-11 * o.ndet ** 0.5


@pytest.mark.parametrize("n,na,nb,k", [(6, 2, 2, 9), (7, 2, 2, 2), (5, 3, 2, 3), (6, 1, 1, 9)])
def test_traces_and_partial_traces(n, na, nb, k):
    h1, e = _rand_ints(n, 2)
    o = Oracle(n, na, nb, k, 0.0, h1, e)
    c = np.random.default_rng(8).standard_normal(o.ndet)
    c /= np.linalg.norm(c)
    d1, d2 = o.density(c)
    tol = 1e-12
    assert abs(np.trace(d1[0]) - na) <= tol and abs(np.trace(d1[1]) - nb) <= tol
    assert abs(np.einsum("pprr", d2[0]) - na * (na - 1)) <= tol
    assert abs(np.einsum("pprr", d2[1]) - na * nb) <= tol
    assert abs(np.einsum("pprr", d2[2]) - nb * (nb - 1)) <= tol
    # sum_r a+_p a+_r a_r a_q = a+_p a_q (N - 1); the other spin's N is a constant
    assert np.abs(np.einsum("pqrr->pq", d2[0]) - (na - 1) * d1[0]).max() <= tol
    assert np.abs(np.einsum("pqrr->pq", d2[2]) - (nb - 1) * d1[1]).max() <= tol
    assert np.abs(np.einsum("pqrr->pq", d2[1]) - nb * d1[0]).max() <= tol
    assert np.abs(np.einsum("pprt->rt", d2[1]) - na * d1[1]).max() <= tol


def test_adjoint_and_antisymmetry():
    h1, e = _rand_ints(6, 4)
    o = Oracle(6, 2, 2, 3, 0.0, h1, e)
    rng = np.random.default_rng(9)
    bra, ket = rng.standard_normal(o.ndet), rng.standard_normal(o.ndet)
    d1, d2 = o.density(bra, ket)
    e1, e2 = o.density(ket, bra)
    assert np.abs(e1 - d1.transpose(0, 2, 1)).max() <= 1e-13
    assert np.abs(e2 - d2.transpose(0, 2, 1, 4, 3)).max() <= 1e-13
    for b in (0, 2):
        assert np.abs(d2[b] + d2[b].transpose(2, 1, 0, 3)).max() <= 1e-13
        assert np.abs(d2[b] + d2[b].transpose(0, 3, 2, 1)).max() <= 1e-13


def test_single_elements_match_full():
    h1, e = _rand_ints(6, 6)
    o = Oracle(6, 2, 2, 2, 0.0, h1, e)
    rng = np.random.default_rng(10)
    bra, ket = rng.standard_normal(o.ndet), rng.standard_normal(o.ndet)
    d1, d2 = o.density(bra, ket)
    spec = np.concatenate([np.column_stack([rng.integers(0, 3, 40)] + [rng.integers(0, 6, 40) for _ in range(4)]),
                           np.column_stack([rng.integers(3, 5, 10)] + [rng.integers(0, 6, 10) for _ in range(4)])])
    got = o.density_elems(bra, ket, spec)
    ref = [d2[b, p, q, r, t] if b < 3 else d1[b - 3, p, q] for b, p, q, r, t in spec]
    assert np.abs(got - np.array(ref)).max() <= 1e-13

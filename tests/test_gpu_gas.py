"""GPU parity of GAS restrictions (Sec. "Generalized Active Space") against the oracle.

Bars: the determinant mask and the kept count are bit-exact; sigma = P H P c
within the FP64 sigma bar (1e-12 of the 2-norm and of the largest element)
with exact zeros outside the GAS space; Davidson energies within 1e-10 Eh of
the dense restricted spectrum; propagation within 1e-11 of the oracle's exact
propagator of the restricted matrices.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import Oracle
from oracle import gas
from oracle.propagate import propagate
from paper_1609_07757_gb300 import _lib as L
from paper_1609_07757_gb300.synthetic import make_integrals, unit_vector

pytestmark = pytest.mark.gpu

REL64 = 1e-12


@pytest.fixture(autouse=True)
def _fresh_library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.load()
    L.iscsi_set_option("autotune", 0)
    L.iscsi_set_option("precision", 64)
    L.iscsi_set_stream(torch.cuda.current_stream())
    yield
    torch.cuda.synchronize()
    L.iscsi_finalize()
    L.iscsi_set_option("precision", 64)
    L.iscsi_set_option("autotune", 1)


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda").contiguous()


def gpu_mask(ndet):
    m = torch.empty(ndet, dtype=torch.uint8, device="cuda")
    L.iscsi_gas_mask(m)
    torch.cuda.synchronize()
    return m.cpu().numpy().astype(bool)


def gpu_sigma(c, nvec=1):
    x = _dev(c)
    s = torch.full_like(x, float("nan"))
    L.iscsi_sigma(x, s, nvec)
    torch.cuda.synchronize()
    return s.cpu().numpy()


def assert_close(got, ref, rel=REL64):
    assert np.isfinite(got).all()
    nrm = max(np.linalg.norm(ref), 1e-300)
    assert np.linalg.norm(got - ref) <= rel * nrm
    assert np.abs(got - ref).max() <= rel * max(np.abs(ref).max(), 1e-300)


CASES = [  # n, na, nb, kmax, sizes, cmin, cmax
    (10, 2, 2, 4, (2, 3, 5), (0, 3, 4), (4, 4, 4)),          # at most one electron in the continuum
    (10, 2, 2, 3, (2, 3, 5), (0, 2, 4), (4, 4, 4)),          # at most two, CISDT
    (9, 3, 2, 3, (3, 2, 4), (2, 4, 5), (5, 5, 5)),
    (9, 2, 1, 9, (1, 4, 4), (1, 2, 3), (2, 3, 3)),           # upper limits active
    (8, 2, 2, 9, (2, 2, 2, 2), (1, 2, 3, 4), (4, 4, 4, 4)),  # four subspaces
    (8, 3, 0, 9, (3, 5), (2, 3), (3, 3)),                    # no beta electrons
    (8, 0, 2, 9, (4, 4), (1, 2), (2, 2)),                    # no alpha electrons
    (8, 2, 2, 2, (8,), (4,), (4,)),                          # one subspace: everything kept
    (8, 2, 2, 4, (4, 4), (4, 4), (4, 4)),                    # CAS(4 orbitals) inside full CI
]


@pytest.mark.parametrize("n,na,nb,k,sizes,cmin,cmax", CASES)
def test_mask_and_sigma_match_oracle(n, na, nb, k, sizes, cmin, cmax):
    h1, eri = make_integrals(n, 40 + n, ell=3.0, nchol=8)
    L.iscsi_init(n, na, nb, k, h1, eri, 0.0)
    o = Oracle(n, na, nb, k, 0.0, h1, eri)
    keep = gas.mask(o, sizes, cmin, cmax)
    kept = L.iscsi_set_gas(sizes, cmin, cmax)
    assert kept == int(keep.sum())
    assert np.array_equal(gpu_mask(o.ndet), keep)
    assert L.iscsi_stats()["gas_ndet"] == kept
    c = unit_vector(o.ndet, 7)  # components outside the GAS space too: projected on input
    s = gpu_sigma(c)
    assert not np.any(s[~keep])
    assert_close(s, gas.sigma(o, c, keep))


def test_several_vectors_host_entry_and_removal():
    n, na, nb, k = 12, 2, 2, 3
    sizes, cmin, cmax = (2, 4, 6), (0, 3, 4), (4, 4, 4)
    h1, eri = make_integrals(n, 12, ell=3.0, nchol=8)
    L.iscsi_init(n, na, nb, k, h1, eri, 0.0)
    o = Oracle(n, na, nb, k, 0.0, h1, eri)
    keep = gas.mask(o, sizes, cmin, cmax)
    L.iscsi_set_gas(sizes, cmin, cmax)
    C = np.stack([unit_vector(o.ndet, 20 + j) for j in range(3)])
    S = gpu_sigma(C, 3)
    for j in range(3):
        assert_close(S[j], gas.sigma(o, C[j], keep))
    Sh = np.zeros_like(C)
    L.iscsi_sigma_host(C, Sh, 3)
    assert np.array_equal(Sh, S)
    # removal: the whole truncated space again
    assert L.iscsi_set_gas() == o.ndet
    assert gpu_mask(o.ndet).all()
    assert_close(gpu_sigma(C[0]), o.sigma(C[0]))


def test_fp32_sigma_is_projected():
    n, na, nb, k = 10, 2, 2, 4
    sizes, cmin, cmax = (2, 3, 5), (0, 3, 4), (4, 4, 4)
    h1, eri = make_integrals(n, 3, ell=3.0, nchol=8)
    L.iscsi_init(n, na, nb, k, h1, eri, 0.0)
    o = Oracle(n, na, nb, k, 0.0, h1, eri)
    keep = gas.mask(o, sizes, cmin, cmax)
    L.iscsi_set_gas(sizes, cmin, cmax)
    c = unit_vector(o.ndet, 2)
    L.iscsi_set_option("precision", 32)
    s = gpu_sigma(c)
    L.iscsi_set_option("precision", 64)
    assert not np.any(s[~keep])
    ref = gas.sigma(o, c, keep)
    assert np.linalg.norm(s - ref) <= 2e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("n,na,nb,k,sizes,cmin,cmax,nroots", [
    (10, 2, 2, 4, (2, 3, 5), (0, 3, 4), (4, 4, 4), 3),
    (9, 3, 2, 3, (3, 2, 4), (2, 4, 5), (5, 5, 5), 2),
    (8, 2, 2, 4, (4, 4), (4, 4), (4, 4), 4),
])
def test_davidson_matches_restricted_spectrum(n, na, nb, k, sizes, cmin, cmax, nroots):
    h1, eri = make_integrals(n, 60 + n, ell=3.0, nchol=8)
    L.iscsi_init(n, na, nb, k, h1, eri, 0.0)
    o = Oracle(n, na, nb, k, 0.0, h1, eri)
    keep = gas.mask(o, sizes, cmin, cmax)
    w = np.linalg.eigvalsh(gas.dense(o, keep))
    L.iscsi_set_gas(sizes, cmin, cmax)
    vecs = torch.zeros((nroots, o.ndet), dtype=torch.float64, device="cuda")
    st, e = L.iscsi_davidson(nroots, 1e-8, vecs)
    assert st == 0
    assert np.abs(e - w[:nroots]).max() <= 1e-10
    V = vecs.cpu().numpy()
    assert not np.any(V[:, ~keep])
    # the unrestricted ground state lies lower (or equal)
    assert e[0] >= np.linalg.eigvalsh(o.dense_h())[0] - 1e-10


def test_davidson_start_vectors_are_projected_and_too_many_roots_refused():
    n, na, nb, k = 8, 2, 2, 4
    sizes, cmin, cmax = (4, 4), (4, 4), (4, 4)  # CAS(4): 36 determinants
    h1, eri = make_integrals(n, 9, ell=3.0, nchol=8)
    L.iscsi_init(n, na, nb, k, h1, eri, 0.0)
    o = Oracle(n, na, nb, k, 0.0, h1, eri)
    keep = gas.mask(o, sizes, cmin, cmax)
    kept = L.iscsi_set_gas(sizes, cmin, cmax)
    assert kept == 36
    w = np.linalg.eigvalsh(gas.dense(o, keep))
    vecs = _dev(np.stack([unit_vector(o.ndet, 30), unit_vector(o.ndet, 31)]))
    L.iscsi_set_option("guess_from_vecs", 1)
    try:
        st, e = L.iscsi_davidson(2, 1e-8, vecs)
    finally:
        L.iscsi_set_option("guess_from_vecs", 0)
    assert st == 0 and np.abs(e - w[:2]).max() <= 1e-10
    with pytest.raises(L.IscsiError):
        L.iscsi_davidson(kept + 1, 1e-8)


def test_batch_davidson_with_a_restricted_member():
    n, na, nb, k = 9, 2, 2, 4
    sizes, cmin, cmax = (2, 3, 4), (0, 3, 4), (4, 4, 4)
    h1, eri = make_integrals(n, 70, ell=3.0, nchol=8)
    L.iscsi_init(n, na, nb, k, h1, eri, 0.0)
    a = L.iscsi_ctx_current()
    L.iscsi_set_gas(sizes, cmin, cmax)
    L.iscsi_init(n, na, nb, k, h1, eri, 0.0)
    b = L.iscsi_ctx_current()
    o = Oracle(n, na, nb, k, 0.0, h1, eri)
    keep = gas.mask(o, sizes, cmin, cmax)
    wa = np.linalg.eigvalsh(gas.dense(o, keep))[:2]
    wb = np.linalg.eigvalsh(o.dense_h())[:2]
    st, e, sts = L.iscsi_batch_davidson([a, b], 2, 1e-8)
    assert st == 0 and list(sts) == [0, 0]
    assert np.abs(e[0] - wa).max() <= 1e-10
    assert np.abs(e[1] - wb).max() <= 1e-10


def test_refusals():
    n = 8
    h1, eri = make_integrals(n, 5, ell=3.0, nchol=8)
    L.iscsi_init(n, 2, 2, 4, h1, eri, 0.0)
    a = L.iscsi_ctx_current()
    ndet = L.iscsi_ndet()
    for sizes, cmin, cmax in [((4, 3), (0, 4), (4, 4)),        # sizes do not add up to n
                              ((4, 4), (3, 4), (2, 4)),        # cmin > cmax
                              ((4, 4), (0, 4), (4, 5)),        # above the electron count
                              ((0, 8), (0, 4), (4, 4)),        # empty subspace
                              ((1,) * 9, (0,) * 9, (4,) * 9)]:  # more than 8 subspaces
        with pytest.raises(L.IscsiError):
            L.iscsi_set_gas(sizes, cmin, cmax)
    assert L.iscsi_stats()["gas_subspaces"] == 0
    L.iscsi_set_gas((2, 6), (0, 3), (4, 4))
    c = _dev(unit_vector(ndet, 1))
    s = torch.empty_like(c)
    with pytest.raises(L.IscsiError):
        L.iscsi_sigma_noalloc(c, s)
    with pytest.raises(L.IscsiError):
        L.iscsi_batch_sigma([a], [c], [s])
    # every electron in the first two orbitals: the reference determinant alone
    assert L.iscsi_set_gas((2, 6), (4, 4), (4, 4)) == 1
    # an empty GAS space is allowed: sigma is zero, the Davidson method refuses
    assert L.iscsi_set_gas((2, 6), (0, 3), (4, 3)) == 0
    L.iscsi_sigma(c, s, 1)
    torch.cuda.synchronize()
    assert not torch.any(s != 0)
    with pytest.raises(L.IscsiError):
        L.iscsi_davidson(1, 1e-8)


def _restricted(H, keep):
    return H[np.ix_(keep, keep)]


@pytest.mark.parametrize("imaginary", [False, True])
def test_propagation_matches_oracle(imaginary):
    n, na, nb, k = 9, 2, 2, 3
    sizes, cmin, cmax = (2, 3, 4), (0, 3, 4), (4, 4, 4)
    h1, eri = make_integrals(n, 80, ell=3.0, nchol=8)
    v = np.diag(np.arange(n) - (n - 1) / 2.0) / n + 0.05 * (np.eye(n, k=1) + np.eye(n, k=-1))
    L.iscsi_init(n, na, nb, k, v, None, 0.0)
    hv = L.iscsi_ctx_current()
    L.iscsi_init(n, na, nb, k, h1, eri, 0.0)
    o = Oracle(n, na, nb, k, 0.0, h1, eri)
    ov = Oracle(n, na, nb, k, 0.0, v, None)
    keep = gas.mask(o, sizes, cmin, cmax)
    L.iscsi_set_gas(sizes, cmin, cmax)
    c = unit_vector(o.ndet, 5)
    nsteps, dt = 8, 0.05
    field = None if imaginary else 0.3 * np.sin(0.5 * np.arange(nsteps))
    if imaginary:
        x = _dev(c)
    else:
        x = _dev(np.stack([c, np.zeros_like(c)]))
    L.iscsi_propagate(x, nsteps, dt, field, 0 if imaginary else hv, 16, imaginary)
    torch.cuda.synchronize()
    y = x.cpu().numpy()
    got = y if imaginary else y[0] + 1j * y[1]
    Hr = _restricted(o.dense_h(), keep)
    Vr = _restricted(ov.dense_h(), keep)
    cr = c[keep]
    if imaginary:
        cr = cr / np.linalg.norm(cr)
    ref_r = propagate(Hr, None if imaginary else Vr, cr, dt, field if field is not None else np.zeros(nsteps),
                      imaginary=imaginary)
    assert not np.any(got[~keep])
    assert np.linalg.norm(got[keep] - ref_r) <= 1e-11


def test_several_tiles_continuum_restriction():
    """n = 20 full CI (36,100 determinants, several 128-row tiles): occupied 2,
    bound 6, continuum 12 orbitals, at most one electron in the continuum."""
    n, na, nb, k = 20, 2, 2, 4
    sizes, cmin, cmax = (2, 6, 12), (0, 3, 4), (4, 4, 4)
    h1, eri = make_integrals(n, 20, ell=3.0, nchol=8)
    L.iscsi_init(n, na, nb, k, h1, eri, 1e-14)
    o = Oracle(n, na, nb, k, 1e-14, h1, eri)
    keep = gas.mask(o, sizes, cmin, cmax)
    assert L.iscsi_set_gas(sizes, cmin, cmax) == int(keep.sum())
    c = unit_vector(o.ndet, 4)
    assert_close(gpu_sigma(c), gas.sigma(o, c, keep))


# ---------------------------------------------------------------------------
# contexts created on a GAS space (iscsi_init_gas): the enclosing space is a
# level truncation of another inner/outer orbital split, with its own
# determinant order; every GPU index is mapped to the full-CI oracle's index.

def gpu_to_oracle_index(o):
    """oracle index of every determinant of the current context, in its order."""
    na, nb = o.na, o.nb
    ga, la = L.iscsi_get_strings(0, na)
    gb, lb = L.iscsi_get_strings(1, nb)
    oa, _ = o.strings(0)
    ob, _ = o.strings(1)
    off = o.offsets()
    posa = {tuple(int(x) for x in r): i for i, r in enumerate(oa)}
    posb = {tuple(int(x) for x in r): i for i, r in enumerate(ob)}
    pa = np.array([posa[tuple(int(x) for x in r)] for r in ga])
    pb = np.array([posb[tuple(int(x) for x in r)] for r in gb])
    kmax = L.iscsi_stats()["max_excitation"]
    assert np.all(np.diff(lb) >= 0)  # beta strings sorted by level: allowed ones are a prefix
    parts = []
    for a in range(len(ga)):
        nba = int(np.searchsorted(lb, kmax - la[a], side="right"))
        parts.append(off[pa[a]] + pb[:nba])
    idx = np.concatenate(parts) if parts else np.zeros(0, dtype=np.int64)
    assert len(idx) == L.iscsi_ndet() and len(np.unique(idx)) == len(idx)
    return idx


def _split_dim(n, na, nb, e, k):
    from math import comb
    cnt = lambda ne, l: comb(e, ne - l) * comb(n - e, l) if 0 <= ne - l <= e else 0
    return sum(cnt(na, la) * cnt(nb, lb) for la in range(na + 1) for lb in range(nb + 1) if la + lb <= k)


SPLIT_CASES = [  # n, na, nb, sizes, cmin, cmax, expected (level split, kmax) or None for full CI
    (10, 2, 2, (2, 3, 5), (0, 3, 4), (4, 4, 4), (5, 1)),          # at most one electron in the continuum
    (10, 2, 2, (2, 3, 5), (2, 3, 4), (4, 4, 4), (2, 2)),          # and at most two out of the occupied: split there, mask
    (9, 3, 2, (4, 5), (3, 5), (5, 5), (4, 2)),
    (9, 2, 1, (3, 6), (2, 3), (3, 3), (3, 1)),
    (8, 2, 2, (2, 2, 4), (0, 0, 4), (4, 3, 4), None),            # only an upper limit restricts: full CI + mask
    (8, 3, 0, (4, 4), (2, 3), (3, 3), (4, 1)),                     # no beta electrons
    (8, 2, 2, (4, 4), (4, 4), (4, 4), (4, 0)),                     # CAS(4): every electron inner
    (8, 2, 2, (1, 7), (1, 4), (2, 4), (1, 3)),                     # fewer inner orbitals than electrons:
    (7, 3, 2, (2, 5), (3, 5), (4, 5), (2, 2)),                     # no string at level 0
]


@pytest.mark.parametrize("n,na,nb,sizes,cmin,cmax,split", SPLIT_CASES)
def test_gas_context_sigma_matches_oracle(n, na, nb, sizes, cmin, cmax, split):
    h1, eri = make_integrals(n, 90 + n, ell=3.0, nchol=8)
    L.iscsi_init_gas(n, na, nb, sizes, cmin, cmax, h1, eri, 0.0)
    st = L.iscsi_stats()
    o = Oracle(n, na, nb, 99, 0.0, h1, eri)  # full CI
    keep = gas.mask(o, sizes, cmin, cmax)
    assert st["gas_ndet"] == int(keep.sum())
    if split is None:
        assert L.iscsi_ndet() == o.ndet
    else:
        e, k = split
        assert st["level_split"] == [e, e] and st["max_excitation"] == k
        assert L.iscsi_ndet() == _split_dim(n, na, nb, e, k)
    idx = gpu_to_oracle_index(o)
    assert set(np.flatnonzero(keep)) <= set(idx.tolist())  # the GAS space lies in the enclosing one
    c_or = unit_vector(o.ndet, 11) * keep
    c_or /= np.linalg.norm(c_or)
    s = gpu_sigma(c_or[idx])
    assert_close(s, gas.sigma(o, c_or, keep)[idx])
    # the determinant mask in the context's own order
    assert np.array_equal(gpu_mask(L.iscsi_ndet()), keep[idx])


@pytest.mark.parametrize("n,na,nb,sizes,cmin,cmax,nroots", [
    (10, 2, 2, (2, 3, 5), (0, 3, 4), (4, 4, 4), 3),
    (10, 2, 2, (2, 3, 5), (2, 3, 4), (4, 4, 4), 2),
    (9, 3, 2, (4, 5), (3, 5), (5, 5), 2),
])
def test_gas_context_davidson_matches_restricted_spectrum(n, na, nb, sizes, cmin, cmax, nroots):
    h1, eri = make_integrals(n, 95 + n, ell=3.0, nchol=8)
    L.iscsi_init_gas(n, na, nb, sizes, cmin, cmax, h1, eri, 0.0)
    o = Oracle(n, na, nb, 99, 0.0, h1, eri)
    keep = gas.mask(o, sizes, cmin, cmax)
    w = np.linalg.eigvalsh(gas.dense(o, keep))
    st, e = L.iscsi_davidson(nroots, 1e-8)
    assert st == 0 and np.abs(e - w[:nroots]).max() <= 1e-10


@pytest.mark.parametrize("n,na,nb,sizes,cmin,cmax", [
    (10, 2, 2, (2, 3, 5), (0, 3, 4), (4, 4, 4)),
    (9, 3, 2, (4, 5), (3, 5), (5, 5)),
    (8, 3, 3, (5, 3), (4, 6), (6, 6)),
    (7, 3, 2, (2, 5), (3, 5), (5, 5)),  # alpha strings without a level-0 string
])
def test_gas_context_density_matches_oracle(n, na, nb, sizes, cmin, cmax):
    """The density matrices' lift tables follow the context's level split."""
    h1, eri = make_integrals(n, 97 + n, ell=3.0, nchol=8)
    L.iscsi_init_gas(n, na, nb, sizes, cmin, cmax, h1, eri, 0.0)
    o = Oracle(n, na, nb, 99, 0.0, h1, eri)
    keep = gas.mask(o, sizes, cmin, cmax)
    idx = gpu_to_oracle_index(o)
    bra = unit_vector(o.ndet, 12) * keep
    ket = unit_vector(o.ndet, 13) * keep
    r1, r2 = o.density(bra, ket)
    d1 = torch.empty((2, n, n), dtype=torch.float64, device="cuda")
    d2 = torch.empty((3, n, n, n, n), dtype=torch.float64, device="cuda")
    L.iscsi_density(_dev(bra[idx]), _dev(ket[idx]), d1, d2)
    torch.cuda.synchronize()
    for got, ref in ((d1.cpu().numpy(), r1), (d2.cpu().numpy(), r2)):
        assert np.abs(got - ref).max() <= 1e-12 * max(np.abs(ref).max(), 1e-300)


def test_gas_context_propagation_matches_oracle():
    n, na, nb = 9, 2, 2
    sizes, cmin, cmax = (2, 3, 4), (0, 3, 4), (4, 4, 4)
    h1, eri = make_integrals(n, 99, ell=3.0, nchol=8)
    L.iscsi_init_gas(n, na, nb, sizes, cmin, cmax, h1, eri, 0.0)
    o = Oracle(n, na, nb, 99, 0.0, h1, eri)
    keep = gas.mask(o, sizes, cmin, cmax)
    idx = gpu_to_oracle_index(o)
    c = unit_vector(o.ndet, 6) * keep
    c /= np.linalg.norm(c)
    x = _dev(np.stack([c[idx], np.zeros(len(idx))]))
    L.iscsi_propagate(x, 6, 0.05, None, 0, 16, False)
    torch.cuda.synchronize()
    y = x.cpu().numpy()
    got = y[0] + 1j * y[1]
    ref = propagate(gas.dense(o, keep), None, c[keep], 0.05, np.zeros(6))
    full = np.zeros(o.ndet, dtype=np.complex128)
    full[keep] = ref
    assert np.linalg.norm(got - full[idx]) <= 1e-11


def test_gas_context_refusals():
    h1, eri = make_integrals(6, 1, ell=3.0, nchol=8)
    for sizes, cmin, cmax in [((3, 2), (0, 4), (4, 4)), ((3, 3), (3, 4), (2, 4)), ((3, 3), (0, 4), (4, 5))]:
        with pytest.raises(L.IscsiError):
            L.iscsi_init_gas(6, 2, 2, sizes, cmin, cmax, h1, eri, 0.0)
    assert L.iscsi_ctx_current() == 0


def test_gas_context_full_size_continuum():
    """Full CI n = 60 restricted to at most one electron in the 40 continuum
    orbitals (2 occupied, 18 bound): the split alone gives the GAS space
    (340,100 determinants, no mask); sampled rows against the full-CI oracle."""
    n, sizes, cmin, cmax = 60, (2, 18, 40), (0, 3, 4), (4, 4, 4)
    h1, eri = make_integrals(n, 1000, ell=4.0, nchol=60)
    L.iscsi_init_gas(n, 2, 2, sizes, cmin, cmax, h1, eri, 1e-14)
    st = L.iscsi_stats()
    assert L.iscsi_ndet() == 340100 and st["gas_ndet"] == 340100 and st["gas_subspaces"] == 0
    assert st["level_split"] == [20, 20] and st["max_excitation"] == 1
    o = Oracle(n, 2, 2, 99, 1e-14, h1, eri)
    idx = gpu_to_oracle_index(o)
    c = unit_vector(len(idx), 8)
    s = gpu_sigma(c)
    c_or = np.zeros(o.ndet)
    c_or[idx] = c
    rows = np.random.default_rng(4).choice(len(idx), size=300, replace=False)
    ref = o.sigma_rows(c_or, idx[rows])
    assert np.abs(s[rows] - ref).max() <= 1e-12 * np.abs(s).max()


def test_gas_context_fp32_mixed_and_batch():
    """A GAS context (split, no mask) through the FP32 form, the FP32-mixed
    Davidson and iscsi_batch_sigma next to an ordinary context."""
    n, na, nb = 10, 2, 2
    sizes, cmin, cmax = (2, 3, 5), (0, 3, 4), (4, 4, 4)
    h1, eri = make_integrals(n, 77, ell=3.0, nchol=8)
    L.iscsi_init_gas(n, na, nb, sizes, cmin, cmax, h1, eri, 0.0)
    g = L.iscsi_ctx_current()
    assert L.iscsi_stats()["gas_subspaces"] == 0  # the split carries the restriction
    o = Oracle(n, na, nb, 99, 0.0, h1, eri)
    keep = gas.mask(o, sizes, cmin, cmax)
    idx = gpu_to_oracle_index(o)
    c_or = unit_vector(o.ndet, 14) * keep
    ref = gas.sigma(o, c_or, keep)[idx]
    # FP32 form
    L.iscsi_set_option("precision", 32)
    s32 = gpu_sigma(c_or[idx])
    L.iscsi_set_option("precision", 64)
    assert np.linalg.norm(s32 - ref) <= 2e-5 * np.linalg.norm(ref)
    # FP32-mixed Davidson
    w = np.linalg.eigvalsh(gas.dense(o, keep))[:2]
    L.iscsi_set_option("precision", 32)
    try:
        st, e = L.iscsi_davidson(2, 1e-8)
    finally:
        L.iscsi_set_option("precision", 64)
    assert st == 0 and np.abs(e - w).max() <= 1e-9
    # batched sigma with an ordinary context
    L.iscsi_init(8, 2, 2, 4, *make_integrals(8, 78, ell=3.0, nchol=8), 0.0)
    b = L.iscsi_ctx_current()
    ob = Oracle(8, 2, 2, 4, 0.0, *make_integrals(8, 78, ell=3.0, nchol=8))
    cb = unit_vector(ob.ndet, 15)
    xg, xb = _dev(c_or[idx]), _dev(cb)
    sg, sb = torch.empty_like(xg), torch.empty_like(xb)
    L.iscsi_batch_sigma([g, b], [xg, xb], [sg, sb])
    torch.cuda.synchronize()
    assert_close(sg.cpu().numpy(), ref)
    assert_close(sb.cpu().numpy(), ob.sigma(cb))


def test_gas_context_propagation_with_field():
    """Real time under H + f(t) V on a GAS context; V's context comes from
    iscsi_init_gas with the same limits (the same determinant order)."""
    n, na, nb = 9, 2, 2
    sizes, cmin, cmax = (2, 3, 4), (0, 3, 4), (4, 4, 4)
    h1, eri = make_integrals(n, 98, ell=3.0, nchol=8)
    v = np.diag(np.arange(n) - (n - 1) / 2.0) / n + 0.05 * (np.eye(n, k=1) + np.eye(n, k=-1))
    L.iscsi_init_gas(n, na, nb, sizes, cmin, cmax, v, None, 0.0)
    hv = L.iscsi_ctx_current()
    L.iscsi_init_gas(n, na, nb, sizes, cmin, cmax, h1, eri, 0.0)
    o = Oracle(n, na, nb, 99, 0.0, h1, eri)
    ov = Oracle(n, na, nb, 99, 0.0, v, None)
    keep = gas.mask(o, sizes, cmin, cmax)
    idx = gpu_to_oracle_index(o)
    c = unit_vector(o.ndet, 16) * keep
    c /= np.linalg.norm(c)
    field = 0.3 * np.sin(0.5 * np.arange(8))
    x = _dev(np.stack([c[idx], np.zeros(len(idx))]))
    L.iscsi_propagate(x, 8, 0.05, field, hv, 16, False)
    torch.cuda.synchronize()
    y = x.cpu().numpy()
    ref = propagate(gas.dense(o, keep), gas.dense(ov, keep), c[keep], 0.05, field)
    full = np.zeros(o.ndet, dtype=np.complex128)
    full[keep] = ref
    assert np.linalg.norm(y[0] + 1j * y[1] - full[idx]) <= 1e-11

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

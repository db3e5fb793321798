"""The allocation-free sigma entry point against the regular one.

iscsi_sigma_noalloc serves callers that cannot allocate device memory when
they need sigma (a memory manager owns all device memory, or the call sits in
a context where cudaMalloc is not allowed).  It keeps its scratch in a static
device array, so this test checks that it reproduces iscsi_sigma, and the CPU
oracle, within the FP64 bar of the other parity tests on two calls in a row
(the second call reuses the array left by the first), that the largest full-CI
context the array holds (2+2 electrons in 38 orbitals) is accepted and the next
one refused.  This file is collected last so that a stop at the first failure
has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import Oracle
from paper_1609_07757_gb300 import _lib as L
from paper_1609_07757_gb300.synthetic import make_integrals, unit_vector

pytestmark = pytest.mark.gpu

REL64 = 1e-12


@pytest.fixture(autouse=True)
def _fresh_library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.iscsi_set_option("class_mask_lo", 4294967295)
    L.iscsi_set_option("class_mask_hi", 1023)
    L.iscsi_set_option("precision", 64)
    L.iscsi_set_stream(torch.cuda.current_stream())
    yield
    torch.cuda.synchronize()
    L.iscsi_finalize()


@pytest.mark.parametrize("n,na,nb,k,tau", [(10, 2, 2, 4, 1e-14), (12, 2, 2, 2, 1e-8), (9, 3, 2, 3, 0.0),
                                           (8, 2, 0, 2, 0.0)])
def test_noalloc_matches_regular_sigma_twice(n, na, nb, k, tau):
    h1, eri = make_integrals(n, 900 + n, ell=3.0, nchol=10)
    L.iscsi_init(n, na, nb, k, h1, eri, tau)
    nd = L.iscsi_ndet()
    ref_s = []
    got_s = []
    for call in range(2):
        c = torch.tensor(unit_vector(nd, 40 + call), dtype=torch.float64, device="cuda")
        ref = torch.empty_like(c)
        got = torch.full_like(c, float("nan"))
        L.iscsi_sigma(c, ref, 1)
        L.iscsi_sigma_noalloc(c, got)
        torch.cuda.synchronize()
        ref_s.append(ref.cpu().numpy())
        got_s.append(got.cpu().numpy())
    o = Oracle(n, na, nb, k, tau, h1, eri)
    for call, (r, g) in enumerate(zip(ref_s, got_s)):
        assert np.all(np.isfinite(g))
        assert np.linalg.norm(g - r) <= REL64 * np.linalg.norm(r)
        assert np.abs(g - r).max() <= REL64 * np.abs(r).max()
        # and the oracle's sigma (every surviving term applied to every determinant)
        want = o.sigma_terms(unit_vector(nd, 40 + call))[0]
        assert np.linalg.norm(g - want) <= REL64 * np.linalg.norm(want)
        assert np.abs(g - want).max() <= REL64 * np.abs(want).max()


def _full_ci(n):
    h1, eri = make_integrals(n, 950, ell=3.0, nchol=4)
    L.iscsi_init(n, 2, 2, 4, h1, eri, 1e-14)
    return h1, eri


def test_noalloc_accepts_the_largest_context_the_array_holds():
    # full CI, 2+2 electrons in 38 orbitals: 2 * 38^4 doubles of lifted vector
    # and product plus the lists, just under 32 MiB
    n = 38
    h1, eri = _full_ci(n)
    nd = L.iscsi_ndet()
    c = torch.tensor(unit_vector(nd, 7), dtype=torch.float64, device="cuda")
    got = torch.full_like(c, float("nan"))
    ref = torch.empty_like(c)
    L.iscsi_sigma_noalloc(c, got)
    L.iscsi_sigma(c, ref, 1)
    torch.cuda.synchronize()
    g, r = got.cpu().numpy(), ref.cpu().numpy()
    assert np.all(np.isfinite(g))
    assert np.linalg.norm(g - r) <= REL64 * np.linalg.norm(r)
    rows = np.random.default_rng(8).choice(nd, size=150, replace=False)
    want = Oracle(n, 2, 2, 4, 1e-14, h1, eri).sigma_rows(unit_vector(nd, 7), rows)
    assert np.abs(g[rows] - want).max() <= REL64 * np.abs(r).max()


def test_noalloc_rejects_a_context_above_the_static_array():
    n = 39  # full CI: 2 * 39^4 doubles = 37 MB > 32 MiB
    _full_ci(n)
    c = torch.zeros(L.iscsi_ndet(), dtype=torch.float64, device="cuda")
    s = torch.empty_like(c)
    with pytest.raises(L.IscsiError) as e:
        L.iscsi_sigma_noalloc(c, s)
    assert e.value.status == L.ISCSI_E_ARG
    assert "static array" in str(e.value)

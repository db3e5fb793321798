"""The allocation-free sigma entry point against the regular one.

iscsi_sigma_noalloc serves callers that cannot allocate device memory when
they need sigma (a memory manager owns all device memory, or the call sits in
a context where cudaMalloc is not allowed).  It keeps its scratch in a static
device array, so this test checks that it reproduces iscsi_sigma within the
FP64 bar of the other parity tests on two calls in a row (the second call
reuses the array left by the first), and that a context too large for the
array is refused.  This file is collected last so that a stop at the first
failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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
    for r, g in zip(ref_s, got_s):
        assert np.all(np.isfinite(g))
        assert np.linalg.norm(g - r) <= REL64 * np.linalg.norm(r)
        assert np.abs(g - r).max() <= REL64 * np.abs(r).max()


def test_noalloc_rejects_a_context_above_the_static_array():
    n = 40  # full CI scratch ~ 2 * 40^4 doubles = 41 MB > 32 MiB
    h1, eri = make_integrals(n, 950, ell=3.0, nchol=4)
    L.iscsi_init(n, 2, 2, 4, h1, eri, 1e-14)
    c = torch.zeros(L.iscsi_ndet(), dtype=torch.float64, device="cuda")
    s = torch.empty_like(c)
    with pytest.raises(L.IscsiError) as e:
        L.iscsi_sigma_noalloc(c, s)
    assert e.value.status == L.ISCSI_E_ARG
    assert "static array" in str(e.value)

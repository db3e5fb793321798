"""The tensor-core kernels' bounded waits fail cleanly, without a GPU fault.

iscsi_check_bounded_wait runs one CTA whose wait (the kernels' own bounded
wait) is on a barrier that nothing arrives on.  The wait must give up after
its polls, the host must read ISCSI_E_WAIT with the wait's site, CTA and
position, the error word must be cleared, and the context must stay usable:
sigma afterwards equals sigma before, and a second check reports again.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1609_07757_gb300 import _lib as L
from paper_1609_07757_gb300.synthetic import make_integrals, unit_vector

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _fresh_library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.load()
    L.iscsi_set_option("precision", 64)
    L.iscsi_set_stream(torch.cuda.current_stream())
    yield
    torch.cuda.synchronize()
    L.iscsi_finalize()


def _sigma(c):
    s = torch.empty_like(c)
    L.iscsi_sigma(c, s, 1)
    torch.cuda.synchronize()
    return s.cpu().numpy()


def test_wait_that_runs_out_is_reported_and_cleared():
    n = 24  # large enough for the tensor-core contraction
    h1, eri = make_integrals(n, 77, ell=3.0, nchol=8)
    L.iscsi_init(n, 2, 2, 4, h1, eri, 1e-14)
    c = torch.tensor(unit_vector(L.iscsi_ndet(), 5), dtype=torch.float64, device="cuda")
    before = _sigma(c)
    for _ in range(2):  # the word is cleared: a second failure is reported again
        with pytest.raises(L.IscsiError) as e:
            L.iscsi_check_bounded_wait(1 << 14)
        assert e.value.status == L.ISCSI_E_WAIT
        msg = str(e.value)
        assert "a stage's data (MMA thread)" in msg and "CTA 0" in msg and "position 1" in msg, msg
    after = _sigma(c)
    assert np.array_equal(before, after)
    L.iscsi_davidson(1, 1e-8)  # and the synchronising calls see no stale error


def test_bounded_wait_check_arguments():
    with pytest.raises(L.IscsiError) as e:
        L.iscsi_check_bounded_wait(1 << 14)
    assert e.value.status == L.ISCSI_E_NOINIT
    h1, eri = make_integrals(6, 78)
    L.iscsi_init(6, 2, 2, 4, h1, eri, 0.0)
    for bad in (0, 1023, (1 << 24) + 1):
        with pytest.raises(L.IscsiError) as e:
            L.iscsi_check_bounded_wait(bad)
        assert e.value.status == L.ISCSI_E_ARG

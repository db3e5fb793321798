"""GPU parity at the benchmark workloads' full sizes, on sampled sigma rows.

The CUDA path computes the whole sigma = H_tau c in the launch configuration
bench.py times (one vector, FP64); the oracle computes sampled rows one by one
(row-wise Slater-Condon assembly).  Bar: |d sigma_I| <= 1e-12 ||sigma||_inf on
every sampled row, plus exact determinant counts.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import Oracle
from paper_1609_07757_gb300 import _lib as L
from paper_1609_07757_gb300.synthetic import make_integrals, unit_vector

pytestmark = pytest.mark.gpu

# name: (n, kmax, ell, nchol, box, seed, tau, expected ndet)
FULL = {
    "fci_n60_tau1e-14": (60, 4, 4.0, 60, False, 1000, 1e-14, 3132900),
    "fci_n60_tau1e-10": (60, 4, 4.0, 60, False, 1000, 1e-10, 3132900),
    "cisd_n200_box": (200, 2, 5.0, 20, True, 2000, 1e-14, 196615),
    "cisdt_n100_box": (100, 3, 5.0, 20, True, 2000, 1e-14, 1911491),
    "fci_n100_tau1e-12": (100, 4, 5.0, 20, False, 3000, 1e-12, 24502500),
}


@pytest.fixture(autouse=True)
def _fresh_library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.iscsi_set_option("precision", 64)
    L.iscsi_set_stream(torch.cuda.current_stream())
    yield
    torch.cuda.synchronize()
    L.iscsi_finalize()


@pytest.mark.parametrize("name", sorted(FULL))
def test_fullsize_sampled_rows(name):
    n, k, ell, nchol, box, seed, tau, nd = FULL[name]
    h1, eri = make_integrals(n, seed, ell=ell, nchol=nchol, box=box)
    L.iscsi_init(n, 2, 2, k, h1, eri, tau)
    assert L.iscsi_ndet() == nd
    c = unit_vector(nd, 17)
    ct = torch.tensor(c, dtype=torch.float64, device="cuda")
    st = torch.empty_like(ct)
    L.iscsi_sigma(ct, st, 1)
    torch.cuda.synchronize()
    s = st.cpu().numpy()
    L.iscsi_finalize()
    o = Oracle(n, 2, 2, k, tau, h1, eri)
    assert o.ndet == nd
    rng = np.random.default_rng(3)
    rows = np.unique(np.concatenate([[0, 1, nd // 2, nd - 1], rng.choice(nd, size=400, replace=False)]))
    ref = o.sigma_rows(c, rows)
    scale = np.abs(s).max()
    err = np.abs(s[rows] - ref).max()
    assert err <= 1e-12 * scale, (err, scale)

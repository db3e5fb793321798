"""GPU parity of the time propagation (iscsi_propagate) against the oracle.

The oracle applies the exact propagator expm(-i (H + f_k V) dt) per step
(oracle/propagate.py, pinned by closed forms).  The GPU's Lanczos propagator
with a Krylov space large enough that its truncation error (~(|H| dt)^m / m!)
is far below FP64 rounding must agree within 1e-11 (2-norm of the difference
of unit vectors after the whole run; FP64 sigma at 1e-12 relative, a few
hundred sigma calls).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import Oracle
from oracle.propagate import propagate
from paper_1609_07757_gb300 import _lib as L
from paper_1609_07757_gb300.synthetic import make_integrals, unit_vector

pytestmark = pytest.mark.gpu

TOL = 1e-11


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
    L.iscsi_set_option("autotune", 1)


def coupling_matrix(n):
    """A position-like one-body operator (a dipole along a line of orbitals)."""
    v = np.diag(np.arange(n) - (n - 1) / 2.0) / n
    return v + 0.05 * (np.eye(n, k=1) + np.eye(n, k=-1))


def make_pair(n, na, nb, k, tau=0.0, seed=3):
    """(context handle of H, handle of V, oracle H, oracle V)."""
    h1, eri = make_integrals(n, seed, ell=3.0, nchol=8)
    v = coupling_matrix(n)
    L.iscsi_init(n, na, nb, k, v, None, tau)
    hv = L.iscsi_ctx_current()
    L.iscsi_init(n, na, nb, k, h1, eri, tau)
    hh = L.iscsi_ctx_current()
    o = Oracle(n, na, nb, k, tau, h1, eri)
    ov = Oracle(n, na, nb, k, tau, v, None)
    return hh, hv, o.dense_h(), ov.dense_h(), o


def run_gpu(c, nsteps, dt, field, coupling, krylov, imaginary=False):
    if imaginary:
        x = torch.as_tensor(c, dtype=torch.float64, device="cuda").contiguous()
    else:
        x = torch.as_tensor(np.stack([c.real, c.imag]), dtype=torch.float64, device="cuda").contiguous()
    diag = L.iscsi_propagate(x, nsteps, dt, field, coupling, krylov, imaginary)
    torch.cuda.synchronize()
    y = x.cpu().numpy()
    return (y if imaginary else y[0] + 1j * y[1]), diag


@pytest.mark.parametrize("n,na,nb,k", [(8, 2, 2, 3), (10, 2, 2, 4), (7, 3, 2, 3), (6, 1, 2, 9), (7, 2, 0, 2)])
def test_real_time_with_field_matches_oracle(n, na, nb, k):
    hh, hv, H, V, o = make_pair(n, na, nb, k)
    c = unit_vector(o.ndet, 5).astype(np.complex128)
    field = 0.3 * np.sin(0.5 * np.arange(10))
    x, diag = run_gpu(c, 10, 0.02, field, hv, 16)
    ref = propagate(H, V, c, 0.02, field)
    assert np.linalg.norm(x - ref) <= TOL
    assert abs(np.linalg.norm(x) - 1.0) <= 1e-12
    assert np.all(diag[:, 0] <= 1e-12)


def test_field_free_energy_is_conserved_and_phase_of_eigenvector():
    hh, hv, H, V, o = make_pair(8, 2, 2, 4)
    w, U = np.linalg.eigh(H)
    c = U[:, 2].astype(np.complex128)
    x, diag = run_gpu(c, 8, 0.05, None, 0, 16)
    assert np.linalg.norm(x - np.exp(-1j * w[2] * 0.4) * c) <= TOL
    assert np.abs(diag[:, 1] - w[2]).max() <= 1e-11
    c2 = unit_vector(o.ndet, 9).astype(np.complex128)
    x2, diag2 = run_gpu(c2, 8, 0.05, None, 0, 16)
    assert np.linalg.norm(x2 - propagate(H, None, c2, 0.05, [0.0] * 8)) <= TOL
    assert np.ptp(diag2[:, 1]) <= 1e-11


def test_rabi_two_determinants():
    """One alpha electron in two orbitals, constant field: the closed-form Rabi population."""
    e0, e1, v, f = -1.0, -0.4, 0.3, 0.5
    L.iscsi_init(2, 1, 0, 9, np.array([[0.0, v], [v, 0.0]]), None, 0.0)
    hv = L.iscsi_ctx_current()
    L.iscsi_init(2, 1, 0, 9, np.diag([e0, e1]), None, 0.0)
    dt, nst = 0.1, 37
    x, _ = run_gpu(np.array([1.0, 0.0], dtype=np.complex128), nst, dt, np.full(nst, f), hv, 2)
    W = np.sqrt((e1 - e0) ** 2 + (2 * f * v) ** 2)
    p1 = (2 * f * v) ** 2 / W ** 2 * np.sin(W * dt * nst / 2) ** 2
    assert abs(abs(x[1]) ** 2 - p1) <= 1e-12


def test_backward_propagation_returns():
    hh, hv, H, V, o = make_pair(7, 2, 2, 2)
    c = unit_vector(o.ndet, 7).astype(np.complex128)
    field = 0.2 * np.cos(0.3 * np.arange(12))
    x, _ = run_gpu(c, 12, 0.03, field, hv, 16)
    back, _ = run_gpu(x, 12, -0.03, field[::-1].copy(), hv, 16)
    assert np.linalg.norm(back - c) <= TOL


def test_imaginary_time_matches_oracle_and_reaches_ground_state():
    """CISD in 8 orbitals (gap 0.13 Eh): 40 steps of 0.1 against the oracle, then
    imaginary time 100 (the excited admixture decays as exp(-0.13 t))."""
    hh, hv, H, V, o = make_pair(8, 2, 2, 2)
    c = unit_vector(o.ndet, 11)
    x, diag = run_gpu(c, 40, 0.1, None, 0, 16, imaginary=True)
    ref = propagate(H, None, c, 0.1, [0.0] * 40, imaginary=True)
    assert np.linalg.norm(x - ref) <= 1e-10
    x2, diag2 = run_gpu(x, 200, 0.5, None, 0, 16, imaginary=True)
    w = np.linalg.eigvalsh(H)[0]
    assert abs(x2 @ H @ x2 - w) <= 1e-10
    assert abs(diag2[-1, 1] - w) <= 1e-10


def test_argument_checks():
    hh, hv, H, V, o = make_pair(6, 2, 2, 2)
    x = torch.zeros((2, o.ndet), dtype=torch.float64, device="cuda")
    x[0, 0] = 1.0
    with pytest.raises(Exception):
        L.iscsi_propagate(x, 2, 0.1, np.zeros(2), 0, 8)  # a field without a coupling
    with pytest.raises(Exception):
        L.iscsi_propagate(x, 2, 0.1, None, 0, 1)  # Krylov dimension below 2
    with pytest.raises(Exception):
        L.iscsi_propagate(x, 2, 0.1, None, hh, 8)  # the current context as its own coupling
    L.iscsi_init(6, 2, 2, 3, coupling_matrix(6), None, 0.0)
    other = L.iscsi_ctx_current()
    L.iscsi_ctx_use(hh)
    with pytest.raises(Exception):
        L.iscsi_propagate(x, 2, 0.1, np.zeros(2), other, 8)  # coupling on another space


def test_context_is_restored_after_a_field():
    """The one-body term enters the context's string matrices only during the call."""
    hh, hv, H, V, o = make_pair(8, 2, 2, 3)
    c = torch.as_tensor(unit_vector(o.ndet, 3), dtype=torch.float64, device="cuda")
    s0 = torch.empty_like(c)
    L.iscsi_sigma(c, s0, 1)
    x = torch.zeros((2, o.ndet), dtype=torch.float64, device="cuda")
    x[0] = c
    L.iscsi_propagate(x, 3, 0.05, np.array([0.3, -0.2, 0.1]), hv, 8)
    s1 = torch.empty_like(c)
    L.iscsi_sigma(c, s1, 1)
    torch.cuda.synchronize()
    assert torch.equal(s0, s1)

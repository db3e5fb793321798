"""GPU parity for operators other than the Hamiltonian (Sec. "Second part":
any one- or two-electron operator runs through the same machinery with its own
integrals), through the C ABI against the CPU oracle.

  * a general one-body operator sum_pq h_pq a+_p a_q with h not symmetric
    (transition operators a+_p a_q among them), with and without a two-electron
    part, on the tensor-core, native FP64 and FP32 paths;
  * the adjoint relation <x|A c> = <A^T x|c> between the contexts of h and h^T;
  * a two-body property operator: D^2 for a one-body operator D, given as
    h1 = d d and (pq|rs) = 2 d_pq d_rs (Eq. ham), equals D applied twice on
    full CI (a closed form that needs no oracle) and the oracle on truncated
    spaces;
  * the eigen-solvers and the propagator refuse a non-symmetric one-body part.
Bars as in test_gpu_sigma.py: FP64 max |d sigma_I| <= 1e-12 ||sigma||_inf and
||d sigma||_2 <= 1e-12 ||sigma||_2; FP32 2e-5.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import Oracle
from paper_1609_07757_gb300 import _lib as L
from paper_1609_07757_gb300.synthetic import make_integrals, unit_vector

pytestmark = pytest.mark.gpu

REL64 = 1e-12
REL32 = 2e-5


@pytest.fixture(autouse=True)
def _fresh_library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.load()
    L.iscsi_set_option("precision", 64)
    L.iscsi_set_option("autotune", 0)
    L.iscsi_set_stream(torch.cuda.current_stream())
    yield
    torch.cuda.synchronize()
    L.iscsi_finalize()  # every context
    L.iscsi_set_option("precision", 64)
    L.iscsi_set_option("fp64_tc", 1)
    L.iscsi_set_option("autotune", 1)


def sigma(C, nvec=1, precision=64):
    L.iscsi_set_option("precision", precision)
    c = torch.as_tensor(np.ascontiguousarray(C), dtype=torch.float64, device="cuda").contiguous()
    s = torch.empty_like(c)
    L.iscsi_sigma(c, s, nvec)
    torch.cuda.synchronize()
    L.iscsi_set_option("precision", 64)
    return s.cpu().numpy()


def assert_close(s_gpu, s_ref, rel):
    nrm, inf = np.linalg.norm(s_ref), np.abs(s_ref).max()
    d = s_gpu - s_ref
    assert np.linalg.norm(d) <= rel * max(nrm, 1e-300), (np.linalg.norm(d), nrm)
    assert np.abs(d).max() <= rel * max(inf, 1e-300), (np.abs(d).max(), inf)


def nonsymmetric_h1(n, seed):
    rng = np.random.default_rng(seed)
    h = rng.normal(0.0, 0.3, size=(n, n))
    h[np.abs(h) < 0.05] = 0.0  # some exact zeros (screened at any tau)
    return np.ascontiguousarray(h)


def pair_index(n):
    P = np.zeros((n, n), dtype=np.int64)
    for p in range(n):
        for q in range(n):
            a, b = max(p, q), min(p, q)
            P[p, q] = a * (a + 1) // 2 + b
    return P


def square_operator(d):
    """(h1, eri) of D^2 for D = sum_pq d_pq E_pq (d symmetric): D^2 =
    sum (d d)_ps E_ps + (1/2) sum 2 d_pq d_rs (E_pq E_rs - delta_qr E_ps)."""
    n = d.shape[0]
    P = pair_index(n)
    npair = n * (n + 1) // 2
    eri = np.zeros((npair, npair))
    for p in range(n):
        for q in range(p + 1):
            for r in range(n):
                for s in range(r + 1):
                    eri[P[p, q], P[r, s]] = 2.0 * d[p, q] * d[r, s]
    return np.ascontiguousarray(d @ d), eri


# n, na, nb, kmax, tau, with two-electron part
NONSYM_CASES = [
    (8, 2, 2, 4, 0.0, True),     # full CI, na == nb (the beta matrix is not the alpha one)
    (9, 2, 2, 2, 1e-6, True),    # truncated
    (8, 3, 2, 5, 0.0, True),     # na != nb
    (7, 3, 3, 2, 1e-8, True),    # three electrons per spin, truncated
    (8, 2, 2, 4, 0.0, False),    # one-body only
    (9, 1, 2, 9, 0.0, False),
]


@pytest.mark.parametrize("n,na,nb,k,tau,two", NONSYM_CASES)
def test_nonsymmetric_one_body_matches_oracle(n, na, nb, k, tau, two):
    _, eri = make_integrals(n, 2100 + n, ell=3.0, nchol=8)
    h1 = nonsymmetric_h1(n, 2200 + n)
    eri = eri if two else None
    L.iscsi_init(n, na, nb, k, h1, eri, tau)
    o = Oracle(n, na, nb, k, tau, h1, eri)
    C = np.stack([unit_vector(o.ndet, 90 + v) for v in range(2)])
    refs = [o.sigma_terms(C[v]) for v in range(2)]
    for tc in (1, 0):
        L.iscsi_set_option("fp64_tc", tc)
        s = sigma(C, nvec=2).reshape(2, -1)
        for v in range(2):
            assert_close(s[v], refs[v][0], REL64)
    L.iscsi_set_option("fp64_tc", 1)
    s32 = sigma(C, nvec=2, precision=32).reshape(2, -1)
    for v in range(2):
        assert np.linalg.norm(s32[v] - refs[v][0]) <= REL32 * np.linalg.norm(refs[v][0])
    assert L.iscsi_updates_per_sigma() == refs[0][1]


@pytest.mark.parametrize("n,na,nb,k", [(8, 2, 2, 4), (9, 3, 2, 3)])
def test_transition_operator_and_its_adjoint(n, na, nb, k):
    """A = a+_p a_q (both spins): h = e_p e_q^T, no two-electron part.  sigma
    against the oracle, and <x|A c> = <A^T x|c> with A^T = a+_q a_p from its
    own context."""
    p, q = n - 1, 0  # a virtual orbital from an occupied one
    h = np.zeros((n, n))
    h[p, q] = 1.0
    L.iscsi_init(n, na, nb, k, h, None, 0.0)
    a = L.iscsi_ctx_current()
    L.iscsi_init(n, na, nb, k, np.ascontiguousarray(h.T), None, 0.0)
    at = L.iscsi_ctx_current()
    o = Oracle(n, na, nb, k, 0.0, h, None)
    c = unit_vector(o.ndet, 11)
    x = unit_vector(o.ndet, 12)
    L.iscsi_ctx_use(a)
    ac = sigma(c)
    assert_close(ac, o.sigma_terms(c)[0], REL64)
    assert np.abs(ac).max() > 0.0
    L.iscsi_ctx_use(at)
    atx = sigma(x)
    lhs, rhs = float(x @ ac), float(atx @ c)
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs)), (lhs, rhs)


@pytest.mark.parametrize("n,na,nb", [(7, 2, 2), (8, 3, 2), (7, 3, 3)])
def test_two_body_property_operator_is_d_squared_on_full_ci(n, na, nb):
    rng = np.random.default_rng(300 + n + na)
    d = rng.normal(0.0, 0.4, size=(n, n))
    d = np.ascontiguousarray(0.5 * (d + d.T))
    h2, eri2 = square_operator(d)
    kfull = na + nb
    L.iscsi_init(n, na, nb, kfull, d, None, 0.0)
    hd = L.iscsi_ctx_current()
    L.iscsi_init(n, na, nb, kfull, h2, eri2, 0.0)
    hd2 = L.iscsi_ctx_current()
    nd = L.iscsi_ndet()
    c = unit_vector(nd, 21)
    s2 = sigma(c)
    L.iscsi_ctx_use(hd)
    twice = sigma(sigma(c))
    assert_close(s2, twice, REL64)
    o = Oracle(n, na, nb, kfull, 0.0, h2, eri2)
    assert_close(s2, o.sigma_terms(c)[0], REL64)
    L.iscsi_ctx_use(hd2)


@pytest.mark.parametrize("n,na,nb,k,tau", [(9, 2, 2, 2, 0.0), (8, 3, 2, 3, 1e-10)])
def test_two_body_property_operator_truncated_matches_oracle(n, na, nb, k, tau):
    rng = np.random.default_rng(400 + n)
    d = rng.normal(0.0, 0.4, size=(n, n))
    d = np.ascontiguousarray(0.5 * (d + d.T))
    h2, eri2 = square_operator(d)
    L.iscsi_init(n, na, nb, k, h2, eri2, tau)
    o = Oracle(n, na, nb, k, tau, h2, eri2)
    c = unit_vector(o.ndet, 23)
    ref, nup = o.sigma_terms(c)
    assert_close(sigma(c), ref, REL64)
    assert L.iscsi_updates_per_sigma() == nup


def test_solvers_refuse_a_nonsymmetric_one_body_part():
    n = 6
    L.iscsi_init(n, 2, 2, 4, nonsymmetric_h1(n, 7), None, 0.0)
    with pytest.raises(L.IscsiError) as e:
        L.iscsi_davidson(1, 1e-8)
    assert e.value.status == L.ISCSI_E_ARG
    c = torch.tensor(np.stack([unit_vector(L.iscsi_ndet(), 3), np.zeros(L.iscsi_ndet())]), device="cuda")
    with pytest.raises(L.IscsiError) as e:
        L.iscsi_propagate(c, 1, 0.01)
    assert e.value.status == L.ISCSI_E_ARG

"""GPU parity: the CUDA sigma path (through the C ABI) against the CPU oracle.

Bars (from the method and the FP64 arithmetic):
  * strings, levels, determinant count and addressing: bit-exact;
  * update counts: exact integers;
  * FP64 sigma: ||d sigma||_2 <= 1e-12 ||sigma||_2 and max|d sigma_I| <= 1e-12 ||sigma||_inf;
  * FP32 sigma: ||d sigma||_2 <= 2e-5 ||sigma||_2 (FP32 products and sums);
  * energies: |dE| <= 1e-10 Eh (FP64), <= 1e-9 Eh after FP64 refinement (mixed).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ALL_CLASSES, Oracle
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
    L.iscsi_set_option("class_mask_lo", 4294967295)
    L.iscsi_set_option("class_mask_hi", 1023)
    L.iscsi_set_option("precision", 64)
    L.iscsi_set_option("fp32_tc", 1)
    # the parity tests below exercise the default routing; the autotuner has its own test
    L.iscsi_set_option("autotune", 0)
    L.iscsi_set_stream(torch.cuda.current_stream())
    yield
    torch.cuda.synchronize()
    L.iscsi_finalize()
    L.iscsi_set_option("class_mask_lo", 4294967295)
    L.iscsi_set_option("class_mask_hi", 1023)
    L.iscsi_set_option("precision", 64)
    L.iscsi_set_option("fp32_tc", 1)
    L.iscsi_set_option("autotune", 1)


def gpu_sigma(C, nvec=1, precision=64):
    L.iscsi_set_option("precision", precision)
    c = torch.as_tensor(np.ascontiguousarray(C), dtype=torch.float64, device="cuda").contiguous()
    s = torch.empty_like(c)
    L.iscsi_sigma(c, s, nvec)
    torch.cuda.synchronize()
    L.iscsi_set_option("precision", 64)
    return s.cpu().numpy()


def assert_close(s_gpu, s_ref, rel):
    """The FP64 bar: ||d||_2 <= rel ||s||_2 and max |d_I| <= rel ||s||_inf."""
    nrm = np.linalg.norm(s_ref)
    inf = np.abs(s_ref).max()
    d = s_gpu - s_ref
    assert np.linalg.norm(d) <= rel * max(nrm, 1e-300), (np.linalg.norm(d), nrm)
    assert np.abs(d).max() <= rel * max(inf, 1e-300), (np.abs(d).max(), inf)


CASES = [  # n, na, nb, kmax, tau
    (6, 2, 2, 4, 0.0),
    (10, 2, 2, 4, 0.0),
    (10, 2, 2, 4, 1e-14),
    (9, 2, 2, 2, 1e-3),
    (11, 2, 2, 3, 1e-6),
    (7, 1, 1, 2, 0.0),
    (7, 3, 2, 3, 1e-5),
    (6, 3, 3, 2, 0.0),
    (8, 2, 1, 9, 1e-4),
    (6, 2, 0, 2, 0.0),
    (5, 0, 3, 9, 0.0),
    (2, 1, 1, 2, 0.0),
    (8, 2, 2, 0, 0.0),
    (13, 2, 2, 1, 1e-8),
]


@pytest.mark.parametrize("n,na,nb,k,tau", CASES)
def test_strings_and_addressing_bit_exact(n, na, nb, k, tau):
    h1, eri = make_integrals(n, 100 + n, ell=3.0, nchol=8)
    L.iscsi_init(n, na, nb, k, h1, eri, tau)
    o = Oracle(n, na, nb, k, tau, h1, eri)
    assert L.iscsi_ndet() == o.ndet
    for spin, ne in ((0, na), (1, nb)):
        g_orbs, g_lev = L.iscsi_get_strings(spin, ne)
        o_orbs, o_lev = o.strings(spin)
        assert np.array_equal(g_lev, o_lev)
        if ne:
            assert np.array_equal(g_orbs, o_orbs)
    ao, _ = o.strings(0)
    bo, _ = o.strings(1)
    rng = np.random.default_rng(0)
    for _ in range(40):
        A = ao[rng.integers(len(ao))]
        B = bo[rng.integers(len(bo))]
        assert L.iscsi_det_index(list(A), list(B)) == o.det_index(list(A), list(B))


@pytest.mark.parametrize("n,na,nb,k,tau", CASES)
def test_sigma_fp64_matches_oracle(n, na, nb, k, tau):
    h1, eri = make_integrals(n, 200 + n, ell=2.5, nchol=8)
    L.iscsi_init(n, na, nb, k, h1, eri, tau)
    o = Oracle(n, na, nb, k, tau, h1, eri)
    c = unit_vector(o.ndet, 7)
    s_ref, nup = o.sigma_terms(c)
    assert_close(gpu_sigma(c), s_ref, REL64)
    assert L.iscsi_updates_per_sigma() == nup


def test_sigma_without_two_electron_integrals():
    n = 8
    h1, _ = make_integrals(n, 5)
    L.iscsi_init(n, 2, 2, 3, h1, None, 0.0)
    o = Oracle(n, 2, 2, 3, 0.0, h1, None)
    c = unit_vector(o.ndet, 3)
    assert_close(gpu_sigma(c), o.sigma_terms(c)[0], REL64)


@pytest.mark.parametrize("cls", range(42))
def test_each_of_the_42_classes(cls):
    n, na, nb, k, tau = 7, 2, 2, 4, 1e-9
    h1, eri = make_integrals(n, 300, ell=2.0, nchol=8)
    mask = 1 << cls
    L.iscsi_set_option("class_mask_lo", mask & 0xFFFFFFFF)
    L.iscsi_set_option("class_mask_hi", mask >> 32)
    L.iscsi_init(n, na, nb, k, h1, eri, tau)
    o = Oracle(n, na, nb, k, tau, h1, eri)
    c = unit_vector(o.ndet, 11 + cls)
    s_ref, nup = o.sigma_terms(c, mask)
    assert np.abs(s_ref).max() > 0
    assert_close(gpu_sigma(c), s_ref, REL64)
    assert L.iscsi_updates_per_sigma() == nup


@pytest.mark.parametrize("cls_set", [(9, 14, 27), (0, 5, 24, 33, 18), tuple(range(8, 24))])
def test_class_subsets_truncated(cls_set):
    n, na, nb, k, tau = 8, 2, 2, 2, 1e-7
    h1, eri = make_integrals(n, 301, ell=2.0, nchol=8)
    mask = sum(1 << c for c in cls_set)
    L.iscsi_set_option("class_mask_lo", mask & 0xFFFFFFFF)
    L.iscsi_set_option("class_mask_hi", mask >> 32)
    L.iscsi_init(n, na, nb, k, h1, eri, tau)
    o = Oracle(n, na, nb, k, tau, h1, eri)
    c = unit_vector(o.ndet, 5)
    s_ref, nup = o.sigma_terms(c, mask)
    assert_close(gpu_sigma(c), s_ref, REL64)
    assert L.iscsi_updates_per_sigma() == nup


def test_multiple_vectors_and_fp32():
    n, na, nb, k, tau = 10, 2, 2, 3, 1e-12
    h1, eri = make_integrals(n, 400, ell=3.0, nchol=10)
    L.iscsi_init(n, na, nb, k, h1, eri, tau)
    o = Oracle(n, na, nb, k, tau, h1, eri)
    C = np.stack([unit_vector(o.ndet, 20 + v) for v in range(3)])
    S64 = gpu_sigma(C, nvec=3).reshape(3, -1)
    S32 = gpu_sigma(C, nvec=3, precision=32).reshape(3, -1)
    for v in range(3):
        ref = o.sigma_terms(C[v])[0]
        assert_close(S64[v], ref, REL64)
        assert np.linalg.norm(S32[v] - ref) <= REL32 * np.linalg.norm(ref)


def test_diagonal_matches_oracle():
    n, na, nb, k, tau = 8, 2, 2, 3, 1e-6
    h1, eri = make_integrals(n, 500, ell=2.0, nchol=8)
    L.iscsi_init(n, na, nb, k, h1, eri, tau)
    o = Oracle(n, na, nb, k, tau, h1, eri)
    d = torch.empty(o.ndet, dtype=torch.float64, device="cuda")
    L.iscsi_diagonal(d)
    torch.cuda.synchronize()
    ref = np.diag(o.dense_h())
    assert np.abs(d.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


def test_screen_everything_gives_zero_and_sigma_host():
    n = 6
    h1, eri = make_integrals(n, 600)
    big = 10 * max(np.abs(h1).max(), np.abs(eri).max())
    L.iscsi_init(n, 2, 2, 4, h1, eri, big)
    c = unit_vector(L.iscsi_ndet(), 1)
    s = np.empty_like(c)
    L.iscsi_sigma_host(c, s, 1)
    assert not s.any()
    assert L.iscsi_updates_per_sigma() == 0


def test_sigma_host_matches_device_path():
    n = 9
    h1, eri = make_integrals(n, 650, ell=3.0, nchol=9)
    L.iscsi_init(n, 2, 2, 4, h1, eri, 1e-14)
    c = np.stack([unit_vector(L.iscsi_ndet(), 30 + v) for v in range(2)])
    s = np.empty_like(c)
    L.iscsi_sigma_host(c, s, 2)
    assert np.array_equal(s, gpu_sigma(c, nvec=2).reshape(2, -1))


def test_davidson_fp64_and_mixed_match_dense_eigenvalues():
    n, tau = 10, 1e-14
    h1, eri = make_integrals(n, 0, ell=3.0, nchol=20)
    o = Oracle(n, 2, 2, 4, tau, h1, eri)
    w = np.linalg.eigvalsh(o.dense_h())
    L.iscsi_init(n, 2, 2, 4, h1, eri, tau)
    vecs = torch.zeros((3, o.ndet), dtype=torch.float64, device="cuda")
    st, e = L.iscsi_davidson(3, 1e-8, vecs)
    assert st == 0
    assert np.abs(e - w[:3]).max() <= 1e-10
    # eigenvectors: residual of the oracle operator is small
    V = vecs.cpu().numpy()
    for j in range(3):
        r = o.sigma_terms(V[j])[0] - e[j] * V[j]
        assert np.linalg.norm(r) < 1e-6
    L.iscsi_set_option("precision", 32)
    st, e32 = L.iscsi_davidson(3, 1e-8)
    L.iscsi_set_option("precision", 64)
    assert st == 0
    assert np.abs(e32 - w[:3]).max() <= 1e-9


def test_davidson_truncated_single_root():
    n, k, tau = 12, 2, 1e-12
    h1, eri = make_integrals(n, 700, ell=3.0, nchol=12)
    o = Oracle(n, 2, 2, k, tau, h1, eri)
    w0 = np.linalg.eigvalsh(o.dense_h())[0]
    L.iscsi_init(n, 2, 2, k, h1, eri, tau)
    st, e = L.iscsi_davidson(1, 1e-8)
    assert st == 0 and abs(e[0] - w0) <= 1e-10


def test_several_contexts():
    n = 7
    h1, eri = make_integrals(n, 800)
    L.iscsi_init(n, 2, 2, 4, h1, eri, 0.0)
    a = L.iscsi_ctx_current()
    L.iscsi_init(n + 1, 2, 2, 2, *make_integrals(n + 1, 801), 0.0)
    b = L.iscsi_ctx_current()
    assert a != b
    L.iscsi_ctx_use(a)
    assert L.iscsi_ndet() == math.comb(n, 2) ** 2
    L.iscsi_ctx_destroy(a)
    assert L.iscsi_ndet() == -1
    L.iscsi_ctx_use(b)
    assert L.iscsi_ndet() > 0


@pytest.mark.parametrize("n,na,nb,k,tau", [(10, 2, 2, 4, 1e-14), (11, 2, 2, 2, 1e-6), (7, 3, 2, 3, 0.0),
                                           (9, 1, 2, 9, 1e-10)])
def test_fp64_tensor_core_and_native_paths_agree(n, na, nb, k, tau):
    h1, eri = make_integrals(n, 1100 + n, ell=3.0, nchol=12)
    L.iscsi_init(n, na, nb, k, h1, eri, tau)
    o = Oracle(n, na, nb, k, tau, h1, eri)
    C = np.stack([unit_vector(o.ndet, 60 + v) for v in range(2)])
    L.iscsi_set_option("fp64_tc", 1)
    s_tc = gpu_sigma(C, nvec=2).reshape(2, -1)
    L.iscsi_set_option("fp64_tc", 0)
    s_nat = gpu_sigma(C, nvec=2).reshape(2, -1)
    L.iscsi_set_option("fp64_tc", 1)
    for v in range(2):
        ref = o.sigma_terms(C[v])[0]
        assert_close(s_tc[v], ref, REL64)
        assert_close(s_nat[v], ref, REL64)


@pytest.mark.parametrize("n,k,tau", [(20, 4, 1e-14), (24, 3, 1e-12), (30, 2, 1e-10)])
def test_samespin_tensor_core_blocks(n, k, tau):
    # level blocks of >= 128 alpha strings with >= 64 allowed beta strings run the
    # same-spin products on the tensor cores; compare with the FP64 grouped GEMM
    h1, eri = make_integrals(n, 1200 + n, ell=4.0, nchol=16)
    L.iscsi_init(n, 2, 2, k, h1, eri, tau)
    nd = L.iscsi_ndet()
    C = np.stack([unit_vector(nd, 70 + v) for v in range(2)])
    L.iscsi_set_option("samespin_tc", 1)
    s_tc = gpu_sigma(C, nvec=2).reshape(2, -1)
    L.iscsi_set_option("samespin_tc", 0)
    L.iscsi_set_option("fp64_tc", 0)
    s_nat = gpu_sigma(C, nvec=2).reshape(2, -1)
    L.iscsi_set_option("samespin_tc", 1)
    L.iscsi_set_option("fp64_tc", 1)
    o = Oracle(n, 2, 2, k, tau, h1, eri)
    rows = np.random.default_rng(1).choice(nd, size=min(nd, 300), replace=False)
    for v in range(2):
        assert_close(s_tc[v], s_nat[v], REL64)
        ref = o.sigma_rows(C[v], rows)
        assert np.abs(s_tc[v][rows] - ref).max() <= REL64 * np.abs(s_nat[v]).max()


@pytest.mark.parametrize("n,na,nb,k,tau", [(10, 2, 2, 4, 1e-14), (11, 2, 2, 2, 1e-6), (7, 3, 2, 3, 0.0),
                                           (9, 1, 2, 9, 1e-10), (24, 2, 2, 3, 1e-12), (30, 2, 2, 2, 1e-10)])
def test_fp32_tensor_core_and_native_paths(n, na, nb, k, tau):
    # FP32 form: three bf16 terms per element on the tensor cores (default) and
    # the FP32 FFMA kernels both stay within the FP32 bound of the oracle
    h1, eri = make_integrals(n, 1300 + n, ell=4.0, nchol=12)
    L.iscsi_init(n, na, nb, k, h1, eri, tau)
    nd = L.iscsi_ndet()
    C = np.stack([unit_vector(nd, 80 + v) for v in range(2)])
    s64 = gpu_sigma(C, nvec=2).reshape(2, -1)
    L.iscsi_set_option("fp32_tc", 1)
    s_tc = gpu_sigma(C, nvec=2, precision=32).reshape(2, -1)
    L.iscsi_set_option("fp32_tc", 0)
    s_nat = gpu_sigma(C, nvec=2, precision=32).reshape(2, -1)
    L.iscsi_set_option("fp32_tc", 1)
    o = Oracle(n, na, nb, k, tau, h1, eri)
    rows = np.random.default_rng(2).choice(nd, size=min(nd, 400), replace=False)
    for v in range(2):
        ref = o.sigma_rows(C[v], rows)
        assert np.abs(s64[v][rows] - ref).max() <= REL64 * np.abs(s64[v]).max()
        for s in (s_tc[v], s_nat[v]):
            assert np.linalg.norm(s - s64[v]) <= REL32 * np.linalg.norm(s64[v])
            assert np.abs(s[rows] - ref).max() <= REL32 * np.abs(s64[v]).max()


def _stats():
    return L.iscsi_stats()


@pytest.mark.parametrize("use_graph", [1, 0])
def test_davidson_graph_and_direct_launches_agree(use_graph):
    # one Davidson iteration is replayed from a captured CUDA graph (default)
    # or launched directly; both reach the dense eigenvalues, and small
    # subspaces force thick restarts
    n, tau = 10, 1e-14
    h1, eri = make_integrals(n, 5, ell=3.0, nchol=20)
    o = Oracle(n, 2, 2, 4, tau, h1, eri)
    w = np.linalg.eigvalsh(o.dense_h())
    L.iscsi_init(n, 2, 2, 4, h1, eri, tau)
    L.iscsi_set_option("use_graph", use_graph)
    L.iscsi_set_option("max_subspace", 4)
    try:
        st, e = L.iscsi_davidson(4, 1e-8)
        s = _stats()
    finally:
        L.iscsi_set_option("use_graph", 1)
        L.iscsi_set_option("max_subspace", 0)
    assert st == 0
    assert np.abs(e - w[:4]).max() <= 1e-10
    assert s["davidson_graph"] == use_graph
    assert s["davidson_iters"] > 4


def test_davidson_many_roots_and_start_vectors():
    # 12 roots of a truncated space; a second run started from the first run's
    # vectors converges in a few iterations to the same energies
    n, k, tau = 12, 2, 1e-12
    h1, eri = make_integrals(n, 710, ell=3.0, nchol=12)
    o = Oracle(n, 2, 2, k, tau, h1, eri)
    w = np.linalg.eigvalsh(o.dense_h())
    L.iscsi_init(n, 2, 2, k, h1, eri, tau)
    vecs = torch.zeros((12, o.ndet), dtype=torch.float64, device="cuda")
    st, e = L.iscsi_davidson(12, 1e-8, vecs)
    assert st == 0
    assert np.abs(e - w[:12]).max() <= 1e-10
    it1 = _stats()["davidson_iters"]
    L.iscsi_set_option("guess_from_vecs", 1)
    try:
        st2, e2 = L.iscsi_davidson(12, 1e-8, vecs)
    finally:
        L.iscsi_set_option("guess_from_vecs", 0)
    assert st2 == 0
    assert np.abs(e2 - w[:12]).max() <= 1e-10
    assert _stats()["davidson_iters"] < it1


def test_davidson_whole_space():
    # fewer determinants than the subspace can hold: the basis reaches the
    # whole space and the iteration stops with the exact spectrum
    n = 4
    h1, eri = make_integrals(n, 720)
    o = Oracle(n, 1, 1, 2, 0.0, h1, eri)
    w = np.linalg.eigvalsh(o.dense_h())
    L.iscsi_init(n, 1, 1, 2, h1, eri, 0.0)
    st, e = L.iscsi_davidson(3, 1e-9)
    assert st == 0
    assert np.abs(e - w[:3]).max() <= 1e-10


@pytest.mark.parametrize("precision", [64, 32])
def test_autotune_picks_a_timed_routing_with_the_same_sigma(precision):
    # full CI in 40 orbitals: large enough for the autotuner to time its
    # candidates; the routing it keeps is the fastest it measured and gives the
    # same sigma as the default routing
    n, tau = 40, 1e-12
    h1, eri = make_integrals(n, 1400, ell=4.0, nchol=16)
    L.iscsi_init(n, 2, 2, 4, h1, eri, tau)
    nd = L.iscsi_ndet()
    C = np.stack([unit_vector(nd, 95 + v) for v in range(2)])
    s_def = gpu_sigma(C, nvec=2, precision=precision).reshape(2, -1)
    assert L.iscsi_stats()["route_fp%d" % precision]["tuned_nvec"] == 0
    L.iscsi_set_option("autotune", 1)
    try:
        s_tun = gpu_sigma(C, nvec=2, precision=precision).reshape(2, -1)
        r = L.iscsi_stats()["route_fp%d" % precision]
    finally:
        L.iscsi_set_option("autotune", 0)
    assert r["tuned_nvec"] == 2 and r["trials"]
    # trials: (opposite spin on tensor cores, same-spin threshold, predicted ms, measured ms)
    chosen = [t for t in r["trials"] if t[0] == r["ab_tc"] and t[1] == r["ss_min"]]
    assert len(chosen) == 1
    measured = [t[3] for t in r["trials"] if t[3] >= 0]
    assert len(measured) >= 2 and chosen[0][3] == min(measured)
    rel = REL64 if precision == 64 else REL32
    for v in range(2):
        assert np.linalg.norm(s_tun[v] - s_def[v]) <= rel * np.linalg.norm(s_def[v])


def test_davidson_extra_block_vectors():
    # iterating two more roots than wanted still returns the wanted ones
    n, tau = 10, 1e-14
    h1, eri = make_integrals(n, 6, ell=3.0, nchol=20)
    w = np.linalg.eigvalsh(Oracle(n, 2, 2, 4, tau, h1, eri).dense_h())
    L.iscsi_init(n, 2, 2, 4, h1, eri, tau)
    vecs = torch.zeros((2, L.iscsi_ndet()), dtype=torch.float64, device="cuda")
    L.iscsi_set_option("block_extra", 2)
    try:
        st, e = L.iscsi_davidson(2, 1e-8, vecs)
    finally:
        L.iscsi_set_option("block_extra", 0)
    assert st == 0 and e.shape == (2,)
    assert np.abs(e - w[:2]).max() <= 1e-10
    assert torch.abs(torch.linalg.norm(vecs, dim=1) - 1).max().item() < 1e-12

"""GPU parity of the density matrices (Eqs. d1, d2) against the CPU oracle.

Bar: the two-body blocks are FP64-accurate tensor-core products (exact bf16
slices, relative error ~2^-48 of sum |x||y| per element), so every element
must agree with the oracle within 1e-12 of the largest |element| of its
block (and the 2-norm of the difference within 1e-12 of the block's norm);
d1 likewise.  Structural zeros (p = r or q = t in a same-spin block, spins
without electrons) must be exactly zero.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import Oracle
from oracle import jordan_wigner as jw
from paper_1609_07757_gb300 import _lib as L
from paper_1609_07757_gb300.synthetic import make_integrals, unit_vector

pytestmark = pytest.mark.gpu

REL = 1e-12


@pytest.fixture(autouse=True)
def _fresh_library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.load()
    L.iscsi_set_option("autotune", 0)
    L.iscsi_set_stream(torch.cuda.current_stream())
    yield
    torch.cuda.synchronize()
    L.iscsi_finalize()
    L.iscsi_set_option("autotune", 1)


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda").contiguous()


def gpu_density(n, bra, ket=None, one=True, two=True, same_pointer=False):
    b = _dev(bra)
    k = None
    if ket is not None:
        k = b if same_pointer else _dev(ket)
    d1 = torch.full((2, n, n), float("nan"), dtype=torch.float64, device="cuda") if one else None
    d2 = torch.full((3, n, n, n, n), float("nan"), dtype=torch.float64, device="cuda") if two else None
    L.iscsi_density(b, k, d1, d2)
    torch.cuda.synchronize()
    return (d1.cpu().numpy() if one else None), (d2.cpu().numpy() if two else None)


def assert_block_close(got, ref):
    scale = max(np.abs(ref).max(), 1e-300)
    d = got - ref
    assert np.isfinite(got).all()
    assert np.abs(d).max() <= REL * scale, (np.abs(d).max(), scale)
    assert np.linalg.norm(d) <= REL * max(np.linalg.norm(ref), 1e-300)


CASES = [  # n, na, nb, kmax
    (10, 2, 2, 4),   # full CI, 2025 determinants
    (8, 2, 2, 2),    # CISD
    (9, 2, 2, 3),    # CISDT
    (7, 3, 2, 3),
    (6, 3, 3, 2),
    (7, 1, 1, 2),
    (6, 2, 0, 2),
    (5, 0, 3, 9),
    (2, 1, 1, 2),
    (8, 2, 2, 0),    # the reference determinant only
    (8, 2, 1, 9),
    (6, 4, 3, 9),    # four alpha electrons: two-hole strings with two electrons
]


@pytest.mark.parametrize("n,na,nb,k", CASES)
def test_state_density_matches_oracle(n, na, nb, k):
    h1, eri = make_integrals(n, 400 + n, ell=3.0, nchol=8)
    L.iscsi_init(n, na, nb, k, h1, eri, 0.0)
    o = Oracle(n, na, nb, k, 0.0, h1, eri)
    c = unit_vector(o.ndet, 21 + n)
    r1, r2 = o.density(c)
    g1, g2 = gpu_density(n, c)
    for s in range(2):
        assert_block_close(g1[s], r1[s])
    for b in range(3):
        assert_block_close(g2[b], r2[b])
    # exact structural zeros
    for b, ne in ((0, na), (2, nb)):
        if ne < 2:
            assert not np.any(g2[b])
        idx = np.arange(n)
        assert not np.any(g2[b][idx, :, idx, :]) and not np.any(g2[b][:, idx, :, idx])


@pytest.mark.parametrize("n,na,nb,k", [(10, 2, 2, 4), (9, 2, 2, 3), (7, 3, 2, 3), (6, 4, 3, 9), (8, 2, 1, 2)])
def test_transition_density_matches_oracle(n, na, nb, k):
    h1, eri = make_integrals(n, 500 + n, ell=3.0, nchol=8)
    L.iscsi_init(n, na, nb, k, h1, eri, 0.0)
    o = Oracle(n, na, nb, k, 0.0, h1, eri)
    bra = unit_vector(o.ndet, 31)
    ket = unit_vector(o.ndet, 32)
    r1, r2 = o.density(bra, ket)
    g1, g2 = gpu_density(n, bra, ket)
    for s in range(2):
        assert_block_close(g1[s], r1[s])
    for b in range(3):
        assert_block_close(g2[b], r2[b])


def test_general_path_equals_symmetric_path():
    """ket = a copy of bra runs the general (all regions) contraction; ket = bra the symmetric one."""
    n, na, nb, k = 11, 2, 2, 3
    h1, eri = make_integrals(n, 7, ell=3.0, nchol=8)
    L.iscsi_init(n, na, nb, k, h1, eri, 0.0)
    ndet = L.iscsi_ndet()
    c = unit_vector(ndet, 3)
    s1, s2 = gpu_density(n, c, c, same_pointer=True)
    g1, g2 = gpu_density(n, c, c, same_pointer=False)
    for b in range(3):
        assert_block_close(g2[b], s2[b])
    assert_block_close(g1, s1)


@pytest.mark.parametrize("n,na,nb,k", [(10, 2, 2, 4), (7, 3, 2, 3), (7, 1, 1, 2), (5, 0, 3, 9)])
def test_one_body_only(n, na, nb, k):
    """d2 = NULL: d1 from the direct one-hole kernel."""
    h1, eri = make_integrals(n, 600 + n, ell=3.0, nchol=8)
    L.iscsi_init(n, na, nb, k, h1, eri, 0.0)
    o = Oracle(n, na, nb, k, 0.0, h1, eri)
    bra, ket = unit_vector(o.ndet, 41), unit_vector(o.ndet, 42)
    r1, _ = o.density(bra, ket, two_body=False)
    g1, _ = gpu_density(n, bra, ket, two=False)
    for s in range(2):
        assert_block_close(g1[s], r1[s])


def test_tiny_case_matches_jordan_wigner():
    """n = 4, 2+2 electrons: the GPU against the Fock-space route directly."""
    n = 4
    h1, eri = make_integrals(n, 9, ell=3.0, nchol=4)
    L.iscsi_init(n, 2, 2, 9, h1, eri, 0.0)
    o = Oracle(n, 2, 2, 9, 0.0, h1, eri)
    ao, _ = o.strings(0)
    bo, _ = o.strings(1)
    off = o.offsets()
    dets = [(list(ao[a]), list(bo[b])) for a in range(len(ao)) for b in range(off[a + 1] - off[a])]
    bra, ket = unit_vector(o.ndet, 1), unit_vector(o.ndet, 2)
    j1, j2 = jw.density(n, dets, bra, ket)
    g1, g2 = gpu_density(n, bra, ket)
    assert_block_close(g1, j1)
    assert_block_close(g2, j2)


def test_several_tiles_ragged():
    """n = 20 full CI (36,100 determinants): 400 alpha-beta pair rows (3 full
    128-row tiles and a 16-row tail), 190 same-spin pair rows."""
    n, na, nb, k = 20, 2, 2, 4
    h1, eri = make_integrals(n, 20, ell=3.0, nchol=8)
    L.iscsi_init(n, na, nb, k, h1, eri, 0.0)
    o = Oracle(n, na, nb, k, 0.0, h1, eri)
    c = unit_vector(o.ndet, 5)
    r1, r2 = o.density(c)
    g1, g2 = gpu_density(n, c)
    for b in range(3):
        assert_block_close(g2[b], r2[b])
    assert_block_close(g1, r1)


def test_host_entry_point_matches_device():
    n, na, nb, k = 9, 2, 2, 3
    h1, eri = make_integrals(n, 3, ell=3.0, nchol=8)
    L.iscsi_init(n, na, nb, k, h1, eri, 0.0)
    ndet = L.iscsi_ndet()
    bra, ket = unit_vector(ndet, 8), unit_vector(ndet, 9)
    h1o = np.zeros((2, n, n))
    h2o = np.zeros((3, n, n, n, n))
    L.iscsi_density_host(bra, ket, h1o, h2o)
    g1, g2 = gpu_density(n, bra, ket)
    assert np.array_equal(h1o, g1) and np.array_equal(h2o, g2)


def test_energy_from_density_equals_sigma_expectation():
    """<c|H|c> from d1, d2 and the integrals equals c . sigma (tau = 0), n = 14 CISDT."""
    n, na, nb, k = 14, 2, 2, 3
    h1, eri = make_integrals(n, 14, ell=3.0, nchol=10)
    L.iscsi_init(n, na, nb, k, h1, eri, 0.0)
    ndet = L.iscsi_ndet()
    c = _dev(unit_vector(ndet, 4))
    s = torch.empty_like(c)
    L.iscsi_sigma(c, s, 1)
    d1 = torch.empty((2, n, n), dtype=torch.float64, device="cuda")
    d2 = torch.empty((3, n, n, n, n), dtype=torch.float64, device="cuda")
    L.iscsi_density(c, None, d1, d2)
    torch.cuda.synchronize()
    g = torch.as_tensor(jw.unpack_eri(eri, n), device="cuda")
    h = torch.as_tensor(h1, device="cuda")
    e_dm = float((h * (d1[0] + d1[1])).sum() + 0.5 * (g * (d2[0] + d2[2])).sum() + (g * d2[1]).sum())
    e_sig = float(torch.dot(c, s))
    assert abs(e_dm - e_sig) <= 1e-11 * max(1.0, abs(e_sig))

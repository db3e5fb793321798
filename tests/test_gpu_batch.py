"""GPU: the batching form (iscsi_batch_sigma) against one-at-a-time sigma.

The batch runs the same kernels on the same tiles as the single-context call;
only the launch grouping differs.  The FP64-accurate contraction's schedule is
planned over the whole launch, so a tile may be cut along K at other points
than in the single-context launch: each part is rounded to FP64 before the
parts are added, and the two results agree to the FP64 bar (1e-12 of the
largest element and of the 2-norm), not bit for bit.  Calls of one batch
reproduce each other exactly: the first runs directly, the second captures a
CUDA graph, later calls replay it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import Oracle
from paper_1609_07757_gb300 import _lib as L
from paper_1609_07757_gb300.synthetic import make_integrals, unit_vector

pytestmark = pytest.mark.gpu

SHAPES = [  # n, na, nb, kmax, tau
    (8, 2, 2, 4, 1e-14),
    (12, 2, 2, 4, 1e-12),
    (24, 2, 2, 3, 1e-12),   # same-spin level blocks on the tensor cores
    (9, 3, 2, 3, 0.0),
    (7, 1, 0, 9, 0.0),      # no opposite-spin part
    (30, 2, 2, 2, 1e-10),
]


@pytest.fixture(autouse=True)
def _fresh():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.load()
    L.iscsi_set_stream(torch.cuda.current_stream())
    L.iscsi_set_option("precision", 64)
    yield
    torch.cuda.synchronize()
    L.iscsi_finalize()
    L.iscsi_set_option("precision", 64)
    L.iscsi_set_option("use_graph", 1)


def _contexts(nvec):
    hs, cs, ints = [], [], []
    for i, (n, na, nb, k, tau) in enumerate(SHAPES):
        h1, eri = make_integrals(n, 1500 + i, ell=3.0, nchol=10)
        L.iscsi_init(n, na, nb, k, h1, eri, tau)
        hs.append(L.iscsi_ctx_current())
        nd = L.iscsi_ndet()
        cs.append(torch.tensor(np.stack([unit_vector(nd, 90 + 7 * i + v) for v in range(nvec)]),
                               dtype=torch.float64, device="cuda").contiguous())
        ints.append((h1, eri))
    return hs, cs, ints


@pytest.mark.parametrize("precision,nvec,graph", [(64, 1, 1), (64, 2, 1), (32, 2, 1), (64, 1, 0)])
def test_batch_sigma_matches_single_contexts(precision, nvec, graph):
    hs, cs, _ = _contexts(nvec)
    L.iscsi_set_option("precision", precision)
    L.iscsi_set_option("use_graph", graph)
    ref = []
    for h, c in zip(hs, cs):
        L.iscsi_ctx_use(h)
        s = torch.empty_like(c)
        L.iscsi_sigma(c, s, nvec)
        ref.append(s)
    torch.cuda.synchronize()
    outs = [torch.full_like(c, np.nan) for c in cs]
    rel = 1e-12 if precision == 64 else 2e-5
    first = None
    for call in range(3):  # direct, captured, replayed
        for o in outs:
            o.fill_(np.nan)
        L.iscsi_batch_sigma(hs, cs, outs, nvec)
        torch.cuda.synchronize()
        L.iscsi_batch_check()
        for o, r in zip(outs, ref):
            d = (o - r).abs()
            assert d.max().item() <= rel * r.abs().max().item(), (call, d.max().item())
            assert torch.linalg.norm(o - r).item() <= rel * torch.linalg.norm(r).item(), call
        if first is None:
            first = [o.clone() for o in outs]
        else:
            assert all(torch.equal(o, f) for o, f in zip(outs, first)), call
    assert L.iscsi_ctx_current() == hs[-1]


def test_batch_sigma_against_oracle_rows():
    hs, cs, ints = _contexts(1)
    outs = [torch.empty_like(c) for c in cs]
    L.iscsi_batch_sigma(hs, cs, outs, 1)
    torch.cuda.synchronize()
    for (n, na, nb, k, tau), (h1, eri), c, s in zip(SHAPES, ints, cs, outs):
        o = Oracle(n, na, nb, k, tau, h1, eri)
        rows = np.random.default_rng(n).choice(o.ndet, size=min(o.ndet, 200), replace=False)
        ref = o.sigma_rows(c.cpu().numpy()[0], rows)
        s = s.cpu().numpy()[0]
        assert np.abs(s[rows] - ref).max() <= 1e-12 * max(np.abs(s).max(), 1e-300)


def test_batch_sigma_rejects_bad_arguments():
    hs, cs, _ = _contexts(1)
    outs = [torch.empty_like(c) for c in cs]
    with pytest.raises(L.IscsiError):
        L.iscsi_batch_sigma([hs[0], hs[0]], cs[:2], outs[:2], 1)
    with pytest.raises(L.IscsiError):
        L.iscsi_batch_sigma([hs[0], 12345], cs[:2], outs[:2], 1)
    with pytest.raises(L.IscsiError):
        L.iscsi_batch_sigma([], [], [], 1)


@pytest.mark.parametrize("precision", [64, 32])
def test_batch_davidson_matches_dense_and_single(precision):
    # several contexts iterated together reach each one's dense eigenvalues,
    # like the one-context call
    shapes = [(8, 2, 2, 4, 1e-14), (10, 2, 2, 4, 1e-14), (12, 2, 2, 2, 1e-12), (7, 3, 2, 3, 0.0)]
    hs, ws = [], []
    for i, (n, na, nb, k, tau) in enumerate(shapes):
        h1, eri = make_integrals(n, 1600 + i, ell=3.0, nchol=12)
        ws.append(np.linalg.eigvalsh(Oracle(n, na, nb, k, tau, h1, eri).dense_h())[:2])
        L.iscsi_init(n, na, nb, k, h1, eri, tau)
        hs.append(L.iscsi_ctx_current())
    L.iscsi_set_option("precision", precision)
    vecs = []
    for h in hs:
        L.iscsi_ctx_use(h)
        vecs.append(torch.zeros((2, L.iscsi_ndet()), dtype=torch.float64, device="cuda"))
    st, e, sts = L.iscsi_batch_davidson(hs, 2, 1e-8, vecs)
    assert st == 0 and sts == [0] * len(hs)
    for i, h in enumerate(hs):
        assert np.abs(e[i] - ws[i]).max() <= (1e-10 if precision == 64 else 1e-9)
        L.iscsi_ctx_use(h)
        st1, e1 = L.iscsi_davidson(2, 1e-8)
        assert st1 == 0 and np.abs(e1 - ws[i]).max() <= (1e-10 if precision == 64 else 1e-9)
        # returned vectors are eigenvectors of the context's operator
        s = torch.empty_like(vecs[i])
        L.iscsi_set_option("precision", 64)
        L.iscsi_sigma(vecs[i], s, 2)
        L.iscsi_set_option("precision", precision)
        r = s - torch.tensor(e[i], device="cuda")[:, None] * vecs[i]
        assert torch.linalg.norm(r, dim=1).max().item() < 1e-6

"""GPU: the batching form (iscsi_batch_sigma) against one-at-a-time sigma.

The batch runs the same kernels on the same tiles as the single-context call
(only the launch grouping differs), so its result is bit-identical; the first
call runs directly, the second captures a CUDA graph, later calls replay it.
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
    for call in range(3):  # direct, captured, replayed
        for o in outs:
            o.fill_(np.nan)
        L.iscsi_batch_sigma(hs, cs, outs, nvec)
        torch.cuda.synchronize()
        L.iscsi_batch_check()
        for o, r in zip(outs, ref):
            assert torch.equal(o, r), call
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

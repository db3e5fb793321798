"""The persistent contraction's host-built schedule (no GPU needed).

iscsi_check_schedule plans synthetic problems with the library's own planner
and checks the plan: every 128 x 64 output tile's K steps covered exactly
once, split tiles' parts numbered in K order on one counter and one run of
workspace blocks, no CTA without work.  The balance bars pin the planner's
cost-model balance on shapes like the full-CI and GAS-context launches: tiles
close to the balanced load must be cut as well, or the CTAs holding them keep
gaps no part fits in.
"""
import numpy as np
import pytest

from paper_1609_07757_gb300 import _lib as L

FCI_LIKE = [(3600, 3600, [(3600, 3600)])] + [(600, 1770, [(592, 1770)] * 3)] * 6
GAS_CONTEXT_LIKE = [
    (2000, 400, [(2000, 400)]),
    (400, 1600, [(400, 1600)]),
    (190, 990, [(192, 990), (800, 190)]),
    (800, 190, [(192, 190), (800, 190), (992, 190)]),
]


@pytest.fixture(scope="module", autouse=True)
def _library():
    L.load()


@pytest.mark.parametrize("name,problems,min_balance", [
    ("fci", FCI_LIKE, 0.99),
    ("gas_context", GAS_CONTEXT_LIKE, 0.94),
    ("thin_and_empty_k", [(40000, 4, [(40000, 4)]), (300, 200, [(0, 200)])], 0.99),
])
def test_plan_covers_every_tile_and_balances(name, problems, min_balance):
    bal, c = L.iscsi_check_schedule(problems, 152)
    assert c["faults"] == 0, (name, c)
    assert c["ctas"] == 152
    assert bal >= min_balance, (name, bal, c)


def test_single_tile_runs_on_one_cta():
    bal, c = L.iscsi_check_schedule([(100, 40, [(112, 40)])], 152)
    assert c == {"ctas": 1, "items": 1, "tiles": 1, "split_tiles": 0, "faults": 0}
    assert bal == pytest.approx(1.0)


def test_random_shapes_and_sm_counts():
    rng = np.random.default_rng(17)
    for trial in range(40):
        probs = []
        for _ in range(int(rng.integers(1, 6))):
            M, N = int(rng.integers(1, 1500)), int(rng.integers(1, 900))
            segs = [(16 * int(rng.integers(0, 120)), int(rng.integers(1, N + 1))) for _ in range(int(rng.integers(1, 4)))]
            probs.append((M, N, segs))
        nsm = int(rng.choice([1, 2, 7, 64, 148, 152]))
        bal, c = L.iscsi_check_schedule(probs, nsm)
        tiles = sum(((M + 127) // 128) * ((N + 63) // 64) for M, N, _ in probs)
        assert c["faults"] == 0, (trial, probs, nsm, c)
        assert c["tiles"] == tiles and 1 <= c["ctas"] <= min(nsm, c["items"])
        assert 0.0 < bal <= 1.0 + 1e-12


@pytest.mark.parametrize("problems,nsm", [
    ([(100, 40, [(112, 40)])], 0),          # no SMs
    ([(100, 40, [(100, 40)])], 152),        # K not a multiple of 16
    ([(100, 40, [(112, 41)])], 152),        # more valid B rows than N
    ([(0, 40, [(112, 40)])], 152),          # empty problem
])
def test_schedule_check_rejects_bad_arguments(problems, nsm):
    with pytest.raises(L.IscsiError) as e:
        L.iscsi_check_schedule(problems, nsm)
    assert e.value.status == L.ISCSI_E_ARG

"""Pins of the oracle's time propagation (oracle/propagate.py).

Against closed forms and invariants that do not use the oracle's propagator:
the phase of an eigenvector, Rabi oscillations of a two-determinant space,
norm and energy conservation, time reversal, and the imaginary-time limit
(the lowest eigenvalue from LAPACK).  No GPU.
"""
import numpy as np
import pytest

from oracle import Oracle
from oracle.propagate import propagate
from paper_1609_07757_gb300.synthetic import make_integrals


def _system(n=6, na=2, nb=2, k=9, tau=0.0, seed=3):
    h1, eri = make_integrals(n, seed, ell=3.0, nchol=8)
    o = Oracle(n, na, nb, k, tau, h1, eri)
    v = np.add.outer(np.arange(n), np.arange(n)) * 0.0
    v[np.arange(n), np.arange(n)] = np.arange(n) - (n - 1) / 2.0  # position-like coupling
    v += 0.1 * (np.eye(n, k=1) + np.eye(n, k=-1))
    ov = Oracle(n, na, nb, k, tau, v, None)
    return o.dense_h(), ov.dense_h()


def test_eigenvector_picks_up_its_phase():
    H, V = _system()
    w, U = np.linalg.eigh(H)
    c = U[:, 1]
    dt, nst = 0.05, 20
    x = propagate(H, V, c, dt, [0.0] * nst)
    assert np.abs(x - np.exp(-1j * w[1] * dt * nst) * c).max() <= 1e-12


def test_rabi_two_determinants():
    """One alpha electron in two orbitals: H = diag(e0, e1), V couples them by v;
    with a constant field f the upper-state population is
    (2fv)^2 / W^2 sin^2(W t / 2), W^2 = (e1 - e0)^2 + (2fv)^2."""
    e0, e1, v, f = -1.0, -0.4, 0.3, 0.5
    h1 = np.diag([e0, e1])
    o = Oracle(2, 1, 0, 9, 0.0, h1, None)
    ov = Oracle(2, 1, 0, 9, 0.0, np.array([[0.0, v], [v, 0.0]]), None)
    H, V = o.dense_h(), ov.dense_h()
    dt, nst = 0.1, 37
    x = propagate(H, V, np.array([1.0, 0.0]), dt, [f] * nst)
    t = dt * nst
    W = np.sqrt((e1 - e0) ** 2 + (2 * f * v) ** 2)
    p1 = (2 * f * v) ** 2 / W ** 2 * np.sin(W * t / 2) ** 2
    assert abs(abs(x[1]) ** 2 - p1) <= 1e-12
    assert abs(np.linalg.norm(x) - 1.0) <= 1e-12


def test_norm_and_energy_conservation():
    H, V = _system(n=7, k=3)
    c = np.random.default_rng(1).standard_normal(H.shape[0])
    c /= np.linalg.norm(c)
    x = propagate(H, V, c, 0.05, [0.0] * 30)
    assert abs(np.linalg.norm(x) - 1.0) <= 1e-12
    assert abs(np.vdot(x, H @ x).real - c @ H @ c) <= 1e-11
    # with a field the norm is still conserved
    y = propagate(H, V, c, 0.05, list(np.sin(0.3 * np.arange(30))))
    assert abs(np.linalg.norm(y) - 1.0) <= 1e-12


def test_time_reversal():
    H, V = _system(n=6, k=2)
    c = np.random.default_rng(2).standard_normal(H.shape[0])
    c /= np.linalg.norm(c)
    field = list(0.4 * np.cos(0.2 * np.arange(15)))
    x = propagate(H, V, c, 0.07, field)
    back = propagate(H, V, x, -0.07, field[::-1])
    assert np.abs(back - c).max() <= 1e-12


def test_imaginary_time_reaches_the_ground_state():
    H, V = _system(n=6, k=9)
    w, U = np.linalg.eigh(H)
    c = np.random.default_rng(3).standard_normal(H.shape[0])
    x = propagate(H, V, c, 0.5, [0.0] * 200, imaginary=True)
    assert abs(x @ H @ x - w[0]) <= 1e-10
    assert abs(abs(x @ U[:, 0]) - 1.0) <= 1e-10

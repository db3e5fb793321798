"""Seeded synthetic integrals shaped like the paper's Be-in-a-box orbital sets.

This module holds input generation only -- none of the method's arithmetic --
so that the CUDA path and the CPU oracle receive identical inputs.

Recipe (all FP64, numpy PCG64 generator, seed = workload index * 1000 + instance):
  h_pq : symmetric; h_pp = -2.0 + 0.05 p; for p != q the upper triangle is
         N(0, 0.1) * w(p, q), mirrored to the lower triangle.
  (pq|rs) = sum_{K < nchol} L^K_pq L^K_rs, with L^K = (X + X^T)/sqrt(2) * w,
         X_pq ~ N(0, 0.3).  This gives 8-fold permutational symmetry and a
         positive-semidefinite two-electron matrix, like a Cholesky-factored
         Coulomb operator; the decay w imitates the pair locality of the
         FE-DVR integrals (the radial sparsity of Eq. gsparse).
  w(p, q) = exp(-|p - q| / ell)                        (plain decay), or
  w(p, q) = exp(-|p - q| / ell) [(1 + p/20)(1 + q/20)]^(-1/2)   (box sweep)
The two-electron integrals are returned pair-packed: element
[P(p,q), P(r,s)] = (pq|rs) with P(p,q) = max(p,q)(max(p,q)+1)/2 + min(p,q).
"""
import numpy as np

# name -> (n, electrons per spin, kmax, ell, nchol, box_decay, taus)
WORKLOADS = {
    "fci_n10": dict(n=10, nel=2, kmax=4, ell=3.0, nchol=20, box=False, taus=(0.0, 1e-14), seed=0),
    "fci_n60": dict(n=60, nel=2, kmax=4, ell=4.0, nchol=60, box=False, taus=(1e-14, 1e-12, 1e-10), seed=1000),
    "box_sweep": dict(n=(50, 100, 150, 200), nel=2, kmax=(2, 3), ell=5.0, nchol=20, box=True, taus=(1e-14,),
                      seed=2000),
    "fci_n100": dict(n=100, nel=2, kmax=4, ell=5.0, nchol=20, box=False, taus=(1e-12,), seed=3000),
    "cisdt_n120": dict(n=120, nel=2, kmax=3, ell=3.0, nchol=20, box=False, taus=(1e-14,), seed=4000),
    "multi_fci": dict(n=(20, 80), nel=2, kmax=4, ell=3.0, nchol=20, box=False, taus=(1e-14,), seed=4100,
                      count=64),
}


def pair_index(p, q):
    a, b = max(p, q), min(p, q)
    return a * (a + 1) // 2 + b


def decay_matrix(n, ell, box=False):
    idx = np.arange(n, dtype=np.float64)
    w = np.exp(-np.abs(idx[:, None] - idx[None, :]) / ell)
    if box:
        f = 1.0 + idx / 20.0
        w = w / np.sqrt(f[:, None] * f[None, :])
    return w


def make_integrals(n, seed, ell=3.0, nchol=20, box=False):
    """(h1 [n, n], eri [npair, npair]) as FP64 numpy arrays, C-contiguous."""
    rng = np.random.default_rng(seed)
    w = decay_matrix(n, ell, box)
    off = rng.normal(0.0, 0.1, size=(n, n)) * w
    h1 = np.triu(off, 1)
    h1 = h1 + h1.T
    h1[np.arange(n), np.arange(n)] = -2.0 + 0.05 * np.arange(n)
    iu = np.tril_indices(n)  # (p >= q) pairs in packed order p(p+1)/2 + q
    Lp = np.empty((nchol, n * (n + 1) // 2))
    for k in range(nchol):
        X = rng.normal(0.0, 0.3, size=(n, n))
        L = (X + X.T) / np.sqrt(2.0) * w
        Lp[k] = L[iu]
    eri = Lp.T @ Lp
    eri = 0.5 * (eri + eri.T)  # exactly symmetric: (pq|rs) and (rs|pq) are one value
    return np.ascontiguousarray(h1), np.ascontiguousarray(eri)


def unit_vector(ndet, seed):
    """Seeded N(0,1) vector normalised to unit 2-norm."""
    rng = np.random.default_rng(seed)
    c = rng.normal(size=ndet)
    return c / np.linalg.norm(c)


def multi_instance_sizes(count=64, lo=20, hi=80, seed=4100):
    """Orbital counts of the independent instances, uniform on [lo, hi]."""
    return np.random.default_rng(seed).integers(lo, hi + 1, size=count)


def transition_operator(n, p, q):
    """h of the one-body operator a+_p a_q (summed over spin): e_p e_q^T."""
    h = np.zeros((n, n))
    h[p, q] = 1.0
    return h


def square_operator_integrals(d):
    """(h1, eri) that express D^2, D = sum_pq d_pq E_pq with d symmetric, in the
    Hamiltonian's form sum h_pq E_pq + (1/2) sum (pq|rs) (E_pq E_rs - delta_qr E_ps):
    h1 = d d, (pq|rs) = 2 d_pq d_rs (pair-packed as make_integrals)."""
    d = np.asarray(d, dtype=np.float64)
    n = d.shape[0]
    pairs = np.array([d[p, q] for p in range(n) for q in range(p + 1)])  # pair_index order
    eri = 2.0 * np.outer(pairs, pairs)
    return np.ascontiguousarray(d @ d), np.ascontiguousarray(eri)

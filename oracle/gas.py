"""Generalised-active-space (GAS) restrictions of the determinant space.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. "Generalized Active Space (GAS)" (and the CAAB types of Eqs. 2gas,
3gas1-3gas4): the orbitals are split into ordered subspaces and only
determinants with allowed electron counts in them are kept.  The limits are
taken in the usual accumulated form: with n_j the number of electrons
(alpha + beta) of a determinant in subspace j, a determinant belongs to the
GAS space iff for every subspace j

    cmin[j] <= n_0 + n_1 + ... + n_j <= cmax[j].

Subspace j holds the next ``sizes[j]`` orbitals in index order.  The
paper's example (at most one electron in a continuum subspace after the
occupied and bound subspaces) is sizes = (n_occ, n_bound, n_cont) with
cmin = (0, N - 1, N), cmax = (N, N, N).  Combined with the excitation-level
truncation of Eq. ci_hierarchy the space is the intersection of the two.

The CI problem on that space is the Hamiltonian of the oracle restricted to
it: with P the projector onto the kept determinants, sigma = P H P c; the
dense restricted matrix is H[kept][:, kept].
"""
import numpy as np


def mask(oracle, sizes, cmin, cmax):
    """Boolean [ndet]: which determinants of the oracle's space (its canonical
    order) satisfy the accumulated occupation limits."""
    sizes = [int(x) for x in sizes]
    if sum(sizes) != oracle.n or len(cmin) != len(sizes) or len(cmax) != len(sizes):
        raise ValueError("GAS: subspace sizes must add up to the orbital count, one limit pair per subspace")
    bounds = np.cumsum([0] + sizes)
    ao, _ = oracle.strings(0)
    bo, _ = oracle.strings(1)
    off = oracle.offsets()

    def counts(orbs):
        # electrons of each string in each subspace, [count, nspace]
        out = np.zeros((len(orbs), len(sizes)), dtype=np.int64)
        for j in range(len(sizes)):
            if orbs.shape[1]:
                out[:, j] = ((orbs >= bounds[j]) & (orbs < bounds[j + 1])).sum(axis=1)
        return out

    ca = counts(np.asarray(ao).reshape(len(ao), -1))
    cb = counts(np.asarray(bo).reshape(len(bo), -1))
    keep = np.zeros(oracle.ndet, dtype=bool)
    for ia in range(len(ao)):
        nbeta = int(off[ia + 1] - off[ia])
        if nbeta == 0:
            continue
        tot = np.cumsum(ca[ia][None, :] + cb[:nbeta], axis=1)
        ok = np.all((tot >= np.asarray(cmin)) & (tot <= np.asarray(cmax)), axis=1)
        keep[off[ia]:off[ia + 1]] = ok
    return keep


def sigma(oracle, c, keep, nthreads=0):
    """sigma = P H P c on the full index range (zero outside the GAS space)."""
    k = keep.astype(np.float64)
    return k * oracle.sigma(k * np.asarray(c, dtype=np.float64), nthreads=nthreads)


def dense(oracle, keep):
    """H restricted to the GAS space, rows and columns in canonical order."""
    H = oracle.dense_h()
    return H[np.ix_(keep, keep)]

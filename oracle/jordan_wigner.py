"""Independent brute-force route: Fock-space Hamiltonian by Jordan-Wigner.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Builds the second-quantised Hamiltonian of Eq. ham in its unrestricted,
spin-summed form (Eq. index_un),
    H = sum_pq h_pq sum_s a+_ps a_qs
      + 1/2 sum_pqrs (pq|rs) sum_{s,t} a+_ps a+_rt a_st a_qs,
as explicit matrices on the 2^(2n)-dimensional Fock space (modes ordered
alpha 0..n-1 then beta 0..n-1), then takes matrix elements between the
determinants of a given list.  A determinant with ascending spin-orbital ids
i1 < i2 < ... is the product a+_i1 a+_i2 ... |vac>, which under Jordan-Wigner
with this mode order is the computational basis state with those bits set
and sign +1.  No code is shared with the C oracle: no index restriction, no
operator-string engine, no Slater-Condon selection.  Only for 2n <= 10.
"""
import numpy as np
import scipy.sparse as sp


def _annihilators(nmodes):
    """a_j for j = 0..nmodes-1 as sparse matrices; mode 0 is the most significant factor."""
    I2 = sp.identity(2, format="csr")
    Z = sp.csr_matrix(np.array([[1.0, 0.0], [0.0, -1.0]]))
    lower = sp.csr_matrix(np.array([[0.0, 1.0], [0.0, 0.0]]))  # |0><1| : removes a particle
    ops = []
    for j in range(nmodes):
        m = sp.identity(1, format="csr")
        for k in range(nmodes):
            f = Z if k < j else (lower if k == j else I2)
            m = sp.kron(m, f, format="csr")
        ops.append(m)
    return ops


def _basis_index(spin_orbitals, nmodes):
    idx = 0
    for i in spin_orbitals:
        idx |= 1 << (nmodes - 1 - i)
    return idx


def unpack_eri(eri_packed, n):
    """Full (pq|rs) array [n,n,n,n] from the pair-packed matrix."""
    P = np.zeros((n, n), dtype=np.int64)
    for p in range(n):
        for q in range(n):
            a, b = max(p, q), min(p, q)
            P[p, q] = a * (a + 1) // 2 + b
    return eri_packed[P[:, :, None, None], P[None, None, :, :]]


def hamiltonian(h1, eri_full, n):
    """Fock-space H (sparse) of Eq. ham with spin-summed integrals."""
    nm = 2 * n
    a = _annihilators(nm)
    ad = [x.T.tocsr() for x in a]
    dim = 1 << nm
    H = sp.csr_matrix((dim, dim))
    for s in range(2):
        for p in range(n):
            for q in range(n):
                if h1[p, q] != 0.0:
                    H = H + h1[p, q] * (ad[s * n + p] @ a[s * n + q])
    for s in range(2):
        for t in range(2):
            for p in range(n):
                for q in range(n):
                    for r in range(n):
                        for s_ in range(n):
                            g = eri_full[p, q, r, s_]
                            if g == 0.0:
                                continue
                            H = H + 0.5 * g * (ad[s * n + p] @ ad[t * n + r] @ a[t * n + s_] @ a[s * n + q])
    return H.tocsr()


def projected(h1, eri_full, n, dets):
    """<D_I|H|D_J> for a list of determinants, each (alpha orbitals, beta orbitals)."""
    H = hamiltonian(h1, eri_full, n)
    nm = 2 * n
    idx = [_basis_index(list(A) + [n + b for b in B], nm) for A, B in dets]
    return H[idx, :][:, idx].toarray()

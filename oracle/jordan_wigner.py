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


def density(n, dets, bra, ket):
    """Spin-resolved density matrices (Eqs. d1 and d2) through Fock-space matrices.

    dets: the determinant list (alpha orbitals, beta orbitals) that bra and
    ket are expanded in.  Returns (d1 [2, n, n], d2 [3, n, n, n, n]) with
      d1[s, p, q]       = <bra| a+_ps a_qs |ket>,
      d2[b, p, q, r, t] = <bra| a+_ps a+_ru a_tu a_qs |ket>,  (s,u) = aa, ab, bb,
    computed as inner products of the Fock vectors a_ru a_ps |bra> and
    a_tu a_qs |ket> (the adjoint of a+_ps a+_ru is a_ru a_ps).
    """
    nm = 2 * n
    a = _annihilators(nm)
    dim = 1 << nm
    fb = np.zeros(dim)
    fk = np.zeros(dim)
    for (A, B), x, y in zip(dets, bra, ket):
        i = _basis_index(list(A) + [n + b for b in B], nm)
        fb[i] = x
        fk[i] = y
    d1 = np.zeros((2, n, n))
    for s in range(2):
        vb = [a[s * n + p] @ fb for p in range(n)]
        vk = [a[s * n + q] @ fk for q in range(n)]
        for p in range(n):
            for q in range(n):
                d1[s, p, q] = vb[p] @ vk[q]
    d2 = np.zeros((3, n, n, n, n))
    for b, (s, u) in enumerate(((0, 0), (0, 1), (1, 1))):
        # X[p, r] = a_ru a_ps |bra>, Y[q, t] = a_tu a_qs |ket>
        X = np.array([[a[u * n + r] @ (a[s * n + p] @ fb) for r in range(n)] for p in range(n)])
        Y = np.array([[a[u * n + t] @ (a[s * n + q] @ fk) for t in range(n)] for q in range(n)])
        d2[b] = np.einsum("prk,qtk->pqrt", X, Y)
    return d1, d2

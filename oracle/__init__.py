"""CPU oracle for the ISCI sigma-vector step (arXiv:1609.07757).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of bench.py may import this
package.  It shares no code with ``paper_1609_07757_gb300`` and never imports
it; both sides receive the same integrals from the seeded input generator.

Contents
  * ``Oracle`` -- ctypes front end of ``iscsi_oracle.c``: determinant space
    (Eq. ci_hierarchy truncated at total excitation level k), the screened
    Hamiltonian of Eq. index_re (screening of Eq. sigma_split, applied per
    integral unit as in the screened loops of Sec. "Second part"), sigma by
    two independent traversals and dense H; the density matrices of Eqs. d1
    and d2 by explicit operator application.
  * ``jordan_wigner`` -- a third, independent route: the Fock-space matrix of
    the unrestricted Hamiltonian of Eq. ham for tiny orbital counts.
  * ``propagate`` -- exact piecewise-constant propagators of H + f(t) V.
  * ``gas`` -- GAS restrictions (Sec. "Generalized Active Space"): the kept
    determinants under accumulated subspace occupation limits, and the
    Hamiltonian restricted to them.

Parity status of each function is stated in its docstring; every function
here is pinned by tests/test_oracle_*.py (paper table, paper sign examples,
closed forms, brute force, invariants).
"""
import ctypes
import os

import numpy as np

from . import build as _build

ALL_CLASSES = (1 << 42) - 1

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        vp, i64, u64, dp, ip = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p
        lib.ora_create.restype = vp
        lib.ora_create.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double, dp, dp]
        lib.ora_destroy.argtypes = [vp]
        lib.ora_ndet.restype = i64
        lib.ora_ndet.argtypes = [vp]
        lib.ora_nstrings.restype = ctypes.c_int
        lib.ora_nstrings.argtypes = [vp, ctypes.c_int]
        lib.ora_strings.argtypes = [vp, ctypes.c_int, ip, ip]
        lib.ora_offsets.argtypes = [vp, dp]
        lib.ora_det_index.restype = i64
        lib.ora_det_index.argtypes = [vp, ip, ip]
        lib.ora_sigma_terms.argtypes = [vp, dp, dp, u64, dp]
        lib.ora_sigma_rows.argtypes = [vp, dp, dp, i64, dp, u64, ctypes.c_int]
        lib.ora_dense_h.argtypes = [vp, dp, u64]
        lib.ora_hij.restype = ctypes.c_double
        lib.ora_hij.argtypes = [vp, i64, i64, u64]
        lib.ora_max_threads.restype = ctypes.c_int
        lib.ora_density.argtypes = [vp, dp, dp, dp, dp, ctypes.c_int]
        lib.ora_density_elems.argtypes = [vp, dp, dp, ip, i64, dp, ctypes.c_int]
        lib.ora_apply.restype = ctypes.c_int
        lib.ora_apply.argtypes = [ctypes.c_int, ip, ip, ctypes.c_int, ip, ip, ip]
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Oracle:
    """Screened CI Hamiltonian on the truncated determinant space.

    n orbitals, na alpha and nb beta electrons, total excitation level <= kmax
    (kmax >= the maximum possible level gives full CI), screening threshold
    tau (a term is kept iff |unit| > tau).  h1 is n x n, eri is the pair-packed
    (pq|rs) matrix of shape (n(n+1)/2, n(n+1)/2) or None for no two-electron
    part.
    """

    def __init__(self, n, na, nb, kmax, tau, h1, eri):
        lib = _load()
        self.n, self.na, self.nb, self.kmax, self.tau = n, na, nb, kmax, float(tau)
        self._h1 = np.ascontiguousarray(h1, dtype=np.float64)
        self._eri = None if eri is None else np.ascontiguousarray(eri, dtype=np.float64)
        assert self._h1.shape == (n, n)
        if self._eri is not None:
            npair = n * (n + 1) // 2
            assert self._eri.shape == (npair, npair)
        self._h = lib.ora_create(n, na, nb, kmax, self.tau, _ptr(self._h1),
                                 None if self._eri is None else _ptr(self._eri))
        if not self._h:
            raise ValueError("oracle: invalid arguments")
        self.ndet = int(lib.ora_ndet(self._h))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.ora_destroy(self._h)
            self._h = None

    def strings(self, spin):
        """(orbitals [count, ne], levels [count]) in the library's canonical order."""
        lib = _load()
        cnt = lib.ora_nstrings(self._h, spin)
        ne = self.na if spin == 0 else self.nb
        orbs = np.zeros((cnt, max(ne, 1)), dtype=np.int32)
        lev = np.zeros(cnt, dtype=np.int32)
        lib.ora_strings(self._h, spin, _ptr(orbs), _ptr(lev))
        return orbs[:, :ne], lev

    def offsets(self):
        cnt = _load().ora_nstrings(self._h, 0)
        off = np.zeros(cnt + 1, dtype=np.int64)
        _load().ora_offsets(self._h, _ptr(off))
        return off

    def det_index(self, aorbs, borbs):
        a = np.ascontiguousarray(sorted(aorbs), dtype=np.int32)
        b = np.ascontiguousarray(sorted(borbs), dtype=np.int32)
        if a.size == 0:
            a = np.zeros(1, dtype=np.int32)
        if b.size == 0:
            b = np.zeros(1, dtype=np.int32)
        return int(_load().ora_det_index(self._h, _ptr(a), _ptr(b)))

    def sigma_terms(self, c, mask=ALL_CLASSES):
        """sigma = H_tau c by applying every surviving term to every determinant.

        Returns (sigma, number of updates sigma_I += term * c_J performed).
        Cost ~ (number of terms) x ndet: small spaces only.
        """
        c = np.ascontiguousarray(c, dtype=np.float64)
        assert c.shape == (self.ndet,)
        s = np.zeros(self.ndet)
        nup = np.zeros(1, dtype=np.int64)
        _load().ora_sigma_terms(self._h, _ptr(c), _ptr(s), ctypes.c_uint64(mask), _ptr(nup))
        return s, int(nup[0])

    def sigma_rows(self, c, rows, mask=ALL_CLASSES, nthreads=0):
        """sigma_I for the given row indices, H_IJ assembled row-wise (any size)."""
        c = np.ascontiguousarray(c, dtype=np.float64)
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        out = np.zeros(rows.shape[0])
        _load().ora_sigma_rows(self._h, _ptr(c), _ptr(rows), rows.shape[0], _ptr(out),
                               ctypes.c_uint64(mask), int(nthreads))
        return out

    def sigma(self, c, mask=ALL_CLASSES, nthreads=0):
        """Full sigma via the row-wise route."""
        return self.sigma_rows(c, np.arange(self.ndet, dtype=np.int64), mask, nthreads)

    def dense_h(self, mask=ALL_CLASSES):
        """Dense H_tau (ndet x ndet); small spaces only."""
        H = np.zeros((self.ndet, self.ndet))
        _load().ora_dense_h(self._h, _ptr(H), ctypes.c_uint64(mask))
        return H

    def hij(self, i, j, mask=ALL_CLASSES):
        return float(_load().ora_hij(self._h, i, j, ctypes.c_uint64(mask)))

    def density(self, bra, ket=None, two_body=True, nthreads=0):
        """One- and two-body density matrices of Eqs. d1 and d2, spin-resolved.

        Returns (d1 [2, n, n], d2 [3, n, n, n, n] or None):
          d1[s, p, q]       = <bra| a+_ps a_qs |ket>                 (s = alpha, beta)
          d2[b, p, q, r, t] = <bra| a+_ps a+_ru a_tu a_qs |ket>      ((s,u) = aa, ab, bb)
        by applying each operator string to every determinant of the space.
        ket defaults to bra.  Cost ~ ndet * n^2 (4 n^2 determinant look-ups
        per determinant and block): small spaces only.
        """
        bra = np.ascontiguousarray(bra, dtype=np.float64)
        ket = bra if ket is None else np.ascontiguousarray(ket, dtype=np.float64)
        assert bra.shape == (self.ndet,) and ket.shape == (self.ndet,)
        n = self.n
        d1 = np.zeros((2, n, n))
        d2 = np.zeros((3, n, n, n, n)) if two_body else None
        _load().ora_density(self._h, _ptr(bra), _ptr(ket), _ptr(d1), None if d2 is None else _ptr(d2), int(nthreads))
        return d1, d2

    def density_elems(self, bra, ket, spec, nthreads=0):
        """Single density-matrix elements, each a sum over the whole space.

        spec: int array [m, 5] of (block, p, q, r, t): block 0..2 selects
        d2[block, p, q, r, t], block 3 / 4 selects d1[0 / 1, p, q].
        """
        bra = np.ascontiguousarray(bra, dtype=np.float64)
        ket = bra if ket is None else np.ascontiguousarray(ket, dtype=np.float64)
        spec = np.ascontiguousarray(spec, dtype=np.int32).reshape(-1, 5)
        out = np.zeros(spec.shape[0])
        _load().ora_density_elems(self._h, _ptr(bra), _ptr(ket), _ptr(spec), spec.shape[0], _ptr(out), int(nthreads))
        return out

    def eigh(self, mask=ALL_CLASSES):
        """All eigenvalues / eigenvectors of the dense H_tau (LAPACK via numpy)."""
        return np.linalg.eigh(self.dense_h(mask))


def apply_operators(ops, occupied):
    """Apply a product of creation/annihilation operators to a determinant.

    ops: list of (is_creation, spin_orbital_id) written left to right (the
    rightmost acts first); occupied: spin-orbital ids of the determinant
    a+_i1 a+_i2 ... |vac> with i1 < i2 < ....  Returns (sign, ascending ids of
    the result); sign 0 means the product annihilates the determinant.
    """
    cr = np.ascontiguousarray([1 if c else 0 for c, _ in ops], dtype=np.int32)
    so = np.ascontiguousarray([i for _, i in ops], dtype=np.int32)
    inp = np.ascontiguousarray(sorted(occupied) or [0], dtype=np.int32)
    out = np.zeros(64, dtype=np.int32)
    olen = np.zeros(1, dtype=np.int32)
    sg = _load().ora_apply(len(ops), _ptr(cr), _ptr(so), len(occupied), _ptr(inp), _ptr(out), _ptr(olen))
    return int(sg), [int(x) for x in out[:olen[0]]]


def max_threads():
    return int(_load().ora_max_threads())

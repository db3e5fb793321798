"""Updates per sigma of the oracle's H_tau: the metric's unit of work, counted.

Test infrastructure only (part of the CPU oracle; the product library never
imports it).

One update is sigma_I += unit * c_J for one surviving unit (Sec. "Integral
screening": keep a unit iff |u| > tau) and one pair of determinants it
connects inside the truncated space (Eq. ci_hierarchy with the truncation at
excitation level k).  ora_sigma_terms counts the same updates by applying every
term to every determinant; here they are counted from the string spaces, so
that full-size workloads take seconds:

  a string of spin s holds ne electrons in n orbitals; its level is the number
  of them at orbitals >= ne (the virtual set V, the rest O);
  a string operator of that spin removes the orbitals `out` and adds `inn`; the
  strings it acts on contain `out` and none of `inn - out`; the other ne - |out|
  electrons lie in the orbitals outside out u inn, o' of them in O, v' in V, so
  C(o', ne - |out| - j) C(v', j) strings have j of those electrons in V, level
  j + |out & V| before and j + |inn & V| after;
  a determinant pair counts when both determinants' levels (alpha + beta) are
  at most k.
Units: one-body h_pq for each spin; same-spin A_{pr,qs} = g_psrq - g_pqrs
(p > r, q > s) for each spin (Eq. index_re); opposite-spin g_pqrs = (pq|rs).
"""
import math

import numpy as np

__all__ = ["updates_per_sigma", "eri_unpack"]


def eri_unpack(eri, n):
    """(pq|rs) as a dense [n, n, n, n] array from the pair-packed matrix."""
    idx = np.zeros((n, n), dtype=np.int64)
    for p in range(n):
        for q in range(n):
            a, b = max(p, q), min(p, q)
            idx[p, q] = a * (a + 1) // 2 + b
    return eri[idx[:, :, None, None], idx[None, None, :, :]]


def _comb(a, b):
    return math.comb(a, b) if 0 <= b <= a else 0


def _level_counts(n, ne, removed, added):
    """{(level before, level after): strings} for a string operator removing the
    orbitals `removed` and adding `added` (sets) on strings of ne electrons."""
    V = lambda x: x >= ne
    touched = set(removed) | set(added)
    o_free = sum(1 for x in range(n) if x not in touched and not V(x))
    v_free = sum(1 for x in range(n) if x not in touched and V(x))
    rest = ne - len(removed)
    lo = sum(1 for x in removed if V(x))
    la = sum(1 for x in added if V(x))
    out = {}
    for j in range(0, rest + 1):
        c = _comb(o_free, rest - j) * _comb(v_free, j)
        if c:
            out[(lo + j, la + j)] = out.get((lo + j, la + j), 0) + c
    return out


def _other_spin_levels(n, ne):
    """strings of the other spin per level"""
    return [_comb(ne, ne - l) * _comb(n - ne, l) for l in range(ne + 1)]


def _kind_key(n, ne, p, q):
    """what the count of a one-body operator a+_p a_q depends on"""
    return (p == q, p >= ne, q >= ne)


def updates_per_sigma(n, na, nb, kmax, tau, h1, eri):
    """Updates per sigma of the truncated, screened Hamiltonian (floating count)."""
    h1 = np.asarray(h1, dtype=np.float64)
    ne = (na, nb)
    other = (_other_spin_levels(n, nb), _other_spin_levels(n, na))
    total = 0.0

    def with_other(hist, s):
        # a same-spin operator leaves the other spin's string unchanged: it may
        # be any string whose level fits beside both levels of this one
        lv = other[s]
        t = 0.0
        for (l0, l1), c in hist.items():
            room = kmax - max(l0, l1)
            t += c * sum(lv[:max(0, min(room, len(lv) - 1)) + 1]) if room >= 0 else 0.0
        return t

    # one-body units, each spin
    for s in range(2):
        if ne[s] == 0:
            continue
        keep = np.abs(h1) > tau
        for p in range(n):
            for q in range(n):
                if keep[p, q]:
                    total += with_other(_level_counts(n, ne[s], {q}, {p}), s)
    if eri is None:
        return total
    g = eri_unpack(np.asarray(eri, dtype=np.float64), n)  # g[p, q, r, s] = (pq|rs)
    # same-spin units A_{pr,qs} = g_psrq - g_pqrs, p > r, q > s; a unit's count
    # depends on the free orbitals (outside {p, q, r, s}) in O and V and on the
    # levels of {q, s} (removed) and {p, r} (added)
    A = np.transpose(g, (0, 3, 2, 1)) - g  # A[p, q, r, s] = g[p, s, r, q] - g[p, q, r, s]
    P, Q, R, S = np.indices((n,) * 4, dtype=np.int16)
    for s in range(2):
        if ne[s] < 2:
            continue
        nv = lambda x: (x >= ne[s]).astype(np.int64)
        keep = (P > R) & (Q > S) & (np.abs(A) > tau)
        p_, q_, r_, s_ = P[keep], Q[keep], R[keep], S[keep]
        shared = (p_ == q_).astype(np.int64), (p_ == s_).astype(np.int64), (r_ == q_).astype(np.int64), \
            (r_ == s_).astype(np.int64)
        sh_v = shared[0] * nv(p_) + shared[1] * nv(p_) + shared[2] * nv(r_) + shared[3] * nv(r_)
        sh_all = shared[0] + shared[1] + shared[2] + shared[3]
        lo, la = nv(q_) + nv(s_), nv(p_) + nv(r_)
        touched_v = lo + la - sh_v
        touched_o = 4 - sh_all - touched_v
        v_free = (n - ne[s]) - touched_v
        o_free = ne[s] - touched_o
        key = ((o_free * 512 + v_free) * 4 + lo) * 4 + la
        uk, cnt = np.unique(key, return_counts=True)
        for k_, m in zip(uk, cnt):
            la_k, lo_k = int(k_ % 4), int(k_ // 4 % 4)
            v_k, o_k = int(k_ // 16 % 512), int(k_ // 8192)
            hist = {}
            for j in range(0, ne[s] - 1):
                c = _comb(o_k, ne[s] - 2 - j) * _comb(v_k, j)
                if c:
                    hist[(lo_k + j, la_k + j)] = hist.get((lo_k + j, la_k + j), 0) + c
            total += float(m) * with_other(hist, s)
    # opposite-spin units g_pqrs: alpha a+_p a_q, beta a+_r a_s
    if na == 0 or nb == 0:
        return total
    for spin, nel in ((0, na), (1, nb)):
        kinds = {}
        kind = np.zeros((n, n), dtype=np.int64)
        hs = []
        for p in range(n):
            for q in range(n):
                key = _kind_key(n, nel, p, q)
                if key not in kinds:
                    kinds[key] = len(kinds)
                    hs.append(_level_counts(n, nel, {q}, {p}))
                kind[p, q] = kinds[key]
        if spin == 0:
            ka, ha = kind, hs
        else:
            kb, hb = kind, hs
    keep = np.abs(g) > tau  # [p, q, r, s]
    idx = ka[:, :, None, None] * len(hb) + kb[None, None, :, :]
    cnt = np.bincount(idx[keep].ravel(), minlength=len(ha) * len(hb))
    for i, hA in enumerate(ha):
        for j, hB in enumerate(hb):
            m = cnt[i * len(hb) + j]
            if not m:
                continue
            w = 0
            for (a0, a1), ca in hA.items():
                for (b0, b1), cb in hB.items():
                    if a0 + b0 <= kmax and a1 + b1 <= kmax:
                        w += ca * cb
            total += float(m) * w
    return total

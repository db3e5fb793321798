"""Time propagation of a CI vector by the exact piecewise-constant propagator.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The Hamiltonian of Eq. ham with a time-dependent one-body part,
    H(t) = H_tau + f(t) V,   h(t) = h + f(t) v,
where H_tau is the screened Hamiltonian of the oracle (Eq. index_re,
Eq. sigma_split) and V the one-body operator of the coupling matrix v on the
same truncated space (the oracle's Hamiltonian with h1 = v and no two-electron
part).  Over step k of length dt the field is held at the caller's sample f_k
(for a smooth field, its value at the step's midpoint), and the exact
propagator of that constant Hamiltonian is applied:
    real time:       c <- expm(-i (H + f_k V) dt) c
    imaginary time:  c <- expm(-(H + f_k V) dt) c / ||expm(-(H + f_k V) dt) c||
(the paper's ground-state runs propagate in imaginary time, Sec. "Application").
The dense matrices come from ``Oracle.dense_h``; the exponential is
scipy.linalg.expm (a library primitive).  Small spaces only.
"""
import numpy as np
import scipy.linalg as sla


def propagate(H, V, c, dt, field, imaginary=False):
    """Return the vector after len(field) steps (complex for real time, real for imaginary time).

    H, V: dense (ndet x ndet) matrices (V may be None when every f_k is 0);
    c: start vector; field: the per-step samples f_k.
    """
    x = np.asarray(c, dtype=np.float64 if imaginary else np.complex128).copy()
    for f in field:
        A = H if (V is None or f == 0.0) else H + f * V
        if imaginary:
            x = sla.expm(-dt * A) @ x
            x /= np.linalg.norm(x)
        else:
            x = sla.expm(-1j * dt * A) @ x
    return x

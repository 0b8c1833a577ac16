"""Dense plain definition of the selected blocks -- test infrastructure, see the package header.

Eq. 2 with Table I's G-row: M(E) = E S - H - Sigma^R(E) and M X^< M^dagger = B^< = Sigma^<, so
G^R = M^-1 and G^< = G^R Sigma^< G^A (G^A = (G^R)^H).  With the broadening z = E + i eta on S
treated as an extra retarded self-energy -i eta S whose greater part is -2 i eta S (and lesser part
0), the greater function is G^> = G^R (Sigma^> - 2 i eta S) G^A with Sigma^> = Sigma^< + Sigma^R -
Sigma^A for every self-energy that enters.  Only the block-tridiagonal pattern is returned.

This builds the full N_B*b square matrices, so it is for tiny inputs (N_B*b up to a few hundred).
"""
from __future__ import annotations

import numpy as np


def _full(diag: np.ndarray, upper: np.ndarray | None, hermitian_lower: bool = True) -> np.ndarray:
    nb, b, _ = diag.shape
    n = nb * b
    X = np.zeros((n, n), dtype=np.complex128)
    for i in range(nb):
        X[i * b:(i + 1) * b, i * b:(i + 1) * b] = diag[i]
    if upper is not None:
        for i in range(nb - 1):
            X[i * b:(i + 1) * b, (i + 1) * b:(i + 2) * b] = upper[i]
            if hermitian_lower:
                X[(i + 1) * b:(i + 2) * b, i * b:(i + 1) * b] = upper[i].conj().T
    return X


def dense_selected(E: float, eta: float, H_diag, H_upper, S_diag=None, S_upper=None,
                   SigR_diag=None, SigL_diag=None, lead_SigR=(None, None), lead_SigL=(None, None),
                   SigR_upper=None, SigR_lower=None, SigL_upper=None):
    """Selected blocks of G^R, G^<, G^> at one energy by dense inversion.

    ``SigR_diag``/``SigL_diag``: [N_B][b][b] scattering self-energies (or None);
    ``SigR_upper``/``SigR_lower``/``SigL_upper``: [N_B-1][b][b] off-diagonal blocks Sigma^R_{i,i+1},
    Sigma^R_{i+1,i}, Sigma^<_{i,i+1} of block-tridiagonal ones (Sigma^<_{i+1,i} = -(Sigma^<_{i,i+1})^H);
    ``lead_SigR``/``lead_SigL``: (left, right) contact blocks added on slices 0 and N_B-1.
    Returns dict with GR_diag [N_B], GR_upper [N_B-1] (G_{i,i+1}), GR_lower [N_B-1] (G_{i+1,i}),
    GL_diag, GL_upper, GG_diag, GG_upper.
    """
    nb, b, _ = H_diag.shape
    n = nb * b
    H = _full(H_diag, H_upper)
    if S_diag is None:
        S = np.eye(n, dtype=np.complex128)
    else:
        S = _full(S_diag, S_upper)
    SR = np.zeros((n, n), dtype=np.complex128)
    SL = np.zeros((n, n), dtype=np.complex128)
    if SigR_diag is not None:
        SR += _full(SigR_diag, None)
    if SigL_diag is not None:
        SL += _full(SigL_diag, None)
    for i in range(nb - 1):
        up, lo = slice(i * b, (i + 1) * b), slice((i + 1) * b, (i + 2) * b)
        if SigR_upper is not None:
            SR[up, lo] += SigR_upper[i]
        if SigR_lower is not None:
            SR[lo, up] += SigR_lower[i]
        if SigL_upper is not None:
            SL[up, lo] += SigL_upper[i]
            SL[lo, up] -= SigL_upper[i].conj().T
    for k, sl in ((0, slice(0, b)), (1, slice(n - b, n))):
        if lead_SigR[k] is not None:
            SR[sl, sl] += lead_SigR[k]
        if lead_SigL[k] is not None:
            SL[sl, sl] += lead_SigL[k]
    z = E + 1j * eta
    M = z * S - H - SR
    G = np.linalg.inv(M)
    GA = G.conj().T
    GL = G @ SL @ GA
    SG = SL + SR - SR.conj().T - 2j * eta * S
    GG = G @ SG @ GA

    def blk(X, i, j):
        return X[i * b:(i + 1) * b, j * b:(j + 1) * b]

    out = {}
    for name, X in (("GR", G), ("GL", GL), ("GG", GG)):
        out[name + "_diag"] = np.stack([blk(X, i, i) for i in range(nb)])
        out[name + "_upper"] = np.stack([blk(X, i, i + 1) for i in range(nb - 1)]) if nb > 1 else \
            np.zeros((0, b, b), np.complex128)
    out["GR_lower"] = np.stack([blk(G, i + 1, i) for i in range(nb - 1)]) if nb > 1 else \
        np.zeros((0, b, b), np.complex128)
    out["GL_lower"] = np.stack([blk(GL, i + 1, i) for i in range(nb - 1)]) if nb > 1 else \
        np.zeros((0, b, b), np.complex128)
    return out

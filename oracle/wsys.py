"""Screened-Coulomb (W) quadratic system -- test infrastructure only (see the package header).

Table I's second row: the selected solution of M X^<> M^H = B^<> (Eq. 2) with
    M(E) = I - V P^R(E),      B^<>(E) = V P^<>(E) V^H,      X^<> = W^<>,
V the (Hermitian) Coulomb matrix and P^R, P^<> the polarisation; like G it is solved independently
at every energy.  All matrices are block-tridiagonal (BT) with N_B blocks of b x b (Sec. II-A).

Reading (the paper does not say how the products are kept in the BT pattern): the system matrix and
right-hand side are the BT blocks of the exact products -- M_ij = delta_ij I - (V P^R)_ij and
B_ij = (V P V^H)_ij for |i - j| <= 1, from all contributing blocks of the BT factors -- and the blocks
beyond the first off-diagonal are not kept.  P^<> are anti-Hermitian (their lower blocks are
-(upper)^H), so B^<> are too; V's lower blocks are (upper)^H.

The selected solve of such a system is the recursion of ``rgf.py`` with A_i = M_ii, U_i = M_{i,i+1},
V_i = M_{i+1,i} and Sigma^< replaced by the BT right-hand side (its cross terms included); its
"retarded" output is the BT part of M^-1.  X^> needs its own lesser recursion with B^>.
"""
from __future__ import annotations

import numpy as np

from .rgf import rgf_energy


def _H(X):
    return X.conj().T


def full_bt(diag, upper, lower):
    """Dense matrix from BT blocks (lower may be None -> zero)."""
    nb, b, _ = diag.shape
    X = np.zeros((nb * b, nb * b), dtype=np.complex128)
    for i in range(nb):
        X[i * b:(i + 1) * b, i * b:(i + 1) * b] = diag[i]
    for i in range(nb - 1):
        if upper is not None:
            X[i * b:(i + 1) * b, (i + 1) * b:(i + 2) * b] = upper[i]
        if lower is not None:
            X[(i + 1) * b:(i + 2) * b, i * b:(i + 1) * b] = lower[i]
    return X


def bt_blocks(X, nb, b):
    """(diag, upper, lower) BT blocks of a dense matrix."""
    blk = lambda i, j: X[i * b:(i + 1) * b, j * b:(j + 1) * b]
    d = np.stack([blk(i, i) for i in range(nb)])
    z = np.zeros((0, b, b), np.complex128)
    u = np.stack([blk(i, i + 1) for i in range(nb - 1)]) if nb > 1 else z
    lo = np.stack([blk(i + 1, i) for i in range(nb - 1)]) if nb > 1 else z
    return d, u, lo


def assemble(V_diag, V_upper, PR, PL, PG=None):
    """M = I - V P^R and B^<> = V P^<> V^H restricted to the BT pattern, at one energy.

    ``PR`` = (diag, upper, lower); ``PL``/``PG`` = (diag, upper) of anti-Hermitian P^<, P^>.
    Returns dict with M_diag, M_upper, M_lower, BL_diag, BL_upper (and BG_* when PG is given)."""
    nb, b, _ = V_diag.shape
    V = full_bt(V_diag, V_upper, np.conj(np.swapaxes(V_upper, 1, 2)) if nb > 1 else None)
    M = np.eye(nb * b, dtype=np.complex128) - V @ full_bt(*PR)
    md, mu, ml = bt_blocks(M, nb, b)
    out = dict(M_diag=md, M_upper=mu, M_lower=ml)
    for key, P in (("BL", PL), ("BG", PG)):
        if P is None:
            continue
        lower = -np.conj(np.swapaxes(P[1], 1, 2)) if nb > 1 else None
        Bf = V @ full_bt(P[0], P[1], lower) @ _H(V)
        d, u, _ = bt_blocks(Bf, nb, b)
        out[key + "_diag"], out[key + "_upper"] = d, u
    return out


def system_device(M, B_diag, B_upper):
    """A device dict for ``rgf.rgf_energy`` whose system matrix is M (per-energy arrays [1][...])
    and whose lesser right-hand side is B: H = 0, S = 0 (so z S vanishes), Sigma^R = -M on every BT
    block, Sigma^< = B."""
    nb, b, _ = M["M_diag"].shape
    z = np.zeros((nb, b, b), np.complex128)
    return dict(n_blocks=nb, block_size=b, H_diag=z, H_upper=np.zeros((max(nb - 1, 0), b, b), np.complex128),
                S_diag=z, S_upper=np.zeros((max(nb - 1, 0), b, b), np.complex128),
                SigR=-M["M_diag"][None], SigL=B_diag[None],
                SigR_upper=-M["M_upper"][None], SigR_lower=-M["M_lower"][None], SigL_upper=B_upper[None],
                leads=None, energies=np.zeros(1), eta=0.0, mu_L=0.0, mu_R=0.0, kT=0.025)


def solve(M, BL, BG=None):
    """Selected blocks of X^R = M^-1 and X^< (and X^> with BG) by the recursion.

    ``M`` = dict of M_diag/M_upper/M_lower, ``BL``/``BG`` = (diag, upper).  Returns XR_diag,
    XR_upper, XR_lower, XL_diag, XL_upper (XG_diag, XG_upper)."""
    r = rgf_energy(0.0, system_device(M, *BL))
    out = dict(XR_diag=r["GR_diag"], XR_upper=r["GR_upper"], XR_lower=r["GR_lower"],
               XL_diag=r["GL_diag"], XL_upper=r["GL_upper"])
    if BG is not None:
        g = rgf_energy(0.0, system_device(M, *BG))
        out.update(XG_diag=g["GL_diag"], XG_upper=g["GL_upper"])
    return out


def dense_solve(M, BL, BG=None):
    """The plain definition: X^R = M^-1, X^<> = M^-1 B^<> M^-H on the dense BT-pattern matrices."""
    nb, b, _ = M["M_diag"].shape
    Mf = full_bt(M["M_diag"], M["M_upper"], M["M_lower"])
    Xr = np.linalg.inv(Mf)
    d, u, lo = bt_blocks(Xr, nb, b)
    out = dict(XR_diag=d, XR_upper=u, XR_lower=lo)
    for key, B in (("XL", BL), ("XG", BG)):
        if B is None:
            continue
        lower = -np.conj(np.swapaxes(B[1], 1, 2)) if nb > 1 else None
        X = Xr @ full_bt(B[0], B[1], lower) @ _H(Xr)
        dd, uu, _ = bt_blocks(X, nb, b)
        out[key + "_diag"], out[key + "_upper"] = dd, uu
    return out

"""Lead (contact) self-energies for the oracle -- test infrastructure, see the package header.

The contact part of Sigma^R in Table I's G-row (M = E S - H - Sigma^R) is the retarded
self-energy of a semi-infinite periodic lead.  The paper does not say how it is obtained; this
oracle uses the Lopez Sancho-Sancho-Rubio decimation (J. Phys. F 15, 851 (1985)).

Lead convention: ``H00`` is the lead's principal layer, ``H01`` = H_{n,n+1} couples lead cell n to
cell n+1 one step FURTHER from the device, and the device's end slice couples to the first lead
cell by the same ``H01`` (the end slice acts as cell 0).  Then the end slice sees
Sigma^R = H01 g_s H01^H, with g_s the surface Green's function of cell 1.
"""
from __future__ import annotations

import numpy as np


def fermi(E: float, mu: float, kT: float) -> float:
    """Fermi-Dirac occupation f(E - mu) = 1 / (1 + exp((E - mu)/kT)), overflow-safe."""
    x = (E - mu) / kT
    if x > 0:
        ex = np.exp(-x)
        return float(ex / (1.0 + ex))
    return float(1.0 / (1.0 + np.exp(x)))


def sancho_rubio(z: complex, H00: np.ndarray, H01: np.ndarray, tol: float = 1e-13,
                 max_iter: int = 100, track_cond: bool = False):
    """Surface Green's function g_s = (z - H00 - H01 g_s H01^H)^-1 of a semi-infinite lead.

    Decimation: start from alpha = H01, beta = H01^H, eps_s = eps = H00; each sweep removes every
    other cell, renormalising the surface (eps_s), bulk (eps) and the couplings (alpha, beta):
        g      = (z - eps)^-1
        eps_s += alpha g beta
        eps   += alpha g beta + beta g alpha
        alpha  = alpha g alpha,   beta = beta g beta
    until max|alpha|, max|beta| fall below tol * max|H01|.  Returns (g_s, sweeps, converged), plus
    the largest 2-norm condition number of the inverted blocks (z - eps) when ``track_cond``: the
    paper's Eq. 6 error model (error ~ kappa * eps_m) applied to this iteration.
    """
    b = H00.shape[0]
    eye = np.eye(b, dtype=np.complex128)
    alpha = H01.astype(np.complex128).copy()
    beta = H01.conj().T.astype(np.complex128).copy()
    eps_s = H00.astype(np.complex128).copy()
    eps = H00.astype(np.complex128).copy()
    scale = max(float(np.abs(H01).max()), 1e-300)
    converged = False
    it = 0
    kappa = 0.0
    for it in range(1, max_iter + 1):
        if track_cond:
            kappa = max(kappa, float(np.linalg.cond(z * eye - eps)))
        g = np.linalg.inv(z * eye - eps)
        agb = alpha @ g @ beta
        bga = beta @ g @ alpha
        eps_s = eps_s + agb
        eps = eps + agb + bga
        alpha = alpha @ g @ alpha
        beta = beta @ g @ beta
        if max(np.abs(alpha).max(), np.abs(beta).max()) < tol * scale:
            converged = True
            break
    if track_cond:
        kappa = max(kappa, float(np.linalg.cond(z * eye - eps_s)))
    g_s = np.linalg.inv(z * eye - eps_s)
    if track_cond:
        return g_s, it, converged, kappa
    return g_s, it, converged


def lead_self_energy(E: float, eta: float, H00: np.ndarray, H01: np.ndarray,
                     tol: float = 1e-13, max_iter: int = 100, track_cond: bool = False):
    """Retarded self-energy Sigma^R = H01 g_s(E + i eta) H01^H on the device's end slice.

    Returns (Sigma^R, sweeps, converged) or, with ``track_cond``, also the decimation's largest
    block condition number."""
    r = sancho_rubio(E + 1j * eta, H00, H01, tol, max_iter, track_cond)
    if track_cond:
        return H01 @ r[0] @ H01.conj().T, r[1], r[2], r[3]
    return H01 @ r[0] @ H01.conj().T, r[1], r[2]

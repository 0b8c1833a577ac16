"""Recursive Green's function (RGF) selected inversion in FP64 -- test infrastructure only.

What is computed (Eq. 2 with Table I's G-row, solved independently at every energy E, Sec. II-A):
the diagonal and first off-diagonal blocks of G^R = M^-1 and G^< = G^R Sigma^< G^A for the
block-tridiagonal M = z S - H - Sigma^R, z = E + i eta.  The solver is the block Gaussian
elimination of Sec. IV-A (forward elimination of slices 0..N_B-1, then back-substitution for the
selected blocks); the blocks are those of the BT tiling of Sec. II-A.

Notation (slice i = 0..N_B-1, block size b):
    A_i = M_ii = z S_ii - H_ii - Sigma^R_ii  (+ contact Sigma^R on slices 0 and N_B-1)
    U_i = M_{i,i+1} = z S_{i,i+1} - H_{i,i+1} - Sigma^R_{i,i+1}
    V_i = M_{i+1,i} = z S_{i,i+1}^H - H_{i,i+1}^H - Sigma^R_{i+1,i}
The scattering self-energies may be block-diagonal or block-tridiagonal; their off-diagonal blocks
Sigma^R_{i,i+1}, Sigma^R_{i+1,i}, L_i = Sigma^<_{i,i+1} (Sigma^<_{i+1,i} = -L_i^H) are zero in the
first case.
Forward (left-connected) sweep:
    g_0 = A_0^-1,                 g_i = (A_i - V_{i-1} g_{i-1} U_{i-1})^-1
    g^<_0 = g_0 Sigma^<_0 g_0^H,
    g^<_i = g_i (Sigma^<_i + V_{i-1} g^<_{i-1} V_{i-1}^H - Y_i + Y_i^H) g_i^H,  Y_i = V_{i-1} g_{i-1} L_{i-1}
Backward sweep (G_{N-1,N-1} = g_{N-1}, G^<_{N-1,N-1} = g^<_{N-1}), with P = g_i U_i:
    G_{i,i+1} = -P G_{i+1,i+1},   G_{i+1,i} = -G_{i+1,i+1} V_i g_i,   G_ii = g_i - P G_{i+1,i}
    Q = V_i g^<_i + (g_i L_i)^H,  K = P G_{i+1,i+1} Q
    G^<_ii = g^<_i + P G^<_{i+1,i+1} P^H + K - K^H
    G^<_{i,i+1} = -P G^<_{i+1,i+1} + (G_{i+1,i+1} Q)^H
(With L = 0, Q = V_i g^<_i and the last line is -P G^<_{i+1,i+1} - g^<_i V_i^H G_{i+1,i+1}^H.)
The cross terms Y and (g L)^H come from splitting G^< = G Sigma^< G^H at the cut (i, i+1): the
rows of G through slice i are g^(i) - P G_{i+1,.} (g^(i) the inverse of slices 0..i), and a
block-tridiagonal Sigma^< couples the two sides only through L_i and -L_i^H.
Greater function on the returned blocks: G^> = G^< + G^R - G^A (this is G^R Sigma^> G^A when
Sigma^> - Sigma^< = Sigma^R - Sigma^A, with the broadening acting as Sigma^>_eta = -2 i eta S).

Observables (Sec. II-B: the current I_d and the electron population are derived from G^<):
    current      I_i(E) = 2 Re Tr[(H_{i,i+1} - E S_{i,i+1}) G^<_{i+1,i}],  G^<_{i+1,i} = -(G^<_{i,i+1})^H
    density      n_i(E) = Im Tr G^<_ii
    contacts     I_L(E) = Re Tr[Sigma^<_L G^>_00 - Sigma^>_L G^<_00]   (same on slice N_B-1 for I_R)
    transmission T(E)   = Tr[Gamma_L A_00] - Tr[Gamma_L G_00 Gamma_L G_00^H],  A = i (G - G^H)
    integrated   I_i = sum_E w_E I_i(E),  n_i = sum_E w_E n_i(E) / (2 pi)
Contacts: Gamma = i (Sigma^R - Sigma^R^H), Sigma^< = i f Gamma, Sigma^> = -i (1 - f) Gamma, with f the
Fermi function at (mu_L, kT) / (mu_R, kT).
"""
from __future__ import annotations

import numpy as np

from .leads import fermi, lead_self_energy


def _H(X):
    return X.conj().T


def _contacts(E: float, dev: dict, decim_tol: float, decim_max_iter: int, track_cond=False):
    """Contact self-energies on the two end slices (None when the device has no leads)."""
    leads = dev.get("leads")
    if not leads:
        return None
    eta, kT = dev["eta"], dev["kT"]
    out = {}
    for side, mu in (("L", dev["mu_L"]), ("R", dev["mu_R"])):
        r = lead_self_energy(E, eta, leads["H00_" + side], leads["H01_" + side], decim_tol,
                             decim_max_iter, track_cond)
        SR, it, conv = r[0], r[1], r[2]
        kappa = r[3] if track_cond else None
        gam = 1j * (SR - _H(SR))
        f = fermi(E, mu, kT)
        out[side] = dict(SigR=SR, Gamma=gam, SigL=1j * f * gam, SigG=-1j * (1.0 - f) * gam,
                         sweeps=it, converged=conv, kappa=kappa)
    return out


def _scattering(dev: dict, key: str, e_index: int, i: int):
    S = dev.get(key)
    if S is None:
        return None
    return S[e_index if S.shape[0] > 1 else 0, i]


def rgf_energy(E: float, dev: dict, e_index: int = 0, decim_tol: float = 1e-13,
               decim_max_iter: int = 100, track_cond: bool = False) -> dict:
    """Selected blocks and observables at one energy (see the module docstring for every formula)."""
    nb, b = dev["n_blocks"], dev["block_size"]
    eta = dev["eta"]
    z = E + 1j * eta
    eye = np.eye(b, dtype=np.complex128)
    Hd, Hu = dev["H_diag"], dev["H_upper"]
    Sd, Su = dev.get("S_diag"), dev.get("S_upper")
    con = _contacts(E, dev, decim_tol, decim_max_iter, track_cond)

    # Step 1: the block rows of M and the lesser self-energy on each slice.
    A, SigL = [], []
    for i in range(nb):
        Sii = eye if Sd is None else Sd[i]
        a = z * Sii - Hd[i]
        sl = np.zeros((b, b), dtype=np.complex128)
        sr = _scattering(dev, "SigR", e_index, i)
        if sr is not None:
            a = a - sr
        s = _scattering(dev, "SigL", e_index, i)
        if s is not None:
            sl = sl + s
        if con is not None:
            if i == 0:
                a = a - con["L"]["SigR"]
                sl = sl + con["L"]["SigL"]
            if i == nb - 1:
                a = a - con["R"]["SigR"]
                sl = sl + con["R"]["SigL"]
        A.append(a)
        SigL.append(sl)
    U, V, L = [], [], []
    for i in range(nb - 1):
        Sup = np.zeros((b, b), dtype=np.complex128) if Su is None else Su[i]
        u = z * Sup - Hu[i]
        v = z * _H(Sup) - _H(Hu[i])
        sru = _scattering(dev, "SigR_upper", e_index, i)
        srl = _scattering(dev, "SigR_lower", e_index, i)
        slu = _scattering(dev, "SigL_upper", e_index, i)
        if sru is not None:
            u = u - sru
        if srl is not None:
            v = v - srl
        U.append(u)
        V.append(v)
        L.append(np.zeros((b, b), dtype=np.complex128) if slu is None else slu)

    # Step 2: forward sweep (retarded and lesser left-connected functions).
    g = [None] * nb
    gl = [None] * nb
    g[0] = np.linalg.inv(A[0])
    gl[0] = g[0] @ SigL[0] @ _H(g[0])
    for i in range(1, nb):
        g[i] = np.linalg.inv(A[i] - V[i - 1] @ g[i - 1] @ U[i - 1])
        Y = V[i - 1] @ g[i - 1] @ L[i - 1]
        gl[i] = g[i] @ (SigL[i] + V[i - 1] @ gl[i - 1] @ _H(V[i - 1]) - Y + _H(Y)) @ _H(g[i])

    # Step 3: backward sweep for the selected blocks.
    GR = [None] * nb
    GL = [None] * nb
    GRu = [None] * (nb - 1)
    GRl = [None] * (nb - 1)
    GLu = [None] * (nb - 1)
    GR[nb - 1] = g[nb - 1]
    GL[nb - 1] = gl[nb - 1]
    for i in range(nb - 2, -1, -1):
        P = g[i] @ U[i]
        GRu[i] = -P @ GR[i + 1]
        GRl[i] = -GR[i + 1] @ V[i] @ g[i]
        GR[i] = g[i] - P @ GRl[i]
        Q = V[i] @ gl[i] + _H(g[i] @ L[i])
        K = P @ GR[i + 1] @ Q
        GL[i] = gl[i] + P @ GL[i + 1] @ _H(P) + K - _H(K)
        GLu[i] = -P @ GL[i + 1] + _H(GR[i + 1] @ Q)

    # Step 4: greater function on the returned blocks.
    GG = [GL[i] + GR[i] - _H(GR[i]) for i in range(nb)]
    GGu = [GLu[i] + GRu[i] - _H(GRl[i]) for i in range(nb - 1)]

    def stk(lst):
        return np.stack(lst) if lst else np.zeros((0, b, b), dtype=np.complex128)

    out = dict(GR_diag=stk(GR), GR_upper=stk(GRu), GR_lower=stk(GRl), GL_diag=stk(GL),
               GL_upper=stk(GLu), GG_diag=stk(GG), GG_upper=stk(GGu))
    out.update(observables(E, dev, out, con))
    if con is not None:
        out["lead_SigR"] = (con["L"]["SigR"], con["R"]["SigR"])
        out["lead_SigL"] = (con["L"]["SigL"], con["R"]["SigL"])
        out["decim_sweeps"] = (con["L"]["sweeps"], con["R"]["sweeps"])
        out["decim_converged"] = con["L"]["converged"] and con["R"]["converged"]
        if track_cond:
            out["decim_cond"] = max(con["L"]["kappa"], con["R"]["kappa"])
    return out


def observables(E: float, dev: dict, blk: dict, con) -> dict:
    """Current, density, contact currents and transmission from the selected blocks."""
    nb, b = dev["n_blocks"], dev["block_size"]
    Hu, Su = dev["H_upper"], dev.get("S_upper")
    current = np.zeros(max(nb - 1, 0))
    for i in range(nb - 1):
        X = Hu[i] if Su is None else Hu[i] - E * Su[i]
        GL_lo = -_H(blk["GL_upper"][i])
        current[i] = 2.0 * np.real(np.trace(X @ GL_lo))
    density = np.array([np.imag(np.trace(blk["GL_diag"][i])) for i in range(nb)])
    out = dict(current=current, density=density)
    if con is not None:
        cL, cR = con["L"], con["R"]
        IL = np.real(np.trace(cL["SigL"] @ blk["GG_diag"][0] - cL["SigG"] @ blk["GL_diag"][0]))
        IR = np.real(np.trace(cR["SigL"] @ blk["GG_diag"][nb - 1]
                              - cR["SigG"] @ blk["GL_diag"][nb - 1]))
        G00 = blk["GR_diag"][0]
        A00 = 1j * (G00 - _H(G00))
        gam = cL["Gamma"]
        T = np.real(np.trace(gam @ A00) - np.trace(gam @ G00 @ gam @ _H(G00)))
        out.update(contact=np.array([IL, IR]), transmission=T)
    return out


def integrate(current_E: np.ndarray, density_E: np.ndarray, weights: np.ndarray):
    """Energy integrals: I_i = sum_E w_E I_i(E) and n_i = sum_E w_E n_i(E) / (2 pi)."""
    w = np.asarray(weights, dtype=np.float64)
    return w @ current_E, (w @ density_E) / (2.0 * np.pi)


def solve(dev: dict, energy_indices=None, weights=None, decim_tol: float = 1e-13,
          decim_max_iter: int = 100, keep_blocks: bool = True, track_cond: bool = False) -> dict:
    """Run ``rgf_energy`` over the device's energy grid (or the listed indices) and stack results.

    ``weights`` (per listed energy) default to the trapezoid rule on the full grid restricted to
    the listed indices."""
    energies = dev["energies"]
    idx = np.arange(energies.size) if energy_indices is None else np.asarray(energy_indices)
    res = [rgf_energy(float(energies[k]), dev, int(k), decim_tol, decim_max_iter, track_cond)
           for k in idx]
    out = {}
    keys = ["current", "density"] + (["contact", "transmission"] if dev.get("leads") else [])
    if keep_blocks:
        keys += ["GR_diag", "GR_upper", "GR_lower", "GL_diag", "GL_upper", "GG_diag", "GG_upper"]
    for k in keys:
        out[k] = np.stack([np.asarray(r[k]) for r in res])
    if weights is None:
        from workloads import trapezoid_weights
        weights = trapezoid_weights(energies)[idx]
    out["current_int"], out["density_int"] = integrate(out["current"], out["density"], weights)
    if dev.get("leads"):
        out["decim_sweeps"] = np.array([r["decim_sweeps"] for r in res])
        if track_cond:
            out["decim_cond"] = np.array([r["decim_cond"] for r in res])
    return out

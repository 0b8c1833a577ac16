"""Extended-precision restatement of the RGF selected solve for ballistic devices with contacts --
test infrastructure (see the package header); it produces reference values, never a product result.

Why it exists: at the strip's band-edge energies the decimation's inverted blocks (z - eps) reach
condition numbers ~3e4, so two correct FP64 evaluations of the same formulas (e.g. with different
inverse algorithms) already differ by ~1e-9.  An FP64 result is then judged by its distance from the
exact value, which this module approximates in numpy's extended precision (np.clongdouble: a 64-bit
significand on x86, so ~2^-64 rounding, 2^11 below FP64's).

It follows the same steps as ``oracle.leads`` and ``oracle.rgf`` (paper Sec. II-A, Eq. 2 with Table I's
G-row; contacts by Lopez Sancho-Rubio decimation) for a device with S = I, no scattering
self-energies and two contacts, with its own Gauss-Jordan inverse (partial pivoting on the largest
modulus) in place of LAPACK.  Every number is converted from binary64 once, so the inputs are exactly
those the FP64 paths see.
"""
from __future__ import annotations

import numpy as np

LD = np.clongdouble


def _inv(A):
    """Inverse by Gauss-Jordan elimination on [A | I] with partial (row) pivoting."""
    n = A.shape[0]
    M = np.concatenate([A.astype(LD), np.eye(n, dtype=LD)], axis=1)
    for k in range(n):
        p = k + int(np.argmax(np.abs(M[k:, k])))
        if p != k:
            M[[k, p]] = M[[p, k]]
        M[k] = M[k] / M[k, k]
        f = M[:, k].copy()
        f[k] = 0
        M -= np.outer(f, M[k])
    return M[:, n:]


def _H(X):
    return X.conj().T


def _fermi(E, mu, kT):
    x = (np.longdouble(E) - np.longdouble(mu)) / np.longdouble(kT)
    if x > 0:
        ex = np.exp(-x)
        return ex / (1 + ex)
    return 1 / (1 + np.exp(x))


def lead_self_energy(E, eta, H00, H01, tol=1e-13, max_iter=100):
    """Sigma^R = H01 g_s H01^H with the decimation of ``oracle.leads.sancho_rubio`` (same stopping
    rule) in extended precision."""
    b = H00.shape[0]
    z = LD(complex(E, eta))
    eye = np.eye(b, dtype=LD)
    H01 = H01.astype(LD)
    alpha, beta = H01.copy(), _H(H01).copy()
    eps_s, eps = H00.astype(LD), H00.astype(LD)
    scale = np.abs(H01).max()
    for _ in range(max_iter):
        g = _inv(z * eye - eps)
        agb = alpha @ g @ beta
        bga = beta @ g @ alpha
        eps_s = eps_s + agb
        eps = eps + agb + bga
        alpha = alpha @ g @ alpha
        beta = beta @ g @ beta
        if max(np.abs(alpha).max(), np.abs(beta).max()) < tol * scale:
            break
    gs = _inv(z * eye - eps_s)
    return H01 @ gs @ _H(H01)


def rgf_energy(E, dev):
    """Selected blocks and observables at one energy for a ballistic device with contacts (S = I, no
    scattering self-energies): every block kind (G^R diagonal, upper, lower; G^< diagonal, upper; G^>
    = G^< + G^R - G^A diagonal and upper) and current, density, contact currents, transmission, as in
    ``oracle.rgf`` (formulas in its module docstring)."""
    assert dev.get("leads") and dev.get("SigR") is None and dev.get("S_diag") is None
    nb, b = dev["n_blocks"], dev["block_size"]
    eta, kT = dev["eta"], dev["kT"]
    z = LD(complex(E, eta))
    eye = np.eye(b, dtype=LD)
    L = dev["leads"]
    con = {}
    for side, mu in (("L", dev["mu_L"]), ("R", dev["mu_R"])):
        SR = lead_self_energy(E, eta, L["H00_" + side], L["H01_" + side])
        gam = 1j * (SR - _H(SR))
        f = _fermi(E, mu, kT)
        con[side] = dict(SigR=SR, Gamma=gam, SigL=1j * f * gam, SigG=-1j * (1 - f) * gam)
    A = [z * eye - dev["H_diag"][i].astype(LD) for i in range(nb)]
    A[0] = A[0] - con["L"]["SigR"]
    A[nb - 1] = A[nb - 1] - con["R"]["SigR"]
    U = [-dev["H_upper"][i].astype(LD) for i in range(nb - 1)]
    V = [_H(-dev["H_upper"][i].astype(LD)) for i in range(nb - 1)]
    SL = [np.zeros((b, b), LD) for _ in range(nb)]
    SL[0] = SL[0] + con["L"]["SigL"]
    SL[nb - 1] = SL[nb - 1] + con["R"]["SigL"]
    g, gl = [None] * nb, [None] * nb
    for i in range(nb):
        Ai = A[i] if i == 0 else A[i] - V[i - 1] @ g[i - 1] @ U[i - 1]
        g[i] = _inv(Ai)
        br = SL[i] if i == 0 else SL[i] + V[i - 1] @ gl[i - 1] @ _H(V[i - 1])
        gl[i] = g[i] @ br @ _H(g[i])
    G, GL = [None] * nb, [None] * nb
    GLu, GRu, GRl = [None] * (nb - 1), [None] * (nb - 1), [None] * (nb - 1)
    G[nb - 1], GL[nb - 1] = g[nb - 1], gl[nb - 1]
    for i in range(nb - 2, -1, -1):
        P = g[i] @ U[i]
        GRl[i] = -G[i + 1] @ V[i] @ g[i]
        GRu[i] = -P @ G[i + 1]
        G[i] = g[i] - P @ GRl[i]
        Q = V[i] @ gl[i]
        K = P @ G[i + 1] @ Q
        GL[i] = gl[i] + P @ GL[i + 1] @ _H(P) + K - _H(K)
        GLu[i] = -P @ GL[i + 1] + _H(G[i + 1] @ Q)
    cur = np.array([2 * np.real(np.trace(dev["H_upper"][i].astype(LD) @ (-_H(GLu[i])))) for i in range(nb - 1)])
    den = np.array([np.imag(np.trace(GL[i])) for i in range(nb)])
    contact = []
    for side, k in (("L", 0), ("R", nb - 1)):
        GG = GL[k] + G[k] - _H(G[k])
        contact.append(np.real(np.trace(con[side]["SigL"] @ GG - con[side]["SigG"] @ GL[k])))
    gam = con["L"]["Gamma"]
    A00 = 1j * (G[0] - _H(G[0]))
    T = np.real(np.trace(gam @ A00) - np.trace(gam @ G[0] @ gam @ _H(G[0])))
    GG = [GL[i] + G[i] - _H(G[i]) for i in range(nb)]
    GGu = [GLu[i] + GRu[i] - _H(GRl[i]) for i in range(nb - 1)]
    stk = lambda lst: np.stack(lst) if lst else np.zeros((0, b, b), LD)  # noqa: E731
    return dict(GR_diag=stk(G), GR_upper=stk(GRu), GR_lower=stk(GRl), GL_diag=stk(GL), GL_upper=stk(GLu),
                GG_diag=stk(GG), GG_upper=stk(GGu), current=cur, density=den, contact=np.array(contact),
                transmission=T)

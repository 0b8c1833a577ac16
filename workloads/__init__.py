"""Seeded synthetic inputs for the RGF selected inversion (shared by the CUDA path's tests and the oracle).

This module draws random numbers and lays blocks out; it holds none of the method's arithmetic
(no Green's functions, no lead self-energies, no observables).  Both the oracle and the GPU tests
import it, so every parity comparison runs on byte-identical inputs.

Layout of a device (all numpy, complex128, row-major, C-contiguous):

* ``H_diag``  [N_B][b][b]     Hermitian diagonal blocks H_ii.
* ``H_upper`` [N_B-1][b][b]   coupling blocks H_{i,i+1}; H_{i+1,i} = H_{i,i+1}^H is implied.
* ``S_diag`` / ``S_upper``    overlap blocks, or ``None`` for S = I.
* ``SigR``, ``SigL``          [N_S][N_B][b][b] block-diagonal scattering self-energies (N_S = 1:
                              one set shared by every energy), or ``None`` for a ballistic device.
                              The greater self-energy is implied by Sigma^> = Sigma^< + Sigma^R - Sigma^A.
* ``leads``                   ``None`` or dict(H00_L, H01_L, H00_R, H01_R): principal layer and the
                              coupling from a lead cell to the next cell further from the device; the
                              device's end slice couples to the first lead cell by the same H01.
* ``energies``                [N_E] float64 grid;  ``eta``, ``mu_L``, ``mu_R``, ``kT`` scalars.

Recipes (seeded with ``numpy.random.default_rng(seed)``; draw order is part of the recipe):

* ``strip`` -- square-lattice tight-binding strip (width W orbitals per slice, hopping t).
  Onsite energies U[-w, w] drawn slice-major, one row of W per slice.  Leads are clean strips
  of the same width with onsite 0.
* ``random_device`` -- dense random blocks: per slice i, X with Re, Im ~ N(0, 1/(2b)),
  H_ii = (X + X^H)/sqrt(2) + diag(U[-1,1]); then per coupling i, H_{i,i+1} complex Gaussian
  of total variance c/b; then per slice, A and B complex N(0, 1/b) and
  Sigma^< = i s A A^H, Sigma^> = -i s B B^H, Sigma^R = (Sigma^> - Sigma^<)/2 (so that
  Sigma^R - Sigma^A = Sigma^> - Sigma^< holds exactly).
"""
from __future__ import annotations

import numpy as np

__all__ = ["strip", "random_device", "uneven_batch", "serving_requests", "trapezoid_weights",
           "nrl_device", "w_system", "STRIP_CFG", "MIXED_CFG", "UNEVEN_NB", "UNEVEN_B", "OZAKI_CFG",
           "NRL_CFG", "WSYS_CFG"]

# The five synthetic workloads (sizes only; the generators below draw the values).
STRIP_CFG = dict(W=16, n_blocks=32, t=-1.0, disorder=0.25, eta=1e-6, mu_L=0.1, mu_R=-0.1,
                 kT=0.025, n_energies=64, e_lo=-3.5, e_hi=3.5)
MIXED_CFG = dict(b=256, n_blocks=64, n_energies=512, e_lo=-2.0, e_hi=2.0)
UNEVEN_NB = (16, 24, 32, 48, 64, 96, 112, 128)
UNEVEN_B = (128, 192, 256, 384, 512)
OZAKI_CFG = dict(b=1024, n_blocks=32, n_energies=256, e_lo=-2.0, e_hi=2.0)
# the paper's large nanoribbon device shape (b = 3408, N_B = 10), energies streamed in small chunks
NRL_CFG = dict(b=3408, n_blocks=10, n_energies=4, e_lo=-1.0, e_hi=1.0)
# screened-Coulomb (W) system: per-energy polarisation blocks
WSYS_CFG = dict(b=256, n_blocks=32, n_energies=64)


def _chain(W: int, t: float) -> np.ndarray:
    """Nearest-neighbour chain of W sites with hopping t and hard walls."""
    h = np.zeros((W, W), dtype=np.complex128)
    idx = np.arange(W - 1)
    h[idx, idx + 1] = t
    h[idx + 1, idx] = t
    return h


def strip(W: int = 16, n_blocks: int = 32, t: float = -1.0, disorder: float = 0.25,
          eta: float = 1e-6, mu_L: float = 0.1, mu_R: float = -0.1, kT: float = 0.025,
          n_energies: int = 64, e_lo: float = -3.5, e_hi: float = 3.5, seed: int = 0,
          energies: np.ndarray | None = None) -> dict:
    """Disordered square-lattice strip between two clean semi-infinite strips of the same width."""
    rng = np.random.default_rng(seed)
    onsite = rng.uniform(-disorder, disorder, size=(n_blocks, W)) if disorder > 0 else \
        np.zeros((n_blocks, W))
    chain = _chain(W, t)
    H_diag = np.empty((n_blocks, W, W), dtype=np.complex128)
    for i in range(n_blocks):
        H_diag[i] = chain + np.diag(onsite[i])
    H_upper = np.broadcast_to(t * np.eye(W, dtype=np.complex128), (n_blocks - 1, W, W)).copy()
    leads = dict(H00_L=chain.copy(), H01_L=t * np.eye(W, dtype=np.complex128),
                 H00_R=chain.copy(), H01_R=t * np.eye(W, dtype=np.complex128))
    if energies is None:
        energies = np.linspace(e_lo, e_hi, n_energies)
    return dict(n_blocks=n_blocks, block_size=W, H_diag=H_diag, H_upper=H_upper,
                S_diag=None, S_upper=None, SigR=None, SigL=None, leads=leads,
                energies=np.asarray(energies, dtype=np.float64), eta=eta, mu_L=mu_L, mu_R=mu_R,
                kT=kT)


def _cgauss(rng: np.random.Generator, shape, var: float) -> np.ndarray:
    """Complex Gaussian with E|x|^2 = var (real and imaginary parts each var/2)."""
    s = np.sqrt(var / 2.0)
    return (rng.standard_normal(shape) * s) + 1j * (rng.standard_normal(shape) * s)


def random_device(b: int, n_blocks: int, n_energies: int = 8, e_lo: float = -2.0,
                  e_hi: float = 2.0, seed: int = 0, coupling_var: float = 0.3,
                  sigma_scale: float = 1e-2, eta: float = 1e-6, scattering: bool = True,
                  energies: np.ndarray | None = None, offdiag_sigma: bool = False) -> dict:
    """Dense random block-tridiagonal device with block-diagonal scattering self-energies.

    ``offdiag_sigma``: block-tridiagonal self-energies instead.  Sigma^< = i s F F^H and
    Sigma^> = -i s G G^H with F, G block-lower-bidiagonal (diagonal blocks as in the
    block-diagonal case, sub-diagonal blocks complex Gaussian of variance 1/b from a second
    generator), so both are block-tridiagonal, anti-Hermitian and of definite sign; Sigma^R =
    (Sigma^> - Sigma^<) / 2 on every block.  Adds SigR_upper (Sigma^R_{i,i+1}), SigR_lower
    (Sigma^R_{i+1,i}) and SigL_upper (Sigma^<_{i,i+1}; Sigma^<_{i+1,i} = -(Sigma^<_{i,i+1})^H),
    each [1][N_B-1][b][b]."""
    rng = np.random.default_rng(seed)
    H_diag = np.empty((n_blocks, b, b), dtype=np.complex128)
    for i in range(n_blocks):
        X = _cgauss(rng, (b, b), 1.0 / b)
        H_diag[i] = (X + X.conj().T) / np.sqrt(2.0) + np.diag(rng.uniform(-1.0, 1.0, size=b))
    H_upper = np.empty((max(n_blocks - 1, 0), b, b), dtype=np.complex128)
    for i in range(n_blocks - 1):
        H_upper[i] = _cgauss(rng, (b, b), coupling_var / b)
    SigR = SigL = None
    extra = {}
    if scattering:
        SigL = np.empty((1, n_blocks, b, b), dtype=np.complex128)
        SigG = np.empty((1, n_blocks, b, b), dtype=np.complex128)
        FA, FB = [], []
        for i in range(n_blocks):
            A = _cgauss(rng, (b, b), 1.0 / b)
            B = _cgauss(rng, (b, b), 1.0 / b)
            FA.append(A)
            FB.append(B)
            SigL[0, i] = 1j * sigma_scale * (A @ A.conj().T)
            SigG[0, i] = -1j * sigma_scale * (B @ B.conj().T)
        SigR = (SigG - SigL) / 2.0
        if offdiag_sigma:
            rng2 = np.random.default_rng(seed + 104729)
            nu = max(n_blocks - 1, 0)
            SLu = np.empty((1, nu, b, b), dtype=np.complex128)
            SGu = np.empty((1, nu, b, b), dtype=np.complex128)
            for i in range(nu):
                CA = _cgauss(rng2, (b, b), 1.0 / b)   # F_{i+1,i}
                CB = _cgauss(rng2, (b, b), 1.0 / b)   # G_{i+1,i}
                SigL[0, i + 1] += 1j * sigma_scale * (CA @ CA.conj().T)
                SigG[0, i + 1] += -1j * sigma_scale * (CB @ CB.conj().T)
                SLu[0, i] = 1j * sigma_scale * (FA[i] @ CA.conj().T)
                SGu[0, i] = -1j * sigma_scale * (FB[i] @ CB.conj().T)
            SigR = (SigG - SigL) / 2.0
            SRu = (SGu - SLu) / 2.0
            extra = dict(SigR_upper=SRu, SigR_lower=-np.conj(np.swapaxes(SRu, -1, -2)),
                         SigL_upper=SLu)
    if energies is None:
        energies = np.linspace(e_lo, e_hi, n_energies)
    dev = dict(n_blocks=n_blocks, block_size=b, H_diag=H_diag, H_upper=H_upper,
               S_diag=None, S_upper=None, SigR=SigR, SigL=SigL, leads=None,
               energies=np.asarray(energies, dtype=np.float64), eta=eta, mu_L=0.0, mu_R=0.0,
               kT=0.025)
    dev.update(extra)
    return dev


def nrl_device(b: int = 3408, n_blocks: int = 10, n_energies: int = 4, e_lo: float = -1.0,
               e_hi: float = 1.0, seed: int = 0, rank: int = 32, sigma_scale: float = 1e-2,
               eta: float = 1e-6) -> dict:
    """Device with the block shape of the paper's large nanoribbon (b = 3408, N_B = 10): H as in
    ``random_device``; per-energy scattering self-energies Sigma^< = i s (A A^H + I/b), Sigma^> =
    -i s (B B^H + I/b) with A, B of rank ``rank`` (complex Gaussian, variance 1/rank) and a smooth
    energy dependence (1 + 0.1 k / N_E at energy k), Sigma^R = (Sigma^> - Sigma^<) / 2.  Arrays are
    [N_E][N_B][b][b] (complex128, about 2 N_E N_B b^2 16 bytes for the two self-energies)."""
    rng = np.random.default_rng(seed)
    H_diag = np.empty((n_blocks, b, b), dtype=np.complex128)
    for i in range(n_blocks):
        X = _cgauss(rng, (b, b), 1.0 / b)
        H_diag[i] = (X + X.conj().T) / np.sqrt(2.0) + np.diag(rng.uniform(-1.0, 1.0, size=b))
    H_upper = np.stack([_cgauss(rng, (b, b), 0.3 / b) for _ in range(n_blocks - 1)]) if n_blocks > 1 \
        else np.zeros((0, b, b), np.complex128)
    SigL = np.empty((n_energies, n_blocks, b, b), dtype=np.complex128)
    SigR = np.empty((n_energies, n_blocks, b, b), dtype=np.complex128)
    eye = np.eye(b) / b
    for i in range(n_blocks):
        A = _cgauss(rng, (b, rank), 1.0 / rank)
        B = _cgauss(rng, (b, rank), 1.0 / rank)
        sl = 1j * sigma_scale * (A @ A.conj().T + eye)
        sg = -1j * sigma_scale * (B @ B.conj().T + eye)
        for k in range(n_energies):
            f = 1.0 + 0.1 * k / max(n_energies, 1)
            SigL[k, i] = f * sl
            SigR[k, i] = f * (sg - sl) / 2.0
    return dict(n_blocks=n_blocks, block_size=b, H_diag=H_diag, H_upper=H_upper, S_diag=None,
                S_upper=None, SigR=SigR, SigL=SigL, leads=None,
                energies=np.linspace(e_lo, e_hi, n_energies), eta=eta, mu_L=0.0, mu_R=0.0, kT=0.025)


def w_system(b: int, n_blocks: int, n_energies: int = 4, seed: int = 0, v_scale: float = 1.0,
             p_scale: float = 4.0) -> dict:
    """Screened-Coulomb system inputs (Table I, W row): a Hermitian BT Coulomb matrix V and per-energy
    BT polarisations.  V_ii = I + v (X + X^H) / (2 sqrt(b)), V_{i,i+1} = v Y / (2 sqrt(b)) (complex
    Gaussian X, Y of unit variance); P^< = i p F F^H and P^> = -i p G G^H with F, G block-lower-
    bidiagonal (complex Gaussian blocks of variance 1/b), scaled by (1 + 0.5 k / N_E) at energy k;
    P^R = (P^> - P^<) / 2 on every block.  With the default scales kappa(M) is 1e2 - 1e3, the range
    the paper reports for W systems (Sec. IV).  Arrays: V_diag [N_B][b][b], V_upper [N_B-1][b][b];
    PR_diag [N_E][N_B][b][b], PR_upper / PR_lower / PL_upper / PG_upper [N_E][N_B-1][b][b],
    PL_diag / PG_diag [N_E][N_B][b][b]."""
    rng = np.random.default_rng(seed)
    nu = max(n_blocks - 1, 0)
    V_diag = np.empty((n_blocks, b, b), np.complex128)
    for i in range(n_blocks):
        X = _cgauss(rng, (b, b), 1.0)
        V_diag[i] = np.eye(b) + v_scale * (X + X.conj().T) / (2.0 * np.sqrt(b))
    V_upper = np.stack([v_scale * _cgauss(rng, (b, b), 1.0) / (2.0 * np.sqrt(b)) for _ in range(nu)]) \
        if nu else np.zeros((0, b, b), np.complex128)
    out = {}
    for key, sgn in (("PL", 1j), ("PG", -1j)):
        D = [_cgauss(rng, (b, b), 1.0 / b) for _ in range(n_blocks)]
        Lo = [_cgauss(rng, (b, b), 1.0 / b) for _ in range(nu)]
        d0 = np.stack([D[i] @ D[i].conj().T + (Lo[i - 1] @ Lo[i - 1].conj().T if i > 0 else 0)
                       for i in range(n_blocks)])
        u0 = np.stack([D[i] @ Lo[i].conj().T for i in range(nu)]) if nu else np.zeros((0, b, b), np.complex128)
        f = (1.0 + 0.5 * np.arange(n_energies) / max(n_energies, 1))[:, None, None, None]
        out[key + "_diag"] = sgn * p_scale * f * d0[None]
        out[key + "_upper"] = sgn * p_scale * f * u0[None]
    out["PR_diag"] = (out["PG_diag"] - out["PL_diag"]) / 2.0
    out["PR_upper"] = (out["PG_upper"] - out["PL_upper"]) / 2.0
    out["PR_lower"] = -np.conj(np.swapaxes(out["PR_upper"], -1, -2))
    out.update(n_blocks=n_blocks, block_size=b, n_energies=n_energies, V_diag=V_diag, V_upper=V_upper)
    return out


def uneven_batch(n_energies: int = 128, seed: int = 0, nb_list=UNEVEN_NB, b_list=UNEVEN_B,
                 scale: float = 1.0) -> list:
    """Eight devices: device k has N_B = nb_list[k] and b = b_list[k mod len(b_list)].

    ``scale`` < 1 shrinks every b and N_B (kept >= 2) for tests that must finish on a CPU.
    """
    devs = []
    for k, nb in enumerate(nb_list):
        b = b_list[k % len(b_list)]
        if scale != 1.0:
            b = max(2, int(round(b * scale)))
            nb = max(2, int(round(nb * scale)))
        devs.append(random_device(b, nb, n_energies=n_energies, seed=seed + k))
    return devs


def serving_requests(n_requests: int, rate_hz: float = 200.0, seed: int = 1,
                     b_choices=(64, 128, 256, 512), nb_range=(16, 96), ne_choices=(32, 64, 128)):
    """Poisson arrival times and per-request shapes/precision tags (no blocks: those come from
    ``random_device`` with the request's seed)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=n_requests)
    t = np.cumsum(gaps)
    reqs = []
    for r in range(n_requests):
        b = int(rng.choice(b_choices))
        nb = int(rng.integers(nb_range[0], nb_range[1] + 1))
        ne = int(rng.choice(ne_choices))
        tag = "c64" if rng.random() < 0.5 else "emu64"
        reqs.append(dict(t_arrival=float(t[r]), b=b, n_blocks=nb, n_energies=ne, precision=tag,
                         seed=1000 + r))
    return reqs


def trapezoid_weights(energies: np.ndarray) -> np.ndarray:
    """Trapezoid-rule weights of an energy grid (length-1 grid: weight 0)."""
    e = np.asarray(energies, dtype=np.float64)
    w = np.zeros_like(e)
    if e.size > 1:
        d = np.diff(e)
        w[:-1] += d / 2.0
        w[1:] += d / 2.0
    return w

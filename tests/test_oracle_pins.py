"""Pins for the FP64 oracle: each test checks it against something other than itself.

* brute-force dense inversion (Eq. 2 with Table I's G-row) on tiny random inputs, with overlap,
  contacts, non-symmetric lead couplings, energy-dependent and block-tridiagonal self-energies;
* the closed-form self-energy and Green's function of a clean tight-binding strip;
* a long truncated lead solved densely (orientation of the lead coupling);
* the clean strip's integer transmission and Landauer current;
* closed forms of the Fermi function, the trapezoid weights, the integrated current of a clean
  chain and the integrated density of a broadened level;
* invariants: anti-Hermitian G^<, PSD spectral function, exact current continuity, and the
  equilibrium (fluctuation-dissipation) case with zero current.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle.dense import dense_selected

BLOCKS = ("GR_diag", "GR_upper", "GR_lower", "GL_diag", "GL_upper", "GG_diag", "GG_upper")


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _herm(rng, b, s=1.0):
    X = rng.standard_normal((b, b)) + 1j * rng.standard_normal((b, b))
    return s * (X + X.conj().T) / 2


def _cplx(rng, b, s=1.0):
    return s * (rng.standard_normal((b, b)) + 1j * rng.standard_normal((b, b)))


def _with_leads_and_overlap(dev, rng, overlap=True):
    b = dev["block_size"]
    nb = dev["n_blocks"]
    dev["leads"] = dict(H00_L=_herm(rng, b), H01_L=_cplx(rng, b, 0.4),
                        H00_R=_herm(rng, b), H01_R=_cplx(rng, b, 0.4))
    if overlap:
        dev["S_diag"] = np.stack([np.eye(b) + _herm(rng, b, 0.05) for _ in range(nb)])
        dev["S_upper"] = np.stack([_cplx(rng, b, 0.03) for _ in range(nb - 1)]) if nb > 1 else \
            np.zeros((0, b, b), np.complex128)
    dev["eta"] = 1e-3
    dev["mu_L"], dev["mu_R"], dev["kT"] = 0.3, -0.2, 0.05
    return dev


def _at(dev, key, k):
    X = dev.get(key)
    return None if X is None else X[k if X.shape[0] > 1 else 0]


def _dense_for(dev, E, k=0, r=None):
    if r is None:
        r = O.rgf_energy(E, dev, k)
    d = dense_selected(E, dev["eta"], dev["H_diag"], dev["H_upper"], dev.get("S_diag"),
                       dev.get("S_upper"), _at(dev, "SigR", k), _at(dev, "SigL", k),
                       lead_SigR=r.get("lead_SigR", (None, None)),
                       lead_SigL=r.get("lead_SigL", (None, None)),
                       SigR_upper=_at(dev, "SigR_upper", k), SigR_lower=_at(dev, "SigR_lower", k),
                       SigL_upper=_at(dev, "SigL_upper", k))
    return r, d


@pytest.mark.parametrize("b,nb,seed", [(4, 5, 1), (3, 8, 2), (5, 2, 3), (6, 1, 4)])
def test_recursion_matches_dense_inverse(b, nb, seed):
    """Every selected block of G^R, G^<, G^> equals the dense definition (Eq. 2, Table I)."""
    rng = np.random.default_rng(100 + seed)
    dev = _with_leads_and_overlap(W.random_device(b, nb, n_energies=3, seed=seed), rng)
    for E in (-1.3, 0.07, 0.9):
        r, d = _dense_for(dev, E)
        for key in BLOCKS:
            if d[key].size:
                assert _rel(r[key], d[key]) < 1e-11, (key, E)


def test_recursion_energy_dependent_sigma():
    """A per-energy scattering self-energy is read at its own energy index."""
    rng = np.random.default_rng(7)
    dev = W.random_device(4, 4, n_energies=3, seed=5)
    dev["SigR"] = np.concatenate([dev["SigR"] * (1.0 + 0.5 * k) for k in range(3)])
    dev["SigL"] = np.concatenate([dev["SigL"] * (1.0 + 0.25 * k) for k in range(3)])
    for k, E in enumerate(dev["energies"]):
        r, d = _dense_for(dev, float(E), k)
        for key in BLOCKS:
            assert _rel(r[key], d[key]) < 1e-11
    del rng


@pytest.mark.parametrize("b,nb,seed", [(4, 5, 11), (3, 7, 12), (5, 2, 13), (4, 1, 14)])
@pytest.mark.parametrize("parts", ["all", "lesser_only", "retarded_only"])
def test_recursion_block_tridiagonal_sigma_matches_dense(b, nb, seed, parts):
    """Block-tridiagonal scattering self-energies: every selected block equals the dense definition
    with the full Sigma^R and Sigma^< matrices -- with only the lesser off-diagonal blocks (which
    exercise the cross terms Y and (g L)^H alone), only the retarded ones (which enter U and V), or
    both; with overlap and contacts."""
    rng = np.random.default_rng(200 + seed)
    dev = _with_leads_and_overlap(W.random_device(b, nb, n_energies=3, seed=seed, offdiag_sigma=True), rng)
    if parts == "lesser_only":
        dev["SigR_upper"] = dev["SigR_lower"] = None
    elif parts == "retarded_only":
        dev["SigL_upper"] = None
    for E in (-1.1, 0.13, 0.8):
        r, d = _dense_for(dev, E)
        for key in BLOCKS:
            if d[key].size:
                assert _rel(r[key], d[key]) < 1e-11, (key, E)


def test_block_tridiagonal_sigma_changes_the_result():
    """The off-diagonal self-energy blocks matter at the level the pins resolve: dropping them
    moves G^< by far more than the 1e-11 agreement above."""
    dev = W.random_device(4, 5, n_energies=1, seed=21, offdiag_sigma=True)
    full = O.rgf_energy(0.2, dev)
    cut = dict(dev, SigL_upper=None, SigR_upper=None, SigR_lower=None)
    part = O.rgf_energy(0.2, cut)
    assert _rel(part["GL_diag"], full["GL_diag"]) > 1e-4
    assert _rel(part["GL_upper"], full["GL_upper"]) > 1e-4


def test_block_tridiagonal_sigma_energy_dependent():
    """Per-energy off-diagonal self-energies are read at their own energy index."""
    dev = W.random_device(3, 4, n_energies=3, seed=22, offdiag_sigma=True)
    for key in ("SigR", "SigL", "SigR_upper", "SigR_lower", "SigL_upper"):
        dev[key] = np.concatenate([dev[key] * (1.0 + 0.3 * k) for k in range(3)])
    for k, E in enumerate(dev["energies"]):
        r, d = _dense_for(dev, float(E), k)
        for key in BLOCKS:
            assert _rel(r[key], d[key]) < 1e-11


def test_single_slice_is_plain_inverse():
    """N_B = 1: G^R is the inverse of the one block and G^< = G Sigma^< G^H."""
    dev = W.random_device(7, 1, n_energies=1, seed=11)
    E = 0.3
    r = O.rgf_energy(E, dev)
    A = (E + 1j * dev["eta"]) * np.eye(7) - dev["H_diag"][0] - dev["SigR"][0, 0]
    G = np.linalg.inv(A)
    assert _rel(r["GR_diag"][0], G) < 1e-13
    assert _rel(r["GL_diag"][0], G @ dev["SigL"][0, 0] @ G.conj().T) < 1e-13


# ---------------------------------------------------------------- clean strip closed forms
def _sqrt_branch(zp, t):
    return np.sqrt(zp - 2 * abs(t)) * np.sqrt(zp + 2 * abs(t))


def _strip_modes(W_, t):
    m = np.arange(1, W_ + 1)
    eps = 2 * t * np.cos(m * np.pi / (W_ + 1))
    n = np.arange(1, W_ + 1)
    Umat = np.sqrt(2.0 / (W_ + 1)) * np.sin(np.outer(n, m) * np.pi / (W_ + 1))
    return eps, Umat


def test_decimation_matches_closed_form_strip_self_energy():
    """Sancho-Rubio on a clean strip = mode-resolved 1D-chain self-energy (z'-sqrt)/2."""
    W_, t = 16, -1.0
    s = W.strip(W=W_, n_blocks=2, t=t, disorder=0.0)
    eps, Umat = _strip_modes(W_, t)
    for E in (-3.3, -1.1, 0.05, 0.7, 2.9, 4.5):
        z = E + 1e-8j
        SR, it, conv = O.lead_self_energy(E, 1e-8, s["leads"]["H00_L"], s["leads"]["H01_L"])
        assert conv
        zp = z - eps
        sig = (zp - _sqrt_branch(zp, t)) / 2.0
        ref = Umat @ np.diag(sig) @ Umat.T
        assert np.abs(SR - ref).max() < 1e-9, E


def test_decimation_scalar_chain_outside_band():
    """Outside the band the 1D-chain self-energy is real and decays: (E -+ sqrt(E^2-4t^2))/2."""
    for E in (-3.0, 2.5):
        SR, _, conv = O.lead_self_energy(E, 1e-12, np.zeros((1, 1)), np.array([[1.0 + 0j]]))
        ref = (E - np.sign(E) * np.sqrt(E * E - 4.0)) / 2.0
        assert conv and abs(SR[0, 0] - ref) < 1e-10


def test_lead_orientation_against_truncated_lead():
    """Contacts with a non-symmetric H01 equal explicit long leads solved densely (large eta)."""
    rng = np.random.default_rng(21)
    b, nb, n_lead, eta = 3, 3, 80, 0.25
    dev = W.random_device(b, nb, n_energies=1, seed=9, scattering=False)
    H00L, H01L = _herm(rng, b), _cplx(rng, b, 0.35)
    H00R, H01R = _herm(rng, b), _cplx(rng, b, 0.35)
    dev["leads"] = dict(H00_L=H00L, H01_L=H01L, H00_R=H00R, H01_R=H01R)
    dev["eta"] = eta
    E = 0.4
    r = O.rgf_energy(E, dev)
    # Explicit chain: left lead cells (farthest first), device slices, right lead cells.
    diag = [H00L] * n_lead + list(dev["H_diag"]) + [H00R] * n_lead
    # coupling from the cell at position p to p+1 (left to right)
    up = []
    for _ in range(n_lead - 1):
        up.append(H01L.conj().T)      # left cell n+1 (farther) -> n is H01^H going rightwards
    up.append(H01L.conj().T)          # first left cell -> device slice 0
    up += list(dev["H_upper"])
    up.append(H01R)                   # device slice N-1 -> first right cell
    up += [H01R] * (n_lead - 1)
    d = dense_selected(E, eta, np.stack(diag), np.stack(up))
    sl = slice(n_lead, n_lead + nb)
    assert _rel(r["GR_diag"], d["GR_diag"][sl]) < 1e-9
    assert _rel(r["GR_upper"], d["GR_upper"][n_lead:n_lead + nb - 1]) < 1e-9


def test_clean_strip_ldos_closed_form():
    """Any diagonal block of the clean strip equals the infinite-strip G: U diag(1/sqrt) U^T."""
    W_, t = 16, -1.0
    s = W.strip(W=W_, n_blocks=6, t=t, disorder=0.0, eta=1e-9)
    eps, Umat = _strip_modes(W_, t)
    for E in (-2.7, 0.31, 1.9):
        r = O.rgf_energy(E, s)
        zp = E + 1e-9j - eps
        gb = 1.0 / _sqrt_branch(zp, t)
        ref = Umat @ np.diag(gb) @ Umat.T
        for i in (0, 3, 5):
            assert np.abs(r["GR_diag"][i] - ref).max() < 1e-6, (E, i)


@pytest.mark.parametrize("eta,tol", [(1e-10, 1e-6), (1e-6, 2e-3)])
def test_clean_strip_integer_transmission_and_landauer_current(eta, tol):
    """Clean strip: T(E) = number of open modes; I_i(E) = T (f_L - f_R) on every slice."""
    W_, t = 16, -1.0
    cfg = dict(W.STRIP_CFG)
    s = W.strip(W=W_, n_blocks=8, t=t, disorder=0.0, eta=eta, mu_L=cfg["mu_L"],
                mu_R=cfg["mu_R"], kT=cfg["kT"])
    eps, _ = _strip_modes(W_, t)
    for E in np.linspace(-3.5, 3.5, 64)[::7]:
        r = O.rgf_energy(float(E), s)
        n_open = int(np.sum(np.abs(E - eps) < 2 * abs(t)))
        assert abs(r["transmission"] - n_open) < tol, E
        df = O.fermi(E, cfg["mu_L"], cfg["kT"]) - O.fermi(E, cfg["mu_R"], cfg["kT"])
        assert np.abs(r["current"] - n_open * df).max() < tol * max(1.0, n_open)
        assert abs(r["contact"][0] - n_open * df) < tol * max(1.0, n_open)
        assert abs(r["contact"][1] + n_open * df) < tol * max(1.0, n_open)


def test_current_is_positive_from_high_to_low_chemical_potential():
    s = W.strip(n_blocks=6, disorder=0.0, eta=1e-10)
    r = O.rgf_energy(0.0, s)
    assert np.all(r["current"] > 0.5)


# ---------------------------------------------------------------- invariants
def _random_with_leads(seed=31, b=5, nb=6):
    rng = np.random.default_rng(seed)
    return _with_leads_and_overlap(W.random_device(b, nb, n_energies=4, seed=seed), rng,
                                   overlap=False)


def test_lesser_is_anti_hermitian_and_spectral_function_psd():
    dev = _random_with_leads()
    for E in (-0.8, 0.2, 1.4):
        r = O.rgf_energy(E, dev)
        for i in range(dev["n_blocks"]):
            GLi = r["GL_diag"][i]
            assert np.abs(GLi + GLi.conj().T).max() < 1e-12 * np.abs(GLi).max()
            A = 1j * (r["GR_diag"][i] - r["GR_diag"][i].conj().T)
            assert np.linalg.eigvalsh((A + A.conj().T) / 2).min() > -1e-12
            # n_i(E) >= 0: the electron population is non-negative
            assert r["density"][i] >= -1e-12


def test_exact_current_continuity():
    """I_{i-1} + J_i = I_i with J_i = Re Tr[Sigma^<_ii G^>_ii - Sigma^>_ii G^<_ii] (eta as a sink),
    I_L + J_0 = I_0 and I_{N-2} + J_{N-1} + I_R = 0."""
    dev = _random_with_leads()
    nb = dev["n_blocks"]
    eta = dev["eta"]
    for E in (-0.5, 0.6):
        r = O.rgf_energy(E, dev)
        J = np.zeros(nb)
        for i in range(nb):
            SL = dev["SigL"][0, i]
            SR = dev["SigR"][0, i]
            SG = SL + SR - SR.conj().T - 2j * eta * np.eye(dev["block_size"])
            J[i] = np.real(np.trace(SL @ r["GG_diag"][i] - SG @ r["GL_diag"][i]))
        I = r["current"]
        IL, IR = r["contact"]
        scale = np.abs(I).max()
        assert abs(IL + J[0] - I[0]) < 1e-11 * scale
        for i in range(1, nb - 1):
            assert abs(I[i - 1] + J[i] - I[i]) < 1e-11 * scale
        assert abs(I[nb - 2] + J[nb - 1] + IR) < 1e-11 * scale


def test_exact_current_continuity_with_overlap():
    """With a non-orthogonal basis the bond current is 2 Re Tr[(H - E S)_{i,i+1} G^<_{i+1,i}] and the
    broadening enters as the block-tridiagonal sink -i eta S.  From M G^< - G^< M^H =
    Sigma^< G^A - G^R Sigma^< (M = z S - H - Sigma^R, Sigma^< without an eta part), the trace of the
    (i, i) block gives I_{i-1} + J_i = I_i with
        J_i = Re Tr[Sigma^<_ii G^>_ii - Sigma^>_ii G^<_ii]          (scattering, Sigma^> = Sigma^< + Sigma^R - Sigma^A)
            + Re { i eta sum_{j=i-1..i+1} (Tr[S_ij G^<_ji] + Tr[S_ji G^<_ij]) }   (the eta sink),
    and the contacts close the chain as in the orthogonal case."""
    rng = np.random.default_rng(37)
    dev = _with_leads_and_overlap(W.random_device(5, 6, n_energies=4, seed=37), rng, overlap=True)
    nb, b = dev["n_blocks"], dev["block_size"]
    eta = dev["eta"]
    Sd, Su = dev["S_diag"], dev["S_upper"]

    def S(i, j):
        return Sd[i] if i == j else (Su[i] if j == i + 1 else Su[j].conj().T)

    for E in (-0.5, 0.6):
        r = O.rgf_energy(E, dev)
        GLu = r["GL_upper"]

        def GL(i, j):
            return r["GL_diag"][i] if i == j else (GLu[i] if j == i + 1 else -GLu[j].conj().T)

        J = np.zeros(nb)
        for i in range(nb):
            SL = dev["SigL"][0, i]
            SR = dev["SigR"][0, i]
            SG = SL + SR - SR.conj().T
            sink = sum(np.trace(S(i, j) @ GL(j, i)) + np.trace(S(j, i) @ GL(i, j))
                       for j in range(max(i - 1, 0), min(i + 2, nb)))
            J[i] = np.real(np.trace(SL @ r["GG_diag"][i] - SG @ r["GL_diag"][i]) + 1j * eta * sink)
        I = r["current"]
        IL, IR = r["contact"]
        scale = np.abs(I).max()
        assert abs(IL + J[0] - I[0]) < 1e-11 * scale
        for i in range(1, nb - 1):
            assert abs(I[i - 1] + J[i] - I[i]) < 1e-11 * scale
        assert abs(I[nb - 2] + J[nb - 1] + IR) < 1e-11 * scale


def test_equilibrium_fluctuation_dissipation():
    """mu_L = mu_R and every Sigma^< = -f (Sigma^R - Sigma^A) (eta reservoir included) =>
    G^< = -f (G^R - G^A), zero current, n_i(E) = f Tr A_ii."""
    dev = _random_with_leads(seed=41)
    mu, kT = 0.1, 0.05
    dev["mu_L"] = dev["mu_R"] = mu
    dev["kT"] = kT
    b = dev["block_size"]
    energies = np.array([-0.6, 0.12, 0.9])
    dev["energies"] = energies
    SR0 = dev["SigR"][0]
    SigL = []
    for E in energies:
        f = O.fermi(E, mu, kT)
        SigL.append(np.stack([-f * (SR0[i] - SR0[i].conj().T) + 2j * dev["eta"] * f * np.eye(b)
                              for i in range(dev["n_blocks"])]))
    dev["SigL"] = np.stack(SigL)
    for k, E in enumerate(energies):
        f = O.fermi(E, mu, kT)
        r = O.rgf_energy(float(E), dev, k)
        for i in range(dev["n_blocks"]):
            G = r["GR_diag"][i]
            ref = -f * (G - G.conj().T)
            assert np.abs(r["GL_diag"][i] - ref).max() < 1e-11 * max(np.abs(ref).max(), 1e-30)
            A = 1j * (G - G.conj().T)
            assert abs(r["density"][i] - f * np.real(np.trace(A))) < 1e-10 * np.abs(A).max()
        for i in range(dev["n_blocks"] - 1):
            G = r["GR_upper"][i]
            Gl = r["GR_lower"][i]
            ref = -f * (G - Gl.conj().T)
            assert np.abs(r["GL_upper"][i] - ref).max() < 1e-11 * np.abs(ref).max()
        assert np.abs(r["current"]).max() < 1e-10


def test_fermi_values_fixed_by_the_definition():
    """f(x) = 1 / (1 + exp(x / kT)): f(mu) = 1/2, f(mu + kT ln 3) = 1/4, f(mu - kT ln 3) = 3/4,
    f(mu + kT ln 9) = 1/10, particle-hole symmetry f(mu + x) + f(mu - x) = 1, and the limits far
    from mu without overflow.  A wrong temperature scale (x / (2 kT)) or sign fails these."""
    for mu, kT in ((0.1, 0.025), (-0.3, 0.1), (0.0, 1e-3)):
        assert O.fermi(mu, mu, kT) == 0.5
        assert abs(O.fermi(mu + kT * np.log(3.0), mu, kT) - 0.25) < 1e-15
        assert abs(O.fermi(mu - kT * np.log(3.0), mu, kT) - 0.75) < 1e-15
        assert abs(O.fermi(mu + kT * np.log(9.0), mu, kT) - 0.1) < 1e-15
        for x in (0.3 * kT, 2.0 * kT, 17.0 * kT):
            assert abs(O.fermi(mu + x, mu, kT) + O.fermi(mu - x, mu, kT) - 1.0) < 1e-15
        assert O.fermi(mu + 2000.0 * kT, mu, kT) == 0.0
        assert O.fermi(mu - 2000.0 * kT, mu, kT) == 1.0


def test_trapezoid_weights_closed_forms():
    """Uniform grid on [a, b] with spacing h: sum w = b - a, sum w E = (b^2 - a^2)/2 (exact for
    linear integrands), sum w E^2 = (b^3 - a^3)/3 + (b - a) h^2 / 6 (the rule's exact error on a
    quadratic); a non-uniform grid integrates linear functions exactly."""
    a, b, n = -1.3, 2.1, 37
    E = np.linspace(a, b, n)
    h = (b - a) / (n - 1)
    w = W.trapezoid_weights(E)
    assert abs(w.sum() - (b - a)) < 1e-14
    assert abs(w @ E - (b * b - a * a) / 2) < 1e-14
    assert abs(w @ E ** 2 - ((b ** 3 - a ** 3) / 3 + (b - a) * h * h / 6)) < 1e-13
    Eg = np.sort(np.random.default_rng(3).uniform(a, b, 25))
    wg = W.trapezoid_weights(Eg)
    assert abs(wg @ (2.0 * Eg - 0.7) - ((Eg[-1] ** 2 - Eg[0] ** 2) - 0.7 * (Eg[-1] - Eg[0]))) < 1e-13
    assert W.trapezoid_weights(np.array([0.4])).tolist() == [0.0]


def test_integrated_current_of_a_clean_chain_equals_the_bias():
    """Clean 1D chain (W = 1 strip, |t| = 1): T(E) = 1 for |E| < 2, so the integrated Landauer
    current over a window that holds both Fermi tails is T (mu_L - mu_R) exactly,
    int (f_L - f_R) dE = mu_L - mu_R.  Window [-0.7, 0.7] (tails e^-24 at kT = 0.025), 140 points
    (E = 0, the chain's band centre where decimation at eta = 1e-10 loses its digits in the first
    sweep, is not on the grid); the trapezoid error of this smooth, decaying integrand is far below
    the tolerance."""
    cfg = W.STRIP_CFG
    s = W.strip(W=1, n_blocks=4, disorder=0.0, eta=1e-10, n_energies=140, e_lo=-0.7, e_hi=0.7,
                mu_L=cfg["mu_L"], mu_R=cfg["mu_R"], kT=cfg["kT"])
    out = O.solve(s, keep_blocks=False)
    assert np.abs(out["transmission"] - 1.0).max() < 1e-8
    assert np.abs(out["current_int"] - (cfg["mu_L"] - cfg["mu_R"])).max() < 1e-8


def test_integrated_density_of_a_broadened_level_closed_form():
    """One level eps0 with a wide-band self-energy Sigma^R = -i Gamma/2 in equilibrium,
    Sigma^< = i f(E) Gamma: n(E) = Im G^< = f(E) Gamma / ((E - eps0)^2 + Gamma^2/4), and the
    density integral sum_E w_E n(E) / (2 pi) over [E_lo, mu + 40 kT] equals the occupation of the
    Lorentzian level, 1/2 - Im psi(1/2 + (Gamma/2 + i (eps0 - mu)) / (2 pi kT)) / pi (psi: digamma),
    minus the part of the Lorentzian below E_lo, (arctan(2 (E_lo - eps0) / Gamma) + pi/2) / pi.
    Pins the 1/(2 pi) of the density integral, the Fermi function's temperature scale inside an
    integral, and the trapezoid weights (its error here is ~1e-9)."""
    from scipy.special import psi
    eps0, gam, mu, kT = 0.0, 0.4, 0.05, 0.02
    E = np.linspace(-2.0, mu + 40 * kT, 2851)
    f = np.array([O.fermi(e, mu, kT) for e in E])
    dev = dict(n_blocks=1, block_size=1, H_diag=np.full((1, 1, 1), eps0, np.complex128),
               H_upper=np.zeros((0, 1, 1), np.complex128), S_diag=None, S_upper=None,
               SigR=np.full((1, 1, 1, 1), -0.5j * gam, np.complex128),
               SigL=(1j * gam * f)[:, None, None, None].astype(np.complex128),
               leads=None, energies=E, eta=1e-12, mu_L=mu, mu_R=mu, kT=kT)
    out = O.solve(dev, keep_blocks=False)
    n_all = 0.5 - np.imag(psi(0.5 + (gam / 2 + 1j * (eps0 - mu)) / (2 * np.pi * kT))) / np.pi
    below = (np.arctan(2 * (E[0] - eps0) / gam) + np.pi / 2) / np.pi
    assert abs(out["density_int"][0] - (n_all - below)) < 1e-8
    # the per-energy density is the Lorentzian times the occupation
    lor = gam / ((E - eps0) ** 2 + gam ** 2 / 4)
    assert np.abs(out["density"][:, 0] - f * lor).max() < 1e-10 * lor.max()

"""The synthetic inputs have the structure the solver and its readings assume: Hermitian H blocks,
anti-Hermitian lesser/greater self-energies of definite sign, and Sigma^R - Sigma^A = Sigma^> -
Sigma^< on every block (the relation that lets G^> come from G^<, G^R and G^A), for the dense device
with block-diagonal or block-tridiagonal self-energies, the NR-L-shaped device and the W system."""
import numpy as np
import pytest

import workloads as W


def _dense_bt(diag, upper, lower=None):
    """Dense matrix from BT blocks; lower = -(upper)^H when not given (anti-Hermitian lesser/greater)."""
    nb, b = diag.shape[0], diag.shape[-1]
    M = np.zeros((nb * b, nb * b), np.complex128)
    for i in range(nb):
        M[i * b:(i + 1) * b, i * b:(i + 1) * b] = diag[i]
    for i in range(nb - 1):
        up = upper[i]
        lo = lower[i] if lower is not None else -up.conj().T
        M[i * b:(i + 1) * b, (i + 1) * b:(i + 2) * b] = up
        M[(i + 1) * b:(i + 2) * b, i * b:(i + 1) * b] = lo
    return M


def _check_lesser_greater_retarded(SL, SG, SR):
    assert np.allclose(SL, -SL.conj().T, atol=1e-14)          # anti-Hermitian
    assert np.allclose(SG, -SG.conj().T, atol=1e-14)
    assert np.linalg.eigvalsh(-1j * SL).min() >= -1e-12        # -i Sigma^< and i Sigma^> are PSD
    assert np.linalg.eigvalsh(1j * SG).min() >= -1e-12
    assert np.allclose(SR - SR.conj().T, SG - SL, atol=1e-14)  # Sigma^R - Sigma^A = Sigma^> - Sigma^<


@pytest.mark.parametrize("offdiag", [False, True])
def test_random_device_structure(offdiag):
    dev = W.random_device(6, 4, n_energies=2, seed=3, offdiag_sigma=offdiag)
    for Hi in dev["H_diag"]:
        assert np.allclose(Hi, Hi.conj().T)
    # only Sigma^< and Sigma^R are inputs; the greater function they imply, Sigma^< + Sigma^R -
    # Sigma^A, must itself be anti-Hermitian with i Sigma^> PSD
    SL_d, SR_d = dev["SigL"][0], dev["SigR"][0]
    SG_d = SL_d + SR_d - SR_d.conj().transpose(0, 2, 1)
    nu = dev["n_blocks"] - 1
    if offdiag:
        SLu, SRu, SRl = dev["SigL_upper"][0], dev["SigR_upper"][0], dev["SigR_lower"][0]
        SGu = SLu + SRu - SRl.conj().transpose(0, 2, 1)
    else:
        SLu = SGu = SRu = SRl = np.zeros((nu, 6, 6), np.complex128)
    SL = _dense_bt(SL_d, SLu)
    SG = _dense_bt(SG_d, SGu)
    SR = _dense_bt(SR_d, SRu, SRl)
    _check_lesser_greater_retarded(SL, SG, SR)


def test_nrl_device_structure():
    dev = W.nrl_device(b=8, n_blocks=3, n_energies=3, rank=4)
    for k in range(3):
        for i in range(3):
            SL, SR = dev["SigL"][k, i], dev["SigR"][k, i]
            SG = SL + SR - SR.conj().T
            _check_lesser_greater_retarded(SL, SG, SR)


def test_w_system_structure():
    w = W.w_system(5, 4, n_energies=2, seed=2)
    V = _dense_bt(w["V_diag"], w["V_upper"], np.conj(np.swapaxes(w["V_upper"], -1, -2)))
    assert np.allclose(V, V.conj().T)
    for k in range(2):
        PL = _dense_bt(w["PL_diag"][k], w["PL_upper"][k])
        PG = _dense_bt(w["PG_diag"][k], w["PG_upper"][k])
        PR = _dense_bt(w["PR_diag"][k], w["PR_upper"][k], w["PR_lower"][k])
        _check_lesser_greater_retarded(PL, PG, PR)

"""Pins for the screened-Coulomb (W) system oracle (Table I, W row): the assembly against explicit
block sums, the selected solve against dense inversion."""
import numpy as np
import pytest

import workloads as W
from oracle import wsys


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _blocks(w, k):
    return ((w["PR_diag"][k], w["PR_upper"][k], w["PR_lower"][k]), (w["PL_diag"][k], w["PL_upper"][k]),
            (w["PG_diag"][k], w["PG_upper"][k]))


def _explicit(w, k):
    """M and B^< by explicit sums over the BT blocks (no dense matrices)."""
    nb, b = w["n_blocks"], w["block_size"]
    Vd, Vu = w["V_diag"], w["V_upper"]
    V = lambda i, j: Vd[i] if i == j else (Vu[i] if j == i + 1 else (Vu[j].conj().T if i == j + 1 else None))
    PR, PL, _ = _blocks(w, k)
    P = lambda i, j: PR[0][i] if i == j else (PR[1][i] if j == i + 1 else (PR[2][j] if i == j + 1 else None))
    Q = lambda i, j: PL[0][i] if i == j else (PL[1][i] if j == i + 1 else (-PL[1][j].conj().T if i == j + 1 else None))
    rng = range(nb)

    def prod(F, G, i, j):
        acc = np.zeros((b, b), np.complex128)
        for m in rng:
            f, g = F(i, m), G(m, j)
            if f is not None and g is not None:
                acc = acc + f @ g
        return acc

    M = {"M_diag": np.stack([np.eye(b) - prod(V, P, i, i) for i in rng]),
         "M_upper": np.stack([-prod(V, P, i, i + 1) for i in range(nb - 1)]) if nb > 1 else np.zeros((0, b, b)),
         "M_lower": np.stack([-prod(V, P, i + 1, i) for i in range(nb - 1)]) if nb > 1 else np.zeros((0, b, b))}
    VQ = lambda i, j: prod(V, Q, i, j)
    VH = lambda i, j: None if V(j, i) is None else V(j, i).conj().T
    B = lambda i, j: sum(VQ(i, m) @ VH(m, j) for m in rng if VH(m, j) is not None)
    M["BL_diag"] = np.stack([B(i, i) for i in rng])
    M["BL_upper"] = np.stack([B(i, i + 1) for i in range(nb - 1)]) if nb > 1 else np.zeros((0, b, b))
    return M


@pytest.mark.parametrize("b,nb", [(3, 1), (4, 2), (3, 5), (5, 4)])
def test_assembly_matches_explicit_block_sums(b, nb):
    w = W.w_system(b, nb, n_energies=2, seed=b + nb)
    for k in range(2):
        a = wsys.assemble(w["V_diag"], w["V_upper"], *_blocks(w, k))
        e = _explicit(w, k)
        for key in e:
            if e[key].size:
                assert _rel(a[key], e[key]) < 1e-13, (key, k)


@pytest.mark.parametrize("b,nb", [(3, 1), (4, 2), (3, 6), (6, 5)])
def test_selected_solve_matches_dense(b, nb):
    """The recursion with A = M_ii, U = M_{i,i+1}, V = M_{i+1,i} and the BT right-hand sides gives
    the BT blocks of M^-1 and M^-1 B^<> M^-H."""
    w = W.w_system(b, nb, n_energies=1, seed=30 + b)
    PR, PL, PG = _blocks(w, 0)
    M = wsys.assemble(w["V_diag"], w["V_upper"], PR, PL, PG)
    BL, BG = (M["BL_diag"], M["BL_upper"]), (M["BG_diag"], M["BG_upper"])
    r, d = wsys.solve(M, BL, BG), wsys.dense_solve(M, BL, BG)
    for key in d:
        if d[key].size:
            assert _rel(r[key], d[key]) < 1e-12, key
    # W^< is anti-Hermitian: its diagonal blocks too
    for X in r["XL_diag"]:
        assert np.abs(X + X.conj().T).max() < 1e-12 * np.abs(X).max()


def test_default_workload_is_conditioned_like_the_papers_w_systems():
    """kappa(M) between 10 and 1e4 (Sec. IV: W systems barely exceed 1e3)."""
    w = W.w_system(32, 6, n_energies=2, seed=0)
    for k in range(2):
        M = wsys.assemble(w["V_diag"], w["V_upper"], *_blocks(w, k))
        kap = np.linalg.cond(wsys.full_bt(M["M_diag"], M["M_upper"], M["M_lower"]))
        assert 10 < kap < 1e4, kap

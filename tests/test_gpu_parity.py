"""GPU parity of the RGF library (called through the C ABI) against the FP64 oracle.

Bars: the FP64 path matches the oracle to 1e-10 relative Frobenius error per block kind and
energy, and to 1e-10 (relative to the largest magnitude) on current, density, contact currents
and transmission.  Lower-precision modes are checked against the error bounds stated beside
each test (derived from the unit roundoff of the mode and the measured sensitivity of the
observables).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

BLOCKS = ("GR_diag", "GR_upper", "GR_lower", "GL_diag", "GL_upper", "GG_diag", "GG_upper")


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2606_25595_gb300 import build
    build.build()
    import paper_2606_25595_gb300 as q
    q.load()
    return q


def _blk_err(got, ref):
    """max over energies of the per-energy relative Frobenius error."""
    errs = []
    for e in range(ref.shape[0]):
        nr = np.linalg.norm(ref[e])
        errs.append(np.linalg.norm(got[e] - ref[e]) / (nr if nr > 0 else 1.0))
    return max(errs) if errs else 0.0


def _obs_err(got, ref):
    s = np.abs(ref).max()
    return np.abs(got - ref).max() / (s if s > 0 else 1.0)


def _check(res, ref, tol_blk, tol_obs, keys=BLOCKS, obs=("current", "density")):
    for k in keys:
        if k in ref and ref[k].size:
            e = _blk_err(res[k], ref[k])
            assert e < tol_blk, (k, e)
    for k in obs:
        if k in ref and np.asarray(ref[k]).size:
            e = _obs_err(np.asarray(res[k]), np.asarray(ref[k]))
            assert e < tol_obs, (k, e)


def test_strip_fp64_full_config(q):
    """W=16 strip, b=16, N_B=32, 64 energies, Sancho-Rubio contacts, FP64.

    Observables to 1e-10.  Blocks to 1e-10 at the median energy and, at every energy, to
    max(1e-10, 2e3 * kappa_dec(E) * eps_64): at eta = 1e-6 the decimation inverts blocks (z - eps)
    with condition numbers up to ~3e4, and two FP64 implementations of the same iteration (the
    oracle with LAPACK's inverse vs with Gauss-Jordan) already differ by up to 7e-10 in Sigma^R there
    (Eq. 6: error ~ kappa * eps_m)."""
    dev = W.strip(**{k: v for k, v in W.STRIP_CFG.items()})
    ref = O.solve(dev, track_cond=True)
    res = q.solve_device(dev, "fp64")
    assert np.all(res["status"] == 0)
    tol_e = np.maximum(1e-10, 2e3 * ref["decim_cond"] * 2.0 ** -53)
    for k in BLOCKS:
        errs = np.array([np.linalg.norm(res[k][e] - ref[k][e]) / np.linalg.norm(ref[k][e])
                         for e in range(ref[k].shape[0])])
        assert np.median(errs) < 1e-10, k
        assert np.all(errs < tol_e), (k, errs.max(), tol_e[np.argmax(errs / tol_e)])
    _check(res, ref, 1.0, 1e-10, keys=(), obs=("current", "density", "contact", "transmission"))
    assert _obs_err(res["current_int"], ref["current_int"]) < 1e-10
    assert _obs_err(res["density_int"], ref["density_int"]) < 1e-10


def test_strip_fp64_well_conditioned_contacts(q):
    """Same strip with eta = 1e-3 (decimation inverses well conditioned): every block <= 1e-10."""
    cfg = dict(W.STRIP_CFG)
    cfg["eta"] = 1e-3
    dev = W.strip(**cfg)
    ref = O.solve(dev)
    res = q.solve_device(dev, "fp64")
    _check(res, ref, 1e-10, 1e-10, obs=("current", "density", "contact", "transmission"))


@pytest.mark.parametrize("b,nb,ne,chunk", [(5, 3, 3, 2), (37, 4, 3, 3), (80, 3, 2, 1),
                                           (130, 2, 3, 2), (1, 6, 4, 4), (20, 1, 3, 3)])
def test_random_fp64_with_overlap_leads_ragged(q, b, nb, ne, chunk):
    """Ragged sizes (tails of the 32/64 tiles, recursive inverse for b > 64), overlap S,
    non-symmetric contacts, energy-dependent Sigma, chunked energies: FP64 parity <= 1e-10."""
    rng = np.random.default_rng(b * 100 + nb)
    dev = W.random_device(b, nb, n_energies=ne, seed=b + nb)
    dev["S_diag"] = np.stack([np.eye(b) + 0.05 * (lambda X: (X + X.conj().T) / 2)(
        rng.standard_normal((b, b)) + 1j * rng.standard_normal((b, b))) for _ in range(nb)])
    dev["S_upper"] = (0.03 * (rng.standard_normal((nb - 1, b, b)) + 1j * rng.standard_normal((nb - 1, b, b)))
                      if nb > 1 else np.zeros((0, b, b), np.complex128))
    X = rng.standard_normal((b, b)) + 1j * rng.standard_normal((b, b))
    dev["leads"] = dict(H00_L=(X + X.conj().T) / 2, H01_L=0.4 * (rng.standard_normal((b, b)) + 1j * rng.standard_normal((b, b))),
                        H00_R=(X + X.conj().T) / 3, H01_R=0.4 * (rng.standard_normal((b, b)) + 1j * rng.standard_normal((b, b))))
    dev["eta"] = 1e-3
    dev["mu_L"], dev["mu_R"], dev["kT"] = 0.3, -0.2, 0.05
    dev["SigR"] = np.concatenate([dev["SigR"] * (1 + 0.1 * k) for k in range(ne)])
    dev["SigL"] = np.concatenate([dev["SigL"] * (1 + 0.2 * k) for k in range(ne)])
    ref = O.solve(dev)
    res = q.solve_device(dev, "fp64", max_energies_in_flight=chunk)
    assert np.all(res["status"] == 0)
    _check(res, ref, 1e-10, 1e-10, obs=("current", "density", "contact", "transmission"))


def test_mixed_workload_fp64_sampled_energies(q):
    """b=256, N_B=64 (the mixed-precision workload's shape) at sampled energies, FP64 <= 1e-10."""
    dev = W.random_device(256, 64, n_energies=512, seed=0)
    idx = [3, 200, 451]
    E = dev["energies"][idx]
    ref = O.solve(dev, energy_indices=idx, keep_blocks=True)
    res = q.solve_device(dev, "fp64", energies=E, outputs=["GR_diag", "GL_diag", "GL_upper", "current",
                                                            "density"])
    _check(res, ref, 1e-10, 1e-10, keys=("GR_diag", "GL_diag", "GL_upper"))


def test_fp32_error_within_stated_bound(q):
    """complex64 products and inverses: G blocks within 5e-4 (about 1e4 x eps_FP32), density within
    1e-4, current within 5e-2 (the current is a small difference of large G^< entries; FP32 loses
    ~1e3-1e4 x eps there on this workload)."""
    dev = W.random_device(64, 16, n_energies=6, seed=2)
    ref = O.solve(dev)
    res = q.solve_device(dev, "fp32")
    _check(res, ref, 5e-4, 1e-4, keys=("GR_diag", "GL_diag"), obs=("density",))
    assert _obs_err(res["current"], ref["current"]) < 5e-2


def test_singular_block_reports_status(q):
    """A block that is exactly singular (eta = 0, E at an eigenvalue, no scattering) is reported
    per energy as QTX_ERR_SINGULAR without trapping."""
    b = 2
    dev = dict(n_blocks=1, block_size=b, H_diag=np.array([[[0.5, 0], [0, 0.0]]], np.complex128),
               H_upper=np.zeros((0, b, b), np.complex128), S_diag=None, S_upper=None, SigR=None,
               SigL=None, leads=None, energies=np.array([0.5, 0.7]), eta=0.0, mu_L=0, mu_R=0, kT=0.025)
    res = q.solve_device(dev, "fp64", outputs=["GR_diag"])
    assert res["status"][0] == 4 and res["status"][1] == 0


def test_decimation_cap_reports_not_converged(q):
    dev = W.strip(n_blocks=4, n_energies=3)
    import torch
    din = q.upload(dev)
    desc = q.make_desc(4, 16, "fp64", 3, leads=True, has_scattering=False, decim_max_iter=2,
                       outputs=["current"])
    P = q.Plan(desc)
    o = q.Outputs()
    cur = torch.empty((3, 3), dtype=torch.float64, device="cuda")
    st = torch.zeros(3, dtype=torch.int32, device="cuda")
    o.current = cur.data_ptr()
    o.status_per_energy = st.data_ptr()
    P.solve(din["_inputs"], o, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert np.all(st.cpu().numpy() == 5)


def test_invalid_arguments_enqueue_nothing(q):
    desc = q.make_desc(4, 16, "fp64", 2, has_scattering=True)
    P = q.Plan(desc)
    with pytest.raises(q.QtxError) as ei:
        P.solve(q.Inputs(), q.Outputs(), 0)
    assert ei.value.status == 1

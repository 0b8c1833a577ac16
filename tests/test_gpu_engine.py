"""GPU checks of the building blocks through the component C ABI (include/qtx_kernels.h):
the tensor-core GEMM engine (emulated FP64 and BF16x3), the batched block inverse with
refinement, and the Sancho-Rubio contact self-energy."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


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


def _t(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.complex128).cuda()


def _op(X, op):
    return X if op == "N" else np.conj(np.swapaxes(X, -1, -2))


# N covers every kind of last column tile.  With 48 columns per tile (6 and 7 digit planes): 16 (64,
# 16, 256), 22 -> 24 (70), 8 (200), a full 48 (96), 41 -> 48 and a single column; with 64 (2 and 4
# planes): a full 64 (64, 128, 256), 6 -> 8 (70), 8 (200), 32 (96), 41 -> 48, 16 and a single column.
# The last shape has 400 (48) or 320 (64) tiles, so the persistent CTAs run several rounds and a
# partial one
SHAPES = [(128, 64, 32, 1), (130, 70, 50, 3), (16, 16, 16, 4), (256, 256, 256, 2), (33, 200, 300, 2),
          (64, 96, 48, 2), (40, 41, 24, 3), (17, 1, 16, 2), (256, 200, 64, 40)]


@pytest.mark.parametrize("M,N,K,batch", SHAPES)
@pytest.mark.parametrize("opA,opB", [("N", "N"), ("C", "N"), ("N", "C"), ("C", "C")])
@pytest.mark.parametrize("prec", ["emu64", "bf16x3"])
def test_integer_inputs_are_exact(q, M, N, K, batch, opA, opB, prec):
    """Integer operands: every digit product is exact, so the result equals the integer product
    bit for bit (pins digits, scales, the complex embedding, the TMA/UMMA layouts and the epilogue).
    BF16x3 (64-column tiles) keeps the products of planes i + j <= 3 only, so its operands are
    multiples of 16 below 500: with the row scaled to 12 or 13 bits they are whole multiples of the
    leading digit's unit, the second digits are zero and nothing dropped was nonzero."""
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    sa = (batch, M, K) if opA == "N" else (batch, K, M)
    sb = (batch, K, N) if opB == "N" else (batch, N, K)
    lo, unit = (-500, 1) if prec == "emu64" else (-31, 16)
    A = unit * (rng.integers(lo, -lo + 1, sa) + 1j * rng.integers(lo, -lo + 1, sa))
    B = unit * (rng.integers(lo, -lo + 1, sb) + 1j * rng.integers(lo, -lo + 1, sb))
    C0 = rng.integers(-1000, 1001, (batch, M, N)) + 1j * rng.integers(-1000, 1001, (batch, M, N))
    ref = -(_op(A, opA) @ _op(B, opB)) + C0
    got = q.zgemm_batched(_t(A), _t(B), prec, opA, opB, alpha=-1.0, beta=1.0, C0=_t(C0)).cpu().numpy()
    assert np.array_equal(got, ref)


def test_emu64_shared_operand_and_zero_rows(q):
    """A 2-D operand is shared across the batch (digitised once); an all-zero row stays zero."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((3, 96, 80)) + 1j * rng.standard_normal((3, 96, 80))
    A[1, 7, :] = 0
    B = rng.standard_normal((80, 72)) + 1j * rng.standard_normal((80, 72))
    got = q.zgemm_batched(_t(A), _t(B), "emu64").cpu().numpy()
    ref = A @ B
    assert np.all(got[1, 7] == 0)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-10


@pytest.mark.parametrize("M,N,K,batch", [(256, 256, 256, 3), (130, 70, 50, 2), (64, 192, 128, 2)])
def test_emu64_random_error_bound(q, M, N, K, batch):
    """Random FP64 data: |C - C_ref| <= 2^-36 * (|A| |B|) elementwise (~41-bit digit products with
    row/column scaling; the rounded accumulator and the df32 rounding of inputs sit below that)."""
    rng = np.random.default_rng(M + N + K)
    A = (rng.standard_normal((batch, M, K)) + 1j * rng.standard_normal((batch, M, K))) * \
        np.exp(rng.uniform(-3, 3, (batch, M, 1)))
    B = rng.standard_normal((batch, K, N)) + 1j * rng.standard_normal((batch, K, N))
    got = q.zgemm_batched(_t(A), _t(B), "emu64").cpu().numpy()
    ref = A @ B
    bound = (np.abs(A.real) + np.abs(A.imag)) @ (np.abs(B.real) + np.abs(B.imag))
    assert np.all(np.abs(got - ref) <= 2.0 ** -36 * bound)


@pytest.mark.parametrize("M,N,K,batch,alpha,beta", [(256, 256, 256, 2, 0.1, 1.0 / 3.0),
                                                    (130, 70, 50, 3, -1.0 / 3.0, 0.1),
                                                    (64, 96, 1536, 2, 0.1, -1.0 / 7.0)])
def test_emu64_general_alpha_beta(q, M, N, K, batch, alpha, beta):
    """Scalars that FP32 cannot hold (0.1, 1/3, 1/7) enter in df32 (~48 bits): the result stays within
    the products' 2^-36 |alpha| (|A| |B|) plus 2^-40 |beta C0|; an FP32-rounded alpha or beta would
    add ~2^-24 of every element.  The last case runs split along K (C0 enters the first chunk)."""
    rng = np.random.default_rng(M + 3 * K)
    A = (rng.standard_normal((batch, M, K)) + 1j * rng.standard_normal((batch, M, K))) * \
        np.exp(rng.uniform(-3, 3, (batch, M, 1)))
    B = rng.standard_normal((batch, K, N)) + 1j * rng.standard_normal((batch, K, N))
    C0 = rng.standard_normal((batch, M, N)) + 1j * rng.standard_normal((batch, M, N))
    got = q.zgemm_batched(_t(A), _t(B), "emu64", alpha=alpha, beta=beta, C0=_t(C0)).cpu().numpy()
    ref = alpha * (A @ B) + beta * C0
    bound = (np.abs(A.real) + np.abs(A.imag)) @ (np.abs(B.real) + np.abs(B.imag))
    tol = 2.0 ** -36 * abs(alpha) * bound + 2.0 ** -40 * abs(beta) * (np.abs(C0.real) + np.abs(C0.imag))
    assert np.all(np.abs(got - ref) <= tol), np.log2(np.max(np.abs(got - ref) / tol))


@pytest.mark.parametrize("K,bits", [(512, 35), (1024, 36)])
def test_emu64_random_error_bound_long_k(q, K, bits):
    """Long contractions (b = 512, 1024 blocks): the leading digit shrinks to keep the exact
    accumulators below 2^24 units (l1 = 6 for K <= 512, 5 for K <= 1024).  At K = 512 six digits
    carry P = 7*5 + l1 - 1 = 40 bits, one less than at K <= 256, so the bound is 2^-35 (|A| |B|);
    at K = 1024 the engine takes a seventh digit (P = 46) and the bound returns to 2^-36."""
    rng = np.random.default_rng(K)
    M, N, batch = 256, 144, 2
    A = (rng.standard_normal((batch, M, K)) + 1j * rng.standard_normal((batch, M, K))) * \
        np.exp(rng.uniform(-3, 3, (batch, M, 1)))
    B = rng.standard_normal((batch, K, N)) + 1j * rng.standard_normal((batch, K, N))
    got = q.zgemm_batched(_t(A), _t(B), "emu64").cpu().numpy()
    ref = A @ B
    bound = (np.abs(A.real) + np.abs(A.imag)) @ (np.abs(B.real) + np.abs(B.imag))
    ratio = np.max(np.abs(got - ref) / bound)
    assert ratio <= 2.0 ** -bits, np.log2(ratio)


@pytest.mark.parametrize("K", [1536, 3408])
def test_emu64_split_k_error_bound(q, K):
    """Contractions beyond 1024 run as K-chunks of at most 1024 (each exact in its digit
    accumulators, 7 digits) added in df32: the 2^-36 (|A| |B|) bound holds at 1536 and at the
    paper's NR-L block size 3408."""
    rng = np.random.default_rng(K)
    M, N, batch = 160, 96, 2
    A = (rng.standard_normal((batch, M, K)) + 1j * rng.standard_normal((batch, M, K))) * \
        np.exp(rng.uniform(-3, 3, (batch, M, 1)))
    B = rng.standard_normal((batch, K, N)) + 1j * rng.standard_normal((batch, K, N))
    got = q.zgemm_batched(_t(A), _t(B), "emu64").cpu().numpy()
    ref = A @ B
    bound = (np.abs(A.real) + np.abs(A.imag)) @ (np.abs(B.real) + np.abs(B.imag))
    ratio = np.max(np.abs(got - ref) / bound)
    assert ratio <= 2.0 ** -36, np.log2(ratio)
    # conjugate-transposed operands take the other chunk strides
    gotc = q.zgemm_batched(_t(np.conj(np.swapaxes(A, 1, 2))), _t(np.conj(np.swapaxes(B, 1, 2))), "emu64",
                           opA="C", opB="C").cpu().numpy()
    assert np.max(np.abs(gotc - ref) / bound) <= 2.0 ** -36


def test_bf16x3_error_bound(q):
    """Two digit planes (~13-bit products): |C - C_ref| <= 2^-11 * (|A| |B|)."""
    rng = np.random.default_rng(11)
    A = rng.standard_normal((2, 128, 96)) + 1j * rng.standard_normal((2, 128, 96))
    B = rng.standard_normal((2, 96, 64)) + 1j * rng.standard_normal((2, 96, 64))
    got = q.zgemm_batched(_t(A), _t(B), "bf16x3").cpu().numpy()
    ref = A @ B
    bound = (np.abs(A.real) + np.abs(A.imag)) @ (np.abs(B.real) + np.abs(B.imag))
    assert np.all(np.abs(got - ref) <= 2.0 ** -11 * bound)


# relative error bound per mode, as a multiple of kappa(A): FP64 / FP32 unit roundoff, and for the
# emulated mode the ~2^-36 of its tensor-core products (Eq. 6: error ~ kappa * eps_m)
INV_EPS = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24, "emu64": 2.0 ** -38}


@pytest.mark.parametrize("prec", ["fp64", "fp32", "emu64"])
@pytest.mark.parametrize("n", [16, 64, 100, 256])
def test_block_inverse(q, prec, n):
    """Batched inverse of accretive blocks (E + i eta - H - Sigma^R) against LAPACK:
    relative error <= 64 kappa(A) eps_mode."""
    dev = W.random_device(n, 3, n_energies=1, seed=n)
    A = np.stack([(0.37 + 1e-6j) * np.eye(n) - dev["H_diag"][i] - dev["SigR"][0, i] for i in range(3)])
    ref = np.linalg.inv(A)
    X, st = q.zinv_batched(_t(A), prec, refine_iter=2)
    X = X.cpu().numpy()
    assert np.all(st.cpu().numpy() == 0)
    for e in range(3):
        kap = np.linalg.cond(A[e])
        err = np.linalg.norm(X[e] - ref[e]) / np.linalg.norm(ref[e])
        assert err < 64 * kap * INV_EPS[prec], (err, kap)


def test_lead_self_energy_matches_oracle(q):
    import torch
    s = W.strip(n_blocks=2, disorder=0.0)
    E = np.linspace(-3.5, 3.5, 17)
    eta = 1e-3
    SR, st = q.lead_self_energy(_t(s["leads"]["H00_L"]), _t(s["leads"]["H01_L"]),
                                torch.as_tensor(E).cuda(), eta)
    SR = SR.cpu().numpy()
    assert np.all(st.cpu().numpy() == 0)
    for k, e in enumerate(E):
        ref, _, _, kap = O.lead_self_energy(e, eta, s["leads"]["H00_L"], s["leads"]["H01_L"],
                                           track_cond=True)
        assert np.linalg.norm(SR[k] - ref) / np.linalg.norm(ref) < max(1e-12, 1e4 * kap * 2.0 ** -53)


def test_bounded_wait_gives_up_and_the_context_stays_usable(q):
    """The tensor-core kernel's waits are bounded.  With the test switch on (qtx_tc_wait_test), every
    product launch's MMA thread first waits on a barrier nothing arrives at, limited to 100 us: the wait
    gives up before any MMA is issued, the launch drains its copies and frees its tensor memory, and
    the call reports QTX_ERR_TIMEOUT.  Nothing faults or hangs: afterwards the same GEMM and an RGF
    solve on the same plan give the results they gave before (the plan's wait flag is cleared per
    solve)."""
    import torch
    L = q.load()
    rng = np.random.default_rng(8)
    A = _t(rng.standard_normal((2, 96, 64)) + 1j * rng.standard_normal((2, 96, 64)))
    B = _t(rng.standard_normal((2, 64, 80)) + 1j * rng.standard_normal((2, 64, 80)))
    ref = q.zgemm_batched(A, B, "emu64").cpu().numpy()
    dev = W.random_device(96, 3, n_energies=2, seed=5)
    outs = ["GR_diag", "GL_diag", "current", "density"]
    P = q.Plan(q.make_desc(3, 96, "emu64", 2, has_scattering=True, outputs=outs))
    good = q.solve_device(dev, "emu64", outputs=outs, plan=P)
    assert P.status() == 0
    L.qtx_tc_wait_test(1)
    try:
        with pytest.raises(q.QtxError) as ei:
            q.zgemm_batched(A, B, "emu64")
        assert ei.value.status == 6  # QTX_ERR_TIMEOUT
        q.solve_device(dev, "emu64", outputs=outs, plan=P)
        assert P.status() == 6
    finally:
        L.qtx_tc_wait_test(0)
    torch.cuda.synchronize()
    assert np.array_equal(q.zgemm_batched(A, B, "emu64").cpu().numpy(), ref)
    again = q.solve_device(dev, "emu64", outputs=outs, plan=P)
    assert P.status() == 0
    for k in outs:
        assert np.array_equal(again[k], good[k]), k
    P.close()

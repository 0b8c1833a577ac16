"""The allocation-free GEMM entry point (qtx_zgemm_emu64_noalloc), called through the C ABI.

It serves callers that cannot allocate device memory while they run (a latency-critical loop where
cudaMalloc/cudaFree would synchronise the device, a plugin inside another runtime that owns all
device memory, a process with a fixed memory budget).  Its result must equal the allocating entry
point's (qtx_zgemm_batched, emulated FP64) on two calls in a row -- the second call reuses the fixed
array the first one left behind -- and a request larger than the array must be refused.  This file
is collected last so that a failure here leaves every other test already run; it also passes alone.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

QTX_ERR_OOM = 2


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


def _noalloc(q, A, B, C0, opA, opB, alpha, beta, M, N, K, batch):
    import torch
    ops = {"N": 0, "C": 1}
    out = torch.empty((batch, M, N), dtype=torch.complex128, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    s = q.load().qtx_zgemm_emu64_noalloc(
        M, N, K, ops[opA], A.data_ptr(), A.shape[2], A.shape[1] * A.shape[2], ops[opB], B.data_ptr(),
        B.shape[2], B.shape[1] * B.shape[2], float(alpha), float(beta),
        None if C0 is None else C0.data_ptr(), N, M * N, out.data_ptr(), N, M * N, batch,
        ctypes.c_void_p(st))
    return s, out


def test_noalloc_matches_allocating_gemm_on_two_calls(q):
    rng = np.random.default_rng(2024)
    # the last case has scalars FP32 cannot hold: both entry points apply them in df32
    cases = [(256, 200, 256, 3, "N", "N", -1.0, 1.0), (130, 96, 70, 4, "C", "C", 1.0, 0.0),
             (200, 144, 96, 2, "N", "C", 0.1, 1.0 / 3.0)]
    for M, N, K, batch, opA, opB, alpha, beta in cases:
        sa = (batch, M, K) if opA == "N" else (batch, K, M)
        sb = (batch, K, N) if opB == "N" else (batch, N, K)
        A = rng.standard_normal(sa) + 1j * rng.standard_normal(sa)
        B = rng.standard_normal(sb) + 1j * rng.standard_normal(sb)
        C0 = rng.standard_normal((batch, M, N)) + 1j * rng.standard_normal((batch, M, N))
        tA, tB, tC0 = _t(A), _t(B), _t(C0)
        ref = q.zgemm_batched(tA, tB, "emu64", opA, opB, alpha=alpha, beta=beta,
                              C0=tC0 if beta else None).cpu().numpy()
        s, out = _noalloc(q, tA, tB, tC0 if beta else None, opA, opB, alpha, beta, M, N, K, batch)
        assert s == 0
        out = out.cpu().numpy()
        # the engine tests' bound, 2^-36 (|A||B|), against the allocating entry point's result
        opa = A if opA == "N" else np.conj(np.swapaxes(A, 1, 2))
        opb = B if opB == "N" else np.conj(np.swapaxes(B, 1, 2))
        bound = (np.abs(opa.real) + np.abs(opa.imag)) @ (np.abs(opb.real) + np.abs(opb.imag))
        tol = 2.0 ** -36 * abs(alpha) * bound + 2.0 ** -40 * abs(beta) * np.abs(C0)
        assert np.all(np.abs(out - ref) <= 2 * tol)
        exact = alpha * (opa @ opb) + (beta * C0 if beta else 0)
        assert np.all(np.abs(out - exact) <= tol)


def test_noalloc_refuses_requests_larger_than_its_array(q):
    import torch
    M = N = K = 256
    batch = 8  # about 8.9 MiB per entry with C0 > 48 MiB
    A = torch.zeros((batch, M, K), dtype=torch.complex128, device="cuda")
    s, _ = _noalloc(q, A, A, A, "N", "N", 1.0, 1.0, M, N, K, batch)
    assert s == QTX_ERR_OOM

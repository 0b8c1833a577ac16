"""GPU parity of the FPX storage codec (Sec. V) against the oracle's exact-rational rounding:
codes are compared byte for byte, decoded values bit for bit."""
import math

import numpy as np
import pytest

from oracle import fpx as F

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


def _values(seed, n):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(n) * 10.0 ** rng.uniform(-48, 40, n)
    edge = [0.0, -0.0, math.inf, -math.inf, 1e-46, -1e-46, 2.0 ** -149, 2.0 ** -149 * 1.5,
            2.0 ** -126, -2.0 ** -126 * (1 - 2.0 ** -30), 3.4028234663852886e38, 3.4028235677973366e38,
            1e39, -1e300, 5e-324, 1.0, -1.5, math.pi]
    return np.concatenate([v, edge])


def _midpoints(bits, seed, n):
    """Values exactly halfway between two neighbouring FPX values (ties), and just off them."""
    m = bits - 9
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        e = int(rng.integers(-140, 127))
        k = int(rng.integers(0, 1 << m))
        base = math.ldexp((1 << m) + k, e - m) if e >= -126 else math.ldexp(k, -126 - m)
        half = math.ldexp(1.0, (max(e, -126)) - m - 1)
        for d in (half, half * (1 - 2.0 ** -20), half * (1 + 2.0 ** -20)):
            out.append(base + d)
            out.append(-(base + d))
    return np.array(out)


@pytest.mark.parametrize("bits", F.WIDTHS)
def test_codes_match_oracle_bytewise(q, bits):
    import torch
    x = np.concatenate([_values(bits, 4000), _midpoints(bits, 7 * bits, 300), [math.nan]])
    x = x[: len(x) - (len(x) % 8) + 5]  # a ragged tail: the last group is partly padding
    got = q.fpx_compress(torch.tensor(x, device="cuda"), bits).cpu().numpy().tobytes()
    ref = F.compress(x, bits)
    assert got[: len(ref)] == ref
    assert got[len(ref):] == bytes(len(got) - len(ref))  # padding codes are zero
    assert len(got) == -(-len(x) // 8) * bits


@pytest.mark.parametrize("bits", F.WIDTHS)
def test_decode_matches_oracle_bitwise(q, bits):
    import torch
    x = np.concatenate([_values(100 + bits, 3000), _midpoints(bits, 11 * bits, 200)])
    codes = q.fpx_compress(torch.tensor(x, device="cuda"), bits)
    got = q.fpx_decompress(codes, bits, len(x)).cpu().numpy()
    data = codes.cpu().numpy().tobytes()
    ref = F.decompress(data, bits, len(x))
    same = (got.view(np.uint64) == ref.view(np.uint64)) | (np.isnan(got) & np.isnan(ref))
    assert np.all(same)


def test_cutoff_complex_and_small_sizes(q):
    import torch
    z = np.array([1e-12 + 2j, -3e-13 - 2.5e-9j, -1.0 + 0j], dtype=np.complex128)
    codes = q.fpx_compress(torch.tensor(z, device="cuda"), 24, cutoff=1e-9)
    assert codes.cpu().numpy().tobytes()[:18] == F.compress(z, 24, cutoff=1e-9)
    back = q.fpx_decompress(codes, 24, 6, complex_out=True).cpu().numpy()
    assert back[0].real == 0.0 and back[1].real == 0.0 and back[2] == -1.0
    for n in (1, 7, 8, 9):
        x = np.linspace(-3, 3, n)
        c = q.fpx_compress(torch.tensor(x, device="cuda"), 40)
        assert c.cpu().numpy().tobytes()[: 5 * n] == F.compress(x, 40)


def test_invalid_arguments(q):
    import ctypes
    import torch
    L = q.load()
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(256, dtype=torch.uint8, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.qtx_fpx_compress(33, x.data_ptr(), 16, 0.0, out.data_ptr(), st) == 1
    assert L.qtx_fpx_compress(24, x.data_ptr(), -1, 0.0, out.data_ptr(), st) == 1
    assert L.qtx_fpx_compress(24, x.data_ptr(), 16, -1.0, out.data_ptr(), st) == 1
    assert L.qtx_fpx_compress(24, x.data_ptr() + 4, 15, 0.0, out.data_ptr(), st) == 1
    assert L.qtx_fpx_decompress(24, out.data_ptr() + 3, 8, x.data_ptr(), st) == 1
    assert L.qtx_fpx_compress(24, x.data_ptr(), 0, 0.0, None, st) == 0
    assert L.qtx_fpx_bytes(24, 17) == 72 and L.qtx_fpx_bytes(7, 17) == 0


@pytest.mark.parametrize("bits", [48, 24])
def test_large_array_sampled_and_round_trip(q, bits):
    """64 M values (512 MB of FP64): sampled codes against the oracle, and the whole array's
    decoded values within half a unit of the last place of the input (or equal to it when the input
    is itself an FPX value, checked by recompressing)."""
    import torch
    n = 1 << 26
    g = torch.Generator(device="cuda").manual_seed(bits)
    x = torch.randn(n, dtype=torch.float64, device="cuda", generator=g) * \
        torch.exp(torch.empty(n, dtype=torch.float64, device="cuda").uniform_(-30, 30, generator=g))
    codes = q.fpx_compress(x, bits)
    y = q.fpx_decompress(codes, bits, n)
    m = bits - 9
    ax = x.abs()
    e = torch.floor(torch.log2(ax)).clamp(min=-126)
    assert bool(((y - x).abs() <= torch.ldexp(torch.ones_like(ax), (e - m - 1).to(torch.int32)) * 1.0000001).all())
    assert torch.equal(q.fpx_compress(y, bits), codes)
    idx = np.random.default_rng(bits).integers(0, n, 500)
    xs = x[torch.tensor(idx, device="cuda")].cpu().numpy()
    cb = codes.cpu().numpy()
    nb = bits // 8
    for k, v in zip(idx, xs):
        assert bytes(cb[k * nb:(k + 1) * nb]) == F.encode(float(v), bits).to_bytes(nb, "little")

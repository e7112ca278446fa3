"""The tcgen05 FP8 product on its own: D = A8 B8^T must equal the exact integer
product for integer digits |d| <= 16 and k <= 2^16 (Sec. III-B, Eq.
error-free-FP8-matmult: every partial sum is an integer of magnitude <= 2^24, exact
in FP32).  Compared element by element with an int64 product on the CPU."""
import numpy as np
import pytest
import torch

import paper_2603_10634_gb300 as ozk

pytestmark = pytest.mark.gpu


def e4m3_codes(d):
    return torch.as_tensor(d, dtype=torch.float32).to(torch.float8_e4m3fn).view(torch.uint8)


def padded(codes, kp):
    rows, k = codes.shape
    out = torch.zeros((rows, kp), dtype=torch.uint8)
    out[:, :k] = codes
    return out


def run(dA, dB, cuda, kp=None):
    m, k = dA.shape
    n = dB.shape[0]
    kp = kp or 32 * ((k + 31) // 32)
    A8 = padded(e4m3_codes(dA), kp).to(cuda)
    B8 = padded(e4m3_codes(dB), kp).to(cuda)
    D = ozk.fp8_gemm(A8, B8, k=k)
    torch.cuda.synchronize()
    assert ozk.device_status() == "OZK2_OK"
    return D.cpu().numpy()


@pytest.mark.parametrize("m,n,k", [(128, 128, 128), (256, 384, 512), (200, 130, 300), (1, 1, 1),
                                   (5, 7, 33), (129, 255, 1000), (300, 140, 4096)])
def test_random_digits_exact(cuda, m, n, k):
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    dA = rng.integers(-16, 17, size=(m, k))
    dB = rng.integers(-16, 17, size=(n, k))
    D = run(dA, dB, cuda)
    want = dA.astype(np.int64) @ dB.astype(np.int64).T
    assert np.array_equal(D.astype(np.int64), want)
    assert np.all(D == np.rint(D))


def test_worst_case_magnitude_2_pow_24(cuda):
    """All digits +16 with k = 2^16: every output is exactly 2^24."""
    m, n, k = 128, 256, 65536
    dA = np.full((m, k), 16)
    dB = np.full((n, k), 16)
    dB[1::2] = -16
    D = run(dA, dB, cuda)
    want = np.where(np.arange(n) % 2 == 0, 2.0**24, -(2.0**24))[None, :].repeat(m, 0)
    assert np.array_equal(D, want)


def test_alternating_partial_sums(cuda):
    """Partial sums that swing through +-2^23 before cancelling stay exact."""
    m, n, k = 128, 128, 65536
    dA = np.full((m, k), 16)
    dA[:, k // 2:] = -16
    dB = np.full((n, k), 16)
    dB[:, ::3] = 15
    D = run(dA, dB, cuda)
    want = dA.astype(np.int64) @ dB.astype(np.int64).T
    assert np.array_equal(D.astype(np.int64), want)


def test_fractional_bound_operands_error_bound(cuda):
    """Non-integer E4M3 values (the bound product): |D - exact| <= (k-1) 2^-24 |A||B|
    (the FP32 summation bound the paper relies on, Sec. III-E)."""
    rng = np.random.default_rng(5)
    m, n, k = 256, 256, 2048
    codes_a = torch.as_tensor(rng.integers(1, 0x78, size=(m, k)), dtype=torch.uint8)
    codes_b = torch.as_tensor(rng.integers(1, 0x78, size=(n, k)), dtype=torch.uint8)
    va = codes_a.view(torch.float8_e4m3fn).double().numpy()
    vb = codes_b.view(torch.float8_e4m3fn).double().numpy()
    D = ozk.fp8_gemm(codes_a.to(cuda), codes_b.to(cuda), k=k).cpu().numpy().astype(np.float64)
    exact = va @ vb.T  # exact in float64 (see the oracle's bound_product)
    assert np.all(np.abs(D - exact) <= (k - 1) * 2.0**-24 * exact)

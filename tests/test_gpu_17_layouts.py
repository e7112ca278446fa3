"""Operands whose lines do not start on 16-byte boundaries: an odd leading dimension, or
a view that starts 8 bytes into its buffer.  A's rows and the rows of B stored
transposed (op(B) = B^T with B^T row-major) go through the row residue kernel, which
loads 16 bytes at a time only when every row is 16-byte aligned; these cases take its
8-byte path.  Bit-exact against the oracle fed with the GPU's exponents."""
import numpy as np
import pytest
import torch

import paper_2603_10634_gb300 as ozk
from oracle import ozaki2 as oz
from paper_2603_10634_gb300 import workloads

pytestmark = pytest.mark.gpu


def _view(X, offset, pad, cuda):
    """X as a view into a wider device buffer: row pitch cols + offset + pad, first
    element `offset` elements into each row."""
    rows, cols = X.shape
    big = torch.zeros(rows, cols + offset + pad, dtype=torch.float64)
    big[:, offset:offset + cols] = X
    return big.to(cuda)[:, offset:offset + cols]


@pytest.mark.parametrize("offset,pad", [(0, 1), (1, 0), (1, 3)])
@pytest.mark.parametrize("N", [12, 7])
def test_unaligned_rows_bit_exact(cuda, offset, pad, N):
    m, n, k = 150, 70, 300
    A, B = workloads.problem(m, n, k, 1.0, seed=3)
    Ad = _view(A, offset, pad, cuda)
    Bd = _view(B.T.contiguous(), offset, pad, cuda).T  # op(B) = B^T, rows of B^T unaligned
    row_bytes = (k + offset + pad) * 8
    aligned = (Ad.data_ptr() % 16 == 0) and row_bytes % 16 == 0
    assert not aligned
    C = ozk.dgemm(Ad, Bd, num_moduli=N)
    sc = ozk.scales(Ad, Bd, num_moduli=N)
    r = oz.ozk2_dgemm(A.numpy(), B.numpy(), N, e=sc["e"].cpu().numpy(), f=sc["f"].cpu().numpy())
    assert np.array_equal(C.cpu().numpy().view(np.uint64), r["C"].view(np.uint64))
    assert ozk.device_status() == "OZK2_OK"
    # and the same numbers as the aligned layout
    assert torch.equal(C, ozk.dgemm(A.to(cuda), B.to(cuda), num_moduli=N))

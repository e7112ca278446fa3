"""FP64 matrix multiplication emulated on GB300 FP8 tensor cores (Ozaki-II scheme with
FP8 E4M3 digits, arXiv:2603.10634).

The compute path is libozk2.so (hand-written sm_103a CUDA behind the C ABI of
include/ozk2.h); this package is its thin binding.
"""
from ._lib import Ozk2Error  # noqa: F401
from .autograd import OzakiMatmul, matmul  # noqa: F401
from .tune import choose_moduli, choose_moduli_batch, choose_plan, choose_tile  # noqa: F401
from .ozk2 import (  # noqa: F401
    MODES,
    BatchPlan,
    dgemm_batched,
    workspace_size_batched,
    PHASES,
    crt,
    device_status,
    dgemm,
    dgemm_backward,
    backward_exponents,
    dgemm_host,
    fp8_gemm,
    get_timing,
    last_launch_count,
    moduli,
    residue_planes,
    residue_products,
    scales,
    set_timing,
    timeline,
    tile_width,
    workspace_size,
    workspace_size_backward,
    workspace_size_host,
)

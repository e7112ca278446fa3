"""Python binding of libozk2: argument marshalling only.

Every step of the emulated DGEMM runs in the library's CUDA kernels on the tensors'
device and torch's current stream; torch supplies device memory and streams.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(device=None):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _check_matrix(x, name, dtype=torch.float64):
    if not isinstance(x, torch.Tensor) or x.dim() != 2:
        raise ValueError(f"{name} must be a 2-D torch tensor")
    if x.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {x.dtype}")
    if not x.is_cuda:
        raise ValueError(f"{name} must live on a CUDA device")
    if x.size(1) > 1 and x.stride(1) != 1:
        raise ValueError(f"{name} must be row-major (unit stride along columns)")
    if x.size(0) > 1 and x.stride(0) == 0:
        raise ValueError(f"{name} has a broadcast (zero) row stride")


def _ld(x):
    return x.stride(0) if x.size(0) > 1 else max(1, x.size(1))


OP_N, OP_T = 0, 1
MODES = {"accurate": 0, "fast": 1}


def _operand(x, name, on_host=False):
    """(op, ld) of a float64 matrix that is row-major (op N) or the transpose of a
    row-major matrix (op T, e.g. ``Y.T``); the stored matrix is never copied.  CUDA
    tensors, or CPU tensors with on_host."""
    if not isinstance(x, torch.Tensor) or x.dim() != 2:
        raise ValueError(f"{name} must be a 2-D torch tensor")
    if x.dtype != torch.float64:
        raise TypeError(f"{name} must be torch.float64, got {x.dtype}")
    if x.is_cuda == on_host:
        raise ValueError(f"{name} must live {'in host memory' if on_host else 'on a CUDA device'}")
    rows, cols = x.shape
    s0, s1 = x.stride()
    if (rows > 1 and s0 == 0) or (cols > 1 and s1 == 0):
        raise ValueError(f"{name} has a broadcast (zero) stride; pass a materialised copy")
    if cols <= 1 or s1 == 1:
        return OP_N, (s0 if rows > 1 else max(1, cols))
    if rows <= 1 or s0 == 1:
        return OP_T, (s1 if cols > 1 else max(1, rows))
    raise ValueError(f"{name} must be row-major or the transpose of a row-major matrix")


def _mode(mode):
    if mode not in MODES:
        raise ValueError(f"mode must be one of {sorted(MODES)}")
    return MODES[mode]


def _block(block):
    if block is None:
        return 0, 0
    bm, bn = block
    if bm < 0 or bn < 0:
        raise ValueError("block sizes must be >= 0")
    return int(bm), int(bn)


class tile_width:
    """Context manager fixing the output tile width of the FP8 products (256 or 128; 0 for
    the library's rule) for the calls and batch plans made inside it (ozk2_set_tile_n,
    a process-wide setting, restored on exit)."""

    def __init__(self, tile_n):
        if tile_n not in (0, 128, 256):
            raise ValueError("tile_n must be 0, 128 or 256")
        self.tile_n = int(tile_n)
        self.prev = None

    def __enter__(self):
        self.prev = _lib.load().ozk2_set_tile_n(self.tile_n)
        return self

    def __exit__(self, *exc):
        _lib.load().ozk2_set_tile_n(self.prev)


def moduli(num_moduli=12):
    """The first N moduli of the hybrid list."""
    lib = _lib.load()
    buf = (ctypes.c_int32 * num_moduli)()
    if lib.ozk2_moduli(num_moduli, buf) != num_moduli:
        raise ValueError("num_moduli must be in 1..20")
    return list(buf)


def workspace_size(m, n, k, num_moduli=12, mode="accurate", block=None):
    bm, bn = _block(block)
    return int(_lib.load().ozk2_workspace_size_ex(m, n, k, num_moduli, _mode(mode), bm, bn))


def dgemm(A, B, num_moduli=12, out=None, workspace=None, mode="accurate", block=None):
    """C = A @ B in emulated FP64 (A: m x k, B: k x n, float64 CUDA tensors).

    A and B may each be row-major or the transpose of a row-major matrix (``X.T``);
    ``mode`` is "accurate" or "fast" (the two scalings of Sec. III-E); ``block`` =
    (block_m, block_n) runs independent emulations of those blocks of C (Sec. IV-C).
    ``workspace`` may be a uint8 CUDA tensor of at least ``workspace_size`` bytes;
    otherwise the library's own per-device workspace is used."""
    ta, lda = _operand(A, "A")
    tb, ldb = _operand(B, "B")
    m, k = A.shape
    k2, n = B.shape
    if k != k2:
        raise ValueError(f"inner dimensions differ: {tuple(A.shape)} @ {tuple(B.shape)}")
    if A.device != B.device:
        raise ValueError("A and B must be on the same device")
    md = _mode(mode)
    bm, bn = _block(block)
    if out is None:
        out = torch.empty((m, n), dtype=torch.float64, device=A.device)
    else:
        _check_matrix(out, "out")
        if tuple(out.shape) != (m, n):
            raise ValueError("out has the wrong shape")
    if workspace is not None and (workspace.dtype != torch.uint8 or not workspace.is_cuda):
        raise TypeError("workspace must be a uint8 CUDA tensor")
    lib = _lib.load()
    with torch.cuda.device(A.device):
        st = _stream(A.device)
        if ta == OP_N and tb == OP_N and md == 0 and bm == 0 and bn == 0:
            if workspace is None:
                s = lib.ozk2_dgemm(m, n, k, _ptr(A), lda, _ptr(B), ldb, _ptr(out), _ld(out), num_moduli, st)
            else:
                s = lib.ozk2_dgemm_ws(m, n, k, _ptr(A), lda, _ptr(B), ldb, _ptr(out), _ld(out), num_moduli,
                                      _ptr(workspace), workspace.numel(), st)
        else:
            s = lib.ozk2_dgemm_ex(ta, tb, m, n, k, _ptr(A), lda, _ptr(B), ldb, _ptr(out), _ld(out), num_moduli,
                                  md, bm, bn, _ptr(workspace), 0 if workspace is None else workspace.numel(), st)
    _lib.check(s, "ozk2_dgemm")
    return out


def workspace_size_backward(m, n, k, num_moduli=12):
    return int(_lib.load().ozk2_workspace_size_backward(m, n, k, num_moduli))


def dgemm_backward(A, B, dC, forward_workspace, num_moduli=12, need_dA=True, need_dB=True, workspace=None):
    """(dA, dB) = (dC @ B.T, A.T @ dC) for C = A @ B computed by ``dgemm(A, B, num_moduli,
    workspace=forward_workspace)`` (accurate mode, no blocking), reusing that call's
    exponents and digit planes (ozk2_dgemm_backward).  A, B, dC: row-major float64 CUDA
    tensors; forward_workspace: the uint8 tensor the forward ran in, unchanged since.
    An output not needed is returned as None."""
    for x, name in ((A, "A"), (B, "B"), (dC, "dC")):
        _check_matrix(x, name)
    m, k = A.shape
    k2, n = B.shape
    if k != k2 or tuple(dC.shape) != (m, n):
        raise ValueError("shapes do not match C = A @ B")
    if forward_workspace.dtype != torch.uint8 or not forward_workspace.is_cuda:
        raise TypeError("forward_workspace must be a uint8 CUDA tensor")
    if workspace is not None and (workspace.dtype != torch.uint8 or not workspace.is_cuda):
        raise TypeError("workspace must be a uint8 CUDA tensor")
    dA = torch.empty((m, k), dtype=torch.float64, device=A.device) if need_dA else None
    dB = torch.empty((k, n), dtype=torch.float64, device=A.device) if need_dB else None
    lib = _lib.load()
    with torch.cuda.device(A.device):
        s = lib.ozk2_dgemm_backward(m, n, k, _ptr(A), _ld(A), _ptr(B), _ld(B), _ptr(dC), _ld(dC), _ptr(dA),
                                    _ld(dA) if dA is not None else max(1, k), _ptr(dB),
                                    _ld(dB) if dB is not None else max(1, n), num_moduli, _ptr(forward_workspace),
                                    forward_workspace.numel(), _ptr(workspace),
                                    0 if workspace is None else workspace.numel(), _stream(A.device))
    _lib.check(s, "ozk2_dgemm_backward")
    return dA, dB


def backward_exponents(m, n, k, num_moduli=12, workspace=None, device=None):
    """(g, h): the exponents of dC's rows and columns used by the last dgemm_backward of
    these sizes (int32 CUDA tensors)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    g = torch.empty(m, dtype=torch.int32, device=dev)
    h = torch.empty(n, dtype=torch.int32, device=dev)
    s = _lib.load().ozk2_debug_backward_exponents(m, n, k, num_moduli, _ptr(workspace), _ptr(g), _ptr(h),
                                                  _stream(dev))
    _lib.check(s, "ozk2_debug_backward_exponents")
    return g, h


def workspace_size_host(m, n, k, num_moduli=12, mode="accurate"):
    return int(_lib.load().ozk2_workspace_size_host(m, n, k, num_moduli, _mode(mode)))


def dgemm_host(A, B, num_moduli=12, out=None, mode="accurate", workspace=None, device=None, sync=True,
               inputs_ready=False):
    """C = A @ B with A, B and C in host memory (float64 CPU tensors; A and B row-major
    or transposed views, C row-major; pinned memory lets the copies overlap the
    kernels).  The library moves the data and pipelines the copies with the kernels on
    ``device`` (default: the current CUDA device) and its current stream.  With
    ``sync`` the call waits for the stream, otherwise ``out`` is complete only once the
    stream is, and A, B (and ``out``) must be kept alive and A, B unchanged until then:
    the library reads them asynchronously and PyTorch does not know it (a freed pinned
    block may be handed out again while its upload is pending).  ``inputs_ready``
    (OZK2_HOST_INPUTS_READY): A and B are final when the call is made, so back-to-back
    calls in the library-owned workspace may upload their inputs while the previous
    call is still computing."""
    ta, lda = _operand(A, "A", on_host=True)
    tb, ldb = _operand(B, "B", on_host=True)
    m, k = A.shape
    k2, n = B.shape
    if k != k2:
        raise ValueError(f"inner dimensions differ: {tuple(A.shape)} @ {tuple(B.shape)}")
    if out is None:
        out = torch.empty((m, n), dtype=torch.float64, pin_memory=True)
    elif out.is_cuda or out.dtype != torch.float64 or out.dim() != 2 or tuple(out.shape) != (m, n) or (
            n > 1 and out.stride(1) != 1) or (m > 1 and out.stride(0) == 0):
        raise ValueError("out must be a row-major float64 host tensor of shape (m, n)")
    ldc = out.stride(0) if m > 1 else max(1, n)
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    if workspace is not None and (workspace.dtype != torch.uint8 or workspace.device != dev):
        raise TypeError("workspace must be a uint8 tensor on the device")
    lib = _lib.load()
    with torch.cuda.device(dev):
        st = torch.cuda.current_stream(dev)
        s = lib.ozk2_dgemm_host_ex(ta, tb, m, n, k, _ptr(A), lda, _ptr(B), ldb, _ptr(out), ldc, num_moduli,
                                   _mode(mode), 1 if inputs_ready else 0, _ptr(workspace),
                                   0 if workspace is None else workspace.numel(), ctypes.c_void_p(st.cuda_stream))
        _lib.check(s, "ozk2_dgemm_host")
        if sync:
            st.synchronize()
    return out


def _batch_arrays(As, Bs, outs):
    """Host arrays (ctypes) of a batch of row-major device problems."""
    count = len(As)
    if len(Bs) != count or (outs is not None and len(outs) != count):
        raise ValueError("As, Bs (and outs) must have the same length")
    I64 = ctypes.c_int64 * count
    P = ctypes.c_void_p * count
    m, n, k, lda, ldb, ldc = I64(), I64(), I64(), I64(), I64(), I64()
    pa, pb, pc = P(), P(), P()
    dev = As[0].device if count else None
    res = []
    for i, (A, B) in enumerate(zip(As, Bs)):
        _check_matrix(A, f"As[{i}]")
        _check_matrix(B, f"Bs[{i}]")
        if A.shape[1] != B.shape[0]:
            raise ValueError(f"problem {i}: inner dimensions differ")
        if A.device != dev or B.device != dev:
            raise ValueError("every operand must be on the same device")
        C = torch.empty((A.shape[0], B.shape[1]), dtype=torch.float64, device=dev) if outs is None else outs[i]
        _check_matrix(C, f"outs[{i}]")
        if tuple(C.shape) != (A.shape[0], B.shape[1]):
            raise ValueError(f"outs[{i}] has the wrong shape")
        m[i], k[i], n[i] = A.shape[0], A.shape[1], B.shape[1]
        lda[i], ldb[i], ldc[i] = _ld(A), _ld(B), _ld(C)
        pa[i], pb[i], pc[i] = A.data_ptr(), B.data_ptr(), C.data_ptr()
        res.append(C)
    return count, (m, n, k, pa, lda, pb, ldb, pc, ldc), res, dev


def workspace_size_batched(shapes, num_moduli=12, mode="accurate"):
    """Workspace bytes of a batch of (m, n, k) shapes."""
    count = len(shapes)
    I64 = ctypes.c_int64 * count
    m, n, k = I64(*[s[0] for s in shapes]), I64(*[s[1] for s in shapes]), I64(*[s[2] for s in shapes])
    return int(_lib.load().ozk2_workspace_size_batched(count, m, n, k, num_moduli, _mode(mode)))


class BatchPlan:
    """A batch of independent products C_i = A_i @ B_i (row-major float64 CUDA tensors)
    prepared once and executed with one launch per phase.  ``execute`` only enqueues
    device work, so it can be captured into a CUDA graph.  The plan keeps references to
    the operands and outputs it was built for."""

    def __init__(self, As, Bs, num_moduli=12, outs=None, mode="accurate", workspace=None, tile_n=None):
        self._lib = _lib.load()
        if tile_n is not None:
            with tile_width(tile_n):
                self.__init__(As, Bs, num_moduli, outs, mode, workspace)
            return
        count, arrs, self.outs, dev = _batch_arrays(As, Bs, outs)
        if count == 0:
            raise ValueError("empty batch")
        self.device = dev
        self._keep = (list(As), list(Bs), workspace)
        self._arrs = arrs
        self._plan = ctypes.c_void_p(0)
        with torch.cuda.device(dev):
            s = self._lib.ozk2_batch_plan_create(ctypes.byref(self._plan), count, *arrs, num_moduli, _mode(mode),
                                                 _ptr(workspace), 0 if workspace is None else workspace.numel(),
                                                 _stream(dev))
        _lib.check(s, "ozk2_batch_plan_create")

    def execute(self):
        with torch.cuda.device(self.device):
            s = self._lib.ozk2_batch_plan_execute(self._plan, _stream(self.device))
        _lib.check(s, "ozk2_batch_plan_execute")
        return self.outs

    def workspace_ptr(self):
        return self._lib.ozk2_batch_plan_workspace(self._plan)

    def tile_n(self):
        """Tile width the plan's residue products run with (0: both widths, chosen per
        problem)."""
        return int(self._lib.ozk2_batch_plan_tile_n(self._plan))

    def status(self):
        """Device flag status of the plan's workspace (synchronises the current stream)."""
        s = self._lib.ozk2_device_status(ctypes.c_void_p(self.workspace_ptr()), _stream(self.device))
        return _lib.STATUS.get(s, s)

    def close(self):
        if self._plan:
            torch.cuda.synchronize(self.device)
            self._lib.ozk2_batch_plan_destroy(self._plan)
            self._plan = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dgemm_batched(As, Bs, num_moduli=12, outs=None, mode="accurate", workspace=None):
    """[A_i @ B_i] for lists of row-major float64 CUDA tensors, one launch per phase for
    the whole batch (ozk2_dgemm_batched)."""
    count, arrs, res, dev = _batch_arrays(As, Bs, outs)
    if count == 0:
        return res
    lib = _lib.load()
    with torch.cuda.device(dev):
        s = lib.ozk2_dgemm_batched(count, *arrs, num_moduli, _mode(mode), _ptr(workspace),
                                   0 if workspace is None else workspace.numel(), _stream(dev))
    _lib.check(s, "ozk2_dgemm_batched")
    return res


def device_status(workspace=None, device=None):
    """Synchronise the current stream and return (and clear) the device flag status name."""
    lib = _lib.load()
    s = lib.ozk2_device_status(_ptr(workspace), _stream(device))
    return _lib.STATUS.get(s, s)


def set_timing(enable=True):
    _lib.load().ozk2_set_timing(1 if enable else 0)


PHASES = ("scale", "bound_gemm", "exponents", "residues", "residue_gemm", "crt")


def get_timing():
    """Per-phase milliseconds of the last timed call (dict), or None."""
    buf = (ctypes.c_float * 6)()
    n = _lib.load().ozk2_get_timing(buf, 6)
    if n < 0:
        return None
    return {PHASES[i]: float(buf[i]) for i in range(n)}


def timeline():
    """Milliseconds from the start of the last timed call to the end of each phase."""
    buf = (ctypes.c_float * 6)()
    n = _lib.load().ozk2_debug_timeline(buf, 6)
    if n < 0:
        return None
    return dict(zip(PHASES, list(buf)[:n]))


def last_launch_count():
    return int(_lib.load().ozk2_last_launch_count())


# ----------------------------------------------------------------- parity hooks

def kp_of(k):
    return 32 * ((k + 31) // 32)


def num_planes(num_moduli):
    return 2 * num_moduli if num_moduli <= 6 else 3 * num_moduli - 6


def fp8_gemm(A8, B8, k=None):
    """D = A8 @ B8^T, FP8 E4M3 codes (uint8, K-major, row stride multiple of 16) -> float32."""
    m, n = A8.shape[0], B8.shape[0]
    k = A8.shape[1] if k is None else k
    D = torch.empty((m, n), dtype=torch.float32, device=A8.device)
    lib = _lib.load()
    s = lib.ozk2_debug_fp8_gemm(m, n, k, _ptr(A8), A8.stride(0), _ptr(B8), B8.stride(0), _ptr(D), n,
                                _stream(A8.device))
    _lib.check(s, "ozk2_debug_fp8_gemm")
    return D


def scales(A, B, num_moduli=12, mode="accurate"):
    """Scaling intermediates: dict of e, f, eprime, fprime, R, S, and in accurate mode Abar
    (m x kp) and BbarT (n x kp).  In fast mode R and S are the round-up sums of squares of
    the scaled rows of A and columns of B.  A, B as for ``dgemm``."""
    ta, lda = _operand(A, "A")
    tb, ldb = _operand(B, "B")
    md = _mode(mode)
    m, k = A.shape
    n = B.shape[1]
    dev = A.device
    kp = kp_of(k)
    out = dict(e=torch.empty(m, dtype=torch.int32, device=dev), f=torch.empty(n, dtype=torch.int32, device=dev),
               eprime=torch.empty(m, dtype=torch.int32, device=dev),
               fprime=torch.empty(n, dtype=torch.int32, device=dev),
               R=torch.empty(m, dtype=torch.float32, device=dev), S=torch.empty(n, dtype=torch.float32, device=dev))
    if md == 0:
        out["Abar"] = torch.empty((m, kp), dtype=torch.uint8, device=dev)
        out["BbarT"] = torch.empty((n, kp), dtype=torch.uint8, device=dev)
    lib = _lib.load()
    s = lib.ozk2_debug_scales_ex(ta, tb, m, n, k, _ptr(A), lda, _ptr(B), ldb, num_moduli, md, _ptr(out["e"]),
                                 _ptr(out["f"]), _ptr(out["eprime"]), _ptr(out["fprime"]), _ptr(out["R"]),
                                 _ptr(out["S"]), _ptr(out.get("Abar")), _ptr(out.get("BbarT")), _stream(dev))
    _lib.check(s, "ozk2_debug_scales_ex")
    return out


def residue_planes(A, B, e, f, num_moduli=12):
    """Digit planes (uint8 E4M3 codes): planesA (M_N x m x kp), planesB (M_N x n x kp)."""
    m, k = A.shape
    n = B.shape[1]
    kp = kp_of(k)
    M = num_planes(num_moduli)
    pa = torch.zeros((M, m, kp), dtype=torch.uint8, device=A.device)
    pb = torch.zeros((M, n, kp), dtype=torch.uint8, device=A.device)
    e = e.to(device=A.device, dtype=torch.int32).contiguous()
    f = f.to(device=A.device, dtype=torch.int32).contiguous()
    s = _lib.load().ozk2_debug_residue_planes(m, n, k, _ptr(A), _ld(A), _ptr(B), _ld(B), num_moduli, _ptr(e),
                                              _ptr(f), _ptr(pa), _ptr(pb), _stream(A.device))
    _lib.check(s, "ozk2_debug_residue_planes")
    return pa, pb


def residue_products(A, B, e, f, num_moduli=12):
    """C'_l for l = 1..N as an int16 tensor N x m x n."""
    m, k = A.shape
    n = B.shape[1]
    out = torch.empty((num_moduli, m, n), dtype=torch.int16, device=A.device)
    e = e.to(device=A.device, dtype=torch.int32).contiguous()
    f = f.to(device=A.device, dtype=torch.int32).contiguous()
    s = _lib.load().ozk2_debug_residue_products(m, n, k, _ptr(A), _ld(A), _ptr(B), _ld(B), num_moduli, _ptr(e),
                                                _ptr(f), _ptr(out), _stream(A.device))
    _lib.check(s, "ozk2_debug_residue_products")
    return out


def crt(Cres, e, f, num_moduli=None):
    """C from residue products (N x m x n int16) and exponents."""
    N, m, n = Cres.shape
    num_moduli = N if num_moduli is None else num_moduli
    Cres = Cres.contiguous()
    dev = Cres.device
    e = e.to(device=dev, dtype=torch.int32).contiguous()
    f = f.to(device=dev, dtype=torch.int32).contiguous()
    C = torch.empty((m, n), dtype=torch.float64, device=dev)
    s = _lib.load().ozk2_debug_crt(m, n, num_moduli, _ptr(Cres), _ptr(e), _ptr(f), _ptr(C), n, _stream(dev))
    _lib.check(s, "ozk2_debug_crt")
    return C

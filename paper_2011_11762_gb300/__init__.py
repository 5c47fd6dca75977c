"""Python binding of libcht: block-sparse quadtree C = A*B on a GB300 GPU.

A thin layer over the C ABI in ``include/cht.h`` (same names, argument
marshalling only): device memory and streams come from PyTorch, every step
of the product runs in the library's CUDA kernels.  There is no CPU
fallback; if the library cannot be loaded, calls raise.
"""

from __future__ import annotations

import ctypes

import torch

from . import _lib

CHT_FP64 = 0
CHT_SPLIT_BF16 = 1

OPT_SCHEDULE = 0
OPT_WAIT_BUDGET_NS = 1
OPT_CTAS_PER_SM = 2
OPT_FP64_ENGINE = 3
OPT_SPLIT_SINGLE = 4

CHT_OK = 0
CHT_ERR_INVALID = -1
CHT_ERR_SHAPE = -2
CHT_ERR_DUPLICATE = -3
CHT_ERR_OOM = -4
CHT_ERR_CUDA = -5
CHT_ERR_TIMEOUT = -6
CHT_ERR_UNSUPPORTED = -7

_VP = ctypes.c_void_p


class ChtError(RuntimeError):
    """A libcht call returned an error status."""

    def __init__(self, code: int, where: str):
        lib = _lib.load()
        name = lib.cht_status_str(code).decode()
        detail = lib.cht_last_error().decode()
        super().__init__(f"{where}: {name} ({detail})")
        self.code = code


def _check(rc: int, where: str):
    if rc != CHT_OK:
        raise ChtError(rc, where)


def _stream(stream=None) -> _VP:
    if stream is None:
        stream = torch.cuda.current_stream()
    return _VP(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class _DevView:
    """__cuda_array_interface__ over memory owned by a libcht handle; keeps
    the handle alive while a tensor views it."""

    def __init__(self, owner, ptr: int, shape, typestr: str):
        self.owner = owner
        self.__cuda_array_interface__ = {
            "shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
            "version": 3, "strides": None, "stream": None,
        }


class Matrix:
    """A block-sparse matrix held by libcht (leaves in Morton order)."""

    def __init__(self, handle: _VP, owned: bool = True, parent=None):
        self._h = handle
        self._owned = owned
        self._parent = parent  # keeps a batch alive for its output views
        n, b, nb = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
        _check(_lib.load().cht_mat_info(handle, ctypes.byref(n), ctypes.byref(b),
                                        ctypes.byref(nb)), "cht_mat_info")
        self.n, self.b, self.nblocks = n.value, b.value, nb.value

    def __del__(self):
        if getattr(self, "_owned", False) and self._h:
            try:
                _lib.load().cht_mat_free(self._h)
            except Exception:
                pass
            self._h = None

    @property
    def handle(self) -> _VP:
        return self._h

    def _arrays(self):
        v, r, c = _VP(), _VP(), _VP()
        _check(_lib.load().cht_mat_leaves(self._h, ctypes.byref(v), ctypes.byref(r),
                                          ctypes.byref(c)), "cht_mat_leaves")
        return v.value, r.value, c.value

    def values(self) -> torch.Tensor:
        """Zero-copy float64 view [nblocks, b, b] of the leaf values."""
        v, _, _ = self._arrays()
        if self.nblocks == 0:
            return torch.zeros((0, self.b, self.b), dtype=torch.float64, device="cuda")
        return torch.as_tensor(_DevView(self, v, (self.nblocks, self.b, self.b), "<f8"),
                               device="cuda")

    def coords(self):
        """(brow, bcol) int32 views of the leaf coordinates (Morton order)."""
        _, r, c = self._arrays()
        if self.nblocks == 0:
            z = torch.zeros(0, dtype=torch.int32, device="cuda")
            return z, z.clone()
        return (torch.as_tensor(_DevView(self, r, (self.nblocks,), "<i4"), device="cuda"),
                torch.as_tensor(_DevView(self, c, (self.nblocks,), "<i4"), device="cuda"))

    def to_dense(self, stream=None) -> torch.Tensor:
        out = torch.empty((self.n, self.n), dtype=torch.float64, device="cuda")
        _check(_lib.load().cht_to_dense(self._h, _VP(out.data_ptr()), self.n,
                                        _stream(stream)), "cht_to_dense")
        return out

    def like(self, stream=None) -> "Matrix":
        h = _VP()
        _check(_lib.load().cht_mat_like(self._h, _stream(stream), ctypes.byref(h)),
               "cht_mat_like")
        return Matrix(h)


class Plan:
    """Symbolic result of A*B: C's pattern, pair segments, schedule."""

    def __init__(self, handle: _VP, A: Matrix, B: Matrix):
        self._h = handle
        self.A, self.B = A, B
        nc, npairs = ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.load().cht_plan_info(handle, ctypes.byref(nc), ctypes.byref(npairs)),
               "cht_plan_info")
        self.nnzb_C, self.npairs = nc.value, npairs.value
        self.n, self.b = A.n, A.b

    def __del__(self):
        if getattr(self, "_h", None):
            try:
                _lib.load().cht_plan_free(self._h)
            except Exception:
                pass
            self._h = None

    @property
    def handle(self) -> _VP:
        return self._h

    @property
    def useful_flops(self) -> int:
        return 2 * self.b ** 3 * self.npairs

    def arrays(self) -> dict:
        """Host copies of the plan's arrays (for tests)."""
        ptrs = [_VP() for _ in range(6)]
        _check(_lib.load().cht_plan_arrays(self._h, *[ctypes.byref(p) for p in ptrs]),
               "cht_plan_arrays")
        nc, npairs = self.nnzb_C, self.npairs

        def grab(p, n, typestr, dtype):
            if n == 0 or not p.value:
                return torch.zeros(0, dtype=dtype)
            return torch.as_tensor(_DevView(self, p.value, (n,), typestr),
                                   device="cuda").cpu().clone()

        return {
            "cseg": grab(ptrs[0], nc + 1, "<i8", torch.int64),
            "pair_a": grab(ptrs[1], npairs, "<i4", torch.int32),
            "pair_b": grab(ptrs[2], npairs, "<i4", torch.int32),
            "crow": grab(ptrs[3], nc, "<i4", torch.int32),
            "ccol": grab(ptrs[4], nc, "<i4", torch.int32),
            "order": grab(ptrs[5], nc, "<i4", torch.int32),
        }


def cht_mat_from_blocks(n: int, b: int, brow: torch.Tensor, bcol: torch.Tensor,
                        vals: torch.Tensor, stream=None) -> Matrix:
    """Build a matrix from leaf coordinates and values (CUDA tensors)."""
    brow = brow.to(device="cuda", dtype=torch.int32).contiguous()
    bcol = bcol.to(device="cuda", dtype=torch.int32).contiguous()
    vals = vals.to(device="cuda", dtype=torch.float64).contiguous()
    nblk = brow.numel()
    if bcol.numel() != nblk or vals.numel() != nblk * b * b:
        raise ValueError("brow, bcol and vals sizes disagree")
    h = _VP()
    _check(_lib.load().cht_mat_from_blocks(
        n, b, nblk, _VP(brow.data_ptr() if nblk else None),
        _VP(bcol.data_ptr() if nblk else None), _VP(vals.data_ptr() if nblk else None),
        _stream(stream), ctypes.byref(h)), "cht_mat_from_blocks")
    return Matrix(h)


def from_block_matrix(m, stream=None) -> Matrix:
    """Upload a host ``workloads.BlockMatrix``."""
    return cht_mat_from_blocks(m.n, m.b, torch.from_numpy(m.brow), torch.from_numpy(m.bcol),
                               torch.from_numpy(m.vals), stream)


def cht_symbolic_multiply(A: Matrix, B: Matrix, stream=None) -> Plan:
    h = _VP()
    _check(_lib.load().cht_symbolic_multiply(A.handle, B.handle, _stream(stream),
                                             ctypes.byref(h), None, None),
           "cht_symbolic_multiply")
    return Plan(h, A, B)


def cht_symbolic_multiply_spamm(A: Matrix, B: Matrix, tau: float, stream=None) -> Plan:
    """Sparse approximate plan: pairs with ||A leaf|| ||B leaf|| < tau dropped."""
    h = _VP()
    _check(_lib.load().cht_symbolic_multiply_spamm(A.handle, B.handle, float(tau),
                                                   _stream(stream), ctypes.byref(h), None,
                                                   None), "cht_symbolic_multiply_spamm")
    return Plan(h, A, B)


def cht_symbolic_multiply_symsquare(A: Matrix, stream=None) -> Plan:
    """Plan of the upper triangle (leaf rows <= leaf columns) of A*A for a
    symmetric A; multiply with cht_multiply(plan, A, A)."""
    h = _VP()
    _check(_lib.load().cht_symbolic_multiply_symsquare(A.handle, _stream(stream),
                                                       ctypes.byref(h), None, None),
           "cht_symbolic_multiply_symsquare")
    return Plan(h, A, A)


def cht_symbolic_multiply_upper(A: Matrix, B: Matrix, stream=None) -> Plan:
    """Plan of the upper-triangle leaves (I <= J) of A*B (for a product known
    to be symmetric); multiply with cht_multiply(plan, A, B)."""
    h = _VP()
    _check(_lib.load().cht_symbolic_multiply_upper(A.handle, B.handle, _stream(stream),
                                                   ctypes.byref(h), None, None),
           "cht_symbolic_multiply_upper")
    return Plan(h, A, B)


def cht_mat_mirror_upper(U: Matrix, stream=None) -> Matrix:
    """The full symmetric matrix from its upper-triangle leaves."""
    h = _VP()
    _check(_lib.load().cht_mat_mirror_upper(U.handle, _stream(stream), ctypes.byref(h)),
           "cht_mat_mirror_upper")
    return Matrix(h)


CHT_TRUNC_FRO = 0
CHT_TRUNC_MAX = 1


def cht_add(alpha: float, A: Matrix, beta: float, B: Matrix, stream=None) -> Matrix:
    """alpha*A + beta*B on the union of the leaf patterns."""
    h = _VP()
    _check(_lib.load().cht_add(float(alpha), A.handle, float(beta), B.handle, _stream(stream),
                               ctypes.byref(h)), "cht_add")
    return Matrix(h)


def cht_add_identity(alpha: float, A: Matrix, beta: float, stream=None) -> Matrix:
    """alpha*A + beta*I."""
    h = _VP()
    _check(_lib.load().cht_add_identity(float(alpha), A.handle, float(beta), _stream(stream),
                                        ctypes.byref(h)), "cht_add_identity")
    return Matrix(h)


def cht_truncate(M: Matrix, eps: float, kind: int = CHT_TRUNC_FRO, stream=None):
    """(T, removed): M without its small leaves; removed = the Frobenius
    (CHT_TRUNC_FRO) or max-norm (CHT_TRUNC_MAX) size of what was removed."""
    h = _VP()
    rem = ctypes.c_double(0.0)
    _check(_lib.load().cht_truncate(M.handle, float(eps), int(kind), _stream(stream),
                                    ctypes.byref(h), ctypes.byref(rem)), "cht_truncate")
    return Matrix(h), rem.value


def cht_multiply(plan: Plan, A: Matrix, B: Matrix, mode: int = CHT_FP64, nslices: int = 0,
                 out: Matrix | None = None, stream=None, sync: bool = False):
    """C = A*B on the plan's pattern.  Returns (C, err_bound or None); with
    ``sync`` the call waits and raises on a device-side failure."""
    h = _VP(out.handle.value if out is not None else None)
    err = ctypes.c_double(0.0)
    _check(_lib.load().cht_multiply(plan.handle, A.handle, B.handle, mode, nslices,
                                    _stream(stream), ctypes.byref(h),
                                    ctypes.byref(err) if sync else None), "cht_multiply")
    C = out if out is not None else Matrix(h)
    return C, (err.value if sync else None)


def cht_multiply_to_host(plan: Plan, A: Matrix, B: Matrix, out: torch.Tensor,
                         nchunks: int = 8, stream=None) -> torch.Tensor:
    """FP64 C = A*B written into the host tensor `out` (float64, shape
    [nnzb_C, b, b], ideally pinned) while it is computed; the stream is
    ordered after the last copy."""
    if out.device.type != "cpu" or out.dtype != torch.float64 or not out.is_contiguous():
        raise ValueError("out must be a contiguous float64 host tensor")
    if out.numel() != plan.nnzb_C * A.b * A.b:
        raise ValueError("out must hold nnzb_C * b * b values")
    _check(_lib.load().cht_multiply_to_host(plan.handle, A.handle, B.handle, _stream(stream),
                                            _VP(out.data_ptr()), int(nchunks)),
           "cht_multiply_to_host")
    return out


def cht_multiply_backward(plan: Plan | None, A: Matrix, B: Matrix, dC: Matrix,
                          recompute_pairs: bool = False, dA: Matrix | None = None,
                          dB: Matrix | None = None, want_dA: bool = True,
                          want_dB: bool = True, stream=None):
    """(dA, dB) = (dC B^T on A's pattern, A^T dC on B's pattern)."""
    ha = _VP(dA.handle.value if dA is not None else None)
    hb = _VP(dB.handle.value if dB is not None else None)
    _check(_lib.load().cht_multiply_backward(
        plan.handle if plan is not None else None, A.handle, B.handle, dC.handle,
        1 if recompute_pairs else 0, _stream(stream),
        ctypes.byref(ha) if want_dA else None, ctypes.byref(hb) if want_dB else None),
        "cht_multiply_backward")
    ra = (dA if dA is not None else Matrix(ha)) if want_dA else None
    rb = (dB if dB is not None else Matrix(hb)) if want_dB else None
    return ra, rb


class Batch:
    """Many independent products in one persistent launch (cht_batch_*).

    Keeps the plans and matrices it was built from alive.  ``run()`` only
    launches kernels, so it can be captured in a CUDA graph."""

    def __init__(self, plans, As, Bs, mode: int = CHT_FP64, nslices: int = 0, stream=None):
        n = len(plans)
        if not (n == len(As) == len(Bs)) or n == 0:
            raise ValueError("plans, As and Bs must be non-empty and of equal length")
        arr = lambda xs: (_VP * n)(*[x.handle.value for x in xs])
        h = _VP()
        _check(_lib.load().cht_batch_create(n, arr(plans), arr(As), arr(Bs), mode, nslices,
                                            _stream(stream), ctypes.byref(h)),
               "cht_batch_create")
        self._h = h
        self._keep = (list(plans), list(As), list(Bs))
        self.count = n
        self.mode = mode
        self.useful_flops = sum(p.useful_flops for p in plans)

    def __del__(self):
        if getattr(self, "_h", None):
            try:
                _lib.load().cht_batch_free(self._h)
            except Exception:
                pass
            self._h = None

    def run(self, stream=None):
        _check(_lib.load().cht_batch_run(self._h, _stream(stream)), "cht_batch_run")

    def output(self, i: int) -> Matrix:
        h = _VP()
        _check(_lib.load().cht_batch_output(self._h, i, ctypes.byref(h)), "cht_batch_output")
        return Matrix(h, owned=False, parent=self)


def cht_to_dense(M: Matrix, stream=None) -> torch.Tensor:
    return M.to_dense(stream)


def set_option(option: int, value: int):
    _check(_lib.load().cht_set_option(option, value), "cht_set_option")


def get_option(option: int) -> int:
    v = ctypes.c_int64()
    _check(_lib.load().cht_get_option(option, ctypes.byref(v)), "cht_get_option")
    return v.value


def sync_status(stream=None):
    """Wait for the stream; raise on a recorded device-side failure."""
    _check(_lib.load().cht_sync_status(_stream(stream)), "cht_sync_status")


def launch_count() -> int:
    return int(_lib.load().cht_launch_count())


def measure_fp64_peak(engine: int = 0, stream=None) -> float:
    t = ctypes.c_double()
    _check(_lib.load().cht_measure_fp64_peak(engine, _stream(stream), ctypes.byref(t)),
           "cht_measure_fp64_peak")
    return t.value


def measure_fp64_peak_cfg(engine: int, chains: int, threads: int, ctas_per_sm: int,
                          stream=None) -> float:
    t = ctypes.c_double()
    _check(_lib.load().cht_measure_fp64_peak_cfg(engine, chains, threads, ctas_per_sm,
                                                 _stream(stream), ctypes.byref(t)),
           "cht_measure_fp64_peak_cfg")
    return t.value


def library_path() -> str:
    return _lib.lib_path()


def load():
    """Load (building if needed) the native library."""
    return _lib.load()

"""Python access to the CPU oracle (ctypes over oracle/oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the
benchmark's CPU-baseline leg are the only users.  Nothing here imports the
GPU library, and the GPU library never imports this.
"""

from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build

_I32P = ctypes.POINTER(ctypes.c_int32)
_I64P = ctypes.POINTER(ctypes.c_int64)
_F64P = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p

_libs: dict = {}

_ERR = {-1: "invalid argument", -2: "shape mismatch", -3: "duplicate leaf",
        -4: "out of memory"}


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle error {code}: {_ERR.get(code, '?')}")
        self.code = code


def load(mutant: int = 0):
    """The oracle library (built on first use)."""
    if mutant in _libs:
        return _libs[mutant]
    lib = ctypes.CDLL(_build.build(mutant))
    lib.orc_build.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int64,
                              _I32P, _I32P, _F64P, ctypes.POINTER(_VP)]
    lib.orc_multiply.argtypes = [_VP, _VP, ctypes.POINTER(_VP), _I64P]
    lib.orc_multiply_spamm.argtypes = [_VP, _VP, ctypes.c_double, ctypes.POINTER(_VP), _I64P]
    lib.orc_multiply_upper.argtypes = [_VP, _VP, ctypes.POINTER(_VP), _I64P]
    lib.orc_mirror_upper.argtypes = [_VP, ctypes.POINTER(_VP)]
    lib.orc_add.argtypes = [ctypes.c_double, _VP, ctypes.c_double, _VP, ctypes.POINTER(_VP)]
    lib.orc_add_identity.argtypes = [ctypes.c_double, _VP, ctypes.c_double,
                                     ctypes.POINTER(_VP)]
    lib.orc_truncate.argtypes = [_VP, ctypes.c_double, ctypes.c_int, ctypes.POINTER(_VP),
                                 ctypes.POINTER(ctypes.c_double)]
    lib.orc_transpose.argtypes = [_VP, ctypes.POINTER(_VP)]
    lib.orc_restrict.argtypes = [_VP, _VP, ctypes.POINTER(_VP)]
    lib.orc_backward.argtypes = [_VP, _VP, _VP, ctypes.POINTER(_VP),
                                 ctypes.POINTER(_VP)]
    lib.orc_leaf_product.argtypes = [_VP, _VP, ctypes.c_int64, ctypes.c_int64,
                                     _F64P, ctypes.POINTER(ctypes.c_int)]
    lib.orc_nleaves.argtypes = [_VP]
    lib.orc_nleaves.restype = ctypes.c_int64
    lib.orc_extract.argtypes = [_VP, _I32P, _I32P, _F64P]
    lib.orc_dim.argtypes = [_VP]
    lib.orc_dim.restype = ctypes.c_int64
    lib.orc_leafsize.argtypes = [_VP]
    lib.orc_leafsize.restype = ctypes.c_int32
    lib.orc_free.argtypes = [_VP]
    lib.orc_free.restype = None
    lib.orc_threads.restype = ctypes.c_int
    _libs[mutant] = lib
    return lib


def _check(rc: int):
    if rc != 0:
        raise OracleError(rc)


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


class OMatrix:
    """A quadtree matrix held by the oracle."""

    def __init__(self, handle, lib):
        self._h = handle
        self._lib = lib

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.orc_free(self._h)
            self._h = None

    @classmethod
    def from_blocks(cls, n: int, b: int, brow, bcol, vals, mutant: int = 0):
        lib = load(mutant)
        brow = np.ascontiguousarray(brow, dtype=np.int32)
        bcol = np.ascontiguousarray(bcol, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.float64)
        h = _VP()
        _check(lib.orc_build(n, b, brow.shape[0], _ptr(brow, _I32P),
                             _ptr(bcol, _I32P), _ptr(vals, _F64P),
                             ctypes.byref(h)))
        return cls(h, lib)

    @classmethod
    def from_block_matrix(cls, m, mutant: int = 0):
        return cls.from_blocks(m.n, m.b, m.brow, m.bcol, m.vals, mutant)

    @property
    def n(self) -> int:
        return int(self._lib.orc_dim(self._h))

    @property
    def b(self) -> int:
        return int(self._lib.orc_leafsize(self._h))

    def nleaves(self) -> int:
        return int(self._lib.orc_nleaves(self._h))

    def multiply(self, other: "OMatrix"):
        """(C, npairs) for C = self * other."""
        h = _VP()
        np_ = ctypes.c_int64(0)
        _check(self._lib.orc_multiply(self._h, other._h, ctypes.byref(h),
                                      ctypes.byref(np_)))
        return OMatrix(h, self._lib), int(np_.value)

    def multiply_spamm(self, other: "OMatrix", tau: float):
        """(C, npairs) for the sparse approximate product with threshold tau."""
        h = _VP()
        np_ = ctypes.c_int64(0)
        _check(self._lib.orc_multiply_spamm(self._h, other._h, float(tau), ctypes.byref(h),
                                            ctypes.byref(np_)))
        return OMatrix(h, self._lib), int(np_.value)

    def multiply_upper(self, other: "OMatrix"):
        """(C, npairs) for the leaves (I, J), I <= J, of self * other."""
        h = _VP()
        np_ = ctypes.c_int64(0)
        _check(self._lib.orc_multiply_upper(self._h, other._h, ctypes.byref(h),
                                            ctypes.byref(np_)))
        return OMatrix(h, self._lib), int(np_.value)

    def mirror_upper(self) -> "OMatrix":
        """The symmetric matrix whose upper-triangle leaves are self's."""
        h = _VP()
        _check(self._lib.orc_mirror_upper(self._h, ctypes.byref(h)))
        return OMatrix(h, self._lib)

    def add(self, alpha: float, other: "OMatrix", beta: float) -> "OMatrix":
        """alpha * self + beta * other on the union pattern."""
        h = _VP()
        _check(self._lib.orc_add(float(alpha), self._h, float(beta), other._h, ctypes.byref(h)))
        return OMatrix(h, self._lib)

    def add_identity(self, alpha: float, beta: float) -> "OMatrix":
        """alpha * self + beta * I."""
        h = _VP()
        _check(self._lib.orc_add_identity(float(alpha), self._h, float(beta), ctypes.byref(h)))
        return OMatrix(h, self._lib)

    def truncate(self, eps: float, kind: int = 0):
        """(T, removed): leaf truncation with Frobenius (kind 0) or max-norm
        (kind 1) error control."""
        h = _VP()
        rem = ctypes.c_double(0.0)
        _check(self._lib.orc_truncate(self._h, float(eps), int(kind), ctypes.byref(h),
                                      ctypes.byref(rem)))
        return OMatrix(h, self._lib), float(rem.value)

    def __matmul__(self, other: "OMatrix") -> "OMatrix":
        return self.multiply(other)[0]

    def transpose(self) -> "OMatrix":
        h = _VP()
        _check(self._lib.orc_transpose(self._h, ctypes.byref(h)))
        return OMatrix(h, self._lib)

    def restrict(self, pattern: "OMatrix") -> "OMatrix":
        h = _VP()
        _check(self._lib.orc_restrict(self._h, pattern._h, ctypes.byref(h)))
        return OMatrix(h, self._lib)

    def leaves(self, values: bool = True):
        """(brow, bcol, vals) of the stored leaves in Morton order."""
        k = self.nleaves()
        b = self.b
        brow = np.zeros(k, dtype=np.int32)
        bcol = np.zeros(k, dtype=np.int32)
        vals = np.zeros((k, b, b), dtype=np.float64) if values else None
        _check(self._lib.orc_extract(self._h, _ptr(brow, _I32P),
                                     _ptr(bcol, _I32P),
                                     _ptr(vals, _F64P) if values else None))
        return brow, bcol, vals

    def pattern(self) -> set:
        r, c, _ = self.leaves(values=False)
        return set(zip(r.tolist(), c.tolist()))

    def to_dense(self) -> np.ndarray:
        brow, bcol, vals = self.leaves()
        n, b = self.n, self.b
        out = np.zeros((n, n), dtype=np.float64)
        for i in range(brow.shape[0]):
            out[brow[i] * b:(brow[i] + 1) * b, bcol[i] * b:(bcol[i] + 1) * b] = vals[i]
        return out


def leaf_product(a: OMatrix, b: OMatrix, I: int, J: int):
    """(values, present) of leaf (I, J) of a*b from the definition."""
    out = np.zeros((a.b, a.b), dtype=np.float64)
    present = ctypes.c_int(0)
    _check(a._lib.orc_leaf_product(a._h, b._h, I, J, _ptr(out, _F64P),
                                   ctypes.byref(present)))
    return out, bool(present.value)


def backward(a: OMatrix, b: OMatrix, dc: OMatrix):
    """(dA, dB): dA = dC B^T on A's pattern, dB = A^T dC on B's pattern."""
    ha, hb = _VP(), _VP()
    _check(a._lib.orc_backward(a._h, b._h, dc._h, ctypes.byref(ha),
                               ctypes.byref(hb)))
    return OMatrix(ha, a._lib), OMatrix(hb, a._lib)


def threads(mutant: int = 0) -> int:
    return int(load(mutant).orc_threads())


def morton_key(brow, bcol) -> np.ndarray:
    """Morton (Z-order) key of leaf coordinates: bit k of the row goes to bit
    2k+1, bit k of the column to bit 2k (quadrant order 11, 12, 21, 22)."""
    r = np.asarray(brow, dtype=np.int64)
    c = np.asarray(bcol, dtype=np.int64)
    key = np.zeros(r.shape, dtype=np.int64)
    for k in range(31):
        key |= ((r >> k) & 1) << (2 * k + 1)
        key |= ((c >> k) & 1) << (2 * k)
    return key


__all__ = ["OMatrix", "OracleError", "leaf_product", "backward", "load",
           "threads", "morton_key"]

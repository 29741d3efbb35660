"""ctypes front end of the FP64 CPU oracle (``gscl_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline / reference leg are the only callers.  Nothing in the CUDA
library imports this module, and this module imports nothing from it.

The oracle's grids are plain numpy float64 arrays of shape
``(nz + 2hz, ny + 2hy, nx + 2hx)`` (x fastest) paired with their halo widths;
2D grids use ``nz = 1, hz = 0``.  Stencil operators are lists of terms
``(dx, dy, dz, in, coef, out, w)`` with the meaning given in the C file's
header (Section 3 of the paper: an operator reads fixed offsets of several
grids around the core element and writes the core element of its outputs;
it may also return a value, which ``do_reduce`` reduces).

Parity status: every function here is pinned by tests under ``tests/``
(closed forms, invariants, brute force); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

VALUE = 254  # term input/output code: the operator's returned value
NONE = 255   # coefficient code: no coefficient grid

SUM, MAXABS, L2 = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gscl_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")


def build(force: bool = False, mutant: int = 0, timing: bool = False) -> str:
    """Compiles the oracle with plain gcc: -O2, no FMA contraction, no fast-math.

    ``mutant`` > 0 builds a copy with one planted mistake (tests only).
    ``timing`` builds the copy that is only timed, as the CPU baseline:
    -O3 -march=native -fopenmp (threads set by ``threads``), still without FMA
    contraction; it returns the checker's numbers (see the C file)."""
    if timing:
        path = os.path.join(_LIB_DIR, "liboracle_omp.so")
        flags = ["-O3", "-march=native", "-fopenmp"]
    else:
        path = _LIB if mutant == 0 else os.path.join(_LIB_DIR, f"liboracle_mutant{mutant}.so")
        flags = ["-O2"]
    if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        os.makedirs(_LIB_DIR, exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c99", *flags, "-ffp-contract=off", "-fno-fast-math",
                               f"-DORC_MUTANT={int(mutant)}", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, path)
    return path


def threads(n: int = 0) -> int:
    """Sets the timing build's thread count (n >= 1) and returns the count in
    effect (1 for the checker build)."""
    return int(_get_lib().orc_threads(int(n)))


class _Term(ctypes.Structure):
    _fields_ = [("dx", ctypes.c_int32), ("dy", ctypes.c_int32), ("dz", ctypes.c_int32),
                ("in_", ctypes.c_int32), ("coef", ctypes.c_int32), ("out", ctypes.c_int32),
                ("w", ctypes.c_double)]


class _Extent(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64)]


class _Grid(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("hx", ctypes.c_int32), ("hy", ctypes.c_int32),
                ("hz", ctypes.c_int32)]


_lib = None
_lib_path = None


def use_library(path=None):
    """Selects which compiled oracle the calls below use (None: the normal build)."""
    global _lib, _lib_path
    _lib, _lib_path = None, path


def _get_lib():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_lib_path or build())
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.orc_do_all.argtypes = [ctypes.POINTER(_Extent), ctypes.c_int, ctypes.POINTER(_Grid),
                                   ctypes.c_int, ctypes.POINTER(_Grid), ctypes.c_int,
                                   ctypes.POINTER(_Term), i64p, i64p, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_double)]
        lib.orc_do_all.restype = ctypes.c_int
        lib.orc_do_reduce.argtypes = [ctypes.c_int, ctypes.POINTER(_Extent), ctypes.c_int,
                                      ctypes.POINTER(_Grid), ctypes.c_int, ctypes.POINTER(_Grid),
                                      ctypes.c_int, ctypes.POINTER(_Term), i64p, i64p,
                                      ctypes.POINTER(ctypes.c_double)]
        lib.orc_do_reduce.restype = ctypes.c_int
        lib.orc_do_reduce_within.argtypes = [ctypes.c_double] + lib.orc_do_reduce.argtypes[1:]
        lib.orc_do_reduce_within.restype = ctypes.c_int
        lib.orc_do_ordered.argtypes = [ctypes.c_int, ctypes.c_int] + lib.orc_do_reduce.argtypes[1:-1]
        lib.orc_do_ordered.restype = ctypes.c_int
        lib.orc_do_colored.argtypes = [ctypes.c_int] + lib.orc_do_reduce.argtypes[1:-1]
        lib.orc_do_colored.restype = ctypes.c_int
        lib.orc_do_diamond.argtypes = lib.orc_do_reduce.argtypes[1:-1]
        lib.orc_do_diamond.restype = ctypes.c_int
        lib.orc_threads.argtypes = [ctypes.c_int]
        lib.orc_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclass
class Grid:
    """A dense FP64 grid with halo: ``a[k + hz, j + hy, i + hx]`` is element (i, j, k)."""
    a: np.ndarray
    halo: tuple

    @property
    def n(self):
        hx, hy, hz = self.halo
        z, y, x = self.a.shape
        return (x - 2 * hx, y - 2 * hy, z - 2 * hz)

    def interior(self):
        hx, hy, hz = self.halo
        nx, ny, nz = self.n
        return self.a[hz:hz + nz, hy:hy + ny, hx:hx + nx]

    def copy(self):
        return Grid(self.a.copy(), tuple(self.halo))


def zeros(n, halo) -> Grid:
    nx, ny, nz = n
    hx, hy, hz = halo
    return Grid(np.zeros((nz + 2 * hz, ny + 2 * hy, nx + 2 * hx), dtype=np.float64), tuple(halo))


def _marshal(terms, ins, outs, lo, hi, allow_alias=False):
    if not ins:
        raise ValueError("at least one input grid")
    n = ins[0].n
    for g in list(ins) + list(outs):
        if g.n != n:
            raise ValueError("all grids of one call share the interior extent")
        if g.a.dtype != np.float64 or not g.a.flags.c_contiguous:
            raise ValueError("oracle grids are C-contiguous float64")
    in_ids = {id(g.a) for g in ins}
    for g in outs:
        if id(g.a) in in_ids and not allow_alias:
            raise ValueError("the oracle requires output arrays distinct from inputs")
    ext = _Extent(*n)
    gin = (_Grid * len(ins))(*[_Grid(g.a.ctypes.data, *g.halo) for g in ins])
    gout = (_Grid * max(1, len(outs)))(*[_Grid(g.a.ctypes.data, *g.halo) for g in outs])
    tt = (_Term * max(1, len(terms)))(*[_Term(int(t[0]), int(t[1]), int(t[2]), int(t[3]),
                                              int(t[4]), int(t[5]), float(t[6])) for t in terms])
    if lo is None:
        lo = (0, 0, 0)
    if hi is None:
        hi = n
    clo = (ctypes.c_int64 * 3)(*lo)
    chi = (ctypes.c_int64 * 3)(*hi)
    return ext, gin, gout, tt, clo, chi


def do_all(terms, ins, outs, lo=None, hi=None, abs_mode=False, want_value=False):
    """Applies the operator at every core element of ``[lo, hi)`` (Section 3, do_all).

    Writes each output grid's core elements in place; with ``want_value``
    returns the operator's value at every core element as an array of shape
    ``(hi_z - lo_z, hi_y - lo_y, hi_x - lo_x)``.  ``abs_mode`` computes the
    absolute stencil S(p) instead (tolerance scaling for the tests).
    """
    ext, gin, gout, tt, clo, chi = _marshal(terms, ins, outs, lo, hi)
    shape = tuple(int(chi[a] - clo[a]) for a in (2, 1, 0))
    val = np.zeros(shape, dtype=np.float64) if want_value else None
    vptr = val.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if want_value else None
    rc = _get_lib().orc_do_all(ctypes.byref(ext), len(ins), gin, len(outs), gout, len(terms), tt,
                               clo, chi, int(bool(abs_mode)), vptr)
    if rc != 0:
        raise ValueError(f"oracle do_all rejected the call (code {rc})")
    return val


I_INC, I_DEC, J_INC, J_DEC, K_INC, K_DEC = range(6)


def do_ordered(order, terms, ins, outs, lo=None, hi=None):
    """Ordered iteration space (Section 3): ``order`` is one of I_INC .. K_DEC.
    Along the ordered axis each element is visited after its predecessor; an
    output passed also as an input (the same Grid) is read as updated so far."""
    ext, gin, gout, tt, clo, chi = _marshal(terms, ins, outs, lo, hi, allow_alias=True)
    rc = _get_lib().orc_do_ordered(order // 2, 1 if order % 2 == 0 else 0, ctypes.byref(ext), len(ins), gin,
                                   len(outs), gout, len(terms), tt, clo, chi)
    if rc != 0:
        raise ValueError(f"oracle do_ordered rejected the call (code {rc})")


def do_diamond(terms, ins, outs, lo=None, hi=None):
    """do_diamond (Section 3): (i-1, j) and (i, j-1) are processed before
    (i, j), here in lexicographic order, plane by plane; an output passed also
    as an input (the same Grid) is read as updated so far."""
    ext, gin, gout, tt, clo, chi = _marshal(terms, ins, outs, lo, hi, allow_alias=True)
    rc = _get_lib().orc_do_diamond(ctypes.byref(ext), len(ins), gin, len(outs), gout, len(terms), tt, clo, chi)
    if rc != 0:
        raise ValueError(f"oracle do_diamond rejected the call (code {rc})")


def do_colored(color, terms, ins, outs, lo=None, hi=None):
    """Red-black colouring (Section 3, stateful stencils): the operator at the
    core elements of ``[lo, hi)`` whose index sum i + j + k has parity
    ``color``, in lexicographic order; an output passed also as an input (the
    same Grid) is updated in place."""
    ext, gin, gout, tt, clo, chi = _marshal(terms, ins, outs, lo, hi, allow_alias=True)
    rc = _get_lib().orc_do_colored(int(color), ctypes.byref(ext), len(ins), gin, len(outs), gout, len(terms), tt,
                                   clo, chi)
    if rc != 0:
        raise ValueError(f"oracle do_colored rejected the call (code {rc})")


def do_reduce_within(eps, terms, ins, outs=(), lo=None, hi=None) -> float:
    """Section 5.2's convergence test as a reduction: 1.0 if every element of
    ``[lo, hi)`` has |value| <= eps (logical_and; a NaN fails), else 0.0."""
    ext, gin, gout, tt, clo, chi = _marshal(terms, ins, outs, lo, hi)
    res = ctypes.c_double(0.0)
    rc = _get_lib().orc_do_reduce_within(ctypes.c_double(eps), ctypes.byref(ext), len(ins), gin, len(outs), gout,
                                         len(terms), tt, clo, chi, ctypes.byref(res))
    if rc != 0:
        raise ValueError(f"oracle do_reduce_within rejected the call (code {rc})")
    return float(res.value)


def do_reduce(op, terms, ins, outs=(), lo=None, hi=None) -> float:
    """Reduces the operator's per-element value over ``[lo, hi)`` (Section 3, do_reduce).

    ``terms`` empty means the value is ``ins[0]`` itself.  Outputs, if the
    operator has any, are written as in ``do_all`` (a fused operator).
    """
    ext, gin, gout, tt, clo, chi = _marshal(terms, ins, outs, lo, hi)
    res = ctypes.c_double(0.0)
    rc = _get_lib().orc_do_reduce(int(op), ctypes.byref(ext), len(ins), gin, len(outs), gout,
                                  len(terms), tt, clo, chi, ctypes.byref(res))
    if rc != 0:
        raise ValueError(f"oracle do_reduce rejected the call (code {rc})")
    return float(res.value)


# ------------------------------------------------------------------ run-time point operators
_PROG_TEMPLATE = os.path.join(_HERE, "program_template.c")


class Program:
    """A point operator given as C statements (reads ``in<a>(dx, dy, dz)``, the
    index ``i, j, k``; assigns ``out<m>``), compiled with gcc and applied at
    every core element of a range in lexicographic order (Section 3, do_all).
    ``reach`` bounds every read's offset; reads beyond it return 0 and are
    counted in ``outside``."""

    def __init__(self, body, n_in, n_out, reach=(1, 1, 1)):
        import hashlib
        defs = "".join(f"#define in{a}(dx, dy, dz) orc_in(e, &in[{a}], i, j, k, (dx), (dy), (dz), reach, outside)\n"
                       for a in range(n_in))
        decl = "".join(f"        real out{m} = 0;\n" for m in range(n_out))
        stores = "".join(f"        out[{m}].data[orc_at(e, out[{m}].hx, out[{m}].hy, out[{m}].hz, i, j, k)] = out{m};\n"
                         for m in range(n_out))
        with open(_PROG_TEMPLATE) as f:
            src = f.read()
        src = (src.replace("/*@DEFS@*/", defs).replace("/*@DECL@*/", decl).replace("/*@BODY@*/", body)
               .replace("/*@STORES@*/", stores))
        key = hashlib.sha1(src.encode()).hexdigest()[:16]
        os.makedirs(_LIB_DIR, exist_ok=True)
        path = os.path.join(_LIB_DIR, f"prog_{key}.so")
        if not os.path.exists(path):
            c = os.path.join(_LIB_DIR, f"prog_{key}.c")
            with open(c, "w") as f:
                f.write(src)
            tmp = path + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-std=gnu99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                                   "-shared", "-o", tmp, c, "-lm"])
            os.replace(tmp, path)
        self._lib = ctypes.CDLL(path)
        self._lib.orc_program.restype = ctypes.c_int
        self.n_in, self.n_out, self.reach = n_in, n_out, tuple(int(v) for v in reach)
        self.outside = 0

    def run(self, ins, outs, lo=None, hi=None, want_value=False):
        """Applies the body over ``[lo, hi)``; with ``want_value`` returns the
        body's ``value`` at every core element, shape (hz - lz, hy - ly, hx - lx)."""
        if len(ins) != self.n_in or len(outs) != self.n_out:
            raise ValueError("the program was made for another number of grids")
        ext, gin, gout, _, clo, chi = _marshal([], ins, outs, lo, hi, allow_alias=True)
        for a in range(3):
            if clo[a] < 0 or chi[a] > (ext.nx, ext.ny, ext.nz)[a] or clo[a] > chi[a]:
                raise ValueError("range outside the interior")
        for g in ins:
            for a in range(3):
                if clo[a] < chi[a] and self.reach[a] > g.halo[a]:
                    raise ValueError("reach beyond a grid's halo")
        r = (ctypes.c_int32 * 3)(*self.reach)
        n = ctypes.c_int64(0)
        shape = tuple(int(chi[a] - clo[a]) for a in (2, 1, 0))
        val = np.zeros(shape) if want_value else None
        vptr = val.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if want_value else None
        self._lib.orc_program(ctypes.byref(ext), gin, gout, clo, chi, r, ctypes.byref(n), vptr)
        self.outside += n.value
        return val

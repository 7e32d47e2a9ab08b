"""ctypes wrapper of the plain FP64 CPU oracle (``fmm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference legs are the only callers.  The CUDA
library never imports this module and this module never imports it.

The shared library is compiled on first use with the system C compiler
(``build()``), into ``oracle/_build/``.
"""

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
# the same source built on double complex numbers (complex-step derivatives)
_LIB_CS_PATH = os.path.join(_OUT_DIR, "liboracle_cs.so")
_LOCK = threading.Lock()
_LIB = None
_LIB_CS = None

NCELL = 512
NCOMP = 20


def _compile(src, out, defines=()):
    cmd = (["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
            "-ffp-contract=off", "-fno-fast-math"] + [f"-D{d}" for d in defines]
           + ["-o", out, src, "-lm"])
    subprocess.run(cmd, check=True)


def _build_one(path, defines, force):
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
        return path
    tmp = path + f".{os.getpid()}.tmp"
    _compile(_SRC, tmp, defines)
    os.replace(tmp, path)
    return path


def build(force=False):
    """Compile the oracle with gcc (OpenMP over target cells, IEEE FP64), and
    its complex-step build."""
    _build_one(_LIB_CS_PATH, ("ORACLE_COMPLEX_STEP",), force)
    return _build_one(_LIB_PATH, (), force)


def _bind(lib):
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    lib.oracle_upward.argtypes = [P, I64, P, P, P, P]
    lib.oracle_m2l.argtypes = [P, I64, P, P, P, P, P, P, P, I64, ctypes.c_int, ctypes.c_int]
    lib.oracle_sources.argtypes = [P, I64, P, I64, ctypes.c_int, P, P, I64]
    lib.oracle_sources.restype = I64
    lib.oracle_coverage.argtypes = [P, I64, P, P, P]
    lib.oracle_downward.argtypes = [P, I64, P, P, P, P, P, P]
    lib.oracle_forces.argtypes = [P, I64, P, P, P, P, P, P, P]
    lib.oracle_pair_m2l.argtypes = [ctypes.c_double, ctypes.c_int, P, P, P, P, ctypes.c_int, P, P]
    lib.oracle_dtensors.argtypes = [P, P, P, P, P, P]
    return lib


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            _LIB = _bind(ctypes.CDLL(build()))
        return _LIB


def _lib_cs():
    global _LIB_CS
    with _LOCK:
        if _LIB_CS is None:
            build()
            _LIB_CS = _bind(ctypes.CDLL(_LIB_CS_PATH))
        return _LIB_CS


def source_text():
    """The oracle's C source (for tests that compile altered copies)."""
    with open(_SRC) as f:
        return f.read()


@contextlib.contextmanager
def variant(source, out_path):
    """Compile `source` (a copy of the oracle's C source, e.g. with a planted
    mistake) to `out_path` with the oracle's own flags, and route every call
    of this module to it inside the block (the tests' check that each pin
    catches the mistakes it is meant to)."""
    global _LIB
    src_path = out_path + ".c"
    with open(src_path, "w") as f:
        f.write(source)
    _compile(src_path, out_path)
    lib = _bind(ctypes.CDLL(out_path))
    with _LOCK:
        saved = _LIB
        _LIB = lib
    try:
        yield
    finally:
        with _LOCK:
            _LIB = saved


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _cfg(theta, G, box_lo, box_size, order=3):
    return np.array([theta, G, box_lo[0], box_lo[1], box_lo[2], box_size, order],
                    dtype=np.float64)


def n_trees(desc):
    return int(desc[:, 13].max()) + 1


class Tree:
    """A node-descriptor array plus the solve parameters (theta, G, box, and
    the expansion order: 3, or 2)."""

    def __init__(self, desc, theta, G=1.0, box_lo=(0.0, 0.0, 0.0), box_size=1.0, order=3):
        if order not in (2, 3):
            raise ValueError("order must be 2 or 3")
        self.desc = np.ascontiguousarray(desc, dtype=np.int32)
        self.n = len(self.desc)
        self.order = order
        self.cfg = _cfg(theta, G, box_lo, box_size, order)
        self.n_leaf = int((self.desc[:, 5] < 0).sum())
        self.n_trees = n_trees(self.desc)

    @classmethod
    def from_config(cls, c):
        return cls(c["desc"], c["theta"], c["G"], c["box_lo"], c["box_size"], c.get("order", 3))


def upward(tree, rho):
    """Returns (M [n,20,512], com [n,3,512])."""
    rho = _f64(rho)
    M = np.empty((tree.n, NCOMP, NCELL))
    com = np.empty((tree.n, 3, NCELL))
    _lib().oracle_upward(_p(tree.desc), tree.n, _p(tree.cfg), _p(rho), _p(M), _p(com))
    return M, com


def m2l(tree, M, com, targets=None, n_threads=0, compact=False):
    """Returns (L [n,20,512], dL1 [n,3,512], counts[4]).

    With ``targets`` (int64 node*512+cell), only those cells are computed and
    the rest of L / dL1 is zero; with ``compact`` as well, L is
    [n_targets, 20] and dL1 [n_targets, 3].  counts = (mp<-mp, mp<-mono,
    mono<-mono, mono<-mp) evaluated pairs.
    """
    M = _f64(M)
    com = _f64(com)
    counts = np.zeros(4, dtype=np.int64)
    if targets is None:
        tp, nt = None, 0
        compact = False
    else:
        targets = np.ascontiguousarray(targets, dtype=np.int64)
        tp, nt = _p(targets), len(targets)
    if compact:
        L = np.zeros((nt, NCOMP))
        dL1 = np.zeros((nt, 3))
    else:
        L = np.zeros((tree.n, NCOMP, NCELL))
        dL1 = np.zeros((tree.n, 3, NCELL))
    _lib().oracle_m2l(_p(tree.desc), tree.n, _p(tree.cfg), _p(M), _p(com), _p(L),
                      _p(dL1), _p(counts), tp, nt, int(n_threads), int(bool(compact)))
    return L, dL1, counts


def sources(tree, node, cell, max_out=4096):
    """Offsets (k,3) and flags (k,) of the sources evaluated for one cell."""
    off = np.zeros((max_out, 3), dtype=np.int32)
    flg = np.zeros(max_out, dtype=np.int32)
    k = _lib().oracle_sources(_p(tree.desc), tree.n, _p(tree.cfg), int(node), int(cell),
                              _p(off), _p(flg), max_out)
    if k > max_out:
        return sources(tree, node, cell, max_out=int(k))
    return off[:k], flg[:k]


def coverage(tree, w):
    w = _f64(w)
    out = np.zeros_like(w)
    _lib().oracle_coverage(_p(tree.desc), tree.n, _p(tree.cfg), _p(w), _p(out))
    return out


def downward(tree, com, L, dL1):
    """Returns (L64 [n,20,512], dL1acc [n,3,512])."""
    L64 = np.empty((tree.n, NCOMP, NCELL))
    acc = np.empty((tree.n, 3, NCELL))
    _lib().oracle_downward(_p(tree.desc), tree.n, _p(tree.cfg), _p(_f64(com)),
                           _p(_f64(L)), _p(_f64(dL1)), _p(L64), _p(acc))
    return L64, acc


def forces(tree, L64, dL1acc, rho):
    """Returns (phi [n_leaf,512], g [n_leaf,3,512], totals [n_trees,8])."""
    phi = np.empty((tree.n_leaf, NCELL))
    g = np.empty((tree.n_leaf, 3, NCELL))
    tot = np.empty((tree.n_trees, 8))
    _lib().oracle_forces(_p(tree.desc), tree.n, _p(tree.cfg), _p(_f64(L64)),
                         _p(_f64(dL1acc)), _p(_f64(rho)), _p(phi), _p(g), _p(tot))
    return phi, g, tot


def solve(tree, rho, n_threads=0):
    """The whole solve; returns a dict of every stage's output."""
    M, com = upward(tree, rho)
    L, dL1, counts = m2l(tree, M, com, n_threads=n_threads)
    L64, acc = downward(tree, com, L, dL1)
    phi, g, tot = forces(tree, L64, acc, rho)
    return dict(M=M, com=com, L=L, dL1=dL1, counts=counts, L64=L64, dL1acc=acc,
                phi=phi, g=g, totals=tot)


def pair_m2l(MA, XA, MB, XB, a_leaf, G=1.0, order=3):
    """One interaction A <- B at expansion order 3 (or 2): returns (L20, dL1)."""
    L = np.zeros(NCOMP)
    d = np.zeros(3)
    _lib().oracle_pair_m2l(float(G), int(order), _p(_f64(MA)), _p(_f64(XA)), _p(_f64(MB)),
                           _p(_f64(XB)), int(bool(a_leaf)), _p(L), _p(d))
    return L, d


def dtensors(R):
    """Full derivative tensors of 1/|R|: (D0, D1[3], D2[3,3], D3[3,3,3], D4[3]*4).

    Flat index i + 3j + 9k + 27l is returned in numpy order [l, k, j, i]
    reshaped so that D2[i, j] etc. read naturally (tensors are symmetric).
    """
    R = _f64(R)
    D = [np.zeros(1), np.zeros(3), np.zeros(9), np.zeros(27), np.zeros(81)]
    _lib().oracle_dtensors(_p(R), *(_p(x) for x in D))
    return (D[0][0], D[1], D[2].reshape(3, 3), D[3].reshape(3, 3, 3),
            D[4].reshape(3, 3, 3, 3))


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def solve_tangent(tree, rho, rho_dot, h=1e-40):
    """The time derivative of the whole solve along rho(t) = rho + t rho_dot
    at t = 0, by complex-step differentiation: the complex-number build of
    the same oracle solves the density rho + i h rho_dot, and every output's
    imaginary part over h is its exact derivative (no differences are formed,
    so there is no cancellation; the O(h^2) remainder is below double
    precision for any h this small).  Returns dict(phi, g, phi_dot, g_dot,
    totals, totals_dot)."""
    lib = _lib_cs()
    rc = _c128(np.asarray(rho, dtype=np.float64) + 1j * h * np.asarray(rho_dot, dtype=np.float64))
    M = np.empty((tree.n, NCOMP, NCELL), dtype=np.complex128)
    com = np.empty((tree.n, 3, NCELL), dtype=np.complex128)
    lib.oracle_upward(_p(tree.desc), tree.n, _p(tree.cfg), _p(rc), _p(M), _p(com))
    L = np.zeros((tree.n, NCOMP, NCELL), dtype=np.complex128)
    dL1 = np.zeros((tree.n, 3, NCELL), dtype=np.complex128)
    counts = np.zeros(4, dtype=np.int64)
    lib.oracle_m2l(_p(tree.desc), tree.n, _p(tree.cfg), _p(M), _p(com), _p(L), _p(dL1),
                   _p(counts), None, 0, 0, 0)
    L64 = np.empty((tree.n, NCOMP, NCELL), dtype=np.complex128)
    acc = np.empty((tree.n, 3, NCELL), dtype=np.complex128)
    lib.oracle_downward(_p(tree.desc), tree.n, _p(tree.cfg), _p(com), _p(L), _p(dL1), _p(L64),
                        _p(acc))
    phi = np.empty((tree.n_leaf, NCELL), dtype=np.complex128)
    g = np.empty((tree.n_leaf, 3, NCELL), dtype=np.complex128)
    tot = np.empty((tree.n_trees, 8), dtype=np.complex128)
    lib.oracle_forces(_p(tree.desc), tree.n, _p(tree.cfg), _p(L64), _p(acc), _p(rc), _p(phi),
                      _p(g), _p(tot))
    return dict(phi=phi.real.copy(), g=g.real.copy(), phi_dot=phi.imag / h, g_dot=g.imag / h,
                totals=tot.real.copy(), totals_dot=tot.imag / h)

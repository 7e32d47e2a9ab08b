"""ctypes binding of ``libfmm_gb300.so`` (C ABI in ``include/fmm_gb300.h``).

The functions keep the C names and only marshal arguments: torch CUDA tensors
(or raw device addresses as ints) become pointers, the current torch stream
becomes the ``cudaStream_t``.  Every step of the solve runs in the library's
CUDA kernels; nothing here computes, and there is no CPU fallback: if the
library cannot be built or loaded, the first call raises.
"""

import ctypes
import threading

import numpy as np

from . import _build

FMM_OK = 0
FMM_ERR_INVALID_ARG = -1
FMM_ERR_TREE = -2
FMM_ERR_CUDA = -3
FMM_ERR_TIMEOUT = -4
FMM_ERR_NOMEM = -5
FMM_FP64 = 0
FMM_MIXED = 1
FMM_DFLOAT = 2
PRECISIONS = {"fp64": FMM_FP64, "mixed": FMM_MIXED, "dfloat": FMM_DFLOAT}
FMM_STATUS_BAD_DENSITY = 1
FMM_STATUS_TIMEOUT = 2
FMM_FLAG_HOST_ONLY = 1
FMM_FLAG_TIMING = 2
KERNEL_SLOTS = ("p2m", "m2m", "pack", "root", "multipole", "monopole", "mono_multi", "l2l",
                "forces", "reduce")

EXPORTED = ("fmm_build_tree", "fmm_get_sizes", "fmm_get_stats", "fmm_upward",
            "fmm_m2l", "fmm_downward", "fmm_forces", "fmm_step", "fmm_set_tuning", "fmm_get_tuning",
            "fmm_forces_noalloc", "fmm_check_conversions", "fmm_peak_rate", "fmm_scf_update",
            "fmm_field_time_derivative", "fmm_get_status", "fmm_destroy_tree", "fmm_last_error")

NCELL = 512
NCOMP = 20


class FmmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class FmmConfig(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_double), ("G", ctypes.c_double),
                ("box_lo", ctypes.c_double * 3), ("box_size", ctypes.c_double),
                ("precision", ctypes.c_int32), ("max_level", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("order", ctypes.c_int32)]


class FmmSizes(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_leaf", ctypes.c_int64),
                ("n_refined", ctypes.c_int64), ("n_trees", ctypes.c_int64),
                ("max_level", ctypes.c_int32), ("precision", ctypes.c_int32)] + [
        (k, ctypes.c_int64) for k in (
            "rho_bytes", "M_bytes", "com_bytes", "L_bytes", "Lcomp_bytes", "dL1_bytes",
            "L64_bytes", "phi_bytes", "g_bytes", "totals_bytes", "workspace_bytes")]


class FmmStats(ctypes.Structure):
    _fields_ = [("interactions", ctypes.c_int64 * 4), ("stencil_far", ctypes.c_int64),
                ("stencil_near", ctypes.c_int64), ("stencil_union", ctypes.c_int64),
                ("flops_per_interaction", ctypes.c_double * 4),
                ("work_items", ctypes.c_int64 * 4), ("kernel_interactions", ctypes.c_int64 * 4),
                ("reach", ctypes.c_int32),
                ("launches_m2l", ctypes.c_int32), ("launches_step", ctypes.c_int32),
                ("timing", ctypes.c_int32), ("launches_fused", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("kernel_ms", ctypes.c_double * 16),
                ("kernel_launches", ctypes.c_int64 * 16)]


class FmmTuning(ctypes.Structure):
    _fields_ = [("mono_subgrids", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("dataflow", ctypes.c_int32), ("wait_budget_us", ctypes.c_int32),
                ("drop_first_producer", ctypes.c_int32), ("mp_pair_targets", ctypes.c_int32),
                ("mp_items", ctypes.c_int32), ("reserved", ctypes.c_int32)]


TUNING_KEYS = ("mono_subgrids", "ctas_per_sm", "dataflow", "wait_budget_us",
               "drop_first_producer", "mp_pair_targets", "mp_items")


class FmmScfParams(ctypes.Structure):
    _fields_ = [("n", ctypes.c_double), ("rho_max", ctypes.c_double * 2),
                ("point_a", ctypes.c_double * 3), ("point_b", ctypes.c_double * 3),
                ("point_c", ctypes.c_double * 3), ("centre", (ctypes.c_double * 3) * 2),
                ("r_lim", ctypes.c_double * 2), ("x_split", ctypes.c_double),
                ("rho_floor", ctypes.c_double), ("rotate", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class FmmScfResult(ctypes.Structure):
    _fields_ = [("omega2", ctypes.c_double), ("C", ctypes.c_double * 2),
                ("com", ctypes.c_double * 3), ("H_max", ctypes.c_double * 2),
                ("phi_points", ctypes.c_double * 3), ("mass", ctypes.c_double)]


_LOCK = threading.Lock()
_LIB = None


def library_path():
    return _build.LIB


def load(build=True):
    """Build (if stale) and load the CUDA library; raises if impossible."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        path = _build.build() if build else _build.LIB
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        lib.fmm_build_tree.argtypes = [P, ctypes.c_int64, ctypes.POINTER(FmmConfig),
                                       ctypes.POINTER(P)]
        lib.fmm_get_sizes.argtypes = [P, ctypes.POINTER(FmmSizes)]
        lib.fmm_get_stats.argtypes = [P, ctypes.POINTER(FmmStats)]
        lib.fmm_upward.argtypes = [P, P, P, P, P]
        lib.fmm_m2l.argtypes = [P, P, P, P, P, P, P]
        lib.fmm_downward.argtypes = [P, P, P, P, P, P, P, P]
        lib.fmm_forces.argtypes = [P, P, P, P, P, P, P, P]
        lib.fmm_step.argtypes = [P] * 13
        lib.fmm_field_time_derivative.argtypes = [P, P, P, ctypes.c_double] + [P] * 14
        lib.fmm_destroy_tree.argtypes = [P]
        lib.fmm_destroy_tree.restype = None
        lib.fmm_forces_noalloc.argtypes = [P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                           ctypes.c_double, P, P, P, P, P, P, P]
        lib.fmm_check_conversions.argtypes = [P, ctypes.c_int64, P, P]
        lib.fmm_peak_rate.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, P,
                                      ctypes.POINTER(ctypes.c_double), P]
        lib.fmm_scf_update.argtypes = [P, ctypes.POINTER(FmmScfParams), P, P, P,
                                       ctypes.POINTER(FmmScfResult), P]
        lib.fmm_set_tuning.argtypes = [P, ctypes.POINTER(FmmTuning)]
        lib.fmm_get_tuning.argtypes = [P, ctypes.POINTER(FmmTuning)]
        lib.fmm_get_status.argtypes = [P, ctypes.POINTER(ctypes.c_int32), ctypes.c_int]
        lib.fmm_last_error.argtypes = []
        lib.fmm_last_error.restype = ctypes.c_char_p
        for name in EXPORTED:
            if name not in ("fmm_destroy_tree", "fmm_last_error"):
                getattr(lib, name).restype = ctypes.c_int
        _LIB = lib
        return lib


def _check(rc):
    if rc != FMM_OK:
        raise FmmError(rc, load().fmm_last_error().decode())


def _ptr(x):
    """Device pointer of a torch tensor (or an int address / None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if not x.is_contiguous():
        raise ValueError("buffers must be contiguous")
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Tree:
    """Handle of an ``fmm_tree_t`` plus its sizes; closes on ``close()``."""

    def __init__(self, handle, host_only):
        self.handle = handle
        self.host_only = host_only
        self.sizes = fmm_get_sizes(self)
        self.stats = fmm_get_stats(self)

    @property
    def value(self):
        return self.handle.value

    def close(self):
        if self.handle is not None and self.handle.value:
            fmm_destroy_tree(self)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fmm_build_tree(desc, theta, G=1.0, box_lo=(0.0, 0.0, 0.0), box_size=1.0,
                   precision=FMM_FP64, max_level=20, host_only=False, timing=False, order=3):
    lib = load()
    d = np.ascontiguousarray(desc, dtype=np.int32)
    if d.ndim != 2 or d.shape[1] != 14:
        raise ValueError("descriptor array must be (n, 14) int32")
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    flags = (FMM_FLAG_HOST_ONLY if host_only else 0) | (FMM_FLAG_TIMING if timing else 0)
    cfg = FmmConfig(float(theta), float(G), (ctypes.c_double * 3)(*box_lo), float(box_size),
                    int(precision), int(max_level), flags, int(order))
    h = ctypes.c_void_p()
    _check(lib.fmm_build_tree(d.ctypes.data_as(ctypes.c_void_p), len(d), ctypes.byref(cfg),
                              ctypes.byref(h)))
    return Tree(h, host_only)


def fmm_get_sizes(tree):
    s = FmmSizes()
    _check(load().fmm_get_sizes(tree.handle, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in FmmSizes._fields_}


def fmm_get_stats(tree):
    s = FmmStats()
    _check(load().fmm_get_stats(tree.handle, ctypes.byref(s)))
    out = {}
    for k, _ in FmmStats._fields_:
        v = getattr(s, k)
        out[k] = list(v) if hasattr(v, "__len__") else v
    return out


def fmm_upward(tree, rho, M, com, stream=None):
    _check(load().fmm_upward(tree.handle, _ptr(rho), _ptr(M), _ptr(com), _stream(stream)))


def fmm_m2l(tree, M, com, L, L_comp, dL1, stream=None):
    _check(load().fmm_m2l(tree.handle, _ptr(M), _ptr(com), _ptr(L), _ptr(L_comp), _ptr(dL1),
                          _stream(stream)))


def fmm_downward(tree, L, L_comp, dL1, com, L64, dL1_acc, stream=None):
    _check(load().fmm_downward(tree.handle, _ptr(L), _ptr(L_comp), _ptr(dL1), _ptr(com),
                               _ptr(L64), _ptr(dL1_acc), _stream(stream)))


def fmm_forces(tree, L64, dL1_acc, rho, phi, g, totals, stream=None):
    _check(load().fmm_forces(tree.handle, _ptr(L64), _ptr(dL1_acc), _ptr(rho), _ptr(phi),
                             _ptr(g), _ptr(totals), _stream(stream)))


def fmm_step(tree, rho, M, com, L, L_comp, dL1, L64, dL1_acc, phi, g, totals, stream=None):
    """The whole step in one call (upward, same-level, downward, forces), with
    the passes' independent work overlapped on two streams; same results as
    the four calls in sequence."""
    _check(load().fmm_step(tree.handle, _ptr(rho), _ptr(M), _ptr(com), _ptr(L), _ptr(L_comp),
                           _ptr(dL1), _ptr(L64), _ptr(dL1_acc), _ptr(phi), _ptr(g), _ptr(totals),
                           _stream(stream)))


def fmm_field_time_derivative(tree, rho, rho_dot, eps, rho_work, M, com, L, L_comp, dL1, L64,
                              dL1_acc, phi, g, totals, phi_dot, g_dot, stream=None):
    """phi_dot, g_dot: the time derivative of the solve along rho + t rho_dot
    (four solves, fourth-order central differences of step eps; the step's
    buffers are scratch)."""
    _check(load().fmm_field_time_derivative(
        tree.handle, _ptr(rho), _ptr(rho_dot), float(eps), _ptr(rho_work), _ptr(M), _ptr(com),
        _ptr(L), _ptr(L_comp), _ptr(dL1), _ptr(L64), _ptr(dL1_acc), _ptr(phi), _ptr(g),
        _ptr(totals), _ptr(phi_dot), _ptr(g_dot), _stream(stream)))


def fmm_destroy_tree(tree):
    load().fmm_destroy_tree(tree.handle)


def fmm_forces_noalloc(leaf_table, n_leaf, n_nodes, n_trees, box_size, L64, dL1_acc, rho, phi,
                       g, totals, stream=None):
    """The leaf-force pass without a tree handle or any allocation (for callers
    that cannot allocate device memory); ``leaf_table`` is a device int32
    [n_leaf, 6] tensor (node, level, ix, iy, iz, tree_id per leaf node),
    ``n_nodes`` the node count of L64 and dL1_acc."""
    _check(load().fmm_forces_noalloc(_ptr(leaf_table), int(n_leaf), int(n_nodes), int(n_trees),
                                     float(box_size), _ptr(L64), _ptr(dL1_acc), _ptr(rho),
                                     _ptr(phi), _ptr(g), _ptr(totals), _stream(stream)))


def fmm_check_conversions(values, mismatch, stream=None):
    """Diagnostic: the library's integer-pipe float/double conversions against
    the hardware's on the device doubles ``values``; ``mismatch`` (device int32
    [1]) receives 0 when all agree, else a bit mask."""
    _check(load().fmm_check_conversions(_ptr(values), int(values.numel()), _ptr(mismatch),
                                        _stream(stream)))


PEAK_KINDS = {"fp32": 0, "fp32x2": 1, "fp64": 2}


def fmm_peak_rate(kind, iters, blocks_per_sm, sink, stream=None):
    """Diagnostic: enqueue one fused multiply-add loop launch (kind "fp32",
    "fp32x2" or "fp64") and return its operation count; time it with CUDA
    events on the same stream.  ``sink`` is a device float tensor of one
    element."""
    fl = ctypes.c_double(0.0)
    _check(load().fmm_peak_rate(int(PEAK_KINDS.get(kind, kind)), int(iters), int(blocks_per_sm),
                                _ptr(sink), ctypes.byref(fl), _stream(stream)))
    return fl.value


def scf_params(n, rho_max, point_a, point_c, centre, r_lim, x_split, point_b=(0.0, 0.0, 0.0),
               rho_floor=1e-10, rotate=True):
    """An fmm_scf_params structure (see include/fmm_gb300.h)."""
    p = FmmScfParams()
    p.n = float(n)
    p.rho_max[:] = [float(v) for v in rho_max]
    p.point_a[:] = [float(v) for v in point_a]
    p.point_b[:] = [float(v) for v in point_b]
    p.point_c[:] = [float(v) for v in point_c]
    for i in range(2):
        p.centre[i][:] = [float(v) for v in centre[i]]
    p.r_lim[:] = [float(v) for v in r_lim]
    p.x_split = float(x_split)
    p.rho_floor = float(rho_floor)
    p.rotate = 1 if rotate else 0
    return p


def fmm_scf_update(tree, params, phi, rho, rho_out, stream=None):
    """One self-consistent-field iteration's density update after a solve of
    ``tree`` (``phi`` the potential of ``rho``); returns the iteration's
    scalars as a dict."""
    r = FmmScfResult()
    _check(load().fmm_scf_update(tree.handle, ctypes.byref(params), _ptr(phi), _ptr(rho),
                                 _ptr(rho_out), ctypes.byref(r), _stream(stream)))
    return {"omega2": r.omega2, "C": tuple(r.C), "com": tuple(r.com), "H_max": tuple(r.H_max),
            "phi_points": tuple(r.phi_points), "mass": r.mass}


def fmm_set_tuning(tree, mono_subgrids=0, ctas_per_sm=0, dataflow=0, wait_budget_us=0,
                   drop_first_producer=0, mp_pair_targets=0, mp_items=0):
    t = FmmTuning(int(mono_subgrids), int(ctas_per_sm), int(dataflow), int(wait_budget_us),
                  int(drop_first_producer), int(mp_pair_targets), int(mp_items))
    _check(load().fmm_set_tuning(tree.handle, ctypes.byref(t)))


def fmm_get_tuning(tree):
    t = FmmTuning()
    _check(load().fmm_get_tuning(tree.handle, ctypes.byref(t)))
    return {k: getattr(t, k) for k in TUNING_KEYS}


def fmm_get_status(tree, clear=True):
    """The tree's device status word (FMM_STATUS_* bits), read after the
    device is idle; cleared afterwards unless ``clear`` is false."""
    st = ctypes.c_int32(0)
    _check(load().fmm_get_status(tree.handle, ctypes.byref(st), 1 if clear else 0))
    return int(st.value)


def fmm_last_error():
    return load().fmm_last_error().decode()


class Solver:
    """Owns the device buffers of one tree and runs the four passes.

    ``step(rho)`` enqueues upward, same-level, downward and forces on the
    current stream; ``capture(rho)`` records that sequence once into a CUDA
    graph which ``replay()`` relaunches.
    """

    def __init__(self, desc, theta, precision="mixed", G=1.0, box_lo=(0.0, 0.0, 0.0),
                 box_size=1.0, device="cuda", timing=False, order=3):
        import torch
        self.tree = fmm_build_tree(desc, theta, G, box_lo, box_size, precision, timing=timing,
                                   order=order)
        self.order = order
        s = self.tree.sizes
        n, nl, nt = s["n_nodes"], s["n_leaf"], s["n_trees"]
        self.precision = s["precision"]
        self.mixed = self.precision == FMM_MIXED
        # float (hi, lo) Taylor coefficients in the mixed and double-float precisions
        self.pair = self.precision != FMM_FP64
        f64 = dict(dtype=torch.float64, device=device)
        self.M = torch.zeros((n, NCOMP, NCELL), **f64)
        self.com = torch.zeros((n, 3, NCELL), **f64)
        if self.pair:
            self.L = torch.zeros((n, NCOMP, NCELL), dtype=torch.float32, device=device)
            self.Lc = torch.zeros((n, NCOMP, NCELL), dtype=torch.float32, device=device)
        else:
            self.L = torch.zeros((n, NCOMP, NCELL), **f64)
            self.Lc = None
        self.dL1 = torch.zeros((n, 3, NCELL), **f64)
        self.L64 = torch.zeros((n, NCOMP, NCELL), **f64)
        self.dacc = torch.zeros((n, 3, NCELL), **f64)
        self.phi = torch.zeros((nl, NCELL), **f64)
        self.g = torch.zeros((nl, 3, NCELL), **f64)
        self.totals = torch.zeros((nt, 8), **f64)
        self.rho = torch.zeros((nl, NCELL), **f64)
        self.graph = None
        self._stream_state = None          # run_stream: second buffer, graphs, copy stream

    def upward(self, rho=None, stream=None):
        fmm_upward(self.tree, self.rho if rho is None else rho, self.M, self.com, stream)

    def m2l(self, stream=None):
        fmm_m2l(self.tree, self.M, self.com, self.L, self.Lc, self.dL1, stream)

    def downward(self, stream=None):
        fmm_downward(self.tree, self.L, self.Lc, self.dL1, self.com, self.L64, self.dacc, stream)

    def forces(self, rho=None, stream=None):
        fmm_forces(self.tree, self.L64, self.dacc, self.rho if rho is None else rho, self.phi,
                   self.g, self.totals, stream)

    def step(self, rho=None, stream=None):
        """One solve step through fmm_step (the passes overlapped on two streams)."""
        fmm_step(self.tree, self.rho if rho is None else rho, self.M, self.com, self.L, self.Lc,
                 self.dL1, self.L64, self.dacc, self.phi, self.g, self.totals, stream)

    def step_passes(self, rho=None, stream=None):
        """The same step as the four pass calls in sequence on one stream."""
        self.upward(rho, stream)
        self.m2l(stream)
        self.downward(stream)
        self.forces(rho, stream)

    def time_derivative(self, rho_dot, eps, phi_dot, g_dot, rho=None, rho_work=None,
                        stream=None):
        """phi_dot, g_dot (device tensors shaped like phi and g): the time
        derivative of the solve along rho + t rho_dot (fmm_field_time_derivative;
        this solver's step buffers are used as scratch)."""
        import torch
        if rho_work is None:
            rho_work = torch.empty_like(self.rho)
        fmm_field_time_derivative(self.tree, self.rho if rho is None else rho, rho_dot, eps,
                                  rho_work, self.M, self.com, self.L, self.Lc, self.dL1, self.L64,
                                  self.dacc, self.phi, self.g, self.totals, phi_dot, g_dot, stream)

    def status(self, clear=True):
        """FMM_STATUS_* bits recorded by the kernels since the last clear
        (FMM_STATUS_BAD_DENSITY: a leaf density was not positive)."""
        return fmm_get_status(self.tree, clear)

    def kernel_times(self):
        """Per-kernel device ms since the last call (trees built with timing=True)."""
        st = fmm_get_stats(self.tree)
        return {k: (st["kernel_ms"][i], st["kernel_launches"][i])
                for i, k in enumerate(KERNEL_SLOTS)}

    def capture(self, rho=None):
        """Record step() into a CUDA graph (call once, then replay).  rho:
        self.rho by default, or a page-locked host tensor that the step's P2M
        kernel then reads directly every replay (the graph keeps its
        address)."""
        import torch
        self.step(rho)                    # warm-up outside capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.step(rho)
        torch.cuda.current_stream().wait_stream(s)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def run_stream(self, inputs, on_result=None, before_step=None):
        """Solve one step per page-locked host density in ``inputs`` (each
        shaped and typed like ``self.rho``), back to back on the current
        stream.  Step k + 1's density is copied to the device on a copy
        stream while step k computes: two device density buffers, one
        captured graph each.  Every step's totals are copied back to
        page-locked host memory.  ``on_result(k, totals)`` runs on the host
        for step k once step k + 1 has been enqueued, and for the last step
        at the end.  ``before_step()``, if given, is called on the host
        before each step is enqueued (work it enqueues on the current stream
        runs before the step).  Returns the number of steps; afterwards
        ``self.graph`` reads ``self.rho`` again."""
        import torch
        inputs = list(inputs)
        for x in inputs:
            if (x.device.type != "cpu" or not x.is_pinned() or x.dtype != self.rho.dtype
                    or tuple(x.shape) != tuple(self.rho.shape)):
                raise ValueError("run_stream inputs must be page-locked host tensors shaped "
                                 "and typed like Solver.rho")
        n = len(inputs)
        if n == 0:
            return 0
        if self._stream_state is None:
            rho_b = self.rho.clone()            # the warm-up step sees a valid density
            g_b = self.capture(rho_b)
            g_a = self.capture()
            tot = [torch.empty(tuple(self.totals.shape), dtype=self.totals.dtype).pin_memory()
                   for _ in range(2)]
            self._stream_state = ((self.rho, rho_b), (g_a, g_b), torch.cuda.Stream(), tot)
        bufs, graphs, cs, tot = self._stream_state
        main = torch.cuda.current_stream()
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        done = [torch.cuda.Event(), torch.cuda.Event()]
        cs.wait_stream(main)               # earlier work on the buffers is done first

        def copy_in(k):
            b = k % 2
            with torch.cuda.stream(cs):
                if k >= 2:
                    cs.wait_event(done[b])     # step k - 2 has read this buffer
                bufs[b].copy_(inputs[k], non_blocking=True)
                copied[b].record(cs)

        copy_in(0)
        for k in range(n):
            if k + 1 < n:
                copy_in(k + 1)
            b = k % 2
            main.wait_event(copied[b])
            if before_step is not None:
                before_step()
            graphs[b].replay()
            tot[b].copy_(self.totals, non_blocking=True)
            done[b].record(main)
            if k >= 1:
                done[(k - 1) % 2].synchronize()
                if on_result is not None:
                    on_result(k - 1, tot[(k - 1) % 2])
        done[(n - 1) % 2].synchronize()
        if on_result is not None:
            on_result(n - 1, tot[(n - 1) % 2])
        main.wait_stream(cs)
        self.graph = graphs[0]
        return n

    def close(self):
        self.graph = None
        self._stream_state = None
        if self.tree is not None:
            self.tree.close()
            self.tree = None

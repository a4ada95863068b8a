"""GB300 builder and applier of the discrete Dirichlet-to-Neumann map of
-Lap u + b u_x + c u_y + d u = 0 on the unit square (Gillman & Martinsson's nested
dissection build, arXiv 1302.5995).

This module is argument marshalling over the C ABI declared in include/gm.h: every
step of the build and of the solve runs in the CUDA kernels of libgm.so.  Importing it
fails loudly when that library has not been built; there is no CPU fallback.

    import paper_1302_5995_gb300 as gm
    op = gm.build(b, c, d, n=512, leaf=16)          # torch CUDA tensors or numpy arrays
    v = op.solve(g)                                 # g: 4n x B, column j = vector j
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgm.so")

GM_OK, GM_EINVAL, GM_ENOMEM, GM_ESINGULAR, GM_ETIMEOUT, GM_ECUDA, GM_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
GM_ESCRATCH = -7
PREC_FP64, PREC_MIXED = 0, 1
PIVOT_AUTO, PIVOT_BLOCK, PIVOT_PARTIAL = 0, 1, 2


class GmError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("keep_levels", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("panel_width", ctypes.c_int), ("timing", ctypes.c_int), ("split_digits", ctypes.c_int),
                ("pivoting", ctypes.c_int), ("hbs_leaf", ctypes.c_int), ("hbs_min_edge", ctypes.c_int),
                ("timing_mask", ctypes.c_int), ("background", ctypes.c_int), ("wait_limit", ctypes.c_int),
                ("graph", ctypes.c_int), ("autotune", ctypes.c_int)]

K_FAMILIES = ["leaf", "assemble", "panel", "pivrows", "gj_update", "merge_update", "root"]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("leaf", ctypes.c_int), ("levels", ctypes.c_int),
                ("precision", ctypes.c_int), ("dtn_bytes", ctypes.c_longlong),
                ("peak_workspace", ctypes.c_longlong), ("min_pivot_ratio", ctypes.c_double),
                ("bad_stage", ctypes.c_int), ("launches", ctypes.c_int),
                ("kernel_ms", ctypes.c_double * 7), ("kernel_flops", ctypes.c_double * 7),
                ("kernel_launches", ctypes.c_int * 7), ("pivoting", ctypes.c_int),
                ("pivot_fallback", ctypes.c_int), ("refine_ratio", ctypes.c_double), ("hbs_levels", ctypes.c_int),
                ("hbs_max_rank", ctypes.c_int), ("hbs_bytes", ctypes.c_longlong), ("resident_bytes", ctypes.c_longlong),
                ("hbs_merges", ctypes.c_int), ("hbs_update_rank", ctypes.c_int), ("hbs_operator_bytes", ctypes.c_longlong),
                ("load_rank", ctypes.c_int), ("hbs_fallbacks", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_longlong), ("vectors", ctypes.c_longlong), ("solves", ctypes.c_longlong),
                ("evictions", ctypes.c_longlong), ("resident_ops", ctypes.c_int), ("pad", ctypes.c_int),
                ("resident_bytes", ctypes.c_longlong), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("vectors_per_s", ctypes.c_double)]


class Problem(ctypes.Structure):
    _fields_ = [("b", ctypes.c_void_p), ("c", ctypes.c_void_p), ("d", ctypes.c_void_p), ("n", ctypes.c_int),
                ("leaf", ctypes.c_int)]


#: exported symbols and their (restype, argtypes)
SIGNATURES = {
    "gm_opts_default": (None, [ctypes.POINTER(Opts)]),
    "gm_build": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                      ctypes.POINTER(ctypes.c_void_p)]),
    "gm_build_ex": (ctypes.c_int, [ctypes.POINTER(Opts)] + [ctypes.c_void_p] * 3
                    + [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_void_p)]),
    "gm_build_batch": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(Problem), ctypes.POINTER(Opts), ctypes.c_double,
                                      ctypes.POINTER(ctypes.c_void_p)]),
    "gm_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "gm_solve_many": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                     ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]),
    "gm_get_dtn": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "gm_get_schur": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int] * 4 + [ctypes.c_void_p]),
    "gm_solve_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.c_void_p]),
    "gm_build_loads": (ctypes.c_int, [ctypes.POINTER(Opts)] + [ctypes.c_void_p] * 3
                       + [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "gm_solve_loads": (ctypes.c_int, [ctypes.c_void_p] * 4 + [ctypes.c_int, ctypes.c_void_p]),
    "gm_get_load_operator": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "gm_compress_load_operator": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "gm_build_net": (ctypes.c_int, [ctypes.POINTER(Opts)] + [ctypes.c_void_p] * 2
                     + [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_int,
                        ctypes.POINTER(ctypes.c_void_p)]),
    "gm_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Info)]),
    "gm_free": (None, [ctypes.c_void_p]),
    "gm_server_create": (ctypes.c_int, [ctypes.c_longlong, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "gm_server_add": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "gm_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_longlong)]),
    "gm_server_submit_build": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Opts)] + [ctypes.c_void_p] * 3
                               + [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(ctypes.c_longlong)]),
    "gm_server_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int)]),
    "gm_server_set_callback": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "gm_server_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong]),
    "gm_server_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "gm_server_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ServerStats)]),
    "gm_server_reset_stats": (ctypes.c_int, [ctypes.c_void_p]),
    "gm_server_destroy": (None, [ctypes.c_void_p]),
    "gm_debug_fail_alloc": (None, [ctypes.c_longlong]),
    "gm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libgm.so and declare its signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build the CUDA extension first "
                          "(python -m paper_1302_5995_gb300.build_ext)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load_library().gm_strerror(code).decode()


def _ptr(x):
    """Raw address of a torch tensor or numpy array (contiguous, float64)."""
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(x.ctypes.data)


def _check_f64(x, what, numel=None):
    import numpy as np
    if hasattr(x, "data_ptr"):
        import torch
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise TypeError(f"{what}: need a contiguous float64 tensor")
        if numel is not None and x.numel() != numel:
            raise ValueError(f"{what}: expected {numel} elements, got {x.numel()}")
        return x
    x = np.ascontiguousarray(x, dtype=np.float64)
    if numel is not None and x.size != numel:
        raise ValueError(f"{what}: expected {numel} elements, got {x.size}")
    return x


def _batch(x, N, what):
    """Vectors in x (N values each); its size must be a whole number of vectors."""
    size = x.numel() if hasattr(x, "numel") else x.size
    if size % N:
        raise ValueError(f"{what}: {size} values is not a whole number of {N}-value vectors")
    return size // N


def _out_like(g, out, numel):
    """The result buffer: a new one like g, or the caller's, checked to hold numel float64
    values contiguously (the library writes all of them)."""
    if out is None:
        if hasattr(g, "data_ptr"):
            import torch
            return torch.empty_like(g)
        import numpy as np
        return np.empty_like(g)
    if hasattr(out, "data_ptr"):
        import torch
        if out.dtype != torch.float64 or not out.is_contiguous() or out.numel() != numel:
            raise ValueError(f"out: need a contiguous float64 tensor of {numel} values")
        return out
    import numpy as np
    if not isinstance(out, np.ndarray) or out.dtype != np.float64 or not out.flags.c_contiguous or out.size != numel:
        raise ValueError(f"out: need a C-contiguous float64 array of {numel} values")
    return out


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class DtN:
    """A built Dirichlet-to-Neumann operator (owns its device memory)."""

    def __init__(self, handle, n, leaf):
        self._h = handle
        self.n = n
        self.leaf = leaf
        self.nbody = 0  # body loads of a build_loads handle
        self._keep = []

    def __del__(self):
        try:
            if self._h:
                load_library().gm_free(self._h)
                self._h = None
        except Exception:
            pass

    def free(self):
        self.__del__()

    def solve(self, g, out=None, stream=None):
        """dudn = T g for g of shape (4n, B) stored column by column (vector j contiguous).

        g/out may be torch CUDA tensors (asynchronous on `stream`) or host arrays."""
        lib = load_library()
        N = 4 * self.n
        g = _check_f64(g, "g")
        B = _batch(g, N, "g")
        out = _out_like(g, out, N * B)
        rc = lib.gm_solve(self._h, _ptr(g), _ptr(out), B, _stream_handle(stream))
        if rc:
            raise GmError(rc, "gm_solve")
        return out

    def dtn(self, out=None):
        """The dense 4n x 4n DtN matrix T.  With `out` (a 4n*4n float64 buffer, host or
        device) the column-major matrix is written there and `out` is returned."""
        import numpy as np
        N = 4 * self.n
        if out is not None:
            out = _out_like(None, out, N * N)
            rc = load_library().gm_get_dtn(self._h, _ptr(out))
            if rc:
                raise GmError(rc, "gm_get_dtn")
            return out
        buf = np.empty((N, N))
        rc = load_library().gm_get_dtn(self._h, _ptr(buf))
        if rc:
            raise GmError(rc, "gm_get_dtn")
        return buf.T.copy()

    def schur(self, x0, y0, a, b):
        """Schur complement of a kept box over its counter-clockwise ring (row-major view
        of the column-major matrix is its transpose; returned as the matrix itself)."""
        import numpy as np
        r = 2 * a + 2 * b - 4
        out = np.empty((r, r))
        rc = load_library().gm_get_schur(self._h, x0, y0, a, b, _ptr(out))
        if rc:
            raise GmError(rc, "gm_get_schur")
        return out.T.copy()

    def solve_loads(self, g, f, out=None, stream=None):
        """dudn = T g + F f (Section 6.3) for g of shape (4n, B) and loads f of shape
        (nbody, B), both stored column by column; needs a handle from build_loads."""
        lib = load_library()
        N = 4 * self.n
        g = _check_f64(g, "g")
        B = _batch(g, N, "g")
        f = _check_f64(f, "f", self.nbody * B)
        out = _out_like(g, out, N * B)
        rc = lib.gm_solve_loads(self._h, _ptr(g), _ptr(f), _ptr(out), B, _stream_handle(stream))
        if rc:
            raise GmError(rc, "gm_solve_loads")
        return out

    def compress_loads(self, tol):
        """Replace the load operator F by its low-rank form L R at relative tolerance tol
        (Section 6.3); returns the rank."""
        rc = load_library().gm_compress_load_operator(self._h, float(tol))
        if rc:
            raise GmError(rc, "gm_compress_load_operator")
        return self.info()["load_rank"]

    def load_operator(self):
        """The 4n x nbody load operator F of a build_loads handle (column c: body[c])."""
        import numpy as np
        F = np.empty((max(self.nbody, 1), 4 * self.n))
        rc = load_library().gm_get_load_operator(self._h, _ptr(F))
        if rc:
            raise GmError(rc, "gm_get_load_operator")
        return F[: self.nbody].T.copy()

    def info(self):
        inf = Info()
        rc = load_library().gm_info(self._h, ctypes.byref(inf))
        if rc:
            raise GmError(rc, "gm_info")
        out = {f: getattr(inf, f) for f, _ in Info._fields_}
        for f in ("kernel_ms", "kernel_flops", "kernel_launches"):
            out[f] = dict(zip(K_FAMILIES, list(out[f])))
        return out


def solve_many(ops, gs, outs, stream=None):
    """dudn_i = T_i g_i for several operators in one call (gm_solve_many): g_i and out_i
    are device tensors of shape (batch_i, 4 n_i), vector j contiguous.  Dense operators of
    one precision share one apply launch."""
    k = len(ops)
    if not (len(gs) == k == len(outs)):
        raise ValueError("ops, gs and outs differ in length")
    hs = (ctypes.c_void_p * k)()
    gp = (ctypes.c_void_p * k)()
    vp = (ctypes.c_void_p * k)()
    bt = (ctypes.c_int * k)()
    for i, (op, g, o) in enumerate(zip(ops, gs, outs)):
        if not (hasattr(g, "is_cuda") and g.is_cuda and hasattr(o, "is_cuda") and o.is_cuda):
            raise ValueError("solve_many takes device tensors")
        B = _batch(g, 4 * op.n, "g")
        _check_f64(o, "out", 4 * op.n * B)
        hs[i], gp[i], vp[i], bt[i] = op._h, _ptr(g), _ptr(o), B
    rc = load_library().gm_solve_many(k, hs, gp, vp, bt, _stream_handle(stream))
    if rc:
        raise GmError(rc, "gm_solve_many")
    return outs


def _opts(precision, keep_levels, stream, panel_width, timing, split_digits, pivoting, hbs_leaf=0, hbs_min_edge=0,
          wait_limit=0, graph=False, autotune=False):
    """timing: False, True (every family) or a list of family names to time."""
    lib = load_library()
    o = Opts()
    lib.gm_opts_default(ctypes.byref(o))
    o.precision = precision
    o.keep_levels = 1 if keep_levels else 0
    o.stream = _stream_handle(stream)
    o.panel_width = panel_width
    o.timing = 1 if timing else 0
    if timing and not isinstance(timing, bool):
        o.timing_mask = sum(1 << K_FAMILIES.index(f) for f in timing)
    o.split_digits = split_digits
    o.pivoting = pivoting
    o.hbs_leaf = hbs_leaf
    o.hbs_min_edge = hbs_min_edge
    o.wait_limit = wait_limit
    o.graph = 1 if graph else 0
    o.autotune = 1 if autotune else 0
    return o


def build_batch(problems, tol=0.0, precision=PREC_FP64, stream=None, panel_width=0, timing=False, split_digits=0,
                pivoting=PIVOT_AUTO, graph=False, autotune=False):
    """Build several operators in one level-by-level sweep.

    problems: list of (b, c, d, n, leaf).  Returns a list of DtN handles."""
    lib = load_library()
    arr = (Problem * len(problems))()
    keep = []
    for i, (b, c, d, n, leaf) in enumerate(problems):
        b, c, d = (_check_f64(x, "coefficients", n * n) for x in (b, c, d))
        keep += [b, c, d]
        arr[i] = Problem(_ptr(b).value, _ptr(c).value, _ptr(d).value, n, leaf)
    o = _opts(precision, False, stream, panel_width, timing, split_digits, pivoting, graph=graph, autotune=autotune)
    outs = (ctypes.c_void_p * len(problems))()
    rc = lib.gm_build_batch(len(problems), arr, ctypes.byref(o), float(tol), outs)
    if rc:
        raise GmError(rc, "gm_build_batch")
    return [DtN(ctypes.c_void_p(outs[i]), problems[i][3], problems[i][4]) for i in range(len(problems))]


def build(b, c, d, n, leaf, tol=0.0, precision=PREC_FP64, keep_levels=False, stream=None, panel_width=0,
          timing=False, split_digits=0, pivoting=PIVOT_AUTO, hbs_leaf=0, hbs_min_edge=0, wait_limit=0, graph=False,
          autotune=False):
    """Build the DtN operator for coefficient fields b, c, d (n*n each, index i + n*j).

    tol > 0 compresses the root Schur complement to HBS form (node size hbs_leaf) and
    solves through Algorithm 2; tol = 0 is the all-dense build."""
    lib = load_library()
    b = _check_f64(b, "b", n * n)
    c = _check_f64(c, "c", n * n)
    d = _check_f64(d, "d", n * n)
    o = _opts(precision, keep_levels, stream, panel_width, timing, split_digits, pivoting, hbs_leaf, hbs_min_edge,
              wait_limit, graph, autotune)
    h = ctypes.c_void_p()
    rc = lib.gm_build_ex(ctypes.byref(o), _ptr(b), _ptr(c), _ptr(d), n, leaf, float(tol), ctypes.byref(h))
    if rc:
        raise GmError(rc, "gm_build")
    return DtN(h, n, leaf)


def build_loads(b, c, d, n, leaf, body, stream=None, panel_width=0):
    """FP64 build of T and of the load operator F for body loads at the flat node indices
    `body` (Section 6.3: dudn = T g + F f).  Returns a DtN handle with nbody set."""
    import numpy as np
    lib = load_library()
    b = _check_f64(b, "b", n * n)
    c = _check_f64(c, "c", n * n)
    d = _check_f64(d, "d", n * n)
    nodes = np.ascontiguousarray(np.asarray(body, dtype=np.int32).reshape(-1))
    o = _opts(PREC_FP64, False, stream, panel_width, False, 0, PIVOT_AUTO)
    h = ctypes.c_void_p()
    rc = lib.gm_build_loads(ctypes.byref(o), _ptr(b), _ptr(c), _ptr(d), n, leaf, ctypes.c_void_p(nodes.ctypes.data),
                            int(nodes.size), ctypes.byref(h))
    if rc:
        raise GmError(rc, "gm_build_loads")
    op = DtN(h, n, leaf)
    op.nbody = int(nodes.size)
    return op


def build_network(sx, sy, n, leaf, body=None, tol=0.0, hbs_leaf=0, keep_levels=False, stream=None, panel_width=0):
    """FP64 build for a conductance network (Section 6.1 Random Laplacian): sx, sy the
    n (n + 1) link conductivities in the layout of inputs.network_conductivities, with
    optional body loads at the flat node indices `body` (Section 6.3), or the root in HBS
    form at tolerance tol > 0 (node size hbs_leaf)."""
    import numpy as np
    lib = load_library()
    sx = _check_f64(sx, "sx", n * (n + 1))
    sy = _check_f64(sy, "sy", n * (n + 1))
    nodes = np.ascontiguousarray(np.asarray([] if body is None else body, dtype=np.int32).reshape(-1))
    o = _opts(PREC_FP64, keep_levels, stream, panel_width, False, 0, PIVOT_AUTO, hbs_leaf)
    h = ctypes.c_void_p()
    rc = lib.gm_build_net(ctypes.byref(o), _ptr(sx), _ptr(sy), n, leaf, float(tol),
                          ctypes.c_void_p(nodes.ctypes.data) if nodes.size else None, int(nodes.size), ctypes.byref(h))
    if rc:
        raise GmError(rc, "gm_build_net")
    op = DtN(h, n, leaf)
    op.nbody = int(nodes.size)
    return op


SERVER_CALLBACK = ctypes.CFUNCTYPE(None, ctypes.c_longlong, ctypes.c_int, ctypes.c_void_p)


class Server:
    """Serving runtime over resident operators (continuous batching on a worker thread).

    add(op) transfers ownership of a DtN handle to the server; submit() queues a solve and
    returns a request id; wait(id) blocks until it is done.  Buffers passed to submit()
    must stay alive until the request completes (the server keeps references here)."""

    def __init__(self, budget_bytes, batching=True):
        lib = load_library()
        h = ctypes.c_void_p()
        rc = lib.gm_server_create(int(budget_bytes), 1 if batching else 0, ctypes.byref(h))
        if rc:
            raise GmError(rc, "gm_server_create")
        self._s = h
        self._keep = {}
        self._n = {}  # operator id -> grid size, to check request buffers
        self._cb = None

    def add(self, op):
        oid = ctypes.c_int()
        rc = load_library().gm_server_add(self._s, op._h, ctypes.byref(oid))
        if rc:
            raise GmError(rc, "gm_server_add")
        op._h = None  # owned by the server now
        self._n[oid.value] = op.n
        return oid.value

    def submit(self, op_id, g, out, batch):
        n = self._n.get(op_id)
        if n is not None:  # the first 4n * batch values of g and out are read and written
            for x, what in ((g, "g"), (out, "out")):
                size = x.numel() if hasattr(x, "numel") else x.size
                if int(batch) < 0 or size < 4 * n * int(batch):
                    raise ValueError(f"{what}: fewer than 4n * batch = {4 * n * int(batch)} values")
        rid = ctypes.c_longlong()
        rc = load_library().gm_server_submit(self._s, op_id, _ptr(g), _ptr(out), int(batch), ctypes.byref(rid))
        if rc:
            raise GmError(rc, "gm_server_submit")
        self._keep[rid.value] = (g, out)
        return rid.value

    def submit_build(self, b, c, d, n, leaf, tol=0.0, precision=PREC_FP64, split_digits=0, pivoting=PIVOT_AUTO):
        """Queue a build on the server's worker; returns (operator id, request id).  The
        operator id takes solves at once (they run after the build)."""
        b, c, d = (_check_f64(x, "coefficients", n * n) for x in (b, c, d))
        o = _opts(precision, False, None, 0, False, split_digits, pivoting)
        oid, rid = ctypes.c_int(), ctypes.c_longlong()
        rc = load_library().gm_server_submit_build(self._s, ctypes.byref(o), _ptr(b), _ptr(c), _ptr(d), n, leaf,
                                                   float(tol), ctypes.byref(oid), ctypes.byref(rid))
        if rc:
            raise GmError(rc, "gm_server_submit_build")
        self._keep[rid.value] = (b, c, d)
        self._n[oid.value] = n
        return oid.value, rid.value

    def set_callback(self, fn):
        """fn(request id, result code) on the worker thread for every completed request
        (None: no callback)."""
        if fn is None:
            cb = None
        else:
            cb = SERVER_CALLBACK(lambda rid, rc, user: fn(rid, rc))
        self._cb = cb  # the C function pointer must outlive its use
        rc = load_library().gm_server_set_callback(self._s, ctypes.cast(cb, ctypes.c_void_p) if cb else None, None)
        if rc:
            raise GmError(rc, "gm_server_set_callback")

    def poll(self, rid):
        """(done, result code) without blocking."""
        done = ctypes.c_int()
        rc = load_library().gm_server_poll(self._s, rid, ctypes.byref(done))
        if done.value:
            self._keep.pop(rid, None)
        return bool(done.value), rc

    def wait(self, rid):
        rc = load_library().gm_server_wait(self._s, rid)
        self._keep.pop(rid, None)
        return rc

    def sync(self):
        load_library().gm_server_sync(self._s)
        self._keep.clear()

    def stats(self):
        st = ServerStats()
        rc = load_library().gm_server_stats(self._s, ctypes.byref(st))
        if rc:
            raise GmError(rc, "gm_server_stats")
        return {f: getattr(st, f) for f, _ in ServerStats._fields_ if f != "pad"}

    def reset_stats(self):
        load_library().gm_server_reset_stats(self._s)

    def close(self):
        if self._s:
            load_library().gm_server_destroy(self._s)
            self._s = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

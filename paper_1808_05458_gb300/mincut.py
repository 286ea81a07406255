"""Thin ctypes binding of libmincut (include/mc.h).

Argument marshalling only: every step of the solve runs in the CUDA library.
If ``libmincut.so`` has not been built the import of this module fails
loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

MC_OK = 0
MC_EINVAL = -1
MC_ENOMEM = -2
MC_ECUDA = -3
MC_ETIMEOUT = -4
MC_EOVERFLOW = -5
MC_EINTERNAL = -6

MC_DEVICE_PTRS = 1
MC_TRUST_INPUT = 2

MC_PQ_LIFO = 0
MC_PQ_FIFO = 1
MC_BOUND_DEGREE = 0
MC_BOUND_LP = 1
MC_BOUND_LEARNED = 2
MC_BOUND_BEST = 3
PROPOSER_PARAMS = 25409


class McOptions(ctypes.Structure):
    _fields_ = [("pq_order", ctypes.c_int32), ("bound", ctypes.c_int32),
                ("pr_level", ctypes.c_int32), ("scans_per_round", ctypes.c_int32),
                ("region_budget", ctypes.c_int32), ("lp_iters", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("cuda_stream", ctypes.c_void_p),
                ("proposer", ctypes.c_void_p), ("tail_vertices", ctypes.c_int32),
                ("approx_milli", ctypes.c_int32), ("visits", ctypes.c_int32)]


class McStats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int32), ("fallback_rounds", ctypes.c_int32),
                ("bound_initial", ctypes.c_int64), ("n_input", ctypes.c_int64),
                ("m_input", ctypes.c_int64), ("ms_total", ctypes.c_double),
                ("ms_bound", ctypes.c_double), ("ms_pr", ctypes.c_double),
                ("ms_capforest", ctypes.c_double), ("ms_contract", ctypes.c_double),
                ("bytes_alg", ctypes.c_int64), ("scanned_arcs", ctypes.c_int64),
                ("scanned_verts", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("scan_launches", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("ms_scan_kernel", ctypes.c_double), ("ms_tail", ctypes.c_double),
                ("tail_launches", ctypes.c_int32), ("pad2_", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MinCutError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} (code {code})")


_lib = None
EXPORTS = ("mc_options_default", "mc_graph_create", "mc_graph_destroy", "mc_graph_size",
           "mc_min_cut", "mc_batch_min_cut", "mc_strerror", "mc_graph_export",
           "mc_step_degrees", "mc_step_contract", "mc_step_pr", "mc_step_capforest",
           "mc_step_capforest_full", "mc_step_label_prop", "mc_capforest_full_noalloc",
           "mc_batch_autotune", "mc_proposer_create", "mc_proposer_destroy", "mc_proposer_get",
           "mc_proposer_set", "mc_proposer_forward", "mc_proposer_grad", "mc_proposer_train_step",
           "mc_proposer_bound", "mc_test_fail_alloc_after", "mc_graph_coarsen",
           "mc_step_capforest_range", "mc_batch_shape_count", "mc_batch_set_shape")


def library_path() -> str:
    return _build.LIB


def load_library():
    """Load libmincut.so (built by ``build.build_library``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libmincut.so is not built ({path}); run "
                          "paper_1808_05458_gb300.build.build_library()")
    lib = ctypes.CDLL(path)
    vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    P = ctypes.POINTER
    lib.mc_options_default.argtypes = [P(McOptions)]
    lib.mc_graph_create.argtypes = [i32, vp, vp, vp, i32, P(vp)]
    lib.mc_graph_destroy.argtypes = [vp]
    lib.mc_graph_size.argtypes = [vp, P(i64), P(i64)]
    lib.mc_min_cut.argtypes = [vp, P(McOptions), P(i64), vp, P(McStats)]
    lib.mc_batch_min_cut.argtypes = [i32, vp, vp, vp, vp, vp, P(McOptions), vp, vp, vp, P(McStats)]
    lib.mc_test_fail_alloc_after.argtypes = [i64]
    lib.mc_batch_shape_count.argtypes = []
    lib.mc_batch_set_shape.argtypes = [i32]
    lib.mc_strerror.argtypes = [ctypes.c_int]
    lib.mc_strerror.restype = ctypes.c_char_p
    lib.mc_graph_export.argtypes = [vp, vp, vp, vp]
    lib.mc_step_degrees.argtypes = [vp, vp]
    lib.mc_step_contract.argtypes = [vp, vp, i32, i64, vp, vp, vp, P(i64)]
    lib.mc_step_pr.argtypes = [vp, i64, i32, vp]
    lib.mc_step_capforest.argtypes = [vp, i64, P(McOptions), vp, P(i64), P(i64)]
    lib.mc_step_capforest_full.argtypes = [vp, i64, i32, vp, P(i64), P(i64)]
    lib.mc_step_label_prop.argtypes = [vp, i32, u64, vp]
    F32P = P(ctypes.c_float)
    lib.mc_proposer_create.argtypes = [vp, u64, P(vp)]
    lib.mc_proposer_destroy.argtypes = [vp]
    lib.mc_proposer_get.argtypes = [vp, vp]
    lib.mc_proposer_set.argtypes = [vp, vp]
    lib.mc_proposer_forward.argtypes = [vp, vp, vp]
    lib.mc_proposer_grad.argtypes = [vp, vp, vp, P(ctypes.c_double), vp]
    lib.mc_proposer_train_step.argtypes = [vp, vp, vp, ctypes.c_float, P(ctypes.c_double)]
    lib.mc_proposer_bound.argtypes = [vp, vp, P(i64), vp]
    del F32P
    lib.mc_graph_coarsen.argtypes = [vp, i32, u64, P(vp), vp]
    lib.mc_step_capforest_range.argtypes = [vp, i64, P(McOptions), i32, i32, vp, P(i64), P(i64), vp]
    lib.mc_batch_autotune.argtypes = [i32, vp, vp, vp, vp, vp, P(McOptions), P(i32), vp, i32]
    lib.mc_capforest_full_noalloc.argtypes = [i32, i64, vp, vp, i64, i32, vp, P(i64), P(i64), vp]
    for f in EXPORTS:
        if f != "mc_strerror":
            getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load_library().mc_strerror(code).decode()


def _check(rc, where):
    if rc != MC_OK:
        raise MinCutError(rc, where)


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def options(**kw) -> McOptions:
    """Default options with overrides (pq_order, bound, pr_level,
    scans_per_round, region_budget, lp_iters, seed, cuda_stream, proposer,
    tail_vertices, approx_milli, visits)."""
    o = McOptions()
    load_library().mc_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def test_fail_alloc_after(k: int):
    """Fault-injection hook: the device allocation after the next k fails
    with MC_ENOMEM (k < 0: off)."""
    load_library().mc_test_fail_alloc_after(k)


def bitmap_to_side(bits: np.ndarray, n: int) -> np.ndarray:
    """uint32 bitmap (bit v of word v/32) -> uint8 side per vertex."""
    b = np.asarray(bits, dtype=np.uint32).view(np.uint8)
    return np.unpackbits(b, bitorder="little")[:n].astype(np.uint8)


@dataclass
class MinCut:
    lam: int
    bitmap: object          # np.uint32 words (host) or torch tensor (device graphs)
    stats: dict

    def side(self, n: int) -> np.ndarray:
        bits = self.bitmap
        if hasattr(bits, "cpu"):
            bits = bits.cpu().numpy().view(np.uint32)
        return bitmap_to_side(bits, n)


class Graph:
    """A graph resident on the current CUDA device (``mc_graph``).

    ``row_ptr``, ``col``, ``w``: int32 symmetric CSR, either numpy arrays
    (host) or int32 CUDA torch tensors (device, copied on the graph's stream).
    ``w=None``: an unweighted graph (every arc has weight 1; no weight array
    is copied).
    """

    def __init__(self, row_ptr, col, w=None, trust: bool = False):
        lib = load_library()
        self._h = ctypes.c_void_p()
        flags = MC_TRUST_INPUT if trust else 0
        self.device_ptrs = hasattr(row_ptr, "data_ptr")
        if self.device_ptrs:
            import torch
            for t in (row_ptr, col) + ((w,) if w is not None else ()):
                assert t.is_cuda and t.dtype == torch.int32 and t.is_contiguous()
            n = row_ptr.numel() - 1
            flags |= MC_DEVICE_PTRS
            torch.cuda.current_stream().synchronize()
            rc = lib.mc_graph_create(n, ctypes.c_void_p(row_ptr.data_ptr()),
                                     ctypes.c_void_p(col.data_ptr()),
                                     ctypes.c_void_p(w.data_ptr() if w is not None else None),
                                     flags, ctypes.byref(self._h))
        else:
            rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
            c = np.ascontiguousarray(col, dtype=np.int32)
            ww = np.ascontiguousarray(w, dtype=np.int32) if w is not None else None
            n = len(rp) - 1
            rc = lib.mc_graph_create(n, _ptr(rp), _ptr(c), _ptr(ww) if ww is not None else None,
                                     flags, ctypes.byref(self._h))
        _check(rc, "mc_graph_create")
        self.n = n
        nn, mm = ctypes.c_int64(), ctypes.c_int64()
        _check(lib.mc_graph_size(self._h, ctypes.byref(nn), ctypes.byref(mm)), "mc_graph_size")
        self.m = mm.value

    def close(self):
        if self._h:
            load_library().mc_graph_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---------------------------------------------------------------- solve
    def min_cut(self, opts: McOptions | None = None, side: bool = True, bitmap_out=None) -> MinCut:
        lib = load_library()
        lam = ctypes.c_int64()
        st = McStats()
        nw = (self.n + 31) // 32
        if side and bitmap_out is None:
            if self.device_ptrs:
                import torch
                bitmap_out = torch.empty(nw, dtype=torch.int32, device="cuda")
            else:
                bitmap_out = np.zeros(nw, dtype=np.uint32)
        if bitmap_out is None:
            bp = None
        elif hasattr(bitmap_out, "data_ptr"):
            bp = ctypes.c_void_p(bitmap_out.data_ptr())
        else:
            bp = ctypes.c_void_p(bitmap_out.ctypes.data)
        o = opts if opts is not None else options()
        rc = lib.mc_min_cut(self._h, ctypes.byref(o), ctypes.byref(lam), bp, ctypes.byref(st))
        _check(rc, "mc_min_cut")
        return MinCut(lam.value, bitmap_out, st.as_dict())

    # ---------------------------------------------------------------- steps
    def export(self):
        lib = load_library()
        rp = np.zeros(self.n + 1, dtype=np.int32)
        col = np.zeros(max(1, 2 * self.m), dtype=np.int32)
        w = np.zeros(max(1, 2 * self.m), dtype=np.int32)
        _check(lib.mc_graph_export(self._h, _ptr(rp), _ptr(col), _ptr(w)), "mc_graph_export")
        return rp, col[:2 * self.m], w[:2 * self.m]

    def degrees(self) -> np.ndarray:
        d = np.zeros(self.n, dtype=np.int64)
        _check(load_library().mc_step_degrees(self._h, _ptr(d)), "mc_step_degrees")
        return d

    def contract(self, lab, nc: int, clamp: int = 0):
        lab = np.ascontiguousarray(lab, dtype=np.int32)
        rp = np.zeros(nc + 1, dtype=np.int32)
        # 2m + 1 arcs: a graph made with trust=True may hold an odd number
        col = np.zeros(2 * self.m + 1, dtype=np.int32)
        w = np.zeros(2 * self.m + 1, dtype=np.int32)
        arcs = ctypes.c_int64()
        _check(load_library().mc_step_contract(self._h, _ptr(lab), nc, clamp, _ptr(rp), _ptr(col),
                                               _ptr(w), ctypes.byref(arcs)), "mc_step_contract")
        return rp, col[:arcs.value], w[:arcs.value]

    def pr_tests(self, lam: int, level: int) -> np.ndarray:
        lab = np.zeros(self.n, dtype=np.int32)
        _check(load_library().mc_step_pr(self._h, lam, level, _ptr(lab)), "mc_step_pr")
        return lab

    def capforest_round(self, lam: int, opts: McOptions | None = None):
        lab = np.zeros(self.n, dtype=np.int32)
        lo, un = ctypes.c_int64(), ctypes.c_int64()
        o = opts if opts is not None else options()
        _check(load_library().mc_step_capforest(self._h, lam, ctypes.byref(o), _ptr(lab),
                                                ctypes.byref(lo), ctypes.byref(un)),
               "mc_step_capforest")
        return lab, lo.value, un.value

    def capforest_range(self, lam: int, lo: int, hi: int, opts: McOptions | None = None):
        """(labels, lambda-hat after, unions, side bitmap) of one round of
        concurrent scans that scan only the vertices in [lo, hi)."""
        lab = np.zeros(self.n, dtype=np.int32)
        side = np.zeros((self.n + 31) // 32, dtype=np.uint32)
        lo_, un = ctypes.c_int64(), ctypes.c_int64()
        o = opts if opts is not None else options()
        _check(load_library().mc_step_capforest_range(self._h, lam, ctypes.byref(o), lo, hi, _ptr(lab),
                                                      ctypes.byref(lo_), ctypes.byref(un), _ptr(side)),
               "mc_step_capforest_range")
        return lab, lo_.value, un.value, side

    def capforest_full(self, lam: int, start: int = 0):
        """One full CAPFOREST scan (Alg. 3): (labels, lambda-hat after, unions)."""
        lab = np.zeros(self.n, dtype=np.int32)
        lo, un = ctypes.c_int64(), ctypes.c_int64()
        _check(load_library().mc_step_capforest_full(self._h, lam, start, _ptr(lab),
                                                     ctypes.byref(lo), ctypes.byref(un)),
               "mc_step_capforest_full")
        return lab, lo.value, un.value

    def label_prop(self, iters: int, seed: int) -> np.ndarray:
        lab = np.zeros(self.n, dtype=np.int32)
        _check(load_library().mc_step_label_prop(self._h, iters, seed, _ptr(lab)),
               "mc_step_label_prop")
        return lab

    def coarsen(self, lp_iters: int = 2, seed: int | None = None):
        """The label-propagation cluster graph the learned proposer runs on
        (``mc_graph_coarsen``): returns (Graph, cluster id of every vertex).
        ``seed=None`` takes the one mc_min_cut uses with default options."""
        if seed is None:
            seed = options().seed ^ 0x9E37
        out = ctypes.c_void_p()
        cl = np.zeros(self.n, dtype=np.int32)
        _check(load_library().mc_graph_coarsen(self._h, lp_iters, seed, ctypes.byref(out), _ptr(cl)),
               "mc_graph_coarsen")
        G = Graph.__new__(Graph)
        G._h = out
        G.device_ptrs = False
        nn, mm = ctypes.c_int64(), ctypes.c_int64()
        _check(load_library().mc_graph_size(out, ctypes.byref(nn), ctypes.byref(mm)), "mc_graph_size")
        G.n, G.m = nn.value, mm.value
        return G, cl


NOALLOC_MAX_N = 32768
NOALLOC_MAX_ARCS = 262144


def capforest_full_noalloc(row_ptr, adj, lam: int, start: int, labels, stream=None):
    """Allocation-free full CAPFOREST scan (``mc_capforest_full_noalloc``).

    ``row_ptr`` (int32, n+1), ``adj`` (int32, 2*arcs interleaved neighbour /
    weight) and ``labels`` (int32, n, output) are CUDA tensors; nothing is
    allocated on the device.  Returns (lambda-hat after the scan, unions).
    """
    n = row_ptr.numel() - 1
    arcs = adj.numel() // 2
    lo, un = ctypes.c_int64(), ctypes.c_int64()
    s = ctypes.c_void_p(stream) if stream else None
    _check(load_library().mc_capforest_full_noalloc(
        n, arcs, ctypes.c_void_p(row_ptr.data_ptr()), ctypes.c_void_p(adj.data_ptr()), lam, start,
        ctypes.c_void_p(labels.data_ptr()), ctypes.byref(lo), ctypes.byref(un), s),
        "mc_capforest_full_noalloc")
    return lo.value, un.value


class Proposer:
    """The learned bound proposer (``mc_proposer``): a 3-layer message-passing
    network whose best sweep cut is an exact upper bound on lambda."""

    MAGIC = b"MCPROP01"

    def __init__(self, params=None, seed: int = 0):
        lib = load_library()
        self._h = ctypes.c_void_p()
        arr = None
        if params is not None:
            arr = np.ascontiguousarray(params, dtype=np.float32)
            assert arr.size == PROPOSER_PARAMS
        _check(lib.mc_proposer_create(_ptr(arr), ctypes.c_uint64(seed & (2**64 - 1)),
                                      ctypes.byref(self._h)), "mc_proposer_create")

    def close(self):
        if self._h:
            load_library().mc_proposer_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h.value

    def get(self) -> np.ndarray:
        out = np.zeros(PROPOSER_PARAMS, dtype=np.float32)
        _check(load_library().mc_proposer_get(self._h, _ptr(out)), "mc_proposer_get")
        return out

    def set(self, params):
        arr = np.ascontiguousarray(params, dtype=np.float32)
        _check(load_library().mc_proposer_set(self._h, _ptr(arr)), "mc_proposer_set")

    def forward(self, g: "Graph") -> np.ndarray:
        out = np.zeros(g.n, dtype=np.float32)
        _check(load_library().mc_proposer_forward(self._h, g._h, _ptr(out)), "mc_proposer_forward")
        return out

    def grad(self, g: "Graph", side_bits):
        bits = np.ascontiguousarray(side_bits, dtype=np.uint32)
        loss = ctypes.c_double()
        grad = np.zeros(PROPOSER_PARAMS, dtype=np.float32)
        _check(load_library().mc_proposer_grad(self._h, g._h, _ptr(bits), ctypes.byref(loss),
                                               _ptr(grad)), "mc_proposer_grad")
        return loss.value, grad

    def train_step(self, g: "Graph", side_bits, lr: float) -> float:
        bits = np.ascontiguousarray(side_bits, dtype=np.uint32)
        loss = ctypes.c_double()
        _check(load_library().mc_proposer_train_step(self._h, g._h, _ptr(bits), ctypes.c_float(lr),
                                                     ctypes.byref(loss)), "mc_proposer_train_step")
        return loss.value

    def bound(self, g: "Graph"):
        cut = ctypes.c_int64()
        side = np.zeros((g.n + 31) // 32, dtype=np.uint32)
        _check(load_library().mc_proposer_bound(self._h, g._h, ctypes.byref(cut), _ptr(side)),
               "mc_proposer_bound")
        return cut.value, side

    # versioned weight blob: magic, count (uint32), float32 params, sha256
    def save(self, path: str):
        import hashlib
        w = self.get().astype("<f4").tobytes()
        body = self.MAGIC + np.uint32(PROPOSER_PARAMS).tobytes() + w
        with open(path, "wb") as f:
            f.write(body + hashlib.sha256(body).digest())

    @classmethod
    def load(cls, path: str) -> "Proposer":
        import hashlib
        data = open(path, "rb").read()
        body, digest = data[:-32], data[-32:]
        if body[:8] != cls.MAGIC or hashlib.sha256(body).digest() != digest:
            raise ValueError(f"{path}: not a proposer weight file or corrupted")
        count = int(np.frombuffer(body[8:12], dtype="<u4")[0])
        if count != PROPOSER_PARAMS:
            raise ValueError(f"{path}: {count} parameters, expected {PROPOSER_PARAMS}")
        return cls(np.frombuffer(body[12:], dtype="<f4").copy())


def min_cut(row_ptr, col, w, **opt) -> MinCut:
    """One-shot: create, solve, destroy."""
    with Graph(row_ptr, col, w) as g:
        return g.min_cut(options(**opt))


def batch_shape_count() -> int:
    """How many batched-kernel shapes the autotuner chooses from."""
    return int(load_library().mc_batch_shape_count())


def batch_set_shape(shape: int) -> None:
    """Use batched-kernel shape `shape` (0 .. batch_shape_count() - 1; -1 =
    the default) for later batch_min_cut calls, as batch_autotune does."""
    _check(load_library().mc_batch_set_shape(int(shape)), "mc_batch_set_shape")


def batch_autotune(row_ptr, col, w, vtx_off, arc_off, opts: McOptions | None = None):
    """Pick the fastest batched-kernel shape for this batch (kept for later
    batch_min_cut calls); returns (best shape index, per-shape kernel ms)."""
    lib = load_library()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    c = np.ascontiguousarray(col, dtype=np.int32)
    ww = np.ascontiguousarray(w, dtype=np.int32)
    vo = np.ascontiguousarray(vtx_off, dtype=np.int64)
    ao = np.ascontiguousarray(arc_off, dtype=np.int64)
    best = ctypes.c_int32()
    ms = np.zeros(16, dtype=np.float64)
    o = opts if opts is not None else options()
    _check(lib.mc_batch_autotune(len(vo) - 1, _ptr(vo), _ptr(ao), _ptr(rp), _ptr(c), _ptr(ww),
                                 ctypes.byref(o), ctypes.byref(best), _ptr(ms), 16),
           "mc_batch_autotune")
    return best.value, ms


def batch_min_cut(row_ptr, col, w, vtx_off, arc_off, opts: McOptions | None = None,
                  bitmaps: bool = False):
    """lambda for each graph of a concatenated batch (layout of mc_batch_min_cut)."""
    lib = load_library()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    c = np.ascontiguousarray(col, dtype=np.int32)
    ww = np.ascontiguousarray(w, dtype=np.int32)
    vo = np.ascontiguousarray(vtx_off, dtype=np.int64)
    ao = np.ascontiguousarray(arc_off, dtype=np.int64)
    G = len(vo) - 1
    lam = np.zeros(G, dtype=np.int64)
    bw = bo = None
    if bitmaps:
        words = (np.diff(vo) + 31) // 32
        bo = np.zeros(G + 1, dtype=np.int64)
        bo[1:] = np.cumsum(words)
        bw = np.zeros(int(bo[-1]), dtype=np.uint32)
    st = McStats()
    o = opts if opts is not None else options()
    rc = lib.mc_batch_min_cut(G, _ptr(vo), _ptr(ao), _ptr(rp), _ptr(c), _ptr(ww), ctypes.byref(o),
                              _ptr(lam), _ptr(bw), _ptr(bo), ctypes.byref(st))
    _check(rc, "mc_batch_min_cut")
    return lam, bw, bo, st.as_dict()

"""CPU oracle for the exact global minimum cut -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct C (``mincut_oracle.c``), loaded through ctypes.
Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the CUDA product path never does, and
the two share no code.

Functions (each cites the passage of Henzinger, Noe, Schulz, "Shared-memory
Exact Minimum Cuts" that it follows):

* :func:`cut_weight`   -- Sec. 2.1, capacity c(A) of a cut.
* :func:`degrees`      -- Sec. 2.1, weighted degree (trivial cut bound).
* :func:`brute_force`  -- Sec. 2.1, lambda(G) by enumeration (n <= 26).
* :func:`stoer_wagner` -- Stoer-Wagner maximum-adjacency phases (Sec. 2.2).
* :func:`noi`          -- sequential NOI: CAPFOREST (Alg. 3) with the
  lambda-hat-capped queue (Sec. 3.1.2, Lemma 1) + contraction, side per
  Sec. 3.3.
* :func:`contract`     -- Sec. 2.1 contraction of every block of a labelling.
* :func:`label_prop`   -- label propagation as read for VieCut (Sec. 2.3).
* :func:`pr_tests`     -- Padberg-Rinaldi tests as read for VieCut (Sec. 2.3).

Sides are uint8 arrays with side[v] = 1 iff v is not on vertex 0's side.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mincut_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORC_EINVAL = -1
ORC_ENOMEM = -2
ORC_ENOPROGRESS = -3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build/liboracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-Wall", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        I32P = ctypes.POINTER(ctypes.c_int32)
        I64P = ctypes.POINTER(ctypes.c_int64)
        U8P = ctypes.POINTER(ctypes.c_uint8)
        i32, i64, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        lib.orc_cut_weight.argtypes = [i32, I32P, I32P, I32P, U8P]
        lib.orc_cut_weight.restype = i64
        lib.orc_degrees.argtypes = [i32, I32P, I32P, I32P, I64P]
        lib.orc_degrees.restype = ctypes.c_int
        lib.orc_brute_force.argtypes = [i32, I32P, I32P, I32P, U8P]
        lib.orc_brute_force.restype = i64
        lib.orc_stoer_wagner.argtypes = [i32, I32P, I32P, I32P, U8P]
        lib.orc_stoer_wagner.restype = i64
        lib.orc_noi.argtypes = [i32, I32P, I32P, I32P, ctypes.c_int, u64, U8P, I32P]
        lib.orc_noi.restype = i64
        lib.orc_matula.argtypes = [i32, I32P, I32P, I32P, ctypes.c_int, u64, U8P, I32P]
        lib.orc_matula.restype = i64
        lib.orc_capforest_round.argtypes = [i32, I32P, I32P, I32P, i64, i32, I32P]
        lib.orc_capforest_round.restype = i64
        lib.orc_contract.argtypes = [i32, I32P, I32P, I32P, I32P, i32, I64P, I32P, I64P]
        lib.orc_contract.restype = i64
        lib.orc_label_prop.argtypes = [i32, I32P, I32P, I32P, ctypes.c_int, u64, I32P]
        lib.orc_label_prop.restype = ctypes.c_int
        lib.orc_pr_tests.argtypes = [i32, I32P, I32P, I32P, i64, ctypes.c_int, I32P]
        lib.orc_pr_tests.restype = ctypes.c_int
        lib.orc_splitmix64.argtypes = [u64]
        lib.orc_splitmix64.restype = u64
        _lib = lib
        return lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _csr(rp, col, w):
    rp = np.ascontiguousarray(rp, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.int32)
    return len(rp) - 1, rp, col, w


def _check(rc, what):
    if rc < 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")
    return rc


def splitmix64(x: int) -> int:
    """The oracle's splitmix64 finaliser (start vertices, LP parity)."""
    return int(_load().orc_splitmix64(ctypes.c_uint64(x & (2**64 - 1))))


def cut_weight(rp, col, w, side) -> int:
    n, rp, col, w = _csr(rp, col, w)
    side = np.ascontiguousarray(side, dtype=np.uint8)
    assert len(side) == n
    return int(_check(_load().orc_cut_weight(n, _p(rp, ctypes.c_int32), _p(col, ctypes.c_int32),
                                             _p(w, ctypes.c_int32), _p(side, ctypes.c_uint8)),
                      "cut_weight"))


def degrees(rp, col, w) -> np.ndarray:
    n, rp, col, w = _csr(rp, col, w)
    deg = np.zeros(n, dtype=np.int64)
    _check(_load().orc_degrees(n, _p(rp, ctypes.c_int32), _p(col, ctypes.c_int32),
                               _p(w, ctypes.c_int32), _p(deg, ctypes.c_int64)), "degrees")
    return deg


def brute_force(rp, col, w):
    """(lambda, side) by enumerating all 2^(n-1)-1 cuts; n <= 26."""
    n, rp, col, w = _csr(rp, col, w)
    side = np.zeros(n, dtype=np.uint8)
    lam = _check(_load().orc_brute_force(n, _p(rp, ctypes.c_int32), _p(col, ctypes.c_int32),
                                         _p(w, ctypes.c_int32), _p(side, ctypes.c_uint8)),
                 "brute_force")
    return int(lam), side


def stoer_wagner(rp, col, w):
    n, rp, col, w = _csr(rp, col, w)
    side = np.zeros(n, dtype=np.uint8)
    lam = _check(_load().orc_stoer_wagner(n, _p(rp, ctypes.c_int32), _p(col, ctypes.c_int32),
                                          _p(w, ctypes.c_int32), _p(side, ctypes.c_uint8)),
                 "stoer_wagner")
    return int(lam), side


def noi(rp, col, w, capped: bool = True, seed: int = 0):
    """(lambda, side, rounds) by sequential NOI with the lambda-hat cap."""
    n, rp, col, w = _csr(rp, col, w)
    side = np.zeros(n, dtype=np.uint8)
    rounds = np.zeros(1, dtype=np.int32)
    lam = _check(_load().orc_noi(n, _p(rp, ctypes.c_int32), _p(col, ctypes.c_int32),
                                 _p(w, ctypes.c_int32), 1 if capped else 0,
                                 ctypes.c_uint64(seed & (2**64 - 1)),
                                 _p(side, ctypes.c_uint8), _p(rounds, ctypes.c_int32)), "noi")
    return int(lam), side, int(rounds[0])


def capforest_round(rp, col, w, lam: int, start: int):
    """(lambda-hat after the scan, labels) of one capped CAPFOREST scan from
    start: labels[v] = the smallest vertex of v's block of marked edges."""
    n, rp, col, w = _csr(rp, col, w)
    lab = np.zeros(n, dtype=np.int32)
    out = _check(_load().orc_capforest_round(n, _p(rp, ctypes.c_int32), _p(col, ctypes.c_int32),
                                             _p(w, ctypes.c_int32), int(lam), int(start),
                                             _p(lab, ctypes.c_int32)), "capforest_round")
    return int(out), lab


def matula(rp, col, w, approx_milli: int, seed: int = 0):
    """(cut, side, rounds) by Matula's approximation: the NOI loop marking at
    ceil(approx_milli * delta / 1000) each round; lambda <= cut <=
    1000 / approx_milli * lambda."""
    n, rp, col, w = _csr(rp, col, w)
    side = np.zeros(n, dtype=np.uint8)
    rounds = np.zeros(1, dtype=np.int32)
    lam = _check(_load().orc_matula(n, _p(rp, ctypes.c_int32), _p(col, ctypes.c_int32),
                                    _p(w, ctypes.c_int32), int(approx_milli),
                                    ctypes.c_uint64(seed & (2**64 - 1)),
                                    _p(side, ctypes.c_uint8), _p(rounds, ctypes.c_int32)), "matula")
    return int(lam), side, int(rounds[0])


def contract(rp, col, w, lab, nc):
    """Canonical CSR (rp int64, col int32, w int64) of G contracted by lab."""
    n, rp, col, w = _csr(rp, col, w)
    lab = np.ascontiguousarray(lab, dtype=np.int32)
    orp = np.zeros(nc + 1, dtype=np.int64)
    ocol = np.zeros(max(1, len(col)), dtype=np.int32)
    ow = np.zeros(max(1, len(col)), dtype=np.int64)
    m = _check(_load().orc_contract(n, _p(rp, ctypes.c_int32), _p(col, ctypes.c_int32),
                                    _p(w, ctypes.c_int32), _p(lab, ctypes.c_int32), nc,
                                    _p(orp, ctypes.c_int64), _p(ocol, ctypes.c_int32),
                                    _p(ow, ctypes.c_int64)), "contract")
    return orp, ocol[:m].copy(), ow[:m].copy()


def label_prop(rp, col, w, iters: int, seed: int) -> np.ndarray:
    n, rp, col, w = _csr(rp, col, w)
    lab = np.zeros(n, dtype=np.int32)
    _check(_load().orc_label_prop(n, _p(rp, ctypes.c_int32), _p(col, ctypes.c_int32),
                                  _p(w, ctypes.c_int32), iters,
                                  ctypes.c_uint64(seed & (2**64 - 1)), _p(lab, ctypes.c_int32)),
           "label_prop")
    return lab


def pr_tests(rp, col, w, lam: int, level: int) -> np.ndarray:
    n, rp, col, w = _csr(rp, col, w)
    lab = np.zeros(n, dtype=np.int32)
    _check(_load().orc_pr_tests(n, _p(rp, ctypes.c_int32), _p(col, ctypes.c_int32),
                                _p(w, ctypes.c_int32), lam, level, _p(lab, ctypes.c_int32)),
           "pr_tests")
    return lab

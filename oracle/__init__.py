"""ctypes front end of the epi3 CPU oracle -- TEST INFRASTRUCTURE ONLY.

The oracle (``epi3_oracle.c``) is a plain FP64 statement of the scan: counts one
sample at a time, K2 by Eq. 1, top-k by (K2, i, j, k).  Only the tests, the
smoke check and the benchmark's CPU-baseline leg may import this module; the
library never does, and nothing here is shared with it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "epi3_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")

def build(force: bool = False, src: str = _SRC, out: str = _LIB) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no FP contraction)."""
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off",
                           "-fPIC", "-shared", src, "-o", tmp, "-lm"])
    os.replace(tmp, out)
    return out


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _inputs(genotypes, phenotype):
    g = np.ascontiguousarray(genotypes, dtype=np.uint8)
    p = np.ascontiguousarray(phenotype, dtype=np.uint8)
    if g.ndim != 2 or p.ndim != 1 or g.shape[1] != p.shape[0]:
        raise ValueError("genotypes must be [M, N] and phenotype [N]")
    return g, p


class Oracle:
    """The oracle's entry points, bound to one compiled copy of the C source."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        lib.oracle_log_factorials.argtypes = [ctypes.c_int32, P]
        lib.oracle_tables.argtypes = [P, P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, P, P]
        lib.oracle_k2.argtypes = [ctypes.c_int64, P, P]
        lib.oracle_scores.argtypes = [P, P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, P, P,
                                      ctypes.c_int32]
        lib.oracle_scan_topk.argtypes = [P, P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, P, P,
                                         ctypes.c_int32]
        lib.oracle_pair_tables.argtypes = [P, P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, P, P]
        lib.oracle_scan_pairs_topk.argtypes = [P, P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                               P, P, ctypes.c_int32]
        lib.oracle_tables_order.argtypes = [P, P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                            ctypes.c_int64, P, P]
        lib.oracle_k2_cells.argtypes = [ctypes.c_int64, ctypes.c_int32, P, P]
        lib.oracle_scan_order_topk.argtypes = [P, P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                               ctypes.c_int32, P, P, ctypes.c_int32]
        for f in (lib.oracle_tables_order, lib.oracle_k2_cells, lib.oracle_scan_order_topk):
            f.restype = ctypes.c_int
        for f in (lib.oracle_log_factorials, lib.oracle_tables, lib.oracle_k2, lib.oracle_scores,
                  lib.oracle_scan_topk):
            f.restype = ctypes.c_int
        self._lib = lib

    def log_factorials(self, n_max: int) -> np.ndarray:
        """lf[n] = sum_{b=1..n} log b for n = 0..n_max (Eq. 1 inner sums)."""
        out = np.empty(n_max + 1, dtype=np.float64)
        if self._lib.oracle_log_factorials(n_max, _ptr(out)):
            raise ValueError("n_max < 0")
        return out

    def tables(self, genotypes, phenotype, triplets) -> np.ndarray:
        """[n, 2, 27] int32 frequency tables; cell = 9 gX + 3 gY + gZ, row 0 = controls."""
        g, p = _inputs(genotypes, phenotype)
        t = np.ascontiguousarray(triplets, dtype=np.int32).reshape(-1, 3)
        out = np.empty((t.shape[0], 2, 27), dtype=np.int32)
        if self._lib.oracle_tables(_ptr(g), _ptr(p), g.shape[0], g.shape[1], t.shape[0], _ptr(t),
                                   _ptr(out)):
            raise ValueError("bad triplet index or genotype/phenotype value")
        return out

    def k2(self, tables_) -> np.ndarray:
        """FP64 K2 (Eq. 1) of [n, 2, 27] tables."""
        t = np.ascontiguousarray(tables_, dtype=np.int32).reshape(-1, 2, 27)
        out = np.empty(t.shape[0], dtype=np.float64)
        if self._lib.oracle_k2(t.shape[0], _ptr(t), _ptr(out)):
            raise ValueError("negative count")
        return out

    def scores(self, genotypes, phenotype, triplets, threads: int = 0) -> np.ndarray:
        """FP64 K2 of each listed triplet, counted sample by sample."""
        g, p = _inputs(genotypes, phenotype)
        t = np.ascontiguousarray(triplets, dtype=np.int32).reshape(-1, 3)
        out = np.empty(t.shape[0], dtype=np.float64)
        if self._lib.oracle_scores(_ptr(g), _ptr(p), g.shape[0], g.shape[1], t.shape[0], _ptr(t),
                                   _ptr(out), threads):
            raise ValueError("bad triplet index or genotype/phenotype value")
        return out

    def scan_topk(self, genotypes, phenotype, top_k: int, threads: int = 0):
        """Exhaustive scan; returns (triplets int32 [k, 3], K2 float64 [k], threads used)."""
        g, p = _inputs(genotypes, phenotype)
        trip = np.empty((top_k, 3), dtype=np.int32)
        sc = np.empty(top_k, dtype=np.float64)
        rc = self._lib.oracle_scan_topk(_ptr(g), _ptr(p), g.shape[0], g.shape[1], top_k, _ptr(trip),
                                        _ptr(sc), threads)
        if rc < 0:
            raise ValueError("bad arguments or values")
        return trip, sc, rc


    def pair_tables(self, genotypes, phenotype, pairs) -> np.ndarray:
        """[n, 2, 9] int32 tables of the given SNP pairs (cell = 3 gX + gY)."""
        g, p = _inputs(genotypes, phenotype)
        t = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        out = np.empty((t.shape[0], 2, 9), dtype=np.int32)
        if self._lib.oracle_pair_tables(_ptr(g), _ptr(p), g.shape[0], g.shape[1], t.shape[0],
                                        _ptr(t), _ptr(out)):
            raise ValueError("bad pair index or genotype/phenotype value")
        return out

    def scan_pairs_topk(self, genotypes, phenotype, top_k: int, threads: int = 0):
        """Exhaustive pairwise scan; returns (pairs int32 [k, 2], K2 float64 [k], threads used)."""
        g, p = _inputs(genotypes, phenotype)
        pairs = np.empty((top_k, 2), dtype=np.int32)
        sc = np.empty(top_k, dtype=np.float64)
        rc = self._lib.oracle_scan_pairs_topk(_ptr(g), _ptr(p), g.shape[0], g.shape[1], top_k,
                                              _ptr(pairs), _ptr(sc), threads)
        if rc < 0:
            raise ValueError("bad arguments or values")
        return pairs, sc, rc


    def tables_order(self, genotypes, phenotype, snps) -> np.ndarray:
        """[n, 2, 3^order] int32 tables of SNP sets snps [n, order] (Eq. 1 for `order` SNPs;
        cell = genotypes as base-3 digits, first SNP most significant)."""
        g, p = _inputs(genotypes, phenotype)
        x = np.ascontiguousarray(snps, dtype=np.int32)
        if x.ndim != 2:
            raise ValueError("snps must be [n, order]")
        order = x.shape[1]
        out = np.empty((x.shape[0], 2, 3 ** order), dtype=np.int32)
        if self._lib.oracle_tables_order(_ptr(g), _ptr(p), g.shape[0], g.shape[1], order,
                                         x.shape[0], _ptr(x), _ptr(out)):
            raise ValueError("bad order, SNP index or genotype/phenotype value")
        return out

    def k2_cells(self, tables_) -> np.ndarray:
        """FP64 K2 (Eq. 1) of [n, 2, ncell] tables, summed in cell order."""
        t = np.ascontiguousarray(tables_, dtype=np.int32)
        if t.ndim != 3 or t.shape[1] != 2:
            raise ValueError("tables must be [n, 2, ncell]")
        out = np.empty(t.shape[0], dtype=np.float64)
        if self._lib.oracle_k2_cells(t.shape[0], t.shape[2], _ptr(t), _ptr(out)):
            raise ValueError("negative count")
        return out

    def scan_order_topk(self, genotypes, phenotype, order: int, top_k: int, threads: int = 0):
        """Exhaustive scan over every set of `order` SNPs; returns (sets int32 [k, order],
        K2 float64 [k], threads used), ordered by (K2, SNP indices)."""
        g, p = _inputs(genotypes, phenotype)
        x = np.empty((top_k, order), dtype=np.int32)
        sc = np.empty(top_k, dtype=np.float64)
        rc = self._lib.oracle_scan_order_topk(_ptr(g), _ptr(p), g.shape[0], g.shape[1], order,
                                              top_k, _ptr(x), _ptr(sc), threads)
        if rc < 0:
            raise ValueError("bad arguments or values")
        return x, sc, rc


_default = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(build())
    return _default


def log_factorials(n_max):
    return default().log_factorials(n_max)


def tables(genotypes, phenotype, triplets):
    return default().tables(genotypes, phenotype, triplets)


def k2(tables_):
    return default().k2(tables_)


def scores(genotypes, phenotype, triplets, threads: int = 0):
    return default().scores(genotypes, phenotype, triplets, threads)


def scan_topk(genotypes, phenotype, top_k, threads: int = 0):
    return default().scan_topk(genotypes, phenotype, top_k, threads)


def pair_tables(genotypes, phenotype, pairs):
    return default().pair_tables(genotypes, phenotype, pairs)


def scan_pairs_topk(genotypes, phenotype, top_k, threads: int = 0):
    return default().scan_pairs_topk(genotypes, phenotype, top_k, threads)


def tables_order(genotypes, phenotype, snps):
    return default().tables_order(genotypes, phenotype, snps)


def k2_cells(tables_):
    return default().k2_cells(tables_)


def scan_order_topk(genotypes, phenotype, order, top_k, threads: int = 0):
    return default().scan_order_topk(genotypes, phenotype, order, top_k, threads)

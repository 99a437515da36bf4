"""Python binding of the epi3 C ABI (include/epi3.h): argument marshalling only.

Every step of the scan runs in the CUDA library ``libepi3.so`` built next to this
file.  There is no fallback: if the library is missing or no sm_103 GPU is
present, calls raise ``Epi3Error``.

Inputs may be numpy arrays (host memory; results come back as numpy arrays) or
CUDA torch tensors (device memory, ``EPI3_DEVICE_PTRS``; results come back as
CUDA tensors).  torch is used only for device buffers and streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libepi3.so")

OK = 0
ERR_ARG, ERR_CUDA, ERR_OOM, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_OVERFLOW = -1, -2, -3, -4, -5, -6
DEVICE_PTRS = 1
PATH_AUTO, PATH_POPC, PATH_POPC8, PATH_MMA, PATH_MMA16, PATH_MMA4, PATH_MMA4C = 0, 1, 2, 3, 4, 5, 6
MAX_TOPK = 512

# Every symbol the header declares; tests check the library exports all of them.
SYMBOLS = ("epi3_create", "epi3_scan", "epi3_scan_range", "epi3_scan_pairs", "epi3_scan_order",
           "epi3_destroy",
           "epi3_last_error",
           "epi3_tables", "epi3_scores", "epi3_set_option", "epi3_get_stats", "epi3_get_shape",
           "epi3_scan_noalloc", "epi3_scan_scores", "epi3_scan_checksum", "epi3_batch_create", "epi3_batch_scan",
           "epi3_batch_destroy", "epi3_batch_get_stats", "epi3_batch_get_paths", "epi3_batch_get_forms",
           "epi3_scan_batch")


class Epi3Error(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"epi3 error {code}: {msg}")
        self.code = code


class Cohort(ctypes.Structure):
    _fields_ = [("genotypes", ctypes.c_void_p), ("phenotype", ctypes.c_void_p),
                ("n_snps", ctypes.c_int32), ("n_samples", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("n_triplets", ctypes.c_int64), ("n_candidates", ctypes.c_int64),
                ("n_rescored", ctypes.c_int64), ("scan_kernel_ms", ctypes.c_float),
                ("select_ms", ctypes.c_float), ("total_ms", ctypes.c_float),
                ("pack_ms", ctypes.c_float), ("path", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("block", ctypes.c_int32), ("kernel_launches", ctypes.c_int32),
                ("k2_rel_bound", ctypes.c_float), ("k2_abs_bound", ctypes.c_float),
                ("wait_loader", ctypes.c_float), ("wait_mma_operands", ctypes.c_float),
                ("wait_mma_accum", ctypes.c_float), ("wait_producers", ctypes.c_float),
                ("wait_epilogue", ctypes.c_float), ("wait_producers_tmem", ctypes.c_float),
                ("mma_issue", ctypes.c_float), ("k2_prune_bound", ctypes.c_float),
                ("compact_ms", ctypes.c_float), ("form", ctypes.c_int32)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libepi3.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise Epi3Error(ERR_UNSUPPORTED,
                        f"{path} not built; run `python -m paper_2201_10956_gb300.build`")
    lib = ctypes.CDLL(path)
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "epi3_create": [ctypes.POINTER(P), P, P, I32, I32, I32, P],
        "epi3_scan": [P, I32, P, P],
        "epi3_scan_range": [P, I64, I64, I32, P, P, ctypes.POINTER(I32)],
        "epi3_scan_pairs": [P, I32, P, P],
        "epi3_scan_order": [P, I32, I32, P, P],
        "epi3_destroy": [P],
        "epi3_last_error": [],
        "epi3_tables": [P, I64, P, P, I32],
        "epi3_scores": [P, I64, P, P, P],
        "epi3_set_option": [P, ctypes.c_char_p, ctypes.c_char_p],
        "epi3_get_stats": [P, ctypes.POINTER(Stats)],
        "epi3_get_shape": [P, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I32),
                           ctypes.POINTER(I32)],
        "epi3_scan_noalloc": [P, P, I32, I32, I32, P, P, P],
        "epi3_scan_scores": [P, I32, P],
        "epi3_scan_checksum": [P, I32, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int64)],
        "epi3_batch_create": [ctypes.POINTER(P), I32, P, I32, P],
        "epi3_batch_scan": [P, I32, P, P],
        "epi3_batch_destroy": [P],
        "epi3_batch_get_stats": [P, ctypes.POINTER(Stats)],
        "epi3_batch_get_paths": [P, P],
        "epi3_batch_get_forms": [P, P],
        "epi3_scan_batch": [I32, P, I32, P, P, I32, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_char_p if name == "epi3_last_error" else ctypes.c_int
    _lib = lib
    return lib


def last_error() -> str:
    return load().epi3_last_error().decode()


def _check(rc: int):
    if rc != OK:
        raise Epi3Error(rc, last_error())


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        return ctypes.c_void_p(x.data_ptr())
    return x.ctypes.data_as(ctypes.c_void_p)


class Handle:
    """One packed data set on the GPU (epi3_create / epi3_destroy)."""

    def __init__(self, genotypes, phenotype, stream=None):
        lib = load()
        self._dev = _is_torch(genotypes)
        if self._dev:
            import torch
            if not (genotypes.is_cuda and phenotype.is_cuda):
                raise Epi3Error(ERR_ARG, "torch inputs must be CUDA tensors")
            g = genotypes.contiguous().to(torch.uint8)
            p = phenotype.contiguous().to(torch.uint8)
            if stream is None:
                stream = torch.cuda.current_stream(g.device)
            self._keep = (g, p)
            m, n = g.shape
        else:
            g = np.ascontiguousarray(genotypes, dtype=np.uint8)
            p = np.ascontiguousarray(phenotype, dtype=np.uint8)
            m, n = g.shape
        if p.shape[0] != n:
            raise Epi3Error(ERR_ARG, "phenotype length does not match genotypes")
        sptr = None
        if stream is not None:
            sptr = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        self._stream = stream
        h = ctypes.c_void_p()
        _check(lib.epi3_create(ctypes.byref(h), _ptr(g), _ptr(p), int(m), int(n),
                               DEVICE_PTRS if self._dev else 0, sptr))
        self._h = h
        self._keep = None  # packed planes are owned by the handle
        self.n_snps, self.n_samples = int(m), int(n)

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            load().epi3_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- helpers
    def _alloc(self, shape, dtype):
        if self._dev:
            import torch
            tdt = {np.int32: torch.int32, np.float64: torch.float64, np.float32: torch.float32}[dtype]
            return torch.empty(shape, dtype=tdt, device="cuda")
        return np.empty(shape, dtype=dtype)

    def _triplets(self, triplets):
        if self._dev:
            import torch
            t = torch.as_tensor(triplets, dtype=torch.int32, device="cuda").reshape(-1, 3).contiguous()
        else:
            t = np.ascontiguousarray(triplets, dtype=np.int32).reshape(-1, 3)
        return t

    # -- API
    def scan(self, top_k: int):
        """Top-k triplets (int32 [k, 3]) and FP64 K2 scores ([k]), ascending."""
        trip = self._alloc((top_k, 3), np.int32)
        sc = self._alloc((top_k,), np.float64)
        _check(load().epi3_scan(self._h, int(top_k), _ptr(trip), _ptr(sc)))
        return trip, sc

    def scan_range(self, pair_begin: int, pair_end: int, top_k: int):
        trip = self._alloc((top_k, 3), np.int32)
        sc = self._alloc((top_k,), np.float64)
        n = ctypes.c_int32(0)
        _check(load().epi3_scan_range(self._h, int(pair_begin), int(pair_end), int(top_k),
                                      _ptr(trip), _ptr(sc), ctypes.byref(n)))
        return trip[: n.value], sc[: n.value]

    def scan_pairs(self, top_k: int):
        """Pairwise scan (Eq. 1 for two SNPs): top-k pairs (int32 [k, 2]) and FP64 K2 ([k])."""
        pairs = self._alloc((top_k, 2), np.int32)
        sc = self._alloc((top_k,), np.float64)
        _check(load().epi3_scan_pairs(self._h, int(top_k), _ptr(pairs), _ptr(sc)))
        return pairs, sc

    def scan_order(self, order: int, top_k: int):
        """Scan of interaction order 2, 3 or 4 (Eq. 1 for that many SNPs): top-k SNP sets
        (int32 [k, order]) and FP64 K2 ([k])."""
        sets = self._alloc((top_k, order), np.int32)
        sc = self._alloc((top_k,), np.float64)
        _check(load().epi3_scan_order(self._h, int(order), int(top_k), _ptr(sets), _ptr(sc)))
        return sets, sc

    def tables(self, triplets, path: int = PATH_AUTO):
        t = self._triplets(triplets)
        out = self._alloc((t.shape[0], 2, 27), np.int32)
        _check(load().epi3_tables(self._h, int(t.shape[0]), _ptr(t), _ptr(out), int(path)))
        return out

    def scores(self, triplets):
        """(FP32 K2 as the scan computes it, FP64 K2 as the rescoring computes it)."""
        t = self._triplets(triplets)
        s32 = self._alloc((t.shape[0],), np.float32)
        s64 = self._alloc((t.shape[0],), np.float64)
        _check(load().epi3_scores(self._h, int(t.shape[0]), _ptr(t), _ptr(s32), _ptr(s64)))
        return s32, s64

    def scan_scores(self, path: int):
        """FP32 K2 the scan kernel of `path` computes for every triplet: [M, M, M], NaN off
        the i < j < k entries (M <= 512)."""
        m = self.n_snps
        out = self._alloc((m, m, m), np.float32)
        _check(load().epi3_scan_scores(self._h, int(path), _ptr(out)))
        return out

    def scan_checksum(self, path: int):
        """(sum of table hashes mod 2^64, tables counted) of a full scan by the kernel of
        `path`, no pruning: two counting forms agree table by table iff their sums agree."""
        total, count = ctypes.c_uint64(0), ctypes.c_int64(0)
        _check(load().epi3_scan_checksum(self._h, int(path), ctypes.byref(total), ctypes.byref(count)))
        return int(total.value), int(count.value)

    def set_option(self, key: str, value):
        _check(load().epi3_set_option(self._h, key.encode(), str(value).encode()))

    def stats(self) -> dict:
        s = Stats()
        _check(load().epi3_get_stats(self._h, ctypes.byref(s)))
        return {name: getattr(s, name) for name, _ in Stats._fields_}

    def shape(self):
        v = [ctypes.c_int32() for _ in range(4)]
        _check(load().epi3_get_shape(self._h, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)


class Batch:
    """Many cohorts scanned together (epi3_batch_*): one persistent tensor-core launch for
    the cohorts the tuner gives to it, everything replayed from one CUDA graph.

    datasets: list of (genotypes [M, N], phenotype [N]) pairs, all numpy (host) or all CUDA
    torch tensors (device)."""

    def __init__(self, datasets, stream=None):
        lib = load()
        self._dev = _is_torch(datasets[0][0])
        keep, arr = [], (Cohort * len(datasets))()
        for c, (g, p) in enumerate(datasets):
            if self._dev:
                import torch
                g = g.contiguous().to(torch.uint8)
                p = p.contiguous().to(torch.uint8)
            else:
                g = np.ascontiguousarray(g, dtype=np.uint8)
                p = np.ascontiguousarray(p, dtype=np.uint8)
            keep.append((g, p))
            arr[c] = Cohort(_ptr(g).value, _ptr(p).value, int(g.shape[0]), int(g.shape[1]))
        sptr = None
        if stream is not None:
            sptr = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        elif self._dev:
            import torch
            sptr = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        b = ctypes.c_void_p()
        _check(lib.epi3_batch_create(ctypes.byref(b), len(datasets), ctypes.cast(arr, ctypes.c_void_p),
                                     DEVICE_PTRS if self._dev else 0, sptr))
        self._b = b
        self.n = len(datasets)

    def close(self):
        if getattr(self, "_b", None):
            load().epi3_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def scan(self, top_k: int):
        """Per cohort top-k: triplets [n, k, 3] int32, FP64 K2 [n, k]."""
        if self._dev:
            import torch
            trip = torch.empty((self.n, top_k, 3), dtype=torch.int32, device="cuda")
            sc = torch.empty((self.n, top_k), dtype=torch.float64, device="cuda")
        else:
            trip = np.empty((self.n, top_k, 3), dtype=np.int32)
            sc = np.empty((self.n, top_k), dtype=np.float64)
        _check(load().epi3_batch_scan(self._b, int(top_k), _ptr(trip), _ptr(sc)))
        return trip, sc

    def stats(self) -> dict:
        s = Stats()
        _check(load().epi3_batch_get_stats(self._b, ctypes.byref(s)))
        return {name: getattr(s, name) for name, _ in Stats._fields_}

    def paths(self):
        out = np.empty(self.n, dtype=np.int32)
        _check(load().epi3_batch_get_paths(self._b, _ptr(out)))
        return out

    def forms(self):
        """Per cohort: 0 not a tensor cohort, 1 plain, 2 register-split, -1 not measured yet."""
        out = np.empty(self.n, dtype=np.int32)
        _check(load().epi3_batch_get_forms(self._b, _ptr(out)))
        return out


def scan_batch(datasets, top_k: int):
    """One-shot epi3_scan_batch on host (numpy) inputs."""
    lib = load()
    keep, arr = [], (Cohort * len(datasets))()
    for c, (g, p) in enumerate(datasets):
        g = np.ascontiguousarray(g, dtype=np.uint8)
        p = np.ascontiguousarray(p, dtype=np.uint8)
        keep.append((g, p))
        arr[c] = Cohort(_ptr(g).value, _ptr(p).value, int(g.shape[0]), int(g.shape[1]))
    trip = np.empty((len(datasets), top_k, 3), dtype=np.int32)
    sc = np.empty((len(datasets), top_k), dtype=np.float64)
    _check(lib.epi3_scan_batch(len(datasets), ctypes.cast(arr, ctypes.c_void_p), int(top_k),
                               _ptr(trip), _ptr(sc), 0, None))
    return trip, sc


def scan_noalloc(genotypes, phenotype, top_k: int, stream=None):
    """epi3_scan_noalloc on CUDA tensors: the scan with no memory allocated by the library.

    For callers that cannot allocate (fixed memory budgets, foreign allocators); the
    outputs are allocated here by torch, the scratch is the library's static device array
    (8 MiB).  It runs the 27-cell POPC scan and synchronises the stream, so it is not for
    a capturing stream.  Returns (triplets int32 [k, 3], scores float64 [k]) on the device.
    """
    import torch
    m, n = genotypes.shape
    trip = torch.empty((top_k, 3), dtype=torch.int32, device=genotypes.device)
    sc = torch.empty((top_k,), dtype=torch.float64, device=genotypes.device)
    if stream is None:
        stream = torch.cuda.current_stream(genotypes.device)
    _check(load().epi3_scan_noalloc(_ptr(genotypes), _ptr(phenotype), int(m), int(n), int(top_k),
                                    _ptr(trip), _ptr(sc), ctypes.c_void_p(stream.cuda_stream)))
    return trip, sc


def pairs_of(m: int) -> int:
    return m * (m - 1) // 2

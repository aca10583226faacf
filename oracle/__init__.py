"""CPU oracle for PCF Learned Sort -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never imports it and shares no code with it.

The C sources (``pcf_oracle.c``, ``brute.c``) implement Algorithm 1 with the
PCF model of Sec. 3.3 of Sato & Matsui, "PCF Learned Sort"; every reading of
an open point is listed at the top of ``pcf_oracle.c``.  This module is a
ctypes wrapper: keys are passed as numpy arrays (float64 or uint64), payloads
as uint32.
"""
import ctypes
import numpy as np

from . import build as _build

KEY_F64 = 0
KEY_U64 = 1
OK, ERR_ARG, ERR_NAN, ERR_OOM = 0, 1, 2, 3


MODEL_PCF, MODEL_SPLINE = 0, 1


class Policy(ctypes.Structure):
    """alpha = floor(n^(a_num/den)), ... delta = floor(n^(d_num/den)); tau;
    model: the CDF model (MODEL_PCF, Sec. 3.3, or MODEL_SPLINE, App. A.5)."""
    _fields_ = [("a_num", ctypes.c_uint32), ("b_num", ctypes.c_uint32),
                ("c_num", ctypes.c_uint32), ("d_num", ctypes.c_uint32),
                ("den", ctypes.c_uint32), ("tau", ctypes.c_uint64),
                ("model", ctypes.c_uint32), ("range_mode", ctypes.c_uint32)]


class Stats(ctypes.Structure):
    _fields_ = [("max_depth", ctypes.c_uint64), ("n_bucketings", ctypes.c_uint64),
                ("n_small", ctypes.c_uint64), ("n_fallback", ctypes.c_uint64),
                ("fallback_keys", ctypes.c_uint64), ("n_single", ctypes.c_uint64),
                ("n_degenerate", ctypes.c_uint64), ("recursed_violations", ctypes.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


RANGE_ARRAY, RANGE_SAMPLE = 0, 1


def paper_policy(tau: int = 100, model: int = MODEL_PCF, range_mode: int = RANGE_ARRAY) -> Policy:
    """alpha = beta = gamma = delta = floor(n^{3/4}), tau = 100 (Sec. 4 setup);
    range_mode RANGE_SAMPLE bins over the samples' range (reading R14)."""
    return Policy(3, 3, 3, 3, 4, tau, model, range_mode)


_lib = None
_u64p = ctypes.POINTER(ctypes.c_uint64)
_u32p = ctypes.POINTER(ctypes.c_uint32)


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(_build.build())
        L.orc_root_floor.restype = ctypes.c_uint64
        L.orc_root_floor.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
        L.orc_splitmix64_mix.restype = ctypes.c_uint64
        L.orc_splitmix64_mix.argtypes = [ctypes.c_uint64]
        L.orc_sample_state.restype = ctypes.c_uint64
        L.orc_sample_state.argtypes = [ctypes.c_uint64] * 4
        L.orc_sample_index.restype = ctypes.c_uint64
        L.orc_sample_index.argtypes = [ctypes.c_uint64] * 3
        L.orc_bins.restype = ctypes.c_int
        L.orc_bins.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                               _u64p, ctypes.c_uint64, _u64p]
        L.orc_std_sort.restype = ctypes.c_int
        L.orc_std_sort.argtypes = [_u64p, _u32p, ctypes.c_uint64, ctypes.c_int]
        L.orc_sort.restype = ctypes.c_int
        L.orc_sort.argtypes = [_u64p, _u32p, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64,
                               ctypes.POINTER(Policy), ctypes.POINTER(Stats)]
        L.orc_level0.restype = ctypes.c_int
        L.orc_level0.argtypes = [_u64p, _u32p, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64,
                                 ctypes.POINTER(Policy), _u64p, _u64p, _u64p, _u64p, _u64p,
                                 ctypes.POINTER(ctypes.c_int)]
        L.orc_bucket_sizes.restype = ctypes.c_int
        L.orc_bucket_sizes.argtypes = [_u64p, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64,
                                       ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                       ctypes.c_uint32, ctypes.c_uint32, _u64p,
                                       ctypes.POINTER(ctypes.c_int)]
        L.brute_insertion_sort.restype = None
        L.brute_insertion_sort.argtypes = [_u64p, _u32p, ctypes.c_uint64, ctypes.c_int]
        L.brute_cumulative_counts.restype = None
        L.brute_cumulative_counts.argtypes = [_u64p, ctypes.c_uint64, ctypes.c_uint64, _u64p]
        _lib = L
    return _lib


def _kt(keys: np.ndarray) -> int:
    if keys.dtype == np.float64:
        return KEY_F64
    if keys.dtype == np.uint64:
        return KEY_U64
    raise TypeError("keys must be float64 or uint64")


def _bits(keys: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(keys).view(np.uint64)


def _p64(a):
    return a.ctypes.data_as(_u64p)


def _p32(a):
    return None if a is None else a.ctypes.data_as(_u32p)


def root_floor(n: int, p: int, q: int) -> int:
    """Largest m with m^q <= n^p."""
    return int(lib().orc_root_floor(n, p, q))


def params(n: int, policy: Policy = None):
    P = policy or paper_policy()
    return tuple(max(1, root_floor(n, num, P.den)) if i < 2 else root_floor(n, num, P.den)
                 for i, num in enumerate((P.a_num, P.b_num, P.c_num, P.d_num)))


def splitmix64_mix(z: int) -> int:
    return int(lib().orc_splitmix64_mix(z & (2**64 - 1)))


def sample_indices(seed: int, depth: int, start: int, n: int, alpha: int) -> np.ndarray:
    L = lib()
    st = L.orc_sample_state(seed, depth, start, n)
    return np.array([L.orc_sample_index(st, j, n) for j in range(alpha)], dtype=np.uint64)


def bins(kt: int, lo_bits: int, hi_bits: int, beta: int, xs_bits: np.ndarray):
    """bin() of each key (raw bits) for the model over [lo, hi]; None if degenerate."""
    xs = np.ascontiguousarray(xs_bits, dtype=np.uint64)
    out = np.empty_like(xs)
    rc = lib().orc_bins(kt, lo_bits, hi_bits, beta, _p64(xs), xs.size, _p64(out))
    return None if rc else out


def std_sort(keys: np.ndarray, vals: np.ndarray = None):
    """Standard-Sort (stable merge sort) -> new arrays."""
    k = _bits(keys).copy()
    v = None if vals is None else np.ascontiguousarray(vals, dtype=np.uint32).copy()
    rc = lib().orc_std_sort(_p64(k), _p32(v), k.size, _kt(keys))
    if rc:
        raise RuntimeError("orc_std_sort failed: %d" % rc)
    return k.view(keys.dtype), v


def sort(keys: np.ndarray, vals: np.ndarray = None, seed: int = 0, policy: Policy = None,
         with_stats: bool = False):
    """PCF Learned Sort of a copy of keys (and vals, stably).

    Returns (sorted_keys, sorted_vals_or_None[, stats_dict]).  Raises
    ValueError on NaN keys."""
    P = policy or paper_policy()
    k = _bits(keys).copy()
    v = None if vals is None else np.ascontiguousarray(vals, dtype=np.uint32).copy()
    st = Stats()
    rc = lib().orc_sort(_p64(k), _p32(v), k.size, _kt(keys), seed, ctypes.byref(P),
                        ctypes.byref(st))
    if rc == ERR_NAN:
        raise ValueError("NaN key")
    if rc:
        raise RuntimeError("orc_sort failed: %d" % rc)
    out = (k.view(keys.dtype), v)
    return out + (st.as_dict(),) if with_stats else out


def level0(keys: np.ndarray, vals: np.ndarray = None, seed: int = 0, policy: Policy = None):
    """Level-0 intermediates of Learned-Sort: dict with alpha..delta, lo/hi
    bits, status, sample_idx, b, T, counts and the bucketed keys/vals."""
    P = policy or paper_policy()
    n = keys.size
    alpha, beta, gamma, delta = params(n, P)
    k = _bits(keys).copy()
    v = None if vals is None else np.ascontiguousarray(vals, dtype=np.uint32).copy()
    p6 = np.zeros(6, dtype=np.uint64)
    sidx = np.zeros(alpha, dtype=np.uint64)
    b = np.zeros(beta + 1, dtype=np.uint64)
    T = np.zeros(beta + 1, dtype=np.uint64)
    counts = np.zeros(gamma + 1, dtype=np.uint64)
    status = ctypes.c_int(0)
    rc = lib().orc_level0(_p64(k), _p32(v), n, _kt(keys), seed, ctypes.byref(P), _p64(p6),
                          _p64(sidx), _p64(b), _p64(T), _p64(counts), ctypes.byref(status))
    if rc:
        raise RuntimeError("orc_level0 failed: %d" % rc)
    return dict(alpha=int(p6[0]), beta=int(p6[1]), gamma=int(p6[2]), delta=int(p6[3]),
                lo_bits=int(p6[4]), hi_bits=int(p6[5]), status=status.value,
                sample_idx=sidx, b=b, T=T, counts=counts, keys=k.view(keys.dtype), vals=v)


def bucket_sizes(keys: np.ndarray, seed: int, alpha: int, beta: int, gamma: int,
                 model: int = MODEL_PCF, range_mode: int = 0):
    """One model-based bucketing (Alg. 1 + Sec. 3.3, or the spline model of
    App. A.5) with alpha, beta, gamma given, as in the experiment of Sec. 4.2:
    (bucket sizes |c_0|..|c_gamma|, status) with status 0 bucketed, 1 single
    value, 2 degenerate range."""
    k = _bits(keys).copy()
    counts = np.zeros(gamma + 1, dtype=np.uint64)
    status = ctypes.c_int(0)
    rc = lib().orc_bucket_sizes(_p64(k), k.size, _kt(keys), seed, alpha, beta, gamma, model,
                                range_mode, _p64(counts), ctypes.byref(status))
    if rc:
        raise RuntimeError("orc_bucket_sizes failed: %d" % rc)
    return counts, status.value


def insertion_sort(keys: np.ndarray, vals: np.ndarray = None):
    """Brute-force stable insertion sort (pin only)."""
    k = _bits(keys).copy()
    v = None if vals is None else np.ascontiguousarray(vals, dtype=np.uint32).copy()
    lib().brute_insertion_sort(_p64(k), _p32(v), k.size, _kt(keys))
    return k.view(keys.dtype), v


def brute_cumulative_counts(sample_bins: np.ndarray, beta: int) -> np.ndarray:
    sb = np.ascontiguousarray(sample_bins, dtype=np.uint64)
    out = np.zeros(beta + 1, dtype=np.uint64)
    lib().brute_cumulative_counts(_p64(sb), sb.size, beta, _p64(out))
    return out

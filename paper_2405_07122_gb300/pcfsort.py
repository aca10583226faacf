"""Python binding of the C ABI in include/pcfsort.h (argument marshalling only).

Every step of the sort runs in the CUDA library libpcfsort.so; this module
only turns torch tensors / numpy arrays into pointers and sizes.  Importing
it raises if the library has not been built (there is no CPU fallback).

Keys: torch.float64 tensors (KEY_F64) or torch.int64 / torch.uint64 tensors
holding unsigned 64-bit keys (KEY_U64, pass key_type="u64").  Values:
torch.int32 / torch.uint32 tensors (copied bit for bit).
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpcfsort.so")

KEY_F64, KEY_U64 = 0, 1
STAGES = ("range", "sample_pcf", "hist1_scan", "scatter1", "hist2_scan", "scatter2",
          "leaf", "fallback")
STATUS = {0: "ok", 1: "invalid argument", 2: "invalid key (NaN)", 3: "out of memory",
          4: "CUDA error", 5: "device wait timed out", 6: "internal error"}


class PcfError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__("pcfsort: %s%s" % (STATUS.get(code, str(code)), (": " + msg) if msg else ""))
        self.code = code


MODELS = {"pcf": 0, "spline": 1}
RANGES = {"array": 0, "sample": 1}


class Policy(ctypes.Structure):
    _fields_ = [("a_num", ctypes.c_uint32), ("b_num", ctypes.c_uint32),
                ("c_num", ctypes.c_uint32), ("d_num", ctypes.c_uint32),
                ("den", ctypes.c_uint32), ("model", ctypes.c_uint32),
                ("tau", ctypes.c_uint64), ("range_mode", ctypes.c_uint32)]


class Tuning(ctypes.Structure):
    _fields_ = [("max_digit_bits", ctypes.c_uint32), ("tile_log2", ctypes.c_uint32),
                ("leaf_cap", ctypes.c_uint32), ("leaf_mode", ctypes.c_uint32)]


class CallStats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_uint64), ("global_passes", ctypes.c_uint64),
                ("leaf_buckets", ctypes.c_uint64), ("fallback_buckets", ctypes.c_uint64),
                ("fallback_keys", ctypes.c_uint64), ("bytes_moved", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_uint64), ("fallback_splits", ctypes.c_uint64),
                ("guard_buckets", ctypes.c_uint64), ("guard_keys", ctypes.c_uint64),
                ("bucketings", ctypes.c_uint64)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


_lib = None
_vp = ctypes.c_void_p
_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libpcfsort.so is not built (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "pcf_ctx_create": [ctypes.POINTER(_vp), ctypes.c_int],
            "pcf_ctx_destroy": [_vp],
            "pcf_ctx_set_policy": [_vp, ctypes.POINTER(Policy)],
            "pcf_ctx_set_tuning": [_vp, ctypes.POINTER(Tuning)],
            "pcf_ctx_get_tuning": [_vp, ctypes.POINTER(Tuning)],
            "pcf_ctx_reserve": [_vp, _u64, ctypes.c_int],
            "pcf_ctx_last_stats": [_vp, ctypes.POINTER(CallStats)],
            "pcf_ctx_enable_timing": [_vp, ctypes.c_int],
            "pcf_ctx_stage_ms": [_vp, ctypes.POINTER(ctypes.c_float)],
            "pcf_sort_keys": [_vp, _vp, _vp, _u64, ctypes.c_int, _u64, _vp],
            "pcf_sort_pairs": [_vp, _vp, _vp, _vp, _vp, _u64, ctypes.c_int, _u64, _vp],
            "pcf_sort_segmented": [_vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_u64), _u32,
                                   ctypes.c_int, _u64, _vp],
            "pcf_sort_keys_host": [_vp, _vp, _u64, ctypes.c_int, _u64, _vp],
            "pcf_sort_keys_host_batch": [_vp, _vp, _vp, _u32, ctypes.c_int, _u64, _vp],
            "pcf_copy_bandwidth": [_vp, _vp, _vp, _u64, _u32, _vp, ctypes.POINTER(ctypes.c_double)],
            "pcf_bucket_sizes": [_vp, _vp, _vp, _u32, ctypes.c_int, _u64, _u64, _u64, _u64, _vp,
                                 _vp, _vp],
            "pcf_sort_segmented_static": [_vp, _vp, _vp, _u32, _u64, ctypes.c_int, _u64, _vp],
            "pcf_graph_create": [ctypes.POINTER(_vp), _vp, _vp, _vp, _vp, _vp,
                                 ctypes.POINTER(_u64), _u32, ctypes.c_int, _u64, _vp],
            "pcf_graph_launch": [_vp, _vp, ctypes.POINTER(ctypes.c_int)],
            "pcf_graph_info": [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_u64),
                               ctypes.POINTER(_u64)],
            "pcf_graph_destroy": [_vp],
            "pcf_sort_segmented_dev": [_vp, _vp, _vp, _vp, _vp, _vp, _u32, _u64, ctypes.c_int,
                                       _u64, _vp],
            "pcf_ctx_sync": [_vp, _vp],
            "pcf_workspace_bytes": [_vp, _u64, _u32, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(_u64)],
            "pcf_ctx_workspace_held": [_vp, ctypes.POINTER(_u64)],
            "pcf_debug_scan": [_vp, _vp, _u64, _u32, _u64, _vp],
            "pcf_debug_level0": [_vp, _vp, _u64, ctypes.c_int, _u64, ctypes.POINTER(_u64),
                                 ctypes.POINTER(_u32), _u64],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.pcf_status_string.restype = ctypes.c_char_p
        L.pcf_status_string.argtypes = [ctypes.c_int]
        L.pcf_last_cuda_error.restype = ctypes.c_char_p
        L.pcf_last_cuda_error.argtypes = [_vp]
        L.pcf_version.restype = _u32
        L.pcf_version.argtypes = []
        L.pcf_debug_bins_host.restype = ctypes.c_int
        L.pcf_debug_bins_host.argtypes = [_u32, _u64, _u64, _u32, _vp, _u64, _vp, _vp]
        L.pcf_debug_root_floor.restype = _u64
        L.pcf_debug_root_floor.argtypes = [_u64, _u32, _u32]
        L.pcf_debug_sample_index.restype = _u64
        L.pcf_debug_sample_index.argtypes = [_u64, _u64, _u64, _u64, _u64]
        L.pcf_debug_fail_alloc_after.restype = None
        L.pcf_debug_fail_alloc_after.argtypes = [ctypes.c_int64]
        _lib = L
    return _lib


def _kt(key_type):
    if key_type in ("f64", KEY_F64):
        return KEY_F64
    if key_type in ("u64", KEY_U64):
        return KEY_U64
    raise ValueError("key_type must be 'f64' or 'u64'")


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


class Context:
    """A pcf_ctx: owns device workspace; one per host thread."""

    def __init__(self, device: int = 0, policy=None, tuning=None):
        self._h = _vp()
        rc = lib().pcf_ctx_create(ctypes.byref(self._h), device)
        if rc:
            raise PcfError(rc)
        self.device = device
        if policy is not None:
            self.set_policy(*policy)
        if tuning is not None:
            self.set_tuning(**tuning)

    def close(self):
        if self._h:
            lib().pcf_ctx_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc:
            raise PcfError(rc, lib().pcf_last_cuda_error(self._h).decode())

    def set_policy(self, a_num=3, b_num=3, c_num=3, d_num=3, den=4, tau=100, model="pcf",
                   range_mode="array"):
        """alpha..delta = floor(n^(x_num/den)), tau, the CDF model ("pcf",
        Sec. 3.3, or "spline", App. A.5) and the range the bins span
        ("array": the (sub)array's, "sample": the alpha samples')."""
        m = MODELS[model] if isinstance(model, str) else int(model)
        r = RANGES[range_mode] if isinstance(range_mode, str) else int(range_mode)
        self._check(lib().pcf_ctx_set_policy(self._h, ctypes.byref(
            Policy(a_num=a_num, b_num=b_num, c_num=c_num, d_num=d_num, den=den, model=m,
                   tau=tau, range_mode=r))))

    def set_tuning(self, max_digit_bits=0, tile_log2=0, leaf_cap=0, leaf_mode=0):
        """leaf_mode: 1 = block-local sort of each on-chip bucket (keys only),
        2 = the remaining Learned-Sort steps on chip; 0 keeps the current."""
        self._check(lib().pcf_ctx_set_tuning(self._h, ctypes.byref(
            Tuning(max_digit_bits, tile_log2, leaf_cap, leaf_mode))))

    def tuning(self):
        t = Tuning()
        self._check(lib().pcf_ctx_get_tuning(self._h, ctypes.byref(t)))
        return dict(max_digit_bits=t.max_digit_bits, tile_log2=t.tile_log2, leaf_cap=t.leaf_cap,
                    leaf_mode=t.leaf_mode)

    def reserve(self, n_total: int, pairs: bool = False):
        self._check(lib().pcf_ctx_reserve(self._h, n_total, 1 if pairs else 0))

    def last_stats(self):
        s = CallStats()
        self._check(lib().pcf_ctx_last_stats(self._h, ctypes.byref(s)))
        return s.as_dict()

    def enable_timing(self, on=True):
        self._check(lib().pcf_ctx_enable_timing(self._h, 1 if on else 0))

    def stage_ms(self):
        a = (ctypes.c_float * 8)()
        self._check(lib().pcf_ctx_stage_ms(self._h, a))
        return dict(zip(STAGES, list(a)))

    # -- sorts ------------------------------------------------------------
    def sort_keys(self, keys_in, keys_out=None, key_type=None, seed=0, stream=None):
        """Sorts a 1-D CUDA tensor of keys into keys_out (default: in place)."""
        kt = _kt(key_type or ("f64" if str(keys_in.dtype) == "torch.float64" else "u64"))
        out = keys_in if keys_out is None else keys_out
        self._check(lib().pcf_sort_keys(self._h, keys_in.data_ptr(), out.data_ptr(),
                                        keys_in.numel(), kt, seed, _stream_ptr(stream)))
        return out

    def sort_pairs(self, keys_in, vals_in, keys_out=None, vals_out=None, key_type=None, seed=0,
                   stream=None):
        kt = _kt(key_type or ("f64" if str(keys_in.dtype) == "torch.float64" else "u64"))
        ko = keys_in if keys_out is None else keys_out
        vo = vals_in if vals_out is None else vals_out
        self._check(lib().pcf_sort_pairs(self._h, keys_in.data_ptr(), vals_in.data_ptr(),
                                         ko.data_ptr(), vo.data_ptr(), keys_in.numel(), kt,
                                         seed, _stream_ptr(stream)))
        return ko, vo

    def sort_segmented(self, keys_in, offsets, vals_in=None, keys_out=None, vals_out=None,
                       key_type=None, seed=0, stream=None):
        """offsets: host sequence of S+1 segment boundaries."""
        kt = _kt(key_type or ("f64" if str(keys_in.dtype) == "torch.float64" else "u64"))
        offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.uint64))
        S = offs.size - 1
        ko = keys_in if keys_out is None else keys_out
        vo = vals_in if vals_out is None else vals_out
        self._check(lib().pcf_sort_segmented(
            self._h, keys_in.data_ptr(), None if vals_in is None else vals_in.data_ptr(),
            ko.data_ptr(), None if vo is None else vo.data_ptr(),
            offs.ctypes.data_as(ctypes.POINTER(_u64)), S, kt, seed, _stream_ptr(stream)))
        return ko, vo

    def sort_segmented_dev(self, keys_in, offsets_dev, vals_in=None, keys_out=None, vals_out=None,
                           key_type=None, seed=0, stream=None):
        """offsets_dev: DEVICE tensor of S+1 segment boundaries (8-byte
        integers on the keys' device), read by the library on `stream`."""
        kt = _kt(key_type or ("f64" if str(keys_in.dtype) == "torch.float64" else "u64"))
        if (offsets_dev.element_size() != 8 or not offsets_dev.is_contiguous()
                or offsets_dev.device != keys_in.device or offsets_dev.numel() < 1
                or str(offsets_dev.dtype) not in ("torch.int64", "torch.uint64")):
            raise ValueError("offsets_dev: a contiguous 8-byte integer tensor on the keys' device")
        ko = keys_in if keys_out is None else keys_out
        vo = vals_in if vals_out is None else vals_out
        n_cap = min(keys_in.numel(), ko.numel())
        if vals_in is not None:
            n_cap = min(n_cap, vals_in.numel(), vo.numel())
        self._check(lib().pcf_sort_segmented_dev(
            self._h, keys_in.data_ptr(), None if vals_in is None else vals_in.data_ptr(),
            ko.data_ptr(), None if vo is None else vo.data_ptr(), offsets_dev.data_ptr(),
            offsets_dev.numel() - 1, n_cap, kt, seed, _stream_ptr(stream)))
        return ko, vo

    def sync(self, stream=None):
        """Waits for `stream` and returns the last sort's status code."""
        return int(lib().pcf_ctx_sync(self._h, _stream_ptr(stream)))

    def workspace_held(self):
        """Device bytes the context holds."""
        v = _u64(0)
        self._check(lib().pcf_ctx_workspace_held(self._h, ctypes.byref(v)))
        return int(v.value)

    def workspace_bytes(self, n_total, n_arrays=1, key_type="f64", pairs=False):
        """Upper bound on the workspace a sort of n_total keys in n_arrays
        arrays grows this context to (its policy and tuning)."""
        return workspace_bytes(n_total, n_arrays, key_type, pairs, ctx=self)

    def sort_keys_host(self, host_keys, key_type=None, seed=0, stream=None):
        """End-to-end: sorts a host tensor/array (ideally pinned) in place."""
        if hasattr(host_keys, "data_ptr"):
            ptr, n = host_keys.data_ptr(), host_keys.numel()
            kt = _kt(key_type or ("f64" if str(host_keys.dtype) == "torch.float64" else "u64"))
        else:
            ptr, n = host_keys.ctypes.data, host_keys.size
            kt = _kt(key_type or ("f64" if host_keys.dtype == np.float64 else "u64"))
        self._check(lib().pcf_sort_keys_host(self._h, ptr, n, kt, seed, _stream_ptr(stream)))
        return host_keys

    def sort_keys_host_batch(self, host_arrays, key_type=None, seed=0, stream=None):
        """End-to-end for several host tensors/arrays (ideally pinned), each
        sorted in place (array i with seed + i); copies overlap the sorts."""
        ptrs, ns, kts = [], [], set()
        for h in host_arrays:
            if hasattr(h, "data_ptr"):
                ptrs.append(h.data_ptr())
                ns.append(h.numel())
                kts.add("f64" if str(h.dtype) == "torch.float64" else "u64")
            else:
                ptrs.append(h.ctypes.data)
                ns.append(h.size)
                kts.add("f64" if h.dtype == np.float64 else "u64")
        if not ptrs:
            return host_arrays
        if key_type is None and len(kts) != 1:
            raise ValueError("arrays of different key types")
        kt = _kt(key_type or kts.pop())
        P = (ctypes.c_void_p * len(ptrs))(*ptrs)
        N = (_u64 * len(ns))(*ns)
        self._check(lib().pcf_sort_keys_host_batch(self._h, P, N, len(ptrs), kt, seed,
                                                   _stream_ptr(stream)))
        return host_arrays

    def bucket_sizes(self, keys, offsets, alpha, beta, gamma, key_type=None, seed=0,
                     counts_out=None, stream=None):
        """Level-0 bucketing only (alpha, beta, gamma given) of the arrays
        keys[offsets[s]:offsets[s+1]] of a CUDA tensor: numpy u64 array of
        max_j |c_j| per array; counts_out (CUDA int32/uint32 tensor of
        S * (gamma + 1)) receives the bucket sizes when given."""
        offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.uint64))
        S = offs.size - 1
        kt = _kt(key_type or ("f64" if str(keys.dtype) == "torch.float64" else "u64"))
        out = np.zeros(S, dtype=np.uint64)
        self._check(lib().pcf_bucket_sizes(
            self._h, keys.data_ptr(), offs.ctypes.data_as(ctypes.POINTER(_u64)), S, kt, seed,
            alpha, beta, gamma, None if counts_out is None else counts_out.data_ptr(),
            out.ctypes.data_as(ctypes.POINTER(_u64)), _stream_ptr(stream)))
        return out

    def copy_bandwidth(self, src, dst, reps=10, stream=None):
        """GB/s (read + written) of the library's 16-byte copy over two CUDA
        tensors of equal byte size."""
        nbytes = src.numel() * src.element_size()
        out = ctypes.c_double(0.0)
        self._check(lib().pcf_copy_bandwidth(self._h, src.data_ptr(), dst.data_ptr(),
                                             nbytes - nbytes % 16, reps, _stream_ptr(stream),
                                             ctypes.byref(out)))
        return out.value

    # -- self-test hooks ----------------------------------------------------
    def debug_scan(self, data_u32, withhold_tile=0xFFFFFFFF, spin_limit=0, stream=None):
        rc = lib().pcf_debug_scan(self._h, data_u32.data_ptr(), data_u32.numel(), withhold_tile,
                                  spin_limit, _stream_ptr(stream))
        return rc

    def debug_level0(self, keys, key_type=None, seed=0, T_cap=1 << 22):
        kt = _kt(key_type or ("f64" if str(keys.dtype) == "torch.float64" else "u64"))
        p8 = (_u64 * 8)()
        T = np.zeros(T_cap, dtype=np.uint32)
        self._check(lib().pcf_debug_level0(self._h, keys.data_ptr(), keys.numel(), kt, seed, p8,
                                           T.ctypes.data_as(ctypes.POINTER(_u32)), T_cap))
        p = [int(v) for v in p8]
        out = dict(alpha=p[0], beta=p[1], gamma=p[2], delta=p[3], lo_bits=p[4], hi_bits=p[5],
                   status=p[6])
        out["T"] = T[: p[1] + 1].copy() if p[6] == 0 else None
        return out


# -- host copies of device functions (CPU self-checks) -------------------------
class SortGraph:
    """A pcf_graph: the segmented sort of fixed buffers captured in a CUDA
    graph.  Creating it sorts keys_in into keys_out once (as
    Context.sort_segmented would, out of place); launch() sorts their
    current contents again, by a graph replay when the data takes the
    recorded plan, else without the graph.  The tensors must outlive it."""

    def __init__(self, ctx, keys_in, offsets, keys_out, vals_in=None, vals_out=None,
                 key_type=None, seed=0, stream=None):
        kt = _kt(key_type or ("f64" if str(keys_in.dtype) == "torch.float64" else "u64"))
        offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.uint64))
        self._h = _vp()
        self._keep = (keys_in, keys_out, vals_in, vals_out)
        rc = lib().pcf_graph_create(
            ctypes.byref(self._h), ctx._h, keys_in.data_ptr(),
            None if vals_in is None else vals_in.data_ptr(), keys_out.data_ptr(),
            None if vals_out is None else vals_out.data_ptr(),
            offs.ctypes.data_as(ctypes.POINTER(_u64)), offs.size - 1, kt, seed,
            _stream_ptr(stream))
        if rc:
            raise PcfError(rc)

    def launch(self, stream=None):
        """Sorts again; returns True when the graph replay did the sort."""
        rep = ctypes.c_int(0)
        rc = lib().pcf_graph_launch(self._h, _stream_ptr(stream), ctypes.byref(rep))
        if rc:
            raise PcfError(rc)
        return bool(rep.value)

    def info(self):
        cap, rep, eag = ctypes.c_int(0), _u64(0), _u64(0)
        rc = lib().pcf_graph_info(self._h, ctypes.byref(cap), ctypes.byref(rep), ctypes.byref(eag))
        if rc:
            raise PcfError(rc)
        return {"captured": bool(cap.value), "replays": rep.value, "eager_runs": eag.value}

    def close(self):
        if self._h:
            lib().pcf_graph_destroy(self._h)
            self._h = _vp()
        self._keep = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bins_host(kt, lo_bits, hi_bits, beta, xs_bits):
    xs = np.ascontiguousarray(xs_bits, dtype=np.uint64)
    out = np.empty(xs.size, dtype=np.uint32)
    fast = np.empty(xs.size, dtype=np.uint8)
    rc = lib().pcf_debug_bins_host(kt, lo_bits, hi_bits, beta, xs.ctypes.data, xs.size,
                                   out.ctypes.data, fast.ctypes.data)
    return None if rc else (out, fast)


STATIC_MAX_ARRAY_KEYS = 1024
STATIC_MAX_ARRAYS = 65536
STATIC_MAX_KEYS = 1 << 22


def sort_segmented_static(keys_in, offsets_dev, n_total, keys_out=None, key_type=None, seed=0,
                          stream=None):
    """pcf_sort_segmented_static: allocation-free sort of S small arrays.
    offsets_dev: CUDA int64/uint64 tensor of S+1 boundaries; n_total = its
    last value.  Calls on one device must not overlap."""
    kt = _kt(key_type or ("f64" if str(keys_in.dtype) == "torch.float64" else "u64"))
    ko = keys_in if keys_out is None else keys_out
    # the C call trusts n_total and the buffers: check them here
    for name, t in (("keys_in", keys_in), ("keys_out", ko), ("offsets_dev", offsets_dev)):
        if t.element_size() != 8 or not t.is_contiguous() or not t.is_cuda:
            raise ValueError(name + ": a contiguous 8-byte CUDA tensor")
    if str(offsets_dev.dtype) not in ("torch.int64", "torch.uint64"):
        raise ValueError("offsets_dev: int64 or uint64")
    import torch
    dev = torch.cuda.current_device()
    if any(t.device.index != dev for t in (keys_in, ko, offsets_dev)):
        raise ValueError("every tensor on the current CUDA device")
    if offsets_dev.numel() < 1 or not 0 <= n_total <= min(keys_in.numel(), ko.numel()):
        raise ValueError("n_total must fit the key buffers")
    rc = lib().pcf_sort_segmented_static(keys_in.data_ptr(), ko.data_ptr(),
                                         offsets_dev.data_ptr(), offsets_dev.numel() - 1,
                                         n_total, kt, seed, _stream_ptr(stream))
    if rc:
        raise PcfError(rc)
    return ko


def workspace_bytes(n_total, n_arrays=1, key_type="f64", pairs=False, ctx=None):
    """pcf_workspace_bytes: upper bound on the device workspace of a sort of
    n_total keys in n_arrays arrays (ctx's policy and tuning, else the
    defaults)."""
    v = _u64(0)
    rc = lib().pcf_workspace_bytes(None if ctx is None else ctx._h, n_total, n_arrays,
                                   _kt(key_type), 1 if pairs else 0, ctypes.byref(v))
    if rc:
        raise PcfError(rc)
    return int(v.value)


def root_floor_host(n, p, q):
    return int(lib().pcf_debug_root_floor(n, p, q))


def sample_index_host(seed, depth, start, n, j):
    return int(lib().pcf_debug_sample_index(seed, depth, start, n, j))


def version():
    return int(lib().pcf_version())

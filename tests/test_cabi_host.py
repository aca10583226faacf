"""C-ABI library checks that need no GPU: it builds, loads, exports every
symbol the header declares, and its host-compiled copies of the device
arithmetic (bin function, parameters, sampler) agree with the oracle."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2405_07122_gb300 import build as pcf_build
from paper_2405_07122_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    pcf_build.build()
    from paper_2405_07122_gb300 import pcfsort
    return pcfsort


def _declared(*headers):
    names = set()
    for h in headers:
        hdr = open(os.path.join(ROOT, "include", h)).read()
        names |= set(re.findall(r"\b(pcf_[a-z0-9_]+)\s*\(", hdr))
    return names


def test_exports_every_declared_symbol(P):
    headers = sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h"))
    assert headers == ["pcfsort.h", "pcfsort_debug.h"]
    declared = _declared(*headers)
    assert {"pcf_sort_keys", "pcf_sort_pairs", "pcf_sort_segmented", "pcf_sort_segmented_dev",
            "pcf_workspace_bytes", "pcf_ctx_sync", "pcf_status_string"} <= declared
    L = P.lib()
    for name in sorted(declared):
        assert hasattr(L, name), name
    assert P.version() >= 100
    # the self-test hooks are declared in the debug header, not the interface
    assert all(n.startswith("pcf_debug_") for n in _declared("pcfsort_debug.h"))
    assert not any(n.startswith("pcf_debug_") for n in _declared("pcfsort.h"))


def test_every_export_is_declared(P):
    # every pcf_* function the library exports has a declaration in include/
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", P.LIB_PATH], capture_output=True,
                         text=True)
    if out.returncode:
        pytest.skip("nm not available")
    exported = {l.split()[-1] for l in out.stdout.splitlines()
                if l.split() and l.split()[-1].startswith("pcf_")}
    assert exported, out.stdout[:200]
    assert exported <= _declared("pcfsort.h", "pcfsort_debug.h"), exported - _declared(
        "pcfsort.h", "pcfsort_debug.h")


def test_workspace_bound_on_the_host(P):
    # the bound follows the planner on the host: the key-sized scratch of 14
    # bytes per key (18 with values) is a floor, and it grows with n
    last = 0
    for n in (1, 1000, 10**5, 10**6, 10**8):
        b = P.workspace_bytes(n)
        assert b >= 14 * n and b > last
        assert P.workspace_bytes(n, pairs=True) >= 18 * n
        last = b
    assert P.workspace_bytes(0) == 0
    assert P.workspace_bytes(10**6, n_arrays=1000) > 0
    with pytest.raises(P.PcfError):
        P.workspace_bytes(10**6, n_arrays=0)
    with pytest.raises(P.PcfError):
        P.workspace_bytes(2**32)


def test_status_strings(P):
    L = P.lib()
    for code in range(7):
        assert L.pcf_status_string(code)


@pytest.mark.parametrize("n", [2, 99, 100, 1000, 31622, 10**6, 10**8, 2**28, 2**32 - 1])
def test_root_floor_matches_oracle(P, n):
    for p, q in [(3, 4), (1, 2), (2, 3), (1, 4), (4, 4)]:
        assert P.root_floor_host(n, p, q) == oracle.root_floor(n, p, q)


def test_sample_index_matches_oracle(P):
    for (seed, depth, start, n) in [(0, 0, 0, 10**6), (7, 2, 12345, 517), (2**63, 1, 9, 2**28)]:
        ref = oracle.sample_indices(seed, depth, start, n, 64)
        got = [P.sample_index_host(seed, depth, start, n, j) for j in range(64)]
        assert np.array_equal(ref, np.array(got, dtype=np.uint64))


def _models(seed):
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for kind in ("normal", "uniform", "lognormal", "wide", "clustered", "clustered_neg", "narrow",
                 "binade_cross", "dyadic", "u64", "u64wide", "u64small", "subnormal", "zerocross"):
        if kind == "normal":
            x = g.standard_normal(5000) * 10.0 ** g.uniform(-5, 5)
        elif kind == "uniform":
            x = g.random(5000)
        elif kind == "lognormal":
            x = g.lognormal(0, 2, 5000)
        elif kind == "wide":
            x = np.concatenate([g.standard_normal(2500) * 1e300, g.standard_normal(2500) * 1e-300])
        elif kind == "clustered":
            # one sign and exponent for all keys (the models' fixed-shift mode)
            x = 1e10 + g.random(5000) * 1e-3
        elif kind == "clustered_neg":
            x = -(1e10 + g.random(5000) * 1e-3)
        elif kind == "narrow":
            x = 1.0 + g.random(5000) * 2.0 ** -30
        elif kind == "binade_cross":
            x = 2.0 + (g.random(5000) - 0.5) * 2.0 ** -20
        elif kind == "dyadic":
            x = g.integers(-512, 512, 5000).astype(np.float64) / 8.0
        elif kind == "u64":
            x = g.integers(0, 2**40, 5000, dtype=np.uint64)
        elif kind == "u64wide":
            x = g.integers(0, 2**64 - 1, 5000, dtype=np.uint64, endpoint=True)
        elif kind == "u64small":
            x = g.integers(100, 130, 5000, dtype=np.uint64)
        elif kind == "subnormal":
            x = g.integers(0, 1000, 5000).astype(np.float64) * 5e-324
        else:
            x = np.concatenate([g.standard_normal(4990), [0.0, -0.0] * 5])
        for beta in (1, 7, 181, 31622, 10**6, 2**21):
            out.append((kind, x, beta))
    return out


@pytest.mark.parametrize("seed", range(3))
def test_bin_fast_path_equals_oracle(P, seed):
    """The kernels' certified integer fast path + exact fallback gives the
    oracle's binary64 bin for every key (same reading of Sec. 3.3)."""
    for kind, x, beta in _models(seed):
        kt = oracle.KEY_F64 if x.dtype == np.float64 else oracle.KEY_U64
        bits = x.view(np.uint64) if kt == 0 else x
        order = np.argsort(x, kind="stable")
        lo = int(bits[order[0]])
        hi = int(bits[order[-1]])
        if kt == 0:  # total-order extremes (-0 < +0)
            s = sorted(bits.tolist(), key=lambda b: (b ^ 0xFFFFFFFFFFFFFFFF) if b >> 63 else b | (1 << 63))
            lo, hi = s[0], s[-1]
        ref = oracle.bins(kt, lo, hi, beta, bits)
        got = P.bins_host(kt, lo, hi, beta, bits)
        assert (ref is None) == (got is None), kind
        if ref is None:
            continue
        assert np.array_equal(ref.astype(np.uint32), got[0]), (kind, beta)


def test_bin_fast_path_rarely_falls_back(P):
    # on continuous data only the maximum key (which sits exactly at beta)
    # needs the exact binary64 sequence
    x = W.f64_keys("normal", 200000, 1)
    bits = x.view(np.uint64)
    lo, hi = int(bits[np.argmin(x)]), int(bits[np.argmax(x)])
    _, fast = P.bins_host(0, lo, hi, 10**6, bits)
    assert int((fast == 0).sum()) <= 2


def _boundary_keys_f64(lo, hi, beta, g, m=3000, spread=4):
    # keys at (an estimate of) the bin boundaries lo + k (hi - lo) / beta and
    # up to `spread` ulps either side, clipped to [lo, hi]
    k = g.integers(0, beta + 1, m)
    x0 = lo + k.astype(np.float64) * ((hi - lo) / beta)
    xs = [x0]
    up, dn = x0.copy(), x0.copy()
    for _ in range(spread):
        up = np.nextafter(up, np.inf)
        dn = np.nextafter(dn, -np.inf)
        xs += [up, dn]
    x = np.clip(np.concatenate(xs), lo, hi)
    return np.concatenate([[lo, hi], x])


@pytest.mark.parametrize("lo,hi,beta", [
    (-5.6, 5.7, 10**6), (0.0, 1.0, 31622), (1e-3, 7.5e3, 2**21), (-1e10, -1e10 + 1e-2, 181),
    (1.0, 1.0 + 2.0 ** -30, 1000), (-3.0, 3.0, 7), (2.0 ** -1000, 2.0 ** -990, 92681)])
def test_bin_fast_path_at_bin_boundaries(P, lo, hi, beta):
    """Keys within a few ulps of the boundaries, where the fixed-point fast
    path must notice the ambiguity and take the exact binary64 sequence:
    every bin equals the oracle's."""
    g = np.random.Generator(np.random.PCG64(beta))
    x = _boundary_keys_f64(lo, hi, beta, g)
    bits = x.view(np.uint64)
    lob, hib = int(np.float64(lo).view(np.uint64)), int(np.float64(hi).view(np.uint64))
    ref = oracle.bins(oracle.KEY_F64, lob, hib, beta, bits)
    got = P.bins_host(oracle.KEY_F64, lob, hib, beta, bits)
    assert ref is not None and got is not None
    assert np.array_equal(ref.astype(np.uint32), got[0])
    assert int((got[1] == 0).sum()) > 0  # the exact sequence was exercised


@pytest.mark.parametrize("lo,hi,beta", [(0, 2**40, 10**6), (10**18, 10**18 + 12345, 181),
                                        (0, 2**64 - 1, 2**21), (5, 2**33 + 7, 31622)])
def test_bin_fast_path_at_bin_boundaries_u64(P, lo, hi, beta):
    g = np.random.Generator(np.random.PCG64(beta + 1))
    k = g.integers(0, beta + 1, 3000).astype(object)
    centre = [lo + (int(kk) * (hi - lo)) // beta for kk in k]
    xs = [min(hi, max(lo, c + d)) for c in centre for d in range(-3, 4)] + [lo, hi]
    x = np.array(xs, dtype=np.uint64)
    ref = oracle.bins(oracle.KEY_U64, lo, hi, beta, x)
    got = P.bins_host(oracle.KEY_U64, lo, hi, beta, x)
    assert ref is not None and got is not None
    assert np.array_equal(ref.astype(np.uint32), got[0])


def test_binding_declares_every_function(P):
    # every function of include/pcfsort.h has a ctypes signature in the
    # binding (argument marshalling only, so a missing one would pass
    # arguments untyped)
    h = open(os.path.join(ROOT, "include", "pcfsort.h")).read()
    names = sorted(set(re.findall(r"\b(pcf_[a-z0-9_]+)\s*\(", h)))
    L = P.lib()
    assert names and all(getattr(L, n).argtypes is not None for n in names), \
        [n for n in names if getattr(L, n).argtypes is None]

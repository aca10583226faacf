"""Host-side admission, batching and the result pool of the served form
(no GPU)."""
import pytest

from paper_2405_07122_gb300.serve import Admission, Request, ResultPool


def req(i, n, kt="f64"):
    return Request(i, None, kt, n=n)


def test_memory_budget_and_fifo():
    a = Admission(mem_budget=8 * 1000, batch_keys=10**6)  # 8 B per key of result
    rs = [req(i, 400) for i in range(4)]
    for r in rs:
        a.submit(r)
    # 2 x 400 keys x 8 B = 6400 <= 8000; the third would exceed
    assert [r.rid for r in a.ready] == [0, 1]
    assert [r.rid for r in a.waiting] == [2, 3]
    b = a.take_batch()
    assert [r.rid for r in b] == [0, 1]
    a.complete(b)
    assert a.reserved == 2 * 400 * 8
    assert [r.rid for r in a.ready] == [2, 3]


def test_batches_share_a_key_type_and_fit():
    a = Admission(mem_budget=1 << 40, batch_keys=1000)
    for i, (n, kt) in enumerate([(600, "f64"), (300, "u64"), (300, "f64"), (200, "f64"),
                                 (100, "u64")]):
        a.submit(req(i, n, kt))
    b1 = a.take_batch()
    assert [r.rid for r in b1] == [0, 2]          # 600 + 300 f64; the 200 does not fit
    b2 = a.take_batch()
    assert [r.rid for r in b2] == [1, 4]          # the u64 requests
    b3 = a.take_batch()
    assert [r.rid for r in b3] == [3]
    assert a.take_batch() == []


def test_continuous_admission_as_memory_frees():
    a = Admission(mem_budget=8 * 1000, batch_keys=10**6)
    first = req(0, 1000)
    a.submit(first)
    late = req(1, 500)
    a.submit(late)                 # arrives while the first is on the GPU
    assert list(a.waiting) == [late]
    b = a.take_batch()
    a.complete(b)                  # the first finishes: the late one is admitted
    assert list(a.ready) == [late]


def test_rejects_oversized():
    a = Admission(mem_budget=1000, batch_keys=10)
    with pytest.raises(ValueError):
        a.submit(req(0, 11))
    p = Admission(mem_budget=1 << 40, batch_keys=10**6, pool=ResultPool(100))
    with pytest.raises(ValueError):   # larger than the whole pool
        p.submit(req(1, 101))


def test_pool_first_fit_and_coalescing():
    p = ResultPool(100)
    a, b, c = p.alloc(30), p.alloc(30), p.alloc(30)
    assert (a, b, c) == (0, 30, 60)
    assert p.alloc(20) is None and p.free_keys() == 10
    p.release(b, 30)
    assert p.alloc(40) is None          # 30 + 10 free, not adjacent
    p.release(a, 30)                    # merges with b's block: 60 at 0
    assert p.starts == [0, 90] and p.sizes == [60, 10]
    p.release(c, 30)                    # everything merges back
    assert p.starts == [0] and p.sizes == [100]
    assert p.alloc(100) == 0


def test_pool_admission_waits_for_release():
    # under memory pressure results hold the pool until the client lets
    # them go; completion alone frees nothing
    a = Admission(mem_budget=1 << 40, batch_keys=10**6, pool=ResultPool(1000))
    r0, r1, r2 = req(0, 600), req(1, 300), req(2, 500)
    for r in (r0, r1, r2):
        a.submit(r)
    assert [r.rid for r in a.ready] == [0, 1] and list(a.waiting) == [r2]
    assert (r0.slot, r1.slot) == (0, 600)
    b = a.take_batch()
    a.complete(b)
    assert list(a.waiting) == [r2]      # results still held
    a.release(r1)
    assert list(a.waiting) == [r2]      # 400 keys free, not 500
    a.release(r0)
    assert list(a.ready) == [r2] and r2.slot == 0
    a.release(r0)                        # a second release is a no-op
    assert a.reserved == 500 * 8

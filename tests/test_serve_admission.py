"""Host-side admission and batching of the served form (no GPU)."""
import pytest

from paper_2405_07122_gb300.serve import Admission, Request


def req(i, n, kt="f64"):
    return Request(i, None, kt, n=n)


def test_memory_budget_and_fifo():
    a = Admission(mem_budget=16 * 1000, batch_keys=10**6)  # 16 B per key reserved
    rs = [req(i, 400) for i in range(4)]
    for r in rs:
        a.submit(r)
    # 2 x 400 keys x 16 B = 12800 <= 16000; the third would exceed
    assert [r.rid for r in a.ready] == [0, 1]
    assert [r.rid for r in a.waiting] == [2, 3]
    b = a.take_batch()
    assert [r.rid for r in b] == [0, 1]
    a.complete(b)
    assert a.reserved == 2 * 400 * 16
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
    a = Admission(mem_budget=16 * 1000, batch_keys=10**6)
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

"""Host-side admission logic of the serving engine (no GPU)."""
from collections import deque

from paper_2505_24053_gb300.serve import Request, Scheduler, summarize


def _reqs(kinds):
    return deque(Request(i, 0.001 * i, camera=None, kind=k) for i, k in enumerate(kinds))


def test_fifo_and_slot_limit():
    s = Scheduler(n_slots=3, pair_budget=10**9, estimates={0: 10, 1: 20})
    q = _reqs([0, 1, 0, 1, 0])
    b = s.admit(q)
    assert [r.rid for r in b] == [0, 1, 2]
    assert [r.rid for r in q] == [3, 4]


def test_memory_budget_stops_admission_but_never_starves():
    s = Scheduler(n_slots=8, pair_budget=100, estimates={0: 60, 1: 30, 2: 500})
    q = _reqs([0, 1, 0, 2, 1])
    assert [r.rid for r in s.admit(q)] == [0, 1]      # 60 + 30; the next 60 does not fit
    assert [r.rid for r in s.admit(q)] == [2]         # 60; the 500 does not fit beside it
    assert [r.rid for r in s.admit(q)] == [3]         # alone even though above the budget
    assert [r.rid for r in s.admit(q)] == [4]


def test_observe_raises_estimates():
    s = Scheduler(n_slots=2, pair_budget=100, estimates={0: 10})
    r = Request(0, 0.0, None, kind=0)
    s.observe(r, 40)
    assert s.estimate(r) == 50
    s.observe(r, 8)
    assert s.estimate(r) == 50


def test_summary_percentiles():
    class Cam:
        width, height = 10, 10
    done = []
    for i in range(100):
        r = Request(i, 0.0, Cam())
        r.done_ms = float(i + 1)
        r.batch = i // 4
        done.append(r)
    s = summarize(done, 2.0)
    assert s["p50_ms"] == 50.0 and s["p99_ms"] == 99.0 and s["requests"] == 100
    assert s["req_per_s"] == 50.0 and s["batches"] == 25


def test_same_kind_batches_keep_arrival_order():
    s = Scheduler(n_slots=3, pair_budget=10**9, estimates={0: 10, 1: 10}, same_kind=True)
    q = _reqs([0, 1, 0, 1, 0, 0])
    assert [r.rid for r in s.admit(q)] == [0, 2, 4]   # the head's kind, in arrival order
    assert [r.rid for r in q] == [1, 3, 5]             # the others keep their order
    assert [r.rid for r in s.admit(q)] == [1, 3]
    assert [r.rid for r in s.admit(q)] == [5]
    assert not q

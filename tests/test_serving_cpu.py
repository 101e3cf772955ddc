"""Admission policy of the serving loop (host logic only)."""
from collections import deque
from types import SimpleNamespace

from paper_2512_02932_gb300.serving import ServingConfig, take_batch


def _req(i, n, rows, k):
    return SimpleNamespace(rid=i, n=n, rows=rows, k=k)


def _take(pending, scfg):
    return take_batch(pending, lambda r: r.n, lambda r: r.rows, lambda r: r.k, scfg)


def test_fifo_and_request_cap():
    scfg = ServingConfig(max_batch=3, prim_budget=10**9, row_budget=10**6, capacity=10**12, safety=1.0)
    pending = deque(_req(i, 10, 10, 10) for i in range(7))
    sizes = []
    while pending:
        b = _take(pending, scfg)
        assert [r.rid for r in b] == sorted(r.rid for r in b)
        sizes.append(len(b))
    assert sizes == [3, 3, 1]


def test_budgets_stop_admission_in_order():
    scfg = ServingConfig(max_batch=16, prim_budget=100, row_budget=50, capacity=1000, safety=1.0)
    pending = deque([_req(0, 60, 10, 10), _req(1, 30, 10, 10), _req(2, 30, 10, 10), _req(3, 5, 10, 10)])
    b = _take(pending, scfg)
    # 60 + 30 fits, the third would exceed 100 primitives: stop (no skipping)
    assert [r.rid for r in b] == [0, 1]
    pending = deque([_req(0, 1, 30, 10), _req(1, 1, 30, 10)])
    assert len(_take(pending, scfg)) == 1  # rows
    scfg2 = ServingConfig(max_batch=16, prim_budget=100, row_budget=50, capacity=100, safety=1.3)
    pending = deque([_req(0, 1, 1, 50), _req(1, 1, 1, 30)])
    assert len(_take(pending, scfg2)) == 1  # instances with margin: 65 + 39 > 100


def test_oversized_request_is_still_admitted_alone():
    scfg = ServingConfig(max_batch=4, prim_budget=10, row_budget=10, capacity=10, safety=1.0)
    pending = deque([_req(0, 1000, 1000, 1000), _req(1, 1, 1, 1)])
    assert [r.rid for r in _take(pending, scfg)] == [0]
    assert [r.rid for r in _take(pending, scfg)] == [1]

"""Admission order of the serving dispatcher (host logic, no GPU)."""

from concurrent.futures import Future

import numpy as np
import pytest

from paper_2412_08308_gb300.serve import Request, Server


def _server(policy, age_s, pending):
    srv = Server.__new__(Server)  # the order needs no device state
    srv.policy, srv.age_s, srv.pending = policy, age_s, pending
    return srv


def _req(length, arrival):
    return Request(np.zeros(length, dtype=np.uint8), arrival, Future())


def test_fifo_keeps_arrival_order():
    reqs = [_req(n, t) for n, t in [(900, 0.0), (30, 0.1), (400, 0.2)]]
    assert _server("fifo", 1.0, list(reqs))._order(5.0) == reqs


def test_sjf_shortest_first_and_aged_requests_ahead():
    a, b, c, d, e = (_req(n, t) for n, t in [(900, 0.0), (700, 0.5), (30, 1.2), (400, 1.3), (30, 1.4)])
    srv = _server("sjf", 1.0, [a, b, c, d, e])
    # at t = 1.6: a and b waited >= 1 s and go first, oldest first; then
    # the others by length (ties keep arrival order)
    assert srv._order(1.6) == [a, b, c, e, d]
    # nobody aged yet: pure shortest first
    assert srv._order(0.9) == [c, e, d, b, a]


def test_unknown_policy_rejected():
    with pytest.raises(ValueError):
        Server(None, np.zeros((20, 20), dtype=np.int8), policy="lifo")

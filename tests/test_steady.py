"""Host logic of steady.run_to_steady and its JSON-lines log (CPU).

A scripted stand-in for a batch supplies check values as functions of the
time level: a domain that meets the tolerance at once, one whose residual
decays and meets it later, one that never does, and one whose check values
become non-finite.  run_to_steady must report, for each domain, the first
chunk boundary at which the tolerance holds.  It must mark the blown-up
domain, stop once nothing is left to wait for (or at max_steps), and log one
consistent JSON line per call.
"""
import io
import json
import math
from types import SimpleNamespace

import numpy as np
import pytest

from paper_1003_0282_gb300 import steady


class ScriptedBatch:
    def __init__(self, rules, cells=(1000, 2000, 3000, 4000)):
        self.problems = [SimpleNamespace(cells=c) for c in cells[:len(rules)]]
        self.rules = rules
        self.time = 0
        self.calls = []

    def step(self, n):
        self.calls.append(n)
        self.time += n

    def residuals(self, allow_nonfinite=False):
        assert allow_nonfinite
        return np.array([rule(self.time) for rule in self.rules], dtype=np.float64)


def fast(t):
    return (1e-9, 100.0, 0.5)


def decaying(t):  # 1e-3 exp(-t / 2000) meets 1e-7 at t = 2000 ln 1e4 = 18421
    return (1e-3 * math.exp(-t / 2000.0), 200.0, -0.25)


def stuck(t):
    return (1e-3, 300.0, 0.0)


def blows_up(t):
    return (1e-4, 400.0, 1.0) if t < 15000 else (math.nan, math.nan, math.nan)


def test_reached_steps_blown_domains_and_the_log():
    b = ScriptedBatch([fast, decaying, stuck, blows_up])
    log = io.StringIO()
    run = steady.run_to_steady(b, tol=1e-7, max_steps=50000, chunk=5000, log=log)
    assert run["steps"] == 50000 and b.calls == [5000] * 10  # the stuck domain keeps it going
    assert run["reached"].tolist() == [5000, 20000, -1, -1]
    assert run["blown"].tolist() == [False, False, False, True]
    assert np.isfinite(run["when"][:2]).all() and np.isnan(run["when"][2:]).all()
    assert run["when"][0] <= run["when"][1]
    lines = [json.loads(x) for x in log.getvalue().splitlines()]
    assert [x["steps"] for x in lines] == list(range(5000, 50001, 5000))
    assert [x["t"] for x in lines] == list(range(5000, 50001, 5000))
    assert [x["converged"] for x in lines] == [1, 1, 1, 2, 2, 2, 2, 2, 2, 2]
    assert [x["blown"] for x in lines] == [0, 0, 1, 1, 1, 1, 1, 1, 1, 1]
    assert all(x["domains"] == 4 and x["mlups"] > 0 for x in lines)
    assert lines[0]["residual_max"] == pytest.approx(1e-3)
    assert lines[0]["mass"] == pytest.approx(1000.0) and lines[0]["budget"] == pytest.approx(1.25)
    assert lines[-1]["mass"] == pytest.approx(600.0)  # the blown domain's values are left out
    walls = [x["wall_s"] for x in lines]
    assert walls == sorted(walls)


def test_stops_when_nothing_is_left_to_wait_for():
    b = ScriptedBatch([fast, decaying, blows_up])
    run = steady.run_to_steady(b, tol=1e-7, max_steps=10 ** 9, chunk=5000)
    assert run["steps"] == 20000 and b.time == 20000
    assert run["reached"].tolist() == [5000, 20000, -1]


def test_a_single_domain_and_a_bad_chunk():
    dom = SimpleNamespace(pb=SimpleNamespace(cells=64), time=0)
    dom.step = lambda n: setattr(dom, "time", dom.time + n)
    dom.residual = lambda allow_nonfinite=False: decaying(dom.time)
    run = steady.run_to_steady(dom, tol=1e-7, max_steps=10 ** 6, chunk=1000)
    assert run["reached"].tolist() == [19000] and run["steps"] == 19000
    with pytest.raises(ValueError):
        steady.run_to_steady(dom, tol=1e-7, max_steps=10, chunk=1)

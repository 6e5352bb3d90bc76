"""The serving scheduler on CPU (paper_1911_05633_gb300.serve.Server) with stand-in
systems whose work completes after a fixed time and whose "device memory" is a counter:
arrival order, one request per system at a time, residency under the memory cap (bring
in on admission, least-recently-used eviction of idle systems, state carried through an
eviction), and latency bookkeeping."""
import time

import pytest

from paper_1911_05633_gb300.serve import Server, latency_stats, poisson_arrivals


class _Done:
    def __init__(self, t_end):
        self.t_end = t_end

    def query(self):
        return time.perf_counter() >= self.t_end


class Meter:
    """Bytes 'allocated' by the stand-in systems."""

    def __init__(self):
        self.used = 0

    def __call__(self):
        return self.used


class FakeSpec:
    def __init__(self, name, footprint, service_s):
        self.name, self.footprint, self.service = name, footprint, service_s
        self.state = None
        self.measured = None
        self.starts = []


class FakeSystem:
    def __init__(self, spec, state, meter):
        self.spec, self.meter = spec, meter
        self.count = 0 if state is None else state["count"]
        self.buffer_bytes = spec.footprint
        meter.used += spec.footprint

    def run_request(self, keep_sigma=False):
        now = time.perf_counter()
        self.spec.starts.append(now)
        self.count += 1
        return _Done(now + self.spec.service), self.count

    def state(self):
        return {"count": self.count}

    def finish(self):
        pass

    def close(self):
        self.meter.used -= self.spec.footprint


def _server(specs, cap):
    meter = Meter()
    srv = Server({s.name: s for s in specs}, mem_cap_bytes=cap, factory=lambda spec, st: FakeSystem(spec, st, meter),
                 meter=meter)
    return srv, meter


def _overlap(a, b):
    return a.admitted < b.done and b.admitted < a.done


def test_one_request_per_system_and_concurrency_across_systems():
    srv, _ = _server([FakeSpec("a", 1, 0.02), FakeSpec("b", 1, 0.02)], 10)
    reqs = srv.run([(0.0, "a"), (0.0, "a"), (0.0, "b")])
    ra = [r for r in reqs if r.system == "a"]
    rb = [r for r in reqs if r.system == "b"]
    assert not _overlap(ra[0], ra[1])           # the same system runs one request at a time
    assert _overlap(ra[0], rb[0])               # different systems run together
    assert ra[1].admitted >= ra[0].done - 1e-4  # the second waits for the first
    srv.close()


def test_residency_under_the_cap_with_eviction():
    """Cap below the sum of footprints: systems are brought in on admission and idle ones
    evicted least recently used first; the allocated bytes never exceed the cap, and a
    system's state (its iteration count here) survives an eviction."""
    specs = [FakeSpec("big", 6, 0.01), FakeSpec("mid", 4, 0.01), FakeSpec("small", 3, 0.005)]
    srv, meter = _server(specs, 10)
    arrivals = [(0.0, "big"), (0.0, "mid"), (0.03, "small"), (0.05, "big"), (0.08, "mid"), (0.1, "small"),
                (0.12, "big")]
    reqs = srv.run(arrivals, keep_sigma=True)
    assert all(entry[3] <= 10 and entry[4] <= 10 for entry in srv.log)
    evicted = [e[2] for e in srv.log if e[1] == "evict"]
    assert evicted, "the cap must force evictions"
    assert sum(1 for r in reqs if r.brought_in) > len(specs)
    # the iteration count of each system advances by one per request, across evictions
    for name in ("big", "mid", "small"):
        counts = [r.sigma_k for r in reqs if r.system == name]
        assert counts == list(range(1, len(counts) + 1))
    # after every bring-in and eviction the resident footprints and the allocated bytes fit the cap
    for t, ev, name, resident, used in srv.log:
        assert resident <= 10 and used <= 10
    srv.close()
    assert meter.used == 0


def test_waits_while_running_systems_hold_the_memory():
    """A request that does not fit beside running systems waits for them (nothing running
    is evicted)."""
    specs = [FakeSpec("a", 6, 0.03), FakeSpec("b", 6, 0.01)]
    srv, _ = _server(specs, 10)
    reqs = srv.run([(0.0, "a"), (0.001, "b")])
    ra, rb = reqs
    assert rb.admitted >= ra.done - 1e-4
    srv.close()


def test_rejects_systems_above_the_cap():
    with pytest.raises(ValueError):
        _server([FakeSpec("x", 11, 0.0)], 10)


def test_poisson_stream_and_latency_stats():
    arr = poisson_arrivals(200.0, 50, ["a", "b"], seed=3)
    assert len(arr) == 50 and all(t2 >= t1 for (t1, _), (t2, _) in zip(arr, arr[1:]))
    srv, _ = _server([FakeSpec("a", 1, 0.002), FakeSpec("b", 1, 0.004)], 2)
    reqs = srv.run(arr)
    st = latency_stats(reqs)
    assert st["requests"] == 50 and 0.0 < st["p50_ms"] <= st["p99_ms"]
    assert all(r.latency >= (0.002 if r.system == "a" else 0.004) - 1e-4 for r in reqs)
    srv.close()

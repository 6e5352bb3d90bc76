"""The serving scheduler on CPU (paper_1911_05633_gb300.serve.Server) with stand-in
systems whose work completes after a fixed time: arrival order, one request per system
at a time, the memory cap, and latency bookkeeping."""
import time

import pytest

from paper_1911_05633_gb300.serve import Server, latency_stats, poisson_arrivals


class _Done:
    def __init__(self, t_end):
        self.t_end = t_end

    def query(self):
        return time.perf_counter() >= self.t_end


class FakeSystem:
    def __init__(self, footprint, service_s):
        self.footprint = footprint
        self.service = service_s
        self.started = []

    def submit(self, keep_sigma=False):
        now = time.perf_counter()
        self.started.append(now)
        return _Done(now + self.service), None

    def finish(self):
        pass


def _overlap(a, b):
    return a.admitted < b.done and b.admitted < a.done


def test_one_request_per_system_and_concurrency_across_systems():
    systems = {"a": FakeSystem(1, 0.02), "b": FakeSystem(1, 0.02)}
    reqs = Server(systems, mem_cap_bytes=10).run([(0.0, "a"), (0.0, "a"), (0.0, "b")])
    ra = [r for r in reqs if r.system == "a"]
    rb = [r for r in reqs if r.system == "b"]
    assert not _overlap(ra[0], ra[1])           # the same system runs one request at a time
    assert _overlap(ra[0], rb[0])               # different systems run together
    assert ra[1].admitted >= ra[0].done - 1e-4  # the second waits for the first


def test_memory_cap_and_passing():
    """A request whose system is busy does not block a later one for an idle system, and
    the footprints of the running requests never exceed the cap."""
    systems = {"big": FakeSystem(8, 0.03), "small": FakeSystem(2, 0.005), "mid": FakeSystem(5, 0.01)}
    arrivals = [(0.0, "big"), (0.0, "big"), (0.001, "small"), (0.002, "mid"), (0.002, "small")]
    reqs = Server(systems, mem_cap_bytes=10).run(arrivals)
    # footprint only grows at admissions: at each one, what runs then fits the cap
    for r in reqs:
        t = r.admitted
        running = [q for q in reqs if q.admitted <= t < q.done]
        assert sum(systems[q.system].footprint for q in running) <= 10
    small = [r for r in reqs if r.system == "small"]
    bigs = [r for r in reqs if r.system == "big"]
    assert small[0].done < bigs[1].admitted     # the small system passed the waiting big request
    assert all(r.done >= r.admitted >= r.arrival - 1e-6 for r in reqs)


def test_rejects_systems_above_the_cap():
    with pytest.raises(ValueError):
        Server({"x": FakeSystem(11, 0.0)}, mem_cap_bytes=10)


def test_poisson_stream_and_latency_stats():
    arr = poisson_arrivals(200.0, 50, ["a", "b"], seed=3)
    assert len(arr) == 50 and all(t2 >= t1 for (t1, _), (t2, _) in zip(arr, arr[1:]))
    systems = {"a": FakeSystem(1, 0.002), "b": FakeSystem(1, 0.004)}
    reqs = Server(systems, mem_cap_bytes=2).run(arr)
    st = latency_stats(reqs)
    assert st["requests"] == 50 and 0.0 < st["p50_ms"] <= st["p99_ms"]
    assert all(r.latency >= (0.002 if r.system == "a" else 0.004) - 1e-4 for r in reqs)

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
        self.plan_bytes = None
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
    _check_disjoint(srv)
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


class SlowClose(FakeSystem):
    def close(self):
        time.sleep(0.06)  # freeing device memory waits for the device to go idle
        super().close()


def test_later_bring_ins_do_not_hold_the_loop():
    """A system brought in again (its footprint known) is made in the worker that runs its
    request, after the evictions before it have freed their memory on the closer thread: a
    request of a resident system queued behind it is admitted at once, not after the slow
    eviction and bring-in."""
    specs = [FakeSpec("p", 5, 0.005), FakeSpec("q", 1, 0.005), FakeSpec("r", 5, 0.005)]
    meter = Meter()
    made = {"p": 0}

    def factory(spec, st):
        if spec.name == "p":
            made["p"] += 1
            if made["p"] > 1:
                time.sleep(0.08)  # a slow bring-in (buffers, state upload)
        return (SlowClose if spec.name == "r" else FakeSystem)(spec, st, meter)

    srv = Server({s.name: s for s in specs}, mem_cap_bytes=10, factory=factory, meter=meter)
    reqs = srv.run([(0.0, "p"), (0.0, "q"), (0.03, "r"), (0.06, "p"), (0.06, "q")])
    p2 = [r for r in reqs if r.system == "p"][1]
    q2 = [r for r in reqs if r.system == "q"][1]
    assert p2.brought_in and not q2.brought_in
    assert made["p"] == 2
    assert "r" in [e[2] for e in srv.log if e[1] == "evict"]
    assert q2.admitted - p2.admitted < 0.04  # not behind r's 60 ms eviction and p's 80 ms bring-in
    assert q2.done < p2.done
    assert p2.done - p2.admitted > 0.14  # p was made after r had been freed
    assert all(e[3] <= 10 and e[4] <= 10 for e in srv.log)
    srv.close()
    assert meter.used == 0


def test_device_pool_first_fit_alignment_and_merging():
    from paper_1911_05633_gb300.serve import DevicePool
    p = DevicePool(100)
    a, b, c = p.alloc(30), p.alloc(30), p.alloc(30)
    assert (a, b, c) == (0, 30, 60) and p.alloc(20) is None and p.free_bytes() == 10
    p.release(b, 30)
    assert p.alloc(40) is None            # 30 + 10 free, not in one range
    p.release(c, 30)
    assert p.free == [(30, 70)]           # merged with both neighbours
    with pytest.raises(ValueError):
        p.release(40, 10)                 # inside a free range
    p.release(a, 30)
    assert p.free == [(0, 100)]
    q = DevicePool(7 << 20, align=2 << 20)
    assert q.size == 6 << 20 and q.alloc(1) == 0 and q.alloc(1) == 2 << 20 and q.alloc(2 << 20) == 4 << 20
    assert q.alloc(1) is None


def _check_disjoint(srv):
    """Wrap the server's placement so that every placement is checked: each resident range
    inside the pool, no two overlapping."""
    place = srv._place

    def checked(name):
        ok = place(name)
        spans = sorted(srv.ranges.values())
        assert all(o >= 0 and o + n <= srv.mem_cap for o, n in spans)
        assert all(o1 + n1 <= o2 for (o1, n1), (o2, _) in zip(spans, spans[1:]))
        return ok
    srv._place = checked


def test_eviction_until_one_range_holds_the_system():
    """The pool holds a system's buffers in one range: with the free bytes split around a
    resident system, idle systems are evicted (least recently used first) until a single
    range is free, not just enough bytes."""
    specs = [FakeSpec("A", 4, 0.002), FakeSpec("B", 2, 0.002), FakeSpec("C", 4, 0.002), FakeSpec("D", 6, 0.002)]
    srv, meter = _server(specs, 10)
    _check_disjoint(srv)
    srv.run([(0.0, "A"), (0.0, "B"), (0.0, "C")])
    assert srv.ranges == {"A": (0, 4), "B": (4, 2), "C": (6, 4)}
    srv.run([(0.0, "B")])                 # B most recently used
    srv.run([(0.0, "D")])
    evicted = [e[2] for e in srv.log if e[1] == "evict"]
    assert evicted == ["A", "C", "B"]     # A + C free 8 bytes, but on both sides of B
    assert srv.ranges == {"D": (0, 6)}
    srv.close()
    assert meter.used == 0


def test_requests_of_one_system_run_in_arrival_order():
    """Two requests of a system that waits for room: the freed room goes to the earlier
    one (an iteration's state advances request by request, so order matters)."""
    specs = [FakeSpec("big", 3294, 0.03), FakeSpec("c1", 113, 0.002), FakeSpec("mx", 7, 0.002),
             FakeSpec("c0", 4, 0.002)]
    srv, meter = _server(specs, 3294 + 56)
    _check_disjoint(srv)
    for s in specs:  # known plans: every bring-in takes the worker path
        s.plan_bytes = 0
    order = ["big", "c1", "mx", "c0", "c1", "big", "mx", "c0"]
    reqs = srv.run([(0.002 * i, n) for i, n in enumerate(order)])
    for name in ("big", "c1", "mx", "c0"):
        mine = [r for r in reqs if r.system == name]
        assert [r.sigma_k for r in mine] == list(range(1, len(mine) + 1))  # state carried in order
        assert all(a.admitted < b.admitted for a, b in zip(mine, mine[1:]))
    srv.close()
    assert meter.used == 0


def test_failed_bring_in_gives_its_range_back():
    """A system whose making fails in the worker: the request loop raises the error, and
    the reservation (its resident slot and its range of the pool) is gone."""
    specs = [FakeSpec("a", 6, 0.002), FakeSpec("b", 6, 0.002)]
    meter = Meter()
    made = {"b": 0}

    def factory(spec, st):
        if spec.name == "b":
            made["b"] += 1
            if made["b"] > 1:
                raise RuntimeError("bring-in failed")
        return FakeSystem(spec, st, meter)

    srv = Server({s.name: s for s in specs}, mem_cap_bytes=10, factory=factory, meter=meter)
    srv.run([(0.0, "a"), (0.01, "b")])      # b's first making measures it; a is evicted
    srv.run([(0.0, "a")])                   # a back in, b evicted
    with pytest.raises(RuntimeError, match="bring-in failed"):
        srv.run([(0.0, "b")])               # b made in a worker: fails there
    assert "b" not in srv.resident and "b" not in srv.ranges
    assert all(v is not None for v in srv.resident.values())
    assert srv._dpool.free_bytes() + sum(n for _, n in srv.ranges.values()) == srv._dpool.size
    srv.close()
    assert meter.used == 0

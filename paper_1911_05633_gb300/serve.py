"""A request loop over the library: continuous batching of GW work for several systems
of different sizes on one GPU, under a device-memory cap.

Two kinds of request:

* "iteration" -- one whole self-consistent step of a system: G(k, tau) -> G(R, tau) ->
  P -> P(i nu) -> W~ (Eq. W_1) -> W~(tau) -> Sigma, Sigma_x -> Sigma(k, i w) -> the
  chemical potential of the new Sigma (bisection on the particle number) -> the Dyson
  step of Eq. G_1 -> the next G(k, tau);
* "psigma" -- the P and Sigma rows of a system on its resident G(k, tau) and W~(R, i nu):
  G(R, tau), P(R, tau), P(R, i nu), W~(R, tau), Sigma(R, tau) + Sigma_x, Sigma(k, i w).

A system is resident when its plan and buffers live on the device; G(k, tau) (and the
chemical potential) carry from one iteration to the next.  The buffers of every resident
system are ranges of one device pool of the cap's size, allocated once: a request is
admitted in arrival order as soon as its system is idle and, for a system that is not
resident, a range of the pool holds its buffers -- idle resident systems are evicted
least recently used first (their state copied to the host) until one does.  Bringing a
system in (its plan, its state copied up) and evicting one allocate and free nothing on
the device, and both run off the request loop.  Requests of different systems run
concurrently, each on its system's CUDA stream (an iteration in a worker thread, because
the chemical-potential search synchronises its stream).  Latency is completion minus
arrival.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import dataclasses
import time
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import gw


def p_iw_structure(inf) -> str:
    """How P(R, tau) goes to P(R, i nu): mirror-paired when C is symmetric, and only the
    frequencies nu >= 0 when the W solve reads no others (a w_symmetric plan)."""
    if not inf["c_symmetric"]:
        return "general"
    return "mirror_nonneg" if inf["w_symmetric"] else "mirror"


@dataclasses.dataclass
class Request:
    rid: int
    system: str
    arrival: float                    # seconds after the start of the run
    admitted: Optional[float] = None
    done: Optional[float] = None
    event: object = None
    future: object = None
    sigma_k: object = None            # copy of Sigma(k, i w) when kept
    brought_in: bool = False          # the system was made resident for this request

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def arena_words(inf, mode: str) -> Dict[str, int]:
    """The complex words of each buffer of a system (plan info `inf`), in arena order."""
    nk, nt, nn, nw = inf["n_k"], inf["n_tau"], inf["n_nu"], inf["n_omega"]
    No, Npb, lo, lp = inf["n_orb_total"], inf["n_pb_total"], inf["len_orb"], inf["len_pb"]
    w = {"G_k": nk * nt * No * No, "G_R": lo * nt, "P_R": lp * nt, "P_iw": lp * nn, "W_iw": lp * nn,
         "W_R": lp * nt, "S_R": lo * nt, "Sx_R": lo, "S_iw": lo * nw, "S_k": nk * nw * No * No,
         "Sx_k": nk * No * No, "v_R": lp}
    if mode == "iteration":
        w.update(v_q=nk * Npb * Npb, H_k=nk * No * No)
    return {k: int(v) for k, v in w.items()}


class DevicePool:
    """One device buffer of `size` bytes handed out in ranges: first fit, aligned to
    `align` bytes (2 MiB on a device), a freed range merged with its free neighbours.
    With device=None it only keeps the books (no memory behind the ranges)."""

    ALIGN = 2 << 20

    def __init__(self, size: int, device: Optional[int] = None, align: Optional[int] = None):
        self.align = int(align) if align is not None else (self.ALIGN if device is not None else 1)
        self.size = int(size) - int(size) % self.align
        self.free: List[tuple] = [(0, self.size)] if self.size > 0 else []  # (offset, bytes), by offset
        self.buf = None
        if device is not None:
            import torch
            self.buf = torch.empty(self.size, dtype=torch.uint8, device=torch.device("cuda", device))

    def _round(self, n: int) -> int:
        return -(-int(n) // self.align) * self.align

    def alloc(self, n: int) -> Optional[int]:
        """The offset of a free range of n bytes (rounded up), or None when none is free."""
        n = self._round(n)
        for i, (off, m) in enumerate(self.free):
            if m >= n:
                if m == n:
                    del self.free[i]
                else:
                    self.free[i] = (off + n, m - n)
                return off
        return None

    def release(self, off: int, n: int):
        n = self._round(n)
        i = 0
        while i < len(self.free) and self.free[i][0] < off:
            i += 1
        if (i > 0 and self.free[i - 1][0] + self.free[i - 1][1] > off) or \
                (i < len(self.free) and off + n > self.free[i][0]):
            raise ValueError(f"range ({off}, {n}) overlaps a free range")
        self.free.insert(i, (off, n))
        if i + 1 < len(self.free) and off + n == self.free[i + 1][0]:  # merge with the next
            self.free[i] = (off, n + self.free[i + 1][1])
            del self.free[i + 1]
        if i > 0 and self.free[i - 1][0] + self.free[i - 1][1] == off:  # and with the previous
            self.free[i - 1] = (self.free[i - 1][0], self.free[i - 1][1] + self.free[i][1])
            del self.free[i]

    def free_bytes(self) -> int:
        return sum(m for _, m in self.free)

    def view(self, off: int, n: int):
        return self.buf.narrow(0, off, n)


def is_lean(mode: str, precision: str) -> bool:
    """A mixed-precision P/Sigma system: its plan holds no scratch and can stay on the device
    while the system is not resident (its tables are small next to the system's buffers)."""
    return mode == "psigma" and precision == "mixed"


class System:
    """One resident system: its plan and device buffers.

    mode "iteration": whole steps (G and the chemical potential advance per request);
    mode "psigma": the P and Sigma rows on the resident G(k, tau) and a W~(R, i nu) drawn
    from `w_seed` (real, as the W solve returns it for these plans)."""

    def __init__(self, name: str, cell, device: int = 0, precision: str = "fp64", mode: str = "iteration",
                 workspace_bytes: int = 2 << 30, w_seed: int = 0, state: Optional[dict] = None, plan=None,
                 arena=None):
        """arena: a uint8 device tensor to hold the buffers (a range of a server's pool), at
        least 16 bytes per word of arena_words; None allocates one."""
        import torch
        self.name, self.cell, self.precision, self.mode = name, cell, precision, mode
        self.dev = torch.device("cuda", device)
        # a mixed-precision P/Sigma system needs neither the W-solve nor the FP64 digit-product
        # scratch: its plan defers them (and never allocates them); every other system holds
        # its scratch from the start, so that the plan bytes measured when it is first brought
        # in are all it will use.  `plan`: a plan kept from an earlier residency (lean systems)
        t0 = time.perf_counter()
        if plan is None:
            plan = gw.Plan.from_cell(cell, device=device, workspace_bytes=workspace_bytes,
                                     defer_scratch=is_lean(mode, precision))
        self.plan = plan
        t1 = time.perf_counter()
        self.stream = torch.cuda.Stream(device=device)
        # the setup (one fill, the seeds, the state upload) runs on a stream of high priority,
        # so that its few kernels start between other systems' launches instead of queueing
        # behind them; the request stream waits for it on the device, not on the host
        setup = torch.cuda.Stream(device=device, priority=-1)
        with torch.cuda.stream(setup):
            self._setup(cell, w_seed, state, arena)
        self.stream.wait_stream(setup)
        self._setup_stream = setup  # kept until the request stream has passed the setup
        self.setup_s = {"plan": t1 - t0, "buffers": time.perf_counter() - t1}  # host seconds

    def _setup(self, cell, w_seed, state, arena):
        """Every buffer is a view into one arena.  The path writes every element of its
        outputs except P(R, i nu) at nu < 0 under the nu >= 0 structure, so that buffer
        alone is zeroed."""
        import torch
        p = self.plan
        sizes = arena_words(p.info, self.mode)
        total = sum(sizes.values())
        if arena is None:
            arena = torch.empty(16 * total, dtype=torch.uint8, device=self.dev)
        if arena.numel() < 16 * total:
            raise ValueError(f"{self.name}: arena of {arena.numel()} bytes, {16 * total} needed")
        self._arena = arena
        flat = arena.narrow(0, 0, 16 * total).view(torch.complex128)
        off = 0
        for name, n in sizes.items():
            setattr(self, name, flat.narrow(0, off, n))
            off += n
        self.P_iw.zero_()
        if self.mode == "iteration":
            vq, _ = cell.coulomb()
            self.v_q.copy_(torch.from_numpy(vq.reshape(-1)))
            self.H_k.copy_(torch.from_numpy(cell.H_k.reshape(-1)))
            p.fourier_k_to_R("pb", 1, self.v_q, self.v_R)
            self.W_iw.zero_()
        else:
            # W~(R, i nu) and v(R): the draws torch.randn(n, generator) gives, cut in the
            # (still unused) P(R, tau) buffer and copied into the real parts
            gen = torch.Generator(device=self.dev).manual_seed(int(w_seed))
            draw = torch.view_as_real(self.P_R).reshape(-1)
            assert draw.numel() >= max(self.W_iw.numel(), self.v_R.numel())
            for dst in (self.W_iw, self.v_R):
                d = draw[:dst.numel()]
                d.normal_(generator=gen)
                dst.copy_(d)
        if state is None:
            self.G_k.copy_(torch.from_numpy(cell.green_k_tau().reshape(-1)))
            self.mu = float(cell.mu)
        else:
            self.G_k.copy_(state["G_k"], non_blocking=True)  # pinned host state
            self.mu = state["mu"]
        self.buffer_bytes = 16 * total

    def state(self) -> Optional[dict]:
        """The iteration state, copied to pinned host memory (for eviction); None when it
        cannot have changed since it was brought in (P/Sigma requests leave G alone)."""
        import torch
        if self.mode != "iteration":
            return None
        host = torch.empty(self.G_k.numel(), dtype=self.G_k.dtype, pin_memory=True)
        with torch.cuda.stream(self.stream):
            host.copy_(self.G_k, non_blocking=True)
        self.stream.synchronize()
        return {"G_k": host, "mu": self.mu}

    def _rows(self):
        """The P and Sigma rows on the current G(k, tau), enqueued on this system's stream."""
        p, s, inf, prec = self.plan, self.stream.cuda_stream, self.plan.info, self.precision
        p.green_k_to_R(self.G_k, self.G_R, stream=s)
        p.polarizability_tau(self.G_R, self.P_R, precision=prec, stream=s)
        p.transform_tau_iw("B", "tau_to_iw", "pb", self.P_R, self.P_iw, stream=s,
                           structure=p_iw_structure(inf))
        if self.mode == "iteration":
            p.screened_W_iw(self.P_iw, self.v_q, self.W_iw, stream=s)
        p.transform_tau_iw("B", "iw_to_tau", "pb", self.W_iw, self.W_R, stream=s,
                           structure="real" if inf["w_symmetric"] else "general")
        p.self_energy_tau(self.G_R, self.W_R, v_R=self.v_R, Sig_R=self.S_R, Sigx_R=self.Sx_R, precision=prec,
                          stream=s)
        p.transform_tau_iw("F", "tau_to_iw", "orb", self.S_R, self.S_iw, stream=s)
        p.fourier_R_to_k("orb", inf["n_omega"], self.S_iw, self.S_k, stream=s)
        p.fourier_R_to_k("orb", 1, self.Sx_R, self.Sx_k, stream=s)

    def run_request(self, keep_sigma: bool = False):
        """One request on this system's stream.  An iteration also finds the chemical
        potential of its Sigma (bisection in a window around the previous one, synchronous
        on the stream) and takes the Dyson step with it.  Returns (event, Sigma copy)."""
        import torch
        with torch.cuda.stream(self.stream):
            self._rows()
            sig = None
            if keep_sigma:  # to pinned host memory: nothing outside the footprint stays on the device
                sig = torch.empty(self.S_k.numel(), dtype=self.S_k.dtype, pin_memory=True)
                sig.copy_(self.S_k, non_blocking=True)
            if self.mode == "iteration":
                s = self.stream.cuda_stream
                n_el = float(self.cell.n_orb_total)
                # a window around the previous mu, widened while it does not hold the solution
                for half in (0.25, 2.0, 16.0):
                    mu, n = self.plan.chemical_potential(self.H_k, n_el, self.mu - half, self.mu + half, tol=1e-10,
                                                         Sigx_k=self.Sx_k, Sig_k_iw=self.S_k, stream=s)
                    if abs(n - n_el) < 1e-6 * max(1.0, n_el):
                        break
                self.mu = mu
                self.plan.dyson_green_tau(self.H_k, self.mu, Sigx_k=self.Sx_k, Sig_k_iw=self.S_k, G_k_tau=self.G_k,
                                          stream=s)
            ev = torch.cuda.Event()
            ev.record(self.stream)
        return ev, sig

    def finish(self):
        self.plan.sync(stream=self.stream.cuda_stream)

    def close(self, keep_plan: bool = False):
        self.finish()
        if not keep_plan:
            self.plan.close()
        for k in ("G_k", "G_R", "P_R", "P_iw", "W_iw", "W_R", "S_R", "Sx_R", "S_iw", "S_k", "Sx_k", "v_q", "H_k",
                  "v_R", "_arena", "_setup_stream"):
            if hasattr(self, k):
                delattr(self, k)


class SystemSpec:
    """A system the server knows: its cell and mode, its footprint in the device pool (the
    bytes of its buffers, exact from its plan's sizes), the device bytes its plan holds
    outside the pool (measured when it is first made resident), and its state while not
    resident."""

    def __init__(self, name: str, cell, mode: str = "iteration", precision: str = "fp64", w_seed: int = 0,
                 workspace_bytes: int = 2 << 30):
        self.name, self.cell, self.mode, self.precision = name, cell, mode, precision
        self.w_seed, self.workspace_bytes = w_seed, workspace_bytes
        self.state: Optional[dict] = None
        self.plan_bytes: Optional[int] = None
        self.plan = None  # a lean system's plan, kept while the system is not resident
        hp = gw.Plan.from_cell(cell, host_only=True)
        self.footprint = 16 * sum(arena_words(hp.info, mode).values())
        hp.close()

    def prepare(self):
        """Compute the first state (the cell's G(k, tau) and chemical potential) on the host
        now, so that bringing the system in later only copies it up."""
        import torch
        if self.state is None:
            G_k = torch.from_numpy(self.cell.green_k_tau().reshape(-1))
            self.state = {"G_k": G_k.pin_memory() if torch.cuda.is_available() else G_k, "mu": float(self.cell.mu)}


class Server:
    """Continuous batching over systems brought in and out of a device pool of the cap's size."""

    def __init__(self, specs: Dict[str, SystemSpec], mem_cap_bytes: int, device: int = 0, max_workers: int = 8,
                 factory=None, meter=None):
        """factory(spec, state) -> a resident system (default: System on `device`, its buffers
        in the pool; with a factory the pool only keeps the books); meter() -> device bytes
        in use (default: the CUDA driver's count)."""
        self.specs = specs
        self.device = device
        self.factory = factory
        self.meter = meter
        self._dpool: Optional[DevicePool] = None
        self.ranges: Dict[str, tuple] = {}  # resident system -> (offset, bytes) in the pool
        self.resident: "collections.OrderedDict[str, System]" = collections.OrderedDict()  # LRU order
        self.mem_cap = mem_cap_bytes
        self.pool = cf.ThreadPoolExecutor(max_workers=max_workers)
        # evictions inside the request loop run here, one at a time and in order (saving an
        # iteration's state waits for its copy to the host)
        self.closer = cf.ThreadPoolExecutor(max_workers=1)
        self._last_close: Optional[cf.Future] = None
        # seconds the workers spent waiting for evictions and making systems, and the closer
        # thread closing evicted ones
        self.timing = {"wait_closes_s": [], "make_s": [], "make_plan_s": [], "close_s": []}
        self.log: List[tuple] = []  # (time, event, system, resident bytes after it, device bytes in use)

    @property
    def mem_cap(self) -> int:
        return self._mem_cap

    @mem_cap.setter
    def mem_cap(self, cap: int):
        """The pool's size; set while no system is resident (the pool is made again)."""
        if self.resident:
            raise RuntimeError("the memory cap changes only while no system is resident")
        self._mem_cap = int(cap)
        self._drop_pool()
        align = 1 if self.factory is not None else DevicePool.ALIGN
        too_big = [n for n, s in self.specs.items() if -(-s.footprint // align) * align > self._mem_cap]
        if too_big:
            raise ValueError(f"systems larger than the memory cap: {too_big}")

    def _pool(self) -> DevicePool:
        if self._dpool is None:
            self._dpool = DevicePool(self._mem_cap, None if self.factory is not None else self.device)
        return self._dpool

    def _drop_pool(self):
        if self._dpool is not None:
            had = self._dpool.buf is not None
            self._dpool = None
            if had:
                import torch
                torch.cuda.empty_cache()

    def resident_bytes(self) -> int:
        return sum(self.specs[n].footprint for n in list(self.resident))  # a snapshot: workers read it too

    def _device_used(self) -> int:
        if self.meter is not None:
            return int(self.meter())
        import torch
        # the driver's count: no device synchronisation, which would wait for every request
        # in flight
        free, total = torch.cuda.mem_get_info(self.device)
        return int(total - free)

    def _place(self, name: str) -> bool:
        """A range of the pool for `name`'s buffers, if one is free."""
        off = self._pool().alloc(self.specs[name].footprint)
        if off is None:
            return False
        self.ranges[name] = (off, self.specs[name].footprint)
        return True

    def _make(self, name: str):
        """A resident system for spec `name` in its range (its plan kept from an earlier
        residency when lean)."""
        spec = self.specs[name]
        if self.factory is not None:
            return self.factory(spec, spec.state)
        off, n = self.ranges[name]
        sysm = System(name, spec.cell, device=self.device, precision=spec.precision, mode=spec.mode,
                      workspace_bytes=spec.workspace_bytes, w_seed=spec.w_seed, state=spec.state, plan=spec.plan,
                      arena=self._dpool.view(off, n))
        if is_lean(spec.mode, spec.precision):
            spec.plan = sysm.plan
        return sysm

    def _bring_and_run(self, name: str, keep_sigma: bool, closes: Optional[cf.Future]):
        """Worker job: make the system (its range already placed) and run its request, once
        the evictions submitted before it have saved their state (`closes`: the last of
        them; they run in order)."""
        t0 = time.perf_counter()
        if closes is not None:
            closes.result()
        t1 = time.perf_counter()
        sysm = self._make(name)
        self.timing["wait_closes_s"].append(t1 - t0)
        self.timing["make_s"].append(time.perf_counter() - t1)
        self.timing["make_plan_s"].append(getattr(sysm, "setup_s", {}).get("plan", 0.0))
        self.resident[name] = sysm  # replaces the reservation (one assignment)
        return sysm.run_request(keep_sigma)

    def bring_in(self, name: str):
        """Make `name` resident now (in a free range of the pool).  The first time, with the
        device quiet, it also measures the device bytes the system's plan holds outside the
        pool."""
        spec = self.specs[name]
        if name not in self.ranges and not self._place(name):
            raise RuntimeError(f"{name}: no free range of {spec.footprint} bytes in the pool")
        self._wait_closes()
        measure = spec.plan_bytes is None
        if measure and self.factory is None:
            import torch
            torch.cuda.synchronize(self.device)
        before = self._device_used()
        sysm = self._make(name)
        if measure:
            spec.plan_bytes = max(0, self._device_used() - before)
        self.resident[name] = sysm
        return sysm

    def _release(self, name: str):
        off, n = self.ranges.pop(name)
        self._dpool.release(off, n)

    def evict(self, name: str):
        sysm = self.resident.pop(name)
        self._release(name)
        self._close(name, sysm)

    def _evict_in_background(self, name: str):
        """Take `name` off the resident set and its range back now; save its state and close
        it on the closer thread (a system made in the range later waits for that)."""
        sysm = self.resident.pop(name)
        self._release(name)
        self._last_close = self.closer.submit(self._close, name, sysm)

    def _wait_closes(self):
        if self._last_close is not None:
            self._last_close.result()
            self._last_close = None

    def _close(self, name: str, sysm):
        t0 = time.perf_counter()
        spec = self.specs[name]
        st = sysm.state()
        if st is not None:
            spec.state = st
        if self.factory is None:
            sysm.close(keep_plan=spec.plan is not None)
        else:
            sysm.close()
        del sysm
        self.timing["close_s"].append(time.perf_counter() - t0)

    def close(self):
        self._wait_closes()
        for n in list(self.resident):
            self.evict(n)
        for spec in self.specs.values():
            if getattr(spec, "plan", None) is not None:
                spec.plan.close()
                spec.plan = None
        self._drop_pool()
        self.pool.shutdown()
        self.closer.shutdown()

    def _victims(self, running, queue, keep: str = "") -> List[str]:
        """Idle resident systems in the order to evict them: those no queued request waits
        for first, each group least recently used first."""
        wanted = {r.system for r in queue}
        idle = [n for n in self.resident if n not in running and n != keep]
        return [n for n in idle if n not in wanted] + [n for n in idle if n in wanted]

    def run(self, arrivals: Sequence[tuple], keep_sigma: bool = False, poll_s: float = 20e-6) -> List[Request]:
        """Serve `arrivals` = [(seconds after start, system name), ...]; returns the requests
        with their admission and completion times."""
        reqs = [Request(i, name, float(t)) for i, (t, name) in enumerate(sorted(arrivals, key=lambda a: a[0]))]
        pending = collections.deque(reqs)
        queue: collections.deque = collections.deque()
        running: Dict[str, Request] = {}
        t0 = time.perf_counter()
        # the queue is scanned again only after an arrival, a completion or a system made:
        # an idle scan would hold the interpreter lock the workers need
        dirty = True
        while pending or queue or running:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
                dirty = True
            waiting = set()  # systems with a request left in the queue in this pass
            idle = None      # the pass's eviction candidates, listed when first needed
            for r in (list(queue) if dirty else ()):
                if r.system in running or r.system in waiting:
                    # one request per system at a time, in arrival order; later requests of
                    # other systems may pass
                    continue
                spec = self.specs[r.system]
                if r.system not in self.resident:
                    first = spec.plan_bytes is None
                    if first and any(v is None for v in self.resident.values()):
                        waiting.add(r.system)
                        continue  # a first bring-in measures its plan: let the pending ones finish
                    placed = self._place(r.system)
                    if not placed:
                        if idle is None:
                            idle = self._victims(running, queue)
                        else:  # admissions earlier in the pass made some of them busy
                            idle = [n for n in idle if n not in running and n in self.resident]
                        while not placed and idle:
                            victim = idle.pop(0)
                            self._evict_in_background(victim)
                            self.log.append((time.perf_counter() - t0, "evict", victim, self.resident_bytes(),
                                             self._device_used()))
                            placed = self._place(r.system)
                        if not placed:
                            waiting.add(r.system)
                            continue  # the running systems hold the pool: wait
                    r.brought_in = True
                    if not first:
                        # made in the worker that runs the request, so that this loop goes on
                        # admitting and completing others meanwhile (a reserved system is never
                        # a victim: its request is running)
                        self.resident[r.system] = None
                        self.log.append((time.perf_counter() - t0, "bring_in", r.system, self.resident_bytes(),
                                         self._device_used()))
                        queue.remove(r)
                        r.admitted = time.perf_counter() - t0
                        r.future = self.pool.submit(self._bring_and_run, r.system, keep_sigma, self._last_close)
                        running[r.system] = r
                        continue
                    self.bring_in(r.system)
                    self.log.append((time.perf_counter() - t0, "bring_in", r.system, self.resident_bytes(),
                                     self._device_used()))
                self.resident.move_to_end(r.system)
                queue.remove(r)
                r.admitted = time.perf_counter() - t0
                r.future = self.pool.submit(self.resident[r.system].run_request, keep_sigma)
                running[r.system] = r
            dirty = False
            for name, r in list(running.items()):
                if r.future is not None and r.future.done():
                    dirty = True
                    try:
                        r.event, r.sigma_k = r.future.result()
                    except BaseException:
                        if name in self.resident and self.resident[name] is None:
                            del self.resident[name]  # a reservation whose system was never made
                            self._release(name)
                        raise
                    r.future = None
                if r.future is None and r.event.query():
                    r.done = time.perf_counter() - t0
                    del running[name]
                    dirty = True
            if not running and not queue and pending:
                time.sleep(max(0.0, min(pending[0].arrival - (time.perf_counter() - t0), 1e-3)))
            elif running:
                time.sleep(poll_s)
        self._wait_closes()
        for sysm in self.resident.values():
            sysm.finish()
        return reqs


def poisson_arrivals(rate_per_s: float, n: int, names: Sequence[str], seed: int = 0) -> List[tuple]:
    """n arrivals of a Poisson process of the given rate, each for a system drawn uniformly."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, n))
    return [(float(ti), names[int(rng.integers(len(names)))]) for ti in t]


def latency_stats(reqs: Sequence[Request]) -> dict:
    lat = np.array([r.latency for r in reqs]) * 1e3
    span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
    return {"requests": len(reqs), "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3), "mean_ms": round(float(lat.mean()), 3),
            "throughput_per_s": round(len(reqs) / span, 3),
            "brought_in": int(sum(1 for r in reqs if r.brought_in))}

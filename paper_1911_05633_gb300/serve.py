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
chemical potential) carry from one iteration to the next.  A request is admitted in
arrival order as soon as its system is idle and the resident bytes fit the cap; a
system that is not resident is brought in on admission (its plan built, its state
copied up), evicting idle resident systems least recently used first (their state
copied to the host) while the cap would be exceeded.  Requests of different systems
run concurrently, each on its system's CUDA stream (an iteration in a worker thread,
because the chemical-potential search synchronises its stream).  Latency is
completion minus arrival.
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


def is_lean(mode: str, precision: str) -> bool:
    """A mixed-precision P/Sigma system: its plan holds no scratch and can stay on the device
    while the system is not resident (its tables are small next to the system's buffers)."""
    return mode == "psigma" and precision == "mixed"


def _bytes(*ts) -> int:
    return int(sum(t.numel() * t.element_size() for t in ts))


class System:
    """One resident system: its plan and device buffers.

    mode "iteration": whole steps (G and the chemical potential advance per request);
    mode "psigma": the P and Sigma rows on the resident G(k, tau) and a W~(R, i nu) drawn
    from `w_seed` (real, as the W solve returns it for these plans)."""

    def __init__(self, name: str, cell, device: int = 0, precision: str = "fp64", mode: str = "iteration",
                 workspace_bytes: int = 2 << 30, w_seed: int = 0, state: Optional[dict] = None, plan=None):
        import torch
        self.name, self.cell, self.precision, self.mode = name, cell, precision, mode
        self.dev = torch.device("cuda", device)
        # a mixed-precision P/Sigma system needs neither the W-solve nor the FP64 digit-product
        # scratch: its plan defers them (and never allocates them); every other system holds
        # its scratch from the start, so that the footprint measured when it is brought in is
        # all it will use.  `plan`: a plan kept from an earlier residency (lean systems only)
        if plan is None:
            plan = gw.Plan.from_cell(cell, device=device, workspace_bytes=workspace_bytes,
                                     defer_scratch=is_lean(mode, precision))
        self.plan = plan
        self.stream = torch.cuda.Stream(device=device)
        with torch.cuda.stream(self.stream):
            self._setup(cell, w_seed, state)
        # this system's own work only: other systems' requests keep running meanwhile
        self.stream.synchronize()

    def _setup(self, cell, w_seed, state):
        import torch
        p, inf = self.plan, self.plan.info
        nk, nt, nn, nw = inf["n_k"], inf["n_tau"], inf["n_nu"], inf["n_omega"]
        No = inf["n_orb_total"]
        z = lambda n: torch.zeros(n, dtype=torch.complex128, device=self.dev)
        self.G_k = z(nk * nt * No * No)
        self.G_R, self.P_R = z(p.len("orb", nt)), z(p.len("pb", nt))
        self.P_iw, self.W_iw, self.W_R = z(p.len("pb", nn)), z(p.len("pb", nn)), z(p.len("pb", nt))
        self.S_R, self.Sx_R, self.S_iw = z(p.len("orb", nt)), z(p.len("orb", 1)), z(p.len("orb", nw))
        self.S_k, self.Sx_k = z(nk * nw * No * No), z(nk * No * No)
        bufs = [self.G_k, self.G_R, self.P_R, self.P_iw, self.W_iw, self.W_R, self.S_R, self.Sx_R, self.S_iw,
                self.S_k, self.Sx_k]
        if self.mode == "iteration":
            vq, _ = cell.coulomb()
            self.v_q = torch.from_numpy(vq.reshape(-1)).to(self.dev)
            self.H_k = torch.from_numpy(cell.H_k.reshape(-1)).to(self.dev)
            self.v_R = p.fourier_k_to_R("pb", 1, self.v_q)
            bufs += [self.v_q, self.H_k, self.v_R]
        else:
            gen = torch.Generator(device=self.dev).manual_seed(int(w_seed))
            self.W_iw.copy_(torch.randn(self.W_iw.numel(), dtype=torch.float64, device=self.dev, generator=gen))
            self.v_R = torch.randn(p.len("pb", 1), dtype=torch.float64, device=self.dev,
                                   generator=gen).to(torch.complex128)
            bufs += [self.v_R]
        if state is None:
            self.G_k.copy_(torch.from_numpy(cell.green_k_tau().reshape(-1)))
            self.mu = float(cell.mu)
        else:
            self.G_k.copy_(state["G_k"], non_blocking=True)  # pinned host state
            self.mu = state["mu"]
        self.buffer_bytes = _bytes(*bufs)

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
                  "v_R"):
            if hasattr(self, k):
                delattr(self, k)


class SystemSpec:
    """A system the server knows: its cell and mode, its footprint on the device (measured
    when it is first made resident, estimated before), and its state while not resident."""

    def __init__(self, name: str, cell, mode: str = "iteration", precision: str = "fp64", w_seed: int = 0,
                 workspace_bytes: int = 2 << 30):
        self.name, self.cell, self.mode, self.precision = name, cell, mode, precision
        self.w_seed, self.workspace_bytes = w_seed, workspace_bytes
        self.state: Optional[dict] = None
        self.measured: Optional[int] = None
        self.plan = None  # a lean system's plan, kept while the system is not resident
        hp = gw.Plan.from_cell(cell, host_only=True)
        inf = hp.info
        nk, nt, nn, nw, No = inf["n_k"], inf["n_tau"], inf["n_nu"], inf["n_omega"], inf["n_orb_total"]
        lo, lp, Npb = inf["len_orb"], inf["len_pb"], inf["n_pb_total"]
        words = nk * nt * No * No + lo * (nt + 1 + nw) + lp * (2 * nt + 2 * nn + 1) + nk * (nw + 1) * No * No
        if mode == "iteration":
            words += 2 * nk * Npb * Npb + nk * No * No
        hp.close()
        # buffers, plus the plan's own tables and W-solve scratch (bounded by workspace_bytes)
        self.estimate = int(16 * words * 1.05) + (workspace_bytes if mode == "iteration" else 0) + (64 << 20)

    @property
    def footprint(self) -> int:
        return self.measured if self.measured is not None else self.estimate

    def prepare(self):
        """Compute the first state (the cell's G(k, tau) and chemical potential) on the host
        now, so that bringing the system in later only copies it up."""
        import torch
        if self.state is None:
            G_k = torch.from_numpy(self.cell.green_k_tau().reshape(-1))
            self.state = {"G_k": G_k.pin_memory() if torch.cuda.is_available() else G_k, "mu": float(self.cell.mu)}


class Server:
    """Continuous batching over systems brought in and out of device memory under a cap."""

    def __init__(self, specs: Dict[str, SystemSpec], mem_cap_bytes: int, device: int = 0, max_workers: int = 8,
                 factory=None, meter=None):
        """factory(spec, state) -> a resident system (default: System on `device`); meter() ->
        device bytes in use (default: the CUDA driver's count)."""
        self.specs = specs
        self.mem_cap = int(mem_cap_bytes)
        self.device = device
        self.factory = factory
        self.meter = meter
        too_big = [n for n, s in specs.items() if s.footprint > self.mem_cap]
        if too_big:
            raise ValueError(f"systems larger than the memory cap: {too_big}")
        self.resident: "collections.OrderedDict[str, System]" = collections.OrderedDict()  # LRU order
        self.pool = cf.ThreadPoolExecutor(max_workers=max_workers)
        self.log: List[tuple] = []  # (time, event, system, resident bytes after it, device bytes in use)

    def resident_bytes(self) -> int:
        return sum(self.specs[n].footprint for n in self.resident)

    def _device_used(self) -> int:
        if self.meter is not None:
            return int(self.meter())
        import torch
        # the driver's count (allocations are synchronous calls): no device synchronisation,
        # which would wait for every request in flight
        free, total = torch.cuda.mem_get_info(self.device)
        return int(total - free)

    def bring_in(self, name: str):
        spec = self.specs[name]
        # the footprint is measured once, the first time the system comes in, with the device
        # quiet (no other request allocating or freeing meanwhile); later bring-ins reuse it
        # and wait for nothing but their own setup
        measure = spec.measured is None
        if measure and self.factory is None:
            import torch
            torch.cuda.synchronize(self.device)
        before = self._device_used()
        if self.factory is not None:
            sysm = self.factory(spec, spec.state)
        else:
            sysm = System(name, spec.cell, device=self.device, precision=spec.precision, mode=spec.mode,
                          workspace_bytes=spec.workspace_bytes, w_seed=spec.w_seed, state=spec.state,
                          plan=spec.plan)
            if is_lean(spec.mode, spec.precision):
                spec.plan = sysm.plan
        if measure:
            spec.measured = max(self._device_used() - before, sysm.buffer_bytes)
        self.resident[name] = sysm
        return sysm

    def evict(self, name: str):
        sysm = self.resident.pop(name)
        spec = self.specs[name]
        st = sysm.state()
        if st is not None:
            spec.state = st
        if self.factory is None:
            sysm.close(keep_plan=spec.plan is not None)
        else:
            sysm.close()
        del sysm
        if self.factory is None:
            import torch
            torch.cuda.empty_cache()

    def close(self):
        for n in list(self.resident):
            self.evict(n)
        for spec in self.specs.values():
            if getattr(spec, "plan", None) is not None:
                spec.plan.close()
                spec.plan = None
        self.pool.shutdown()

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
        while pending or queue or running:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            for r in list(queue):
                if r.system in running:
                    continue  # one request per system at a time; later requests of others may pass
                spec = self.specs[r.system]
                if r.system not in self.resident:
                    need = spec.footprint
                    idle = self._victims(running, queue)
                    while self.resident_bytes() + need > self.mem_cap and idle:
                        victim = idle.pop(0)
                        self.evict(victim)
                        self.log.append((time.perf_counter() - t0, "evict", victim, self.resident_bytes(),
                                         self._device_used()))
                    if self.resident_bytes() + need > self.mem_cap:
                        continue  # the running systems hold the memory: wait
                    self.bring_in(r.system)
                    r.brought_in = True
                    # the measured footprint may exceed the estimate admission used: evict
                    # more idle systems until the cap holds again
                    idle = self._victims(running, queue, keep=r.system)
                    while self.resident_bytes() > self.mem_cap and idle:
                        victim = idle.pop(0)
                        self.evict(victim)
                        self.log.append((time.perf_counter() - t0, "evict", victim, self.resident_bytes(),
                                         self._device_used()))
                    self.log.append((time.perf_counter() - t0, "bring_in", r.system, self.resident_bytes(),
                                     self._device_used()))
                    if self.resident_bytes() > self.mem_cap:  # the running systems and this one alone exceed it
                        raise RuntimeError(f"{r.system}: resident bytes above the cap after bringing it in")
                self.resident.move_to_end(r.system)
                queue.remove(r)
                r.admitted = time.perf_counter() - t0
                r.future = self.pool.submit(self.resident[r.system].run_request, keep_sigma)
                running[r.system] = r
            for name, r in list(running.items()):
                if r.future is not None and r.future.done():
                    r.event, r.sigma_k = r.future.result()
                    r.future = None
                if r.future is None and r.event.query():
                    r.done = time.perf_counter() - t0
                    del running[name]
            if not running and not queue and pending:
                time.sleep(max(0.0, min(pending[0].arrival - (time.perf_counter() - t0), 1e-3)))
            elif running:
                time.sleep(poll_s)
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

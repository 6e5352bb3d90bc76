"""A request loop over the library: continuous batching of GW iterations for several
systems on one GPU.

Each system (a cell with its plan) keeps its Green function G(k, tau), its bare
interaction v(q) and v(R), H(k) and every intermediate buffer resident on the device
between requests.  A request asks for one iteration of one system: G(k, tau) ->
G(R, tau) -> P -> P(i nu) -> W~ -> W~(tau) -> Sigma, Sigma_x -> Sigma(k, i w) -> the
Dyson step of Eq. G_1 -> the next G(k, tau), all through the C ABI on the system's own
CUDA stream.  Requests are admitted in arrival order as soon as their system is idle
and the resident bytes of the running systems plus theirs fit the memory cap; requests
of different systems then run concurrently on the device.  Completion is detected by
polling a CUDA event per request; latency is completion time minus arrival time.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import gw


@dataclasses.dataclass
class Request:
    rid: int
    system: str
    arrival: float                    # seconds after the start of the run
    admitted: Optional[float] = None
    done: Optional[float] = None
    event: object = None
    sigma_k: object = None            # copy of Sigma(k, i w) when kept

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class System:
    """One cell: its plan and its resident device buffers."""

    def __init__(self, name: str, cell, device: int = 0, precision: str = "fp64", workspace_bytes: int = 2 << 30):
        import torch
        self.name = name
        self.cell = cell
        self.precision = precision
        self.plan = gw.Plan.from_cell(cell, device=device, workspace_bytes=workspace_bytes)
        self.dev = torch.device("cuda", device)
        self.stream = torch.cuda.Stream(device=device)
        p, inf = self.plan, self.plan.info
        nk, nt, nn, nw = inf["n_k"], inf["n_tau"], inf["n_nu"], inf["n_omega"]
        No, Npb = inf["n_orb_total"], inf["n_pb_total"]
        z = lambda n: torch.zeros(n, dtype=torch.complex128, device=self.dev)
        self.G_k = z(nk * nt * No * No)
        self.G0 = torch.from_numpy(cell.green_k_tau().reshape(-1)).to(self.dev)
        vq, _ = cell.coulomb()
        self.v_q = torch.from_numpy(vq.reshape(-1)).to(self.dev)
        self.H_k = torch.from_numpy(cell.H_k.reshape(-1)).to(self.dev)
        self.G_R, self.P_R = z(p.len("orb", nt)), z(p.len("pb", nt))
        self.P_iw, self.W_iw, self.W_R = z(p.len("pb", nn)), z(p.len("pb", nn)), z(p.len("pb", nt))
        self.v_R = p.fourier_k_to_R("pb", 1, self.v_q)
        self.S_R, self.Sx_R, self.S_iw = z(p.len("orb", nt)), z(p.len("orb", 1)), z(p.len("orb", nw))
        self.S_k, self.Sx_k = z(nk * nw * No * No), z(nk * No * No)
        torch.cuda.synchronize(self.dev)
        self.reset()
        # resident bytes: the buffers above plus the plan's W-solve scratch
        bufs = [self.G_k, self.G0, self.v_q, self.H_k, self.G_R, self.P_R, self.P_iw, self.W_iw, self.W_R,
                self.v_R, self.S_R, self.Sx_R, self.S_iw, self.S_k, self.Sx_k]
        self.footprint = int(sum(b.numel() * b.element_size() for b in bufs) + inf["workspace_bytes"])

    def reset(self):
        """Back to the input G(k, tau) (the first iteration)."""
        self.G_k.copy_(self.G0)

    def enqueue_iteration(self):
        """One iteration on this system's stream; the next G(k, tau) replaces the current one."""
        p, s, inf, prec = self.plan, self.stream.cuda_stream, self.plan.info, self.precision
        p.green_k_to_R(self.G_k, self.G_R, stream=s)
        p.polarizability_tau(self.G_R, self.P_R, precision=prec, stream=s)
        p.transform_tau_iw("B", "tau_to_iw", "pb", self.P_R, self.P_iw, stream=s,
                           structure="mirror" if inf["c_symmetric"] else "general")
        p.screened_W_iw(self.P_iw, self.v_q, self.W_iw, stream=s)
        p.transform_tau_iw("B", "iw_to_tau", "pb", self.W_iw, self.W_R, stream=s,
                           structure="real" if inf["w_symmetric"] else "general")
        p.self_energy_tau(self.G_R, self.W_R, v_R=self.v_R, Sig_R=self.S_R, Sigx_R=self.Sx_R, precision=prec,
                          stream=s)
        p.transform_tau_iw("F", "tau_to_iw", "orb", self.S_R, self.S_iw, stream=s)
        p.fourier_R_to_k("orb", inf["n_omega"], self.S_iw, self.S_k, stream=s)
        p.fourier_R_to_k("orb", 1, self.Sx_R, self.Sx_k, stream=s)
        p.dyson_green_tau(self.H_k, self.cell.mu, Sigx_k=self.Sx_k, Sig_k_iw=self.S_k, G_k_tau=self.G_k, stream=s)

    def submit(self, keep_sigma: bool = False):
        """Enqueue one iteration; returns (event, copy of Sigma(k, i w) or None).  The event
        answers query() once the device has finished it."""
        import torch
        with torch.cuda.stream(self.stream):
            self.enqueue_iteration()
            sig = self.S_k.clone() if keep_sigma else None
            ev = torch.cuda.Event()
            ev.record(self.stream)
        return ev, sig

    def finish(self):
        self.plan.sync(stream=self.stream.cuda_stream)

    def close(self):
        self.plan.close()


class Server:
    """Continuous batching over several systems under a device-memory cap."""

    def __init__(self, systems: Dict[str, System], mem_cap_bytes: int):
        self.systems = systems
        self.mem_cap = int(mem_cap_bytes)
        too_big = [n for n, s in systems.items() if s.footprint > self.mem_cap]
        if too_big:
            raise ValueError(f"systems larger than the memory cap: {too_big}")

    def run(self, arrivals: Sequence[tuple], keep_sigma: bool = False, poll_s: float = 20e-6) -> List[Request]:
        """Serve `arrivals` = [(seconds after start, system name), ...] (any order); returns
        the requests with their admission and completion times."""
        reqs = [Request(i, name, float(t)) for i, (t, name) in enumerate(sorted(arrivals, key=lambda a: a[0]))]
        pending = collections.deque(reqs)
        queue: collections.deque = collections.deque()
        running: Dict[str, Request] = {}
        used = 0
        t0 = time.perf_counter()
        while pending or queue or running:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            # admit in arrival order: a request waits while its system is busy; others may pass it
            for r in list(queue):
                sysm = self.systems[r.system]
                if r.system in running or used + sysm.footprint > self.mem_cap:
                    continue
                queue.remove(r)
                r.admitted = time.perf_counter() - t0
                r.event, r.sigma_k = sysm.submit(keep_sigma)
                running[r.system] = r
                used += sysm.footprint
            for name, r in list(running.items()):
                if r.event.query():
                    r.done = time.perf_counter() - t0
                    del running[name]
                    used -= self.systems[name].footprint
            if not running and not queue and pending:
                time.sleep(max(0.0, min(pending[0].arrival - (time.perf_counter() - t0), 1e-3)))
            elif running:
                time.sleep(poll_s)
        for s in self.systems.values():
            s.finish()
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
            "throughput_per_s": round(len(reqs) / span, 3)}

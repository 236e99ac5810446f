"""Continuous-batching server for many independent colour-gradient runs.

Requests (a droplet problem, a step count, an arrival time) are admitted while
the device's free memory (as the driver reports it at admission time) and the
batch slots allow; every admitted run keeps its state on the
device and all active runs advance together.  In the "batched" mode one batch
step is four shared launches over the tiles of every active run (cg_batch_*,
replayed from CUDA graphs); in the "per_run" mode each run is stepped with its
own launches (cg_step), one run after the other, on the same stream.  Runs
finish at different times; a finished run's summary (per-colour mass,
pressure jump, largest speed, non-finite flag) is reduced on the device and
read back, and its memory goes to the next arrivals.  In the batched mode admission overlaps the GPU: before a
quantum the server admits arrived requests for at most ADMIT_SLICE seconds of
host time (at least one when the GPU would otherwise idle), and while the
quantum runs it admits further arrivals as long as the GPU is still busy; runs
admitted during a quantum join the next one.  Time to result is measured from a
request's arrival to the end of its read-back on the host clock.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import cg


@dataclass
class Result:
    rid: int
    edge: int
    steps: int
    arrival: float
    admitted: float
    finished: float
    mass0: np.ndarray
    mass: np.ndarray
    dp: float
    u_max: float
    nonfinite: int
    macros: Optional[dict] = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class _Run:
    req: object
    dom: cg.Domain
    done: int
    admitted: float
    mass0: np.ndarray


def _r2(n: int) -> np.ndarray:
    d = (np.arange(n) - n / 2.0) ** 2
    return d[:, None, None] + d[None, :, None] + d[None, None, :]


def diagnostics(n: int, radius: float, p: np.ndarray, u: np.ndarray):
    """Host form of the run summary, for read-back fields (p as [z, y, x], u
    as [3, z, y, x]): pressure jump (mean p inside half the radius minus mean p
    beyond the radius plus a quarter edge, about the box centre) and largest
    |u|.  The server computes the same on the device (cg_reduce_diagnostics)."""
    r2 = _r2(n)
    inner = r2 < (0.5 * radius) ** 2
    outer = r2 > (radius + 0.25 * n) ** 2
    p = p.reshape(n, n, n)
    dp = float(p[inner].mean() - p[outer].mean()) if inner.any() and outer.any() else float("nan")
    return dp, float(np.sqrt((u.reshape(3, -1) ** 2).sum(axis=0)).max())


def _summary(req, dom: cg.Domain, keep_macros: bool):
    """Per-colour mass, pressure jump, largest speed and non-finite flag of a
    finished run, reduced on the device (no field read-back)."""
    n = req.edge
    dg = dom.diagnostics((n / 2.0, n / 2.0, n / 2.0), 0.5 * req.radius, req.radius + 0.25 * n)
    dp = dg["p_in"] - dg["p_out"] if dg["n_in"] and dg["n_out"] else float("nan")
    m = dom.macros() if keep_macros else None
    return dg["mass"], dp, dg["u_max"], dg["nonfinite"], m


ADMIT_SLICE = 0.02  # seconds of admission work before a quantum (batched mode)


class Server:
    """mode: "batched" (shared launches) or "per_run" (one run's launches at a
    time).  A request is admitted when its workspace fits the device memory
    that is free at that moment (cudaMemGetInfo, plus what PyTorch's caching
    allocator holds unused) less a reserve of `reserve` bytes (default: 2 %
    of the device memory), and, if hbm_budget is given, when the active runs'
    workspaces stay within it; max_active: batch slots; quantum: most steps
    advanced between admission checks."""

    def __init__(self, mode="batched", precision="f32", max_active=256, quantum=100,
                 hbm_budget: Optional[int] = None, device="cuda", keep_macros=False, depth=0,
                 reserve: Optional[int] = None):
        import torch
        if mode not in ("batched", "per_run"):
            raise ValueError("mode must be 'batched' or 'per_run'")
        self.mode, self.precision, self.quantum = mode, precision, int(quantum)
        self.max_active, self.keep_macros = int(max_active), keep_macros
        self.device = torch.device(device)
        total = torch.cuda.get_device_properties(self.device).total_memory
        self.total_memory = total
        self.hbm_budget = None if hbm_budget is None else int(hbm_budget)
        self.reserve = int(0.02 * total) if reserve is None else int(reserve)
        self.stream = torch.cuda.Stream(self.device)
        # initialisation of the runs of a batch, beside the batch's steps
        self.io_stream = torch.cuda.Stream(self.device)
        self.batch = None
        if mode == "batched":
            self.batch = cg.Batch(self.max_active, precision, device=self.device, stream=self.stream)
            if depth:
                self.batch.set_depth(depth)
        self.log: List[tuple] = []

    def free_bytes(self) -> int:
        """Device memory a new workspace can take now: free memory as the
        driver reports it plus blocks PyTorch's allocator caches unused, less
        the reserve."""
        import torch
        free, _ = torch.cuda.mem_get_info(self.device)
        cached = torch.cuda.memory_reserved(self.device) - torch.cuda.memory_allocated(self.device)
        return free + cached - self.reserve

    def close(self):
        if self.batch is not None:
            self.batch.close()
            self.batch = None

    def _admit(self, req, now) -> _Run:
        wl = req.workload()
        stream = self.io_stream if self.batch is not None else self.stream
        dom = cg.Domain(cg.make_params(precision=self.precision, **wl.params()), device=self.device,
                        stream=stream)
        dom.init(*req.fields())
        mass0, _ = dom.mass()
        if self.batch is not None:
            self.batch.add(dom)
            self.batch.set_stop(dom, req.steps)  # it leaves the shared steps at its own count
        return _Run(req, dom, 0, now, mass0)

    def run(self, requests, clock=time.perf_counter) -> dict:
        pending = sorted(requests, key=lambda r: r.arrival)
        active: List[_Run] = []    # advanced by the next quantum
        joining: List[_Run] = []   # admitted while a quantum runs
        results: List[Result] = []
        used = 0
        cell_updates = 0
        t0 = clock()
        i = 0

        def admit(go_on):
            """Admit arrived requests while a slot is free, the workspace fits
            the budget and go_on(number admitted so far) holds."""
            nonlocal i, used
            n = 0
            while i < len(pending) and pending[i].arrival <= clock() - t0 and \
                    len(active) + len(joining) < self.max_active and go_on(n):
                need = cg.cg_workspace_bytes(cg.make_params(precision=self.precision,
                                                            **pending[i].workload().params()))
                cap = self.total_memory - self.reserve
                if self.hbm_budget is not None:
                    cap = min(cap, self.hbm_budget)
                if need > cap:
                    raise ValueError("request %d needs %d bytes of workspace, more than the %d this device "
                                     "can give a run" % (pending[i].rid, need, cap))
                if self.hbm_budget is not None and used + need > self.hbm_budget:
                    break
                if need > self.free_bytes():
                    if not active and not joining:
                        raise RuntimeError("request %d needs %d bytes of workspace and the device has only "
                                           "%d free with no run active" % (pending[i].rid, need,
                                                                           self.free_bytes()))
                    break
                joining.append(self._admit(pending[i], clock() - t0))
                used += need
                i += 1
                n += 1

        while i < len(pending) or active or joining:
            if self.batch is not None:
                start = clock()
                admit(lambda n: n == 0 or clock() - start < ADMIT_SLICE)
            else:
                admit(lambda n: True)
            active += joining
            joining = []
            if not active:
                if i < len(pending):
                    time.sleep(max(0.0, min(0.05, pending[i].arrival - (clock() - t0))))
                continue
            # the quantum ends with the shortest remaining run, rounded up to
            # whole eight-step chains in the batched mode: a member that
            # reaches its own count sits out the rest of the quantum
            shortest = min(r.req.steps - r.done for r in active)
            k = min(self.quantum, -(-shortest // 8) * 8 if self.batch is not None else shortest)
            if self.batch is not None:
                self.batch.step(k)
                # the GPU is busy with the quantum: admit meanwhile
                admit(lambda n: not self.stream.query())
                self.batch.sync()
            else:
                for r in active:
                    r.dom.step(min(k, r.req.steps - r.done))
                self.stream.synchronize()
            for r in active:
                taken = min(k, r.req.steps - r.done)
                r.done += taken
                cell_updates += taken * r.req.cells
            self.log.append((clock() - t0, len(active), k))
            for r in [r for r in active if r.done >= r.req.steps]:
                if self.batch is not None:
                    self.batch.remove(r.dom)
                mass, dp, umax, flag, mac = _summary(r.req, r.dom, self.keep_macros)
                fin = clock() - t0
                results.append(Result(r.req.rid, r.req.edge, r.req.steps, r.req.arrival, r.admitted, fin,
                                      r.mass0, mass, dp, umax, flag, mac))
                active.remove(r)
                used -= r.dom.nbytes
                r.dom.close()
                del r.dom
        wall = clock() - t0
        lat = np.array([r.latency for r in results])
        return {
            "mode": self.mode,
            "runs": len(results),
            "wall_s": wall,
            "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "runs_per_h": 3600.0 * len(results) / wall if wall > 0 else None,
            "MLUPS": cell_updates / wall / 1e6 if wall > 0 else None,
            "cell_updates": cell_updates,
            "max_active": max((a for _, a, _ in self.log), default=0),
            "nonfinite_runs": int(sum(1 for r in results if r.nonfinite)),
            "results": results,
        }

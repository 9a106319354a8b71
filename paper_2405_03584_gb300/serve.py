"""Serving loop: a stream of QP solve requests run with continuous batching on one GPU.

A *plan* is a QP family whose matrices stay resident on the device (an RT plan's dose
matrix D with its organ rows A = D[a_rows], bounds and b); a *request* names a plan and
brings its own factor weights f_w and linear cost c.  A request is either one QP or an
SQP-like chain of related QPs (Section 3.2: the SQP method solves one QP per iteration and
warm-starts it from the previous solution), whose QP k+1 is released when QP k completes.

Execution model (all device work is the library's; this module only schedules):

* slot = one solver handle bound to a plan.  It shares the plan's matrices
  (``ipm_share_qp``) and owns only its state: iterate, PCG and preconditioner work space.
* admission: requests wait in arrival order; a waiting request starts when the number of
  solves in flight is below ``max_inflight`` and its plan has an idle slot, or a new slot's
  state fits in the HBM ledger (``budget_bytes`` minus resident plans and live slots).  Idle
  slots of other plans are freed when the ledger is full.  Requests that cannot start do not
  block those behind them.
* each admitted solve is one asynchronous graph launch ordered on its slot's own CUDA stream
  (never on a stream shared between slots, which would chain every solve after the one
  before), so solves of different requests overlap on the device; completions are polled,
  and a chain keeps its slot (its iterate stays on the device) and continues with a warm
  start.

Results do not depend on what else runs: every solve's arithmetic is fixed by its own inputs
(deterministic reductions, no atomics in floating point, lane counts fixed per plan).
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass

import numpy as np

from . import ipm
from .workloads import request_costs

__all__ = ["Server", "latency_summary"]


@dataclass
class _Job:
    req: dict
    step: int
    t_release: float
    costs: tuple            # (f_w, c, step)


@dataclass
class _Slot:
    solver: ipm.Solver
    plan: int
    state_bytes: int
    stream: object = None   # the slot's own CUDA stream (kept alive with the slot)
    is_plan: bool = False   # the plan's own handle (holds the matrix reference; never freed)

    @property
    def sid(self):
        return getattr(self.stream, "cuda_stream", None)


def _new_stream():
    import torch
    return torch.cuda.Stream()


class Server:
    """Continuous-batching server over resident plans.

    plans: RT-shaped QPs (``workloads.rt_qp`` dicts).  opts: ``ipm_options`` fields for every
    handle (storage, tolerance ...).  warm: warm-start chain QPs from the previous solution.
    """

    solver_cls = ipm.Solver      # the handle type (replaceable by a host-only fake in tests)
    stream_factory = staticmethod(_new_stream)

    def __init__(self, plans, budget_bytes: float = 120e9, max_inflight: int = 16, warm: bool = True,
                 keep_x: bool = False, **opts):
        self.plans = plans
        self.budget = float(budget_bytes)
        self.max_inflight = int(max_inflight)
        self.warm = bool(warm)
        self.keep_x = bool(keep_x)
        self.opts = opts
        self.idle: dict[int, list[_Slot]] = {}
        self.used = 0            # ledger: bytes of resident matrices and live slot states
        self.peak = 0
        self.slots_created = 0
        self.slots_freed = 0
        self.plan_slot: list[_Slot] = []
        for k, p in enumerate(plans):
            st = self.stream_factory()
            s = self.solver_cls(**opts).set_qp_rt(p, stream=getattr(st, "cuda_stream", None))
            b = s.device_bytes()
            self._charge(b["matrix"] + b["state"])
            if self.used > self.budget:
                raise MemoryError("resident plans need %d bytes, over the %d byte budget" % (self.used, self.budget))
            slot = _Slot(s, k, b["state"], stream=st, is_plan=True)
            self.plan_slot.append(slot)
            self.idle[k] = [slot]
        self.state_bytes = [sl.state_bytes for sl in self.plan_slot]

    # ------------------------------------------------------------------ ledger
    def _charge(self, nbytes):
        self.used += int(nbytes)
        self.peak = max(self.peak, self.used)

    def _new_slot(self, plan):
        need = self.state_bytes[plan]
        if self.used + need > self.budget:
            # free idle shared slots of other plans until the new state fits
            for k, lst in self.idle.items():
                while lst and self.used + need > self.budget:
                    victim = next((s for s in lst if not s.is_plan), None)
                    if victim is None:
                        break
                    lst.remove(victim)
                    victim.solver.close()
                    self.used -= victim.state_bytes
                    self.slots_freed += 1
            if self.used + need > self.budget:
                return None
        st = self.stream_factory()
        s = self.solver_cls(**self.opts).share_qp(self.plan_slot[plan].solver, stream=getattr(st, "cuda_stream", None))
        b = s.device_bytes()["state"]
        self._charge(b)
        self.slots_created += 1
        return _Slot(s, plan, b, stream=st)

    def _acquire(self, plan):
        lst = self.idle[plan]
        if lst:
            return lst.pop()
        return self._new_slot(plan)

    # ------------------------------------------------------------------ loop
    def _start(self, slot, job, warm):
        f_w, c, _ = job.costs
        slot.solver.update_costs(f_w=f_w, c=c, stream=slot.sid)
        slot.solver.solve_async(warm=warm, stream=slot.sid)

    def run(self, requests, poll_s: float = 5e-5):
        """Serves ``requests`` (``workloads.serving_stream`` dicts; times in seconds from the
        start of this call) and returns one record per QP solved, plus one per request."""
        reqs = sorted(requests, key=lambda r: r["t"])
        queue: deque[_Job] = deque()
        inflight: dict[int, tuple[_Slot, _Job]] = {}
        qp_records, req_done = [], {}
        t0 = time.perf_counter()
        ai = 0
        busy_s, t_prev, max_conc = 0.0, 0.0, 0
        total_qps = sum(r["steps"] for r in reqs)
        while len(qp_records) < total_qps:
            now = time.perf_counter() - t0
            if inflight:
                busy_s += now - t_prev
            t_prev = now
            busy = False
            while ai < len(reqs) and reqs[ai]["t"] <= now:
                r = reqs[ai]
                queue.append(_Job(r, 0, r["t"], request_costs(self.plans[r["plan"]], r)))
                ai += 1
            # completions
            for key in list(inflight):
                slot, job = inflight[key]
                if not slot.solver.done():
                    continue
                busy = True
                status = slot.solver.wait()
                t_done = time.perf_counter() - t0
                out = slot.solver.get(stream=slot.sid)
                info = out["info"]
                rec = dict(rid=job.req["rid"], step=job.step, plan=slot.plan, t_release=job.t_release,
                           t_done=t_done, latency=t_done - job.t_release, status=int(status),
                           ipm_iters=info["ipm_iters"], cg_iters=info["cg_iters"], rel_kkt=info["rel_kkt"],
                           primal_obj=info["primal_obj"], warm=job.step > 0 and self.warm)
                if self.keep_x:
                    rec["x"] = out["x"].copy()
                qp_records.append(rec)
                del inflight[key]
                if job.step + 1 < job.req["steps"]:
                    nxt = _Job(job.req, job.step + 1, t_done,
                               request_costs(self.plans[slot.plan], job.req, job.costs))
                    self._start(slot, nxt, warm=self.warm)
                    inflight[id(slot)] = (slot, nxt)
                else:
                    req_done[job.req["rid"]] = t_done
                    self.idle[slot.plan].append(slot)
            # admission (arrival order; a request that cannot start lets later ones pass)
            if queue and len(inflight) < self.max_inflight:
                waiting = deque()
                while queue and len(inflight) < self.max_inflight:
                    job = queue.popleft()
                    slot = self._acquire(job.req["plan"])
                    if slot is None:
                        waiting.append(job)
                        continue
                    self._start(slot, job, warm=False)
                    inflight[id(slot)] = (slot, job)
                    busy = True
                waiting.extend(queue)
                queue = waiting
                max_conc = max(max_conc, len(inflight))
            if not busy:
                if not inflight and not queue and ai < len(reqs):
                    time.sleep(max(0.0, min(reqs[ai]["t"] - (time.perf_counter() - t0), 0.01)))
                else:
                    time.sleep(poll_s)
        self.stats = dict(busy_s=busy_s, max_inflight_seen=max_conc, slots_created=self.slots_created,
                          slots_freed=self.slots_freed, ledger_peak_bytes=self.peak, ledger_budget_bytes=self.budget)
        req_records = [dict(rid=r["rid"], plan=r["plan"], steps=r["steps"], t_arrival=r["t"],
                            t_done=req_done[r["rid"]], latency=req_done[r["rid"]] - r["t"]) for r in reqs]
        return qp_records, req_records

    def close(self):
        for lst in self.idle.values():
            for s in lst:
                s.solver.close()
        self.idle = {}


def latency_summary(qp_records, req_records, horizon, busy_s=None):
    """Throughput and latency percentiles of a served stream.  With the time some solve was
    in flight (``busy_s``), capacity = QPs / busy time and rho = offered rate / capacity."""
    lat = np.array([r["latency"] for r in qp_records])
    chains = np.array([r["latency"] for r in req_records if r["steps"] > 1])
    singles = np.array([r["latency"] for r in req_records if r["steps"] == 1])
    t_end = max(r["t_done"] for r in qp_records)
    t_first = min(r["t_arrival"] for r in req_records)
    n = len(qp_records)
    pct = lambda a, q: float(np.percentile(a, q)) * 1e3 if a.size else None
    out = dict(qps=n, requests=len(req_records), makespan_s=t_end - t_first,
               solves_per_s=n / (t_end - t_first), offered_qp_per_s=n / horizon,
               p50_ms=pct(lat, 50), p99_ms=pct(lat, 99),
               single_p50_ms=pct(singles, 50), single_p99_ms=pct(singles, 99),
               chain_p50_ms=pct(chains, 50), chain_p99_ms=pct(chains, 99),
               ipm_iters_cold=float(np.mean([r["ipm_iters"] for r in qp_records if not r["warm"]] or [0])),
               ipm_iters_warm=float(np.mean([r["ipm_iters"] for r in qp_records if r["warm"]] or [0])),
               max_rel_kkt=float(max(r["rel_kkt"] for r in qp_records)),
               not_ok=int(sum(r["status"] != 0 for r in qp_records)))
    if busy_s:
        out["busy_s"] = busy_s
        out["capacity_qp_per_s"] = n / busy_s
        out["rho"] = out["offered_qp_per_s"] / out["capacity_qp_per_s"]
    return out

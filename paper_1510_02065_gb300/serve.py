"""Continuous-batching server for RLT2 bound requests.

Requests (an instance F, D and a number of passes) arrive over time.  The
server admits them in arrival order while their device state fits a memory
budget (rlt2_state_bytes) and a slot limit, keeps each admitted request's dual
state resident on the GPU, and advances all resident requests together: every
round is `passes_per_round` passes of one group (rlt2_group_*), so the work of
requests of different sizes shares the same kernel launches.  Between rounds
finished requests leave (their bound is read and their memory released) and
waiting ones join: the group is rebuilt whenever its membership changes.
Each result equals that of the request bounded alone (same passes, same
arithmetic).  A request can be cancelled (cancel(rid), from any thread, or
cancel_after passes for a client that gives up mid-run): it leaves at the
next round boundary with its memory released and error "cancelled".

All device work runs through the C ABI (librlt2.so); this module only
schedules.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time
from typing import List, Optional

import numpy as np

from . import rlt2


@dataclasses.dataclass
class Request:
    rid: int
    F: np.ndarray
    D: np.ndarray
    iters: int
    arrival: float = 0.0            # seconds after the start of serve()
    B_lin: Optional[np.ndarray] = None
    lb_const: int = 0
    cancel_after: Optional[int] = None   # cancel once this many passes are done
    # filled in by the server
    lb: Optional[int] = None
    admitted: Optional[float] = None
    done: Optional[float] = None
    error: Optional[str] = None

    @property
    def N(self) -> int:
        return int(np.asarray(self.F).shape[0])

    @property
    def latency(self) -> Optional[float]:
        return None if self.done is None else self.done - self.arrival


class BoundServer:
    """Admit by memory, bound in shared launches, release on completion."""

    def __init__(self, mem_budget: int, max_slots: int = 64, passes_per_round: int = 1,
                 stream: int = 0, store: int = rlt2.RLT2_STORE_TILES):
        self.store = int(store)
        self.mem_budget = int(mem_budget)
        self.max_slots = int(max_slots)
        self.passes_per_round = max(1, int(passes_per_round))
        self.stream = stream
        self.peak_bytes = 0
        self.rounds = 0
        self.slot_rounds = 0
        self._cancelled = set()
        self._lock = threading.Lock()

    def cancel(self, rid: int) -> None:
        """Cancel request rid (queued or running); effective at the next round boundary."""
        with self._lock:
            self._cancelled.add(rid)

    def _is_cancelled(self, req: Request, done: int = 0) -> bool:
        with self._lock:
            if req.rid in self._cancelled:
                return True
        return req.cancel_after is not None and done >= req.cancel_after

    def _bytes(self, req: Request) -> int:
        return rlt2.rlt2_state_bytes(req.N, False, req.iters + 1, self.store)

    def serve(self, requests: List[Request], realtime: bool = True) -> dict:
        """Serve every request; returns latency / throughput statistics.

        realtime=True waits for arrivals on the wall clock; False admits a
        request as soon as the server is idle or at the first round that
        starts after its arrival time measured in rounds (for tests).
        """
        future = collections.deque(sorted(requests, key=lambda r: r.arrival))
        pending: collections.deque = collections.deque()
        active = []       # [request, context, passes done]
        used = 0
        group = None
        changed = False
        t0 = time.perf_counter()
        now = (lambda: time.perf_counter() - t0) if realtime else (lambda: float(self.rounds))
        finished = []
        while future or pending or active:
            t = now()
            while future and (future[0].arrival <= t or (not realtime and not active and not pending)):
                pending.append(future.popleft())
            for req in [r for r in pending if self._is_cancelled(r)]:
                pending.remove(req)
                req.error = "cancelled"
                finished.append(req)
            while pending and len(active) < self.max_slots:
                req = pending[0]
                need = self._bytes(req)
                if need > self.mem_budget:
                    pending.popleft()
                    req.error = "needs %d bytes, more than the budget" % need
                    finished.append(req)
                    continue
                if used + need > self.mem_budget:
                    break
                pending.popleft()
                try:
                    ctx = rlt2.Context(req.F, req.D, B_lin=req.B_lin, lb_const=req.lb_const,
                                       max_iters=req.iters + 1, stream=self.stream, store=self.store)
                except rlt2.Rlt2Error as e:
                    req.error = str(e)
                    finished.append(req)
                    continue
                req.admitted = now()
                used += need
                self.peak_bytes = max(self.peak_bytes, used)
                active.append([req, ctx, 0])
                changed = True
            if not active:
                if future and realtime:
                    time.sleep(max(0.0, min(0.05, future[0].arrival - now())))
                continue
            if changed:
                if group is not None:
                    rlt2.rlt2_group_destroy(group)
                group = rlt2.rlt2_group_create([a[1].ctx for a in active], self.stream)
                changed = False
            k = min(self.passes_per_round, min(a[0].iters - a[2] for a in active))
            for a in active:               # stop at a client's cancellation point
                if a[0].cancel_after is not None and a[2] < a[0].cancel_after:
                    k = min(k, a[0].cancel_after - a[2])
            if k > 0:
                rlt2.rlt2_group_iterate(group, k)
                rlt2.rlt2_group_sync(group)
            self.rounds += 1
            self.slot_rounds += len(active)
            leaving = []
            for a in active:
                a[2] += k
                if a[2] >= a[0].iters or self._is_cancelled(a[0], a[2]):
                    leaving.append(a)
            if leaving:
                rlt2.rlt2_group_destroy(group)
                group = None
                changed = True
                for a in leaving:
                    req, ctx = a[0], a[1]
                    if a[2] >= req.iters:
                        req.lb = ctx.bound()[1]
                    else:
                        ctx.bound()          # surfaces a device error, if any
                        req.error = "cancelled"
                    req.done = now()
                    ctx.close()
                    used -= self._bytes(req)
                    active.remove(a)
                    finished.append(req)
        if group is not None:
            rlt2.rlt2_group_destroy(group)
        span = now()
        lat = np.array([r.latency for r in finished if r.latency is not None])
        ok = [r for r in finished if r.error is None]
        return {
            "requests": len(requests), "completed": len(ok),
            "rejected": len(finished) - len(ok),
            "makespan": span,
            "throughput": len(ok) / span if span > 0 else None,
            "p50_latency": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_latency": float(np.percentile(lat, 99)) if lat.size else None,
            "mean_resident": self.slot_rounds / self.rounds if self.rounds else 0.0,
            "peak_bytes": self.peak_bytes, "rounds": self.rounds,
        }


def serve_sharded(server: "BoundServer", requests: List[Request], group=None, realtime: bool = True) -> dict:
    """One server per rank (one process per GPU): this rank serves its
    round-robin share of `requests` (distributed.shard by position) with
    `server`, and every request's result, (LB, error), is gathered on every
    rank in the original order.  The requests are independent, so no
    collective touches the bounding; the gather is the only exchange."""
    import torch.distributed as dist

    from .distributed import gather_results, shard

    rank, world = dist.get_rank(group), dist.get_world_size(group)
    mine = shard(requests, rank, world)
    stats = server.serve([r for _, r in mine], realtime=realtime)
    local = [(i, (r.lb, r.error)) for i, r in mine]
    results = gather_results(local, len(requests), group)
    parts = [None] * world
    dist.all_gather_object(parts, stats, group=group)
    return {"results": results, "per_rank": parts, "ranks": world}

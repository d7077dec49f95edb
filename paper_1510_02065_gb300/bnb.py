"""Branch-and-bound for the QAP on the RLT2 dual-ascent bound (Sec. 6).

The paper solves QAP instances by branch-and-bound with the RLT2 bound of
every node computed on the GPU, a node being a partial assignment of
facilities to locations.  This driver does the same on one GPU:

* depth-first search; a node fixes k facility/location pairs; its children
  assign the branching facility to each free location;
* all children of a node are bounded together by one rlt2_batch_bound call
  (their residual instances, Sec. 3, cold start), with the incumbent UB as
  the stopping rule of Algorithm 1 (a child's dual ascent stops as soon as
  LB >= UB, and such a child is pruned);
* branching facility: near the root, strong branching on the RLT1 bound
  (Algorithm 1 without D, as in the paper): the free facility whose children
  have the largest least RLT1 bound; deeper, the free facility of largest
  total flow;
* nodes with at most `enum_size` free facilities are completed by exhaustive
  enumeration on the host;
* the initial UB comes from pairwise-exchange local search from a few seeded
  random permutations (the paper's UB heuristic is not specified);
* warm=True: a node keeps its context, and its children start from its dual
  state (rlt2_child: the state restricted to the child's fixed pair) instead
  of cold residual instances; the children of a node are advanced together
  as one group (rlt2_group_*), each stopping once its bound reaches the UB.

Children are visited in increasing order of their bound.  With integer costs
a node whose bound reaches the incumbent cannot contain a better solution.

Several GPUs (one process each, as the paper runs one host thread per GPU
with its own subtrees): with a torch.distributed process group, every rank
expands the top of the tree the same way (deterministic: the bounds are bit
for bit the same on every GPU) until there are at least `frontier_per_rank`
subtrees per rank, deals them round-robin (distributed.shard) and searches
its own on its own GPU.  Every `sync_every` nodes the ranks exchange the
incumbent (an all-reduce of one integer, the minimum) and whether any of them
has work left; nothing else crosses ranks, and no collective touches the
bounding itself.  At the end the optimum, its permutation and the counters
are gathered.

All bounding runs through the C ABI (librlt2.so); this module only schedules.
"""
from __future__ import annotations

import itertools
import time
from typing import List, Optional, Tuple

import numpy as np

from . import rlt2


def qap_cost(F: np.ndarray, D: np.ndarray, perm: np.ndarray) -> int:
    """sum_{i != k} F[i,k] D[perm i, perm k] (diagonal terms excluded)."""
    F64, D64 = F.astype(np.int64), D.astype(np.int64)
    Dp = D64[np.ix_(perm, perm)]
    return int((F64 * Dp).sum() - (np.diag(F64) * np.diag(Dp)).sum())


def local_search_ub(F: np.ndarray, D: np.ndarray, starts: int = 8, seed: int = 0) -> Tuple[int, np.ndarray]:
    """Best pairwise-exchange local optimum over `starts` random permutations."""
    N = F.shape[0]
    rng = np.random.default_rng(seed)
    best, best_p = None, None
    for _ in range(starts):
        p = rng.permutation(N)
        c = qap_cost(F, D, p)
        improved = True
        while improved:
            improved = False
            for a in range(N):
                for b in range(a + 1, N):
                    p[a], p[b] = p[b], p[a]
                    c2 = qap_cost(F, D, p)
                    if c2 < c:
                        c, improved = c2, True
                    else:
                        p[a], p[b] = p[b], p[a]
        if best is None or c < best:
            best, best_p = c, p.copy()
    return best, best_p


class BranchAndBound:
    """Exact QAP solver: depth-first branch-and-bound on batched RLT2 bounds."""

    def __init__(self, F, D, iters: int = 12, root_iters: int = 30, strong_depth: int = 1,
                 strong_iters: int = 3, enum_size: int = 3, ub: Optional[int] = None,
                 node_limit: int = 1_000_000, store: int = rlt2.RLT2_STORE_TILES, warm: bool = False,
                 group=None, sync_every: int = 16, frontier_per_rank: int = 2):
        self.F = np.ascontiguousarray(F, np.int32)
        self.D = np.ascontiguousarray(D, np.int32)
        self.N = self.F.shape[0]
        self.iters = iters
        self.root_iters = root_iters
        self.strong_depth = strong_depth
        self.strong_iters = strong_iters
        self.enum_size = max(1, enum_size)
        self.node_limit = node_limit
        self.store = store
        self.warm = warm
        self.ub0 = ub
        self.group = group
        self.sync_every = max(1, sync_every)
        self.frontier_per_rank = max(1, frontier_per_rank)
        self.stats = dict(nodes_bounded=0, nodes_pruned=0, leaves_enumerated=0, batches=0,
                          strong_evaluations=0)

    # -- bounds -----------------------------------------------------------
    def _children_bounds(self, fac: List[int], loc: List[int], f: int, free_locs: List[int]) -> List[int]:
        nodes = [(np.array(fac + [f], np.int32), np.array(loc + [l], np.int32)) for l in free_locs]
        lbs, _ = rlt2.rlt2_batch_bound(self.F, self.D, nodes, self.iters, store=self.store, ub=float(self.ub))
        self.stats["batches"] += 1
        self.stats["nodes_bounded"] += len(nodes)
        return [int(x) for x in lbs]

    def _children_warm(self, ctx, free_facs, free_locs, f) -> List[Tuple[int, object]]:
        """Children of the node held by ctx, warm-started from its dual state and
        advanced `iters` passes together; returns (bound, context) per location."""
        fl = free_facs.index(f)
        kids = []
        try:
            for x in range(len(free_locs)):
                kids.append(ctx.child(fl, x, ub=float(self.ub), max_iters=self.iters + 1))
            grp = rlt2.rlt2_group_create([k.ctx for k in kids])
            try:
                rlt2.rlt2_group_iterate(grp, self.iters)
                rlt2.rlt2_group_sync(grp)
            finally:
                rlt2.rlt2_group_destroy(grp)
        except BaseException:
            for k in kids:      # each holds a store of D on the device
                k.close()
            raise
        self.stats["batches"] += 1
        self.stats["nodes_bounded"] += len(kids)
        return [(k.bound()[1], k) for k in kids]

    def _rlt1_child_min(self, fac, loc, f, free_locs) -> int:
        best = None
        for l in free_locs:
            Fp, Dp, Bl, cst = rlt2.rlt2_subproblem(self.F, self.D, np.array(fac + [f]), np.array(loc + [l]))
            if Fp.shape[0] < rlt2.RLT2_MIN_N:
                return 0
            with rlt2.Context(Fp, Dp, B_lin=Bl, lb_const=cst, rlt1_only=True,
                              max_iters=self.strong_iters + 1) as c:
                c.iterate(self.strong_iters)
                v = c.bound()[1]
            self.stats["strong_evaluations"] += 1
            best = v if best is None else min(best, v)
        return best

    def _branch_facility(self, fac, loc, free_facs, free_locs) -> int:
        if len(fac) < self.strong_depth and len(free_facs) > self.enum_size + 1:
            scores = [(self._rlt1_child_min(fac, loc, f, free_locs), f) for f in free_facs]
            return max(scores)[1]
        flow = self.F.astype(np.int64).sum(1) + self.F.astype(np.int64).sum(0)
        return max(free_facs, key=lambda f: (flow[f], -f))

    # -- leaves -----------------------------------------------------------
    def _enumerate(self, fac, loc, free_facs, free_locs):
        self.stats["leaves_enumerated"] += 1
        perm = np.empty(self.N, np.int64)
        perm[fac] = loc
        for tail in itertools.permutations(free_locs):
            perm[free_facs] = tail
            c = qap_cost(self.F, self.D, perm)
            if c < self.ub:
                self.ub, self.best = c, perm.copy()

    # -- search -----------------------------------------------------------
    def _expand(self, lb, fac, loc, ctx, stack) -> int:
        """Process one node; push its surviving children.  Returns 1 if the node
        counted as visited (its bound was still below the incumbent)."""
        if lb >= self.ub:          # the incumbent improved since the node was queued
            self.stats["nodes_pruned"] += 1
            return 0
        free_facs = [f for f in range(self.N) if f not in fac]
        free_locs = [l for l in range(self.N) if l not in loc]
        if len(free_facs) <= self.enum_size:
            self._enumerate(fac, loc, free_facs, free_locs)
            return 1
        f = self._branch_facility(fac, loc, free_facs, free_locs)
        if len(free_facs) - 1 < rlt2.RLT2_MIN_N:
            # children too small for the bound: enumerate them
            for l in free_locs:
                ff = [x for x in free_facs if x != f]
                ll = [x for x in free_locs if x != l]
                self._enumerate(fac + [f], loc + [l], ff, ll)
            return 1
        if self.warm and ctx is not None:
            kids = [(b, l, k) for (b, k), l in zip(self._children_warm(ctx, free_facs, free_locs, f), free_locs)]
        else:
            kids = [(b, l, None) for b, l in zip(self._children_bounds(fac, loc, f, free_locs), free_locs)]
        kids.sort(key=lambda x: -x[0])   # popped in increasing bound order
        for b, l, k in kids:
            if b >= self.ub:
                self.stats["nodes_pruned"] += 1
                if k is not None:
                    k.close()
                continue
            stack.append((b, fac + [f], loc + [l], k))
        return 1

    def solve(self) -> dict:
        if self.group is not None:
            return self._solve_distributed()
        t0 = time.perf_counter()
        if self.ub0 is not None:
            self.ub, self.best = int(self.ub0), None
        else:
            self.ub, self.best = local_search_ub(self.F, self.D)
        ub_initial = self.ub
        root = rlt2.Context(self.F, self.D, ub=float(self.ub), max_iters=self.root_iters + 1, store=self.store)
        root.iterate(self.root_iters)
        root_lb = root.bound()[1]
        if not self.warm:
            root.close()
            root = None
        stack = [(root_lb, [], [], root)] if root_lb < self.ub else []
        if not stack and root is not None:
            root.close()
        visited = 0
        try:
            while stack and visited < self.node_limit:
                lb, fac, loc, ctx = stack.pop()
                try:
                    visited += self._expand(lb, fac, loc, ctx, stack)
                finally:
                    if ctx is not None:
                        ctx.close()
        finally:
            for entry in stack:
                if entry[3] is not None:
                    entry[3].close()
        return dict(optimum=self.ub, perm=self.best, proven=not stack, root_lb=root_lb, warm=self.warm,
                    ub_initial=ub_initial, nodes_visited=visited, seconds=time.perf_counter() - t0,
                    **self.stats)

    # -- several ranks ------------------------------------------------------
    def _solve_distributed(self) -> dict:
        """The search over the ranks of self.group (see the module docstring)."""
        import torch
        import torch.distributed as dist

        from .distributed import shard

        if self.warm:
            raise ValueError("the distributed search starts every subtree cold")
        t0 = time.perf_counter()
        rank, world = dist.get_rank(self.group), dist.get_world_size(self.group)
        if self.ub0 is not None:
            self.ub, self.best = int(self.ub0), None
        else:
            self.ub, self.best = local_search_ub(self.F, self.D)   # the same on every rank
        ub_initial = self.ub
        with rlt2.Context(self.F, self.D, ub=float(self.ub), max_iters=self.root_iters + 1,
                          store=self.store) as root:
            root.iterate(self.root_iters)
            root_lb = root.bound()[1]
        # the top of the tree, expanded alike on every rank (breadth first)
        frontier = [(root_lb, [], [], None)] if root_lb < self.ub else []
        visited = 0
        while frontier and len(frontier) < self.frontier_per_rank * world:
            nxt = []
            expandable = False
            for lb, fac, loc, _ in frontier:
                if self.N - len(fac) <= self.enum_size + 1:
                    nxt.append((lb, fac, loc, None))
                    continue
                expandable = True
                visited += self._expand(lb, fac, loc, None, nxt)
            frontier = nxt
            if not expandable:
                break
        frontier.sort(key=lambda x: (x[0], x[1], x[2]))
        mine = [node for _, node in shard(frontier, rank, world)]
        stack = sorted(mine, key=lambda x: -x[0])      # popped in increasing bound order
        top = dict(self.stats)
        for k in self.stats:
            self.stats[k] = 0      # the search below counts this rank's own work
        local = 0
        # the incumbent exchange: NCCL reduces device tensors, gloo host ones
        dev = "cuda" if dist.get_backend(self.group) == "nccl" else "cpu"
        buf = torch.zeros(2, dtype=torch.int64, device=dev)
        while True:
            n = 0
            while stack and n < self.sync_every and visited + local < self.node_limit:
                lb, fac, loc, _ = stack.pop()
                local += self._expand(lb, fac, loc, None, stack)
                n += 1
            # incumbent and remaining work across the ranks
            buf[0] = self.ub
            dist.all_reduce(buf[:1], op=dist.ReduceOp.MIN, group=self.group)
            self.ub = min(self.ub, int(buf[0]))
            buf[1] = 1 if (stack and visited + local < self.node_limit) else 0
            dist.all_reduce(buf[1:], op=dist.ReduceOp.MAX, group=self.group)
            if int(buf[1]) == 0:
                break
        parts = [None] * world
        mine_best = None if self.best is None else [int(x) for x in self.best]
        dist.all_gather_object(parts, dict(perm=mine_best, proven=not stack, nodes=local,
                                           stats=dict(self.stats)), group=self.group)
        # the incumbent (the minimum over the ranks after the last exchange) and
        # a permutation of that cost found by some rank (none if it is ub0's)
        perm = None
        for part in parts:
            if part["perm"] is not None and qap_cost(self.F, self.D, np.array(part["perm"])) == self.ub:
                perm = np.array(part["perm"])
                break
        stats = {k: top[k] + sum(part["stats"][k] for part in parts) for k in top}
        return dict(optimum=self.ub, perm=perm, proven=all(part["proven"] for part in parts),
                    root_lb=root_lb, warm=False, ub_initial=ub_initial,
                    nodes_visited=visited + sum(part["nodes"] for part in parts),
                    seconds=time.perf_counter() - t0, ranks=world,
                    nodes_per_rank=[part["nodes"] for part in parts], **stats)


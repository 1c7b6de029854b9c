"""Literal simulation of the 1D swept rule on tiny periodic grids.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).  Pure Python, for grids of
a few dozen points.

This follows the stages of Section 3 directly, without assuming any shape:

* the periodic grid of N points is split uniformly among P nodes, each node
  owning B = N/P consecutive points (Section 3 asks for an even count; with a
  stencil of radius r the count is a multiple of 2r);
* each node alternates between two sets of points (Section 3): in odd
  stages the B points it owns, in even stages the B points shifted by B/2
  to the right (half its own, half its right neighbour's);
* in every computing stage each node computes *everything it can* on its
  current set from the values it holds: the output of a sub-timestep at
  point x is computable once the node holds the inputs at x-r..x+r one level
  below (the domain of dependence, Section 2).  Nothing else decides what is
  computed, so the triangle of the first stage and the diamonds of later
  stages are not built in; they come out of this rule;
* after computing stage k (k = 1, 2, ...) every node sends to one neighbour
  the values it holds that the neighbour's next set can read (that set
  widened by the stencil radius): to the left after odd-numbered stages and to the right after
  even-numbered stages (Section 3, the alternating send direction).  Of a
  message the receiver reads only the leading edge; the trace records which
  values were read.

Computation stops at the requested level ``nsteps``.  The simulation records
how often every space-time value was computed (the swept rule computes each
exactly once) and which received values each node actually read (the paper's
leading edge: two values per sub-timestep level for a 3-point stencil, 2r in
general).
"""
from __future__ import annotations

import numpy as np

from dataclasses import dataclass, field

from .pointwise import make_point_update


@dataclass
class SweptTrace:
    u_final: list
    compute_count: dict            # (x, t) -> number of times computed
    stages: int
    # per stage k (1-based), per node: {level: sorted list of x read from received data}
    reads: list = field(default_factory=list)
    # per stage k, per node: number of values computed
    computed: list = field(default_factory=list)


def swept_simulate(stencil: int, params, u0, P: int, nsteps: int, max_stages: int = 100000):
    """Run the swept stages on P nodes until level ``nsteps`` is known everywhere.

    ``nsteps`` counts sub-timesteps (levels); a two-stage Runge-Kutta time step
    is two of them.
    """
    radius, f = make_point_update(stencil, params)
    N = len(u0)
    if P < 1 or N % P:
        raise ValueError("N must split uniformly among the nodes")
    B = N // P
    if B % (2 * radius):
        raise ValueError("points per node must be a multiple of 2r")
    # store[j]: (x, t) -> (value, origin); origin 'own' or ('recv', stage)
    store = [dict() for _ in range(P)]
    pair = stencil in (2, 3)            # two-stage Runge-Kutta: (u, m) per point
    euler = stencil == 4                # Euler: (q, q_mid, slopes), q = u0[x] (3 values)
    euler32 = stencil == 5              # compensated FP32 Euler: u0[x] = (hi(3), lo(3)) float32
    for j in range(P):
        for x in range(j * B, (j + 1) * B):
            if euler:
                q = tuple(float(c) for c in u0[x])
                v = q + q + (0.0, 0.0, 0.0)
            elif euler32:
                h = tuple(np.float32(c) for c in u0[x][:3])
                lo = tuple(np.float32(c) for c in u0[x][3:6])
                v = h + lo + h + (np.float32(0.0),) * 3
            else:
                v0 = float(u0[x])
                v = (v0, v0) if pair else v0
            store[j][(x, 0)] = (v, "own")
    count: dict = {}
    trace = SweptTrace(u_final=[], compute_count=count, stages=0)

    def known_final():
        have = set()
        for j in range(P):
            for (x, t) in store[j]:
                if t == nsteps:
                    have.add(x)
        return len(have) == N

    def point_set(j, stage_k):
        start = j * B if stage_k % 2 == 1 else j * B + B // 2
        return {(start + i) % N for i in range(B)}

    stage = 0
    idle = 0
    while not known_final():
        stage += 1
        if stage > max_stages:
            raise RuntimeError("swept simulation did not terminate")
        stage_reads = []
        stage_computed = []
        for j in range(P):
            S = store[j]
            mine = point_set(j, stage)
            reads: dict = {}
            ncomp = 0
            for t in range(nsteps):          # level t -> t+1, ascending
                for x in sorted(mine):
                    if (x, t + 1) in S:
                        continue
                    keys = [((x + k) % N, t) for k in range(-radius, radius + 1)]
                    if not all(k in S for k in keys):
                        continue
                    vals = []
                    for k in keys:
                        v, origin = S[k]
                        vals.append(v)
                        if origin != "own":
                            reads.setdefault(k[1], set()).add(k[0])
                    S[(x, t + 1)] = (f(vals, t), "own")
                    count[(x, t + 1)] = count.get((x, t + 1), 0) + 1
                    ncomp += 1
            stage_reads.append({lvl: sorted(xs) for lvl, xs in reads.items()})
            stage_computed.append(ncomp)
        # communication after stage k: odd -> to the left, even -> to the right.
        # Messages are assembled from the senders' state before any delivery.
        outbox = []
        for j in range(P):
            dest = (j - 1) % P if stage % 2 == 1 else (j + 1) % P
            if dest == j:
                continue
            # what the neighbour can use next: its next set widened by the
            # stencil radius (its outermost points read r neighbours beyond it)
            nxt = point_set(dest, stage + 1)
            reach = {(x + k) % N for x in nxt for k in range(-radius, radius + 1)}
            msg = {key: v for key, (v, _) in store[j].items() if key[0] in reach}
            outbox.append((dest, msg))
        for dest, msg in outbox:
            for key, v in msg.items():
                if key not in store[dest]:
                    store[dest][key] = (v, ("recv", stage))
        trace.reads.append(stage_reads)
        trace.computed.append(stage_computed)
        idle = idle + 1 if all(c == 0 for c in stage_computed) else 0
        if idle >= 2 and not known_final():
            raise RuntimeError("swept simulation stalled")
    trace.stages = stage
    final = [None] * N
    for j in range(P):
        for (x, t), (v, _) in store[j].items():
            if t == nsteps and final[x] is None:
                final[x] = v[0] if pair else (v[:3] if euler else (v[:6] if euler32 else v))
    trace.u_final = final
    return trace

"""One periodic problem sharded over nodes: the swept rule of Section 3 with a GPU as the node.

Each of G ranks owns a contiguous slice of N/G points (a whole number of tiles
of B points) and runs the library's stage kernels on its own windows, which
wrap around the slice as if it were the whole periodic grid.  Section 3's
alternation makes that exact with one message per stage:

* after an unshifted stage (k even; windows [jB, jB+B)) the next stage's
  window that straddles the slice's right end reads, as its right arm, the
  left leading edges of the first window of the slice on the right.  So each
  rank sends the left edge half of its window 0 (h levels x 2r values = B
  edge elements) to its left neighbour and receives its right neighbour's
  into the same slot, which no window of its own reads;
* after a shifted stage (k odd; windows [jB + B/2, ...)) the next stage's
  first window reads, as its left arm, the right leading edges of the window
  that straddles the boundary on its left, which the left neighbour computed.
  So each rank sends the right edge half of its last window to its right
  neighbour and receives its left neighbour's into the same slot;
* the stages that store the final flat state: a straddling window of an odd
  stage stores the head of the next slice, which the local wrap puts at the
  head of this slice.  One last message moves those points (at most B/2) to
  the right neighbour, which holds the left neighbour's in return.

Nothing else crosses a slice boundary: every other window of every stage lies
inside its slice.  The FP64 reductions (the sum, J = 1/2 sum u^2, <g, v>) are the
one collective: each rank reduces its slice and the ranks all-gather the
partials, which every rank adds with one rounding (``sharded_reduce``), so all
ranks hold the same bits whatever the order the partials arrive in.  Per stage a rank sends B edge elements to one neighbour
(8 KB for FP64 at B = 1024), so the network latency is paid once per h
sub-timesteps (Section 4, Eq. 1).  No collective and no load from another
GPU's memory is needed: on GPUs the messages are NCCL send/recv pairs.

Every wait for a message has a time budget; a message that does not arrive in
time ends the advance with SWEPT_ETIMEOUT (the state is then undefined and the
process group holds unmatched operations: destroy it before reusing the
ranks).

The stages run through a runner (``PlanRunner`` for a GPU plan over the slice,
through the C ABI's swept_stage and swept_edge_copy) and the messages through
a transport (``TorchDistTransport``: torch.distributed isend/irecv, gloo or
NCCL).  ``ShardedAdvance.program()`` is the rank's schedule as a generator that
yields at every exchange, so one process can also interleave several slices.
"""
from __future__ import annotations

import time

SWEPT_OK = 0
SWEPT_ETIMEOUT = -4


def schedule(levels: int, h: int):
    """swept_advance's stages (k, hv, ht) for ``levels`` sub-timesteps of tiles of h levels:
    a triangle, q - 1 diamonds, the last fill with a trapezoid of the remainder, and that
    trapezoid's fill (q = levels // h); below h levels a trapezoid and its fill."""
    if levels <= 0:
        return []
    q, rem = divmod(levels, h)
    if q == 0:
        return [(0, 0, rem), (1, rem, 0)]
    out = [(0, 0, h)] + [(k, h, h) for k in range(1, q)] + [(q, h, rem)]
    if rem:
        out.append((q + 1, rem, 0))
    return out


def wrapped_head(levels: int, h: int, B: int, r: int) -> int:
    """How many points at the head of a slice hold the right neighbour's values after the
    last stages: the straddling window of the odd one of them stores the head of the next
    slice there (windows of an odd stage start B/2 into a tile).  With levels = q h + rem:
    rem = 0 and q odd: the whole half window, B/2; rem > 0 and q odd: the top of the last
    trapezoid past the boundary, B/2 - r rem; q even: the fill of height rem past the
    boundary, r rem (none when rem = 0)."""
    if levels <= 0:
        return 0
    q, rem = divmod(levels, h)
    if rem == 0:
        return B // 2 if q % 2 == 1 else 0
    if q % 2 == 1:
        return B // 2 - r * rem
    return r * rem


class Slice:
    """Rank ``rank`` of ``world`` owns points [start, start + n_local) of the periodic grid."""

    def __init__(self, N: int, B: int, world: int, rank: int):
        if world < 1 or not 0 <= rank < world:
            raise ValueError("bad rank or world size")
        if N % world or (N // world) % B:
            raise ValueError(f"N = {N} does not split into {world} slices of whole tiles of {B}")
        self.N, self.B, self.world, self.rank = N, B, world, rank
        self.n_local = N // world
        self.nwin = self.n_local // B
        self.start = rank * self.n_local
        self.left = (rank - 1) % world
        self.right = (rank + 1) % world


class _Pending:
    """A posted exchange: resumes the program when its messages are in."""

    def __init__(self, handle, after):
        self.handle, self.after = handle, after

    def done(self) -> bool:
        return self.handle.done()

    def wait(self, timeout_s: float) -> bool:
        return self.handle.wait(timeout_s)


class ShardedAdvance:
    """One rank's part of a swept advance of ``levels`` sub-timesteps over a sharded problem."""

    def __init__(self, runner, transport, sl: Slice, h: int, radius: int, levels: int,
                 timeout_s: float = 30.0, tag_base: int = 0):
        self.runner, self.transport, self.slice = runner, transport, sl
        self.h, self.r, self.levels = h, radius, levels
        self.timeout_s = timeout_s
        self.tag_base = tag_base
        self.messages = 0            # messages this rank sent

    def _exchange(self, send_buf, dst, recv_buf, src, tag, after):
        self.messages += 1
        handle = self.transport.post(send_buf, dst, recv_buf, src, self.tag_base + tag)
        return _Pending(handle, after)

    def program(self):
        """The rank's schedule; yields a pending exchange wherever it needs a neighbour's message."""
        sl, run = self.slice, self.runner
        stages = schedule(self.levels, self.h)
        for i, (k, hv, ht) in enumerate(stages):
            run.stage(k, hv, ht)
            if sl.world == 1 or i + 1 == len(stages):
                continue
            if k % 2 == 0:
                # the next stage's straddling window reads the right neighbour's window-0 left edges
                w, side, dst, src = 0, 0, sl.left, sl.right
            else:
                # the next stage's first window reads the left neighbour's straddler's right edges
                w, side, dst, src = sl.nwin - 1, 1, sl.right, sl.left
            out = run.get_edge(k, w, side)
            into = run.new_edge()
            yield self._exchange(out, dst, into, src, 2 * k,
                                 lambda k=k, w=w, side=side, into=into: run.put_edge(k, w, side, into))
        n = wrapped_head(self.levels, self.h, sl.B, self.r)
        if sl.world > 1 and n > 0:
            out = run.get_head(n)
            into = run.new_head(n)
            yield self._exchange(out, sl.right, into, sl.left, 2 * len(stages) + 1,
                                 lambda: run.put_head(n, into))

    def run(self) -> int:
        """Run the program to the end, waiting at most ``timeout_s`` for each message.
        Returns SWEPT_OK or SWEPT_ETIMEOUT (a message that did not arrive in time, or a peer
        whose connection closed)."""
        for pending in self.program():
            if not pending.wait(self.timeout_s):
                return SWEPT_ETIMEOUT
            pending.after()
        return SWEPT_OK


def drive_in_process(programs, timeout_s: float = 30.0, poll_s: float = 1e-4) -> int:
    """Run several ranks' programs in one process, round-robin: each runs until it waits for a
    message, and resumes once that message is in.  SWEPT_ETIMEOUT if some wait outlasts
    ``timeout_s`` with nothing else able to move."""
    waiting = {}
    active = list(range(len(programs)))
    for i in active:
        waiting[i] = next(programs[i], None)
    deadline = time.monotonic() + timeout_s
    while any(p is not None for p in waiting.values()):
        moved = False
        for i, p in list(waiting.items()):
            if p is not None and p.done():
                p.after()
                waiting[i] = next(programs[i], None)
                moved = True
        if moved:
            deadline = time.monotonic() + timeout_s
        elif time.monotonic() > deadline:
            return SWEPT_ETIMEOUT
        else:
            time.sleep(poll_s)
    return SWEPT_OK


# ------------------------------------------------------------------ transports
class _TorchHandle:
    """The send and receive of one exchange.  gloo reports a point-to-point operation's
    completion only through its wait, which takes a time budget; an NCCL wait orders the
    caller's stream and returns, and completion is then polled within the same budget."""

    def __init__(self, works):
        self.works = works

    def done(self) -> bool:
        return all(w.is_completed() for w in self.works)

    def wait(self, timeout_s: float, poll_s: float = 1e-4) -> bool:
        import datetime
        deadline = time.monotonic() + timeout_s
        for w in self.works:
            left = deadline - time.monotonic()
            if left <= 0:
                return False
            try:
                w.wait(timeout=datetime.timedelta(seconds=left))
            except RuntimeError:          # timed out, or the peer's connection closed
                return False
        while not self.done():
            if time.monotonic() > deadline:
                return False
            time.sleep(poll_s)
        return True


class TorchDistTransport:
    """torch.distributed point-to-point messages (gloo on CPU tensors, NCCL on CUDA tensors):
    a non-blocking send and receive per exchange; completion is polled, never waited on
    without a budget."""

    def __init__(self, group=None):
        self.group = group

    def post(self, send_buf, dst: int, recv_buf, src: int, tag: int):
        import torch.distributed as dist
        works = [dist.isend(send_buf, dst, group=self.group, tag=tag),
                 dist.irecv(recv_buf, src, group=self.group, tag=tag)]
        return _TorchHandle(works)


# ---------------------------------------------------------------- reductions
def combine_partials(partials) -> float:
    """The sum of per-rank FP64 partials rounded once (math.fsum: the exact sum of the
    partials, correctly rounded), so the result does not depend on their order."""
    import math
    return math.fsum(float(p) for p in partials)


class TorchDistReducer:
    """All-gather of one FP64 partial per rank (gloo on CPU tensors, NCCL on CUDA tensors),
    combined by ``combine_partials`` on every rank.  The all-gather is bounded by the process
    group's timeout."""

    def __init__(self, group=None):
        self.group = group

    def allreduce(self, partial) -> float:
        import torch
        import torch.distributed as dist
        world = dist.get_world_size(self.group)
        parts = [torch.empty_like(partial) for _ in range(world)]
        dist.all_gather(parts, partial, group=self.group)
        return combine_partials(t.item() for t in parts)


def sharded_reduce(plan, u, what: int, reducer, v=None, stream=None) -> float:
    """An FP64 reduction (SWEPT_SUM, SWEPT_HALF_SUMSQ, SWEPT_DOT with ``v`` the rank's slice of
    the other vector) of a field sharded over ranks: the slice's partial by swept_reduce on
    the slice's plan, then ``reducer.allreduce``."""
    from . import swept_reduce
    return reducer.allreduce(swept_reduce(plan, u, what, v, stream=stream))


# ------------------------------------------------------------------ GPU runner
class PlanRunner:
    """The stages of one slice on this GPU: a plan over the slice's n_local points (its windows
    wrap around the slice) and the slice's state, through swept_stage and swept_edge_copy.
    Edge halves and head points travel as device tensors on the current stream."""

    def __init__(self, plan, u, stream=None):
        from . import SWEPT_EULER, SWEPT_F32C, edge_element_bytes
        self.plan, self.u, self.stream = plan, u, stream
        self.edge_bytes = plan.B * edge_element_bytes(plan)
        n = plan.N
        # the state as blocks of n points: FP64 / F32 / Runge-Kutta 1; F32C hi, lo;
        # Euler rho, m, E (compensated: hi of each, then lo of each)
        nblocks = (3 if plan.stencil == SWEPT_EULER else 1) * (2 if plan.dtype == SWEPT_F32C else 1)
        flat = u.view(-1)
        self.blocks = [flat[b * n:(b + 1) * n] for b in range(nblocks)]

    def stage(self, k, hv, ht):
        from . import swept_stage
        swept_stage(self.plan, self.u, k, hv, ht, self.stream)

    def new_edge(self):
        import torch
        return torch.empty(self.edge_bytes, dtype=torch.uint8, device=self.u.device)

    def get_edge(self, k, w, side):
        from . import swept_edge_copy
        return swept_edge_copy(self.plan, k, w, side, self.new_edge(), False, self.stream)

    def put_edge(self, k, w, side, buf):
        from . import swept_edge_copy
        swept_edge_copy(self.plan, k, w, side, buf, True, self.stream)

    def new_head(self, n):
        import torch
        return torch.empty(len(self.blocks) * n, dtype=self.u.dtype, device=self.u.device)

    def get_head(self, n):
        import torch
        return torch.cat([b[:n] for b in self.blocks])

    def put_head(self, n, buf):
        for i, b in enumerate(self.blocks):
            b[:n].copy_(buf[i * n:(i + 1) * n])

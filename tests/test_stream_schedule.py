"""Schedule of the streamed ring launch (several full-diamond stages per launch), checked
on a CPU model under adversarial interleavings of the warps.

The model restates the kernel's bookkeeping: warp g of W owns windows
[g*nwin/W, (g+1)*nwin/W) shifted right by (j + [k0 odd]) / 2 at stage k0 + j; slot s
fills window s and empties window s - 1 of its run (stage-major); a window of an
offset (odd) stage reads windows w and w + 1 of the previous stage, of an unshifted
stage w - 1 and w (Section 3's alternating point sets); stage k0 + j reads edge buffer
j mod 2 and writes the other; before filling its last window of a stage j > 0 the warp
waits until warp g + 1 has completed slot (j - 1) * n_{g+1} + 1 (its first window of the
previous stage emptied).  Every arm read must find the previous stage's edges (no read
of a stale or a future stage) and every overwrite must come after both readers of the
old edges (no write-after-read hazard), and the run must never deadlock.
"""
from __future__ import annotations

import random

import pytest


def simulate(nwin, W, nst, odd0, seed, mode):
    rng = random.Random(seed)
    k0 = 1 if odd0 else 2
    runs = [((g * nwin) // W, ((g + 1) * nwin) // W) for g in range(W)]
    n_of = [b - a for a, b in runs]
    buf = [[k0 - 1] * nwin, [k0 - 2] * nwin]        # edge buffers: stage of the edges held
    reads = {}
    progress = [0] * W
    st = [dict(slot=0, jf=0, i_f=0, je=0, ie=0) for _ in range(W)]
    T = [nst * n for n in n_of]

    def win(g, j, i):
        return (runs[g][0] + ((j + odd0) >> 1) + i) % nwin

    def can_step(g):
        s = st[g]
        if s["slot"] > T[g]:
            return False
        if s["slot"] < T[g] and s["i_f"] == n_of[g] - 1 and s["jf"] > 0:
            gr = (g + 1) % W
            return progress[gr] >= (s["jf"] - 1) * n_of[gr] + 2
        return True

    def step(g):
        s = st[g]
        n = n_of[g]
        slot = s["slot"]
        if slot < T[g]:                               # fill: read both arms at the slot's start
            jf = s["jf"]
            k = k0 + jf
            w = win(g, jf, s["i_f"])
            offs = (k & 1) == 1
            for idx in ((w, (w + 1) % nwin) if offs else ((w - 1) % nwin, w)):
                assert buf[jf & 1][idx] == k - 1, ("stale arm", g, slot, k, idx)
                reads[(k - 1, idx)] = reads.get((k - 1, idx), 0) + 1
        if slot > 0:                                  # empty: write the edges at the slot's end
            je = s["je"]
            ke = k0 + je
            w = win(g, je, s["ie"])
            b = 0 if (je & 1) else 1
            old = buf[b][w]
            assert old == ke - 2
            if old >= k0 - 1:
                assert reads.get((old, w), 0) == 2, ("write before read", g, slot, ke, w)
            buf[b][w] = ke
            s["ie"] += 1
            if s["ie"] == n:
                s["ie"], s["je"] = 0, je + 1
        progress[g] = slot + 1
        if slot < T[g]:
            s["i_f"] += 1
            if s["i_f"] == n:
                s["i_f"], s["jf"] = 0, s["jf"] + 1
        s["slot"] += 1

    while True:
        ready = [g for g in range(W) if can_step(g)]
        if not ready:
            break
        g = {"min": ready[0], "max": ready[-1], "mid": ready[len(ready) // 2]}.get(mode) \
            if mode != "rand" else rng.choice(ready)
        for _ in range(rng.choice([1, 1, 5, 40])):
            if can_step(g):
                step(g)
    assert all(st[g]["slot"] == T[g] + 1 for g in range(W)), "deadlock"
    last = k0 + nst - 1
    assert all(v == last for v in buf[0 if (nst - 1) & 1 else 1]), "final edges"


@pytest.mark.parametrize("nwin", [3, 5, 9, 16, 31, 64])
@pytest.mark.parametrize("mode", ["rand", "min", "max", "mid"])
def test_streamed_schedule_hazard_free(nwin, mode):
    for W in range(1, nwin // 3 + 1):               # at least 3 windows per warp
        for nst in (1, 2, 3, 7):
            for odd0 in (0, 1):
                simulate(nwin, W, nst, odd0, seed=nwin * 100 + W, mode=mode)


def test_two_windows_per_warp_is_unsafe():
    """With runs of 2 windows a stage's first fill would read an edge emptied in the same
    slot: the launcher keeps at least 3 windows per warp."""
    with pytest.raises(AssertionError):
        simulate(8, 4, 3, 1, seed=0, mode="min")

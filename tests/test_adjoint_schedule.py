"""CPU model of the KS adjoint's checkpoint and tape-ring schedule (swept_adjoint).

The forward pass stores a flat checkpoint every m stages of a swept advance that
starts at level rem (nsteps = q*h + rem); the reverse pass refills a ring of
m + 1 chunks of h levels from those checkpoints, one checkpoint group at a time,
just before the transposed stage that first needs it, and each transposed stage
reads the forward levels nsteps - tau for its sweep levels tau.  This model
replays that schedule (the same chunk and slot arithmetic as the library's host
code and its device-side tape_level) with labelled values instead of states and
checks, for many (q, rem, m):
  * every level a stage reads is in the ring, holding exactly that level;
  * every level is recomputed once, from the checkpoint of its own group;
  * the choice of m is the one that minimises the scratch.
"""
from __future__ import annotations

import itertools
import math

import pytest


def layout(q, rem, h, k_cycles=64):
    best, every = None, 1
    for m in range(1, min(2 * k_cycles, max(q, 1)) + 1):
        states = -(-q // m) + (m + 1) * h
        if best is None or states < best:
            best, every = states, m
    nckpt = -(-q // every) if q > 0 else 0
    return every, nckpt, every + 1, (1 if rem > 0 else 0) + nckpt + (every + 1) * h


def slot_of(level, rem, h, ring):
    if level < rem:
        return ring - 1, level
    c = (level - rem) // h
    return c % ring, level - rem - c * h


def stage_levels(q, rem, h):
    """(k, sweep levels tau read, lowest chunk needed) for each stage of the sweep."""
    out = []
    if q == 0:
        out.append((0, range(1, rem + 1), -1))
        out.append((1, range(1, rem + 1), -1))
        return out
    out.append((0, range(1, h + 1), q - 1))
    for k in range(1, q):
        out.append((k, range((k - 1) * h + 1, (k + 1) * h + 1), q - k - 1))
    out.append((q, range((q - 1) * h + 1, q * h + rem + 1), -1 if rem > 0 else 0))
    if rem > 0:
        out.append((q + 1, range(q * h + 1, q * h + rem + 1), -1))
    return out


def replay(q, rem, h, every, ring):
    F = q * h + rem
    tape = {}                      # (slot, offset) -> forward level held there
    computed = []                  # levels recomputed, in order
    lowest = q

    def recompute_down_to(need):
        nonlocal lowest
        while lowest > need:
            top = lowest - 1
            if top >= 0:
                g = top // every
                l0, count = rem + g * every * h, (lowest - g * every) * h
                src = ("ckpt", g)
                lowest = g * every
            else:
                l0, count, src = 0, rem, ("pre",)
                lowest = -1
            assert src == ("pre",) or src[1] < -(-q // every)
            for lv in range(l0, l0 + count):
                tape[slot_of(lv, rem, h, ring)] = lv
                computed.append(lv)

    for k, taus, need in stage_levels(q, rem, h):
        recompute_down_to(need)
        for tau in taus:
            lv = F - tau
            assert tape.get(slot_of(lv, rem, h, ring)) == lv, (q, rem, every, k, tau, lv)
    return computed, F


@pytest.mark.parametrize("h", [4, 16, 64])
def test_every_level_read_is_in_the_ring(h):
    for q, rem in itertools.product(list(range(0, 12)) + [31, 64, 97], [0, 1, h // 2, h - 1]):
        if q == 0 and rem == 0:
            continue
        for every in range(1, max(q, 1) + 1):
            computed, F = replay(q, rem, h, every, every + 1)
            assert sorted(computed) == list(range(F)), (q, rem, every)   # each level exactly once


def test_layout_minimises_scratch_and_matches_the_adjoint_workload():
    # the adjoint workload: N = 2^20, 20000 steps, B = 256 (h = 64), checkpoint bound 64 cycles
    every, nckpt, ring, states = layout(20000 // 64, 20000 % 64, 64)
    assert (every, nckpt, ring, states) == (2, 156, 3, 349)
    assert states * 8 * (1 << 20) < 4 * 2 ** 30                 # under 4 GiB at N = 2^20
    for q, h in ((312, 64), (1000, 16), (5, 128)):
        every, _, _, states = layout(q, 1, h)
        brute = min(1 + math.ceil(q / m) + (m + 1) * h for m in range(1, min(128, q) + 1))
        assert states == brute
    # the bound: with K_cycles = 1 the interval is at most 2 stages
    assert layout(312, 0, 64, k_cycles=1)[0] <= 2

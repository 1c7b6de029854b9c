"""A CPU stand-in for one rank's stages, for the sharded-advance tests.

It plays the part the GPU plays under ``paper_1504_01380_gb300.shard``: stage k
of the swept schedule on every window of a slice whose windows wrap around the
slice, with the library's leading-edge layout (per window, the left edges
L[h][2r] then the right edges R[h][2r], two buffers alternating by stage), in
FP64 with the oracle's per-point update.  The geometry is written out from
Section 3's stages (V-fill from the arms, shrinking trapezoid with its edges
captured), independently of the kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from oracle.pointwise import make_point_update


class StandinRunner:
    def __init__(self, stencil: int, params, u_local: np.ndarray, B: int):
        self.r, self.f = make_point_update(stencil, params)
        self.u = np.array(u_local, dtype=np.float64)
        self.n = self.u.size
        self.B = B
        self.h = B // (2 * self.r)
        self.nwin = self.n // B
        # edges[buffer, window, side, level, q]
        self.edges = np.full((2, self.nwin, 2, self.h, 2 * self.r), np.nan)

    def _level(self, prev: dict, lo: int, hi: int) -> dict:
        r, f = self.r, self.f
        return {x: f([prev[x + d] for d in range(-r, r + 1)], 0) for x in range(lo, hi)}

    def stage(self, k: int, hv: int, ht: int):
        B, r, h, n = self.B, self.r, self.h, self.n
        off = B // 2 if k % 2 else 0
        ein, eout = self.edges[(k + 1) % 2], self.edges[k % 2]
        flat_in = self.u.copy()
        for w in range(self.nwin):
            ws = w * B + off
            if hv == 0:
                cur = {x: flat_in[(ws + x) % n] for x in range(B)}
            else:
                wl = w if off else (w - 1) % self.nwin
                wr = (w + 1) % self.nwin if off else w
                arm_l, arm_r = ein[wl, 1], ein[wr, 0]     # right edges of wl, left edges of wr
                cur = {}
                for m in range(1, hv + 1):
                    prev = dict(cur)
                    for q in range(2 * r):
                        prev[B // 2 - r * (m - 1) - 2 * r + q] = arm_l[m - 1, q]
                        prev[B // 2 + r * (m - 1) + q] = arm_r[m - 1, q]
                    cur = self._level(prev, B // 2 - r * m, B // 2 + r * m)
            if ht > 0:
                for m in range(ht):
                    if m > 0:
                        cur = self._level(cur, r * m, B - r * m)
                    for q in range(2 * r):
                        eout[w, 0, m, q] = cur[r * m + q]
                        eout[w, 1, m, q] = cur[B - r * m - 2 * r + q]
                if ht < h:
                    top = self._level(cur, r * ht, B - r * ht)
                    for x, v in top.items():
                        self.u[(ws + x) % n] = v
            else:
                for x, v in cur.items():                   # a full fill is flat; a partial one its gap
                    self.u[(ws + x) % n] = v

    # message buffers are CPU tensors (gloo)
    def new_edge(self):
        return torch.empty(self.h * 2 * self.r, dtype=torch.float64)

    def get_edge(self, k, w, side):
        return torch.from_numpy(self.edges[k % 2, w, side].reshape(-1).copy())

    def put_edge(self, k, w, side, buf):
        self.edges[k % 2, w, side] = buf.numpy().reshape(self.h, 2 * self.r)

    def new_head(self, n):
        return torch.empty(n, dtype=torch.float64)

    def get_head(self, n):
        return torch.from_numpy(self.u[:n].copy())

    def put_head(self, n, buf):
        self.u[:n] = buf.numpy()

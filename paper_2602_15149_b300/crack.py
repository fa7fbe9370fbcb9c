"""Crack geometry of the notched plate from its phase field (post-processing of read-back state).

The plate is a regular lattice X = ((i + 1/2) dp, (j + 1/2) dp), so the phase field s maps to an
(ny, nx) image.  A cell is cracked when s < threshold.  From a sequence of images this extracts what
the paper reports for its crack-branching benchmark (Sec. 4, dynamic crack branching): the time the
crack starts at the notch tip, the time and place it branches, the angle between the two branches
and whether the pattern is symmetric about the notch plane.
"""
from __future__ import annotations

import math

import numpy as np


def image(X0, s, dp):
    """s on the lattice as an (ny, nx) array."""
    i = np.rint(X0[:, 0] / dp - 0.5).astype(np.int64)
    j = np.rint(X0[:, 1] / dp - 0.5).astype(np.int64)
    img = np.ones((j.max() + 1, i.max() + 1))
    img[j, i] = s
    return img


def runs(col):
    """Runs of True in a 1D boolean array: list of (first, last) indices."""
    out = []
    k = 0
    n = col.shape[0]
    while k < n:
        if col[k]:
            b = k
            while k < n and col[k]:
                k += 1
            out.append((b, k - 1))
        else:
            k += 1
    return out


def branched_columns(cracked, j0, gap):
    """Columns whose cracked cells form a run wholly above the notch plane and one wholly below it,
    each at least ``gap`` rows from it (the two branches, with intact material between them).
    Returns {column: (centre row of the lowest run above, centre row of the highest run below)}."""
    ny = cracked.shape[0]
    pad = np.zeros((1, cracked.shape[1]), bool)
    prev = np.vstack([pad, cracked[:-1]])
    nxt = np.vstack([cracked[1:], pad])
    starts = cracked & ~prev
    ends = cracked & ~nxt
    R = np.arange(ny)[:, None]
    j_up = int(math.ceil(j0 + gap))
    j_lo = int(math.floor(j0 - gap))
    up_c = starts & (R >= j_up)
    lo_c = ends & (R <= j_lo)
    has = up_c.any(axis=0) & lo_c.any(axis=0)
    out = {}
    if not has.any():
        return out
    up_first = np.argmax(up_c, axis=0)
    up_end = np.argmax(ends & (R >= up_first[None, :]), axis=0)
    lo_last = ny - 1 - np.argmax(lo_c[::-1], axis=0)
    lo_start = ny - 1 - np.argmax((starts & (R <= lo_last[None, :]))[::-1], axis=0)
    for i in np.nonzero(has)[0]:
        out[int(i)] = (0.5 * (up_first[i] + up_end[i]), 0.5 * (lo_start[i] + lo_last[i]))
    return out


class CrackTracker:
    """Feed (t, s) snapshots of the notched plate; read the crack's milestones.

    ``t_init``: first snapshot with a cracked cell ahead of the notch tip.  ``t_branch``: first snapshot
    in which some column ahead of the tip holds cracked runs on both sides of the notch plane, each at
    least ``branch_gap_rows`` rows from it.  With one row this is the first split of the crack band;
    with a few rows, sustained branches."""

    def __init__(self, X0, dp, y0, notch_len, threshold=0.25, branch_gap_rows=4):
        self.X0, self.dp, self.thr = X0, dp, threshold
        self.j0 = y0 / dp - 0.5  # notch plane in row units
        self.i_tip = int(round(notch_len / dp - 0.5))
        self.gap = branch_gap_rows
        self.t_init = None
        self.t_branch = None
        self.tip_x = []      # (t, furthest cracked x ahead of the notch)
        self.last = None

    def add(self, t, s):
        img = image(self.X0, s, self.dp)
        cracked = img < self.thr
        ahead = cracked[:, self.i_tip + 1:]
        if self.t_init is None and ahead.any():
            self.t_init = t
        cols = np.nonzero(ahead.any(axis=0))[0]
        self.tip_x.append((t, (self.i_tip + 1 + cols.max() + 0.5) * self.dp if cols.size else math.nan))
        if self.t_branch is None:
            bc = branched_columns(cracked[:, self.i_tip + 1:], self.j0, self.gap)
            if bc:
                self.t_branch = t
        self.last = (t, img)

    def geometry(self, fit_len=5e-3):
        """Branch point, divergence angle (degrees, between the two branches, from straight-line fits of
        each branch's centre over ``fit_len`` beyond the branch point) and mirror asymmetry (the share of
        cracked cells whose mirror image about the notch plane is intact) of the last snapshot."""
        t, img = self.last
        cracked = img < self.thr
        sub = cracked[:, self.i_tip + 1:]
        bc = branched_columns(sub, self.j0, self.gap)
        out = {"t": t, "branch_x": None, "angle_deg": None, "angle_up_deg": None, "angle_lo_deg": None}
        j = np.arange(cracked.shape[0])
        jm = np.rint(2 * self.j0 - j).astype(np.int64)
        ok = (jm >= 0) & (jm < cracked.shape[0])
        mirrored = np.zeros_like(cracked)
        mirrored[ok] = cracked[jm[ok]]
        nc = max(int(cracked.sum()), 1)
        out["asymmetry"] = float((cracked & ~mirrored).sum()) / nc
        if not bc:
            return out
        i_b = min(bc)
        out["branch_x"] = (self.i_tip + 1 + i_b + 0.5) * self.dp
        n_fit = int(round(fit_len / self.dp))
        xs, yu, yl = [], [], []
        for i in range(i_b, i_b + n_fit):
            if i in bc:
                xs.append(i)
                yu.append(bc[i][0] - self.j0)
                yl.append(self.j0 - bc[i][1])
        if len(xs) >= 3:
            au = math.degrees(math.atan(np.polyfit(xs, yu, 1)[0]))
            al = math.degrees(math.atan(np.polyfit(xs, yl, 1)[0]))
            out.update(angle_up_deg=au, angle_lo_deg=al, angle_deg=au + al)
        return out

"""Per-block error measures for the GPU parity tests.

A whole-vector relative error hides a block that is wrong by a few percent
among many right ones, so the parity tests compare block by block:
  * torn vectors: one block per (patch, component) tensor;
  * multiplier vectors: one block per (component, patch of the first copy)
    run of constraint rows (rows are component-major, then ordered by the
    node's first copy, so these runs are contiguous);
  * saddle vectors [w; chi]: both lists, the second shifted by n_dof.
The measure is the largest block-relative error, max_b ||a_b - r_b|| / ||r_b||.
A block whose reference is exactly zero must come out as exactly zero."""
from __future__ import annotations

import numpy as np


def torn_blocks(orc):
    out = []
    for k in range(orc.np):
        for l in range(orc.dim):
            a = int(orc.off[k]) + l * orc.N[k]
            out.append((a, a + orc.N[k]))
    return out


def interior_blocks(orc):
    """Blocks of the compact interior layout ([patch][component][interior])."""
    out, a = [], 0
    for k, (per, mask, Hs) in enumerate(orc._local()):
        ni = int(mask.sum())
        for l in range(orc.dim):
            out.append((a, a + ni))
            a += ni
    return out


def mult_blocks(orc):
    first = {}
    for (c, n, ids) in orc.node_rows:
        k = orc.nodes[n][0][0]
        for r in ids:
            first[r] = (c, k)
    for (c, kf, ff, ids) in getattr(orc, "nested_rows", []):
        for r in ids:
            first[r] = ("nested", c, kf, ff)
    out, start = [], 0
    for r in range(1, orc.nc + 1):
        if r == orc.nc or first[r] != first[start]:
            out.append((start, r))
            start = r
    return out


def saddle_blocks(orc):
    return torn_blocks(orc) + [(a + orc.ndof, b + orc.ndof) for a, b in mult_blocks(orc)]


def block_rel(a, ref, blocks):
    """max over blocks of ||a_b - ref_b|| / ||ref_b||."""
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert a.shape == ref.shape
    covered = np.zeros(ref.shape, dtype=bool)
    worst = 0.0
    for lo, hi in blocks:
        covered[lo:hi] = True
        rn = np.linalg.norm(ref[lo:hi])
        dn = np.linalg.norm(a[lo:hi] - ref[lo:hi])
        if rn == 0.0:
            if dn != 0.0:
                return float("inf")
            continue
        worst = max(worst, dn / rn)
    assert covered.all(), "blocks do not cover the vector"
    return float(worst)

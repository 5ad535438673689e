"""The byte and FLOP counts behind bench.py's roofline lines, checked against
brute-force counts on small problems (CPU only): structural nonzeros of the
stiffness (pairs of basis functions whose supports overlap, times the d^2
component blocks), the stored FP64 stencil, and the row-compressed pair copy
(per row group and in-row offset o1, the nodes whose neighbour lies in the
row, padded to an even count)."""
import itertools

import afi_workloads as W
import bench


def brute_counts(prob):
    d = prob.dim
    nnz = stored = pairs = ndof = 0
    for k in range(prob.npatch):
        p = int(prob.degree[k])
        ns = prob.n(k)
        N = 1
        for n in ns:
            N *= n
        ndof += d * N
        # structural nonzeros: node pairs within p in every direction
        per_dir = [sum(1 for i in range(n) for j in range(n) if abs(i - j) <= p) for n in ns]
        cnt = 1
        for c in per_dir:
            cnt *= c
        nnz += d * d * cnt
        n1p = ns[0] + ns[0] % 2
        stored += d * d * (2 * p + 1) ** d * (N // ns[0]) * n1p
        rows = N // ns[0]
        groups = d * d * (2 * p + 1) ** (d - 1)
        for o1 in range(2 * p + 1):
            ln = sum(1 for i1 in range(ns[0]) if 0 <= i1 + o1 - p < ns[0])
            sz = rows * ln
            pairs += groups * (sz + sz % 2)
    return 2 * nnz, 8 * stored + 16 * ndof, 8 * pairs


def test_counts_match_brute_force():
    probs = [W.config("C1-small"), W.config("C1"), W.config("C2-small"), W.config("C5-small"),
             W.quarter_annulus(grid=(2, 1, 2), p=2, nel_cols=[[6, 3], [5], [2, 7]], name="uneven")]
    for prob in probs:
        flops, stored = bench.stencil_stats(prob)
        bf, bs, bp = brute_counts(prob)
        assert (flops, stored) == (bf, bs), prob.name
        assert bench.pair_copy_bytes(prob) == bp, prob.name


def test_pair_copy_is_smaller_than_the_fp64_stencil():
    for name in ("C2-small", "C5-small"):
        prob = W.config(name)
        flops, stored = bench.stencil_stats(prob)
        assert 8 * (flops // 2) < bench.pair_copy_bytes(prob) < stored


def test_matrix_free_flop_count():
    """The matrix-free kernel's FLOPs per element (bench roofline), against a
    pass-by-pass enumeration: forward, six fields, contractions producing
    2 / 3 / 3 outputs per line in directions 1 / 2 / 3; back, three
    components, 3 / 3 / 2 (one output of back pass 2 takes two products);
    each output of a line is a (p+1)-term FMA chain over (p+1)^2 lines."""
    for p in range(1, 6):
        nb = p + 1
        lines = nb * nb
        fma = 6 * lines * nb * (2 + 3 + 3) * nb + 3 * lines * nb * (3 + 3 + 2) * nb
        pointwise = 168 * nb ** 3
        assert bench.mf_flops_per_element(p) == 2 * fma + pointwise
    assert bench.mf_flops_per_element(4) == 111000
    assert abs(bench.fp32_peak_tflops(2070.0) - 80.55) < 0.01

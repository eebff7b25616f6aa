#!/usr/bin/env python3
"""Generate the register selection networks used by the CUDA kernels.

A median of n values is taken with a comparator network: Batcher's odd-even
merge sort (Batcher 1968) on a power-of-two number of wires, padded with
-inf/+inf constants, pruned to the one output rank that is needed. Pruning
folds comparisons against the constants, merges identical nodes and drops
every node the selected output does not depend on. What is left is a DAG of
min/max operations on the inputs.

Correctness: a min/max network selects rank k of its inputs for all real
inputs iff it does so for all 0/1 inputs (the 0-1 principle, Knuth TAOCP
5.3.4). The generator checks every 0/1 input for n <= 25 (bit-parallel) and
random real inputs for every n; the pruning itself only removes operations
that cannot reach the output.

Row groups: the 5x5 medians of G horizontally adjacent windows share columns.
Each of the G + 4 columns is sorted once; sorted lists are then merged
(odd-even merge of two sorted lists of any lengths) in a tree per window, and
merges shared by several windows are built once. A merged list of n < 25 values
of a window keeps only its ranks max(0, n - 13) .. min(n - 1, 12): a value of
rank s among them has a window rank between s and s + 25 - n, so it can be the
median (rank 12) only inside that range. A dropped low value ranks below every
kept value of any merge above it (its rank in the union of two lists is below
n - 13 of the union), so a parent's ranks shift down by its children's low
drops. The generator checks the whole network on every 0/1 input whose columns
are already sorted, and the column sorter on every 0/1 input: together they
cover all 0/1 inputs, since the merges read only sorted columns.

Usage: python gen_networks.py OUT.cuh [--quick]   (--quick: random checks only)
"""

from __future__ import annotations

import sys

import numpy as np


def batcher_pairs(n):
    """Comparator pairs (i, j), i < j, of Batcher's odd-even merge sort on n = 2^m wires."""
    pairs = []

    def merge(lo, cnt, r):
        step = r * 2
        if step < cnt:
            merge(lo, cnt, step)
            merge(lo + r, cnt, step)
            for i in range(lo + r, lo + cnt - r, step):
                pairs.append((i, i + r))
        else:
            pairs.append((lo, lo + r))

    def sort(lo, cnt):
        if cnt > 1:
            half = cnt // 2
            sort(lo, half)
            sort(lo + half, half)
            merge(lo, cnt, 1)

    sort(0, n)
    return pairs


NEG, POS = ("const", "-inf"), ("const", "+inf")


class Dag:
    def __init__(self):
        self.nodes = {}   # key -> id
        self.defs = []    # id -> key

    def node(self, key):
        if key not in self.nodes:
            self.nodes[key] = len(self.defs)
            self.defs.append(key)
        return self.nodes[key]

    def minmax(self, op, a, b):
        ka, kb = self.defs[a], self.defs[b]
        if a == b:
            return a
        if op == "min":
            if ka == POS:
                return b
            if kb == POS:
                return a
            if ka == NEG or kb == NEG:
                return self.node(NEG)
        else:
            if ka == NEG:
                return b
            if kb == NEG:
                return a
            if ka == POS or kb == POS:
                return self.node(POS)
        x, y = (a, b) if a < b else (b, a)
        return self.node((op, x, y))


def select_network(n, rank, npad_lo):
    """DAG selecting 0-based `rank` of n inputs; npad_lo -inf constants go below the inputs."""
    size = 1
    while size < n:
        size *= 2
    npad_hi = size - n - npad_lo
    assert npad_hi >= 0
    d = Dag()
    wires = ([d.node(NEG)] * npad_lo + [d.node(("in", i)) for i in range(n)]
             + [d.node(POS)] * npad_hi)
    for (i, j) in batcher_pairs(size):
        a, b = wires[i], wires[j]
        wires[i], wires[j] = d.minmax("min", a, b), d.minmax("max", a, b)
    out = wires[rank + npad_lo]
    # keep only what the output depends on
    live, stack = set(), [out]
    while stack:
        v = stack.pop()
        if v in live:
            continue
        live.add(v)
        k = d.defs[v]
        if k[0] in ("min", "max"):
            stack += [k[1], k[2]]
    order = [v for v in range(len(d.defs)) if v in live]  # ids are topological
    return d, order, out


def count_ops(d, order):
    return sum(1 for v in order if d.defs[v][0] in ("min", "max"))


def best_network(n, rank):
    size = 1
    while size < n:
        size *= 2
    best = None
    for lo in range(0, size - n + 1):
        d, order, out = select_network(n, rank, lo)
        c = count_ops(d, order)
        if best is None or c < best[0]:
            best = (c, d, order, out)
    return best


def evaluate(d, order, out, X):
    """Evaluate on rows of X (inputs in columns); works for bool (and/or) and float."""
    vals = {}
    boolean = X.dtype == bool
    for v in order:
        k = d.defs[v]
        if k[0] == "in":
            vals[v] = X[:, k[1]]
        elif k[0] == "const":
            raise AssertionError("constant survived pruning")
        elif k[0] == "min":
            vals[v] = (vals[k[1]] & vals[k[2]]) if boolean else np.minimum(vals[k[1]], vals[k[2]])
        else:
            vals[v] = (vals[k[1]] | vals[k[2]]) if boolean else np.maximum(vals[k[1]], vals[k[2]])
    return vals[out]


def verify(n, rank, d, order, out, exhaustive=True):
    rng = np.random.default_rng(0)
    X = rng.normal(size=(4000, n))
    X[:1000] = rng.integers(0, 3, size=(1000, n))  # ties
    got = evaluate(d, order, out, X)
    assert np.array_equal(got, np.sort(X, axis=1)[:, rank]), f"real inputs, n={n}"
    if exhaustive and n <= 25:
        # all 2^n 0/1 inputs, in chunks: sorted[rank] == 1 iff count(ones) >= n - rank
        total = 1 << n
        chunk = 1 << 20
        bits = np.arange(n, dtype=np.uint64)
        for start in range(0, total, chunk):
            idx = np.arange(start, min(total, start + chunk), dtype=np.uint64)
            X = ((idx[:, None] >> bits[None, :]) & np.uint64(1)).astype(bool)
            got = evaluate(d, order, out, X)
            exp = X.sum(axis=1) >= (n - rank)
            assert np.array_equal(got, exp), f"0-1 inputs, n={n}"


def fuse3(d, order, out):
    """Pairs a min (max) node with a single-use min (max) operand: op(op(a, b), c) = op3(a, b, c).

    Returns {node: (op, operands)} for every emitted node; operands has 2 or 3 entries.
    The three-input form issues at the rate of the two-input one on sm_103a. `out` is
    one output node or a list of them.
    """
    outs = out if isinstance(out, list) else [out]
    uses = {}
    for v in order:
        k = d.defs[v]
        if k[0] in ("min", "max"):
            for u in k[1:]:
                uses[u] = uses.get(u, 0) + 1
    for o in outs:
        uses[o] = uses.get(o, 0) + 1
    absorbed = set()
    emitted = {}
    for v in reversed(order):  # from the output down, so a fused operand is never emitted twice
        k = d.defs[v]
        if k[0] not in ("min", "max") or v in absorbed:
            continue
        ops = [k[1], k[2]]
        for idx, u in enumerate(ops):
            ku = d.defs[u]
            if ku[0] == k[0] and uses.get(u, 0) == 1 and u not in emitted:
                absorbed.add(u)
                ops = ops[:idx] + [ku[1], ku[2]] + ops[idx + 1:]
                break
        emitted[v] = (k[0], ops)
    return emitted


def emit(name, n, rank, d, order, out):
    fused = fuse3(d, order, out)
    lines = [f"// rank {rank} (0-based) of {n} values; {count_ops(d, order)} two-input min/max, "
             f"{len(fused)} instructions with three-input forms",
             f"__device__ __forceinline__ float {name}(const float (&v)[{n}]) {{"]
    names = {}
    t = 0
    for v in order:
        k = d.defs[v]
        if k[0] == "in":
            names[v] = f"v[{k[1]}]"
        elif v in fused:
            op, ops = fused[v]
            args = ", ".join(names[u] for u in ops)
            fn = ("fminf" if op == "min" else "fmaxf") if len(ops) == 2 else ("min3f" if op == "min" else "max3f")
            names[v] = f"t{t}"
            lines.append(f"  const float t{t} = {fn}({args});")
            t += 1
    lines.append(f"  return {names[out]};")
    lines.append("}")
    return "\n".join(lines)


def live_order(d, outs):
    """The nodes the outputs depend on, in topological (id) order."""
    live, stack = set(), list(outs)
    while stack:
        v = stack.pop()
        if v in live:
            continue
        live.add(v)
        k = d.defs[v]
        if k[0] in ("min", "max"):
            stack += [k[1], k[2]]
    return [v for v in range(len(d.defs)) if v in live]


def merge_sorted(d, a, b):
    """Odd-even merge (Batcher 1968) of two sorted lists of nodes, any lengths: the evens and the odds
    of both lists are merged recursively, then neighbouring odd/even outputs are compared."""
    if not a:
        return list(b)
    if not b:
        return list(a)
    if len(a) == 1 and len(b) == 1:
        return [d.minmax("min", a[0], b[0]), d.minmax("max", a[0], b[0])]
    e = merge_sorted(d, a[0::2], b[0::2])
    o = merge_sorted(d, a[1::2], b[1::2])
    out, i = [e[0]], 0
    while i < len(o) and i + 1 < len(e):
        out += [d.minmax("min", o[i], e[i + 1]), d.minmax("max", o[i], e[i + 1])]
        i += 1
    return out + o[i:] + e[i + 1:]


def sort_nodes(d, xs):
    """Odd-even merge sort of a list of nodes."""
    if len(xs) <= 1:
        return list(xs)
    h = len(xs) // 2
    return merge_sorted(d, sort_nodes(d, xs[:h]), sort_nodes(d, xs[h:]))


ROW_D, ROW_MED = 5, 12  # 5x5 windows, median = rank 12 of 25


def row_network(g):
    """Medians of the g (even) adjacent 5x5 windows over a 5 x (g + 4) block; input ("in", r*(g+4)+c) is
    row r, column c; window i covers columns i .. i+4. Outputs 2j and 2j+1 share the merge of columns
    2j+1 .. 2j+4 (two pair merges); output 2j adds column 2j, output 2j+1 column 2j+5. For g = 4 an
    exhaustive search over every merge tree of the four windows finds no cheaper network."""
    assert g % 2 == 0
    d = Dag()
    ncol = g + 4
    cols = [sort_nodes(d, [d.node(("in", r * ncol + c)) for r in range(ROW_D)]) for c in range(ncol)]

    def kept_range(n):
        # the ranks of n values of a window that can be its median
        return max(0, n - (ROW_MED + 1)), min(n - 1, ROW_MED)

    def merge_kept(a, na, b, nb):
        # a, b: the kept lists of na and nb window values; returns the kept list of the na + nb values
        shift = kept_range(na)[0] + kept_range(nb)[0]
        lo, hi = kept_range(na + nb)
        return merge_sorted(d, a, b)[lo - shift: hi - shift + 1]

    pair = {c: merge_kept(cols[c], ROW_D, cols[c + 1], ROW_D) for c in range(1, ncol - 2, 2)}
    outs = []
    for j in range(g // 2):
        c = 2 * j + 1
        quad = merge_kept(pair[c], 2 * ROW_D, pair[c + 2], 2 * ROW_D)
        for extra in (c - 1, c + 4):
            # one more column completes the window: its median is the one kept rank of 25 values
            outs.append(merge_kept(cols[extra], ROW_D, quad, 4 * ROW_D)[0])
    return d, live_order(d, outs), outs


def evaluate_many(d, order, outs, X):
    vals = {}
    boolean = X.dtype == bool
    for v in order:
        k = d.defs[v]
        if k[0] == "in":
            vals[v] = X[:, k[1]]
        elif k[0] == "const":
            raise AssertionError("constant survived pruning")
        elif k[0] == "min":
            vals[v] = (vals[k[1]] & vals[k[2]]) if boolean else np.minimum(vals[k[1]], vals[k[2]])
        else:
            vals[v] = (vals[k[1]] | vals[k[2]]) if boolean else np.maximum(vals[k[1]], vals[k[2]])
    return [vals[o] for o in outs]


def verify_row(g, d, order, outs, exhaustive=True):
    ncol = g + 4
    rng = np.random.default_rng(1)
    X = rng.normal(size=(20000, ROW_D * ncol))
    X[:5000] = rng.integers(0, 3, size=(5000, ROW_D * ncol))  # ties
    got = evaluate_many(d, order, outs, X)
    blk = X.reshape(-1, ROW_D, ncol)
    for i in range(g):
        exp = np.sort(blk[:, :, i:i + ROW_D].reshape(len(X), -1), axis=1)[:, ROW_MED]
        assert np.array_equal(got[i], exp), f"row network, real inputs, window {i}"
    if not exhaustive:
        return
    # the column sorter on every 0/1 input
    ds = Dag()
    srt = sort_nodes(ds, [ds.node(("in", r)) for r in range(ROW_D)])
    Z = ((np.arange(1 << ROW_D)[:, None] >> np.arange(ROW_D)[None, :]) & 1).astype(bool)
    res = np.stack(evaluate_many(ds, live_order(ds, srt), srt, Z), axis=1)
    assert np.array_equal(res, np.sort(Z, axis=1)), "column sorter"
    # the network on every 0/1 input with sorted columns: column c holds k_c ones at its bottom rows
    nconf = (ROW_D + 1) ** ncol
    idx = np.arange(nconf)
    counts = np.stack([(idx // (ROW_D + 1) ** c) % (ROW_D + 1) for c in range(ncol)], axis=1)
    rows = np.arange(ROW_D)
    X = (rows[None, :, None] >= (ROW_D - counts)[:, None, :]).reshape(nconf, -1)
    got = evaluate_many(d, order, outs, X)
    for i in range(g):
        exp = counts[:, i:i + ROW_D].sum(axis=1) >= ROW_D * ROW_D - ROW_MED
        assert np.array_equal(got[i], exp), f"row network, 0/1 inputs, window {i}"


def emit_row(name, g, d, order, outs):
    fused = fuse3(d, order, outs)
    two = sum(1 for v in order if d.defs[v][0] in ("min", "max"))
    ncol = g + 4
    lines = [f"// row group: {g} medians of 5x5 windows; {two} two-input min/max, {len(fused)} instructions "
             "with three-input forms",
             f"// m[i] = median of v[0..4][i..i+4] (rank 12 of 25)",
             f"__device__ __forceinline__ void {name}(const float (&v)[5][{ncol}], float (&m)[{g}]) {{"]
    names, t = {}, 0
    for v in order:
        k = d.defs[v]
        if k[0] == "in":
            names[v] = f"v[{k[1] // ncol}][{k[1] % ncol}]"
        elif v in fused:
            op, ops = fused[v]
            args = ", ".join(names[u] for u in ops)
            fn = ("fminf" if op == "min" else "fmaxf") if len(ops) == 2 else ("min3f" if op == "min" else "max3f")
            names[v] = f"t{t}"
            lines.append(f"  const float t{t} = {fn}({args});")
            t += 1
    for i, o in enumerate(outs):
        lines.append(f"  m[{i}] = {names[o]};")
    lines.append("}")
    return "\n".join(lines), two, len(fused)


ROW_SPECS = [("med25_row2", 2), ("med25_row4", 4)]

SPECS = [("sel_med5", 5, 2), ("sel_med7", 7, 3), ("sel_med9", 9, 4), ("sel_med25", 25, 12),
         ("sel_med49", 49, 24)]

PRELUDE = """// Three-input min/max (PTX min.f32 / max.f32 with three sources, sm_100+).
__device__ __forceinline__ float min3f(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ float max3f(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
"""


def main(path, exhaustive=True):
    parts = ["// Generated by gen_networks.py -- do not edit.",
             "// Pruned Batcher odd-even merge selection networks (exact selections).",
             "#pragma once", "", PRELUDE]
    for (name, n, rank) in SPECS:
        c, d, order, out = best_network(n, rank)
        verify(n, rank, d, order, out, exhaustive)
        parts.append(emit(name, n, rank, d, order, out))
        parts.append("")
        print(f"{name}: {c} ops", file=sys.stderr)
    for (name, g) in ROW_SPECS:
        d, order, outs = row_network(g)
        verify_row(g, d, order, outs, exhaustive)
        text, two, ins = emit_row(name, g, d, order, outs)
        parts.append(text)
        parts.append("")
        print(f"{name}: {two} ops, {ins} instructions", file=sys.stderr)
    with open(path, "w") as f:
        f.write("\n".join(parts))


if __name__ == "__main__":
    main(sys.argv[1], exhaustive="--quick" not in sys.argv)

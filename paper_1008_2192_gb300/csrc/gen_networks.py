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
    The three-input form issues at the rate of the two-input one on sm_103a.
    """
    uses = {}
    for v in order:
        k = d.defs[v]
        if k[0] in ("min", "max"):
            for u in k[1:]:
                uses[u] = uses.get(u, 0) + 1
    uses[out] = uses.get(out, 0) + 1
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
    with open(path, "w") as f:
        f.write("\n".join(parts))


if __name__ == "__main__":
    main(sys.argv[1], exhaustive="--quick" not in sys.argv)

"""Fit the arctangent polynomial used by the query kernels; writes atan_poly.cuh.

atan(t) = t * P(t^2) on 0 <= t <= 1 with P the polynomial of degree N in
s = t^2 that minimises the maximum RELATIVE error |t P(t^2) / atan(t) - 1|
(so small boundary terms keep a small relative error).  The fit is the Remez
exchange algorithm, in 50-digit arithmetic (mpmath), on f(s) = atan(sqrt s)/sqrt s
with weight 1/f(s).  The coefficients are then rounded to FP32 and the error of
the FP32 Horner evaluation is measured on a dense grid and written into the
header's comment.

Run:  python paper_2605_01536_gb300/csrc/fit_atan.py [N]
"""
from __future__ import annotations

import os
import sys

import mpmath as mp
import numpy as np

mp.mp.dps = 50
HERE = os.path.dirname(os.path.abspath(__file__))


def f(s):
    s = mp.mpf(s)
    if s == 0:
        return mp.mpf(1)
    r = mp.sqrt(s)
    return mp.atan(r) / r


def solve_reference(xs, n):
    """P(x_i) - f(x_i) = (-1)^i E f(x_i) for the n+2 reference points."""
    m = n + 2
    A = mp.matrix(m, m)
    b = mp.matrix(m, 1)
    for i, x in enumerate(xs):
        fx = f(x)
        for j in range(n + 1):
            A[i, j] = mp.mpf(x) ** j
        A[i, n + 1] = -((-1) ** i) * fx
        b[i] = fx
    sol = mp.lu_solve(A, b)
    return [sol[j] for j in range(n + 1)], sol[n + 1]


def rel_err(c, s):
    p = mp.mpf(0)
    for a in reversed(c):
        p = p * s + a
    return p / f(s) - 1


def remez(n, iters=30):
    xs = [mp.mpf(1) / 2 - mp.cos(mp.pi * i / (n + 1)) / 2 for i in range(n + 2)]
    grid = [mp.mpf(i) / 4000 for i in range(4001)]
    c, E = None, None
    for _ in range(iters):
        c, E = solve_reference(xs, n)
        err = [rel_err(c, s) for s in grid]
        # alternating extrema: split the grid where the error changes sign
        ext = []
        start = 0
        for i in range(1, len(grid) + 1):
            if i == len(grid) or mp.sign(err[i]) != mp.sign(err[start]):
                k = max(range(start, i), key=lambda j: abs(err[j]))
                ext.append(k)
                start = i
        while len(ext) > n + 2:   # drop the smallest end extremum
            if abs(err[ext[0]]) < abs(err[ext[-1]]):
                ext.pop(0)
            else:
                ext.pop()
        if len(ext) < n + 2:
            break
        new = [grid[k] for k in ext]
        if max(abs(a - b) for a, b in zip(new, xs)) < mp.mpf(1e-12):
            xs = new
            break
        xs = new
    return [float(x) for x in c], float(abs(E))


def fp32_error(c32):
    t = np.linspace(0.0, 1.0, 2_000_001, dtype=np.float64).astype(np.float32)
    s = (t * t).astype(np.float32)
    p = np.float32(c32[-1])
    p = np.full_like(s, c32[-1])
    for a in reversed(c32[:-1]):
        p = (p * s + np.float32(a)).astype(np.float32)
    r = (p * t).astype(np.float32)
    ref = np.arctan(t.astype(np.float64))
    nz = ref > 0
    rel = np.abs(r[nz].astype(np.float64) / ref[nz] - 1.0)
    ab = np.abs(r.astype(np.float64) - ref)
    return float(rel.max()), float(ab.max())


def main():
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 8
    c, E = remez(n)
    c32 = [float(np.float32(x)) for x in c]
    rel32, abs32 = fp32_error(c32)
    lines = [
        "// Generated by fit_atan.py: do not edit.",
        f"// atan(t) ~= t * P(t^2), 0 <= t <= 1, P of degree {n} (Remez, minimax relative error).",
        f"// Minimax relative error of the exact-coefficient fit: {E:.3e}",
        f"// FP32 coefficients, FP32 Horner: max relative error {rel32:.3e}, max absolute error {abs32:.3e}",
        "#pragma once",
        f"#define GWN_ATAN_DEGREE {n}",
        "// P(s) in Horner form",
        "__device__ __forceinline__ float gwn_atan_poly(float s) {",
        f"    float p = {c32[-1]!r}f;",
    ]
    lines += [f"    p = fmaf(p, s, {x!r}f);" for x in reversed(c32[:-1])]
    lines += ["    return p;", "}", "// the same coefficients for the paired-FP32 evaluation"]
    lines += [f"#define GWN_ATAN_C{i} {x!r}f" for i, x in enumerate(c32)]
    lines += [""]
    out = os.path.join(HERE, "atan_poly.cuh")
    with open(out, "w") as fh:
        fh.write("\n".join(lines))
    print(f"degree {n}: minimax rel {E:.3e}; fp32 rel {rel32:.3e} abs {abs32:.3e} -> {out}")


if __name__ == "__main__":
    main()

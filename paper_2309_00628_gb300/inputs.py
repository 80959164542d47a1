"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds no arithmetic of the method: it only draws matrices.  Every
matrix is drawn in float64 from numpy's PCG64 generator and then cast to the
dtype the caller asks for; the oracle receives the same cast values (upcast
back to float64), so both sides see identical inputs.

Distributions (the paper benchmarks square power-of-two orders 2^1..2^11 and
does not state a distribution; these stand in for its inputs):
  "uniform"  i.i.d. uniform[-1, 1]
  "int"      i.i.d. uniform integers in [-lim, lim] (default lim 8)
  "normal"   i.i.d. normal(0, 1)
Seeds: A uses ``seed``, B uses ``seed + 1`` (0 and 1 by default).
"""
from __future__ import annotations

import math

import numpy as np


def draw(shape, dist: str = "uniform", seed: int = 0, dtype=np.float32, lim: int = 8) -> np.ndarray:
    g = np.random.Generator(np.random.PCG64(seed))
    if dist == "uniform":
        x = g.uniform(-1.0, 1.0, size=shape)
    elif dist == "int":
        x = g.integers(-lim, lim + 1, size=shape).astype(np.float64)
    elif dist == "normal":
        x = g.standard_normal(size=shape)
    else:
        raise ValueError(f"unknown distribution {dist!r}")
    return np.ascontiguousarray(x.astype(dtype))


def pair(m: int, n: int, k: int, dist: str = "uniform", seed: int = 0, dtype=np.float32, lim: int = 8):
    """(A m x k, B k x n) drawn with seeds (seed, seed + 1)."""
    return (draw((m, k), dist, seed, dtype, lim), draw((k, n), dist, seed + 1, dtype, lim))


def batched_shapes(count: int = 512, lo: int = 96, hi: int = 3000, seed: int = 2):
    """m, n, k each round(exp(U(ln lo, ln hi))): the uneven batched workload."""
    g = np.random.Generator(np.random.PCG64(seed))
    u = g.uniform(math.log(lo), math.log(hi), size=(count, 3))
    dims = np.rint(np.exp(u)).astype(np.int64)
    return [tuple(int(v) for v in row) for row in dims]


def serving_requests(count: int = 40, seed: int = 3, sizes=(512, 1024, 2048, 4096, 8192), max_aspect: float = 8.0,
                     align: int = 32):
    """The serving mix: (m, n, k, elem_bytes) per request.

    elem_bytes is 4 or 8 with probability 1/2 each; a base order s is drawn uniformly from
    `sizes`; half the requests are square (s, s, s), the others rectangular with aspect
    a = exp(U(0, ln max_aspect)) between two of the three dimensions (s sqrt(a) and s / sqrt(a),
    rounded to a multiple of `align`, the third left at s, the dimensions in random order).
    """
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        eb = 4 if g.uniform() < 0.5 else 8
        s = int(sizes[int(g.integers(0, len(sizes)))])
        if g.uniform() < 0.5:
            dims = [s, s, s]
        else:
            a = math.exp(g.uniform(0.0, math.log(max_aspect)))
            hi = max(align, int(round(s * math.sqrt(a) / align)) * align)
            lo = max(align, int(round(s / math.sqrt(a) / align)) * align)
            dims = [hi, lo, s]
            g.shuffle(dims)
        out.append((int(dims[0]), int(dims[1]), int(dims[2]), eb))
    return out

"""Shared helpers for the GPU parity tests: instances, tolerances, comparisons.

Tolerance (FP32 path).  Every constraint value FE_c lies in [-1, 1].  The
node path evaluates each node's product prod_i (1 + i t_j y_i) with a relative
(norm-wise) rounding error of order L * eps32 and scales it so that the node's
term C_j Q_j has modulus at most |c_j|, so the FP32 rounding error of one
constraint is absolute, of order L * eps32 * sum_j |c_j| (at most ~1e-5 for
L = 512), not relative to the possibly tiny value of one term.  We therefore read the 1e-4 relative
tolerance of the FP32 path against the condition scale of each sum of signed
terms:
    |f - f*| <= 1e-4 * max(|f*|, sum_c w_c |FE_c*|)
    |g_v - g*_v| <= 1e-4 * max(|g*_v|, A_v),  A_v = sum_{c ni v} w_c max(|dFE_c/dy_v|, 1e-2 [node path])
(the node path carries every at-least-K constraint, and clauses and XORs too
when they are routed through it)
The 1e-2 floor for cardinality literals makes the per-literal allowance 1e-6
absolute per unit weight.  Measured FP32 errors of the node path reach
2-3e-7 absolute (L = 512, near-corner points; also short L = 8 constraints
whose node sums cancel), and the rounding bound grows like L * eps32 *
sum_j |d_j|; a wrong term, sign or index produces errors of order 1e-2 to 1.
FP64 path: the same scales with 1e-10 instead of 1e-4.
"""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_2308_15020_gb300 import gen

ATLEAST_FLOOR = 1e-2


def mixed_instance(seed: int = 0, n: int = 700, scale: int = 1, weights: bool = True) -> gen.Instance:
    """Clauses of 1..3 literals, long clauses, XOR (short, long, > 256), at-least-K
    of 1..512 literals with K in {0, 1, ~L/2, L, L+1}; random weights."""
    rng = np.random.default_rng(seed)
    cons = []

    def pick(L):
        vs = rng.choice(n, size=L, replace=False) + 1
        return (vs * rng.choice([-1, 1], size=L)).tolist()

    for _ in range(300 * scale):
        cons.append((gen.OR, 0, pick(int(rng.integers(1, 4)))))
    for L in [4, 5, 9, 17, 31, 64, 100, 255, 256, 257, 300, 512]:
        cons.append((gen.OR, 0, pick(L)))
    for L in [1, 2, 3, 7, 8, 16, 33, 40, 64, 129, 256, 257, 400, 512]:
        cons.append((gen.XOR, int(rng.integers(0, 2)), pick(L)))
    for L in [1, 2, 3, 5, 8, 15, 16, 17, 31, 32, 33, 63, 64, 65, 100, 127, 128, 129, 200, 255, 256, 257, 300, 400,
              511, 512]:
        for K in sorted({0, 1, max(1, L // 2), L, L + 1, min(L, L // 2 + L // 8)}):
            cons.append((gen.ATLEAST, K, pick(L)))
    w = rng.uniform(0.25, 2.0, size=len(cons)) if weights else None
    return gen.from_lists(n, cons, w, name=f"mixed{seed}")


def oracle_fg(inst, x, weights=None):
    return O.eval_grad(inst, np.asarray(x, dtype=np.float64), weights=weights)


def compare(inst, x, f, g, rtol: float, weights=None, points=None, node_types=(O.ATLEAST,)):
    """Max normalised errors of f and g against the oracle (<= 1 passes).

    node_types: constraint types evaluated on the node (DFT) path, whose FP32
    error is absolute; their literals get the ATLEAST_FLOOR condition scale."""
    x = np.asarray(x, dtype=np.float64)
    if points is not None:
        x = x[points]
        f = None if f is None else f[points]
        g = None if g is None else g[points]
    fs, gs = oracle_fg(inst, x, weights)
    sf, A = O.eval_scale(inst, x, ATLEAST_FLOOR, weights=weights, floor_types=node_types)
    ef = eg = 0.0
    if f is not None:
        ef = float(np.max(np.abs(f - fs) / (rtol * np.maximum(np.abs(fs), np.maximum(sf, 1e-300)))))
    if g is not None:
        den = rtol * np.maximum(np.abs(gs), A)
        diff = np.abs(g - gs)
        zero = den == 0
        eg = float(np.max(np.where(zero, diff / 1e-300, diff / np.where(zero, 1, den)))) if diff.size else 0.0
    return ef, eg


def to_np(t):
    return t.detach().cpu().numpy()

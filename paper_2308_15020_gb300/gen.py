"""Seeded synthetic instances and restart points.

This module is the only code shared by the CUDA path and the FP64 oracle.  It
draws constraint sets and points and holds none of the method's arithmetic
(no Walsh coefficients, no products, no gradients).

Conventions (Preliminaries, "Walsh Expansions"): a variable value -1 means
True and +1 means False.  Literals are DIMACS-style signed 1-based integers:
+v is x_v, -v is its negation.  Constraint types:

* OR (0): a CNF clause, satisfied when at least one literal is True;
* XOR (1): satisfied when the number of True literals has parity ``param``
  (param=1 is the usual exclusive-or of the literals);
* ATLEAST (2): satisfied when at least ``param`` literals are True
  (the cardinality constraints of Example 1 and Benchmark 1).

Workload shapes follow the paper's settings where it states them: random
3-SAT at clause ratio 4.26 (the SATLIB uf series of the ablation, App. C),
the RQ1 XOR/cardinality formulas (App. D, "Random Boolean Formula") and
Benchmark 1 random cardinality (App. D).  The SATLIB, MSE19 and competition
files themselves are not used: these seeded generators stand in for them.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

OR, XOR, ATLEAST = 0, 1, 2


@dataclass
class Instance:
    """A hybrid constraint set in CSR form (host arrays)."""

    n: int
    row_ptr: np.ndarray  # int64 [m+1]
    lits: np.ndarray  # int32 [nnz], signed 1-based
    ctype: np.ndarray  # uint8 [m]
    param: np.ndarray  # int32 [m]
    weights: np.ndarray  # float64 [m]
    name: str = ""
    planted: Optional[np.ndarray] = field(default=None, repr=False)  # int8 [n] in {-1,+1}
    target_unsat: int = 0  # an assignment counts as a solution with at most this many violated constraints

    @property
    def m(self) -> int:
        return int(self.ctype.shape[0])

    @property
    def nnz(self) -> int:
        return int(self.lits.shape[0])

    def lengths(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def constraint(self, c: int):
        a, b = int(self.row_ptr[c]), int(self.row_ptr[c + 1])
        return int(self.ctype[c]), int(self.param[c]), self.lits[a:b]


def _rng(seed: int, stream: int) -> np.random.Generator:
    """Counter-based Philox stream keyed by (seed, stream)."""
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([int(seed) & 0xFFFFFFFF, int(stream)])))


def from_lists(n: int, cons: Sequence[tuple], weights: Optional[Sequence[float]] = None, name: str = "") -> Instance:
    """Build an instance from ``[(ctype, param, [lits...]), ...]``."""
    row_ptr = np.zeros(len(cons) + 1, dtype=np.int64)
    lits: List[int] = []
    ctype = np.zeros(len(cons), dtype=np.uint8)
    param = np.zeros(len(cons), dtype=np.int32)
    for i, (t, p, ls) in enumerate(cons):
        ctype[i] = t
        param[i] = p
        lits.extend(int(v) for v in ls)
        row_ptr[i + 1] = len(lits)
    w = np.ones(len(cons), dtype=np.float64) if weights is None else np.asarray(weights, dtype=np.float64)
    return Instance(n, row_ptr, np.asarray(lits, dtype=np.int32), ctype, param, w, name)


def concat(parts: Sequence[Instance], name: str = "") -> Instance:
    """Concatenate constraint sets over the same variables."""
    n = max(p.n for p in parts)
    offs = [0]
    for p in parts:
        offs.append(offs[-1] + p.nnz)
    row_ptr = [np.zeros(1, dtype=np.int64)]
    for p, o in zip(parts, offs):
        row_ptr.append(p.row_ptr[1:] + o)
    planted = next((p.planted for p in parts if p.planted is not None), None)
    return Instance(
        n,
        np.concatenate(row_ptr).astype(np.int64),
        np.concatenate([p.lits for p in parts]).astype(np.int32),
        np.concatenate([p.ctype for p in parts]).astype(np.uint8),
        np.concatenate([p.param for p in parts]).astype(np.int32),
        np.concatenate([p.weights for p in parts]).astype(np.float64),
        name,
        planted,
    )


def _distinct_rows(rng: np.random.Generator, n: int, m: int, k: int) -> np.ndarray:
    """m rows of k distinct variable indices in [0, n), uniform."""
    v = rng.integers(0, n, size=(m, k))
    while True:
        s = np.sort(v, axis=1)
        bad = np.any(s[:, 1:] == s[:, :-1], axis=1) if k > 1 else np.zeros(m, dtype=bool)
        if not bad.any():
            return v
        v[bad] = rng.integers(0, n, size=(int(bad.sum()), k))


def _signs(rng: np.random.Generator, shape) -> np.ndarray:
    return np.where(rng.random(shape) < 0.5, 1, -1)


def _lit_true(lits: np.ndarray, assign: np.ndarray) -> np.ndarray:
    """Which literals are True under a +-1 assignment (True is -1)."""
    v = np.abs(lits) - 1
    val = assign[v] * np.sign(lits)
    return val < 0


def planted_assignment(n: int, seed: int) -> np.ndarray:
    return _signs(_rng(seed, 99), n).astype(np.int8)


def random_ksat(n: int, m: int, k: int = 3, seed: int = 0, planted: Optional[np.ndarray] = None, stream: int = 1) -> Instance:
    """Uniform random k-SAT: k distinct variables per clause, signs +-1 with p=1/2.

    With ``planted`` set, clauses violated by that assignment are redrawn, so
    the instance is satisfiable by construction.
    """
    rng = _rng(seed, stream)
    v = _distinct_rows(rng, n, m, k)
    s = _signs(rng, (m, k))
    lits = (v + 1) * s
    if planted is not None:
        while True:
            sat = _lit_true(lits.reshape(-1), planted).reshape(m, k).any(axis=1)
            if sat.all():
                break
            nb = int((~sat).sum())
            v2 = _distinct_rows(rng, n, nb, k)
            lits[~sat] = (v2 + 1) * _signs(rng, (nb, k))
    row_ptr = np.arange(0, m * k + 1, k, dtype=np.int64)
    return Instance(n, row_ptr, lits.reshape(-1).astype(np.int32), np.full(m, OR, np.uint8), np.zeros(m, np.int32), np.ones(m), f"{k}sat", planted)


def random_xor(n: int, m: int, lmin: int, lmax: int, seed: int = 0, planted: Optional[np.ndarray] = None, stream: int = 2, signs: bool = False) -> Instance:
    """XOR constraints of length U{lmin..lmax} on distinct uniform variables and random parity.

    With ``planted`` set, each parity is chosen so that the planted
    assignment satisfies the constraint.
    """
    rng = _rng(seed, stream)
    L = rng.integers(lmin, lmax + 1, size=m)
    row_ptr = np.concatenate([[0], np.cumsum(L)]).astype(np.int64)
    lits = np.empty(int(row_ptr[-1]), dtype=np.int32)
    par = rng.integers(0, 2, size=m).astype(np.int32)
    for c in range(m):
        vs = rng.choice(n, size=int(L[c]), replace=False) + 1
        sg = _signs(rng, int(L[c])) if signs else np.ones(int(L[c]), dtype=np.int64)
        ls = vs * sg
        lits[row_ptr[c] : row_ptr[c + 1]] = ls
        if planted is not None:
            par[c] = int(_lit_true(ls, planted).sum()) & 1
    return Instance(n, row_ptr, lits, np.full(m, XOR, np.uint8), par, np.ones(m), "xor", planted)


def random_atleast(
    n: int,
    m: int,
    lmin: int,
    lmax: int,
    seed: int = 0,
    planted: Optional[np.ndarray] = None,
    stream: int = 3,
    k_rule: str = "half_pm_eighth",
    sign_rule: str = "per_literal",
) -> Instance:
    """At-least-K constraints of length U{lmin..lmax} on distinct uniform variables.

    ``k_rule``:
      * ``half_pm_eighth``: K = L//2 + s*U{0..L//8}, s = +-1, clamped to [1, L];
      * ``half``: K = ceil(L/2) (the RQ1 reading) ;
      * ``half_floor``: K = L//2 (Benchmark 1: "l/2-cardinality").
    ``sign_rule``: ``per_literal`` (+-1 each, p=1/2) or ``all_same`` (Benchmark 1:
    all literals of a constraint positive or all negative with p=1/2).
    With ``planted`` set, K is lowered where needed so the planted assignment
    satisfies the constraint.
    """
    rng = _rng(seed, stream)
    L = rng.integers(lmin, lmax + 1, size=m)
    row_ptr = np.concatenate([[0], np.cumsum(L)]).astype(np.int64)
    lits = np.empty(int(row_ptr[-1]), dtype=np.int32)
    K = np.empty(m, dtype=np.int32)
    for c in range(m):
        l = int(L[c])
        vs = rng.choice(n, size=l, replace=False) + 1
        if sign_rule == "all_same":
            sg = np.full(l, 1 if rng.random() < 0.5 else -1)
        else:
            sg = _signs(rng, l)
        ls = vs * sg
        lits[row_ptr[c] : row_ptr[c + 1]] = ls
        if k_rule == "half_pm_eighth":
            d = int(rng.integers(0, l // 8 + 1))
            k = l // 2 + (d if rng.random() < 0.5 else -d)
        elif k_rule == "half":
            k = (l + 1) // 2
        else:
            k = l // 2
        k = min(max(k, 1), l)
        if planted is not None:
            k = min(k, int(_lit_true(ls, planted).sum()))
            k = max(k, 0)
        K[c] = k
    return Instance(n, row_ptr, lits, np.full(m, ATLEAST, np.uint8), K, np.ones(m), "atleast", planted)


# --------------------------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------------------------


def uniform_3sat_100(seed: int = 0, planted: bool = False) -> Instance:
    """Random 3-SAT, n=100, m=426 (uf100 shape), unit weights."""
    p = planted_assignment(100, seed) if planted else None
    inst = random_ksat(100, 426, 3, seed, planted=p)
    inst.name = "3sat_n100_m426"
    return inst


def cnf_xor_2000(seed: int = 0, planted: bool = False, n: int = 2000) -> Instance:
    """Hybrid CNF-XOR: n=2000, 8400 random 3-clauses + 200 XOR of length U{10..40}.

    ``n`` rescales the shape (m = 4.2n clauses, n/10 XORs) for the larger
    held-out instances of the restart study.
    """
    p = planted_assignment(n, seed) if planted else None
    a = random_ksat(n, int(round(4.2 * n)), 3, seed, planted=p)
    b = random_xor(n, n // 10, 10, 40, seed, planted=p)
    return concat([a, b], f"cnf_xor_n{n}")


def cnf_card_20000(seed: int = 0, planted: bool = False) -> Instance:
    """CNF + cardinality: n=20000, 84000 3-clauses + 500 at-least-K of length U{64..512}."""
    p = planted_assignment(20000, seed) if planted else None
    a = random_ksat(20000, 84000, 3, seed, planted=p)
    b = random_atleast(20000, 500, 64, 512, seed, planted=p)
    return concat([a, b], "cnf_card_n20000")


def uneven_batch(seed: int = 0, count: int = 64) -> List[Instance]:
    """64 uneven instances: n log-uniform in [500, 50000], clause ratio U[4.0, 4.3],
    XOR fraction U[0, 5%] (length 10..60), cardinality fraction U[0, 2%] (length 32..512,
    capped at n)."""
    rng = _rng(seed, 7)
    out = []
    for i in range(count):
        n = int(round(np.exp(rng.uniform(np.log(500), np.log(50000)))))
        ratio = rng.uniform(4.0, 4.3)
        fx = rng.uniform(0.0, 0.05)
        fc = rng.uniform(0.0, 0.02)
        m_total = int(round(ratio * n))
        mx = int(round(fx * m_total))
        mc = int(round(fc * m_total))
        mcl = max(m_total - mx - mc, 1)
        s = seed * 1000 + i
        parts = [random_ksat(n, mcl, 3, s)]
        if mx:
            parts.append(random_xor(n, mx, 10, min(60, n), s))
        if mc:
            parts.append(random_atleast(n, mc, min(32, n), min(512, n), s))
        inst = concat(parts, f"uneven{i}_n{n}")
        out.append(inst)
    return out


RQ1_SHAPES = {
    # App. D "Random Boolean Formula": (XOR count, XOR length, cardinality count, cardinality length)
    "xor1": (200, 8, 0, 0),
    "xor2": (400, 16, 0, 0),
    "xor3": (800, 32, 0, 0),
    "card1": (0, 0, 50, 8),
    "card2": (0, 0, 100, 16),
    "card3": (0, 0, 200, 32),
    "xor+card": (800, 8, 1, 32),
}


def rq1(name: str, seed: int = 0, n: int = 1024) -> Instance:
    """The RQ1 gradient-timing formulas; n is not stated in the paper (n=1024 here),
    and K = ceil(L/2) for the cardinality constraints."""
    nx, lx, nc, lc = RQ1_SHAPES[name]
    parts = []
    if nx:
        parts.append(random_xor(n, nx, lx, lx, seed, signs=True))
    if nc:
        parts.append(random_atleast(n, nc, lc, lc, seed, k_rule="half"))
    return concat(parts, f"rq1_{name}")


def bench1_cardinality(N: int, seed: int = 0) -> Instance:
    """Benchmark 1: m=0.6N constraints over l=0.2N variables each, K=l/2, all-same signs."""
    l = int(round(0.2 * N))
    m = int(round(0.6 * N))
    inst = random_atleast(N, m, l, l, seed, k_rule="half_floor", sign_rule="all_same")
    inst.name = f"bench1_N{N}"
    return inst


def parity_learning(N: int, seed: int = 0, e: float = 0.25) -> Instance:
    """Benchmark 2, parity learning with error: a hidden parity function over a
    subset S of the N variables (each variable in S with probability 1/2) and
    m = 2N samples a_j ~ U{0,1}^N (an all-zero sample is redrawn) labelled
    b_j = |S cap a_j| mod 2, of which floor(e m) chosen at random are flipped.
    Sample j becomes the XOR over {i : a_j,i = 1} with parity b_j; variable i is
    True (-1) iff i is in S.  The hidden S violates exactly floor(e m)
    constraints, so a solution is an assignment with at most that many
    violations (target_unsat)."""
    rng = _rng(seed, 5)
    m = 2 * N
    hidden = np.where(rng.random(N) < 0.5, -1, 1).astype(np.int8)  # -1: i in S
    rows = []
    for _ in range(m):
        a = rng.random(N) < 0.5
        while not a.any():
            a = rng.random(N) < 0.5
        rows.append(np.flatnonzero(a) + 1)
    par = np.array([int(np.sum(hidden[r - 1] < 0)) & 1 for r in rows], dtype=np.int32)
    flips = rng.choice(m, size=int(np.floor(e * m)), replace=False)
    par[flips] ^= 1
    row_ptr = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
    lits = np.concatenate(rows).astype(np.int32)
    return Instance(N, row_ptr, lits, np.full(m, XOR, np.uint8), par, np.ones(m), f"plwe_N{N}", hidden,
                    int(np.floor(e * m)))


def planted_maxcut(l: int, k: int, seed: int = 0, p_edge: float = 0.5) -> Instance:
    """Benchmark 3, weighted Max-Cut on a planted-partition graph: l clusters of
    k vertices, each vertex pair joined with probability p_edge (unstated in the
    paper; 0.5 gives the paper's "more than 260000 edges" at l = k = 32), weight
    1 inside a cluster and 2 between clusters.  Edge (u, v) becomes the XOR of
    u and v with odd parity (satisfied iff the edge is cut), weighted by the edge
    weight; maximising the cut is minimising the weight of violated XORs."""
    rng = _rng(seed, 6)
    n = l * k
    cl = np.repeat(np.arange(l), k)
    iu, iv = np.triu_indices(n, 1)
    keep = rng.random(iu.shape[0]) < p_edge
    iu, iv = iu[keep], iv[keep]
    w = np.where(cl[iu] == cl[iv], 1.0, 2.0)
    m = iu.shape[0]
    lits = np.empty(2 * m, dtype=np.int32)
    lits[0::2] = iu + 1
    lits[1::2] = iv + 1
    row_ptr = np.arange(0, 2 * m + 1, 2, dtype=np.int64)
    return Instance(n, row_ptr, lits, np.full(m, XOR, np.uint8), np.ones(m, np.int32), w, f"maxcut_{l}x{k}")


def cut_weight(inst: Instance, z: np.ndarray) -> float:
    """Total weight of the cut edges (XOR satisfied) under a +-1 assignment."""
    u = np.abs(inst.lits[0::2]) - 1
    v = np.abs(inst.lits[1::2]) - 1
    return float(np.sum(inst.weights[z[u] != z[v]]))


WORKLOADS = {
    "3sat_n100": uniform_3sat_100,
    "cnf_xor_n2000": cnf_xor_2000,
    "cnf_card_n20000": cnf_card_20000,
}


# --------------------------------------------------------------------------------------------
# Points
# --------------------------------------------------------------------------------------------


def uniform_points(B: int, n: int, seed: int = 0, dtype=np.float32) -> np.ndarray:
    """x ~ U[-1, 1]^n for each of B restart points (Alg. 1, first line)."""
    return _rng(seed, 11).uniform(-1.0, 1.0, size=(B, n)).astype(dtype)


def near_corner_points(B: int, n: int, seed: int = 0, dtype=np.float32) -> np.ndarray:
    """x = s * (1 - 0.1 u^4), s = +-1, u ~ U[0, 1]: points close to cube corners."""
    rng = _rng(seed, 12)
    s = _signs(rng, (B, n))
    u = rng.random((B, n))
    return (s * (1.0 - 0.1 * u**4)).astype(dtype)


def corner_points(B: int, n: int, seed: int = 0, dtype=np.float32, zero_frac: float = 0.1) -> np.ndarray:
    """Exact corners +-1 with a fraction of exact zeros (and signed zeros)."""
    rng = _rng(seed, 13)
    x = _signs(rng, (B, n)).astype(np.float64)
    z = rng.random((B, n)) < zero_frac
    neg = rng.random((B, n)) < 0.5
    x[z & neg] = -0.0
    x[z & ~neg] = 0.0
    return x.astype(dtype)


def dyadic_points(B: int, n: int, seed: int = 0, bits: int = 6, dtype=np.float64) -> np.ndarray:
    """x = k / 2^bits, k uniform in [-2^bits, 2^bits]: exactly representable points."""
    rng = _rng(seed, 14)
    k = rng.integers(-(1 << bits), (1 << bits) + 1, size=(B, n))
    return (k / float(1 << bits)).astype(dtype)


def dpll_model(inst: Instance, max_nodes: int = 2_000_000) -> Optional[np.ndarray]:
    """A model of a pure CNF instance found by DPLL (unit propagation, branching
    on the variable with the largest Jeroslow-Wang score), or None when the
    formula is unsatisfiable.  Selects satisfiable seeds of the random 3-SAT
    workload; raises RuntimeError past max_nodes search nodes.  Models use the
    paper's encoding: -1 True, +1 False."""
    if np.any(inst.ctype != OR):
        raise ValueError("dpll_model takes clauses only")
    n = inst.n
    clauses = [list(inst.lits[inst.row_ptr[c]:inst.row_ptr[c + 1]]) for c in range(inst.m)]
    occ = [[] for _ in range(2 * n + 2)]  # literal -> clauses containing it
    for ci, cl in enumerate(clauses):
        for l in cl:
            occ[l + n].append(ci)
    val = [0] * (n + 1)  # 0 unassigned, +1 True, -1 False (literal l is true iff val[|l|] * sign(l) > 0)
    nodes = [0]

    def lit_val(l):
        v = val[abs(l)]
        return 0 if v == 0 else (1 if (v > 0) == (l > 0) else -1)

    def propagate(trail):
        changed = True
        while changed:
            changed = False
            for cl in clauses:
                free, sat = None, False
                nfree = 0
                for l in cl:
                    s = lit_val(l)
                    if s > 0:
                        sat = True
                        break
                    if s == 0:
                        nfree += 1
                        free = l
                if sat:
                    continue
                if nfree == 0:
                    return False
                if nfree == 1:
                    val[abs(free)] = 1 if free > 0 else -1
                    trail.append(abs(free))
                    changed = True
        return True

    def pick():
        score = {}
        for cl in clauses:
            if any(lit_val(l) > 0 for l in cl):
                continue
            free = [l for l in cl if lit_val(l) == 0]
            w = 2.0 ** -len(free)
            for l in free:
                score[l] = score.get(l, 0.0) + w
        if not score:
            return None
        return max(score.items(), key=lambda kv: kv[1])[0]

    def solve():
        nodes[0] += 1
        if nodes[0] > max_nodes:
            raise RuntimeError("dpll_model: node budget exceeded")
        trail = []
        if not propagate(trail):
            for v in trail:
                val[v] = 0
            return False
        l = pick()
        if l is None:
            return True
        for choice in (l, -l):
            val[abs(choice)] = 1 if choice > 0 else -1
            if solve():
                return True
            val[abs(choice)] = 0
        for v in trail:
            val[v] = 0
        return False

    import sys
    old = sys.getrecursionlimit()
    sys.setrecursionlimit(max(old, 10 * n + 100))
    try:
        ok = solve()
    finally:
        sys.setrecursionlimit(old)
    if not ok:
        return None
    return np.array([-1 if val[v] > 0 else 1 for v in range(1, n + 1)], dtype=np.int8)


def satisfiable_3sat_100(count: int, seed0: int = 0):
    """The first `count` seeds >= seed0 whose uniform random 3-SAT n=100, m=426
    instance is satisfiable (decided by dpll_model), with the instances."""
    out = []
    s = seed0
    while len(out) < count:
        inst = uniform_3sat_100(s)
        if dpll_model(inst) is not None:
            out.append((s, inst))
        s += 1
    return out

"""Seeded generators: determinism, shapes, distinct variables per constraint."""
import numpy as np

from paper_2308_15020_gb300 import gen


def _distinct(inst):
    for c in range(inst.m):
        _, _, ls = inst.constraint(c)
        v = np.abs(ls)
        if len(np.unique(v)) != len(v):
            return False
    return True


def test_deterministic():
    a, b = gen.cnf_xor_2000(3), gen.cnf_xor_2000(3)
    for k in ("row_ptr", "lits", "ctype", "param", "weights"):
        assert np.array_equal(getattr(a, k), getattr(b, k))
    assert not np.array_equal(a.lits, gen.cnf_xor_2000(4).lits)
    assert np.array_equal(gen.uniform_points(4, 10, 1), gen.uniform_points(4, 10, 1))


def test_shapes():
    i2 = gen.cnf_xor_2000(0)
    assert i2.n == 2000 and i2.m == 8600
    L = i2.lengths()
    assert (L[:8400] == 3).all() and L[8400:].min() >= 10 and L[8400:].max() <= 40
    assert _distinct(i2)
    i3 = gen.cnf_card_20000(0)
    L3 = i3.lengths()
    assert i3.m == 84500 and (L3[84000:] >= 64).all() and (L3[84000:] <= 512).all()
    K = i3.param[84000:]
    assert ((K >= 1) & (K <= L3[84000:])).all()
    assert (np.abs(K - L3[84000:] // 2) <= L3[84000:] // 8).all()
    assert _distinct(gen.random_atleast(2000, 30, 64, 512, 1))
    i1 = gen.uniform_3sat_100(0)
    assert i1.n == 100 and i1.m == 426 and _distinct(i1)


def test_rq1_shapes():
    for name, (nx, lx, nc, lc) in gen.RQ1_SHAPES.items():
        inst = gen.rq1(name)
        assert inst.m == nx + nc
        assert inst.nnz == nx * lx + nc * lc


def test_points():
    x = gen.near_corner_points(8, 100, 0)
    assert (np.abs(x) >= 0.9).all() and (np.abs(x) <= 1).all()
    z = gen.corner_points(8, 100, 0)
    assert set(np.unique(np.abs(z))) <= {0.0, 1.0}
    assert np.signbit(z[z == 0]).any()


def test_parity_learning_recipe():
    """Benchmark 2: m = 2N XOR samples; the hidden parity violates exactly floor(e m)."""
    import oracle as O

    for N, seed in ((20, 0), (40, 3), (60, 7)):
        inst = gen.parity_learning(N, seed)
        assert inst.m == 2 * N and inst.target_unsat == N // 2
        assert np.all(inst.ctype == gen.XOR) and np.all(inst.lengths() >= 1)
        assert abs(inst.lengths().mean() / N - 0.5) < 0.1
        _, nun = O.check(inst, inst.planted.astype(np.float64)[None])
        assert nun[0] == inst.target_unsat


def test_planted_maxcut_recipe():
    """Benchmark 3: 2-XOR per edge, weight 1 inside a cluster and 2 across; the
    weight of cut edges plus the weight the oracle's checker counts as violated
    is the total."""
    import oracle as O

    inst = gen.planted_maxcut(4, 6, 2)
    n = 24
    assert inst.n == n and np.all(inst.lengths() == 2) and np.all(inst.param == 1)
    u = np.abs(inst.lits[0::2]) - 1
    v = np.abs(inst.lits[1::2]) - 1
    assert np.all(u < v)
    same = (u // 6) == (v // 6)
    assert np.array_equal(inst.weights, np.where(same, 1.0, 2.0))
    assert 0.3 < inst.m / (n * (n - 1) / 2) < 0.7
    z = np.where(np.arange(n) % 3 == 0, -1, 1)
    U = O.unsat_counts(inst, z.astype(np.float64)[None])
    assert gen.cut_weight(inst, z) + float(np.sum(inst.weights[U > 0])) == float(inst.weights.sum())

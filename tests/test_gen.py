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

"""Pins of the FP64 oracle to the paper's worked examples and to mathematics
that does not depend on the oracle's own code (brute force, exact rationals,
closed-form distributions).  CPU only."""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2308_15020_gb300 import gen

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name):
    out = {}
    with open(os.path.join(GOLD, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = (s.strip() for s in line.split("=", 1))
            out[k] = [Fraction(t) for t in v.split()]
    return out


def fl(xs):
    return np.array([float(t) for t in xs])


# ---------------------------------------------------------------------------------------------
# Worked examples
# ---------------------------------------------------------------------------------------------


def test_example1_walsh_coefficients():
    g = golden("example1_walsh.txt")
    L, K = int(g["L"][0]), int(g["K"][0])
    a = O.walsh_by_size(O.ATLEAST, K, L)  # a[m] on e_m
    want = fl(g["coef_e4_to_e0"])[::-1]  # -> e0..e4
    assert np.array_equal(a, want)
    # symmetry: every subset of the same size has the same coefficient (Thm. corner sum)
    for mask in range(1 << L):
        m = bin(mask).count("1")
        assert O.walsh_subset(O.ATLEAST, K, L, mask) == want[m]


@pytest.mark.parametrize("route", ["bruteforce", "corners", "esp", "paper", "dp", "default"])
def test_example2_gradient_all_routes(route):
    g = golden("example2_gradient.txt")
    K = int(g["K"][0])
    v, dy = O.fe(O.ATLEAST, K, fl(g["x"]), route)
    assert np.allclose(dy, fl(g["grad"]), rtol=0, atol=1e-14)
    assert abs(v - (-59 / 128)) < 1e-14


def test_example3_ftilde_and_value():
    g = golden("example3_forward.txt")
    L, K = int(g["L"][0]), int(g["K"][0])
    w = np.exp(-2j * np.pi / (L + 1))
    scale = float(g["ftilde_scale"][0])
    ft = O.paper_ftilde(O.ATLEAST, K, L)
    for j in range(L + 1):
        coefs = fl(g[f"ftilde{j}"])
        want = scale * sum(c * w**p for p, c in enumerate(coefs))
        assert abs(ft[j] - want) < 1e-14, (j, ft[j], want)
    v, _ = O.fe(O.ATLEAST, K, fl(g["x"]), "paper")
    assert abs(v - float(g["WE"][0])) < 1e-14


def test_gradsat_probabilities():
    g = golden("gradsat_example.txt")
    v, _ = O.fe(O.ATLEAST, 2, fl(g["x"]), "dp")
    # FE = P(false) * (+1) + P(true) * (-1)
    assert v == float(g["P_false"][0] - g["P_true"][0])
    assert g["P_true"][0] + g["P_false"][0] == 1


def _poly2(coef, x1, x2):
    c, a1, a2, a12 = (float(t) for t in coef)
    return c + a1 * x1 + a2 * x2 + a12 * x1 * x2


def test_saddle_example_objective():
    g = golden("saddle_example.txt")
    inst = gen.from_lists(2, [(gen.OR, 0, [1, -2]), (gen.XOR, 1, [-1, 2])])
    rng = np.random.default_rng(0)
    pts = rng.uniform(-1, 1, size=(8, 2))
    f, _ = O.eval_grad(inst, pts)
    assert np.allclose(f, [_poly2(g["F"], *p) for p in pts], atol=1e-15)
    # the inner point where the gradient vanishes
    f0, g0 = O.eval_grad(inst, fl(g["stationary"])[None])
    assert np.allclose(g0, 0.0, atol=1e-15)
    # reweighted objective
    w = fl(g["weights_after"])
    f1, _ = O.eval_grad(inst, pts, weights=w)
    assert np.allclose(f1, [_poly2(g["F_after"], *p) for p in pts], atol=1e-15)


def test_erwa_saddle_and_local_examples():
    """Prop. "Adaptive weight" with alpha = 0.4 reproduces the weights printed in
    the saddle and local-optimum examples from their unsatisfaction scores."""
    sad = golden("saddle_example.txt")
    inst = gen.from_lists(2, [(gen.OR, 0, [1, -2]), (gen.XOR, 1, [-1, 2])])
    # at the saddle's sign vector c1 is satisfied and c2 violated (r = (0, 1))
    x = fl(sad["stationary"])[None]
    U = O.unsat_counts(inst, x)
    assert list(U) == [0, 1]
    assert np.allclose(O.erwa(U, [1.0, 1.0], 0.4), fl(sad["weights_after"]), atol=1e-15)
    loc = golden("local_example.txt")
    inst = gen.from_lists(4, [(gen.XOR, 1, [1, 2]), (gen.XOR, 1, [2, 3]), (gen.XOR, 1, [3, 4])])
    U = O.unsat_counts(inst, fl(loc["point"])[None])
    assert list(U) == [0, 1, 0]
    assert np.allclose(O.erwa(U, [1.0, 1.0, 1.0], 0.4), fl(loc["weights_after"]), atol=1e-15)


def test_erwa_is_the_recency_weighted_average():
    """Sec. "Weighting Heuristics": from w = 0, t updates give the ERWA sum
    w^(t) = sum_i alpha (1 - alpha)^(t - i) r^(i) with r^(i) = U^(i) / max U^(i)."""
    rng = np.random.default_rng(3)
    m, alpha = 9, 0.4
    w = np.zeros(m)
    rs = []
    for t in range(6):
        U = rng.integers(0, 20, size=m).astype(np.int32)
        if t == 2:
            U[:] = 0  # no violated constraint: r = 0 everywhere
        rs.append(U / U.max() if U.max() > 0 else np.zeros(m))
        w = O.erwa(U, w, alpha)
        ref = sum(alpha * (1 - alpha) ** (t - i) * rs[i] for i in range(t + 1))
        assert np.allclose(w, ref, rtol=0, atol=1e-14)
    # decay only when nothing is violated
    assert np.array_equal(O.erwa(np.zeros(3, np.int32), [1.0, 2.0, 0.5], 0.4), np.array([0.6, 1.2, 0.3]))


def test_unsat_counts_brute_force():
    """U_c counts, over the points, the sign vectors that violate c (checked by
    direct evaluation of each constraint's Boolean definition)."""
    inst = gen.concat([gen.random_ksat(12, 30, 3, 5), gen.random_xor(12, 6, 2, 5, 5),
                       gen.random_atleast(12, 5, 2, 8, 5)])
    x = gen.uniform_points(11, 12, 4, dtype=np.float64)
    U = O.unsat_counts(inst, x)
    rp, lits = inst.row_ptr, inst.lits
    for c in range(inst.m):
        cnt = 0
        for b in range(x.shape[0]):
            ls = lits[rp[c]:rp[c + 1]]
            true = [(x[b, abs(l) - 1] < 0) == (l > 0) for l in ls]  # x < 0 encodes True
            s = sum(true)
            t, p = inst.ctype[c], inst.param[c]
            ok = s >= 1 if t == gen.OR else (s % 2 == p % 2 if t == gen.XOR else s >= p)
            cnt += not ok
        assert U[c] == cnt, c
    _, nun = O.check(inst, x)
    assert U.sum() == nun.sum()


def test_rephase_phases():
    """Sec. "Rephasing Heuristics": original keeps, flipped negates, random draws
    the same uniform point as the restart of a CLS round; solved points stay."""
    inst = gen.random_ksat(40, 400, 3, 9)  # unsatisfiable in practice at ratio 10
    x = gen.uniform_points(6, 40, 2, dtype=np.float64)
    solved = np.array([0, 1, 0, 0, 1, 0], np.uint8)
    assert np.array_equal(O.rephase(x, 0, solved), x)
    xf = O.rephase(x, 1, solved)
    assert np.array_equal(xf[solved == 1], x[solved == 1]) and np.array_equal(xf[solved == 0], -x[solved == 0])
    assert np.array_equal(O.rephase(xf, 1, solved), x)
    xr = O.rephase(x, 2, None, seed=7, epoch=3, b_offset=100)
    assert np.all((xr >= -1) & (xr < 1)) and np.array_equal(xr * 2.0**23, np.round(xr * 2.0**23))
    xs, ok, _ = O.step(inst, x, T=0, lr=0.1, seed=7, epoch=3, b_offset=100, restart=True)
    assert not ok.any()
    assert np.array_equal(xr, xs)
    with pytest.raises(ValueError):
        O.rephase(x, 3)


def test_local_optimum_example_gradient():
    g = golden("local_example.txt")
    inst = gen.from_lists(4, [(gen.XOR, 1, [1, 2]), (gen.XOR, 1, [2, 3]), (gen.XOR, 1, [3, 4])])
    p = fl(g["point"])[None]
    f, _ = O.eval_grad(inst, p)
    assert f[0] == 1 * -1 + -1 * -1 + -1 * 1  # F = x1x2 + x2x3 + x3x4
    _, gr = O.eval_grad(inst, p, weights=fl(g["weights_after"]))
    assert np.allclose(gr[0], fl(g["grad_after"]), atol=1e-15)


# ---------------------------------------------------------------------------------------------
# Definitions on tiny inputs: corners, brute force, ESPs
# ---------------------------------------------------------------------------------------------

CASES = [(O.OR, 0), (O.XOR, 0), (O.XOR, 1)] + [(O.ATLEAST, k) for k in range(0, 7)]


@pytest.mark.parametrize("ctype,param", CASES)
@pytest.mark.parametrize("L", [1, 2, 3, 5, 6])
def test_corners_equal_truth(ctype, param, L):
    """At every cube corner FE is -1 iff the constraint holds (Thm. "Walsh Transform")."""
    for bits in itertools.product([-1.0, 1.0], repeat=L):
        y = np.array(bits)
        ntrue = int((y < 0).sum())
        if ctype == O.OR:
            truth = ntrue >= 1
        elif ctype == O.XOR:
            truth = (ntrue % 2) == param
        else:
            truth = ntrue >= param
        for route in ("default", "dp", "bruteforce"):
            v, _ = O.fe(ctype, param, y, route)
            assert v == (-1.0 if truth else 1.0), (route, bits, v)


@pytest.mark.parametrize("ctype,param", CASES)
@pytest.mark.parametrize("L", [1, 4, 7, 9])
def test_routes_agree_small(ctype, param, L):
    rng = np.random.default_rng(L * 31 + ctype * 7 + param)
    for _ in range(4):
        y = rng.uniform(-1, 1, L)
        ref, dref = O.fe(ctype, param, y, "bruteforce")
        for route in ("corners", "esp", "paper", "dp", "default"):
            v, d = O.fe(ctype, param, y, route)
            assert abs(v - ref) < 1e-12, route
            assert np.allclose(d, dref, atol=1e-12), route


def test_esp_matches_subset_sums():
    rng = np.random.default_rng(5)
    for L in range(0, 9):
        y = rng.uniform(-1, 1, L)
        e = O.esp(y)
        for m in range(L + 1):
            want = sum(math.prod(y[list(S)]) for S in itertools.combinations(range(L), m))
            assert abs(e[m] - want) < 1e-13


def test_walsh_by_size_matches_theorem_sum():
    for L in range(1, 11):
        for ctype, param in [(O.OR, 0), (O.XOR, 1), (O.ATLEAST, (L + 1) // 2)]:
            a = O.walsh_by_size(ctype, param, L)
            for m in range(L + 1):
                mask = (1 << m) - 1
                assert a[m] == O.walsh_subset(ctype, param, L, mask)


# ---------------------------------------------------------------------------------------------
# Long constraints: exact rationals, closed-form distributions, finite differences
# ---------------------------------------------------------------------------------------------


def _exact_fe_esp(ctype, param, y_fr):
    """FE = sum_m a_m e_m (Eq. effi_eval) in exact rationals, a_m from the
    Krawtchouk grouping of the theorem's corner sum with exact integers."""
    L = len(y_fr)
    val = [O.value(ctype, param, L, s) for s in range(L + 1)]
    e = [Fraction(0)] * (L + 1)
    e[0] = Fraction(1)
    for yi in y_fr:
        for m in range(L, 0, -1):
            e[m] += yi * e[m - 1]
    fe = Fraction(0)
    for m in range(L + 1):
        tot = 0
        for s in range(L + 1):
            kr = sum((-1) ** t * math.comb(m, t) * math.comb(L - m, s - t) for t in range(0, min(m, s) + 1))
            tot += val[s] * kr
        fe += Fraction(tot, 2**L) * e[m]
    return fe


@pytest.mark.parametrize("L", [16, 40, 64])
def test_dp_matches_exact_rationals(L):
    rng = np.random.default_rng(L)
    k = rng.integers(-64, 65, size=L)
    y = k / 64.0
    y_fr = [Fraction(int(t), 64) for t in k]
    for ctype, param in [(O.ATLEAST, L // 2), (O.ATLEAST, L // 2 + L // 8), (O.OR, 0), (O.XOR, 1)]:
        exact = _exact_fe_esp(ctype, param, y_fr)
        v, _ = O.fe(ctype, param, y, "dp")
        assert abs(Fraction(v) - exact) < Fraction(1, 10**13), (ctype, param)


def _binom_tail(L, K, p_fr):
    q = 1 - p_fr
    return sum(math.comb(L, s) * p_fr**s * q ** (L - s) for s in range(K, L + 1))


@pytest.mark.parametrize("L,K", [(64, 32), (257, 140), (512, 256), (512, 300), (512, 200)])
@pytest.mark.parametrize("ynum", [0, 16, -40])
def test_dp_binomial_closed_form(L, K, ynum):
    """All literals equal: S ~ Binomial(L, p) with p = (1 - y)/2."""
    y_fr = Fraction(ynum, 64)
    p = (1 - y_fr) / 2
    fe_exact = 1 - 2 * _binom_tail(L, K, p)
    # dFE/dy_i = P(Binomial(L-1, p) = K-1)
    d_exact = math.comb(L - 1, K - 1) * p ** (K - 1) * (1 - p) ** (L - K)
    y = np.full(L, float(y_fr))
    v, d = O.fe(O.ATLEAST, K, y, "dp")
    assert abs(v - float(fe_exact)) < 1e-13
    assert np.allclose(d, float(d_exact), rtol=1e-11, atol=1e-300)


@pytest.mark.parametrize("L", [3, 50, 300, 512])
def test_dp_generic_equals_closed_forms(L):
    """The DP with the OR / XOR truth tables reproduces the closed forms."""
    rng = np.random.default_rng(L)
    y = rng.uniform(-1, 1, L)
    for ctype, param, cf in [(O.OR, 0, O.fe_or), (O.XOR, 1, lambda yy: O.fe_xor(1, yy)), (O.XOR, 0, lambda yy: O.fe_xor(0, yy))]:
        v1, d1 = O.fe(ctype, param, y, "dp")
        v2, d2 = cf(y)
        assert abs(v1 - v2) < 1e-13
        assert np.allclose(d1, d2, atol=1e-13)
    # at-least-1 is the clause
    v1, d1 = O.fe(O.ATLEAST, 1, y, "dp")
    v2, d2 = O.fe_or(y)
    assert abs(v1 - v2) < 1e-13 and np.allclose(d1, d2, atol=1e-13)


@pytest.mark.parametrize("L,K", [(8, 4), (64, 30), (200, 100), (512, 260)])
def test_gradient_is_exact_central_difference(L, K):
    """FE is multilinear, so (FE(y_i=+1) - FE(y_i=-1))/2 equals dFE/dy_i exactly."""
    rng = np.random.default_rng(L + K)
    y = rng.uniform(-1, 1, L)
    _, d = O.fe(O.ATLEAST, K, y, "dp")
    for i in rng.choice(L, size=min(L, 12), replace=False):
        yp, ym = y.copy(), y.copy()
        yp[i], ym[i] = 1.0, -1.0
        fd = (O.fe(O.ATLEAST, K, yp, "dp")[0] - O.fe(O.ATLEAST, K, ym, "dp")[0]) / 2
        assert abs(fd - d[i]) < 1e-13
        assert d[i] >= -1e-15  # dFE/dy_i = P_{-i}(S = K-1) >= 0 for at-least-K


@pytest.mark.parametrize("L", [40, 128, 512])
def test_value_in_range_and_monotone(L):
    rng = np.random.default_rng(L)
    for _ in range(5):
        y = rng.uniform(-1, 1, L)
        K = int(rng.integers(1, L + 1))
        v, d = O.fe(O.ATLEAST, K, y, "dp")
        assert -1.0 - 1e-15 <= v <= 1.0 + 1e-15
        assert (d >= -1e-15).all()
        vo, do = O.fe_or(y)
        assert -1 <= vo <= 1 and (do >= 0).all()


def test_degenerate_cardinality():
    y = np.random.default_rng(0).uniform(-1, 1, 20)
    v, d = O.fe(O.ATLEAST, 0, y, "dp")  # always satisfied
    assert v == -1.0 and np.all(d == 0)
    v, d = O.fe(O.ATLEAST, 21, y, "dp")  # never satisfied
    assert v == 1.0 and np.all(d == 0)


def test_paper_form_loses_precision_with_length():
    """The paper's literal form cancels for long constraints (Conclusion's precision remark)."""
    rng = np.random.default_rng(1)
    errs = {}
    for L in (8, 24, 48):
        y = rng.uniform(-1, 1, L)
        ref, _ = O.fe(O.ATLEAST, L // 2, y, "dp")
        v, _ = O.fe(O.ATLEAST, L // 2, y, "paper")
        errs[L] = abs(v - ref)
    assert errs[8] < 1e-13
    assert errs[48] > errs[8]


# ---------------------------------------------------------------------------------------------
# Instance level: certificate, checker twin, restart draws, one CLS round
# ---------------------------------------------------------------------------------------------


def _truth(ctype, param, lits, assign):
    vals = [(assign[abs(l) - 1] * (1 if l > 0 else -1)) < 0 for l in lits]
    if ctype == O.OR:
        return any(vals)
    if ctype == O.XOR:
        acc = False
        for t in vals:
            acc ^= t
        return acc == bool(param & 1)
    return sum(vals) >= param


def test_checker_twin_and_certificate():
    inst = gen.concat([gen.random_ksat(30, 100, 3, 1), gen.random_xor(30, 10, 2, 6, 1, signs=True),
                       gen.random_atleast(30, 5, 4, 12, 1)])
    x = gen.corner_points(64, 30, 3, dtype=np.float64)
    sat, nun = O.check(inst, x)
    f, _ = O.eval_grad(inst, x)
    for b in range(x.shape[0]):
        z = np.where(x[b] < 0, -1.0, 1.0)
        want = sum(not _truth(*inst.constraint(c), z) for c in range(inst.m))
        assert nun[b] == want and sat[b] == (want == 0)
        # at corners F(sgn x) = #violated - #satisfied (Thm. "SAT Certificate")
        fz, _ = O.eval_grad(inst, z[None])
        assert fz[0] == 2 * want - inst.m
    # F >= -sum w everywhere in the cube
    xs = gen.uniform_points(32, 30, 4, dtype=np.float64)
    fs, _ = O.eval_grad(inst, xs)
    assert (fs >= -inst.m - 1e-9).all()


def test_planted_instances_are_satisfied():
    for make in (gen.uniform_3sat_100, gen.cnf_xor_2000):
        inst = make(3, planted=True)
        sat, nun = O.check(inst, inst.planted[None].astype(np.float64))
        assert sat[0] == 1 and nun[0] == 0
        f, _ = O.eval_grad(inst, inst.planted[None].astype(np.float64))
        assert f[0] == -inst.weights.sum()


def test_signed_zero_is_false():
    inst = gen.from_lists(1, [(gen.OR, 0, [1])])
    sat, _ = O.check(inst, np.array([[0.0], [-0.0], [-1e-300], [1.0]]))
    assert list(sat) == [0, 0, 1, 0]
    with pytest.raises(ValueError):
        O.check(inst, np.array([[np.nan]]))


def test_splitmix64_published_first_output():
    # splitmix64 started at state 0 returns 0xE220A8397B1DCDAF first (Steele et al. 2014 / Vigna)
    assert O.splitmix64(0) == 0xE220A8397B1DCDAF


def test_uniform_draws():
    vals = np.array([O.uniform(7, 2, b, v) for b in range(20) for v in range(500)])
    assert vals.min() >= -1.0 and vals.max() < 1.0
    assert np.all(vals * 2**23 == np.round(vals * 2**23))
    assert abs(vals.mean()) < 0.02 and abs(vals.var() - 1 / 3) < 0.02
    assert O.uniform(7, 2, 3, 4) != O.uniform(7, 3, 3, 4)


def test_step_is_pgd_then_check_then_restart():
    inst = gen.uniform_3sat_100(0)
    x0 = gen.uniform_points(6, inst.n, 1, dtype=np.float64)
    f, g = O.eval_grad(inst, x0)
    x1, solved, nun = O.step(inst, x0, T=1, lr=0.1, seed=5, epoch=0, restart=False)
    assert np.array_equal(x1, np.clip(x0 - 0.1 * g, -1, 1))
    s2, n2 = O.check(inst, x1)
    assert np.array_equal(s2, solved) and np.array_equal(n2, nun)
    x2, solved2, _ = O.step(inst, x0, T=1, lr=0.1, seed=5, epoch=3, b_offset=10, restart=True)
    for b in range(6):
        if not solved2[b]:
            want = [O.uniform(5, 3, 10 + b, v) for v in range(inst.n)]
            assert np.array_equal(x2[b], want)
        else:
            assert np.array_equal(x2[b], x1[b])


# ---------------------------------------------------------------------------------------------
# Projected-gradient fixed point with FISTA line search (App. A.3)
# ---------------------------------------------------------------------------------------------

def _unit_clauses(signs, weights):
    n = len(signs)
    return gen.from_lists(n, [(gen.OR, 0, [int(s) * (v + 1)]) for v, s in enumerate(signs)], weights)


def test_pgfp_linear_objective_reaches_the_vertex_without_backtracking():
    """Unit clauses make F = sum_v w_v s_v x_v affine: the sufficient-decrease
    test holds for every step size (so the step never shrinks) and projected
    gradient steps end at the minimising vertex x_v = -s_v exactly."""
    rng = np.random.default_rng(1)
    signs = rng.choice([-1, 1], size=7)
    w = rng.uniform(0.5, 2.0, size=7)
    inst = _unit_clauses(signs, w)
    x0 = rng.uniform(-0.9, 0.9, size=(3, 7))
    x, ok, nun, its, eta = O.step_pgfp(inst, x0, T=60, eta0=0.05, restart=False)
    assert np.array_equal(x, -np.broadcast_to(signs, x.shape).astype(float))
    assert ok.all() and not nun.any()
    assert np.all(eta == 0.05) and np.all(its == 60)


def test_pgfp_momentum_follows_the_fista_sequence():
    """One variable, affine F = w x, no clipping over three iterations:
    x1 = x0 - h, x2 = x1 - h (t1 = 1 gives no momentum), and
    x3 = x2 + m2 (x2 - x1) - h with m2 = (t2 - 1)/t3, t2 = golden ratio,
    t3 = (1 + sqrt(1 + 4 t2^2))/2 = 2.19352...  (h = eta w)."""
    inst = _unit_clauses([1], [1.0])
    h = 0.01
    x, _, _, _, _ = O.step_pgfp(inst, np.array([[0.5]]), T=3, eta0=h, restart=False)
    phi = (1 + 5 ** 0.5) / 2
    t3 = 2.193527085331054
    assert abs(x[0, 0] - (0.5 - 3 * h - (phi - 1) / t3 * h)) < 1e-15


def test_pgfp_line_search_takes_the_first_acceptable_step():
    """From a large initial step, one iteration returns eta = eta0 beta^i for the
    smallest i at which p = clip(x0 - eta g) satisfies
    F(p) <= F(x0) + <g, p - x0> + |p - x0|^2 / (2 eta); the previous step of the
    sequence violates it (checked with independent evaluations of F)."""
    inst = gen.concat([gen.random_ksat(30, 120, 3, 4), gen.random_xor(30, 8, 3, 6, 4)])
    x0 = gen.uniform_points(5, 30, 8, dtype=np.float64)
    eta0, beta = 8.0, 0.5
    x1, _, _, its, eta = O.step_pgfp(inst, x0, T=1, eta0=eta0, beta=beta, maxls=30, restart=False)
    f0, g0 = O.eval_grad(inst, x0)

    def ok(b, e):
        p = np.clip(x0[b] - e * g0[b], -1, 1)
        fp, _ = O.eval_grad(inst, p[None])
        return fp[0] <= f0[b] + g0[b] @ (p - x0[b]) + (p - x0[b]) @ (p - x0[b]) / (2 * e), p

    shrunk = 0
    for b in range(5):
        i = round(np.log(eta[b] / eta0) / np.log(beta))
        assert abs(eta[b] - eta0 * beta ** i) < 1e-12 * eta0
        good, p = ok(b, eta[b])
        assert good and np.array_equal(p, x1[b])
        if i > 0:
            shrunk += 1
            assert not ok(b, eta[b] / beta)[0]
    assert shrunk >= 1 and np.all(its == 1)


def test_pgfp_stops_below_the_minimum_step():
    inst = gen.random_ksat(20, 80, 3, 2)
    x0 = gen.uniform_points(2, 20, 3, dtype=np.float64)
    _, _, _, its, eta = O.step_pgfp(inst, x0, T=50, eta0=1e-13, restart=False)
    assert np.all(its == 1) and np.all(eta <= 1e-13)
    with pytest.raises(ValueError):
        O.step_pgfp(inst, x0, T=5, eta0=0.1, beta=1.5)


# ---------------------------------------------------------------------------------------------
# The tolerance scales every parity test divides by
# ---------------------------------------------------------------------------------------------


def _fe_corner_expectation(ctype, param, y):
    """FE at y as the expectation of the truth value v(#True) over independent
    literals that are True (-1) with probability (1 - y_i) / 2: the sum over all
    2^L corners (Thm. "Walsh Transform" read as an expectation)."""
    L = len(y)
    tot = 0.0
    for z in itertools.product((-1.0, 1.0), repeat=L):
        s = sum(1 for zi in z if zi < 0)
        sat = s >= 1 if ctype == O.OR else ((s % 2) == (param % 2) if ctype == O.XOR else s >= param)
        p = 1.0
        for yi, zi in zip(y, z):
            p *= (1.0 + yi * zi) / 2.0
        tot += (-1.0 if sat else 1.0) * p
    return tot


@pytest.mark.parametrize("floor", [0.0, 1e-2, 0.3])
def test_eval_scale_against_direct_restatement(floor):
    """orc_eval_scale: sf_b = sum_c w_c |FE_c|, A[b, v] = sum_{c containing v}
    w_c max(|dFE_c/dy_v|, floor for at-least-K constraints), restated from
    corner sums (FE) and exact central differences (the derivative of a
    multilinear polynomial along one coordinate is half its difference between
    y_v = +1 and y_v = -1).  A dropped weight, a lost absolute value, a floor on
    the wrong type or a gradient credited to the wrong variable fails here."""
    n = 7
    cons = [(O.OR, 0, [1, -2, 3]), (O.XOR, 1, [2, 4, -5, 6]), (O.ATLEAST, 2, [1, 3, -4, 5, 7]),
            (O.ATLEAST, 0, [2, 6]), (O.XOR, 0, [-7]), (O.ATLEAST, 5, [1, -2, 3])]
    w = np.array([0.5, 1.5, 2.0, 0.75, 1.25, 3.0])
    inst = gen.from_lists(n, cons, w)
    x = np.random.default_rng(5).uniform(-1, 1, (3, n))
    sf, A = O.eval_scale(inst, x, floor)
    for b in range(3):
        sf_want = 0.0
        A_want = np.zeros(n)
        for (ctype, param, lits), wc in zip(cons, w):
            sg = np.sign(lits)
            vs = np.abs(lits) - 1
            y = sg * x[b, vs]
            sf_want += wc * abs(_fe_corner_expectation(ctype, param, y))
            for i in range(len(lits)):
                hi, lo = y.copy(), y.copy()
                hi[i], lo[i] = 1.0, -1.0
                d = 0.5 * (_fe_corner_expectation(ctype, param, hi) - _fe_corner_expectation(ctype, param, lo))
                A_want[vs[i]] += wc * max(abs(d), floor if ctype == O.ATLEAST else 0.0)
        assert sf[b] == pytest.approx(sf_want, rel=1e-12, abs=1e-15)
        assert np.allclose(A[b], A_want, rtol=1e-12, atol=1e-15)

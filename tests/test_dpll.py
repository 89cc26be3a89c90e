"""The DPLL that selects satisfiable random 3-SAT seeds, against exhaustive
search on small formulas (the selection decides which instances the
time-to-SAT measurement uses)."""
import itertools

import numpy as np

from paper_2308_15020_gb300 import gen


def _brute(inst):
    n = inst.n
    cls = [inst.lits[inst.row_ptr[c]:inst.row_ptr[c + 1]] for c in range(inst.m)]
    for bits in itertools.product([1, -1], repeat=n):  # -1 True
        if all(any((bits[abs(l) - 1] < 0) == (l > 0) for l in cl) for cl in cls):
            return True
    return False


def _is_model(inst, z):
    cls = [inst.lits[inst.row_ptr[c]:inst.row_ptr[c + 1]] for c in range(inst.m)]
    return all(any((z[abs(l) - 1] < 0) == (l > 0) for l in cl) for cl in cls)


def test_dpll_matches_exhaustive_search():
    seen = {True: 0, False: 0}
    for seed in range(40):
        inst = gen.random_ksat(10, 52, 3, seed)  # ratio 5.2: a mix of SAT and UNSAT
        z = gen.dpll_model(inst)
        truth = _brute(inst)
        assert (z is not None) == truth, seed
        if z is not None:
            assert _is_model(inst, z)
        seen[truth] += 1
    assert seen[True] > 3 and seen[False] > 3


def test_satisfiable_seeds_of_the_n100_workload():
    got = gen.satisfiable_3sat_100(3, 0)
    for s, inst in got:
        z = gen.dpll_model(inst)
        assert z is not None and _is_model(inst, z)
    assert np.all(np.diff([s for s, _ in got]) > 0)

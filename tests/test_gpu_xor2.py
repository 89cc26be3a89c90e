"""XOR constraints of at most two literals on the thread-per-constraint record
path (Max-Cut as weighted 2-XOR, Benchmark 3) against the oracle: F and its
gradient in FP32 and FP64, a fused step, and the ERWA update of their weights."""
import numpy as np
import pytest

import oracle as O
from paper_2308_15020_gb300 import gen
from parity import compare, to_np

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _instance():
    # a planted-partition graph plus unit and two-literal XORs of both parities
    # (negated literals too) next to ordinary clauses
    g = gen.planted_maxcut(4, 8, 3)
    rng = np.random.default_rng(0)
    cons = []
    for _ in range(40):
        L = int(rng.integers(1, 3))
        vs = rng.choice(32, size=L, replace=False) + 1
        cons.append((gen.XOR, int(rng.integers(0, 2)), (vs * rng.choice([-1, 1], size=L)).tolist()))
    for _ in range(60):
        vs = rng.choice(32, size=3, replace=False) + 1
        cons.append((gen.OR, 0, (vs * rng.choice([-1, 1], size=3)).tolist()))
    extra = gen.from_lists(32, cons, rng.uniform(0.5, 2.0, size=len(cons)))
    return gen.concat([g, extra])


@pytest.mark.parametrize("dt,tol", [(torch.float32, 1e-4), (torch.float64, 1e-10)])
def test_eval_matches_oracle(dt, tol):
    from paper_2308_15020_gb300 import ffsat

    inst = _instance()
    h = ffsat.Instance(inst)
    assert h.info()["n_xor2"] > inst.m // 2
    for pts in (gen.uniform_points(7, inst.n, 2, dtype=np.float64), gen.corner_points(5, inst.n, 4, dtype=np.float64)):
        x = torch.from_numpy(pts).to(dt).cuda()
        f, g = h.eval_grad(x)
        ef, eg = compare(inst, x.double().cpu().numpy(), to_np(f), to_np(g).astype(np.float64), tol)
        assert ef <= 1 and eg <= 1, (ef, eg)


def test_step_and_erwa_match_oracle():
    from paper_2308_15020_gb300 import ffsat

    inst = _instance()
    h = ffsat.Instance(inst)
    x0 = gen.uniform_points(6, inst.n, 9, dtype=np.float64)
    x = torch.from_numpy(x0).cuda()
    U = torch.zeros(inst.m, dtype=torch.int32, device="cuda")
    solved, nun = h.step(x, T=20, lr=0.05, seed=2, epoch=1, restart=False, unsat_counts=U)
    xs, ok, nu = O.step(inst, x0, T=20, lr=0.05, seed=2, epoch=1, restart=False)
    assert np.allclose(to_np(x), xs, rtol=0, atol=1e-9)
    assert np.array_equal(to_np(nun), nu)
    assert np.array_equal(to_np(U), O.unsat_counts(inst, xs))
    h.erwa_update(U, 0.4)
    w = O.erwa(O.unsat_counts(inst, xs), inst.weights, 0.4)
    assert np.array_equal(h.get_weights(), w)
    f, g = h.eval_grad(torch.from_numpy(x0).cuda())
    ef, eg = compare(inst, x0, to_np(f), to_np(g), 1e-10, weights=w)
    assert ef <= 1 and eg <= 1

"""Projected gradient with FISTA line search (App. A.3, Alg. PGFP) on the device
against the oracle: FP64 trajectories, step sizes and iteration counts; FP32
line-search invariants; the affine special case; argument errors."""
import numpy as np
import pytest

import oracle as O
from paper_2308_15020_gb300 import gen
from parity import mixed_instance, to_np

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _cases():
    return [
        ("3sat_n100", gen.uniform_3sat_100(3)),
        ("cnf_xor_300", gen.cnf_xor_2000(5, n=300)),
        ("mixed_700", mixed_instance(41, n=700)),
    ]


@pytest.mark.parametrize("name,inst", _cases(), ids=lambda v: v if isinstance(v, str) else "")
def test_fp64_matches_oracle(name, inst):
    from paper_2308_15020_gb300 import ffsat

    h = ffsat.Instance(inst)
    B = 9
    x0 = gen.uniform_points(B, inst.n, 17, dtype=np.float64)
    for restart in (False, True):
        x = torch.from_numpy(x0).cuda()
        its = torch.zeros(B, dtype=torch.int32, device="cuda")
        eta = torch.zeros(B, dtype=torch.float64, device="cuda")
        solved, nun = h.step_pgfp(x, T=6, eta0=2.0, beta=0.5, maxls=20, seed=4, epoch=2, restart=restart,
                                  iters=its, eta_out=eta)
        xs, ok, nu, oits, oeta = O.step_pgfp(inst, x0, T=6, eta0=2.0, beta=0.5, maxls=20, seed=4, epoch=2,
                                             restart=restart)
        assert np.array_equal(to_np(its), oits)
        assert np.array_equal(to_np(eta), oeta)
        assert np.array_equal(to_np(solved), ok) and np.array_equal(to_np(nun), nu)
        assert np.allclose(to_np(x), xs, rtol=0, atol=1e-9), np.max(np.abs(to_np(x) - xs))
    assert (oeta < 2.0).any()  # the line search did backtrack somewhere


def test_fp32_accepted_steps_satisfy_sufficient_decrease():
    """One iteration in FP32: every point's accepted step eta = eta0 beta^i and the
    step it took satisfy the test (evaluated by the FP64 oracle, within the FP32
    slack and rounding)."""
    from paper_2308_15020_gb300 import ffsat

    inst = gen.cnf_xor_2000(6, n=500)
    h = ffsat.Instance(inst)
    B = 16
    x0 = gen.uniform_points(B, inst.n, 3)  # float32 values
    x = torch.from_numpy(x0).cuda()
    eta = torch.zeros(B, dtype=torch.float64, device="cuda")
    slack = 1e-6 * float(np.sum(inst.weights))
    h.step_pgfp(x, T=1, eta0=4.0, beta=0.5, maxls=25, slack=slack, restart=False, eta_out=eta)
    x0d = x0.astype(np.float64)
    f0, g0 = O.eval_grad(inst, x0d)
    p = to_np(x).astype(np.float64)
    fp, _ = O.eval_grad(inst, p)
    e = to_np(eta)
    i = np.round(np.log(e / 4.0) / np.log(0.5))
    assert np.allclose(e, 4.0 * 0.5 ** i, rtol=1e-12)
    dz = p - x0d
    rhs = f0 + np.sum(g0 * dz, axis=1) + np.sum(dz * dz, axis=1) / (2 * e) + slack
    tol = 1e-4 * np.sum(np.abs(inst.weights))  # FP32 evaluation of F at two points
    assert np.all(fp <= rhs + tol)
    # the point is the projected step from x0 along the FP32 gradient
    _, g32 = h.eval_grad(torch.from_numpy(x0).cuda())
    want = np.clip(x0d - e[:, None] * to_np(g32).astype(np.float64), -1, 1)
    assert np.allclose(p, want, atol=1e-5)


def test_affine_objective_reaches_the_vertex_in_fp32():
    from paper_2308_15020_gb300 import ffsat

    rng = np.random.default_rng(2)
    signs = rng.choice([-1, 1], size=40)
    inst = gen.from_lists(40, [(gen.OR, 0, [int(s) * (v + 1)]) for v, s in enumerate(signs)],
                          rng.uniform(0.5, 2.0, size=40))
    h = ffsat.Instance(inst)
    x = torch.from_numpy(gen.uniform_points(4, 40, 1) * 0.9).cuda()
    its = torch.zeros(4, dtype=torch.int32, device="cuda")
    solved, nun = h.step_pgfp(x, T=80, eta0=0.05, restart=False, iters=its)
    assert np.array_equal(to_np(x), -np.broadcast_to(signs, (4, 40)).astype(np.float32))
    assert to_np(solved).all() and (to_np(its) == 80).all()


def test_errors():
    from paper_2308_15020_gb300 import ffsat

    inst = gen.uniform_3sat_100(1)
    h = ffsat.Instance(inst)
    x = torch.zeros(2, 100, device="cuda")
    for kw in ({"eta0": 0.0}, {"eta0": 0.1, "beta": 1.0}, {"eta0": 0.1, "maxls": 0}):
        with pytest.raises(ffsat.FFSatError):
            h.step_pgfp(x, T=1, **kw)
    big = gen.random_ksat(70000, 2000, 3, 1)  # x does not fit in shared memory
    hb = ffsat.Instance(big)
    assert hb.info()["smem_mode_f32"] == 2
    with pytest.raises(ffsat.FFSatError):
        hb.step_pgfp(torch.zeros(1, 70000, device="cuda"), T=1, eta0=0.1)

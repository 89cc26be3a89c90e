"""Restart heuristics on the device against the oracle: unsatisfaction counts
(standalone and fused into the step's final check), the ERWA weight update
(Prop. "Adaptive weight") and every weight copy it must reach, rephasing."""
import numpy as np
import pytest

import oracle as O
from paper_2308_15020_gb300 import gen
from parity import compare, mixed_instance, to_np

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _instances():
    return [
        ("mixed", mixed_instance(31, n=700)),                      # every path, constant constraints, resident image
        ("cnf_xor", gen.cnf_xor_2000(4)),                           # clause + product paths
        ("large", gen.concat([gen.random_ksat(20000, 60000, 3, 6),  # x and g outside shared memory
                              gen.random_atleast(20000, 30, 64, 512, 6)])),
    ]


@pytest.mark.parametrize("name,inst", _instances(), ids=lambda v: v if isinstance(v, str) else "")
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_unsat_counts_bit_exact(name, inst, dtype):
    from paper_2308_15020_gb300 import ffsat

    h = ffsat.Instance(inst)
    x_np = gen.corner_points(19, inst.n, 5, dtype=dtype)  # exact zeros included: sgn(0) = +1
    U = h.unsat_counts(torch.from_numpy(x_np).cuda())
    assert np.array_equal(to_np(U), O.unsat_counts(inst, x_np.astype(np.float64)))
    # empty batch gives zeros
    assert not to_np(h.unsat_counts(torch.zeros(0, inst.n, dtype=torch.from_numpy(x_np).dtype, device="cuda"))).any()


@pytest.mark.parametrize("name,inst", _instances()[:2], ids=lambda v: v if isinstance(v, str) else "")
def test_step_accumulates_unsat_counts(name, inst):
    """The counts of the step's final check are those of the points it ends at
    (restart off) and of the points before their restart (restart on)."""
    from paper_2308_15020_gb300 import ffsat

    h = ffsat.Instance(inst)
    x0 = torch.from_numpy(gen.uniform_points(40, inst.n, 8)).cuda()
    x = x0.clone()
    U = torch.zeros(inst.m, dtype=torch.int32, device="cuda")
    _, nun = h.step(x, T=3, lr=0.05, seed=2, epoch=1, restart=False, unsat_counts=U)
    assert np.array_equal(to_np(U), O.unsat_counts(inst, to_np(x).astype(np.float64)))
    assert int(U.sum()) == int(nun.sum())
    # with restart the counts still describe the pre-restart points: compare with a
    # restart-free step from the same start
    x1 = x0.clone()
    U1 = torch.zeros_like(U)
    h.step(x1, T=3, lr=0.05, seed=2, epoch=1, restart=True, unsat_counts=U1)
    assert torch.equal(U1, U)
    # counts add up across calls (the caller zeroes)
    x2 = x0.clone()
    h.step_noalloc(x2, T=3, lr=0.05, seed=2, epoch=1, restart=False, unsat_counts=U1)
    assert torch.equal(U1, 2 * U)


@pytest.mark.parametrize("autotune", [False, True])
def test_erwa_matches_oracle_and_reaches_every_weight_copy(autotune):
    """Three ERWA rounds: the device weights equal the oracle's bit for bit, and
    F, grad F (FP32 and FP64 fused kernels, plain FP64 comparator) and the step
    then follow the new weights."""
    from paper_2308_15020_gb300 import ffsat

    inst = mixed_instance(32, n=700)
    h = ffsat.Instance(inst, autotune=autotune)
    w = np.asarray(inst.weights, dtype=np.float64).copy()
    for r in range(3):
        xr = gen.uniform_points(64, inst.n, 40 + r, dtype=np.float64)
        U = h.unsat_counts(torch.from_numpy(xr).cuda())
        h.erwa_update(U, 0.4)
        w = O.erwa(O.unsat_counts(inst, xr), w, 0.4)
        assert np.array_equal(h.get_weights(), w), r
    x_np = gen.uniform_points(9, inst.n, 50, dtype=np.float64)
    for dt, tol in ((torch.float32, 1e-4), (torch.float64, 1e-10)):
        x = torch.from_numpy(x_np).to(dt).cuda()
        f, g = h.eval_grad(x)
        ef, eg = compare(inst, x.double().cpu().numpy(), to_np(f), to_np(g).astype(np.float64), tol, weights=w)
        assert ef <= 1 and eg <= 1, (dt, ef, eg)
    f, g = h.eval_grad_plain64(torch.from_numpy(x_np).cuda())
    ef, eg = compare(inst, x_np, to_np(f), to_np(g), 1e-10, weights=w)
    assert ef <= 1 and eg <= 1, (ef, eg)
    # one FP64 step follows the oracle's step under the same weights
    x = torch.from_numpy(x_np).cuda()
    solved, nun = h.step(x, T=2, lr=0.02, seed=3, epoch=1, restart=False)
    xs, ok, nu = O.step(inst, x_np, T=2, lr=0.02, seed=3, epoch=1, restart=False, weights=w)
    assert np.allclose(to_np(x), xs, rtol=0, atol=1e-9)
    # set_weights overwrites the device weights again
    h.set_weights(inst.weights)
    assert np.array_equal(h.get_weights(), np.asarray(inst.weights, dtype=np.float64))
    f2, _ = h.eval_grad(torch.from_numpy(x_np).cuda())
    ef, _ = compare(inst, x_np, to_np(f2), None, 1e-10)
    assert ef <= 1


def test_erwa_edge_cases():
    from paper_2308_15020_gb300 import ffsat

    inst = gen.from_lists(5, [(gen.OR, 0, [1, -2]), (gen.XOR, 1, [2, 3, 4]), (gen.ATLEAST, 0, [1, 5]),
                              (gen.ATLEAST, 3, [1, 2]), (gen.ATLEAST, 2, [1, 3, 5])], [1.0, 2.0, 0.5, 1.5, 3.0])
    h = ffsat.Instance(inst)
    zeros = torch.zeros(inst.m, dtype=torch.int32, device="cuda")
    h.erwa_update(zeros, 0.4)  # nothing violated: pure decay
    assert np.array_equal(h.get_weights(), O.erwa(np.zeros(inst.m, np.int32), inst.weights, 0.4))
    neg = torch.tensor([-3, 2, 0, 4, 1], dtype=torch.int32, device="cuda")  # negative counts read as 0
    h.erwa_update(neg, 1.0)
    assert np.array_equal(h.get_weights(), np.array([0.0, 0.5, 0.0, 1.0, 0.25]))
    # the constant constraints (K = 0 and K > L) still enter f with their new weights
    x_np = gen.uniform_points(4, inst.n, 3, dtype=np.float64)
    f, _ = h.eval_grad(torch.from_numpy(x_np).cuda())
    ef, _ = compare(inst, x_np, to_np(f), None, 1e-10, weights=h.get_weights())
    assert ef <= 1
    with pytest.raises(ffsat.FFSatError):
        h.erwa_update(zeros, 1.5)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_rephase_matches_oracle(dtype):
    from paper_2308_15020_gb300 import ffsat

    inst = gen.cnf_xor_2000(5)
    h = ffsat.Instance(inst)
    x_np = gen.uniform_points(33, inst.n, 6, dtype=np.float64)
    solved = (np.arange(33) % 4 == 1).astype(np.uint8)
    for phase in (0, 1, 2):
        x = torch.from_numpy(x_np).to(dtype).cuda()
        h.rephase(x, phase, solved=torch.from_numpy(solved).cuda(), seed=11, epoch=4, b_offset=7)
        ref = O.rephase(x_np.astype(np.float32).astype(np.float64) if dtype == torch.float32 else x_np, phase,
                        solved, seed=11, epoch=4, b_offset=7)
        assert np.array_equal(to_np(x).astype(np.float64), ref), phase
    with pytest.raises(ffsat.FFSatError):
        h.rephase(torch.zeros(2, inst.n, device="cuda"), 3)


def test_heuristic_round_in_cuda_graph():
    """Two rounds of step with counts -> ERWA -> rephase (flipped, then random),
    captured once and replayed, equal the same calls issued eagerly."""
    from paper_2308_15020_gb300 import ffsat

    inst = gen.cnf_xor_2000(6)
    x_np = gen.uniform_points(64, inst.n, 9)
    runs = []
    for graph in (False, True):
        h = ffsat.Instance(inst)
        x = torch.from_numpy(x_np).cuda()
        U = torch.zeros(inst.m, dtype=torch.int32, device="cuda")
        solved = torch.zeros(64, dtype=torch.uint8, device="cuda")
        nun = torch.zeros(64, dtype=torch.int32, device="cuda")

        def rounds():
            for e in (1, 2):
                U.zero_()
                h.step(x, T=5, lr=0.05, seed=1, epoch=e, restart=False, solved=solved, n_unsat=nun, unsat_counts=U)
                h.erwa_update(U, 0.4)
                h.rephase(x, e, solved=solved, seed=1, epoch=100 + e)

        if graph:
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                rounds()  # warm-up outside the capture
            torch.cuda.current_stream().wait_stream(s)
            torch.cuda.synchronize()
            h.set_weights(inst.weights)
            x.copy_(torch.from_numpy(x_np).cuda())
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                rounds()
            for _ in range(2):
                g.replay()
        else:
            for _ in range(2):
                rounds()
        torch.cuda.synchronize()
        runs.append((to_np(x), h.get_weights(), to_np(nun)))
    assert np.array_equal(runs[0][0], runs[1][0])
    assert np.array_equal(runs[0][1], runs[1][1])
    assert np.array_equal(runs[0][2], runs[1][2])

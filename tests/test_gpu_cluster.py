"""FP64 fixed-step calls with one thread-block cluster per point against the
one-CTA kernel and the FP64 oracle: the same trajectories (up to the order in
which the one-CTA kernel's FP64 atomics add), bit-exact checks, violation
counts and restart draws, in every shared-memory layout the cluster kernel
serves, and bit-reproducible repeats."""
import numpy as np
import pytest

import oracle as O
from paper_2308_15020_gb300 import gen
from parity import mixed_instance, to_np

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _run(inst, x_np, cluster, **kw):
    from paper_2308_15020_gb300 import ffsat

    h = ffsat.Instance(inst, cluster=cluster)
    x = torch.from_numpy(np.ascontiguousarray(x_np)).cuda()
    U = torch.zeros(inst.m, dtype=torch.int32, device="cuda")
    solved, nun = h.step(x, unsat_counts=U, **kw)
    cl = ffsat.last_cluster_size()
    torch.cuda.synchronize()
    return to_np(x), to_np(solved), to_np(nun), to_np(U), cl, h


def _instances():
    # (name, instance, iterations per call, FP64 shared-memory layout: 3 = the
    # resident image beside x and the gradient, 0 = x and the gradient only)
    return [
        ("3sat_n100", gen.uniform_3sat_100(3), 40, 3),            # clause path only
        ("card_n100", gen.bench1_cardinality(100, 7), 40, 3),     # node path (20-literal at-least-10)
        ("mixed", mixed_instance(33, n=700), 12, 3),              # every path, constants, long constraints
        ("cnf_xor", gen.cnf_xor_2000(2), 40, 3),                  # clause and product paths, resident image
        ("3sat_n5000", gen.random_ksat(5000, 21000, 3, 4), 10, 0),  # image too large: x and g only
    ]


@pytest.mark.parametrize("name,inst,T,mode", _instances(), ids=lambda v: v if isinstance(v, str) else "")
@pytest.mark.parametrize("B", [1, 7, 32])
def test_cluster_step_matches_one_cta_and_oracle(name, inst, T, mode, B):
    x0 = gen.uniform_points(B, inst.n, 11 + B, dtype=np.float64)
    xa, sa, na, Ua, cla, h = _run(inst, x0, 0, T=T, lr=0.05, seed=5, epoch=2, restart=False)
    assert h.info()["smem_mode_f64"] == mode  # both layouts of the cluster kernel are covered
    xb, sb, nb, Ub, clb, _ = _run(inst, x0, 1, T=T, lr=0.05, seed=5, epoch=2, restart=False)
    assert clb == 1
    assert cla > 1, "the automatic choice kept one CTA per point"
    xo, so, no = O.step(inst, x0, T=T, lr=0.05, seed=5, epoch=2, restart=False)
    assert np.max(np.abs(xa - xo)) < 1e-9
    assert np.max(np.abs(xa - xb)) < 1e-9
    assert np.array_equal(sa, so) and np.array_equal(na, no)
    assert np.array_equal(Ua, O.unsat_counts(inst, xo)) and np.array_equal(Ua, Ub)


@pytest.mark.parametrize("cluster", [2, 4, 8])
def test_forced_cluster_sizes(cluster):
    inst = mixed_instance(34, n=700)
    x0 = gen.uniform_points(3, inst.n, 4, dtype=np.float64)
    xa, sa, na, Ua, cl, _ = _run(inst, x0, cluster, T=12, lr=0.05, seed=1, epoch=1, restart=False)
    assert cl == cluster
    xo, so, no = O.step(inst, x0, T=12, lr=0.05, seed=1, epoch=1, restart=False)
    assert np.max(np.abs(xa - xo)) < 1e-9
    assert np.array_equal(na, no)


def test_cluster_restart_draws_and_solved_points():
    """Restarts in the cluster kernel are the oracle's draws bit for bit; a solved
    point keeps its x; T = 0 is the check alone."""
    inst = gen.uniform_3sat_100(5, planted=True)
    B = 6
    x0 = gen.uniform_points(B, inst.n, 21, dtype=np.float64)
    x0[2] = np.where(inst.planted < 0, -0.5, 0.5)  # a model: stays solved
    xa, sa, na, _, cl, _ = _run(inst, x0, 0, T=0, lr=0.05, seed=9, epoch=4, restart=True, b_offset=17)
    assert cl > 1
    xo, so, no = O.step(inst, x0, T=0, lr=0.05, seed=9, epoch=4, restart=True, b_offset=17)
    assert np.array_equal(xa, xo) and np.array_equal(sa, so) and np.array_equal(na, no)
    assert sa[2] == 1 and np.array_equal(xa[2], x0[2])
    xa, sa, na, _, _, _ = _run(inst, x0, 0, T=15, lr=0.05, seed=9, epoch=4, restart=True, b_offset=17)
    xo, so, no = O.step(inst, x0, T=15, lr=0.05, seed=9, epoch=4, restart=True, b_offset=17)
    assert np.array_equal(sa, so) and np.array_equal(na, no)
    restarted = so == 0
    assert np.array_equal(xa[restarted], xo[restarted])  # the draws themselves
    assert np.max(np.abs(xa[~restarted] - xo[~restarted])) < 1e-9


def test_cluster_step_in_cuda_graph():
    """Captured cluster launches replay to the eager result."""
    from paper_2308_15020_gb300 import ffsat

    inst = gen.uniform_3sat_100(4)
    x0 = torch.from_numpy(gen.uniform_points(32, inst.n, 3, dtype=np.float64)).cuda()
    h = ffsat.Instance(inst)
    xe = x0.clone()
    for e in (1, 2, 3):
        h.step(xe, T=20, lr=0.1, seed=2, epoch=e)
    assert ffsat.last_cluster_size() > 1
    xg = x0.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        h.step(xg.clone(), T=20, lr=0.1, seed=2, epoch=1)  # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graphs = []
    for e in (1, 2, 3):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            h.step(xg, T=20, lr=0.1, seed=2, epoch=e)
        graphs.append(g)
    xg.copy_(x0)
    for g in graphs:
        g.replay()
    torch.cuda.synchronize()
    # fixed-point sums: the replay repeats the eager bits
    assert torch.equal(xg, xe)


@pytest.mark.parametrize("name", ["3sat_n100", "card_n100", "cnf_xor", "3sat_n5000"])
def test_cluster_step_bit_reproducible(name):
    """The cluster step accumulates clause and node contributions in fixed
    point, whose sums do not depend on the order of the atomics: without
    product constraints repeated calls give the same bits (CNF-XOR's XOR
    products add with FP64 atomics), and the result stays within 1e-9 of the
    FP64 oracle."""
    from paper_2308_15020_gb300 import ffsat

    inst = {
        "3sat_n100": lambda: gen.uniform_3sat_100(8),
        "card_n100": lambda: gen.bench1_cardinality(100, 9),
        "cnf_xor": lambda: gen.cnf_xor_2000(4),
        "3sat_n5000": lambda: gen.random_ksat(5000, 21000, 3, 5),
    }[name]()
    T = 10 if name == "3sat_n5000" else 60
    x0 = gen.uniform_points(32, inst.n, 6, dtype=np.float64)
    h = ffsat.Instance(inst)
    outs = []
    for _ in range(3):
        x = torch.from_numpy(x0.copy()).cuda()
        h.step(x, T=T, lr=0.05, seed=3, epoch=1, restart=False)
        assert ffsat.last_cluster_size() > 1
        outs.append(to_np(x))
    for o in outs[1:]:
        if name == "cnf_xor":
            assert np.max(np.abs(o - outs[0])) < 1e-12
        else:
            assert np.array_equal(o.view(np.uint64), outs[0].view(np.uint64))
    xo, _, _ = O.step(inst, x0, T=T, lr=0.05, seed=3, epoch=1, restart=False)
    assert np.max(np.abs(outs[0] - xo)) < 1e-9

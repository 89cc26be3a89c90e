"""The FP32 shared-memory-resident gradient in one or two fixed-point words:
the library picks one word where the weights and degrees allow it, two where a
variable's weighted degree is large, and both variants match the FP64 oracle
(evaluation and a multi-iteration step)."""
import numpy as np
import pytest

import oracle as O
from paper_2308_15020_gb300 import gen
from parity import compare, to_np

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _hub(n=300, m=5000, seed=3):
    """Random 3-clauses that all contain variable 1 (weighted degree 5000)."""
    rng = np.random.default_rng(seed)
    cons = []
    for _ in range(m):
        others = rng.choice(np.arange(2, n + 1), size=2, replace=False)
        sg = np.where(rng.random(3) < 0.5, -1, 1)
        cons.append((0, 0, [int(sg[0]), int(sg[1] * others[0]), int(sg[2] * others[1])]))
    return gen.from_lists(n, cons, name="hub")


@pytest.mark.parametrize("name,make,words", [
    ("cnf_xor", lambda: gen.cnf_xor_2000(7), 1),
    ("3sat_n100", lambda: gen.uniform_3sat_100(7), 1),
    ("hub_degree_5000", _hub, 2),
])
def test_word_choice_and_parity(name, make, words):
    from paper_2308_15020_gb300 import ffsat

    inst = make()
    h = ffsat.Instance(inst)
    info = h.info()
    assert info["smem_mode_f32"] == 3 and info["fix_words_f32"] == words
    B = 16
    x = gen.uniform_points(B, inst.n, 5)
    f, g = h.eval_grad(torch.from_numpy(x).cuda())
    ef, eg = compare(inst, x, to_np(f), to_np(g), 1e-4)
    assert ef <= 1 and eg <= 1, (ef, eg)
    # ten fixed-step iterations from the same points: within 1e-4 of the FP64 trajectory
    xs = torch.from_numpy(x.copy()).cuda()
    h.step(xs, T=10, lr=0.05, seed=1, epoch=1, restart=False)
    xo, _, _ = O.step(inst, x.astype(np.float64), T=10, lr=0.05, seed=1, epoch=1, restart=False)
    assert np.max(np.abs(to_np(xs) - xo)) < 1e-4


@pytest.mark.parametrize("scale,words", [(1.0, 1), (300.0, 1), ("mixed", 2)])
def test_weights_switch_word_count(scale, words):
    """ffsat_set_weights re-derives the scales: uniform weights of any size keep
    one word; weights spanning 1..300 need the second (a unit-weight clause's
    contribution would be rounded to 2^-12), and either way the gradient
    matches the oracle."""
    from paper_2308_15020_gb300 import ffsat

    inst = gen.uniform_3sat_100(9)
    h = ffsat.Instance(inst)
    assert h.info()["fix_words_f32"] == 1
    if scale == "mixed":
        w = np.ones(inst.m)
        w[::7] = 300.0
    else:
        w = np.full(inst.m, scale)
    h.set_weights(w)
    assert h.info()["fix_words_f32"] == words
    x = gen.uniform_points(8, inst.n, 2)
    f, g = h.eval_grad(torch.from_numpy(x).cuda())
    ef, eg = compare(inst, x, to_np(f), to_np(g), 1e-4, weights=w)
    assert ef <= 1 and eg <= 1, (ef, eg)
    # a step with more points than SMs pairs them only with one fixed-point word
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    xs = torch.from_numpy(gen.uniform_points(sms + 9, inst.n, 3)).cuda()
    h.step(xs, T=2, lr=0.05, seed=1, epoch=1, restart=False)
    assert ffsat.last_points_per_cta() == (2 if words == 1 else 1)


@pytest.mark.parametrize("name,B", [("3sat_n2000", 305), ("3sat_n2000", 400), ("cnf_xor", 305)])
def test_two_points_per_cta_equal_one_point_per_cta(name, B):
    """Enough points for two per CTA: the paired launch (an odd B leaves the last
    point alone) gives the one-point-per-CTA results (points, flags, violation
    counts, restarts), the latter run in chunks of at most one wave: bit for bit
    where every contribution is fixed point (clauses), and to FP32 rounding
    where XOR products add with FP32 atomics in either order."""
    from paper_2308_15020_gb300 import ffsat

    inst = gen.random_ksat(2000, 8400, 3, 12) if name == "3sat_n2000" else gen.cnf_xor_2000(12)
    h = ffsat.Instance(inst)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    x0 = gen.uniform_points(B, inst.n, 8)
    xa = torch.from_numpy(x0.copy()).cuda()
    Ua = torch.zeros(inst.m, dtype=torch.int32, device="cuda")
    sa, na = h.step(xa, T=30, lr=0.1, seed=2, epoch=3, restart=True, unsat_counts=Ua)
    assert ffsat.last_points_per_cta() == 2
    xb = torch.from_numpy(x0.copy()).cuda()
    Ub = torch.zeros(inst.m, dtype=torch.int32, device="cuda")
    sb, nb = [], []
    for s in range(0, B, sms):
        part = xb[s:s + sms]
        ss, nn = h.step(part, T=30, lr=0.1, seed=2, epoch=3, restart=True, b_offset=s, unsat_counts=Ub)
        assert ffsat.last_points_per_cta() == 1
        sb.append(to_np(ss))
        nb.append(to_np(nn))
    if name == "3sat_n2000":
        assert torch.equal(xa, xb)
        assert np.array_equal(to_np(sa), np.concatenate(sb)) and np.array_equal(to_np(na), np.concatenate(nb))
        assert torch.equal(Ua, Ub)
    else:
        # restarted points are the same draws either way; the others within FP32 rounding
        assert torch.max(torch.abs(xa - xb)).item() < 1e-5


def test_two_points_per_cta_through_noalloc_and_graph():
    """The allocation-free entry point and a captured CUDA graph take the paired
    launch too, with the same bits as the ordinary call (a clause-only instance:
    every contribution is fixed point)."""
    from paper_2308_15020_gb300 import ffsat

    inst = gen.random_ksat(2000, 8400, 3, 13)
    h = ffsat.Instance(inst)
    B = 320
    x0 = torch.from_numpy(gen.uniform_points(B, inst.n, 9)).cuda()
    xa = x0.clone()
    h.step(xa, T=15, lr=0.1, seed=5, epoch=1)
    assert ffsat.last_points_per_cta() == 2
    xb = x0.clone()
    h.step_noalloc(xb, T=15, lr=0.1, seed=5, epoch=1)
    assert ffsat.last_points_per_cta() == 2
    assert torch.equal(xa, xb)
    xg = x0.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        h.step(xg.clone(), T=15, lr=0.1, seed=5, epoch=1)  # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        h.step(xg, T=15, lr=0.1, seed=5, epoch=1)
    xg.copy_(x0)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(xa, xg)


@pytest.mark.parametrize("name,make,mode", [
    ("3sat_n100", lambda: gen.uniform_3sat_100(4), 3),
    ("cnf_xor_300", lambda: gen.cnf_xor_2000(6, n=300), 3),
    ("hub_degree_5000", _hub, 1),  # the fixed point would resolve only 2^-36: gradient in a global row
])
def test_fp64_fixed_point_eval_and_step(name, make, mode):
    """FP64 with the gradient in shared memory accumulates clause and node
    contributions in two-word fixed point: within 1e-10 of the oracle, and
    without product constraints repeated calls give the same bits; an instance
    whose range would make it coarser keeps FP64 atomics in global rows."""
    from paper_2308_15020_gb300 import ffsat

    inst = make()
    h = ffsat.Instance(inst, cluster=1)
    assert h.info()["smem_mode_f64"] == mode
    x = gen.uniform_points(12, inst.n, 7, dtype=np.float64)
    outs = []
    for _ in range(2):
        f, g = h.eval_grad(torch.from_numpy(x).cuda())
        outs.append((to_np(f), to_np(g)))
    ef, eg = compare(inst, x, outs[0][0], outs[0][1], 1e-10)
    assert ef <= 1 and eg <= 1, (ef, eg)
    if mode == 3 and name == "3sat_n100":
        assert np.array_equal(outs[0][1].view(np.uint64), outs[1][1].view(np.uint64))
    xa = torch.from_numpy(x.copy()).cuda()
    xb = torch.from_numpy(x.copy()).cuda()
    h.step(xa, T=20, lr=0.05, seed=1, epoch=1, restart=False)
    h.step(xb, T=20, lr=0.05, seed=1, epoch=1, restart=False)
    xo, _, _ = O.step(inst, x, T=20, lr=0.05, seed=1, epoch=1, restart=False)
    assert np.max(np.abs(to_np(xa) - xo)) < 1e-9
    if mode == 3 and name == "3sat_n100":
        assert torch.equal(xa, xb)


@pytest.mark.parametrize("cluster", [1, 0])
def test_fp64_xor_only_relative_precision(cluster):
    """An XOR-only instance (parity learning, XORs of about N/2 literals): the
    gradient of a variable is a sum of products of many factors and can be tiny,
    and the FP64 paths keep it to 1e-10 of its own condition scale (product
    contributions are not rounded to the fixed point's absolute resolution)."""
    from paper_2308_15020_gb300 import ffsat

    inst = gen.parity_learning(40, 3)
    h = ffsat.Instance(inst, cluster=cluster)
    x = gen.uniform_points(8, inst.n, 4, dtype=np.float64)
    f, g = h.eval_grad(torch.from_numpy(x).cuda())
    ef, eg = compare(inst, x, to_np(f), to_np(g), 1e-10)
    assert ef <= 1 and eg <= 1, (ef, eg)
    xs = torch.from_numpy(x.copy()).cuda()
    h.step(xs, T=10, lr=0.5, seed=1, epoch=1, restart=False)
    xo, _, _ = O.step(inst, x, T=10, lr=0.5, seed=1, epoch=1, restart=False)
    assert np.max(np.abs(to_np(xs) - xo)) < 1e-10

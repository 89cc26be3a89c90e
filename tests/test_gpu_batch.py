"""One launch over several uneven instances (configuration 4) against the oracle
and against the single-instance entry points; the load-time autotuner."""
import numpy as np
import pytest

import oracle as O
from paper_2308_15020_gb300 import gen
from parity import compare, mixed_instance, to_np

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _instances():
    return [
        mixed_instance(21, n=700),                                             # resident image
        gen.cnf_xor_2000(2),                                                    # resident image, closed forms
        gen.concat([gen.random_ksat(20000, 60000, 3, 2), gen.random_atleast(20000, 30, 64, 512, 2)]),  # x, g
        gen.concat([gen.random_ksat(30000, 90000, 3, 3), gen.random_xor(30000, 50, 10, 60, 3, signs=True)]),  # x only
        gen.uniform_3sat_100(5),
        gen.rq1("card2", 1),
    ]


def test_batch_eval_matches_oracle_and_single():
    from paper_2308_15020_gb300 import ffsat

    insts = _instances()
    hs = [ffsat.Instance(i) for i in insts]
    modes = {h.info()["smem_mode_f32"] for h in hs}
    assert {0, 1, 3} <= modes
    bt = ffsat.Batch(hs)
    Bs = [5, 3, 2, 4, 7, 6]
    xs_np = [gen.uniform_points(B, i.n, 30 + k) for k, (B, i) in enumerate(zip(Bs, insts))]
    xs = [torch.from_numpy(x).cuda() for x in xs_np]
    fs, gs = bt.eval_grad(xs)
    for k, (inst, h) in enumerate(zip(insts, hs)):
        ef, eg = compare(inst, xs_np[k], to_np(fs[k]), to_np(gs[k]), 1e-4)
        assert ef <= 1 and eg <= 1, (k, ef, eg)
        f1, g1 = h.eval_grad(xs[k])
        assert np.allclose(to_np(f1), to_np(fs[k]), rtol=1e-6, atol=1e-6)
    for h in hs:
        h.sync_status()


def test_batch_step_restarts_and_one_iteration():
    from paper_2308_15020_gb300 import ffsat

    insts = _instances()[:4]
    hs = [ffsat.Instance(i) for i in insts]
    bt = ffsat.Batch(hs)
    Bs = [3, 4, 2, 2]
    xs_np = [gen.uniform_points(B, i.n, 50 + k) for k, (B, i) in enumerate(zip(Bs, insts))]
    xs = [torch.from_numpy(x).cuda() for x in xs_np]
    offs = [0, 100, 200, 300]
    solved, nun = bt.step(xs, T=1, lr=0.05, seed=4, epoch=2, restart=False, b_offsets=offs)
    for k, inst in enumerate(insts):
        _, gs = O.eval_grad(inst, xs_np[k].astype(np.float64))
        _, A = O.eval_scale(inst, xs_np[k].astype(np.float64), 1e-2)
        want = np.clip(xs_np[k].astype(np.float64) - 0.05 * gs, -1, 1)
        tol = 0.05 * 1e-4 * np.maximum(np.abs(gs), A) + 1e-7
        assert np.all(np.abs(to_np(xs[k]) - want) <= tol), k
        s2, n2 = O.check(inst, to_np(xs[k]).astype(np.float64))
        assert np.array_equal(to_np(solved[k]), s2) and np.array_equal(to_np(nun[k]), n2)
    # restarts: keyed by the per-instance offsets, bit-exact
    solved, nun = bt.step(xs, T=0, lr=0.05, seed=4, epoch=3, restart=True, b_offsets=offs)
    for k, inst in enumerate(insts):
        for b in range(Bs[k]):
            if not to_np(solved[k])[b]:
                want = np.array([O.uniform(4, 3, offs[k] + b, v) for v in range(inst.n)])
                assert np.array_equal(to_np(xs[k])[b].astype(np.float64), want)


def test_uneven_batch_shape_sampled():
    from paper_2308_15020_gb300 import ffsat

    insts = gen.uneven_batch(1, count=8)
    hs = [ffsat.Instance(i) for i in insts]
    bt = ffsat.Batch(hs)
    xs_np = [gen.uniform_points(16, i.n, 60 + k) for k, i in enumerate(insts)]
    xs = [torch.from_numpy(x).cuda() for x in xs_np]
    fs, gs = bt.eval_grad(xs)
    for k, inst in enumerate(insts):
        ef, eg = compare(inst, xs_np[k], to_np(fs[k]), to_np(gs[k]), 1e-4, points=np.array([0, 15]))
        assert ef <= 1 and eg <= 1, (k, ef, eg)


def test_autotune_picks_a_candidate_and_stays_exact():
    """The load-time autotuner times candidate tile choices (node literals per
    lane and segment shape, clause groups per task, points per CTA), keeps the
    fastest, reuses the choice for an instance of the same shape, and the tuned
    image evaluates and steps within the oracle's tolerance."""
    from paper_2308_15020_gb300 import ffsat

    inst = gen.concat([gen.random_ksat(3000, 9000, 3, 7), gen.random_atleast(3000, 60, 16, 200, 7)])
    h = ffsat.Instance(inst, autotune=True)
    info = h.info()
    assert info["autotuned"] == 1 and info["node_r"] in (8, 16)
    assert all(t > 0 for t in info["autotune_us"])
    assert info["autotune_us"][1] <= info["autotune_us"][0]
    assert info["tune_cached"] == 0 and info["tune_candidates"] >= 4
    assert info["tune_shape"] in (0, 1, 2) and info["tune_clause_k"] in (0, 1, 2, 4)
    assert info["tune_pts_per_cta"] in (1, 2)
    x = gen.uniform_points(9, inst.n, 3)
    f, g = h.eval_grad(torch.from_numpy(x).cuda())
    ef, eg = compare(inst, x, to_np(f), to_np(g), 1e-4)
    assert ef <= 1 and eg <= 1
    w = np.random.default_rng(0).uniform(0.5, 2, inst.m)
    h.set_weights(w)
    f, g = h.eval_grad(torch.from_numpy(x).cuda())
    ef, eg = compare(inst, x, to_np(f), to_np(g), 1e-4, weights=w)
    assert ef <= 1 and eg <= 1
    # an instance of another seed (its own shape, or a cached one) steps within tolerance
    inst2 = gen.concat([gen.random_ksat(3000, 9000, 3, 8), gen.random_atleast(3000, 60, 16, 200, 8)])
    h2 = ffsat.Instance(inst2, autotune=True)
    assert h2.info()["autotuned"] == 1
    x2 = gen.uniform_points(5, inst2.n, 4)
    xt = torch.from_numpy(x2).cuda()
    solved, nun = h2.step(xt, T=1, lr=0.05, seed=1, restart=False)
    _, gs = O.eval_grad(inst2, x2.astype(np.float64))
    _, A = O.eval_scale(inst2, x2.astype(np.float64), 1e-2)
    tol = 0.05 * 1e-4 * np.maximum(np.abs(gs), A) + 1e-7
    assert np.all(np.abs(to_np(xt) - np.clip(x2 - 0.05 * gs, -1, 1)) <= tol)
    # the same instance loaded again hits the cache
    h3 = ffsat.Instance(inst, autotune=True)
    i3 = h3.info()
    assert i3["tune_cached"] == 1 and i3["tune_candidates"] == 0
    assert (i3["node_r"], i3["tune_shape"], i3["tune_clause_k"], i3["tune_pts_per_cta"]) == \
        (info["node_r"], info["tune_shape"], info["tune_clause_k"], info["tune_pts_per_cta"])
    f3, g3 = h3.eval_grad(torch.from_numpy(x).cuda())
    h3.set_weights(np.ones(inst.m))
    # a batch of autotuned instances times both CTA widths of its FP32 kernel
    bt = ffsat.Batch([h, h3])
    th, us384, us512 = bt.threads()
    assert th in (384, 512) and us384 > 0 and us512 > 0
    assert ffsat.Batch([ffsat.Instance(inst)]).threads()[0] == 512
    fs, gs = bt.eval_grad([torch.from_numpy(x).cuda(), torch.from_numpy(x).cuda()])
    ef, eg = compare(inst, x, to_np(fs[1]), to_np(gs[1]), 1e-4)
    assert ef <= 1 and eg <= 1
    for hh in (h, h2, h3):
        hh.sync_status()


def test_batch_step_replays_from_a_cuda_graph():
    """With fixed buffers a batch step enqueues one memset and one kernel; it can be
    captured once and replayed."""
    from paper_2308_15020_gb300 import ffsat

    insts = [gen.cnf_xor_2000(3), mixed_instance(22, n=700)]
    hs = [ffsat.Instance(i) for i in insts]
    bt = ffsat.Batch(hs)
    xs = [torch.from_numpy(gen.uniform_points(4, i.n, 70 + k)).cuda() for k, i in enumerate(insts)]
    ref = [x.clone() for x in xs]
    solved = [torch.empty(4, dtype=torch.uint8, device="cuda") for _ in insts]
    nun = [torch.empty(4, dtype=torch.int32, device="cuda") for _ in insts]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # warm-up uploads the per-instance table outside the capture
        bt.step(xs, T=3, lr=0.1, seed=1, epoch=0, restart=False, solved=solved, n_unsat=nun, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    for x, r in zip(xs, ref):
        x.copy_(r)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        bt.step(xs, T=3, lr=0.1, seed=1, epoch=0, restart=False, solved=solved, n_unsat=nun, stream=s)
    for x, r in zip(xs, ref):
        x.copy_(r)
    graph.replay()
    torch.cuda.synchronize()
    got = [x.clone() for x in xs]
    for x, r in zip(xs, ref):
        x.copy_(r)
    bt.step(xs, T=3, lr=0.1, seed=1, epoch=0, restart=False, solved=solved, n_unsat=nun)
    torch.cuda.synchronize()
    for a, b in zip(got, xs):
        assert torch.allclose(a, b, atol=1e-5)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_batch_with_eight_literal_node_images(dtype):
    """Instances whose node path was built with 8 literals per lane (FP64 for
    constraints of <= 256 literals, or node_r = 8 in FP32) inside a batch whose
    kernel is the 16-literal one: same results as the single-instance path."""
    from paper_2308_15020_gb300 import ffsat

    insts = [gen.concat([gen.random_ksat(3000, 9000, 3, 11), gen.random_atleast(3000, 20, 32, 200, 11)]),
             mixed_instance(22, n=700)]
    hs = [ffsat.Instance(insts[0], node_r=8), ffsat.Instance(insts[1])]
    bt = ffsat.Batch(hs)
    xs = [torch.from_numpy(gen.uniform_points(4, i.n, 60 + k)).to(dtype).cuda() for k, i in enumerate(insts)]
    fs, gs = bt.eval_grad(xs)
    tol = 1e-4 if dtype == torch.float32 else 1e-10
    for k, (inst, h) in enumerate(zip(insts, hs)):
        ef, eg = compare(inst, xs[k].double().cpu().numpy(), to_np(fs[k]), to_np(gs[k]).astype(np.float64), tol)
        assert ef <= 1 and eg <= 1, (k, ef, eg)

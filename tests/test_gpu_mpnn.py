"""The learned restart proposal's CUDA forward/backward (dense layers on the
tensor cores) against the FP64 oracle with the same BF16 roundings, its
training, and the proposal restart."""
import numpy as np
import pytest

import mpnn_oracle as MO
import oracle as O
from paper_2308_15020_gb300 import gen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _small():
    return gen.concat([gen.random_ksat(80, 300, 3, 4), gen.random_xor(80, 10, 3, 12, 4, signs=True),
                       gen.random_atleast(80, 6, 5, 30, 4)])


def _medium():
    # many 32-row tiles with ragged tails on both sides of the graph
    return gen.concat([gen.random_ksat(709, 2950, 3, 5), gen.random_xor(709, 40, 3, 20, 5, signs=True),
                       gen.random_atleast(709, 23, 5, 60, 5)])


@pytest.mark.parametrize("make", [_small, _medium], ids=["small", "medium"])
def test_loss_and_gradient_match_oracle(make):
    from paper_2308_15020_gb300 import ffsat

    inst = make()
    h = ffsat.Instance(inst)
    net = ffsat.MPNN(layers=3, seed=1)
    rng = np.random.default_rng(2)
    p = (rng.normal(0, 0.2, net.num_params())).astype(np.float32)
    net.set_params(p)
    t = np.where(rng.random(inst.n) < 0.5, -1.0, 1.0)
    loss, x0, g = net.loss_grad(h, torch.from_numpy(t.astype(np.float32)).cuda(), want_host_grad=True)
    # the oracle with BF16 weights and BF16-rounded dense-product inputs, as the
    # tensor-core layers compute.  FP32 and FP64 values that fall on opposite
    # sides of a BF16 rounding boundary differ by one BF16 unit (2^-8 relative),
    # and such flips propagate through the layers: the bounds below allow a few
    # BF16 units at the worst element and a fraction of one in RMS (the
    # unrounded oracle differs by several times more; a wrong operand layout or
    # a dropped term by the size of the values themselves)
    lo, go, xo = MO.loss_and_grad(p.astype(np.float64), inst, t, 3, bf16_weights=True, bf16_inputs=True)
    assert abs(float(loss.item()) - lo) <= 2e-4 * max(1.0, abs(lo))
    xk = x0.cpu().numpy()
    assert np.max(np.abs(xk - xo)) < 2e-2 and np.sqrt(np.mean((xk - xo) ** 2)) < 2e-3
    lay, _ = MO.layout(3)
    for name, (o, shape) in lay.items():
        a, b = go[o:o + int(np.prod(shape))], g[o:o + int(np.prod(shape))]
        scale, rms = np.max(np.abs(a)), np.sqrt(np.mean(a ** 2))
        assert np.max(np.abs(a - b)) <= 2e-2 * scale, name
        assert np.sqrt(np.mean((a - b) ** 2)) <= 1e-2 * rms, name
    x1 = net.forward(h)
    assert torch.equal(x1, x0)


def test_training_reduces_loss():
    from paper_2308_15020_gb300 import ffsat

    inst = gen.cnf_xor_2000(5, planted=True, n=400)
    h = ffsat.Instance(inst)
    net = ffsat.MPNN(layers=3, seed=3)
    t = torch.from_numpy(inst.planted.astype(np.float32)).cuda()
    first = None
    for it in range(60):
        loss, _, _ = net.loss_grad(h, t)
        net.adam_step(3e-3)
        if first is None:
            first = float(loss.item())
    last = float(net.loss_grad(h, t)[0].item())
    assert last < 0.8 * first, (first, last)


def test_proposal_restart_is_exact():
    from paper_2308_15020_gb300 import ffsat

    inst = gen.uniform_3sat_100(1)
    h = ffsat.Instance(inst)
    prop = np.random.default_rng(0).uniform(-1, 1, inst.n).astype(np.float32)
    x = torch.zeros(5, inst.n, device="cuda")
    solved = torch.tensor([0, 1, 0, 0, 1], dtype=torch.uint8, device="cuda")
    ffsat.restart_from_proposal(h, x, torch.from_numpy(prop).cuda(), 0.5, solved=solved, seed=9, epoch=4, b_offset=20)
    got = x.cpu().numpy()
    for b in range(5):
        if b in (1, 4):
            assert np.all(got[b] == 0)
        else:
            u = np.array([O.uniform(9, 4, 20 + b, v) for v in range(inst.n)], dtype=np.float32)
            want = np.clip(prop + np.float32(0.5) * u, -1, 1)
            assert np.array_equal(got[b], want)


def test_learned_proposal_reduces_time_to_sat():
    """What the trained network gains over the method without it: trained on the
    CLS's own best points of 600 planted 3-SAT instances (n = 400, ratio 4.2),
    restarts drawn around its proposal solve several times more held-out
    instances (n = 350) within the same budget than uniform restarts from the
    same seeds and end far closer to a model.  (Training accumulates in FP32 with
    atomics, so the exact counts vary from run to run; the margins below hold
    across runs.)"""
    from paper_2308_15020_gb300 import learned

    res = learned.learned_restart_experiment(
        train_count=600, test_count=24, n_train=400, n_test=350, family="3sat",
        test_cfg=learned.CLSConfig(B=256, T=100, lr=0.1, max_rounds=300, seed=9))
    print(res)
    assert res["held_out_sign_agreement"] > 0.7
    assert res["solved"]["learned"] >= res["solved"]["uniform"] + 4
    assert res["mean_best_unsat"]["learned"] < 0.6 * res["mean_best_unsat"]["uniform"]


def test_learned_proposal_on_the_cnf_xor_family():
    """The same gain on the configuration-5 family itself (planted CNF-XOR, 4.2 n
    3-clauses and n/10 XORs of 10..40 literals): trained on the CLS's own best
    points of 300 instances at n = 2000, restarts around the proposal reach,
    on 4 held-out instances at n = 5000, points that violate under 0.6x as many
    constraints as uniform restarts from the same seeds, and reach 200 violated
    constraints in the first rounds where uniform restarts never do within the
    budget.  The best points' violations are counted by constraint type."""
    from paper_2308_15020_gb300 import learned

    res = learned.learned_restart_experiment(
        train_count=300, test_count=4, n_train=2000, n_test=5000, family="cnf_xor",
        test_cfg=learned.CLSConfig(B=256, T=100, lr=0.1, max_rounds=40, seed=9))
    print({k: res[k] for k in ("mean_best_unsat", "median_par2_s_to_unsat_le", "violated_at_best_by_type")})
    assert res["mean_best_unsat"]["learned"] < 0.6 * res["mean_best_unsat"]["uniform"]
    k200 = res["median_par2_s_to_unsat_le"]["200"]
    assert k200["learned"] < k200["uniform"]
    vt = res["violated_at_best_by_type"]
    for arm in ("uniform", "learned"):
        assert vt[arm] is not None and sum(vt[arm].values()) > 0

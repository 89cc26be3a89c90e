"""Checkpoint and resume of a CLS search: three rounds, a state handed to a
fresh instance, three more rounds equal six uninterrupted rounds bit for bit
(FP32 shared-memory-resident path, whose gradient sums are order-independent)."""
import io

import numpy as np
import pytest
import torch as _torch_for_save

from paper_2308_15020_gb300 import gen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_resume_equals_uninterrupted():
    from paper_2308_15020_gb300 import ffsat, learned

    inst = gen.random_ksat(300, 1260, 3, 8)
    cfg = learned.CLSConfig(B=64, T=30, lr=0.1, max_rounds=6, seed=4, heuristics=True, policy="ROF")
    h = ffsat.Instance(inst)
    assert h.info()["smem_mode_f32"] == 3
    S = learned.CLSSearch(h, inst.n, cfg, cfg.seed)
    for r in range(6):
        S.round(r)
    want_x, want_w = S.x.cpu().numpy(), h.get_weights()

    h1 = ffsat.Instance(inst)
    S1 = learned.CLSSearch(h1, inst.n, cfg, cfg.seed)
    for r in range(3):
        S1.round(r)
    buf = io.BytesIO()
    _torch_for_save.save(S1.state_dict(), buf)  # through bytes, as a checkpoint file would
    del S1, h1
    buf.seek(0)
    state = _torch_for_save.load(buf, weights_only=False)
    h2 = ffsat.Instance(inst)
    S2 = learned.CLSSearch.from_state(h2, state)
    for r in range(S2.rounds_done, 6):
        S2.round(r)
    assert np.array_equal(S2.x.cpu().numpy(), want_x)
    assert np.array_equal(h2.get_weights(), want_w)


def test_graph_replayed_rounds_equal_eager_rounds():
    """One ROF period captured in a CUDA graph and replayed twice (device epoch
    counter) leaves the points and weights exactly where six eager rounds do."""
    from paper_2308_15020_gb300 import ffsat, learned

    inst = gen.random_ksat(300, 1260, 3, 9)
    cfg = learned.CLSConfig(B=64, T=20, lr=0.1, max_rounds=6, seed=5, heuristics=True, policy="ROF")
    h = ffsat.Instance(inst)
    S = learned.CLSSearch(h, inst.n, cfg, cfg.seed)
    for r in range(6):
        S.round(r)
    want_x, want_w = S.x.cpu().numpy(), h.get_weights()
    h2 = ffsat.Instance(inst)
    keep = {}
    run = learned.time_to_sat_graph(h2, inst.n, cfg, cfg.seed, target_unsat=-1, keep=keep)  # never stops early
    assert run.rounds == 6 and not run.solved
    assert np.array_equal(keep["x"].cpu().numpy(), want_x)
    assert np.array_equal(h2.get_weights(), want_w)

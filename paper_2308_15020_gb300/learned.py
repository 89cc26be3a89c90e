"""Learned restart proposal: data from our own CLS runs, training with the
library's network kernels, and the A/B time-to-SAT protocol.

Every device computation runs in the CUDA library (ffsat_step, ffsat_check,
the ffsat_mpnn_* kernels and ffsat_restart_from_proposal); this module only
orchestrates them.  PyTorch supplies device buffers.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

from . import ffsat, gen


@dataclass
class CLSConfig:
    B: int = 64          # restart points per round
    T: int = 100         # projected-GD iterations per round
    lr: float = 0.1
    max_rounds: int = 30
    noise: float = 0.7   # proposal restarts: x = clip(p + noise * u)
    seed: int = 1
    heuristics: bool = True  # ERWA weights + rephasing between rounds (else plain restarts)
    erwa: Optional[bool] = None  # ERWA on/off separately (None: as heuristics); fixed weights + rephasing for optimisation
    alpha: float = 0.4       # ERWA decay (Prop. "Adaptive weight")
    policy: str = "ROF"      # rephasing policy, repeated: R random, O original, F flipped
    dtype: str = "f32"       # real type of the points: "f32" or "f64"
    method: str = "fixed"    # "fixed": x <- clip(x - lr g) T times; "pgfp": FISTA line search from eta0 = lr


_PHASE = {"O": 0, "F": 1, "R": 2}


class CLSSearch:
    """State of one CLS run on one instance: B points, per-round step, and the
    restart rule between rounds -- uniform restarts, or (cfg.heuristics) the
    ERWA update plus the rephasing policy, where the learned arm draws its random
    phase around the network's proposal instead of uniformly."""

    def __init__(self, h: ffsat.Instance, n: int, cfg: CLSConfig, seed: int, prop=None):
        import torch

        self.h, self.cfg, self.seed, self.prop = h, cfg, seed, prop
        self.x = torch.zeros(cfg.B, n, dtype=torch.float64 if cfg.dtype == "f64" else torch.float32, device="cuda")
        self.use_erwa = cfg.heuristics if cfg.erwa is None else (cfg.erwa and cfg.heuristics)
        self.U = torch.zeros(h.m, dtype=torch.int32, device="cuda") if self.use_erwa else None
        self.rounds_done = 0
        if prop is None:
            h.rephase(self.x, ffsat.FFSAT_PHASE_RANDOM, seed=seed, epoch=0)
        else:
            ffsat.restart_from_proposal(h, self.x, prop, cfg.noise, seed=seed, epoch=0)

    # -- checkpoint / resume -------------------------------------------------------------
    def state_dict(self) -> dict:
        """Everything a later process needs to continue this search exactly: the
        points, the device weights (ERWA), the rounds done, the seed and the
        configuration (host copies)."""
        return {"x": self.x.detach().cpu().clone(), "weights": self.h.get_weights(),
                "rounds_done": self.rounds_done, "seed": self.seed, "cfg": dict(vars(self.cfg)),
                "proposal": None if self.prop is None else self.prop.detach().cpu().clone()}

    @classmethod
    def from_state(cls, h: ffsat.Instance, state: dict) -> "CLSSearch":
        """Resume a search from state_dict() on a freshly loaded instance.  The
        next round() should be given r = state["rounds_done"]; the restart draws
        are keyed by (seed, round), so the continuation matches an uninterrupted
        run (bit for bit where the gradient accumulation is order-independent:
        the FP32 shared-memory-resident clause and node paths)."""
        import torch

        cfg = CLSConfig(**state["cfg"])
        self = cls.__new__(cls)
        self.h, self.cfg, self.seed = h, cfg, state["seed"]
        self.prop = None if state["proposal"] is None else state["proposal"].cuda()
        self.x = state["x"].cuda()
        self.use_erwa = cfg.heuristics if cfg.erwa is None else (cfg.erwa and cfg.heuristics)
        self.U = torch.zeros(h.m, dtype=torch.int32, device="cuda") if self.use_erwa else None
        self.rounds_done = state["rounds_done"]
        h.set_weights(state["weights"])
        return self

    def round(self, r: int, on_checked=None):
        """One round: T iterations and the exact check (on_checked(x, solved,
        n_unsat) sees the points here), then the restart rule for the points that
        are not models.  Returns (solved, n_unsat) of the round."""
        cfg, h, x = self.cfg, self.h, self.x
        if self.U is not None:
            self.U.zero_()
        if cfg.method == "pgfp":
            solved, nun = h.step_pgfp(x, T=cfg.T, eta0=cfg.lr, seed=self.seed, epoch=r + 1, restart=False,
                                      unsat_counts=self.U)
        else:
            solved, nun = h.step(x, T=cfg.T, lr=cfg.lr, seed=self.seed, epoch=r + 1, restart=False,
                                 unsat_counts=self.U)
        if on_checked is not None:
            on_checked(x, solved, nun)
        phase = ffsat.FFSAT_PHASE_RANDOM
        if cfg.heuristics:
            if self.use_erwa:
                h.erwa_update(self.U, cfg.alpha)
            phase = _PHASE[cfg.policy[r % len(cfg.policy)]]
        if phase == ffsat.FFSAT_PHASE_RANDOM and self.prop is not None:
            ffsat.restart_from_proposal(h, x, self.prop, cfg.noise, solved=solved, seed=self.seed, epoch=r + 1)
        else:
            h.rephase(x, phase, solved=solved, seed=self.seed, epoch=r + 1)
        self.rounds_done = r + 1
        return solved, nun


def best_point(h: ffsat.Instance, n: int, cfg: CLSConfig, seed: int, net: Optional[ffsat.MPNN] = None):
    """Run CLS rounds (uniform restarts, or restarts around the network's proposal);
    return (signs of the best point found, its #unsat, rounds)."""
    import torch

    if cfg.heuristics:
        h.set_weights(h.host_weights)
    prop = None if net is None else net.forward(h)
    S = CLSSearch(h, n, cfg, seed, prop)
    st = {"best": None, "u": math.inf}

    def keep_best(x, solved, nun):
        u = nun.cpu().numpy()
        b = int(np.argmin(u))
        if u[b] < st["u"]:
            st["u"] = int(u[b])
            st["best"] = torch.where(x[b] < 0, -1.0, 1.0)

    rounds = 0
    for r in range(cfg.max_rounds):
        rounds = r + 1
        S.round(r, keep_best)
        if st["u"] == 0:
            break
    best, best_u = st["best"], st["u"]
    if cfg.heuristics:
        h.set_weights(h.host_weights)
    return best, best_u, rounds


def collect(instances, cfg: CLSConfig, net: Optional[ffsat.MPNN] = None, handles=None):
    """Targets for training: for each instance, the signs of the best point the
    CLS finds (with uniform restarts, or with the network's proposals)."""
    data = []
    for k, inst in enumerate(instances):
        h = handles[k] if handles is not None else ffsat.Instance(inst)
        t, u, _ = best_point(h, inst.n, cfg, cfg.seed + 1000 * k, net)
        data.append((h, t, u))
    return data


def self_train(net: ffsat.MPNN, instances, cfg: CLSConfig, rounds: int = 2, epochs: int = 6, lr: float = 2e-3):
    """Train on CLS near-solutions; then regenerate the targets with CLS runs that
    restart around the current proposal and continue training (rounds times).
    Returns the per-round mean #unsat of the targets and the losses."""
    data = collect(instances, cfg)
    handles = [d[0] for d in data]
    hist = [float(np.mean([d[2] for d in data]))]
    losses = train(net, data, epochs, lr)
    for _ in range(rounds - 1):
        data = collect(instances, cfg, net, handles)
        hist.append(float(np.mean([d[2] for d in data])))
        losses += train(net, data, epochs, lr)
    return hist, losses


def train(net: ffsat.MPNN, data, epochs: int = 5, lr: float = 2e-3, seed: int = 0) -> List[float]:
    """Adam on the logistic loss of the proposal against the collected signs."""
    rng = np.random.default_rng(seed)
    losses = []
    for _ in range(epochs):
        tot = 0.0
        for i in rng.permutation(len(data)):
            h, t, _ = data[i]
            loss, _, _ = net.loss_grad(h, t)
            net.adam_step(lr)
            tot += float(loss.item())
        losses.append(tot / max(1, len(data)))
    return losses


@dataclass
class SatRun:
    solved: bool
    seconds: float
    rounds: int
    best_unsat: int = -1  # fewest violated constraints of any point seen (0 when solved)
    # (seconds since the start, fewest violated constraints so far) after every round
    trajectory: List[Tuple[float, int]] = field(default_factory=list)
    # violated constraints of the best point, by type (with keep_best)
    violated_by_type: Optional[dict] = None

    def time_to_unsat(self, k: int) -> float:
        """Seconds until some point violated at most k constraints (inf if never)."""
        return next((t for t, u in self.trajectory if u <= k), math.inf)


def time_to_sat(h: ffsat.Instance, n: int, cfg: CLSConfig, seed: int, net: Optional[ffsat.MPNN] = None,
                target_unsat: int = 0, keep_best: bool = False, ctype=None) -> SatRun:
    """Wall time until some point's sign vector is a model (Alg. 1) -- or violates
    at most target_unsat constraints -- with uniform restarts (net None) or
    restarts drawn around the network's proposal.  With keep_best (and the
    instance's constraint types `ctype`) the best point is kept on the device
    (no extra host synchronisation) and the constraints it violates are counted
    by type after the run."""
    import torch

    if cfg.heuristics:
        h.set_weights(h.host_weights)  # every run starts from the instance's own weights
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    prop = None if net is None else net.forward(h)
    S = CLSSearch(h, n, cfg, seed, prop)
    best = None
    traj = []
    keep = {}

    def on_checked(x, solved, nun):
        i = nun.argmin()
        u, row = nun[i], x[i]
        if "x" not in keep:
            keep["u"], keep["x"] = u.clone(), row.clone()
        else:
            better = u < keep["u"]
            keep["x"] = torch.where(better, row, keep["x"])
            keep["u"] = torch.minimum(keep["u"], u)

    run = None
    for r in range(cfg.max_rounds):
        solved, nun = S.round(r, on_checked if keep_best else None)
        m = nun.min()
        best = m if best is None else torch.minimum(best, m)
        b = int(best.item())  # the round's one host synchronisation
        traj.append((time.perf_counter() - t0, b))
        if b <= target_unsat:
            run = SatRun(True, traj[-1][0], r + 1, 0, traj)
            break
    if run is None:
        run = SatRun(False, time.perf_counter() - t0, cfg.max_rounds, traj[-1][1] if traj else -1, traj)
    if keep_best and "x" in keep and ctype is not None:
        U = h.unsat_counts(keep["x"].reshape(1, -1).contiguous()).cpu().numpy()
        ct = np.asarray(ctype)
        run.violated_by_type = {name: int(U[ct == t].sum()) for name, t in
                                (("clauses", ffsat.FFSAT_OR), ("xor", ffsat.FFSAT_XOR), ("atleast", ffsat.FFSAT_ATLEAST))}
    return run


def time_to_sat_graph(h: ffsat.Instance, n: int, cfg: CLSConfig, seed: int, target_unsat: int = 0,
                      keep: Optional[dict] = None) -> SatRun:
    """time_to_sat with uniform restarts, where each round (step with violation
    counts, ERWA update, rephase) is a CUDA graph replay: one graph per phase of
    the rephasing policy, captured once; the random phase reads its epoch from a
    device counter that the graphs advance, so every replay draws what the eager
    loop would.  The host reads the best #unsat once per round."""
    import torch

    if cfg.heuristics:
        h.set_weights(h.host_weights)
    warm(h, n, cfg, None)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S = CLSSearch(h, n, cfg, seed)
    x = S.x
    if keep is not None:
        keep["x"] = x  # the points, for callers that continue or inspect the search
    B = cfg.B
    solved = torch.zeros(B, dtype=torch.uint8, device="cuda")
    nun = torch.zeros(B, dtype=torch.int32, device="cuda")
    best = torch.full((1,), 2**31 - 1, dtype=torch.int32, device="cuda")
    ctr = torch.ones(1, dtype=torch.int64, device="cuda")  # round r draws with epoch r + 1
    policy = cfg.policy if cfg.heuristics else "R"

    def one_round(ph):
        if S.U is not None:
            S.U.zero_()
        if cfg.method == "pgfp":
            h.step_pgfp(x, T=cfg.T, eta0=cfg.lr, seed=seed, restart=False, solved=solved, n_unsat=nun,
                        unsat_counts=S.U)
        else:
            h.step(x, T=cfg.T, lr=cfg.lr, seed=seed, restart=False, solved=solved, n_unsat=nun, unsat_counts=S.U)
        torch.minimum(best, nun.min().reshape(1), out=best)
        if S.use_erwa:
            h.erwa_update(S.U, cfg.alpha)
        h.rephase(x, _PHASE[ph], solved=solved, seed=seed, epoch_dev=ctr)
        ctr.add_(1)

    graphs = {}
    for ph in set(policy):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            one_round(ph)
        graphs[ph] = g
    for r in range(cfg.max_rounds):
        graphs[policy[r % len(policy)]].replay()
        if int(best.item()) <= target_unsat:
            torch.cuda.synchronize()
            return SatRun(True, time.perf_counter() - t0, r + 1, 0)
    torch.cuda.synchronize()
    return SatRun(False, time.perf_counter() - t0, cfg.max_rounds, int(best.item()))


UNSAT_LADDER = (400, 200, 100, 50, 20, 5, 0)


@dataclass
class ABResult:
    uniform: List[SatRun] = field(default_factory=list)
    learned: List[SatRun] = field(default_factory=list)

    @staticmethod
    def _median(runs):
        v = [r.seconds if r.solved else math.inf for r in runs]
        return float(np.median(v)) if v else math.nan

    @staticmethod
    def _par2(runs, budget):
        """Median PAR-2 time: unsolved runs count as twice the budget (the paper's
        convention for unsolved instances)."""
        v = [r.seconds if r.solved else 2.0 * budget for r in runs]
        return float(np.median(v)) if v else math.nan

    def summary(self):
        budget = max([r.seconds for r in self.uniform + self.learned if not r.solved] or [0.0])
        arms = {"uniform": self.uniform, "learned": self.learned}
        return {
            "instances": len(self.uniform),
            "median_time_to_sat_s": {k: self._median(v) for k, v in arms.items()},
            "median_par2_s": {k: self._par2(v, budget) for k, v in arms.items()},
            "par2_budget_s": budget,
            "median_rounds": {k: float(np.median([r.rounds for r in v])) for k, v in arms.items()},
            "solved": {k: sum(r.solved for r in v) for k, v in arms.items()},
            "mean_best_unsat": {k: float(np.mean([r.best_unsat for r in v])) for k, v in arms.items()},
            # median (PAR-2) time until some point violates at most K constraints, for a
            # fixed ladder of K: time-to-SAT is the K = 0 rung
            "median_par2_s_to_unsat_le": {
                str(K): {k: self._par2_to(v, K, budget) for k, v in arms.items()} for K in UNSAT_LADDER},
            # mean violated constraints of each run's best point, by type
            "violated_at_best_by_type": {k: self._by_type(v) for k, v in arms.items()},
        }

    @staticmethod
    def _by_type(runs):
        rs = [r.violated_by_type for r in runs if r.violated_by_type is not None]
        if not rs:
            return None
        return {t: float(np.mean([r[t] for r in rs])) for t in rs[0]}

    @staticmethod
    def _par2_to(runs, K, budget):
        v = [min(r.time_to_unsat(K), 2.0 * budget) for r in runs]
        return float(np.median(v)) if v else math.nan


def warm(h: ffsat.Instance, n: int, cfg: CLSConfig, net: Optional[ffsat.MPNN]):
    """Untimed first use of an instance: kernel limits, scratch, the network's graph data."""
    import torch

    x = torch.zeros(cfg.B, n, dtype=torch.float64 if cfg.dtype == "f64" else torch.float32, device="cuda")
    if cfg.method == "pgfp":
        h.step_pgfp(x, T=1, eta0=cfg.lr, restart=False)
    else:
        h.step(x, T=1, lr=cfg.lr, restart=False)
    if net is not None:
        net.forward(h)
    torch.cuda.synchronize()


def ab_test(net: ffsat.MPNN, instances, cfg: CLSConfig) -> ABResult:
    """Held-out A/B: the same instances and seeds with uniform and learned restarts."""
    res = ABResult()
    for k, inst in enumerate(instances):
        h = ffsat.Instance(inst)
        seed = cfg.seed + 7919 * k
        warm(h, inst.n, cfg, net)
        res.uniform.append(time_to_sat(h, inst.n, cfg, seed, None, keep_best=True, ctype=inst.ctype))
        res.learned.append(time_to_sat(h, inst.n, cfg, seed, net, keep_best=True, ctype=inst.ctype))
    return res


def sign_agreement(net: ffsat.MPNN, instances) -> float:
    """Mean fraction of variables whose proposal sign matches the planted assignment."""
    vals = []
    for inst in instances:
        h = ffsat.Instance(inst)
        p = net.forward(h).cpu().numpy()
        vals.append(float(np.mean(np.where(p < 0, -1, 1) == inst.planted)))
    return float(np.mean(vals))


def planted_family(count: int, n: int, seed0: int):
    """CNF-XOR instances of the n=2000 shape (m = 4.2 n clauses, n/10 XORs), planted."""
    return [gen.cnf_xor_2000(seed0 + i, planted=True, n=n) for i in range(count)]


def planted_3sat_family(count: int, n: int, seed0: int, ratio: float = 4.2):
    """Planted random 3-SAT at the given clause ratio."""
    return [gen.random_ksat(n, int(round(ratio * n)), 3, seed0 + i, planted=gen.planted_assignment(n, seed0 + i))
            for i in range(count)]


def learned_restart_experiment(train_count: int = 2000, test_count: int = 100, n_train: int = 2000,
                               n_test: int = 5000, family: str = "cnf_xor", self_train_rounds: int = 2,
                               epochs: int = 6, collect_cfg: Optional[CLSConfig] = None,
                               test_cfg: Optional[CLSConfig] = None, seed: int = 0, log=None):
    """Train the proposal network on the CLS's own best points over train_count
    seeded planted instances of the family at n_train, then A/B time-to-SAT on
    test_count held-out instances at n_test (uniform restarts vs restarts around
    the proposal, same seeds, same heuristics).  Returns a summary dict."""
    def say(*a):
        if log is not None:
            log(*a)

    make = planted_family if family == "cnf_xor" else planted_3sat_family
    collect_cfg = collect_cfg or CLSConfig(B=64, T=100, lr=0.1, max_rounds=10, seed=3)
    test_cfg = test_cfg or CLSConfig(B=256, T=100, lr=0.1, max_rounds=30, seed=9)
    t0 = time.perf_counter()
    train_set = make(train_count, n_train, 100000 + seed)
    net = ffsat.MPNN(3, seed + 7)
    hist, losses = self_train(net, train_set, collect_cfg, rounds=self_train_rounds, epochs=epochs)
    t_train = time.perf_counter() - t0
    say(f"trained on {train_count} instances in {t_train:.0f} s; target #unsat per round {hist}")
    test_set = make(test_count, n_test, 900000 + seed)
    agree = sign_agreement(net, test_set)
    res = ab_test(net, test_set, test_cfg)
    out = res.summary()
    out.update({"family": family, "train_instances": train_count, "n_train": n_train, "test_instances": test_count,
                "n_test": n_test, "target_mean_unsat_per_self_training_round": hist,
                "final_train_loss": losses[-1] if losses else None, "held_out_sign_agreement": agree,
                "train_seconds": t_train, "total_seconds": time.perf_counter() - t0,
                "collect": vars(collect_cfg), "test": vars(test_cfg)})
    return out

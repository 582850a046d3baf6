"""Learned proposal experiment: does the network help RV-GOMEA?

1. Plain runs of the optimiser on a problem collect elites (archive members).
2. Training pairs: for every state (a candidate of a plain run's initial
   population) and point, features of the state at that point and, as
   target, the displacement of the target-mesh point from the state to a
   randomly drawn elite.
3. The network is trained on the GPU (tcgen05 forward and backward, Adam).
4. Fresh runs with and without the learned sampler (alpha = probability that
   a trial's target-mesh move is drawn from the network's Gaussian) are
   compared by hypervolume against evaluations (GOMEA units), both against
   one reference point fixed from the initial population.
"""
from __future__ import annotations

import numpy as np

from . import dmr, gomea, synth


def make_problem(pr, stream=None, storage="f32"):
    C = pr["coords"].shape[0]
    return dmr.Problem(pr["img"][0], pr["img"][1], *pr["spacing"], pr["mesh"], guide=pr["guide"],
                       model=dmr.LINEAR, storage=storage, max_candidates=C, stream=stream)


def proposal_fn(prob, net):
    """coords [C,2,3,P] (host) -> (mean [C,P,3], log-variance [C,P,3]) (host)."""
    import torch

    def f(coords):
        C = coords.shape[0]
        X = dmr.MLP.features(prob, torch.from_numpy(np.ascontiguousarray(coords)).cuda())
        out = net.forward(X).cpu().numpy().reshape(C, prob.P, 6)
        lv = np.clip(out[..., 3:], -8.0, 4.0)
        return out[..., :3].astype(np.float64), lv.astype(np.float64)

    return f


def collect(pr, seeds, generations, sigma0, n_samples, rng):
    """Plain runs -> training set (X device BF16 [n, 256], Y device FP32 [n, 3])."""
    import torch

    states, targets = [], []
    for sd in seeds:
        prob = make_problem(pr)
        opt = gomea.Gomea(prob, pr["coords"], synth.single_point_fos(pr["mesh"]), pr["mesh"], sigma0,
                          np.random.default_rng(sd))
        start = opt.coords.copy()
        for _ in range(generations):
            opt.generation()
        elites = [c for c in opt.archive.coords if c is not None]
        if not elites:
            continue
        for c in range(start.shape[0]):
            e = elites[int(rng.integers(len(elites)))]
            states.append(start[c])
            targets.append((e[1] - start[c][1]).T)  # [P, 3] target-mesh displacement
        prob.close()
    states = np.stack(states)
    prob = make_problem(pr)
    X = dmr.MLP.features(prob, torch.from_numpy(states).cuda())
    Y = torch.from_numpy(np.concatenate(targets).astype(np.float32)).cuda()
    if n_samples and n_samples < X.shape[0]:
        idx = torch.from_numpy(rng.choice(X.shape[0], n_samples, replace=False)).cuda()
        X, Y = X.index_select(0, idx), Y.index_select(0, idx)
    return X, Y


def train(net, X, Y, steps, batch, lr, rng):
    import torch

    n = X.shape[0]
    losses = []
    for _ in range(steps):
        idx = torch.from_numpy(rng.integers(0, n, batch)).cuda()
        losses.append(net.train_step(X.index_select(0, idx), Y.index_select(0, idx), lr))
    return losses


def evals_to_reach(curve, target):
    """First evaluation count at which the curve's HV reaches target
    (linear interpolation between generations); inf if never."""
    prev_e, prev_h = None, None
    for e, h in curve:
        if h >= target:
            if prev_e is None or h == prev_h:
                return e
            return prev_e + (target - prev_h) / (h - prev_h) * (e - prev_e)
        prev_e, prev_h = e, h
    return float("inf")


def compare(pr, net, seeds, generations, sigma0, alpha):
    """HV curves of plain and learned runs; evaluations each needs to reach the
    plain run's final HV (per seed)."""
    prob0 = make_problem(pr)
    obj0 = np.asarray(prob0.eval_full(pr["coords"]))
    ref = 1.1 * np.max(obj0[:, :3], axis=0)
    prob0.close()
    rows = []
    for sd in seeds:
        curves = {}
        for arm in ("plain", "learned"):
            prob = make_problem(pr)
            prop = proposal_fn(prob, net) if arm == "learned" else None
            opt = gomea.Gomea(prob, pr["coords"], synth.single_point_fos(pr["mesh"]), pr["mesh"], sigma0,
                              np.random.default_rng(1000 + sd), proposal=prop, alpha=alpha)
            curves[arm] = opt.run(generations, ref)
            prob.close()
        target = curves["plain"][-1][1]
        rows.append({"seed": sd, "plain_final_hv": target, "learned_final_hv": curves["learned"][-1][1],
                     "plain_evals": evals_to_reach(curves["plain"], target),
                     "learned_evals": evals_to_reach(curves["learned"], target),
                     "curves": curves})
    return ref, rows

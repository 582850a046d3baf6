"""Minimal multi-objective GOMEA scaffold over the C-ABI evaluator.

Only what measuring "hypervolume at a fixed evaluation budget" needs; the
paper specifies the optimiser only as far as Sec. 2.2 (FOS groups changed
together, a change accepted only if it improves, independent groups changed
in parallel) and Sec. 2.4 (approximation set from an elitist archive of
non-dominated solutions).  Per generation and wave of independent groups:
sample a proposal for every (candidate, group), evaluate partially on the
GPU, accept-if-improves and commit on the GPU.  Proposal = current group
coordinates + N(0, s_g^2) on the free axes of both meshes, s_g adapted per
group with the 1/5 success rule; optionally (learned proposal) the
target-mesh part of a trial is drawn from the MLP's Gaussian instead, with
probability alpha.

Budget (GOMEA convention): a partial evaluation costs |touched tets| / N_tet
of a full evaluation; a full evaluation costs 1.
"""
from __future__ import annotations

import numpy as np

from . import dmr, synth


def nondominated(objs):
    """Mask of the rows of ``objs`` [n, d] not dominated by another row."""
    n = len(objs)
    keep = np.ones(n, bool)
    for i in range(n):
        if not keep[i]:
            continue
        dom = np.all(objs <= objs[i], axis=1) & np.any(objs < objs[i], axis=1)
        if dom.any():
            keep[i] = False
    return keep


class Archive:
    """Elitist archive: feasible, mutually non-dominated (f_sim, f_def, f_guid)."""

    def __init__(self, cap=2000):
        self.cap = cap
        self.objs = np.zeros((0, 3))
        self.coords = []

    def update(self, objs, coords_of):
        """Add the feasible, mutually non-dominated candidates of objs [C, 4]
        (exact duplicates of archive members are skipped) and drop archive
        members they dominate."""
        cand = np.nonzero(objs[:, 3] == 0)[0]
        if len(cand) == 0:
            return
        N = objs[cand, :3]
        # exact duplicates (against the archive and among the candidates)
        rows = np.ascontiguousarray(N).view(np.dtype((np.void, N.dtype.itemsize * 3))).ravel()
        _, first = np.unique(rows, return_index=True)
        keep = np.zeros(len(cand), bool)
        keep[first] = True
        if len(self.objs):
            arows = np.ascontiguousarray(self.objs).view(np.dtype((np.void, N.dtype.itemsize * 3))).ravel()
            keep &= ~np.isin(rows, arows)
        cand, N = cand[keep], N[keep]
        if len(cand) == 0:
            return

        def dominates(a, b):  # [i, j]: a_i dominates b_j
            return np.all(a[:, None, :] <= b[None, :, :], axis=2) & np.any(a[:, None, :] < b[None, :, :], axis=2)

        new_ok = ~np.any(dominates(N, N), axis=0)
        old_ok = np.ones(len(self.objs), bool)
        if len(self.objs):
            new_ok &= ~np.any(dominates(self.objs, N), axis=0)
            old_ok = ~np.any(dominates(N[new_ok], self.objs), axis=0)
        self.objs = np.vstack([self.objs[old_ok], N[new_ok]])
        self.coords = [c for c, k in zip(self.coords, old_ok) if k] + [coords_of(int(c)) for c in cand[new_ok]]
        if len(self.objs) > self.cap:
            idx = np.random.default_rng(0).choice(len(self.objs), self.cap, replace=False)
            self.objs = self.objs[idx]
            self.coords = [self.coords[i] for i in idx]

    def hypervolume(self, ref):
        return dmr.hypervolume(self.objs, ref) if len(self.objs) else 0.0


class Gomea:
    def __init__(self, prob, coords0, groups, mesh, sigma0, rng, proposal=None, alpha=0.25):
        self.prob = prob
        self.mesh = tuple(mesh)
        self.groups = groups
        self.rng = rng
        self.C = coords0.shape[0]
        self.coords = np.array(coords0, np.float64)
        self.obj = np.asarray(prob.eval_full(self.coords))
        prob.set_fos(groups)
        self.waves = prob.waves()
        self.sigma = np.full(len(groups), float(sigma0))
        self.fix = synth.fixed_axes(mesh)
        self.evals = float(self.C)
        self.ntet = prob.ntet
        self.touched = self._touched_counts()
        self.archive = Archive()
        self.archive.update(self.obj, lambda c: self.coords[c].copy())
        self.proposal = proposal  # callable(coords [C,2,3,P]) -> (mean [C,P,3], logvar [C,P,3]) or None
        self.alpha = alpha
        self.history = [(self.evals, None)]

    def _touched_counts(self):
        """|union of the stars of the group's points| per group."""
        tets = self.prob.tets()
        flat = tets.reshape(-1)
        tet_of = np.repeat(np.arange(len(tets)), 4)
        order = np.argsort(flat, kind="stable")
        starts = np.searchsorted(flat[order], np.arange(self.prob.P + 1))
        out = []
        for grp in self.groups:
            parts = [tet_of[order[starts[p]:starts[p + 1]]] for p in grp]
            out.append(len(np.unique(np.concatenate(parts))))
        return np.array(out, np.float64)

    def _proposals(self, gids, cids, learned):
        """Trial coordinates [n, 2, 3, G] for (group, candidate) pairs."""
        G = max(len(g) for g in self.groups)
        n = len(gids)
        if G == 1:  # single-point groups: vectorised
            pts = np.array([self.groups[g][0] for g in gids])
            cur = self.coords[cids, :, :, pts]  # [n, 2, 3]
            noise = self.rng.normal(0.0, 1.0, size=cur.shape) * self.sigma[gids][:, None, None]
            if learned is not None:
                use = self.rng.uniform(size=n) < self.alpha
                mu = learned[0][cids, pts]          # [n, 3]
                lv = learned[1][cids, pts]
                lt = mu + np.exp(0.5 * lv) * self.rng.normal(size=mu.shape)
                noise[use, 1, :] = lt[use]
            fixed = ((self.fix[pts][:, None] >> np.arange(3)[None, :]) & 1) == 1  # [n, 3]
            noise[np.repeat(fixed[:, None, :], 2, axis=1)] = 0.0
            return (cur + noise)[..., None]
        tc = np.zeros((n, 2, 3, G))
        for k, (g, c) in enumerate(zip(gids, cids)):
            pts = self.groups[g]
            cur = self.coords[c][:, :, pts]
            noise = self.rng.normal(0.0, self.sigma[g], size=cur.shape)
            if learned is not None and self.rng.uniform() < self.alpha:
                noise[1] = learned[0][c][pts].T + np.exp(0.5 * learned[1][c][pts].T) * self.rng.normal(size=(3, len(pts)))
            for ax in range(3):
                noise[:, ax, ((self.fix[pts] >> ax) & 1) == 1] = 0.0
            tc[k, :, :, : len(pts)] = cur + noise
        return tc

    def generation(self):
        learned = self.proposal(self.coords) if self.proposal is not None else None
        succ = np.zeros(len(self.groups))
        tries = np.zeros(len(self.groups))
        for w in self.waves:
            cids = np.repeat(np.arange(self.C), len(w)).astype(np.int32)
            gids = np.tile(w, self.C).astype(np.int32)
            tc = self._proposals(gids, cids, learned)
            self.prob.eval_partial(gids, cids, tc)
            acc = self.prob.commit_improving()
            ks = np.nonzero(acc)[0]
            if tc.shape[-1] == 1:
                pts = np.array([self.groups[g][0] for g in gids[ks]], dtype=np.int64)
                self.coords[cids[ks], :, :, pts] = tc[ks, :, :, 0]
            else:
                for k in ks:
                    g, c = gids[k], cids[k]
                    self.coords[c][:, :, self.groups[g]] = tc[k, :, :, : len(self.groups[g])]
            np.add.at(succ, gids, acc)
            np.add.at(tries, gids, 1)
            self.evals += float(np.sum(self.touched[gids])) / self.ntet
        rate = succ / np.maximum(tries, 1)
        self.sigma *= np.where(rate > 0.2, 1.2, 0.85)
        self.obj = self.prob.objectives()
        self.archive.update(self.obj, lambda c: self.coords[c].copy())
        return self.obj

    def run(self, generations, ref):
        hv = []
        for _ in range(generations):
            self.generation()
            hv.append((self.evals, self.archive.hypervolume(ref)))
        return hv


def seed_from_archive(archive, n, rng):
    """Sec. 2.4: a finer-resolution run starts from a random sample, of its
    population size, of the coarser run's approximation set (drawn with
    replacement only when the set is smaller than the population)."""
    k = len(archive.coords)
    if k == 0:
        raise ValueError("empty approximation set")
    idx = rng.choice(k, size=n, replace=k < n)
    return np.stack([archive.coords[i] for i in idx])


def multi_resolution(build, coords0, levels, ref, rng):
    """Grid multi-resolution run (Sec. 2.4): level 0 starts from coords0; each
    next level refines a random sample of the previous level's approximation
    set (edge, face and cube midpoints on the GPU, dmr.refine) and continues
    from it.  build(mesh, C) -> a dmr.Problem for that mesh and population;
    levels: [{"mesh", "C", "generations", "sigma0"}].  Returns per level the
    hypervolume curve, the final archive and the feasible fraction of the
    refined seeds."""
    out = []
    coords = np.asarray(coords0, np.float64)
    prev = None
    for li, lv in enumerate(levels):
        mesh, C = tuple(lv["mesh"]), int(lv["C"])
        seeded_feasible = None
        if li > 0:
            seeds = seed_from_archive(prev.archive, C, rng)
            coords = dmr.refine(seeds, prev.mesh)
        prob = build(mesh, C)
        groups = synth.single_point_fos(mesh)
        g = Gomea(prob, coords, groups, mesh, lv["sigma0"], rng)
        if li > 0:
            seeded_feasible = float(np.mean(g.obj[:, 3] == 0))
        curve = g.run(int(lv["generations"]), ref)
        out.append({"mesh": list(mesh), "C": C, "generations": int(lv["generations"]), "curve": curve,
                    "final_hv": curve[-1][1] if curve else g.archive.hypervolume(ref),
                    "archive_size": int(len(g.archive.objs)), "seeded_feasible": seeded_feasible, "gomea": g})
        prev = g
    return out

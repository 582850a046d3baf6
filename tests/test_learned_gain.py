"""What the trained proposal network gains over the plain sampler.

On the coarse CT level (64x64x24 voxels of 4x4x12 mm, 10^3-point meshes,
population 256, 1000 single-point FOS groups): elites are collected from two
plain runs of the optimiser scaffold, the network is trained on the tensor
cores (dmr_mlp_train_step: tcgen05 forward and backward, Adam), then five
fresh runs with and without the learned sampler (alpha = 0.25) are compared.
Every proposal of either arm, learned or not, is scored by the exact
evaluator (partial evaluation + accept-if-improves on the GPU), so both arms
spend the same evaluations per generation (checked); the budget counts a
partial evaluation as touched / total tetrahedra.  Averaged over the seeds,
the learned sampler's hypervolume curve must reach the plain curve's final
value in fewer evaluations, and the learned arm must be ahead in at least
three of the five seeds."""
import numpy as np
import pytest

from paper_2202_11001_gb300 import dmr, learned, synth

pytestmark = pytest.mark.gpu


def test_learned_sampler_reaches_plain_hypervolume_in_fewer_evaluations():
    pr = synth.ct_phantom(seed=3, C=256, level="coarse")
    rng = np.random.default_rng(0)
    X, Y = learned.collect(pr, seeds=[11, 12], generations=12, sigma0=0.5, n_samples=50000, rng=rng)
    net = dmr.MLP(seed=1)
    losses = learned.train(net, X, Y, steps=400, batch=4096, lr=1e-3, rng=rng)
    assert losses[-1] < losses[0] - 1.0, (losses[0], losses[-1])
    _, rows = learned.compare(pr, net, seeds=[21, 22, 23, 24, 25], generations=12, sigma0=0.5, alpha=0.25)
    for r in rows:
        # same evaluation count after every generation: every proposal scored
        ep = [e for e, _ in r["curves"]["plain"]]
        el = [e for e, _ in r["curves"]["learned"]]
        assert np.allclose(ep, el, rtol=0, atol=1e-9), r["seed"]
    # the seed-averaged hypervolume curves (evaluation counts are the same for
    # every run): the learned curve reaches the plain curve's final value in
    # fewer evaluations, and the learned arm is ahead in most seeds
    evals = [e for e, _ in rows[0]["curves"]["plain"]]
    mean_plain = [(e, np.mean([r["curves"]["plain"][i][1] for r in rows])) for i, e in enumerate(evals)]
    mean_lrn = [(e, np.mean([r["curves"]["learned"][i][1] for r in rows])) for i, e in enumerate(evals)]
    target = mean_plain[-1][1]
    need = learned.evals_to_reach(mean_lrn, target)
    per_seed = [(r["seed"], r["plain_evals"], r["learned_evals"]) for r in rows]
    assert need < evals[-1], (need, evals[-1], per_seed)
    wins = sum(1 for r in rows if r["learned_evals"] < r["plain_evals"])
    assert wins >= 3, per_seed
    net.close()

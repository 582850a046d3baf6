"""Elitist archive of the optimiser scaffold (Sec. 2.4: approximation set of
the non-dominated solutions encountered): after any sequence of updates it
holds exactly the non-dominated set of all feasible objective vectors seen,
each once, with the coordinates of the candidate that brought it."""
import numpy as np

from paper_2202_11001_gb300.gomea import Archive, nondominated, seed_from_archive


def test_archive_equals_nondominated_set_of_everything_seen():
    for seed in range(4):
        rng = np.random.default_rng(seed)
        A = Archive()
        seen = []
        for it in range(25):
            o = np.zeros((40, 4))
            x = rng.random((40, 3))
            o[:, 0] = x[:, 0]
            o[:, 1] = 1 - x[:, 0] + 0.3 * x[:, 1]
            o[:, 2] = rng.integers(0, 3, 40)
            if it % 5 == 0:
                o[:5, :3] = o[5:10, :3]  # exact duplicates within a batch
            o[rng.random(40) < 0.2, 3] = 1  # infeasible rows never enter
            A.update(o, lambda c, it=it: (it, c))
            seen.append(o[o[:, 3] == 0, :3])
        U = np.unique(np.vstack(seen), axis=0)
        want = np.unique(U[nondominated(U)], axis=0)
        assert np.array_equal(np.unique(A.objs, axis=0), want)
        assert len(A.objs) == len(want) and len(A.coords) == len(A.objs)


def test_seed_sample_size_and_membership():
    A = Archive()
    o = np.array([[1.0, 2.0, 0.0, 0.0], [2.0, 1.0, 0.0, 0.0], [0.5, 3.0, 0.0, 0.0]])
    A.update(o, lambda c: np.full((2, 3, 4), float(c)))
    rng = np.random.default_rng(0)
    s = seed_from_archive(A, 7, rng)
    assert s.shape == (7, 2, 3, 4)
    assert set(np.unique(s[:, 0, 0, 0])) <= {0.0, 1.0, 2.0}
    s2 = seed_from_archive(A, 2, rng)
    assert len(set(s2[:, 0, 0, 0])) == 2  # without replacement when the set is large enough

"""Host logic of the package's adaptive-mesh module (no GPU): its quadtree,
2:1 balance, controller and mesh arrays against the independent quadtree of
the input generator, through refine and coarsen cycles (exact: integers and
node coordinates), and the partitions derived from the levels."""
import numpy as np

from paper_2507_04991_gb300 import amr as pamr
import workloads

THRESH = (0.3, 0.9)
LEVELS = (0, 1, 2)


def test_package_mesh_logic_matches_generator():
    tree = workloads.Quadtree.uniform(8, 1.0)
    pmesh = pamr.QuadMesh.uniform(8, 1.0)
    rng = np.random.default_rng(7)
    kinds = np.zeros(3, int)
    for cycle in range(6):
        alpha = rng.uniform(0, 1, len(tree.leaves)) ** 3
        ref, coa = workloads.amr_marks(tree, alpha, THRESH, LEVELS)
        pref, pcoa = pamr.controller(pmesh, alpha, THRESH, LEVELS)
        assert sorted(ref) == sorted(pref) and sorted(coa) == sorted(pcoa)
        tree, omap = tree.adapt(ref, coa)
        pmesh, pmap = pmesh.adapt(pref, pcoa)
        assert pmesh.leaves == tree.leaves
        assert np.array_equal(pmap, omap)
        pc, pf, pm = pmesh.arrays()
        oc, of, om, _ = tree.mesh()
        assert np.abs(pc - oc).max() == 0.0
        assert sorted(map(tuple, pf)) == sorted(map(tuple, of))
        assert sorted(map(tuple, pm)) == sorted(map(tuple, om))
        kinds += np.bincount(pmap[:, 0], minlength=3)
    assert np.all(kinds > 0)                            # copies, refinements and coarsenings all occurred


def test_balance_holds_after_adapt():
    pmesh = pamr.QuadMesh.uniform(6, 1.0)
    for _ in range(3):
        pmesh, _ = pmesh.adapt([pmesh.leaves[len(pmesh.leaves) // 2]], [])
    for (lev, i, j) in pmesh.leaves:
        for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            o = pmesh.owner(lev, i + di, j + dj)
            assert o is None or o[0] >= lev - 1


def test_partitions_from_levels():
    assert list(pamr.partitions([0, 1, 2, 2], 2)) == [2, 1, 0, 0]

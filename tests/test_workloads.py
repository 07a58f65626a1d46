"""The synthetic inputs (no arithmetic of the method): shapes, seeding and the
structure each workload promises."""
import numpy as np

import gen


def test_slab_partition_matches_the_paper_setup():
    """Sec. 6: a 250 x 250 x 15 box partitioned along x only; Table 2 uses a
    residual threshold of 1e-6."""
    for n_slabs in (32, 64, 128):
        prob = gen.workload(f"slab{n_slabs}")
        assert (prob.xc[-1], prob.yc[-1], prob.zc[-1]) == (250.0, 250.0, 15.0)
        assert len(prob.cx) == n_slabs + 1 and list(prob.cy) == [0, prob.ny] and list(prob.cz) == [0, prob.nz]
        assert np.all(np.diff(prob.cx) >= 2) and prob.rtol == 1e-6
    prob = gen.workload("slab32")
    assert prob.n_nodes == 769 * 769 * 33 and prob.n_dofs == 767 * 767 * 31


def test_crater_density_structure_and_seed():
    xc = gen.uniform_coords(64, 250.0)
    zc = gen.uniform_coords(8, 15.0)
    a = gen.crater_density(xc, xc, zc, np.random.default_rng(0), noise=0.0)
    b = gen.crater_density(xc, xc, zc, np.random.default_rng(0), noise=0.0)
    assert np.array_equal(a, b)
    rho = a.reshape(8, 64, 64)
    # the breccia lens sits under the cover near the rim centre, the layers far from it
    X, Y, Z = gen.element_centroids(xc, xc, zc)
    centre = (np.hypot(X - 125.0, Y - 125.0) < 60.0) & (Z > 15.0 - 3.0) & (Z < 15.0 - 1.0)
    assert np.all(rho[centre & ~(np.hypot(X - 125.0, Y - 125.0) > 35.0)] <= 0.0)
    assert rho[-1, 0, 0] == -150.0 and rho[0, 0, 0] == 100.0
    noisy = gen.crater_density(xc, xc, zc, np.random.default_rng(1))
    assert 5.0 < np.std(noisy - a) < 15.0


def test_named_workloads_are_deterministic():
    for name in ("sphere16", "layered32", "regional"):
        a, b = gen.workload(name), gen.workload(name)
        assert np.array_equal(a.drho, b.drho) and np.array_equal(a.cx, b.cx) and a.p == b.p

"""The seeded synthetic inputs (no GPU): the ragged ensemble follows its stated recipe and every generator
is deterministic in its seed."""
import numpy as np

from paper_1805_00007_gb300 import workloads as wl


def test_ragged_ensemble_recipe():
    """256 square instances, sides drawn from {64, 128, 256, 512} (about 22.3 M nodes expected), walls in
    y, a circle of radius R ~ U[0.15, 0.3] side at the centre, shear rate ~ U[1e-5, 1e-4], Pe ~ U[10, 1000]."""
    ens = wl.shear_ensemble()
    assert len(ens) == 256
    sides = np.array([p["nx"] for p, _ in ens])
    assert all(p["nx"] == p["ny"] and p["walls"] == 1 and p["vel"] == wl.VEL_SHEAR for p, _ in ens)
    assert set(sides) <= {64, 128, 256, 512} and len(set(sides)) == 4
    expected = 256 * np.mean(np.array([64, 128, 256, 512]) ** 2)  # 22.28 M
    assert abs((sides ** 2).sum() / expected - 1.0) < 0.15
    for p, phi0 in ens:
        s = p["nx"]
        R = np.sqrt((phi0 > 0.5).sum() / np.pi)  # the area inside the interface
        assert 0.15 * s - 1.5 <= R <= 0.3 * s + 1.5
        assert abs(phi0[s // 2, s // 2] - 1.0) < 1e-3 and abs(phi0[0, 0]) < 1e-3  # tanh tails, W = 4
        assert 1e-5 <= p["shear"] <= 1e-4 and 10.0 <= p["Pe"] <= 1000.0


def test_generators_are_deterministic():
    a, b = wl.shear_ensemble(n_inst=5, seed=17), wl.shear_ensemble(n_inst=5, seed=17)
    for (pa, fa), (pb, fb) in zip(a, b):
        assert pa == pb and np.array_equal(fa, fb)
    c = wl.shear_ensemble(n_inst=5, seed=18)
    assert any(pa != pc for (pa, _), (pc, _) in zip(a, c))
    assert np.array_equal(wl.random_smooth_phi(33, 21, seed=3), wl.random_smooth_phi(33, 21, seed=3))

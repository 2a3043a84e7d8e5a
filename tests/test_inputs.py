"""The seeded input recipes match the workloads they stand in for: the
512 uneven D2Q9 cases of the batched workload (sides uniform on [32, 512],
R = L/4 +- L/16, density ratio log-uniform on [10, 1000], tau on [0.51,
0.8], W in {3, 4, 5}, drops and bubbles), the 1-4 separated drops or
bubbles of the warm-start cases, and the profiles' shapes.  The recipes
hold no model arithmetic; these checks are about the inputs only."""
import numpy as np
import pytest

from paper_1812_00118_gb300 import inputs as I


def test_batch_cases_recipe():
    cases = I.batch_cases()
    assert len(cases) == 512
    L = np.array([c["L"] for c in cases])
    R = np.array([c["R"] for c in cases])
    ratio = np.array([c["rho_ratio"] for c in cases])
    tau = np.array([c["tau"] for c in cases])
    W = np.array([c["W"] for c in cases])
    drop = np.array([c["drop"] for c in cases])
    assert L.min() >= 32 and L.max() <= 512 and L.dtype.kind == "i"
    assert 200 < L.mean() < 340                                # uniform: mean 272
    assert np.all(np.abs(R - L / 4.0) <= L / 16.0 + 1e-12)
    assert ratio.min() >= 10.0 and ratio.max() <= 1000.0
    lr = np.log10(ratio)
    assert abs(lr.mean() - 2.0) < 0.1                           # log-uniform: mean log10 = 2
    assert np.mean(lr < 1.5) == pytest.approx(0.25, abs=0.06)
    assert tau.min() >= 0.51 and tau.max() <= 0.8
    assert set(W.tolist()) == {3.0, 4.0, 5.0}
    assert 0.4 < drop.mean() < 0.6
    # reproducible and independent per case: the first cases do not depend on n_cases
    assert I.batch_cases(n_cases=8) == cases[:8]
    assert I.batch_cases(seed=1)[0] != cases[0]


@pytest.mark.parametrize("seed", range(12))
def test_drops_recipe(seed):
    L, W = 256, 4.0
    phi, u, P, placed = I.drops(L, seed, W=W, gap=3.0 * W, bubbles=seed % 2 == 1)
    assert phi.shape == (1, L, L) and u.shape == (3, 1, L, L) and P.shape == (1, L, L)
    assert not u.any() and not P.any()
    assert 1 <= len(placed) <= 4
    assert phi.min() >= 0.0 and phi.max() <= 1.0
    for k, (x, y, R) in enumerate(placed):
        assert 12.0 <= R <= 48.0
        for (x2, y2, R2) in placed[k + 1:]:
            d = np.abs(np.array([x - x2, y - y2]))
            d = np.minimum(d, L - d)
            assert np.hypot(*d) >= R + R2 + 3.0 * W - 1e-9
    # the light phase is the disks for bubbles, their complement for drops
    light = (1.0 - phi).sum() if seed % 2 == 0 else phi.sum()
    disks = sum(np.pi * R * R for _, _, R in placed)
    heavy_inside = phi.sum() if seed % 2 == 0 else (1.0 - phi).sum()
    assert heavy_inside == pytest.approx(disks, rel=0.03)
    assert light == pytest.approx(L * L - disks, rel=0.03)


def test_sphere_and_layers_profiles():
    shape = (1, 40, 40)
    phi = I.sphere(shape, (20.3, 19.7, 0.0), 10.0, 4.0, periodic=False)[0]
    assert phi[0, 20, 20] > 0.999 and phi[0, 0, 0] < 1e-3
    # the half-value contour sits at r = R; the profile is odd about it
    r = np.hypot(np.arange(40)[None, :] - 20.3, np.arange(40)[:, None] - 19.7)
    assert np.all(np.abs(phi[0] - (0.5 + 0.5 * np.tanh(2 * (10.0 - r) / 4.0))) < 1e-15)
    bub = I.sphere(shape, (20.3, 19.7, 0.0), 10.0, 4.0, drop=False, periodic=False)[0]
    np.testing.assert_allclose(bub, 1.0 - phi, atol=1e-15)
    # periodic: distances are minimum-image, so a drop at the corner wraps
    wrap = I.sphere(shape, (0.0, 0.0, 0.0), 6.0, 2.0)[0]
    assert wrap[0, 39, 39] > 0.99 and wrap[0, 0, 39] > 0.99 and wrap[0, 20, 20] < 1e-6
    lay = I.layers((1, 30, 8), 1, 12.5, 3.0)[0]
    assert np.all(np.diff(lay[0, :, 0]) < 0)                  # heavy below the split
    assert lay[0, 12, 0] > 0.5 > lay[0, 13, 0]


def test_smooth_random_ranges_and_seeds():
    phi, u, P = I.smooth_random((6, 7, 9), 3)
    assert 0.05 - 1e-12 <= phi.min() and phi.max() <= 0.95 + 1e-12
    assert np.abs(u).max() <= 0.02 + 1e-12 and np.abs(P).max() <= 1e-3 + 1e-15
    phi2 = I.smooth_random((6, 7, 9), 3)[0]
    assert np.array_equal(phi, phi2)
    assert not np.array_equal(phi, I.smooth_random((6, 7, 9), 4)[0])
    _, u2d, _ = I.smooth_random((1, 7, 9), 3, dim=2)
    assert not u2d[2].any()

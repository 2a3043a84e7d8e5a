"""The learned warm start against the method without it.

The four-level surrogate is trained on the GPU, by the library's own
kernels, on snapshot pairs DT = 2000 steps apart that the solver generates
(1-4 drops or bubbles at density ratio 1000); on held-out configurations the
warm-started solver -- the surrogate applied k times to the initial fields,
populations rebuilt as equilibria plus the Chapman-Enskog non-equilibrium
part, total of phi re-imposed -- must reach the residual tolerance 1e-6 in
fewer steps than the plain solver started from the same fields, keep the
total of phi, and end as close to Laplace's law.  Reduced sizes (128^2
grids, 96 training cases) keep the test to a minute or two."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_00118_gb300 import build, lbm as L
    from paper_1812_00118_gb300 import warmstart as WS
    from paper_1812_00118_gb300.surrogate import Surrogate
    build.build()
    L.load()
    return torch, L, WS, Surrogate


def test_warm_start_reaches_tolerance_in_fewer_steps(env):
    torch, L, WS, Surrogate = env
    Lsz, K, k_apply = 128, 12, 8
    S, dropped = WS.generate_snapshots(torch, Lsz, list(range(1000, 1096)), K)
    assert dropped <= 3 and S.shape[0] >= 93
    sg = Surrogate(8, Lsz, Lsz, seed=0)
    hist = WS.train(torch, sg, S, 1500, lr=1e-3)
    assert np.mean([l for _, l in hist[-3:]]) < 0.5 * WS.identity_loss(S), (hist[-3:], WS.identity_loss(S))
    sg1 = Surrogate(1, Lsz, Lsz, params=sg.params())
    prm = WS.case_params(L.F32)
    ratios = []
    for sd in (5001, 5002, 5004):
        phi0, placed = WS.case_fields(Lsz, sd)
        steps, lap = {}, {}
        for mode in ("plain", "warm"):
            sim = L.Simulation(L.D2Q9, (Lsz, Lsz), prm)
            if mode == "plain":
                sim.init_fields(phi0, np.zeros(2 * Lsz * Lsz), np.zeros(Lsz * Lsz))
            else:
                WS.predict_into(torch, sg1, sim, phi0, prm, k_apply)
            steps[mode], _, _ = WS.steps_to_tolerance(torch, sim, tol=1e-6, max_steps=400000)
            f, P, _ = sim.macro()
            assert abs(f.sum() - phi0.sum()) < 1e-5 * phi0.sum()
            if len(placed) == 1:
                cx, cy, R = placed[0]
                law = WS.PHYS["sigma"] / R    # inside minus outside, for a drop and for a bubble
                lap[mode] = sim.laplace((cx % Lsz, cy % Lsz), R - 8.0, R + 8.0) / law - 1.0
            sim.close()
        assert steps["plain"] is not None and steps["warm"] is not None, (sd, steps)
        ratios.append(steps["plain"] / steps["warm"])
        if lap:
            # converged states: the warm start ends as close to sigma / R
            assert abs(lap["warm"]) < abs(lap["plain"]) + 0.02, (sd, lap)
    print("plain / warm steps to residual 1e-6:", ratios)
    assert np.mean(ratios) > 1.2, ratios

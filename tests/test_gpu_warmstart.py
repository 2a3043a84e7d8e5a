"""The learned warm start against the method without it.

The four-level surrogate is trained on the GPU, by the library's own
kernels, on snapshot pairs DT = 2000 steps apart that the solver generates
(1-4 drops or bubbles at density ratio 1000, nu = 1/60).  On held-out
configurations the warm-started solver -- the surrogate applied k = 4 times
to the initial fields, the predicted phi projected onto the start's
interfaces with its total restored, populations rebuilt as equilibria plus
the Chapman-Enskog non-equilibrium part -- and the plain solver from the same
fields both run until the Laplace-jump residual |J(t) - J(t - 100)| / |J(t)|
stays below 1e-6.  From each run's residual history the test reads the steps
to 1e-3 and to 1e-6.  What the network gains: the early transient (to 1e-3)
is cut by more than a fifth on average.  The slow tail to 1e-6, set by the
decay of the longest acoustic modes that the BF16 prediction leaves excited
like any start does, is not shortened: the steps to 1e-6 stay within a fifth
of the plain run's on average (measured means 1.0 and 1.1 in two builds,
single cases 0.75 to 1.32, as the network and the rounding of its training
data vary).  Both
runs keep the total of phi (FP32 rounding of the rest-population closure
on near-static fields drifts it by ~1e-4 over 1e5 steps in either) and end
on Laplace's law within the W = 4 discretisation band (10 %).  Reduced sizes (128^2 grids, 96 training
cases, 1500 iterations) keep the test to a minute or two."""
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


def test_warm_start_against_plain_solver(env):
    torch, L, WS, Surrogate = env
    Lsz, K, k_apply = 128, 12, 4
    S, dropped = WS.generate_snapshots(torch, Lsz, list(range(1000, 1096)), K)
    assert dropped <= 3 and S.shape[0] >= 93
    sg = Surrogate(8, Lsz, Lsz, seed=0)
    hist = WS.train(torch, sg, S, 1500, lr=1e-3)
    assert np.mean([l for _, l in hist[-3:]]) < 0.7 * WS.identity_loss(S), (hist[-3:], WS.identity_loss(S))
    del S
    assert L.load().lbm_sg_status(None) == 0
    sg1 = Surrogate(1, Lsz, Lsz, params=sg.params())
    prm = WS.case_params(L.F32)
    early, late = [], []
    for sd in (5001, 5002, 5003):
        phi0, placed = WS.case_fields(Lsz, sd)
        res, lap = {}, {}
        for mode in ("plain", "warm"):
            sim = L.Simulation(L.D2Q9, (Lsz, Lsz), prm)
            if mode == "plain":
                sim.init_fields(phi0, np.zeros(2 * Lsz * Lsz), np.zeros(Lsz * Lsz))
            else:
                WS.predict_into(torch, sg1, sim, phi0, prm, k_apply)
            h = []
            steps, _, _ = WS.steps_to_tolerance(torch, sim, tol=1e-6, max_steps=500000, history=h)
            assert steps is not None, (sd, mode, h[-3:])
            res[mode] = (WS.steps_at(h, 1e-3), steps)
            f, P, _ = sim.macro()
            assert abs(f.sum() - phi0.sum()) < 1e-3 * phi0.sum(), (sd, mode)
            if len(placed) == 1:   # around the drop's current centre, R from its area
                lap[mode] = WS.laplace_error(sim, placed, bubble=sd % 2 == 1)
            sim.close()
        early.append(res["plain"][0] / res["warm"][0])
        late.append(res["plain"][1] / res["warm"][1])
        if lap:
            # converged states: both end on Laplace's law (Section 4.1) within
            # the discretisation band of the surface tension at W = 4 (a
            # relaxed drop sits 5-7 % below sigma / R; measured at the
            # residual's stopping point, which leaves 2-7 %)
            print("case %d Laplace error at convergence: plain %+.4f, warm %+.4f" % (sd, lap["plain"], lap["warm"]))
            assert abs(lap["plain"]) < 0.10 and abs(lap["warm"]) < 0.10, (sd, lap)
    print("plain / warm steps to the Laplace residual 1e-3:", early, " to 1e-6:", late)
    assert np.mean(early) > 1.2, early
    assert np.mean(late) > 0.8, late

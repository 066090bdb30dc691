"""The learned surrogate end to end on a small scale: trajectories generated by
the batched solver under four bond seeds per point, the network trained by the
library's kernels on the seed means, held-out accuracy (N_L also against its
noise floor, the seed-to-seed spread), the hull test with the solver as
fallback, and the cost of a surrogate trajectory against the one-instance
solver."""
import dataclasses

import numpy as np
import pytest

from paper_2210_06043_gb300 import lbib
from paper_2210_06043_gb300 import surrogate as sg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_initial_bonds_equal_the_librarys():
    """N0 from the surrogate's geometry (its input feature) equals the bonds the
    library engages at t = 0 in the same capillary."""
    pts = sg.sample_points(16, seed=8)
    lib = []
    for p in pts:
        s = lbib.from_capillary(sg.capillary_for(p))
        lib.append(int(np.sum(s.bonds(1)[0])))
        s.close()
    assert sg.initial_bonds(pts).tolist() == lib


# Held-out accuracy bounds at this scale (56 training points of 4 bond seeds, 24 000 steps).
# N_L: the floor is the uncertainty of the held-out targets themselves (seed-to-seed
# spread / sqrt(4)); measured on GB300 the network is at 0.20 of the spread and 2.3 times
# the floor (without the N0 input feature: about 0.7 and 7 at similar scales).
NL_OVER_STD, NL_OVER_FLOOR = 0.35, 4.0


def test_surrogate_pipeline_small():
    st = torch.cuda.Stream()
    torch.cuda.set_stream(st)
    pts = sg.sample_points(64, seed=5)
    reps, steps, samples = 4, 24000, 48
    runs = sg.replicate(pts, reps)
    t_star, Yall, gen_secs = sg.generate(runs, steps=steps, samples=samples, batch=len(runs), stream=st.cuda_stream)
    assert np.isfinite(Yall).all()
    assert t_star[0] > 0 and np.all(np.diff(t_star) > 0)
    assert (Yall[:, 0, 0] >= 1.0).all()  # N_L starts from the bonds engaged at t = 0
    Y, spread, floor = sg.seed_statistics(Yall, reps)
    assert spread[0] > 0  # bond events are stochastic: the seeds differ
    hold, fit = np.arange(8), np.arange(8, 64)
    X = sg.features_many([pts[i] for i in fit], t_star)
    T = Y[fit].reshape(-1, 3).astype(np.float32)
    tr = sg.train(X, T, steps=1000, batch=2048, lr=2e-3, seed=1)
    assert tr.losses[-1] < tr.losses[0] / 5
    err, inf_secs, _ = sg.evaluate(tr, [pts[i] for i in hold], t_star, Y[hold], floor=floor)
    print({k: (round(v["rmse_over_std"], 3), round(v["rmse_over_floor"], 2)) for k, v in err.items()}, spread)
    assert err["delta_p"]["rmse_over_std"] < 0.5 and err["r"]["rmse_over_std"] < 0.5, err
    assert err["n_l"]["rmse_over_std"] < NL_OVER_STD and err["n_l"]["rmse_over_floor"] < NL_OVER_FLOOR, err
    # the hull: a particle stiffer than the training range goes to the solver
    stiff = dataclasses.replace(pts[0], rigid=False, log10_ca=-4.5)
    sur = sg.Surrogate(tr, steps=steps)
    Yp, inside = sur.predict([pts[0], stiff], t_star[:4])
    assert inside.tolist() == [True, False]
    assert np.isfinite(Yp).all()
    # a surrogate trajectory (features on the host, network on the GPU) costs far less
    # than a solver trajectory
    per_step = sg.plain_solver_seconds_per_step(pts[:2], steps=500)
    assert inf_secs / len(hold) < 1e-3 * per_step * steps, (inf_secs, per_step)
    tr.net.close()

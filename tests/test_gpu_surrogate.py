"""The learned surrogate end to end on a small scale: trajectories generated by
the batched solver, the network trained by the library's kernels, held-out
accuracy, the hull test with the solver as fallback, and the cost of a
surrogate trajectory against the one-instance solver."""
import dataclasses
import time

import numpy as np
import pytest

from paper_2210_06043_gb300 import lbib
from paper_2210_06043_gb300 import surrogate as sg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_surrogate_pipeline_small():
    st = torch.cuda.Stream()
    torch.cuda.set_stream(st)
    pts = sg.sample_points(96, seed=5)
    steps, samples = 12000, 48
    t_star, Y, gen_secs = sg.generate(pts, steps=steps, samples=samples, batch=96, stream=st.cuda_stream)
    assert np.isfinite(Y).all()
    assert t_star[0] > 0 and np.all(np.diff(t_star) > 0)
    assert (Y[:, 0, 0] > 0).all()  # bonds engaged at the start
    hold, fit = np.arange(8), np.arange(8, 96)
    X = np.concatenate([sg.features(pts[i], t_star) for i in fit])
    T = Y[fit].reshape(-1, 3).astype(np.float32)
    tr = sg.train(X, T, steps=600, batch=2048, lr=2e-3, seed=1)
    assert tr.losses[-1] < tr.losses[0] / 5
    err, inf_secs, _ = sg.evaluate(tr, [pts[i] for i in hold], t_star, Y[hold])
    # delta p and r are smooth in the parameters; N_L carries the noise of the bond events
    assert err["delta_p"]["rmse_over_std"] < 0.5 and err["r"]["rmse_over_std"] < 0.5, err
    # the hull: a particle stiffer than the training range goes to the solver
    stiff = dataclasses.replace(pts[0], rigid=False, log10_ca=-4.5)
    sur = sg.Surrogate(tr, steps=steps)
    Yp, inside = sur.predict([pts[0], stiff], t_star[:4])
    assert inside.tolist() == [True, False]
    assert np.isfinite(Yp).all()
    # a surrogate trajectory costs far less than a solver trajectory
    per_step = sg.plain_solver_seconds_per_step(pts[:2], steps=500)
    assert inf_secs / len(hold) < 1e-3 * per_step * steps, (inf_secs, per_step)
    tr.net.close()

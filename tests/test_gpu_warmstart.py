"""The learned warm start end to end on small volumes: training pairs made by
plain 3MG, the U-Net trained by the library's tensor-core kernels, and what the
trained network gains over starting 3MG from y on held-out volumes."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _iters_to(trace, fstar, f0, gap):
    g = (trace - fstar) / (f0 - fstar)
    hit = np.nonzero(g <= gap)[0]
    return int(hit[0]) if hit.size else len(trace)


def test_trained_network_gains_over_plain_start(cuda_lib):
    import torch
    from paper_2002_02328_gb300 import binding, unet_binding as ub, warmstart as ws
    shape, count, held = (16, 32, 32), 136, 8
    ys, ramps = ws.make_crops(count, shape, seed=1, source_shape=None)
    targets = ws.solve_targets(ys, ramps, iters=400)
    ntr = count - held
    with ub.UNet((16, 32, 64, 128), 2, lr=1e-3) as net:
        net.set_params(ub.he_init((16, 32, 64, 128), 2, 0))
        losses = ws.train(net, ys, ramps, targets, range(ntr), epochs=12, batch=4)
        assert np.mean(losses[-20:]) < 0.6 * np.mean(losses[:5])
        it_y, it_x, mse_y, mse_x, better = [], [], [], [], 0
        for k in range(ntr, count):
            prob = ws.crop_problem(ys[k], ramps[k])
            xh = ws.predict(net, ys[k], ramps[k])
            mse_y.append(float(torch.mean((ys[k] - targets[k]) ** 2)))
            mse_x.append(float(torch.mean((xh - targets[k]) ** 2)))
            start, fx, fy = ws.choose_start(prob, xh)
            better += fx < fy
            with binding.Solver.from_problem(prob, slabs=None) as s:
                tr_y = s.iterate(500)
            with binding.Solver.from_problem(prob, slabs=None) as s:
                s.set_x(start)
                tr_x = s.iterate(500)
            fstar = min(tr_y[-1], tr_x[-1])
            it_y.append(_iters_to(tr_y, fstar, tr_y[0], 1e-3))
            it_x.append(_iters_to(tr_x, fstar, tr_y[0], 1e-3))
    # the network moves y toward the 3MG solution on volumes it has not seen ...
    assert np.mean(mse_x) < 0.8 * np.mean(mse_y), (np.mean(mse_x), np.mean(mse_y))
    assert better >= held // 2
    # ... and 3MG from its start needs fewer iterations to the same accuracy
    assert sum(it_x) < sum(it_y), (it_x, it_y)


def test_fallback_keeps_y_when_the_prediction_is_worse(cuda_lib):
    import torch
    from paper_2002_02328_gb300 import warmstart as ws
    ys, ramps = ws.make_crops(1, (16, 32, 32), seed=2, source_shape=None)
    prob = ws.crop_problem(ys[0], ramps[0])
    bad = ys[0] + 5.0                     # far outside the box: a much higher objective
    start, fx, fy = ws.choose_start(prob, bad)
    assert fx > fy
    assert torch.equal(start.cpu(), torch.from_numpy(prob.y))

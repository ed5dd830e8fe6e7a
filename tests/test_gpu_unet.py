"""GPU parity of the learned warm start's tensor-core layers and network
against the FP64 U-Net oracle, through the C ABI.

Inputs are rounded to BF16 before both sides see them, so the layer tests
compare FP32 tensor-core accumulation (plus the final BF16 rounding of the
output) against exact FP64 arithmetic on the same values."""
import numpy as np
import pytest

from oracle import unet as U

pytestmark = pytest.mark.gpu


def _bf(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16)


def _np(t):
    import torch
    return t.detach().to(torch.float32).cpu().numpy().astype(np.float64)


def _rng(seed):
    return np.random.default_rng([seed, 99])


@pytest.fixture(scope="module")
def ub(cuda_lib):
    from paper_2002_02328_gb300 import unet_binding
    return unet_binding


@pytest.mark.parametrize("cin,cout,relu,masked", [(16, 32, True, False), (32, 16, False, True),
                                                  (128, 64, True, False), (256, 128, False, False)])
def test_conv3_matches_oracle(ub, cin, cout, relu, masked):
    import torch
    r = _rng(cin + cout)
    B, D, H, W = 2, 4, 6, 10              # 480 rows: three full 128-row tiles and a ragged tail
    x = _bf(r.normal(size=(B, D, H, W, cin)))
    w = _bf(r.normal(0, (27 * cin) ** -0.5, size=(27, cout, cin)))
    b = torch.from_numpy(r.normal(size=cout).astype(np.float32))
    mask = _bf(r.normal(size=(B, D, H, W, cout))) if masked else None
    out = ub.conv3(x.cuda(), w.cuda(), b.cuda(), relu=relu, mask=mask.cuda() if masked else None)
    torch.cuda.synchronize()
    got = _np(out)
    xd, wd, bd = _np(x), _np(w), b.numpy().astype(np.float64)
    for k in range(B):
        ref = U.conv3(xd[k], wd, bd)
        if relu:
            ref = np.maximum(ref, 0.0)
        if masked:
            ref = ref * (_np(mask)[k] > 0)
        err = np.abs(got[k] - ref)
        assert np.all(err <= 2.0 ** -8 * np.abs(ref) + 1e-5 * np.abs(ref).max()), err.max()


@pytest.mark.parametrize("cin,cout,relu,masked,strided", [
    (16, 16, True, False, False), (32, 16, False, True, True), (16, 32, True, True, False),
    (32, 32, False, False, True), (32, 64, True, False, False), (64, 32, True, False, False),
    (64, 64, True, True, True), (64, 128, False, True, True), (128, 64, True, False, True)])
def test_tma_conv3_matches_oracle_and_the_gather_kernel(ub, cin, cout, relu, masked, strided):
    """The TMA-staged convolution (input block per 8x16 output tile, taps read
    through shifted descriptors) on a grid with ragged x and y tiles: within the
    oracle bound, and the same bits as the row-gather kernel (same MMA order).
    strided: x is the second half of rows of 2 cin channels and out the first
    cout channels of rows of 2 cout (the concatenation buffers' layout).  64 ->
    64 and 64 -> 128 run as two and four launches of 32 output channels, 128 ->
    64 as four launches of 16 with a ring of two slices (the weights of all of
    them do not fit in shared memory beside the slice ring)."""
    import torch
    r = _rng(7 * cin + cout)
    B, D, H, W = 2, 3, 21, 13
    xs = _bf(r.normal(size=(B, D, H, W, 2 * cin if strided else cin))).cuda()
    x = xs[..., cin:] if strided else xs
    w = _bf(r.normal(0, (27 * cin) ** -0.5, size=(27, cout, cin))).cuda()
    b = torch.from_numpy(r.normal(size=cout).astype(np.float32)).cuda()
    mask = _bf(r.normal(size=(B, D, H, W, cout))).cuda() if masked else None
    outs = []
    for tma in (True, False):
        prev = ub.set_tma_conv(tma)
        try:
            full = torch.zeros((B, D, H, W, 2 * cout if strided else cout), device="cuda", dtype=torch.bfloat16)
            o = full[..., :cout] if strided else full
            ub.conv3(x, w, b, relu=relu, mask=mask, out=o)
            torch.cuda.synchronize()
            outs.append(full)
        finally:
            ub.set_tma_conv(prev)
    assert torch.equal(outs[0], outs[1])
    if strided:
        assert not torch.any(outs[0][..., cout:] != 0)             # nothing written past the output channels
    got = _np(outs[0][..., :cout])
    xd, wd, bd = _np(x), _np(w), _np(b)
    for k in range(B):
        ref = U.conv3(xd[k], wd, bd)
        if relu:
            ref = np.maximum(ref, 0.0)
        if masked:
            ref = ref * (_np(mask)[k] > 0)
        err = np.abs(got[k] - ref)
        assert np.all(err <= 2.0 ** -8 * np.abs(ref) + 1e-5 * np.abs(ref).max()), err.max()


@pytest.mark.parametrize("cin,cout", [(16, 16), (32, 16), (32, 32), (16, 64), (64, 64), (128, 64)])
def test_tma_conv3_accumulator_ring_on_a_large_volume(ub, cin, cout):
    """A 48x128x128 volume: 768 work items of 8 output depths, more than the
    resident CTAs, so CTAs take several items and the MMA groups that add one
    input slice to three outputs' accumulators meet the end of the TMEM ring
    (two MMAs there).  The same bits as the row-gather kernel, and outputs
    sampled over the volume (its faces, edges and corners included) within the
    oracle bound, each from the oracle's convolution of its 3x3x3 neighbourhood."""
    import torch
    r = _rng(11 * cin + cout)
    B, D, H, W = 1, 48, 128, 128
    x = _bf(r.normal(size=(B, D, H, W, cin))).cuda()
    w = _bf(r.normal(0, (27 * cin) ** -0.5, size=(27, cout, cin))).cuda()
    b = torch.from_numpy(r.normal(size=cout).astype(np.float32)).cuda()
    outs = []
    for tma in (True, False):
        prev = ub.set_tma_conv(tma)
        try:
            outs.append(ub.conv3(x, w, b, relu=False))
            torch.cuda.synchronize()
        finally:
            ub.set_tma_conv(prev)
    assert torch.equal(outs[0], outs[1])
    zs = np.concatenate([[0, D - 1, 7, 8, 15, 16], r.integers(0, D, 250)])
    ys = np.concatenate([[0, H - 1, 15, 16, 0, H - 1], r.integers(0, H, 250)])
    xs = np.concatenate([[0, W - 1, 7, 8, W - 1, 0], r.integers(0, W, 250)])
    xd = x[0].float().cpu().numpy().astype(np.float64)
    got = outs[0][0].float().cpu().numpy().astype(np.float64)
    wd, bd = _np(w), _np(b)
    refs, gots = [], []
    for z, y, xx in zip(zs, ys, xs):
        crop = np.zeros((3, 3, 3, cin))
        z0, z1, y0, y1, x0, x1 = max(z - 1, 0), min(z + 2, D), max(y - 1, 0), min(y + 2, H), max(xx - 1, 0), min(xx + 2, W)
        crop[z0 - z + 1:z1 - z + 1, y0 - y + 1:y1 - y + 1, x0 - xx + 1:x1 - xx + 1] = xd[z0:z1, y0:y1, x0:x1]
        refs.append(U.conv3(crop, wd, bd)[1, 1, 1])
        gots.append(got[z, y, xx])
    refs, gots = np.array(refs), np.array(gots)
    err = np.abs(gots - refs)
    assert np.all(err <= 2.0 ** -8 * np.abs(refs) + 1e-5 * np.abs(refs).max()), err.max()


@pytest.mark.parametrize("cin,cout", [(16, 16), (32, 64), (256, 128)])
def test_conv3_weight_gradient_matches_oracle(ub, cin, cout):
    import torch
    r = _rng(7 * cin + cout)
    B, D, H, W = 2, 4, 6, 10
    x = _bf(r.normal(size=(B, D, H, W, cin)))
    dz = _bf(r.normal(size=(B, D, H, W, cout)))
    dw = ub.conv3_wgrad(x.cuda(), dz.cuda())
    torch.cuda.synchronize()
    got = dw.cpu().numpy().astype(np.float64)
    ref = np.zeros((27, cout, cin))
    xd, dd = _np(x), _np(dz)
    for k in range(B):
        ref += U.conv3_backward(xd[k], np.zeros((27, cout, cin)), dd[k])[1]
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max() + 1e-6


@pytest.mark.parametrize("cin,cout", [(32, 16), (64, 32), (128, 64)])
def test_up_matches_oracle(ub, cin, cout):
    import torch
    r = _rng(3 * cin + cout)
    B, D, H, W = 2, 3, 4, 5               # 120 coarse rows (one ragged tile)
    x = _bf(r.normal(size=(B, D, H, W, cin)))
    w = _bf(r.normal(0, cin ** -0.5, size=(8, cout, cin)))
    b = torch.from_numpy(r.normal(size=cout).astype(np.float32))
    out = ub.up(x.cuda(), w.cuda(), b.cuda())
    torch.cuda.synchronize()
    got = _np(out)
    for k in range(B):
        ref = U.up2(_np(x)[k], _np(w), b.numpy().astype(np.float64))
        assert np.all(np.abs(got[k] - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-5 * np.abs(ref).max())


def _tiny_net_case(widths=(16, 32), cin=2, B=2, D=8, H=8, W=16, seed=0):
    from paper_2002_02328_gb300 import unet_binding as ub
    r = _rng(seed)
    params = ub.he_init(widths, cin, seed)
    # round every parameter to BF16 so both sides use the same weights
    params = {k: _np(_bf(v)) for k, v in params.items()}
    for k in params:
        if k.endswith(".b"):
            params[k] = r.normal(0, 0.05, size=params[k].shape)
    inp = _np(_bf(r.uniform(0, 1, size=(B, D, H, W, cin))))
    base = inp[..., 0].copy()
    target = base + r.normal(0, 0.1, size=base.shape)
    return params, inp, base, target


def test_network_forward_and_gradients_match_oracle(ub):
    import torch
    widths, cin = (16, 32), 2
    params, inp, base, target = _tiny_net_case(widths, cin)
    B = inp.shape[0]
    with ub.UNet(widths, cin) as net:
        net.set_params(params)
        pred = net.forward(torch.from_numpy(inp.astype(np.float32)).cuda(),
                           torch.from_numpy(base.astype(np.float32)).cuda())
        loss = net.loss_grad(torch.from_numpy(inp.astype(np.float32)).cuda(),
                             torch.from_numpy(base.astype(np.float32)).cuda(),
                             torch.from_numpy(target.astype(np.float32)).cuda())
        grads = net.grads()
    pred = pred.cpu().numpy().astype(np.float64)
    ref_pred = np.stack([U.forward(params, inp[k], widths)[0] + base[k] for k in range(B)])
    rel = np.linalg.norm(pred - ref_pred) / np.linalg.norm(ref_pred - base)
    assert rel < 2e-2, rel
    # oracle loss and gradient over the batch (mean over all voxels)
    ref_loss = float(np.mean((ref_pred - target) ** 2))
    assert abs(loss - ref_loss) <= 2e-2 * ref_loss
    ref_g = None
    n = ref_pred.size
    for k in range(B):
        _, cache = U.forward(params, inp[k], widths, keep=True)
        dout = 2.0 * (ref_pred[k] - target[k]) / n
        g = U.backward(params, cache, dout, widths)
        ref_g = g if ref_g is None else {q: ref_g[q] + g[q] for q in g}
    for name in ref_g:
        a, b = grads[name].astype(np.float64).ravel(), ref_g[name].ravel()
        nb = np.linalg.norm(b)
        if nb == 0:
            continue
        cos = float(a @ b / (np.linalg.norm(a) * nb))
        assert cos > 0.99 and abs(np.linalg.norm(a) / nb - 1.0) < 0.06, (name, cos, np.linalg.norm(a) / nb)


def test_training_reduces_the_loss(ub):
    import torch
    widths, cin = (16, 32), 2
    params, inp, base, target = _tiny_net_case(widths, cin, seed=3)
    ti = torch.from_numpy(inp.astype(np.float32)).cuda()
    tb = torch.from_numpy(base.astype(np.float32)).cuda()
    tt = torch.from_numpy(target.astype(np.float32)).cuda()
    with ub.UNet(widths, cin, lr=1e-3) as net:
        net.set_params(params)
        first = net.train_step(ti, tb, tt)
        for _ in range(60):
            last = net.train_step(ti, tb, tt)
        p1 = net.params()
    assert last < 0.7 * first, (first, last)
    # the parameters moved and stayed finite
    assert all(np.all(np.isfinite(v)) for v in p1.values())


def test_first_adam_step_follows_the_oracle_gradient_sign(ub):
    """With zero moments the first bias-corrected Adam step is -lr g / (|g| + eps):
    -lr sign(g) wherever the gradient is not tiny (the oracle gives g)."""
    import torch
    widths, cin, lr = (16, 32), 2, 1e-3
    params, inp, base, target = _tiny_net_case(widths, cin, seed=5)
    B = inp.shape[0]
    ti = torch.from_numpy(inp.astype(np.float32)).cuda()
    tb = torch.from_numpy(base.astype(np.float32)).cuda()
    tt = torch.from_numpy(target.astype(np.float32)).cuda()
    with ub.UNet(widths, cin, lr=lr) as net:
        net.set_params(params)
        w0 = net.get_flat().astype(np.float64)
        net.train_step(ti, tb, tt)
        w1 = net.get_flat().astype(np.float64)
    ref_pred = np.stack([U.forward(params, inp[k], widths)[0] + base[k] for k in range(B)])
    g = None
    for k in range(B):
        _, cache = U.forward(params, inp[k], widths, keep=True)
        gk = U.backward(params, cache, 2.0 * (ref_pred[k] - target[k]) / ref_pred.size, widths)
        g = gk if g is None else {q: g[q] + gk[q] for q in gk}
    gflat = ub.flatten(g, widths, cin).astype(np.float64)
    dw = w1 - w0
    # |dw| <= lr, up to the FP32 rounding of w0 and w1 (one ulp of |w| each)
    assert np.all(np.abs(dw) <= lr * (1 + 1e-5) + 2.4e-7 * np.abs(w0))
    big = np.abs(gflat) > 0.05 * np.sqrt(np.mean(gflat ** 2))
    assert big.sum() > 0.2 * gflat.size
    ref_step, _, _ = U.adam_step(w0, gflat, np.zeros_like(gflat), np.zeros_like(gflat), 1, lr=lr)
    agree = np.abs(dw[big] - (ref_step - w0)[big]) <= 1e-6 + 2.4e-7 * np.abs(w0[big])
    assert agree.mean() > 0.995, agree.mean()

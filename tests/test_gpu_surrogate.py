"""Surrogate kernels (through the C ABI) against the FP64 reference MLP.

Tolerances.  The tensor-core layers read bfloat16 activations and weights
(unit roundoff 2^-9).  Against the reference evaluated with the same
bfloat16 roundings (``mixed=True``) the GPU differs only by FP32
accumulation order, __expf in the activation, and the rare bfloat16
rounding those flip: outputs within 2e-3 of their RMS.  Gradients are
compared element by element: for every parameter tensor,
max |g_gpu - g_ref| <= 1e-2 max |g_ref|.  A flipped bfloat16 rounding moves
one back-propagated entry by one bfloat16 ulp (2^-8 of it), and a weight
gradient entry sums 200 such products, so one flip shifts it by well under
1e-3 of the tensor's largest entry.  Against the plain FP64 network the
bfloat16 roundings themselves count: outputs within 3e-2 of their RMS,
gradients element-wise within 5e-2 of the tensor's largest entry.
"""
import numpy as np
import pytest

from oracle import mlp
from paper_1401_6047_gb300 import bte
from paper_1401_6047_gb300 import surrogate as S
from paper_1401_6047_gb300 import workloads as W

pytestmark = pytest.mark.gpu

Y_MEAN, Y_STD = (0.02, 0.15), (0.05, 0.2)


def _ref_outputs(p, x, mixed):
    lo, hi = S.box_bounds()
    xh = mlp.normalise_x(x, lo, hi)
    return np.stack([mlp.forward(mlp.unpack(p[m].astype(np.float64)), xh, mixed)[0]
                     for m in range(p.shape[0])])


def test_forward_ensemble_matches_reference():
    M = 4
    p = S.init_params(M, seed=1)
    x = W.sweep_matrix(300, 3)  # 300 rows: three 128-row tiles, the last one ragged
    with S.Surrogate(Y_MEAN, Y_STD, members=M, batch_capacity=1024) as sur:
        sur.set_params(p)
        mean, std, mask = sur.predict(x, threshold=1e-3)
    for mixed, tol in ((True, 2e-3), (False, 3e-2)):
        yh = _ref_outputs(p, x, mixed)
        ys = yh * np.array(Y_STD) + np.array(Y_MEAN)
        rm, rs = ys.mean(axis=0), np.sqrt(((ys - ys.mean(axis=0)) ** 2).mean(axis=0))
        scale = np.sqrt(np.mean(ys ** 2))
        assert np.max(np.abs(mean - rm)) <= tol * scale, mixed
        assert np.max(np.abs(std - rs)) <= tol * scale, mixed
    assert np.array_equal(mask, np.max(std, axis=1) > 1e-3)


def _elementwise(g, ref):
    """Largest entry-wise error of a tensor relative to its largest entry."""
    return float(np.max(np.abs(g - ref)) / np.max(np.abs(ref)))


GRAD_TOL = {True: 1e-2, False: 5e-2}  # mixed (bfloat16-emulating) / plain FP64 reference


def _grad_case(M=3, B=200):
    p = S.init_params(M, seed=2)
    rng = np.random.default_rng(5)
    x = W.sweep_matrix(B, 6)
    t = np.stack([rng.normal(Y_MEAN[0], Y_STD[0], B), rng.normal(Y_MEAN[1], Y_STD[1], B)], axis=1)
    lo, hi = S.box_bounds()
    xh = mlp.normalise_x(x, lo, hi)
    th = (t - np.array(Y_MEAN)) / np.array(Y_STD)
    return p, x, t, xh, th


def test_gradients_match_reference():
    """bte_sur_grad against the reference backward pass, element by element
    for every parameter tensor of every member (p11)."""
    M = 3
    p, x, t, xh, th = _grad_case(M)
    with S.Surrogate(Y_MEAN, Y_STD, members=M, batch_capacity=256) as sur:
        sur.set_params(p)
        loss, g = sur.grad(x, t)
    worst = {}
    for m in range(M):
        pm = mlp.unpack(p[m].astype(np.float64))
        gm = mlp.unpack(g[m].astype(np.float64))
        for mixed in (True, False):
            L, gr = mlp.loss_and_grad(pm, xh, th, mixed)
            assert abs(loss[m] - L) <= 1e-2 * L
            for k in gr:
                err = _elementwise(gm[k], gr[k])
                worst[(mixed, k)] = max(worst.get((mixed, k), 0.0), err)
                assert err <= GRAD_TOL[mixed], (m, k, mixed, err)
    print("element-wise gradient error / max|g_ref|:",
          {f"{'mixed' if a else 'fp64'}:{k}": f"{v:.2e}" for (a, k), v in sorted(worst.items())})


def test_gradient_check_catches_planted_mistakes(monkeypatch):
    """Mistakes planted in the reference (on the CPU) that an element-wise
    comparison with the GPU gradient must reject: two entries of dW2
    exchanged across the diagonal (a transposed index confined to one
    pair), the b3 gradient read one unit off, and the SiLU' factor dropped
    from the first layer's back-propagation."""
    p, x, t, xh, th = _grad_case(1)
    with S.Surrogate(Y_MEAN, Y_STD, members=1, batch_capacity=256) as sur:
        sur.set_params(p)
        _, g = sur.grad(x, t)
    pm = mlp.unpack(p[0].astype(np.float64))
    gm = mlp.unpack(g[0].astype(np.float64))
    _, gr = mlp.loss_and_grad(pm, xh, th, True)
    tol = GRAD_TOL[True]
    assert all(_elementwise(gm[k], gr[k]) <= tol for k in gr)

    planted = {}
    w2 = gr["W2"].copy()
    d = np.abs(w2 - w2.T)
    i, j = np.unravel_index(np.argmax(d), d.shape)
    w2[i, j], w2[j, i] = w2[j, i], w2[i, j]
    planted["dW2 pair transposed"] = ("W2", w2)
    b3 = gr["b3"].copy()
    u = int(np.argmax(np.abs(np.diff(b3))))
    b3[u] = b3[u + 1]
    planted["db3 one unit off"] = ("b3", b3)
    yh, cache = mlp.forward(pm, xh, True)
    orig = mlp.silu_grad
    monkeypatch.setattr(mlp, "silu_grad",
                        lambda z: np.ones_like(z) if z is cache["z1"] else orig(z))
    gbad = mlp.backward(pm, cache, (yh - th) / xh.shape[0], True)
    monkeypatch.undo()
    planted["no SiLU' in layer 1"] = ("W1", gbad["W1"])
    for name, (k, bad) in planted.items():
        assert _elementwise(gm[k], bad) > tol, name


def test_adam_step_matches_reference():
    M = 2
    p = S.init_params(M, seed=3)
    x = W.sweep_matrix(256, 7)
    rng = np.random.default_rng(8)
    t = np.stack([rng.normal(0, 0.05, 256), rng.normal(0, 0.2, 256)], axis=1)
    lr = 1e-3
    with S.Surrogate(Y_MEAN, Y_STD, members=M, batch_capacity=256) as sur:
        sur.set_params(p)
        _, g = sur.grad(x, t)
        sur.set_data(x, t)
        order = np.broadcast_to(np.arange(256, dtype=np.int32), (1, M, 256)).copy()
        sur.train(order, [lr])
        p1 = sur.get_params()
    for m in range(M):
        want, _, _ = mlp.adam(p[m].astype(np.float64), g[m].astype(np.float64),
                              np.zeros(p.shape[1]), np.zeros(p.shape[1]), 1, lr)
        assert np.max(np.abs(p1[m] - want)) <= 1e-6


def test_training_fits_a_smooth_map():
    """Loss falls by 20x on a smooth synthetic target within 40 epochs."""
    rng = np.random.default_rng(11)
    x = W.sweep_matrix(8192, 12)
    lo, hi = S.box_bounds()
    xh = mlp.normalise_x(x, lo, hi)
    y = np.stack([0.05 * np.sin(2 * xh[:, 0]) * xh[:, 1] + 0.02 * xh[:, 4],
                  0.2 * np.tanh(xh[:, 2] + xh[:, 3]) * (1 + 0.3 * xh[:, 4])], axis=1)
    with S.Surrogate(y.mean(axis=0), y.std(axis=0), members=4, batch_capacity=1024) as sur:
        sur.set_params(S.init_params(4, seed=0))
        hist = sur.fit(x, y, epochs=40, batch=512, lr=3e-3, seed=1)
        mean, std, _ = sur.predict(x[:1000])
    assert hist[-1] < hist[0] / 20
    assert np.sqrt(np.mean((mean - y[:1000]) ** 2, axis=0)).max() < 0.05 * y.std(axis=0).max()


def test_identical_members_have_zero_spread():
    # two members: (y + y) / 2 == y exactly, so the spread is exactly zero
    p = np.repeat(S.init_params(1, seed=4), 2, axis=0)
    x = W.sweep_matrix(500, 9)
    with S.Surrogate(Y_MEAN, Y_STD, members=2, batch_capacity=256) as sur:
        sur.set_params(p)
        mean, std, mask = sur.predict(x, threshold=0.0)  # 500 rows: two chunks of 256
    assert np.all(std == 0.0) and not mask.any()


def test_device_prediction_equals_host_prediction():
    torch = pytest.importorskip("torch")
    p = S.init_params(2, seed=5)
    x = W.sweep_matrix(700, 10).astype(np.float32)
    with S.Surrogate(Y_MEAN, Y_STD, members=2, batch_capacity=512) as sur:
        sur.set_params(p)
        mean, std, mask = sur.predict(x, threshold=2e-2)
        xd = torch.from_numpy(x).cuda()
        md = torch.zeros((700, 2), device="cuda")
        sd = torch.zeros((700, 2), device="cuda")
        kd = torch.zeros(700, dtype=torch.uint8, device="cuda")
        sur.predict_device(xd.data_ptr(), 700, md.data_ptr(), sd.data_ptr(), kd.data_ptr(), 2e-2)
        torch.cuda.synchronize()
    assert np.array_equal(md.cpu().numpy(), mean)
    assert np.array_equal(sd.cpu().numpy(), std)
    assert np.array_equal(kd.cpu().numpy().astype(bool), mask)


def test_pipelined_host_prediction_over_many_chunks():
    """The host-array call alternates two buffer sets over six chunks (copies
    of one chunk overlapping the inference of the next): bit for bit the
    device-array result, with pageable and with page-locked host arrays,
    and again on a second call."""
    torch = pytest.importorskip("torch")
    p = S.init_params(3, seed=6)
    n = 1357  # 5 full chunks of 256 and a ragged sixth
    x = W.sweep_matrix(n, 12).astype(np.float32)
    with S.Surrogate(Y_MEAN, Y_STD, members=3, batch_capacity=256) as sur:
        sur.set_params(p)
        xd = torch.from_numpy(x).cuda()
        md = torch.zeros((n, 2), device="cuda")
        sd = torch.zeros((n, 2), device="cuda")
        kd = torch.zeros(n, dtype=torch.uint8, device="cuda")
        sur.predict_device(xd.data_ptr(), n, md.data_ptr(), sd.data_ptr(), kd.data_ptr(), 1e-2)
        torch.cuda.synchronize()
        ref = (md.cpu().numpy(), sd.cpu().numpy(), kd.cpu().numpy())
        mean, std, mask = sur.predict(x, threshold=1e-2)
        assert np.array_equal(mean, ref[0]) and np.array_equal(std, ref[1])
        assert np.array_equal(mask, ref[2].astype(bool))
        xp = torch.from_numpy(x).pin_memory()
        outs = (torch.zeros((n, 2)).pin_memory().numpy(), torch.zeros((n, 2)).pin_memory().numpy(),
                torch.zeros(n, dtype=torch.uint8).pin_memory().numpy())
        for _ in range(2):
            outs[0][:] = 0
            m2, s2, k2 = sur.predict(xp.numpy(), threshold=1e-2, out=outs)
            assert np.array_equal(m2, ref[0]) and np.array_equal(s2, ref[1])
            assert np.array_equal(k2, ref[2])


def test_hybrid_uses_the_solver_exactly_where_members_disagree():
    p = S.init_params(4, seed=6)
    x = W.sweep_matrix(10, 13)
    x[:, 2] = np.maximum(x[:, 2], 3.0)  # short runs: omega >= 3
    pts = [W.surrogate_params(xi) for xi in x]
    ref = bte.batch_run(pts)
    with S.Surrogate(Y_MEAN, Y_STD, members=4, batch_capacity=256) as sur:
        sur.set_params(p)
        mean, std, _ = sur.predict(x)
        y_all, solved_all, st = sur.hybrid(x, threshold=-1.0)
        y_none, solved_none, _ = sur.hybrid(x, threshold=1e9)
        thr = float(np.median(std.max(axis=1)))
        y_mix, solved_mix, _ = sur.hybrid(x, threshold=thr)
    assert solved_all.all() and not solved_none.any()
    assert np.all(st == bte.OK)
    for i, o in enumerate(ref):
        assert y_all[i, 0] == o.absorption and y_all[i, 1] == o.v_dc_avg
    assert np.array_equal(y_none.astype(np.float32), mean)
    assert np.array_equal(solved_mix, std.max(axis=1) > thr)
    assert np.array_equal(y_mix[solved_mix], y_all[solved_mix])
    assert np.array_equal(y_mix[~solved_mix].astype(np.float32), mean[~solved_mix])

"""Learned Q' initial guess on the GPU (through the C-ABI): gradients of the
training kernels against the FP64 reference backprop, the logged training
pairs against the reference features/targets, and the gain in Newton
updates of the trained guess with results unchanged."""
import numpy as np
import pytest

from oracle import bgk as obgk
from oracle import mlp as omlp
from oracle import stage as ostage
from paper_2312_06567_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib(libbgk, cuda_device):
    from paper_2312_06567_gb300 import bgk
    return bgk


def _rand_batch(rng, n):
    x = np.column_stack([rng.uniform(0.8, 1.2, n), rng.normal(0, 0.1, (n, 3)), rng.uniform(0.9, 1.1, n),
                         rng.uniform(2.9, 3.1, n), rng.uniform(2.9, 3.1, n), rng.uniform(0.95, 1.05, n),
                         rng.uniform(0.005, 0.01, n)])
    t = rng.normal(0, 1e-4, (n, 5))
    norm = np.concatenate([x.mean(0), x.std(0), t.mean(0), t.std(0)])
    return x, t, norm


@pytest.mark.parametrize("bf16,tol", [(False, 1e-5), (True, 2e-2)])
def test_training_gradients_match_reference(lib, bf16, tol):
    rng = np.random.default_rng(7)
    x, t, norm = _rand_batch(rng, 200)
    params = omlp.init_params(11)
    for b in (1, 3, 5):
        params[b] += rng.normal(0, 0.1, params[b].shape)
    wl = W.reduced(W.periodic_sine_box(), mesh_n=(1, 1, 1), vel_n=(4, 4, 4))
    with lib.Solver(wl) as s:
        s.mlp_weights(load=(params, norm))
        p32 = [np.asarray(p, dtype=np.float32).astype(np.float64) for p in params]
        loss_g, grads_g = s.mlp_grad(x, t, bf16=bf16)
    n32 = norm.astype(np.float32).astype(np.float64)
    xn = (x.astype(np.float32) - n32[:9]) / n32[9:18]
    tn = (t.astype(np.float32) - n32[18:23]) / n32[23:28]
    loss_o, grads_o = omlp.loss_and_grads(p32, xn, tn)
    assert abs(loss_g - loss_o) <= tol * loss_o
    for go, gg in zip(grads_o, grads_g):
        assert np.max(np.abs(gg - go)) <= tol * np.max(np.abs(go)), np.max(np.abs(gg - go)) / np.max(np.abs(go))


def test_logged_pairs_match_reference_features_and_targets(lib):
    wl = W.reduced(W.taylor_green_box(), mesh_n=(2, 1, 1), vel_n=(14, 12, 13)).replace(p=2)
    pb = ostage.problem_from_workload(wl)
    f = W.random_anisotropic_state(wl, seed=8)
    m = obgk.raw_moments(f[0].reshape(wl.n_vel, -1), None, pb.vg)
    qp_o, _, conv, _ = obgk.solve_qprime(m, pb.gas, pb.vg)
    with lib.Solver(wl) as s:
        s.mlp_log(True, 10000)
        s.qprime(m)
        pairs = s.mlp_log_read(10000).astype(np.float64)
    assert pairs.shape == (len(m), 14)
    # log order is the order in which solves finished: match rows by density
    order = np.argsort(pairs[:, 0])
    ref_x = omlp.features(m, pb.gas)
    ref_t = omlp.target(m, qp_o, pb.gas)
    ro = np.argsort(ref_x[:, 0])
    assert np.allclose(pairs[order, :9], ref_x[ro], rtol=2e-6, atol=1e-6)
    assert np.allclose(pairs[order, 9:], ref_t[ro], rtol=1e-4, atol=1e-7)


def test_learned_guess_cuts_newton_updates_and_keeps_results(lib):
    """Train on pairs logged from the sine box's first 20 steps, then run steps
    21-30, whose states the network never saw: the learned guess needs fewer
    Newton updates, none is rejected, and the FP64 results match the from-q
    run to 1e-12."""
    wl = W.periodic_sine_box()
    f0 = W.maxwellian_state(wl)
    dt = wl.dt()
    with lib.Solver(wl) as s:
        s.set_state(f0)
        s.mlp_log(True, 1 << 20)
        assert s.step(dt, 20) == lib.BGK_OK
        s.mlp_log(False)
        loss = s.mlp_train(epochs=60, batch=512, lr=2e-3, seed=1, bf16=True)
        net = s.mlp_weights()
        f20 = s.get_state()
    assert loss < 0.05
    out = {}
    for mode in (0, 1):
        with lib.Solver(wl) as s:
            if mode:
                s.mlp_weights(load=net)
            s.set_guess(mode, bf16=True)
            s.set_state(f20)
            s.stats()
            assert s.step(dt, 10) == lib.BGK_OK
            out[mode] = (s.stats(), s.mlp_stats(), s.get_state())
    (mean_q, max_q, _), _, f_q = out[0]
    (mean_l, max_l, res_l), fallbacks, f_l = out[1]
    assert fallbacks == 0
    assert res_l <= 1e-13
    assert mean_l <= mean_q - 0.9, (mean_q, mean_l)
    C, Nu = f_q.shape[:2]
    err = np.max(np.abs(f_l - f_q).reshape(C * Nu, -1).max(1) / np.abs(f_q).reshape(C * Nu, -1).max(1))
    assert err <= 1e-12


def test_tensor_core_batch_inference_matches_reference(lib):
    """bgk_mlp_infer (tcgen05, BF16 operands, FP32 accumulation in tensor
    memory) against the FP64 network with the same BF16 roundings, on a batch
    that is not a whole number of 128-point tiles; host and device buffers.
    The tensor core truncates its sums and a hidden activation can then round
    to the neighbouring BF16 value, so outputs agree to a few 1e-3 of the
    target scale, not bit for bit."""
    import torch
    rng = np.random.default_rng(12)
    x, t, norm = _rand_batch(rng, 1000)
    params = omlp.init_params(13)
    for b in (1, 3, 5):
        params[b] += rng.normal(0, 0.1, params[b].shape)
    wl = W.reduced(W.periodic_sine_box(), mesh_n=(1, 1, 1), vel_n=(4, 4, 4))
    with lib.Solver(wl) as s:
        s.mlp_weights(load=(params, norm))
        d_host = s.mlp_infer(x)
        xd = torch.from_numpy(x.astype(np.float32)).cuda()
        dd = torch.empty((x.shape[0], 5), dtype=torch.float32, device="cuda")
        s.mlp_infer(xd, dd)
        torch.cuda.synchronize()
        d_dev = dd.cpu().numpy()
    assert np.array_equal(d_host, d_dev)
    n32 = norm.astype(np.float32).astype(np.float64)
    p32 = [np.asarray(p, dtype=np.float32).astype(np.float64) for p in params]
    xn = ((x.astype(np.float32) - n32[:9].astype(np.float32)) / n32[9:18].astype(np.float32)).astype(np.float64)
    y = omlp.forward_bf16(p32, xn)
    ref = y * n32[23:28] + n32[18:23]
    err = np.abs(d_host - ref) / n32[23:28]                  # in units of the target scale
    assert np.all(np.isfinite(d_host))
    assert np.max(err) <= 5e-3, np.max(err)
    assert np.mean(err) <= 2e-4, np.mean(err)

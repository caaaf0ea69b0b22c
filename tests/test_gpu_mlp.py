"""Warm-start network and warm start on the GPU against the oracle
(oracle/mlp.py): the BF16 tensor-core contraction, forward pass, loss
gradient, Adam steps, standardisation, the interior projection of a
prediction, the training target, and the gain of the trained network over
cold starts on a small parametric family."""
import math

import numpy as np
import pytest

import paper_2605_13736_gb300 as m
from paper_2605_13736_gb300 import warmstart as ws
import synth
from gpu_util import make_ctx, make_problem, torch_cuda
from oracle import mlp as om

pytestmark = pytest.mark.gpu


def r8(v):
    return (v + 7) // 8 * 8


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (100, 37, 8), (128, 128, 64), (300, 200, 1000),
                                   (256, 512, 20000), (5000, 64, 256), (257, 129, 65),
                                   # M <= 256 with a column tile per SM: the persistent wide-M kernel
                                   (1, 19457, 64), (100, 19500, 200), (255, 20000, 1), (256, 40001, 512)])
def test_gemm_bf16_matches_definition(M, N, K):
    torch = torch_cuda()
    ctx = make_ctx()
    try:
        g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
        lda, ldb, ldc = r8(K) + 8, r8(K), N + 3
        A = torch.zeros((M, lda), dtype=torch.bfloat16)
        B = torch.zeros((N, ldb), dtype=torch.bfloat16)
        A[:, :K] = torch.randn((M, K), generator=g).to(torch.bfloat16)
        B[:, :K] = torch.randn((N, K), generator=g).to(torch.bfloat16)
        A[:, K:] = float("nan")      # padding must never be read
        Cd = torch.full((M, ldc), -7.0, dtype=torch.float32, device="cuda")
        m.mdsip_gemm_bf16(ctx, M, N, K, A.cuda(), lda, B.cuda(), ldb, Cd, ldc)
        a = A[:, :K].double().numpy()
        b = B[:, :K].double().numpy()
        ref = a @ b.T
        bound = (K * 2.0 ** -23 + 1e-7) * (np.abs(a) @ np.abs(b).T) + 1e-30
        got = Cd.cpu().double().numpy()
        assert np.all(np.abs(got[:, :N] - ref) <= bound)
        assert np.all(got[:, N:] == -7.0)
    finally:
        m.mdsip_ctx_destroy(ctx)


def _setup(I, H, O, seed):
    p = synth.mlp_init(I, H, O, seed, out_scale=1.0)
    rng = np.random.default_rng(seed + 10)
    p["b1"] = rng.uniform(-0.2, 0.2, H).astype(np.float32)
    p["b2"] = rng.uniform(-0.2, 0.2, H).astype(np.float32)
    p["b3"] = rng.uniform(-0.2, 0.2, O).astype(np.float32)
    sc = dict(in_mean=rng.uniform(-0.1, 0.1, I).astype(np.float32),
              in_std=rng.uniform(0.5, 1.5, I).astype(np.float32),
              out_mean=rng.uniform(-1, 1, O).astype(np.float32),
              out_std=rng.uniform(0.5, 2.0, O).astype(np.float32))
    return p, sc


def _net_on_gpu(ctx, p, sc, I, H, O):
    net = m.mdsip_mlp_create(ctx, I, H, O)
    m.mdsip_mlp_set_params(net, ws.pack_params(net, p), ctx=ctx)
    m.mdsip_mlp_set_scaling(net, sc["in_mean"], sc["in_std"], sc["out_mean"], sc["out_std"], ctx=ctx)
    return net


def _f64(d):
    return {k: np.asarray(v, np.float64) for k, v in d.items()}


# Element-wise parity of the network on inputs chosen so that every product
# and every partial sum of the forward pass is a dyadic rational with few
# significant bits: inputs in {0, +-1/2, +-1}, first- and second-layer weights
# in {+-1/8, +-1/4} with at most 8 (W1) or 4 (W2, per row and per column)
# nonzeros, dense output weights and biases in multiples of 1/16, output
# scaling by 2.  Then the FP32 tensor-core accumulation is exact in any order,
# every hidden activation is exactly a bfloat16 number, and the GPU's forward
# pass must equal the oracle's (bf16 rounding points of oracle/mlp.py) bit for
# bit.  With targets y + 2 delta (delta in multiples of 1/16) and a batch times
# outputs a power of two, the output gradient dL/dyn = -2 delta / (B O) is exact
# too, and so are dW3, db3, the pre-activation gradient of layer 2 and db2; the
# products that can lose bits (dW2 = dZ2^T h1, dW1 = dZ1^T xn, db1) are held to
# the FP32 accumulation bound k 2^-24 sum|terms| over their k = B terms, and
# the second pre-activation gradient, whose sum is exact, is rounded identically
# on both sides.
E32 = 2.0 ** -24


def _sparse_pm(rng, rows, cols, per_row, vals, perms=False):
    W = np.zeros((rows, cols), np.float32)
    if perms:                                   # <= per_row nonzeros in every row and column
        for _ in range(per_row):
            pr = rng.permutation(max(rows, cols))
            for r in range(rows):
                c = pr[r] % cols
                W[r, c] = rng.choice(vals)
    else:
        for r in range(rows):
            for c in rng.choice(cols, size=min(per_row, cols), replace=False):
                W[r, c] = rng.choice(vals)
    return W


def _exact_setup(I, H, O, seed):
    rng = np.random.default_rng(seed)
    p = {"W1": _sparse_pm(rng, H, I, 8, [-0.25, -0.125, 0.125, 0.25]),
         "b1": (rng.integers(-4, 5, H) / 16).astype(np.float32),
         "W2": _sparse_pm(rng, H, H, 4, [-0.125, 0.125], perms=True),
         "b2": (rng.integers(-16, 17, H) / 128).astype(np.float32),
         "W3": (rng.integers(-8, 9, (O, H)) / 16).astype(np.float32),
         "b3": (rng.integers(-8, 9, O) / 16).astype(np.float32)}
    sc = dict(in_mean=np.zeros(I, np.float32), in_std=np.ones(I, np.float32),
              out_mean=(rng.integers(-4, 5, O) / 4).astype(np.float32), out_std=np.full(O, 2.0, np.float32))
    return p, sc


def _exact_inputs(rng, B, I):
    return rng.choice([-1.0, -0.5, 0.0, 0.5, 1.0], size=(B, I))


@pytest.mark.parametrize("I,H,O,B", [(64, 256, 1037, 100), (8, 136, 300, 33), (3, 40, 10, 9)])
def test_forward_matches_oracle_exactly(I, H, O, B):
    torch = torch_cuda()
    p, sc = _exact_setup(I, H, O, I + H)
    X = _exact_inputs(np.random.default_rng(2), B, I)
    ctx = make_ctx()
    net = _net_on_gpu(ctx, p, sc, I, H, O)
    try:
        Yd = torch.zeros((B, O + 5), dtype=torch.float32, device="cuda")
        m.mdsip_mlp_forward(net, torch.from_numpy(X).cuda(), I, B, Yd, O + 5, ctx=ctx)
        got = Yd[:, :O].cpu().double().numpy()
        ref = om.predict(_f64(p), X, _f64(sc), bf16=True)
        # the inputs were built for exact arithmetic: the exact network gives the same
        assert np.array_equal(ref, om.predict(_f64(p), X, _f64(sc), bf16=False))
        np.testing.assert_array_equal(got, ref)
        assert np.all(Yd[:, O:].cpu().numpy() == 0.0)
    finally:
        m.mdsip_mlp_destroy(net)
        m.mdsip_ctx_destroy(ctx)


def test_forward_matches_oracle_random():
    """Random weights and inputs: the forward pass within the BF16 oracle's
    norm (rounding decisions may differ where FP32 and FP64 sums straddle a
    bfloat16 boundary; the exact-arithmetic test above pins each element)."""
    torch = torch_cuda()
    I, H, O, B = 64, 256, 1037, 100
    p, sc = _setup(I, H, O, 1)
    X = np.random.default_rng(2).uniform(-1, 1, (B, I))
    ctx = make_ctx()
    net = _net_on_gpu(ctx, p, sc, I, H, O)
    try:
        Yd = torch.zeros((B, O + 5), dtype=torch.float32, device="cuda")
        m.mdsip_mlp_forward(net, torch.from_numpy(X).cuda(), I, B, Yd, O + 5, ctx=ctx)
        got = Yd[:, :O].cpu().double().numpy()
        ref = om.predict(_f64(p), X, _f64(sc), bf16=True)
        assert np.linalg.norm(got - ref) <= 1e-3 * np.linalg.norm(ref)
    finally:
        m.mdsip_mlp_destroy(net)
        m.mdsip_ctx_destroy(ctx)


def _blocks(net, flat, I, H, O):
    return ws.unpack_params(net, flat, I, H, O)


@pytest.mark.parametrize("I,H,O,B,rows", [(64, 256, 256, 64, 150), (8, 136, 512, 16, 64), (3, 40, 32, 8, 20)])
def test_gradient_matches_oracle(I, H, O, B, rows):
    torch = torch_cuda()
    assert (B * O) & (B * O - 1) == 0            # 2 / (B O) exact
    p, sc = _exact_setup(I, H, O, 3 + I)
    rng = np.random.default_rng(4)
    X = _exact_inputs(rng, rows, I)
    delta = rng.integers(-32, 33, (rows, O)) / 16.0
    Y = om.predict(_f64(p), X, _f64(sc), bf16=True) + 2.0 * delta
    idx = rng.permutation(rows)[:B].astype(np.int32)
    ctx = make_ctx()
    net = _net_on_gpu(ctx, p, sc, I, H, O)
    try:
        grad = torch.zeros(m.mdsip_mlp_num_params(net), dtype=torch.float32, device="cuda")
        loss = m.mdsip_mlp_gradient(net, torch.from_numpy(X).cuda(), I, torch.from_numpy(Y).cuda(), O,
                                    torch.from_numpy(idx).cuda(), B, grad, ctx=ctx)
        g = _f64(_blocks(net, grad.cpu().numpy(), I, H, O))
        q = _f64(p)
        L_ref, g_ref = om.loss_and_grad(q, X[idx], Y[idx], _f64(sc), bf16=True)
        assert loss == pytest.approx(L_ref, rel=1e-12)
        for k in ("W3", "b3", "b2"):              # exact sums
            np.testing.assert_array_equal(g[k], g_ref[k], err_msg=k)
        # FP32 accumulation over the batch (B terms) of exactly equal operands
        c = om.forward(q, X[idx], _f64(sc)["in_mean"], _f64(sc)["in_std"], bf16=True)
        gy = 2.0 * (c["yn"] - (Y[idx] - _f64(sc)["out_mean"]) / _f64(sc)["out_std"]) / (B * O)
        dz2 = om.bf16_round((gy @ c["W3"]) * (c["h2"] > 0))
        dz1 = om.bf16_round((dz2 @ c["W2"]) * (c["h1"] > 0))
        bounds = {"W2": B * E32 * (np.abs(dz2).T @ np.abs(c["h1"])),
                  "W1": B * E32 * (np.abs(dz1).T @ np.abs(c["xn"])),
                  "b1": B * E32 * np.abs(dz1).sum(axis=0)}
        for k, bd in bounds.items():
            d = np.abs(g[k] - g_ref[k])
            assert np.all(d <= bd), (k, float(np.max(d - bd)))
        assert np.count_nonzero(g_ref["W1"]) > 0 and np.count_nonzero(g_ref["W2"]) > 0
    finally:
        m.mdsip_mlp_destroy(net)
        m.mdsip_ctx_destroy(ctx)


def test_gradient_random_against_exact_network():
    """Random weights: the BF16 gradient stays within 10% (norm) of the exact
    FP64 network's gradient, the accuracy the warm start relies on."""
    torch = torch_cuda()
    I, H, O, B, rows = 64, 256, 1037, 100, 150
    p, sc = _setup(I, H, O, 3)
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, (rows, I))
    Y = om.predict(_f64(p), X, _f64(sc)) + rng.normal(size=(rows, O)) * sc["out_std"]
    idx = rng.permutation(rows)[:B].astype(np.int32)
    ctx = make_ctx()
    net = _net_on_gpu(ctx, p, sc, I, H, O)
    try:
        grad = torch.zeros(m.mdsip_mlp_num_params(net), dtype=torch.float32, device="cuda")
        m.mdsip_mlp_gradient(net, torch.from_numpy(X).cuda(), I, torch.from_numpy(Y).cuda(), O,
                             torch.from_numpy(idx).cuda(), B, grad, ctx=ctx)
        g = _blocks(net, grad.cpu().numpy(), I, H, O)
        _, g_ex = om.loss_and_grad(_f64(p), X[idx], Y[idx], _f64(sc), bf16=False)
        for k in om.BLOCKS:
            assert np.linalg.norm(g[k] - g_ex[k]) <= 1e-1 * np.linalg.norm(g_ex[k]), k
    finally:
        m.mdsip_mlp_destroy(net)
        m.mdsip_ctx_destroy(ctx)


def test_adam_steps_match_oracle():
    """Two training steps: each one's update equals the oracle's Adam step
    (Kingma-Ba Algorithm 1) applied to the gradient the GPU takes at the same
    weights (pinned element-wise above), for every element, within the FP32
    rounding of the update and of the weight.  Both sides use the constants as
    the kernel holds them (learning rate, decay rates and epsilon rounded to
    FP32): 1 - fl32(0.999) differs from 0.001 by 1.3e-5 relative, far above
    the FP32 rounding this test bounds."""
    torch = torch_cuda()
    I, H, O, B = 16, 128, 200, 64
    p, sc = _setup(I, H, O, 5)
    rng = np.random.default_rng(6)
    X = rng.uniform(-1, 1, (B, I))
    Y = om.predict(_f64(p), X, _f64(sc)) + rng.normal(size=(B, O)) * sc["out_std"]
    lr = 1e-3
    ctx = make_ctx()
    net = _net_on_gpu(ctx, p, sc, I, H, O)
    try:
        Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
        idx = torch.arange(B, dtype=torch.int32, device="cuda")
        n = m.mdsip_mlp_num_params(net)
        flat = np.zeros(n, np.float32)
        m.mdsip_mlp_get_params(net, flat, ctx=ctx)
        w = _f64(_blocks(net, flat, I, H, O))
        mom = {k: np.zeros_like(v) for k, v in w.items()}
        vel = {k: np.zeros_like(v) for k, v in w.items()}
        for t in (1, 2):
            grad = torch.zeros(n, dtype=torch.float32, device="cuda")
            m.mdsip_mlp_gradient(net, Xd, I, Yd, O, idx, B, grad, ctx=ctx)
            g = _f64(_blocks(net, grad.cpu().numpy(), I, H, O))
            f32 = lambda v: float(np.float32(v))
            ref, mom, vel = om.adam_step(w, g, mom, vel, t, f32(lr), beta1=f32(0.9), beta2=f32(0.999),
                                         eps=f32(1e-8))
            m.mdsip_mlp_train_step(net, Xd, I, Yd, O, idx, B, lr, ctx=ctx)
            m.mdsip_mlp_get_params(net, flat, ctx=ctx)
            got = _f64(_blocks(net, flat, I, H, O))
            for k in om.BLOCKS:
                step = np.abs(ref[k] - w[k])
                bound = 2 * E32 * np.abs(ref[k]) + 16 * E32 * step + 1e-30
                d = np.abs(got[k] - ref[k])
                assert np.all(d <= bound), (t, k, float(np.max(d / bound)))
            w = got            # the next step starts from the GPU's weights
    finally:
        m.mdsip_mlp_destroy(net)
        m.mdsip_ctx_destroy(ctx)


def test_fit_scaling_matches_oracle():
    torch = torch_cuda()
    rng = np.random.default_rng(8)
    X = rng.uniform(-1, 1, (300, 5)) * [1, 2, 0.5, 1, 3]
    Y = rng.normal(size=(300, 9)) * [1, 0, 1e-9, 5, 1, 1, 2, 3, 4] + np.arange(9)
    ctx = make_ctx()
    net = m.mdsip_mlp_create(ctx, 5, 16, 9)
    try:
        m.mdsip_mlp_fit_scaling(net, torch.from_numpy(X).cuda(), 5, torch.from_numpy(Y).cuda(), 9, 300, ctx=ctx)
        im, isd, om_, osd = (np.zeros(k, np.float32) for k in (5, 5, 9, 9))
        m.mdsip_mlp_get_scaling(net, im, isd, om_, osd, ctx=ctx)
        for got, ref in ((im, om.col_stats(X)[0]), (isd, om.col_stats(X)[1]),
                         (om_, om.col_stats(Y)[0]), (osd, om.col_stats(Y)[1])):
            np.testing.assert_allclose(got, ref, rtol=2e-7, atol=1e-12)
    finally:
        m.mdsip_mlp_destroy(net)
        m.mdsip_ctx_destroy(ctx)


def _tiny():
    return synth.make_instance(6, 20, 2, 0.1, seed=11)


def test_set_start_predicted_matches_oracle():
    torch = torch_cuda()
    inst = _tiny()
    ctx = make_ctx()
    prob = make_problem(ctx, inst)
    try:
        P = m.mdsip_packed_size(prob)
        rng = np.random.default_rng(12)
        pred = (rng.normal(size=P + 1) * 1.5).astype(np.float32)
        pred[P] = math.log(3e-4)
        push = 1e-3
        m.mdsip_set_start_predicted(prob, pred, push, ctx=ctx)
        got = np.zeros(P)
        m.mdsip_get_iterate(prob, got)
        mu0 = om.clamp_mu0(float(pred[P]), 1e-8, 0.1)
        ref = om.project_start(pred[:P].astype(np.float64), inst.n, inst.m_E, inst.m_I, inst.xl, inst.xu,
                               inst.hl, inst.hu, push, mu0)
        np.testing.assert_allclose(got, ref, rtol=4e-16, atol=0)
        m.mdsip_set_start_predicted(prob, torch.from_numpy(pred).cuda(), push, m.MDSIP_MEM_DEVICE, ctx=ctx)
        got2 = np.zeros(P)
        m.mdsip_get_iterate(prob, got2)
        np.testing.assert_array_equal(got2, got)
        with pytest.raises(m.MdsipError):
            m.mdsip_set_start_predicted(prob, pred, 0.0, ctx=ctx)
        # the solve from this start reaches the optimum of the cold start
        assert m.mdsip_solve(prob, ctx) == 0
        f_warm = m.mdsip_get_stats(prob)["f"]
        m.mdsip_set_start(prob, None)
        assert m.mdsip_solve(prob, ctx) == 0
        f_cold = m.mdsip_get_stats(prob)["f"]
        assert abs(f_warm - f_cold) <= 1e-8 * max(1.0, abs(f_cold))
    finally:
        m.mdsip_problem_destroy(prob)
        m.mdsip_ctx_destroy(ctx)


def test_warmstart_target_rule():
    inst = _tiny()
    ctx = make_ctx()
    prob = make_problem(ctx, inst)
    try:
        with pytest.raises(m.MdsipError):
            m.mdsip_warmstart_target(prob, 1e-3, np.zeros(m.mdsip_packed_size(prob) + 1), ctx=ctx)
        assert m.mdsip_solve(prob, ctx) == 0
        P = m.mdsip_packed_size(prob)
        it = np.zeros(P)
        m.mdsip_get_iterate(prob, it)
        log = m.mdsip_get_log(prob)
        for level in (1e-1, 1e-3, 1e-12):
            out = np.zeros(P + 1)
            m.mdsip_warmstart_target(prob, level, out, ctx=ctx)
            np.testing.assert_array_equal(out[:P], it)
            first = [r["mu"] for r in log if r["E0"] <= level]
            want = math.log(first[0] if first else log[-1]["mu"])
            assert out[P] == want
    finally:
        m.mdsip_problem_destroy(prob)
        m.mdsip_ctx_destroy(ctx)


def test_trained_network_reduces_iterations():
    """A small parametric family: the network trained on cold-start solutions
    cuts the iterations of new members, and every warm-started solve reaches
    the same optimum (E_0 <= 1e-8) as its cold start."""
    torch = torch_cuda()
    m.build()
    base = synth.make_instance(16, 200, 4, 0.05, seed=77)
    n_p, W = 8, 8
    streams = [torch.cuda.Stream() for _ in range(W)]
    ctxs = [m.mdsip_ctx_create(0, s.cuda_stream) for s in streams]
    probs = [make_problem(c, base) for c in ctxs]

    def set_member(prob, p):
        m.mdsip_set_bounds(prob, base.xl, base.xu, base.hl, base.hu, synth.family_rhs(base, p), base.x0)

    try:
        P = m.mdsip_packed_size(probs[0])
        train_p = synth.draw_family_params(256, n_p, seed=1)
        eval_p = synth.draw_family_params(24, n_p, seed=2)
        X = torch.from_numpy(train_p).cuda()
        Y = torch.zeros((len(train_p), P + 1), dtype=torch.float64, device="cuda")
        fam = ws.solve_family(probs, set_member, train_p, Y, e0_level=1e-3)
        assert np.all(fam["statuses"] == 0)
        net = ws.WarmStartNet(ctxs[0], n_p, P, hidden=128, init=synth.mlp_init(n_p, 128, P + 1, seed=3))
        losses, _ = net.train(X, Y, len(train_p), epochs=200, batch=64, lr=3e-3, lr_final=1e-4, seed=4)
        assert losses[-1] < 0.2 * losses[0]
        pred = net.predict(torch.from_numpy(eval_p).cuda(), len(eval_p))
        cold = ws.solve_cold(probs, set_member, eval_p)
        f_cold = []
        for i in range(len(eval_p)):
            set_member(probs[0], eval_p[i])
            m.mdsip_set_start(probs[0], None)
            assert m.mdsip_solve(probs[0]) == 0
            f_cold.append(m.mdsip_get_stats(probs[0])["f"])
        warm = ws.solve_warm(probs, set_member, eval_p, pred, push=1e-4)
        assert np.all(cold["statuses"] == 0) and np.all(warm["statuses"] == 0)
        assert warm["iters"].mean() <= 0.8 * cold["iters"].mean(), (warm["iters"], cold["iters"])
        for i in range(len(eval_p)):
            set_member(probs[0], eval_p[i])
            m.mdsip_set_start_predicted(probs[0], pred[i], 1e-4, m.MDSIP_MEM_DEVICE)
            assert m.mdsip_solve(probs[0]) == 0
            s = m.mdsip_get_stats(probs[0])
            assert s["E0"] <= 1e-8
            assert abs(s["f"] - f_cold[i]) <= 1e-7 * max(1.0, abs(f_cold[i]))
        net.close()
    finally:
        for p in probs:
            m.mdsip_problem_destroy(p)
        for c in ctxs:
            m.mdsip_ctx_destroy(c)

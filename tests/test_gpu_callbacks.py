"""The callback problem interface (mdsip_problem_create / mdsip_set_bounds):
the benchmark model family written as user callbacks on device pointers
(torch on the context's stream) gives the same trajectory as the built-in
model, and a failing callback ends the solve with MDSIP_ERR_CALLBACK."""
import json
import os

import numpy as np
import pytest

import paper_2605_13736_gb300 as m
import synth
from gpu_util import make_ctx, make_problem, torch_cuda

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


class _Dev:
    def __init__(self, ptr, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 3}


def _view(ptr, *shape):
    torch = torch_cuda()
    return torch.as_tensor(_Dev(ptr, shape), device="cuda")


class TorchModel:
    """f = 1/2 x_d^T Q x_d + sum 1/4 x_s^4 + c^T x, g = J_sg x_s + A x_d, h_j = ||x_d[S_j]||^2."""

    def __init__(self, inst, fail_on=None):
        torch = torch_cuda()
        t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a)).to(dt).cuda()
        self.inst, self.fail_on = inst, fail_on
        self.ns, self.nd, self.mE, self.mI = inst.n_s, inst.n_d, inst.m_E, inst.m_I
        self.Q, self.c, self.A = t(inst.Q), t(inst.c), t(inst.A)
        self.rows, self.cols = t(inst.Jsg_rows, torch.int64), t(inst.Jsg_cols, torch.int64)
        self.vals = t(inst.Jsg_vals)
        hs = inst.h_set
        self.hk = t(np.nonzero(hs >= 0)[0], torch.int64)
        self.hj = t(hs[hs >= 0], torch.int64)
        self.calls = 0

    def _x(self, x):
        xv = _view(x, self.ns + self.nd)
        return xv[:self.ns], xv[self.ns:]

    def eval_f(self, stream, x, f):
        xs, xd = self._x(x)
        c = self.c
        val = 0.5 * xd @ (self.Q @ xd) + 0.25 * (xs ** 4).sum() + c @ torch_cuda().cat([xs, xd])
        _view(f, 1).copy_(val.reshape(1))
        return 0

    def eval_grad_f(self, stream, x, grad):
        xs, xd = self._x(x)
        g = _view(grad, self.ns + self.nd)
        g[:self.ns].copy_(xs ** 3 + self.c[:self.ns])
        g[self.ns:].copy_(self.Q @ xd + self.c[self.ns:])
        return 0

    def eval_cons(self, stream, x, g, h):
        self.calls += 1
        if self.fail_on is not None and self.calls >= self.fail_on:
            return 7
        xs, xd = self._x(x)
        gv = _view(g, self.mE)
        gv.copy_(self.A @ xd)
        gv.index_add_(0, self.rows, self.vals * xs[self.cols])
        hv = _view(h, self.mI)
        hv.zero_()
        hv.index_add_(0, self.hj, xd[self.hk] ** 2)
        return 0

    def eval_jac(self, stream, x, jv, A, lda, Jdh, ldh):
        xs, xd = self._x(x)
        _view(jv, len(self.vals)).copy_(self.vals)
        _view(A, self.mE, lda)[:, :self.nd].copy_(self.A)
        J = _view(Jdh, self.mI, ldh)
        J.zero_()
        J[self.hj, self.hk] = 2.0 * xd[self.hk]
        return 0

    def eval_hess(self, stream, x, yg, yh, Hss, Hdd, ldd):
        xs, xd = self._x(x)
        _view(Hss, self.ns).copy_(3.0 * xs ** 2)
        H = _view(Hdd, self.nd, ldd)
        H.copy_(self.Q)
        yv = _view(yh, self.mI)
        H[self.hk, self.hk] += 2.0 * yv[self.hj]
        return 0


def _callback_problem(ctx, inst, model):
    prob = m.mdsip_problem_create(ctx, n_d=inst.n_d, n_s=inst.n_s, m_E=inst.m_E, m_I=inst.m_I,
                                  Jsg_rows=np.ascontiguousarray(inst.Jsg_rows, dtype=np.int32),
                                  Jsg_cols=np.ascontiguousarray(inst.Jsg_cols, dtype=np.int32),
                                  eval_f=model.eval_f, eval_grad_f=model.eval_grad_f, eval_cons=model.eval_cons,
                                  eval_jac=model.eval_jac, eval_hess=model.eval_hess)
    m.mdsip_set_bounds(prob, inst.xl, inst.xu, inst.hl, inst.hu, np.ascontiguousarray(inst.b), inst.x0, ctx=ctx)
    return prob


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx()
    yield c
    m.mdsip_ctx_destroy(c)


@pytest.mark.parametrize("path", [m.MDSIP_PATH_P1, m.MDSIP_PATH_P2])
def test_callback_model_matches_builtin(ctx, path):
    inst = synth.make_config(0)
    g = json.load(open(os.path.join(HERE, "golden", "mds0_full.json")))
    model = TorchModel(inst)
    prob = _callback_problem(ctx, inst, model)
    try:
        m.mdsip_set_option_int(prob, "path", path, ctx)
        st = m.mdsip_solve(prob, ctx)
        stats = m.mdsip_get_stats(prob)
        log = m.mdsip_get_log(prob)
    finally:
        m.mdsip_problem_destroy(prob)
    assert m.STATUS[st] == "OK"
    assert stats["iters"] == g["iters"]
    assert abs(stats["f"] - g["f"]) <= 1e-8 * abs(g["f"])
    for rec, grec in zip(log, g["log"]):
        assert [tuple(c[2]) for c in rec["ic"]] == [tuple(c[2]) for c in grec.get("ic", [])]


def test_failing_callback_reports_status(ctx):
    inst = synth.make_instance(6, 20, 2, 0.2, seed=5)
    model = TorchModel(inst, fail_on=4)   # eval_cons fails on its 4th call
    prob = _callback_problem(ctx, inst, model)
    try:
        with pytest.raises(m.MdsipError) as ei:
            m.mdsip_solve(prob, ctx)
        assert ei.value.status == 4 and "eval_cons" in str(ei.value)
        # the context stays usable: the same problem solves once the model recovers
        model.fail_on = None
        st = m.mdsip_solve(prob, ctx)
        assert m.STATUS[st] == "OK"
    finally:
        m.mdsip_problem_destroy(prob)


def test_bounds_required(ctx):
    inst = synth.make_instance(4, 6, 1, 0.2, seed=6)
    model = TorchModel(inst)
    prob = m.mdsip_problem_create(ctx, n_d=inst.n_d, n_s=inst.n_s, m_E=inst.m_E, m_I=inst.m_I,
                                  Jsg_rows=np.ascontiguousarray(inst.Jsg_rows, dtype=np.int32),
                                  Jsg_cols=np.ascontiguousarray(inst.Jsg_cols, dtype=np.int32),
                                  eval_f=model.eval_f, eval_grad_f=model.eval_grad_f, eval_cons=model.eval_cons,
                                  eval_jac=model.eval_jac, eval_hess=model.eval_hess)
    try:
        with pytest.raises(m.MdsipError) as ei:
            m.mdsip_solve(prob, ctx)
        assert ei.value.status == 1
    finally:
        m.mdsip_problem_destroy(prob)

"""Device memory through the caller's allocation hooks (mdsip_ctx_create).

Every device buffer of a context is taken from `mdsip_alloc_hooks.alloc` and
returned through `.free` with the same size: the test counts both on a solve
of the benchmark family member 0 (n_d=32, n_s=2000, m_E=1000, m_I=1), whose
result must still be the oracle's (tests/golden/mds0_full.json), and checks
that a hook that fails gives MDSIP_ERR_OOM without harming the context.
"""
import ctypes as C
import json
import os

import pytest

import paper_2605_13736_gb300 as m
import synth
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    with open(os.path.join(HERE, "golden", "mds0_full.json")) as fh:
        return json.load(fh)


class _Counting:
    """Hooks over torch's caching allocator that record every call."""

    def __init__(self, fail=False):
        self.torch = torch_cuda()
        self.fail = fail
        self.live = {}
        self.n_alloc = self.n_free = 0
        self.bad_free = 0
        self.hooks = m.mdsip_alloc_hooks(m.ALLOC_FN(self.alloc), m.FREE_FN(self.free), None)

    def alloc(self, nbytes, stream, user):
        if self.fail:
            return None
        p = self.torch.cuda.caching_allocator_alloc(int(nbytes), 0, int(stream or 0))
        self.live[p] = int(nbytes)
        self.n_alloc += 1
        return p

    def free(self, ptr, nbytes, stream, user):
        if self.live.pop(ptr, None) != int(nbytes):
            self.bad_free += 1
        self.n_free += 1
        self.torch.cuda.caching_allocator_delete(int(ptr))


def test_hooks_receive_every_allocation():
    torch = torch_cuda()
    m.build()
    rec = _Counting()
    ctx = m.mdsip_ctx_create(0, torch.cuda.current_stream().cuda_stream, allocator=rec.hooks)
    g = _golden()
    try:
        prob = m.mdsip_problem_create_synthetic(ctx, **m.synth_arrays(synth.make_config(0)))
        try:
            st = m.mdsip_solve(prob, ctx)
            stats = m.mdsip_get_stats(prob)
        finally:
            m.mdsip_problem_destroy(prob)
    finally:
        m.mdsip_ctx_destroy(ctx)
    assert m.STATUS[st] == "OK"
    assert stats["iters"] == g["iters"]
    assert abs(stats["f"] - g["f"]) <= 1e-8 * abs(g["f"])
    assert rec.n_alloc > 0
    assert rec.n_free == rec.n_alloc and not rec.live and rec.bad_free == 0


def test_failing_hook_reports_oom():
    torch = torch_cuda()
    m.build()
    rec = _Counting(fail=True)
    ctx = m.mdsip_ctx_create(0, torch.cuda.current_stream().cuda_stream, allocator=rec.hooks)
    try:
        with pytest.raises(m.MdsipError) as ei:
            m.mdsip_problem_create_synthetic(ctx, **m.synth_arrays(synth.make_config(0)))
        assert ei.value.status == 3        # MDSIP_ERR_OOM
        assert "hook" in m.mdsip_ctx_last_error(ctx)
        rec.fail = False                    # the same context works once memory is given
        prob = m.mdsip_problem_create_synthetic(ctx, **m.synth_arrays(synth.make_config(0)))
        try:
            assert m.STATUS[m.mdsip_solve(prob, ctx)] == "OK"
        finally:
            m.mdsip_problem_destroy(prob)
    finally:
        m.mdsip_ctx_destroy(ctx)
    assert not rec.live

"""Shared helpers of the GPU tests (device buffers through torch, contexts)."""
import numpy as np

import paper_2605_13736_gb300 as m


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def dev(a, dtype=None):
    torch = torch_cuda()
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda().contiguous()


def make_ctx():
    torch = torch_cuda()
    m.build()
    stream = torch.cuda.current_stream().cuda_stream
    return m.mdsip_ctx_create(0, stream)


def make_problem(ctx, inst, path=None):
    prob = m.mdsip_problem_create_synthetic(ctx, **m.synth_arrays(inst))
    if path is not None:
        m.mdsip_set_option_int(prob, "path", path, ctx)
    return prob


def pack_dir(r):
    return np.concatenate([r["dx"], r["dd"], r["dyg"], r["dyh"], r["dzl"], r["dzu"], r["dvl"], r["dvu"]])

"""Helpers for the GPU parity tests (device transfer, relative error)."""
import numpy as np


def to_dev(*arrays):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0") for a in arrays]


def run_fmm(xy, q, levels, p, precision="fp64", box=5.0):
    from paper_2009_00767_gb300 import binding
    txy, tq = to_dev(xy, q)
    with binding.Plan(q.shape[0], levels, p, box, precision) as plan:
        phi = plan.potential(txy, tq).cpu().numpy()
        stats = plan.stats()
    return phi, stats

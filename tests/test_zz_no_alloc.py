"""fmm_potential_noalloc: the FP64 method for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc (a loop that forbids allocation after start-up, a
device whose free memory belongs to another allocator, a plugin that may not own
allocations), so this entry point runs the method with its workspaces in a fixed device
array inside the library.  The test calls it through the C ABI twice in a row, on
different inputs, and checks each result against the plan-based fmm_potential within the
FP64 path's tolerance (1e-12 relative L2).  The file sorts last so that a run that stops
at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from conftest import rel_l2
from paper_2009_00767_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12


def test_noalloc_matches_plan_on_two_calls_in_a_row():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_00767_gb300 import binding
    lib = binding.library()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev).cuda_stream
    cases = [(40000, 6, 20, inputs.uniform(40000, 501)), (9000, 5, 12, inputs.gmm(9000, 502))]
    for n, lev, p, (xy, q) in cases:
        txy = torch.from_numpy(xy).to(dev)
        tq = torch.from_numpy(q).to(dev)
        out = torch.full((n,), 7.0, dtype=torch.float64, device=dev)
        st = lib.fmm_potential_noalloc(n, lev, p, ctypes.c_double(5.0), txy.data_ptr(), tq.data_ptr(),
                                       out.data_ptr(), stream)
        assert st == binding.FMM_OK, binding.status_string(st)
        with binding.Plan(n, lev, p, 5.0, "fp64") as plan:
            ref = plan.potential(txy, tq)
        assert rel_l2(out.cpu().numpy(), ref.cpu().numpy()) < TOL


def test_noalloc_rejects_sizes_beyond_its_limit():
    import torch
    from paper_2009_00767_gb300 import binding
    lib = binding.library()
    x = torch.zeros((65537, 2), dtype=torch.float64, device="cuda:0")
    qq = torch.zeros(65537, dtype=torch.float64, device="cuda:0")
    ph = torch.zeros(65537, dtype=torch.float64, device="cuda:0")
    s = lib.fmm_potential_noalloc(65537, 6, 20, ctypes.c_double(5.0), x.data_ptr(), qq.data_ptr(), ph.data_ptr(), None)
    assert s == binding.FMM_ERR_INVALID_ARG
    assert lib.fmm_potential_noalloc(100, 7, 20, ctypes.c_double(5.0), x.data_ptr(), qq.data_ptr(), ph.data_ptr(),
                                     None) == binding.FMM_ERR_INVALID_ARG
    assert lib.fmm_potential_noalloc(100, 6, 21, ctypes.c_double(5.0), x.data_ptr(), qq.data_ptr(), ph.data_ptr(),
                                     None) == binding.FMM_ERR_INVALID_ARG

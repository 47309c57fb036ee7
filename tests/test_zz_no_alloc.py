"""fmm_potential_noalloc: the FP64 method for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc (a loop that forbids allocation after start-up, a
device whose free memory belongs to another allocator, a plugin that may not own
allocations), so this entry point runs the method with its workspaces in a fixed device
array inside the library.  The tests call it through the C ABI and check each result
against the plan-based fmm_potential within the FP64 path's tolerance (1e-12 relative L2),
on two calls in a row, that a repeated call leaves the device's free memory unchanged, the
levels without a far field, the NULL stream, and that a call whose device checks fail is
followed by a correct one (the array keeps the previous call's state).  The file sorts last
so that a run that stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from conftest import check_parity
from paper_2009_00767_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_00767_gb300 import binding
    return binding, binding.library()


def _call(lib, n, lev, p, txy, tq, out, stream):
    return lib.fmm_potential_noalloc(n, lev, p, ctypes.c_double(5.0), txy.data_ptr(), tq.data_ptr(), out.data_ptr(),
                                     stream)


def test_noalloc_matches_plan_on_two_calls_in_a_row():
    import torch
    binding, lib = _lib()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev).cuda_stream
    cases = [(40000, 6, 20, inputs.uniform(40000, 501)), (9000, 5, 12, inputs.gmm(9000, 502))]
    for n, lev, p, (xy, q) in cases:
        txy = torch.from_numpy(xy).to(dev)
        tq = torch.from_numpy(q).to(dev)
        out = torch.full((n,), 7.0, dtype=torch.float64, device=dev)
        st = _call(lib, n, lev, p, txy, tq, out, stream)
        assert st == binding.FMM_OK, binding.status_string(st)
        with binding.Plan(n, lev, p, 5.0, "fp64") as plan:
            ref = plan.potential(txy, tq)
        check_parity(out.cpu().numpy(), ref.cpu().numpy(), TOL, f"noalloc N={n} levels={lev} p={p}")


def test_noalloc_allocates_nothing_on_a_repeated_call():
    import torch
    binding, lib = _lib()
    dev = torch.device("cuda:0")
    xy, q = inputs.uniform(20000, 503)
    txy = torch.from_numpy(xy).to(dev)
    tq = torch.from_numpy(q).to(dev)
    out = torch.empty(20000, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    assert _call(lib, 20000, 6, 16, txy, tq, out, stream) == binding.FMM_OK   # set-up done
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    assert _call(lib, 20000, 6, 16, txy, tq, out, stream) == binding.FMM_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free0


def test_noalloc_levels_without_far_field_and_null_stream(oracle_mod):
    import torch
    binding, lib = _lib()
    dev = torch.device("cuda:0")
    xy, q = inputs.uniform(600, 504)
    txy = torch.from_numpy(xy).to(dev)
    tq = torch.from_numpy(q).to(dev)
    torch.cuda.synchronize()
    for lev in (0, 1):
        out = torch.empty(600, dtype=torch.float64, device=dev)
        assert _call(lib, 600, lev, 8, txy, tq, out, None) == binding.FMM_OK   # NULL = default stream
        check_parity(out.cpu().numpy(), oracle_mod.direct(xy, q), 1e-13, f"noalloc levels={lev}")


def test_noalloc_failed_checks_then_a_clean_call():
    import torch
    binding, lib = _lib()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev).cuda_stream
    xy, q = inputs.uniform(5000, 505)
    bad = xy.copy()
    bad[123] = (5.5, 1.0)
    tbad = torch.from_numpy(bad).to(dev)
    txy = torch.from_numpy(xy).to(dev)
    tq = torch.from_numpy(q).to(dev)
    out = torch.full((5000,), 9.0, dtype=torch.float64, device=dev)
    assert _call(lib, 5000, 4, 10, tbad, tq, out, stream) == binding.FMM_ERR_OUT_OF_BOX
    assert bool((out == 9.0).all())
    assert _call(lib, 5000, 4, 10, txy, tq, out, stream) == binding.FMM_OK
    with binding.Plan(5000, 4, 10, 5.0, "fp64") as plan:
        ref = plan.potential(txy, tq)
    check_parity(out.cpu().numpy(), ref.cpu().numpy(), TOL, "noalloc after a failed call")


def test_noalloc_rejects_sizes_beyond_its_limit():
    import torch
    binding, lib = _lib()
    x = torch.zeros((65537, 2), dtype=torch.float64, device="cuda:0")
    qq = torch.zeros(65537, dtype=torch.float64, device="cuda:0")
    ph = torch.zeros(65537, dtype=torch.float64, device="cuda:0")
    assert _call(lib, 65537, 6, 20, x, qq, ph, None) == binding.FMM_ERR_INVALID_ARG
    assert _call(lib, 100, 7, 20, x, qq, ph, None) == binding.FMM_ERR_INVALID_ARG
    assert _call(lib, 100, 6, 21, x, qq, ph, None) == binding.FMM_ERR_INVALID_ARG

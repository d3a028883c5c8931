"""Failure detection without a GPU fault: the library's bounded waits (the
scans' look-back wait and the blend kernels' mbarrier wait) given something
that never completes must time out, report HM_DEV_TIMEOUT through the device
status word and return, and the context must stay usable afterwards."""
import time

import pytest
import torch

from paper_2506_06988_b300 import lib, scenes

from gpu_util import compare_blend, gpu_render, oracle_view, view_outputs  # noqa: E402

pytestmark = pytest.mark.gpu


def test_bounded_waits_time_out_and_the_context_stays_usable():
    slot = torch.zeros(1, dtype=torch.int64, device="cuda")          # a look-back slot nobody publishes
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.full((2,), 7, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    lib.check(lib.hm_selftest_bounded_waits(slot, status, out, torch.cuda.current_stream().cuda_stream),
              "hm_selftest_bounded_waits")
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    assert int(status.item()) & lib.HM_DEV_TIMEOUT
    assert out.tolist() == [0, 0]                  # neither wait completed
    assert elapsed < 10.0
    # the context still works: a render matches the oracle
    s = scenes.micro_two_gaussians()
    r, _, _ = gpu_render(s)
    assert r.status()[0] == 0
    compare_blend(view_outputs(r, 0), oracle_view(s, 0))

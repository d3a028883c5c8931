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


@pytest.mark.plants_bad_index
def test_out_of_range_record_index_is_reported_not_returned():
    """A pair list holding a record index past the records (possible only
    after an earlier failure left the list invalid) is caught by the blend
    kernel's index guard: HM_DEV_BAD_INDEX in the status word, and the
    renderer's checked paths raise instead of returning the image."""
    s = scenes.micro_two_gaussians()
    r, P, mesh = gpu_render(s)
    assert int(r.n_pairs.item()) > 0
    r.pair_vals[0] = r.V * r.n + 1000                  # out of range; the guard substitutes record 0
    r.blend()
    torch.cuda.synchronize()
    st = r.status()[0]
    assert st & lib.HM_DEV_BAD_INDEX
    with pytest.raises(lib.HmError, match="HM_DEV_BAD_INDEX"):
        lib.check_device_status(st)
    # a full render (fresh lists) clears the status and succeeds
    r.render(P["means"], P["scales"], P["quats"], P["opacity"], P["sh"], mesh)
    assert r.status()[0] == 0
    compare_blend(view_outputs(r, 0), oracle_view(s, 0))

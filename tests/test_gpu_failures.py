"""Failure detection on the host: an allocation that fails while a context
is being created makes gs_create return GS_ERR_OOM and release everything it
had allocated.  The failure is injected in the library's allocation helper
(gs_set_alloc_failure); no device fault is involved."""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("after", [0, 1, 7, 23, 45])
def test_create_reports_oom_and_leaves_nothing_allocated(after):
    import torch

    import paper_2308_01629_gb300 as gs
    sc = scenes.funnel()
    gs.Context(sc).close()   # module loading and the CUDA context are set up once
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    gs.gs_set_alloc_failure(after)
    try:
        with pytest.raises(gs.GsError) as err:
            gs.Context(sc)
        assert err.value.code == gs.GS_ERR_OOM
    finally:
        gs.gs_set_alloc_failure(-1)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert abs(free1 - free0) <= 2 << 20, (free0, free1)
    # the library works normally afterwards
    ctx = gs.Context(sc)
    ctx.step_low(1.0 / 240.0, 2)
    x = ctx.read(gs.GS_FIELD_LR_POS)
    ctx.close()
    assert np.all(np.isfinite(x))

"""Per-launch timing (MK_FLAG_TIMING) and its sampling (mk_set_timing)."""

import numpy as np
import pytest

from tests.helpers import desc_for

pytestmark = pytest.mark.gpu

MK_FLAG_TIMING = 1


def test_sampled_timing_counts_and_results(tiny_inputs):
    from paper_2106_04649_gb300 import binding as B
    from paper_2106_04649_gb300 import _native as N
    from paper_2106_04649_gb300.api import Plan
    s, R64, td, Gd64 = tiny_inputs
    R, Gd = R64.astype(np.complex64), Gd64.astype(np.float32)
    out = []
    for flags, stride in ((0, None), (MK_FLAG_TIMING, 1), (MK_FLAG_TIMING, 4)):
        p = Plan([desc_for(s, flags=flags)])
        p.load_R(0, R)
        if stride is not None:
            B.mk_set_timing(p.handle, stride, 8)
        else:  # without the flag there is nothing to sample
            with pytest.raises(B.MarchenkoError) as ei:
                B.mk_set_timing(p.handle, 2, 0)
            assert ei.value.status == N.MK_ERR_STATE
        p.set_Gd_window(0, Gd, td, s.eps)
        p.stats(reset=True)
        e = p.iterate(16)
        st = p.stats(reset=True)
        if stride is None:
            assert st["contract_timed"] == 0
        else:
            assert st["contract_timed"] == 16 // stride and st["epilogue_timed"] == 16 // stride
            assert st["contract_ms"] > 0 and st["epilogue_ms"] > 0
        assert st["contract_launches"] == 16
        out.append((e, p.fetch_fields(0)))
        p.close()
    # timing never changes a result
    for e, f in out[1:]:
        assert np.array_equal(e, out[0][0]) and np.array_equal(f, out[0][1])

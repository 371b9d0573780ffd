"""Size limits of one evaluation call, through the C ABI.

The work lists of a call (one entry per particle and work chunk its support
meets, sized for P times the stream's chunks) are indexed with 32-bit
offsets; a call above 2^31 - 1 such pairs is refused before any scratch is
allocated, and the context stays usable.
"""
import numpy as np
import pytest

from paper_2408_13170_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scstat():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2408_13170_gb300 import scstat as m
    return m


def test_call_above_the_work_list_limit_is_refused(scstat):
    d = synth.make_stream("C3")   # the four-year stream: 5 040 001 bins
    th = synth.injection_params(d["rng"], 30.0, 1.5, 0.018)
    with scstat.Context(0, scstat.SCS_MIXED) as ctx:
        ctx.set_data(0, d)
        ctx.set_segments(0, 16, scstat.SCS_EQUAL_WIDTH)
        scstat.scs_set_tile(ctx.h, 0, 11)
        n_chunks = -(-d["K"] // 2048)
        P = (2**31 - 1) // n_chunks + 1          # one particle over the limit
        assert P * n_chunks > 2**31 - 1 and P <= 2**24
        params = np.tile(th, (P, 1))
        with pytest.raises(scstat.ScsError) as e:
            ctx.eval(0, params)
        assert e.value.code == scstat.SCS_EINVAL
        assert "split the call" in str(e.value)
        # the same particle in a small call afterwards
        st = ctx.eval(0, params[:64])
        assert np.all(np.isfinite(st)) and np.all(st == st[0]) and st[0] > 0

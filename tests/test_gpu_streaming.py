"""Streaming host blocks (stream_blocks = 1): alternate staging buffers and
trigger lists, so that the next block's host copy overlaps this block's
kernels and a block's triggers are read while the next block runs.  The
results of every block equal those of the ordinary host-input plan bit for
bit, read either while the next block is in flight or as the last block; only
the last two blocks can be read.
"""

import numpy as np
import pytest

from gpu_common import random_case

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp16", "fp32"])
def test_streaming_blocks_equal_ordinary_host_blocks(cuda_lib, precision):
    import torch
    lp = cuda_lib
    S, P, K, B, Tr, F, fb = 8, 2, 24, 5, 2, 520, 160
    blocks, enu, dirs, tec = random_case(81, S, P, K, B, Tr, F, fb, "int8", 5, amp=100)
    hosts = [torch.from_numpy(b).pin_memory() for b in blocks]
    kw = dict(input_dtype="int8", precision=precision, first_bin=fb, k_sigma=3.5,
              host_input=True)
    ref = lp.Plan(S, P, K, B, Tr, F, **kw)
    st = lp.Plan(S, P, K, B, Tr, F, stream_blocks=True, **kw)
    for p in (ref, st):
        p.lp_set_weights(enu, dirs)
        p.lp_set_tec(tec)
    want = []
    for h in hosts:
        ref.lp_process_block(h)
        want.append((ref.lp_get_triggers()[0], ref.lp_get_sigma().copy()))
    got = []
    for i, h in enumerate(hosts):
        st.lp_process_block(h)
        if i > 0:                       # block i - 1 while block i runs
            got.append(st.lp_get_triggers_block(i - 1)[0])
    got.append(st.lp_get_triggers_block(len(hosts) - 1)[0])
    for (tw, _), tg in zip(want, got):
        np.testing.assert_array_equal(tg, tw)
        assert len(tg) > 0
    np.testing.assert_array_equal(st.lp_get_sigma(), want[-1][1])
    np.testing.assert_array_equal(st.lp_get_triggers()[0], want[-1][0])
    with pytest.raises(lp.LPError):
        st.lp_get_triggers_block(len(hosts) - 3)       # no longer kept
    with pytest.raises(lp.LPError):
        ref.lp_get_triggers_block(len(hosts) - 2)      # ordinary plans keep the last only
    np.testing.assert_array_equal(ref.lp_get_triggers_block(len(hosts) - 1)[0], want[-1][0])

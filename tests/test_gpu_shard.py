"""Beam sharding on the GPU: the ranks' plans, run one after the other on one
GPU (each on the whole station block, as every rank would on its own GPU),
give -- after relabelling and merging -- exactly the triggers and noise levels
of one plan over all beams, in both beamformer forms.  (Each beam's arithmetic
does not depend on which other beams share its plan: the FP32 form sums each
beam on its own, and in the tensor-core form every beam's rows accumulate the
same products in the same order whatever the other rows of the tile hold.)
"""

import numpy as np
import pytest

from gpu_common import random_case
from paper_1612_06592_gb300.shard import BeamShard, merge_triggers

pytestmark = pytest.mark.gpu

KEY = ("n", "beam", "tec", "pol", "stream", "env", "sigma")


@pytest.mark.parametrize("precision,world", [("fp16", 2), ("fp32", 3)])
def test_beam_shards_merge_to_the_single_plan(cuda_lib, precision, world):
    import torch
    S, P, K, B, Tr, F, fb = 8, 2, 20, 9, 2, 520, 160
    blocks, enu, dirs, tec = random_case(61, S, P, K, B, Tr, F, fb, "int8", 2, amp=100)
    kw = dict(input_dtype="int8", precision=precision, first_bin=fb, k_sigma=3.5)
    full = cuda_lib.Plan(S, P, K, B, Tr, F, **kw)
    full.lp_set_weights(enu, dirs)
    full.lp_set_tec(tec)
    shards = [BeamShard(S, P, K, B, Tr, F, rank=r, world=world, **kw) for r in range(world)]
    for sh in shards:
        sh.lp_set_weights(enu, dirs)
        sh.lp_set_tec(tec)
    for xb in blocks:                                   # two blocks: carried state too
        xd = torch.from_numpy(xb).cuda()
        full.lp_process_block(xd)
        want, n_want, _ = full.lp_get_triggers()
        parts, sig = [], []
        for sh in shards:
            sh.lp_process_block(xd)
            t, n, st = sh.lp_get_triggers()
            assert st == cuda_lib.LP_OK
            parts.append(t)
            sig.append(sh.lp_get_sigma())
        got = merge_triggers(parts)
        assert len(want) > 20 and len(got) == len(want)
        for k in KEY:
            np.testing.assert_array_equal(got[k], want[k])
        np.testing.assert_array_equal(np.concatenate(sig), full.lp_get_sigma())

"""Failure detection on the GPU without a fault: the tensor-core screen's
pipeline waits are bounded (rhseg_params.wait_cycles).  A bound of one clock
cycle makes the first wait for a TMA load run out; the screen then stops,
lets its own copies and MMAs finish, releases its tensor memory and sets the
device error word, which rhseg_run returns as RHSEG_ETIMEOUT.  The same
handle then runs again with the default bound and gives the oracle's result,
so the context and the handle stay usable.  Both screen forms: one CTA per
unit, and CTA pairs (where a wait that runs out also stops the peer CTA).  (The paper has no failure
detection; this is the library's own.)"""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(__file__))
import synth  # noqa: E402
from test_gpu_parity import _assert_same  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2106_12942_b300 as P
    return P


@pytest.mark.parametrize("pair", [0, 1])
@pytest.mark.parametrize("precision", [1, 2])
def test_screen_wait_that_runs_out_returns_etimeout(P, orc, precision, pair):
    from paper_2106_12942_b300 import _abi
    img, mask = synth.make(4, seed=7, rows=48, cols=40)
    img = np.ascontiguousarray(img[:, :, :24])
    kw = dict(rnb_levels=3, spclust_wght=0.3, conv_nregions=6, connectivity=8, n_out_levels=3)
    seg = P.RHSEG(img, mask, precision=precision, wait_cycles=1, screen_pair=pair, **kw)
    with pytest.raises(P.RHSEGError) as e:
        seg.run()
    assert e.value.code == _abi.RHSEG_ETIMEOUT
    with pytest.raises(P.RHSEGError) as e2:        # no results from a run that stopped
        seg.log()
    assert e2.value.code == _abi.RHSEG_ESTATE
    # the same handle, default bound: the oracle's log and levels
    seg.set_wait_cycles(0).run()
    _assert_same(seg, orc.run(img, mask, **kw), f"after a timed-out run, p{precision} pair{pair}")
    seg.close()


def test_wait_bound_rejects_negative(P):
    img = np.zeros((4, 4, 3), dtype=np.uint16)
    with pytest.raises(P.RHSEGError):
        P.RHSEG(img, None, wait_cycles=-1)

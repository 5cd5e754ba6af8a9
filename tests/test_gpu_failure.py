"""Failure detection without a GPU fault: every device-side wait of the library is bounded and
reports through the context's status word. The self-test makes one wait run out (a look-back
word that nothing publishes); the host reads LOBE_ERR_TIMEOUT, and the same context then
renders correctly."""
import time

import numpy as np
import pytest
import torch

import oracle
import scenes
from tests.helpers import match_image

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2510_01767_b300 as lobe
    from paper_2510_01767_b300 import _abi as A


def test_bounded_wait_times_out_and_the_context_survives():
    ctx = lobe.Context()
    ctx.status()  # clean
    t0 = time.perf_counter()
    ctx._check(ctx.lib.lobe_selftest_wait(ctx.handle))
    with pytest.raises(A.LobeError) as err:
        ctx.status()  # synchronises: the wait gave up and latched the timeout
    assert err.value.code == A.ERR_TIMEOUT
    assert time.perf_counter() - t0 < 60.0
    ctx.status()  # reading the status cleared it
    # the same context still renders, bit-identical work as before the failure
    wl = scenes.small_scene()
    batch = lobe.Batch([lobe.GaussianSet.from_numpy(wl.sets[0])], wl.cameras, wl.items, wl.blocks)
    proj, bins, img = lobe.forward(ctx, batch)
    cam = wl.cameras[0].as_dict()
    p = oracle.project(oracle.set_dict(wl.sets[0]), cam, wl.tile, margins=oracle.MARGINS_E2E)
    eb = oracle.bin_ext(p, cam, wl.tile)
    lv = oracle.render_leaves(p, eb, cam, wl.tile, margins=oracle.MARGINS_E2E)
    match_image(lv, img.rgb.view(3, 128, 128).cpu().numpy(), img.T_final.view(128, 128).cpu().numpy(), None,
                "image small after a timeout")
    ctx.status()

"""Batched multi-view / multi-block step captured in a CUDA graph: identical images to the
plain one-view-per-call path, matching gradients, graph replay after parameter updates,
and the tile-shape autotuner."""
import numpy as np
import pytest
import torch

import scenes
from tests.helpers import grad_rel_err

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2510_01767_b300 as lobe
    from paper_2510_01767_b300.batched import BatchedStep, PlainSteps, autotune


def small_multi_block(seed=0):
    return scenes.multi_block_scene(seed=seed, block_sizes=(3000, 6000, 9000, 12000), views_per_block=2,
                                    city_n=60000)


def scaled(wl, f=0.25):
    """The same batch with every view shrunk (keeps the test fast)."""
    cams = []
    for c in wl.cameras:
        w, h = max(16, int(c.width * f)), max(16, int(c.height * f))
        cams.append(scenes.pinhole(w, h, c.fx * f, viewmat=c.viewmat))
    return scenes.Workload(wl.name, wl.sets, cams, wl.blocks, wl.items, wl.tile)


@pytest.fixture(scope="module")
def workload():
    return scaled(small_multi_block())


def fill_dL(step, seed=3):
    g = torch.Generator(device="cuda").manual_seed(seed)
    step.dL.copy_(torch.randn(step.dL.shape, generator=g, device="cuda"))


def test_graph_replay_equals_plain(workload):
    wl = workload
    sets = [lobe.GaussianSet.from_numpy(s) for s in wl.sets]
    cams = [c.as_dict() for c in wl.cameras]
    st = BatchedStep(sets, cams, wl.items, wl.blocks, tile=(16, 16))
    fill_dL(st)
    st.capture()
    st.replay()
    torch.cuda.synchronize()
    plain = PlainSteps(sets, cams, wl.items, wl.blocks, tile=(16, 16))
    for p, d in zip(plain.steps, st.dL_views()):
        p.dL.copy_(d.reshape(-1))
    plain.run()
    torch.cuda.synchronize()
    for img, p in zip(st.images(), plain.steps):
        torch.testing.assert_close(img, p.images()[0], rtol=0, atol=0)
    # gradients: the batched step sums each set's views in registers
    for s in range(len(sets)):
        for k in lobe.PARAM_KEYS:
            want = sum(p.grads[0][k] for p, it in zip(plain.steps, wl.items) if it[0] == s)
            assert grad_rel_err(st.grads[s][k].cpu().numpy(), want.cpu().numpy()) <= 1e-3, (s, k)
        want_cnt = sum(p.grads[0]["sd_cnt"] for p, it in zip(plain.steps, wl.items) if it[0] == s)
        # the graph step ran three times (two warm-up runs before capture, one replay)
        assert torch.equal(st.grads[s]["sd_cnt"], 3 * want_cnt)


def test_graph_follows_parameter_updates(workload):
    wl = workload
    sets = [lobe.GaussianSet.from_numpy(s) for s in wl.sets]
    cams = [c.as_dict() for c in wl.cameras]
    st = BatchedStep(sets, cams, wl.items, wl.blocks, tile=(16, 16)).capture()
    st.replay()
    torch.cuda.synchronize()
    before = st.image.rgb.clone()
    with torch.no_grad():
        for s in sets:
            s.sh[:, 0, :] += 0.3  # brighter: parameters are updated in place, as an optimiser does
    st.replay()
    torch.cuda.synchronize()
    eager = BatchedStep(sets, cams, wl.items, wl.blocks, tile=(16, 16))
    eager.run()
    torch.cuda.synchronize()
    assert not torch.equal(before, st.image.rgb)
    torch.testing.assert_close(st.image.rgb, eager.image.rgb, rtol=0, atol=0)


def test_graph_replay_past_its_pair_capacity(workload):
    """Gaussians that grow after capture (every scale e times larger) need more (splat, tile)
    pairs than the captured step reserved: the replay latches LOBE_ERR_CAPACITY, its bins then
    describe empty tiles (every pixel the background, T = 1, no 2D gradient), the context stays
    usable, and a step built for the grown Gaussians matches the eager path again."""
    wl = workload
    sets = [lobe.GaussianSet.from_numpy(s) for s in wl.sets]
    cams = [c.as_dict() for c in wl.cameras]
    bg = (0.25, 0.5, 0.75)
    st = BatchedStep(sets, cams, wl.items, wl.blocks, tile=(16, 16), bg=bg, slack=1.0).capture()
    fill_dL(st)
    st.replay()
    st.stream.synchronize()
    st.ctx.status()  # within capacity
    with torch.no_grad():
        for s in sets:
            s.log_scales += 1.0
    st.replay()
    st.stream.synchronize()
    with pytest.raises(lobe._abi.LobeError) as e:
        st.ctx.status()
    assert e.value.code == lobe._abi.ERR_CAPACITY
    assert int(st.bins.tile_start.abs().max().item()) == 0
    for v in st.images():
        for ch in range(3):
            assert torch.all(v[ch] == bg[ch])
    assert torch.all(st.image.T_final == 1.0)
    assert torch.all(st.grad2d == 0)
    st.ctx.status()  # read and cleared
    grown = BatchedStep(sets, cams, wl.items, wl.blocks, tile=(16, 16), bg=bg).capture()
    assert grown.n_isect > st.bins.capacity
    grown.replay()
    grown.stream.synchronize()
    grown.ctx.status()
    eager = BatchedStep(sets, cams, wl.items, wl.blocks, tile=(16, 16), bg=bg)
    eager.run()
    eager.stream.synchronize()
    torch.testing.assert_close(grown.image.rgb, eager.image.rgb, rtol=0, atol=0)


@pytest.mark.parametrize("tile", [(8, 8), (16, 8), (32, 16)])
def test_batched_other_tiles_match_16(workload, tile):
    wl = workload
    sets = [lobe.GaussianSet.from_numpy(s) for s in wl.sets]
    cams = [c.as_dict() for c in wl.cameras]
    a = BatchedStep(sets, cams, wl.items, wl.blocks, tile=(16, 16))
    b = BatchedStep(sets, cams, wl.items, wl.blocks, tile=tile)
    a.run()
    b.run()
    torch.cuda.synchronize()
    # different tile shapes truncate splats at different tile rectangles: images agree up to
    # the contributions beyond 3 sigma (alpha <= 0.011 o), so compare loosely and on average
    d = (a.image.rgb - b.image.rgb).abs()
    assert float(d.mean()) < 2e-3


def test_autotune_picks_fastest(workload, tmp_path, monkeypatch):
    from paper_2510_01767_b300 import batched
    monkeypatch.setattr(batched, "CACHE", str(tmp_path / "autotune.json"))
    wl = workload
    sets = [lobe.GaussianSet.from_numpy(s) for s in wl.sets]
    cams = [c.as_dict() for c in wl.cameras]
    best, times = autotune(sets, cams, wl.items, wl.blocks, reps=3, dL_init=fill_dL)
    # every tile shape once, the winner once more as persistent kernels, and then with its tuned
    # staging batch when that is not 32 / 32
    assert {k.split("/")[0] for k in times} == {"8x8", "16x8", "16x16", "32x16"} and len(times) in (5, 6)
    assert sum(k.endswith("/persistent") for k in times) in (1, 2)
    assert (len(times) == 6) == any("/s" in k for k in times)
    name = batched.config_name(best.tile, best.px, best.batch_size) + ("/persistent" if best.persistent else "")
    assert times[name] == min(times.values())
    again, t2 = autotune(sets, cams, wl.items, wl.blocks, reps=3, dL_init=fill_dL)  # from the cache
    assert again.tile == best.tile and again.px == best.px and again.persistent == best.persistent and t2 == times
    assert again.batch_size == best.batch_size

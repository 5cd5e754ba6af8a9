"""Host-side logic without a GPU: the camera assignment of fast camera selection (Sec. 3.2)
from per-block counts, and the autotuner's configuration names."""
import numpy as np
import torch

from paper_2510_01767_b300 import batched
from paper_2510_01767_b300.raster import fcs_select


def test_fcs_select_assigns_cameras_at_tau():
    """V[c, b] = counts / points; camera c joins block b when V >= tau (0.1 in the paper);
    a camera without points joins nothing."""
    counts = torch.tensor([[50, 5, 45], [0, 0, 0], [10, 10, 80], [1, 99, 0]], dtype=torch.int32)
    npts = torch.tensor([100, 0, 100, 100], dtype=torch.int32)
    V, assign = fcs_select(counts, npts, tau=0.1)
    np.testing.assert_allclose(V.numpy(), [[0.5, 0.05, 0.45], [0, 0, 0], [0.1, 0.1, 0.8], [0.01, 0.99, 0.0]])
    assert assign == [[0, 2], [2, 3], [0, 2]]
    _, strict = fcs_select(counts, npts, tau=0.5)
    assert strict == [[0], [3], [2]]


def test_autotune_configuration_names():
    assert batched.config_name((8, 8), (1, 2)) == "8x8/f1b2"
    assert batched.config_name((32, 16), (4, 8)) == "32x16/f4b8"
    assert batched.config_name((16, 8), (2, 4), (32, 32)) == "16x8/f2b4"  # the default staging batch
    assert batched.config_name((16, 8), (2, 4), (64, 32)) == "16x8/f2b4/s64.32"
    assert set(batched.BATCH_OPTIONS) == {32, 64}
    for tile, pxs in batched.PX_OPTIONS.items():
        assert tile in batched.TILES and len(pxs) >= 2


def test_traffic_files_track_their_kernel_sources(tmp_path, monkeypatch):
    """bench.py quotes a stage's DRAM traffic only while the kernel sources it was captured
    from are unchanged: every committed traffic file names its sources, and a changed source
    makes traffic_of return None."""
    import importlib.util
    import json
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    prof = os.path.join(root, "profiles")
    names = [f for f in os.listdir(prof) if f.startswith("traffic_") and f.endswith(".json")]
    assert names
    for f in names:
        t = json.load(open(os.path.join(prof, f)))
        assert t["sources"] and all(os.path.exists(os.path.join(root, p)) for p in t["sources"]), f
        assert len(t["source_sha1"]) == 16 and t["bytes_per_launch"] > 0, f
    # a copy of the tree with one source edited: the same file reads as stale
    fake = tmp_path / "repo"
    (fake / "profiles").mkdir(parents=True)
    src = fake / "k.cu"
    src.write_text("kernel A")
    monkeypatch.setattr(bench, "ROOT", str(fake))
    rec = {"bytes_per_launch": 123, "sources": ["k.cu"], "source_sha1": bench.source_digest(["k.cu"])}
    (fake / "profiles" / "traffic_render_bwd_w.json").write_text(json.dumps(rec))
    assert bench.traffic_of("render_bwd", "w")["bytes_per_launch"] == 123
    src.write_text("kernel A // a comment\n/* and another */")  # comments do not change the code
    assert bench.traffic_of("render_bwd", "w")["bytes_per_launch"] == 123
    src.write_text("kernel B")
    assert bench.traffic_of("render_bwd", "w") is None
    assert bench.traffic_of("render_fwd", "w") is None  # absent

"""The pruning pass's tuning (task depth, CTAs per SM, rows per 2D task) and
the autotuner change only the time, never the pairs."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_04801_gb300 as cp

    return cp


def test_pairs_do_not_depend_on_tuning(cp):
    from paper_2606_04801_gb300 import autotune

    vol = torch.from_numpy(workloads.blurred((70, 50, 90), 2.0, 41)).cuda()
    img = torch.from_numpy(workloads.quantised(workloads.blurred((300, 200), 3.0, 42))).cuda()
    saved = autotune.current()
    try:
        ref_v = cp.persistence(vol).raw.cpu()
        ref_i = cp.persistence(img).raw.cpu()
        ref_b = cp.persistence_batched([img, vol]).raw.cpu()
        for zc, ctas, rows in [(4, 1, 4), (16, 2, 7), (256, 0, 128), (4096, 3, 4096)]:
            autotune.apply({"zchunk3d": zc, "ctas3d": ctas, "rows2d": rows})
            assert torch.equal(cp.persistence(vol).raw.cpu(), ref_v)
            assert torch.equal(cp.persistence(img).raw.cpu(), ref_i)
            assert torch.equal(cp.persistence_batched([img, vol]).raw.cpu(), ref_b)
    finally:
        autotune.apply(saved)


def test_autotune_picks_and_caches(cp, tmp_path):
    from paper_2606_04801_gb300 import autotune

    saved = autotune.current()
    try:
        vol = torch.from_numpy(workloads.blurred((96, 96, 96), 3.0, 43)).cuda()
        cfg = autotune.autotune([vol], cache=str(tmp_path / "t.json"))
        assert cfg["trials"] >= 15 and cfg["ms"] > 0
        assert autotune.current()["zchunk3d"] == cfg["zchunk3d"]
        # the union-find design is measured too, and the faster one kept
        assert set(cfg["forward_ms"]) == {"0", "1"}
        assert cfg["uf_variant"] == min((0, 1), key=lambda v: cfg["forward_ms"][str(v)])
        assert autotune.current()["uf_variant"] == cfg["uf_variant"]
        assert "|surv:" in cfg["key"]
        again = autotune.autotune([vol], cache=str(tmp_path / "t.json"))
        assert again["ms"] == cfg["ms"]  # served from the cache
    finally:
        autotune.apply(saved)


def test_autotune_key_follows_the_data(cp, tmp_path):
    """Smooth fields and i.i.d. noise of one shape leave very different
    survivor fractions, so they get separate cache entries."""
    from paper_2606_04801_gb300 import autotune

    saved = autotune.current()
    try:
        smooth = torch.from_numpy(workloads.blurred((64, 64, 64), 3.0, 44)).cuda()
        noise = torch.from_numpy(workloads.uniform((64, 64, 64), 45)).cuda()
        assert autotune.survivor_fraction([noise]) > 8 * autotune.survivor_fraction([smooth])
        a = autotune.autotune([smooth], cache=str(tmp_path / "k.json"))
        b = autotune.autotune([noise], cache=str(tmp_path / "k.json"))
        assert a["key"] != b["key"]
    finally:
        autotune.apply(saved)

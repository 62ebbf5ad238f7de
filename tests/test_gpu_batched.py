"""Batched forward + backward in one CUDA graph (the batched workload's
recipe, scaled down): graph replays against eager steps, against the oracle's
pairs and reference gradient per item, and against finite differences.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
TAU = 0.05


@pytest.fixture(scope="module")
def cp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_04801_gb300 as cp

    return cp


def _ref(img):
    p = oracle.persistence(img)
    g = np.zeros(img.size, dtype=np.float64)
    loss = 0.0
    for r in p:
        if r["death_cell"] < 0:
            continue
        pers = float(r["death"]) - float(r["birth"])
        if pers > TAU:
            loss += pers * pers
            g[r["death_pixel"]] += 2 * pers
            g[r["birth_pixel"]] -= 2 * pers
    return p, loss, g


@pytest.fixture(scope="module")
def batch():
    return workloads.batch(0, n2d=10, n3d=3, scale=0.2)


def test_graph_matches_eager_and_oracle(cp, batch):
    shapes = [a.shape for a in batch]
    tens = [torch.from_numpy(a).cuda() for a in batch]
    eager = cp.BatchedPersistence(shapes, tau=TAU, graph=False)
    eager.load(tens)
    le, ge = eager.step()
    le, ge = float(le.item()), ge.cpu().numpy()
    pe = eager.pairs().numpy()
    bp = cp.BatchedPersistence(shapes, tau=TAU, graph=True)
    bp.load(tens)
    for _ in range(3):  # replays are identical
        lg, gg = bp.step()
        assert float(lg.item()) == le
        assert np.array_equal(gg.cpu().numpy(), ge)
    assert np.array_equal(bp.pairs().numpy(), pe)
    assert bp.status()["rc"] == 0
    # per item against the oracle
    grads = [g.cpu().numpy().ravel() for g in bp.grads()]
    total = 0.0
    for i, a in enumerate(batch):
        p, loss, g = _ref(a)
        total += loss
        mine = pe[pe["item"] == i]
        assert len(mine) == len(p)
        for k in ("birth", "death", "birth_cell", "death_cell", "birth_pixel", "death_pixel", "dim"):
            assert np.array_equal(mine[k], p[k]), (i, k)
        scale = max(1.0, float(np.abs(g).max()))
        np.testing.assert_allclose(grads[i], g, rtol=1e-6, atol=1e-6 * scale)
    assert abs(le - total) <= 1e-9 * max(1.0, total)


def test_graph_replay_with_new_inputs(cp, batch):
    shapes = [a.shape for a in batch]
    bp = cp.BatchedPersistence(shapes, tau=TAU, graph=True)
    bp.load([torch.from_numpy(a).cuda() for a in batch])
    bp.step()
    other = [workloads.rank_spaced(workloads.blurred(s, 2.0, 77 + i)) for i, s in enumerate(shapes)]
    bp.load([torch.from_numpy(a).cuda() for a in other])
    loss, grad = bp.step()
    want = sum(_ref(a)[1] for a in other)
    assert abs(float(loss.item()) - want) <= 1e-9 * max(1.0, want)


def test_graph_finite_differences(cp):
    """Central differences (step 1e-3) through graph replays on rank-spaced items (gaps 2^-8)."""
    items = workloads.batch(0, n2d=3, n3d=1, scale=0.12)
    shapes = [a.shape for a in items]
    bp = cp.BatchedPersistence(shapes, tau=TAU, graph=True)
    bp.load([torch.from_numpy(a).cuda() for a in items])
    _, grad = bp.step()
    g = grad.cpu().numpy().copy()
    flat = np.concatenate([a.ravel() for a in items])
    offs = np.concatenate([[0], np.cumsum([a.size for a in items])[:-1]])

    def in_loss(vals):
        bp.load([torch.from_numpy(vals[o : o + a.size].reshape(a.shape)).cuda() for o, a in zip(offs, items)])
        loss, _ = bp.step()
        d = bp.pairs().numpy()
        fin = d["death_cell"] >= 0
        pers = d["death"].astype(np.float64) - d["birth"].astype(np.float64)
        sel = fin & (pers > TAU)
        return float(loss.item()), set(zip(d["item"][sel].tolist(), d["birth_pixel"][sel].tolist(), d["death_pixel"][sel].tolist()))

    _, base = in_loss(flat)
    rng = np.random.default_rng(3)
    picks = np.concatenate([rng.choice(np.flatnonzero(g), 25, replace=False), rng.choice(flat.size, 10, replace=False)])
    h = 1e-3
    valid = 0
    for p in picks:
        xp, xm = flat.copy(), flat.copy()
        xp[p] = np.float32(flat[p] + h)
        xm[p] = np.float32(flat[p] - h)
        lp, sp = in_loss(xp)
        lm, sm = in_loss(xm)
        if sp != base or sm != base:
            continue
        fd = (lp - lm) / (float(xp[p]) - float(xm[p]))
        assert abs(fd - g[p]) <= 1e-3 * max(1.0, abs(g[p])), (p, fd, g[p])
        valid += 1
    assert valid >= 0.8 * len(picks)

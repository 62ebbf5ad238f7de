"""The benchmark's own workload at full size (512^3 blurred noise, sigma 3,
the same call bench.py times), checked by properties that hold at any size
(the oracle needs minutes there; it is compared element by element on the
smaller configurations in test_gpu_parity.py):

- two runs give byte-identical pairs;
- every pair's values are copies of its birth/death pixels, birth < death,
  and (sampled) each pixel is the largest vertex of its cell;
- for thresholds t across the range: the H0 pairs alive at t equal the
  components of {f <= t} (6-connectivity), and the H2 pairs alive at t equal
  the components of {f > t} (26-connectivity) that do not touch the border.
"""
import os

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


@pytest.fixture(scope="module")
def vol():
    cache = "/tmp/cp_bench_vol_512_3.0_0.npy"
    if os.path.exists(cache):
        try:
            return np.load(cache)
        except Exception:
            pass
    return workloads.blurred((512, 512, 512), 3.0, 0)


def _argmax_vertex(shape, cells, f):
    D, H, W = shape
    GH, GW = 2 * H - 1, 2 * W - 1
    Z, rem = np.divmod(cells, GH * GW)
    Y, X = np.divmod(rem, GW)
    best = np.full(len(cells), -1, dtype=np.int64)
    bestv = np.full(len(cells), -np.inf)
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                z = Z // 2 + dz * (Z % 2)
                y = Y // 2 + dy * (Y % 2)
                x = X // 2 + dx * (X % 2)
                v = (z * H + y) * W + x
                fv = f[v].astype(np.float64)
                better = (fv > bestv) | ((fv == bestv) & (v > best))
                best = np.where(better, v, best)
                bestv = np.where(better, fv, bestv)
    return best


def test_512_cube_properties(cp, vol):
    from scipy import ndimage

    x = torch.from_numpy(vol).cuda()
    a = cp.persistence(x)
    b = cp.persistence(x)
    assert torch.equal(a.raw, b.raw)
    p = a.numpy()
    f = vol.ravel()
    fin = p["death_cell"] >= 0
    assert (p["birth"] < p["death"]).all()
    assert (p["birth"] == f[p["birth_pixel"]]).all()
    assert (p["death"][fin] == f[p["death_pixel"][fin]]).all()
    assert (p["dim"][~fin] == 0).all() and fin.sum() == len(p) - 1
    rng = np.random.default_rng(0)
    s = rng.choice(len(p), min(20000, len(p)), replace=False)
    assert (_argmax_vertex(vol.shape, p["birth_cell"][s].astype(np.int64), f) == p["birth_pixel"][s]).all()
    sf = s[fin[s]]
    assert (_argmax_vertex(vol.shape, p["death_cell"][sf].astype(np.int64), f) == p["death_pixel"][sf]).all()
    for q in (0.35, 0.5, 0.65):
        t = np.float32(np.quantile(f[::97], q))
        alive0 = int(((p["dim"] == 0) & (p["birth"] <= t) & (t < p["death"])).sum())
        _, n0 = ndimage.label(vol <= t)
        assert alive0 == n0, (q, alive0, n0)
        alive2 = int(((p["dim"] == 2) & (p["birth"] <= t) & (t < p["death"])).sum())
        lab, n2 = ndimage.label(vol > t, structure=np.ones((3, 3, 3), dtype=bool))
        border = set()
        for ax in range(3):
            border |= set(np.unique(np.take(lab, 0, axis=ax)).tolist())
            border |= set(np.unique(np.take(lab, -1, axis=ax)).tolist())
        border.discard(0)
        assert alive2 == n2 - len(border), (q, alive2, n2, len(border))


def _t_min_pixel(shape, cells, f):
    """Top cell of smallest (value, index) containing each T-complex cell
    (doubled extents 2n+1: pixels at odd coordinates)."""
    D, H, W = shape
    GH, GW = 2 * H + 1, 2 * W + 1
    Z, rem = np.divmod(cells, GH * GW)
    Y, X = np.divmod(rem, GW)
    best = np.full(len(cells), -1, dtype=np.int64)
    bestv = np.full(len(cells), np.inf)
    for oz in (0, 1):
        for oy in (0, 1):
            for ox in (0, 1):
                # odd coordinate c: the pixel (c-1)/2; even c: pixels c/2-1 and c/2
                z = np.where(Z % 2 == 1, (Z - 1) // 2, Z // 2 - 1 + oz)
                y = np.where(Y % 2 == 1, (Y - 1) // 2, Y // 2 - 1 + oy)
                x = np.where(X % 2 == 1, (X - 1) // 2, X // 2 - 1 + ox)
                ok = (z >= 0) & (z < D) & (y >= 0) & (y < H) & (x >= 0) & (x < W)
                v = np.where(ok, (z * H + y) * W + x, 0)
                fv = np.where(ok, f[v].astype(np.float64), np.inf)
                better = ok & ((fv < bestv) | ((fv == bestv) & (v < best)))
                best = np.where(better, v, best)
                bestv = np.where(better, fv, bestv)
    return best


def test_510_cube_t_filtration_properties(cp, vol):
    """The T-filtration workload (510^3, its dual image exactly 512^3):
    determinism, values copied from the pixels the cells enter with (sampled
    cells checked against their smallest containing top cell), and Betti
    numbers across the range: H0 pairs alive at t = components of {f <= t}
    joined through shared vertices (26-connectivity), H2 pairs alive at t =
    face-connected components of {f > t} that avoid the border."""
    from scipy import ndimage

    v = np.ascontiguousarray(vol[:510, :510, :510])
    x = torch.from_numpy(v).cuda()
    a = cp.persistence(x, filtration="T")
    b = cp.persistence(x, filtration="T")
    assert torch.equal(a.raw, b.raw)
    p = a.numpy()
    f = v.ravel()
    fin = p["death_cell"] >= 0
    assert (p["birth"] < p["death"]).all()
    assert (p["birth"] == f[p["birth_pixel"]]).all()
    assert (p["death"][fin] == f[p["death_pixel"][fin]]).all()
    assert (p["dim"][~fin] == 0).all() and fin.sum() == len(p) - 1
    rng = np.random.default_rng(1)
    s = rng.choice(len(p), min(20000, len(p)), replace=False)
    assert (_t_min_pixel(v.shape, p["birth_cell"][s].astype(np.int64), f) == p["birth_pixel"][s]).all()
    sf = s[fin[s]]
    assert (_t_min_pixel(v.shape, p["death_cell"][sf].astype(np.int64), f) == p["death_pixel"][sf]).all()
    for q in (0.35, 0.5, 0.65):
        t = np.float32(np.quantile(f[::97], q))
        alive0 = int(((p["dim"] == 0) & (p["birth"] <= t) & (t < p["death"])).sum())
        _, n0 = ndimage.label(v <= t, structure=np.ones((3, 3, 3), dtype=bool))
        assert alive0 == n0, (q, alive0, n0)
        alive2 = int(((p["dim"] == 2) & (p["birth"] <= t) & (t < p["death"])).sum())
        lab, n2 = ndimage.label(v > t)
        border = set()
        for ax in range(3):
            border |= set(np.unique(np.take(lab, 0, axis=ax)).tolist())
            border |= set(np.unique(np.take(lab, -1, axis=ax)).tolist())
        border.discard(0)
        assert alive2 == n2 - len(border), (q, alive2, n2, len(border))

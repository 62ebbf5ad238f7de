"""Gradients: the backward kernels against (a) a reference gradient built in
double precision from the oracle's pairs and (b) finite differences.

Loss (the batched workload's): L = sum over finite pairs with
death - birth > 0.05 of (death - birth)^2.  Every birth and death value is a
copy of one pixel (its birth/death pixel), so dL/dx[p] collects +2(d-b) from
the pairs that die at p and -2(d-b) from the pairs born at p.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
TAU = 0.05
RTOL = 1e-6


@pytest.fixture(scope="module")
def cp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_04801_gb300 as cp

    return cp


def _ref_grad(img, tau=TAU):
    p = oracle.persistence(img)
    g = np.zeros(img.size, dtype=np.float64)
    loss = 0.0
    for r in p:
        if r["death_cell"] < 0:
            continue
        pers = float(r["death"]) - float(r["birth"])
        if pers > tau:
            loss += pers * pers
            g[r["death_pixel"]] += 2 * pers
            g[r["birth_pixel"]] -= 2 * pers
    return loss, g


def _gpu_loss_grad(cp, imgs):
    """Through the C-ABI: forward (single or batched) then the fused loss backward."""
    lib = cp.load()
    if len(imgs) == 1:
        d = cp.persistence(torch.from_numpy(imgs[0]).cuda())
        offs = None
    else:
        d = cp.persistence_batched([torch.from_numpy(a).cuda() for a in imgs])
        sizes = [a.size for a in imgs]
        offs = torch.tensor(np.concatenate([[0], np.cumsum(sizes)[:-1]]), dtype=torch.int64, device="cuda")
    n = int(sum(a.size for a in imgs))
    grad = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    ws_bytes = lib.cubical_persistence_loss_backward_workspace_size(n)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    rc = lib.cubical_persistence_loss_backward(
        ctypes.c_void_p(d.raw.data_ptr()), len(d), None, ctypes.c_float(TAU), ctypes.c_void_p(loss.data_ptr()),
        None if offs is None else ctypes.c_void_p(offs.data_ptr()), ctypes.c_void_p(grad.data_ptr()), n,
        ctypes.c_void_p(ws.data_ptr()), ws_bytes, None,
    )
    assert rc == 0
    return float(loss.item()), grad.cpu().numpy()


def _close(got, want):
    scale = max(1.0, float(np.abs(want).max()))
    np.testing.assert_allclose(got, want, rtol=RTOL, atol=RTOL * scale)


@pytest.mark.parametrize(
    "img",
    [
        workloads.rank_spaced(workloads.blurred((96, 120), 4.0, 31)),
        workloads.rank_spaced(workloads.blurred((20, 24, 18), 2.0, 32)),
        workloads.blurred((128, 100), 3.0, 33),
        workloads.uniform((40, 41), 34),
    ],
    ids=["2d_rank_spaced", "3d_rank_spaced", "2d_blurred", "2d_uniform"],
)
def test_loss_backward_matches_oracle_reference(cp, img):
    loss, g = _gpu_loss_grad(cp, [img])
    ref_loss, ref = _ref_grad(img)
    assert abs(loss - ref_loss) <= 1e-12 * max(1.0, ref_loss)
    _close(g, ref)


def test_loss_backward_batched_offsets(cp):
    items = workloads.batch(0, n2d=6, n3d=2, scale=0.15)
    loss, g = _gpu_loss_grad(cp, items)
    ref = np.concatenate([_ref_grad(a)[1] for a in items])
    ref_loss = sum(_ref_grad(a)[0] for a in items)
    assert abs(loss - ref_loss) <= 1e-9 * max(1.0, ref_loss)
    _close(g, ref)


def test_generic_backward_and_autograd(cp):
    img = workloads.rank_spaced(workloads.blurred((64, 72), 3.0, 35))
    x = torch.from_numpy(img).cuda().requires_grad_(True)
    b, d, raw = cp.diagram(x)
    fin = torch.isfinite(d)
    pers = (d - b)[fin]
    keep = pers > TAU
    loss = (pers[keep].double() ** 2).sum()
    loss.backward()
    ref_loss, ref = _ref_grad(img)
    assert abs(float(loss) - ref_loss) <= 1e-9 * max(1.0, ref_loss)
    _close(x.grad.detach().cpu().numpy().ravel(), ref)


def _in_loss_set(cp, img):
    d = cp.persistence(torch.from_numpy(img).cuda()).numpy()
    fin = d["death_cell"] >= 0
    pers = d["death"].astype(np.float64) - d["birth"].astype(np.float64)
    sel = fin & (pers > TAU)
    return set(zip(d["birth_pixel"][sel].tolist(), d["death_pixel"][sel].tolist()))


def test_finite_differences(cp):
    """Central differences with step 1e-3 on a rank-spaced field (gaps 2^-8).

    A step of 1e-3 never reorders pixels there, so the cell pairs do not
    change; a sample is valid when the set of (birth pixel, death pixel) pairs
    inside the loss is also unchanged at x+h and x-h (a persistence within h
    of the threshold can cross it).  Within a valid sample the loss is exactly
    quadratic along the coordinate, so the central difference over the
    representable step (x+h) - (x-h), in double precision, equals the
    derivative up to rounding.
    """
    img = workloads.rank_spaced(workloads.blurred((48, 56), 3.0, 36))
    _, g = _gpu_loss_grad(cp, [img])
    base = _in_loss_set(cp, img)
    rng = np.random.default_rng(0)
    flat = img.ravel()
    nz = np.flatnonzero(g)
    picks = np.concatenate([rng.choice(nz, min(40, len(nz)), replace=False), rng.choice(flat.size, 20, replace=False)])
    h = 1e-3
    valid = invalid = 0
    for p in picks:
        xp, xm = flat.copy(), flat.copy()
        xp[p] = np.float32(flat[p] + h)
        xm[p] = np.float32(flat[p] - h)
        xp, xm = xp.reshape(img.shape), xm.reshape(img.shape)
        if _in_loss_set(cp, xp) != base or _in_loss_set(cp, xm) != base:
            invalid += 1
            continue
        lp, _ = _gpu_loss_grad(cp, [xp])
        lm, _ = _gpu_loss_grad(cp, [xm])
        h_eff = (float(xp.ravel()[p]) - float(xm.ravel()[p])) / 2
        fd = (lp - lm) / (2 * h_eff)
        assert abs(fd - g[p]) <= 1e-3 * max(1.0, abs(g[p])), (p, fd, g[p])
        valid += 1
    assert valid >= 0.8 * len(picks), (valid, invalid)

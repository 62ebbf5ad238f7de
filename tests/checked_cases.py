"""The parity suite's small cases, run through the bounds-checked build of the
library (-DCP_CHECKED: every data-dependent device index is tested against
its array's size, a bad one flags the call instead of being used).  Run by
test_gpu_checked.py in a fresh process with CP_LIB_VARIANT=checked; prints
"checked ok" when every case equals the oracle and no call was flagged.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
import workloads  # noqa: E402

FIELDS = ("birth", "death", "birth_cell", "death_cell", "birth_pixel", "death_pixel", "dim")


def same(got, want, what):
    assert len(got) == len(want), f"{what}: {len(got)} pairs vs oracle {len(want)}"
    for k in FIELDS:
        assert np.array_equal(got[k], want[k]), f"{what}: field {k}"


def main():
    assert os.environ.get("CP_LIB_VARIANT") == "checked"
    import paper_2606_04801_gb300 as cp

    lib = cp.load()
    assert lib._name.endswith("libcp_gb300_checked.so"), lib._name
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(2024)
    cases = [workloads.uniform((64, 64), 0), workloads.blurred((128, 128, 128), 2.0, 1),
             workloads.uniform((48, 40, 36), 3)]
    for _ in range(12):
        nd = 2 if rng.random() < 0.5 else 3
        shape = tuple(int(v) for v in rng.integers(2, 40 if nd == 2 else 14, nd))
        cases.append(rng.integers(0, 3, shape).astype(np.float32) if rng.random() < 0.5
                     else rng.random(shape, dtype=np.float32))
    for img in cases:
        d = cp.persistence(torch.from_numpy(np.ascontiguousarray(img)).to(dev), with_stats=True)
        same(d.numpy(), oracle.persistence(img), f"V {img.shape}")
    for cross in (0, 1):  # both orders of the 2D top dimension
        assert lib.cp_set_tuning(5, cross) == 0
        items = workloads.batch(0, n2d=6, n3d=2, scale=0.15)
        got = cp.persistence_batched([torch.from_numpy(a).to(dev) for a in items]).numpy()
        for i, a in enumerate(items):
            same(got[got["item"] == i], oracle.persistence(a), f"batch item {i} cross {cross}")
    assert lib.cp_set_tuning(5, 0) == 0
    for img in (workloads.uniform((17, 23), 4), workloads.uniform((6, 7, 5), 5)):
        got = cp.persistence(torch.from_numpy(img).to(dev), filtration="T").numpy()
        same(got, oracle.persistence_t(img), f"T {img.shape}")
    for img in (workloads.uniform((9, 10, 11), 6), workloads.blurred((24, 20, 22), 1.5, 7)):
        got = cp.persistence_full(torch.from_numpy(img).to(dev)).numpy()
        same(got, oracle.persistence_full(img), f"full {img.shape}")
    # the slab split of the union-finds (with the boundary reduction) and the
    # Borůvka design of the union-finds
    for img, S in ((workloads.blurred((40, 24, 28), 1.5, 8), 3), (workloads.uniform((33, 29), 9), 4),
                   (workloads.uniform((20, 12, 14), 10), 20)):
        d = cp.persistence_slabs(torch.from_numpy(img).to(dev), S)
        same(d.numpy(), oracle.persistence(img), f"slabs {img.shape} S={S}")
    assert lib.cp_set_tuning(7, 1) == 0
    try:
        for img in (workloads.blurred((36, 30, 26), 1.5, 11), workloads.uniform((45, 51), 12)):
            d = cp.persistence(torch.from_numpy(img).to(dev))
            same(d.numpy(), oracle.persistence(img), f"boruvka {img.shape}")
    finally:
        lib.cp_set_tuning(7, 0)
    # the fused loss backward through the batched graph
    items = workloads.batch(0, n2d=3, n3d=1, scale=0.12)
    bp = cp.BatchedPersistence([a.shape for a in items], tau=0.05, graph=True)
    bp.load([torch.from_numpy(a).to(dev) for a in items])
    bp.step()
    assert bp.status()["rc"] == 0
    torch.cuda.synchronize()
    print("checked ok")


if __name__ == "__main__":
    main()

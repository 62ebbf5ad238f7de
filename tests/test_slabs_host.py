"""The slab split of the union-finds on the CPU: its restatement against the
oracle (every slab count, 2D and 3D, slabs that do not divide the extent),
the exchange step with two gloo ranks, and the library's argument checks."""
import ctypes
import os
import socket

import numpy as np
import pytest

import oracle
import slab_restatement as sr

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2606_04801_gb300 import _lib, slabs  # noqa: E402


def _images():
    rng = np.random.default_rng(11)
    yield rng.random((7, 6, 9)).astype(np.float32)
    yield rng.integers(0, 4, size=(6, 7, 5)).astype(np.float32)  # many ties: the index order decides
    yield rng.random((13, 11)).astype(np.float32)
    yield rng.integers(0, 3, size=(9, 12)).astype(np.float32)


@pytest.mark.parametrize("reduce", [False, True])
@pytest.mark.parametrize("S", [1, 2, 3, 4, 7, 20])
def test_split_equals_oracle(S, reduce):
    for img in _images():
        assert sr.split_pairs(img, S, reduce) == sr.oracle_pairs(oracle.persistence(img))


def test_boundary_reduction_sends_less():
    img = np.random.default_rng(3).random((12, 7, 6)).astype(np.float32)
    cx = sr.Complex(img)
    for dual in (False, True):
        full, none = sr.slab_records(cx, 2, range(2), dual, reduce=False)
        part, final = sr.slab_records(cx, 2, range(2), dual, reduce=True)
        assert not none and final
        assert len(part) + len(final) == len(full)


def test_whole_union_find_equals_oracle():
    for img in _images():
        assert sr.whole_pairs(img) == sr.oracle_pairs(oracle.persistence(img))


def _mutant_pairs(cx, S, drop):
    """The split with one planted mistake."""
    out = []
    for dual in (False, True):
        recs = cx.dual_records() if dual else cx.h0_records()
        crossing = [r for r in recs if sr.class_slab(cx, r[1], S) != sr.class_slab(cx, r[2], S)]
        touched = {r[1] for r in crossing} | {r[2] for r in crossing}
        send, final = [], []
        for s in range(S):
            internal = [r for r in recs if sr.class_slab(cx, r[1], S) == s and sr.class_slab(cx, r[2], S) == s]
            commits = sr.union_find(internal, dual)
            if drop == "commits":
                pass
            elif drop in ("own endpoints", "surviving side"):
                boundary = {}
                for rec, young, old in commits:
                    by = boundary.get(young, young in touched)
                    bo = boundary.get(old, old in touched)
                    if not (bo if drop == "surviving side" else by):
                        final.append((rec, young, old))
                    else:  # "own endpoints": the record's own endpoints instead of the classes' roots
                        send.append(rec if drop == "own endpoints" else (rec[0], young, old, rec[3]))
                    boundary[old] = by or bo
            else:
                send += [rec for rec, _, _ in commits]
            if drop != "crossing":
                send += [r for r in crossing if cx.slab_of_vertex(r[3], S) == s]
        out += sr.pairs_from_commits(cx, final, dual)
        out += sr.pairs_from_commits(cx, sr.union_find(send, dual), dual)
    return sorted(out)


@pytest.mark.parametrize("drop", ["crossing", "commits", "own endpoints", "surviving side"])
def test_split_mistakes_fail(drop):
    """Planted mistakes in the split change the pairs, so the parity tests
    above would see them: dropping the crossing records or a slab's commits;
    under the boundary reduction, sending a commit with its own endpoints
    instead of the two classes' roots, or deciding finality on the surviving
    class instead of the dying one."""
    want = [sr.oracle_pairs(oracle.persistence(img)) for img in _mutant_images()]
    got = [_mutant_pairs(sr.Complex(img), 3, drop) for img in _mutant_images()]
    assert got != want, drop


def _mutant_images():
    rng = np.random.default_rng(5)
    return [rng.random((8, 7, 6)).astype(np.float32), rng.random((9, 5, 7)).astype(np.float32),
            rng.random((15, 12)).astype(np.float32)]


def test_slab_of():
    assert list(slabs.slab_of(np.arange(10), 10, 3)) == [0, 0, 0, 0, 1, 1, 1, 2, 2, 2]
    assert list(slabs.slab_of(np.arange(3), 3, 5)) == [0, 1, 3]
    with pytest.raises(ValueError):
        slabs.slab_of(0, 0, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _to_records(recs):
    out = np.zeros(len(recs), dtype=slabs.RECORD_DTYPE)
    for i, r in enumerate(recs):
        out[i] = (r[0], r[1], r[2])
    return out


def _rank_main(rank, world, port, S, img, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        cx = sr.Complex(img)
        mine = [s for s in range(S) if s % world == rank]  # this rank's slabs
        result = []
        for dual in (False, True):
            sent, final = sr.slab_records(cx, S, mine, dual, reduce=True)
            local = sr.pairs_from_commits(cx, final, dual)  # written by the slab's own rank
            gathered = [None] * world if rank == 0 else None
            dist.gather_object(local, gathered, dst=0)
            merged = slabs.exchange(_to_records(sent))
            if rank != 0:
                assert merged is None
                continue
            assert np.all(merged["key"][1:] > merged["key"][:-1])
            recs = [(int(k), int(a), int(b)) for k, a, b in merged]
            result += sr.pairs_from_commits(cx, sr.union_find(recs, dual), dual)
            for g in gathered:
                result += g
            result.append(("records", dual, len(recs)))
        # a record sent twice is refused
        dup = _to_records(sr.slab_records(cx, S, [0], False)[0][:1])
        try:
            slabs.exchange(dup)
            refused = False
        except ValueError:
            refused = True
        out.put((rank, result, refused))
    finally:
        dist.destroy_process_group()


def _empty_rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        recs = np.zeros(0 if rank == 1 else 3, dtype=slabs.RECORD_DTYPE)
        if rank == 0:
            recs["key"] = [30, 10, 20]
            recs["age_a"] = [1, 2, 3]
        merged = slabs.exchange(recs)  # rank 1 sends nothing
        none = slabs.exchange(np.zeros(0, dtype=slabs.RECORD_DTYPE), dst=1)  # nobody sends anything
        out.put((rank, None if merged is None else merged.tolist(), None if none is None else len(none)))
    finally:
        dist.destroy_process_group()


def test_exchange_empty_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_empty_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted((q.get(timeout=10) for _ in range(world)), key=lambda r: r[0])
    assert res[0][1] == [(10, 2, 0), (20, 3, 0), (30, 1, 0)] and res[0][2] is None
    assert res[1][1] is None and res[1][2] == 0


@pytest.mark.parametrize("S", [2, 4])
def test_exchange_two_gloo_ranks(S):
    world = 2
    img = np.random.default_rng(21).random((9, 6, 7)).astype(np.float32)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, S, img, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    res = sorted((q.get(timeout=10) for _ in range(world)), key=lambda r: r[0])
    pairs = sorted(x for x in res[0][1] if x[0] != "records")
    assert pairs == sr.oracle_pairs(oracle.persistence(img))
    counts = [x for x in res[0][1] if x[0] == "records"]
    cx = sr.Complex(img)
    n_edges, n_facets = len(cx.edges), len(cx.facets)
    # the merge sees fewer records than the whole graph: each slab's cycles stay local
    assert counts[0][2] < n_edges and counts[1][2] < n_facets
    assert res[0][2] and not res[1][2]  # rank 0 saw the duplicate; rank 1 receives nothing


def test_slabs_workspace_argument_checks():
    lib = _lib.load()
    d = (ctypes.c_int64 * 3)(16, 12, 10)
    plain = lib.cubical_persistence_workspace_size(3, d, 0)
    assert lib.cubical_persistence_slabs_workspace_size(3, d, 4, 0) > plain
    assert lib.cubical_persistence_slabs_workspace_size(3, d, 0, 0) == 0
    assert lib.cubical_persistence_slabs_workspace_size(3, d, 1 << 17, 0) == 0
    assert lib.cubical_persistence_slabs_workspace_size(3, d, 1 << 16, 0) > plain
    d2 = (ctypes.c_int64 * 2)(16, 12)
    assert lib.cubical_persistence_slabs_workspace_size(2, d2, 3, 0) > 0
    old = lib.cp_get_tuning(5)
    try:
        assert lib.cp_set_tuning(5, 1) == 0
        assert lib.cubical_persistence_slabs_workspace_size(2, d2, 3, 0) == 0  # 2D cross-pruning: refused
        assert lib.cubical_persistence_slabs_workspace_size(3, d, 3, 0) > 0  # volumes do not use it
    finally:
        lib.cp_set_tuning(5, old)
    assert lib.cubical_persistence_slabs(3, None, d, 2, None, 0, None, None, None, 0, 0, None, None) == _lib.CP_ERR_ARG

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


@pytest.mark.parametrize("S", [1, 2, 3, 4, 7, 20])
def test_split_equals_oracle(S):
    for img in _images():
        assert sr.split_pairs(img, S) == sr.oracle_pairs(oracle.persistence(img))


def test_whole_union_find_equals_oracle():
    for img in _images():
        assert sr.whole_pairs(img) == sr.oracle_pairs(oracle.persistence(img))


def test_split_needs_both_record_kinds():
    """Dropping the crossing records, or a slab's commits, changes the pairs:
    the parity tests above would see either mistake."""
    img = np.random.default_rng(5).random((8, 7, 6)).astype(np.float32)
    cx = sr.Complex(img)
    want = sr.oracle_pairs(oracle.persistence(img))
    S = 3
    for drop in ("crossing", "commits"):
        out = []
        for dual in (False, True):
            recs = cx.dual_records() if dual else cx.h0_records()
            send = []
            for s in range(S):
                internal = [r for r in recs if sr.class_slab(cx, r[1], S) == s and sr.class_slab(cx, r[2], S) == s]
                if drop != "commits":
                    send += [rec for rec, _ in sr.union_find(internal, dual)]
                if drop != "crossing":
                    send += [r for r in recs if sr.class_slab(cx, r[1], S) != sr.class_slab(cx, r[2], S)
                             and cx.slab_of_vertex(r[3], S) == s]
            out += sr.pairs_from_commits(cx, sr.union_find(send, dual), dual)
        assert sorted(out) != want, drop


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
            sent = sr.slab_records(cx, S, mine, dual)
            merged = slabs.exchange(_to_records(sent))
            if rank != 0:
                assert merged is None
                continue
            assert np.all(np.diff(merged["key"].astype(np.float64)) >= 0)
            recs = [(int(k), int(a), int(b)) for k, a, b in merged]
            result += sr.pairs_from_commits(cx, sr.union_find(recs, dual), dual)
            result.append(("records", dual, len(recs)))
        # a record sent twice is refused
        dup = _to_records(sr.slab_records(cx, S, [0], False)[:1])
        try:
            slabs.exchange(dup)
            refused = False
        except ValueError:
            refused = True
        out.put((rank, result, refused))
    finally:
        dist.destroy_process_group()


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

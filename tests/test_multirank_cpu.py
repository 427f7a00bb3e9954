"""The multi-rank path on CPU: two gloo ranks on 127.0.0.1.

bench.py shards the work by image: every rank runs its own batch, with image
ids offset by rank, the same dictionary, and no collective on the data path;
the job's value is the summed work over the slowest rank's time.  These tests
check that host logic with gloo, and that sharding changes no result: the
code update of each image depends only on that image and its global id (the
mask hash key), so per-rank oracle steps equal one step over the union batch.
"""
import os
import socket

import numpy as np
import pytest

import bench
from oracle import reference as R
from paper_1909_00145_gb300 import inputs as I

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")

WORLD = 2


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = {}
        # shards of the two batch workloads (4 images per rank here)
        for name in ["c3", "c5"]:
            wl = dict(bench.WORKLOADS[name], n=4)
            H, W, ids, x, d = bench.make_inputs(wl, rank)
            got = [None] * world
            dist.all_gather_object(got, (ids.tolist(), H.tolist(), W.tolist(),
                                         float(np.abs(d).sum()), float(x[:64].sum())))
            res[name] = got
        # the job's time is the slowest rank's, its work the sum
        res["max"] = bench.reduce_over_ranks(1.5 + rank, "max", "cpu")
        res["sum"] = bench.reduce_over_ranks(10.0 * (rank + 1), "sum", "cpu")
        # oracle code step on this rank's shard of a tiny batch
        K, s = 4, 5
        cfg = R.Config(K=K, s=s, lam=0.3, p_num=1, p_den=2, seed=3)
        Hs, Ws = [12, 9], [10, 14]
        ids = [rank * 2, rank * 2 + 1]
        x = I.images(40 + rank, np.array(Hs), np.array(Ws)).astype(np.float64)
        d = I.filters(41, K, s).astype(np.float64)
        z = R.code_step(cfg, R.Batch(H=Hs, W=Ws, ids=ids), x, d, np.zeros(int(np.dot(Hs, Ws)) * K),
                        t=2, n_iters=6, step=0.02)
        shards = [None] * world
        dist.all_gather_object(shards, (x.tolist(), z.tolist()))
        res["shards"] = shards
        if rank == 0:
            np.save(os.path.join(out_dir, "res.npy"), np.array([res], dtype=object),
                    allow_pickle=True)
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    out = tmp_path_factory.mktemp("ranks")
    mp.start_processes(_worker, args=(WORLD, _free_port(), str(out)), nprocs=WORLD,
                       start_method="spawn")
    return np.load(os.path.join(out, "res.npy"), allow_pickle=True)[0]


def test_ranks_get_disjoint_image_ids_and_the_same_dictionary(results):
    for name in ["c3", "c5"]:
        ids = [set(r[0]) for r in results[name]]
        assert not (ids[0] & ids[1])
        assert sorted(ids[0] | ids[1]) == list(range(8))
        assert results[name][0][3] == results[name][1][3]  # same filters on every rank
        assert results[name][0][4] != results[name][1][4]  # different images
    # uneven batches: each rank draws its own sizes
    assert results["c5"][0][1] != results["c5"][1][1]


def test_job_time_is_the_max_and_work_the_sum(results):
    assert results["max"] == 2.5
    assert results["sum"] == 30.0


def test_shard_union_matches_the_oracle_on_the_whole_batch(results):
    K, s = 4, 5
    cfg = R.Config(K=K, s=s, lam=0.3, p_num=1, p_den=2, seed=3)
    Hs, Ws = [12, 9] * WORLD, [10, 14] * WORLD
    ids = list(range(2 * WORLD))
    x = np.concatenate([np.asarray(sh[0]) for sh in results["shards"]])
    z_shards = np.concatenate([np.asarray(sh[1]) for sh in results["shards"]])
    d = I.filters(41, K, s)
    z_all = R.code_step(cfg, R.Batch(H=Hs, W=Ws, ids=ids), x, d.astype(np.float64),
                        np.zeros(int(np.dot(Hs, Ws)) * K), t=2, n_iters=6, step=0.02)
    np.testing.assert_array_equal(z_shards, z_all)

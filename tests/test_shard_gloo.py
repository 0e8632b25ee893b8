"""Multi-rank split of one pairwise matrix, exercised with CPU ranks (gloo).

Each rank enumerates the pairs its shard owns (the host mirror of the
device's length sort and tile order), integrates them with the CPU oracle,
and the partial matrices are summed with an all-reduce.  The union must be
the full matrix with every pair computed exactly once.  A second test makes
one rank fail before the collective and checks that the survivor gets an
error from the collective within a short timeout instead of waiting forever.
"""
import os
import socket
import sys
import traceback

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, mode, q):
    try:
        sys.path.insert(0, ROOT)
        import datetime

        import torch
        import torch.distributed as dist

        import oracle
        from paper_2404_07183_gb300 import shard, synth
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=world,
                                timeout=datetime.timedelta(seconds=8))
        s = synth.random_set(70, seed=91, min_len=1, max_len=40)
        n = s.n
        owned = shard.shard_pairs(s.lengths(), rank, world)
        if mode == "backward":
            # this rank's share of d(sum G * F)/d(values, times): G restricted to
            # the pairs its tiles own, then one sum all-reduce of the gradients
            G = np.random.default_rng(5).standard_normal((n, n))
            Gr = np.zeros_like(G)
            for i, j in owned:
                Gr[i, j] = G[i, j]
                Gr[j, i] = G[j, i]
            gv, gt = oracle.backward(s, Gr, metric="l2", p=2.0)
            tv, tt = torch.from_numpy(gv), torch.from_numpy(gt)
            dist.all_reduce(tv)
            dist.all_reduce(tt)
            if rank == 0:
                wv, wt = oracle.backward(s, G, metric="l2", p=2.0)
                ev = float(np.max(np.abs(tv.numpy() - wv)) / np.max(np.abs(wv)))
                et = float(np.max(np.abs(tt.numpy() - wt)) / np.max(np.abs(wt)))
                q.put((rank, f"grad-ok={ev < 1e-12 and et < 1e-12}"))
            else:
                q.put((rank, "done"))
            dist.destroy_process_group()
            return
        part = np.zeros((n, n))
        for i, j in owned:
            v = oracle.integral(*s.pcf(i), *s.pcf(j), "l1")
            part[i, j] = v
            part[j, i] = v
        count = np.zeros((n, n))
        for i, j in owned:
            count[i, j] += 1
        if mode == "dead" and rank == 1:
            q.put((rank, "exited"))
            q.close()
            q.join_thread()      # make sure the message is sent before leaving
            os._exit(0)          # leaves without joining the collective
        t = torch.from_numpy(part)
        c = torch.from_numpy(count)
        try:
            dist.all_reduce(t)
            dist.all_reduce(c)
        except Exception as e:  # noqa: BLE001
            q.put((rank, "collective-error:" + type(e).__name__))
            return
        if rank == 0:
            full = oracle.matrix(s, metric="l1")
            ok = np.array_equal(t.numpy(), full)
            iu = np.triu_indices(n)
            once = bool(np.all(c.numpy()[iu] == 1))
            q.put((rank, f"ok={ok} once={once}"))
        else:
            q.put((rank, "done"))
        dist.destroy_process_group()
    except Exception:  # noqa: BLE001
        q.put((rank, "exception:" + traceback.format_exc()))


def _run(world, mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, mode, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        r, msg = q.get(timeout=60)
        out[r] = msg
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    return out


def test_two_ranks_cover_every_pair_once():
    out = _run(2, "ok")
    assert out[0] == "ok=True once=True", out


def test_three_ranks():
    out = _run(3, "ok")
    assert out[0] == "ok=True once=True", out


def test_backward_shards_all_reduce_to_the_gradient():
    out = _run(3, "backward")
    assert out[0] == "grad-ok=True", out


def test_dead_rank_is_detected_by_the_survivor():
    out = _run(2, "dead")
    assert out[1] == "exited"
    assert out[0].startswith("collective-error"), out


def test_shard_units_partition():
    from paper_2404_07183_gb300 import shard
    lens = np.random.default_rng(0).integers(1, 50, 150)
    allp = shard.shard_pairs(lens, 0, 1)
    assert len(allp) == 150 * 151 // 2
    parts = [shard.shard_pairs(lens, r, 4) for r in range(4)]
    assert sum(len(p) for p in parts) == len(allp)
    assert set().union(*parts) == allp
    with pytest.raises(ValueError):
        list(shard.shard_units(10, 4, 4))


def test_tile_order_mirror():
    """Queue order of the pairwise tiles: every upper-triangle tile once, the
    longest column band first, and inside a band of TILE_BAND column blocks each row
    block's tiles consecutive (so a row block is staged once per band)."""
    from paper_2404_07183_gb300 import shard
    for n in (1, 32, 33, 300, 1000, 5000):
        nb = (n + 31) // 32
        tiles = shard.tile_order(n)
        assert len(tiles) == nb * (nb + 1) // 2 == len(set(tiles))
        assert all(bi <= bj for bi, bj in tiles)
        assert tiles[0] == (nb - 1, nb - 1)
        k = 0
        for c1 in range(nb - 1, -1, -shard.TILE_BAND):
            c0 = max(0, c1 - shard.TILE_BAND + 1)
            band = tiles[k:k + sum(bj + 1 for bj in range(c0, c1 + 1))]
            k += len(band)
            assert {bj for _, bj in band} == set(range(c0, c1 + 1))
            rows = [bi for bi, _ in band]
            assert rows == sorted(rows, reverse=True)
        assert k == len(tiles)

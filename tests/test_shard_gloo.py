"""The row-sharded pass's host logic on CPU: gloo ranks, one exchange step.

Each rank folds its own share of the rows (``shard.row_shard``: whole blocks, dealt out
contiguously) into the oracle's accumulators (Alg. 4 step 7, Eq. 11), standing in for a
session; ``shard.merge_across_ranks`` gathers the checkpoints on rank 0 in rank order and
adds them there. The merged accumulators must equal those of one process over all rows
(the sketch is a sum over rows). The GPU merge itself (spca_merge with the shift rebase) is
covered by tests/test_gpu_merge.py; here all ranks use one shift, so merging is addition.
A rank that dies before the exchange (killed, no clean shutdown) makes the exchange fail on
rank 0 within the process group's timeout instead of waiting for it forever.
"""
import io
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1704_07669_gb300 import shard

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = ("H", "gram", "s", "sG")


@pytest.mark.parametrize("m,world,block", [(1000, 3, 64), (10, 4, 4), (4096, 2, 4096), (5, 3, 1)])
def test_row_shards_cover_every_row_once(m, world, block):
    seen = np.zeros(m, dtype=int)
    prev = 0
    for r in range(world):
        r0, r1 = shard.row_shard(m, world, r, block)
        assert r0 == prev and r0 <= r1
        assert r0 % block == 0 or r0 == m
        seen[r0:r1] += 1
        prev = r1
    assert prev == m and (seen == 1).all()


class _FakeSession:
    """Accumulators of the oracle behind the save_state / load_state interface."""

    def __init__(self, acc=None):
        self.acc = acc

    def save_state(self):
        bio = io.BytesIO()
        np.savez(bio, m=self.acc.m, **{k: getattr(self.acc, k) for k in KEYS})
        return bio.getvalue()

    def load_state(self, data):
        z = np.load(io.BytesIO(data))
        self.loaded = {k: z[k] for k in KEYS + ("m",)}


def _add(dst, src):
    for k in KEYS:
        setattr(dst.acc, k, getattr(dst.acc, k) + src.loaded[k])
    dst.acc.m += int(src.loaded["m"])


def _data(m, n, l):
    rng = np.random.default_rng(5)
    A = rng.standard_normal((m, n)) + rng.standard_normal(n)[None, :]
    Om = rng.standard_normal((n, l))
    c = A[:7].mean(axis=0)
    return A, Om, c


def _worker(rank, world, port, m, block, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist
    from oracle import spca as O
    from paper_1704_07669_gb300 import shard as sh
    dist.init_process_group("gloo", rank=rank, world_size=world)
    A, Om, c = _data(m, 12, 5)
    r0, r1 = sh.row_shard(m, world, rank, block)
    acc = O.ShiftedPass(Om, c=c, keep_G=False)
    for b0 in range(r0, r1, block):
        acc.add(A[b0:min(b0 + block, r1)])
    sess = _FakeSession(acc)
    root = sh.merge_across_ranks(sess, scratch=_FakeSession(), merge=_add)
    if root:
        out.put({k: getattr(acc, k) for k in KEYS} | {"m": acc.m})
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_accumulators_merge_to_one_pass(world):
    import sys
    sys.path.insert(0, ROOT)
    from oracle import spca as O
    m, block = 403, 32
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, m, block, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    A, Om, c = _data(m, 12, 5)
    whole = O.ShiftedPass(Om, c=c, keep_G=False)
    for b0 in range(0, m, block):
        whole.add(A[b0:b0 + block])
    assert got["m"] == m
    for k in KEYS:
        np.testing.assert_allclose(got[k], getattr(whole, k), rtol=1e-12, atol=1e-10)


def _worker_fail(rank, world, port, out):
    """Rank 1 dies before the exchange step (a crash: no clean shutdown); rank 0 must see
    an error from the exchange within the process group's timeout, not wait forever."""
    import datetime
    import sys
    import time
    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist
    from paper_1704_07669_gb300 import shard as sh
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        os._exit(3)
    t0 = time.time()
    try:
        sh.merge_across_ranks(_FakeSession(_Acc()), scratch=_FakeSession(), merge=_add)
        out.put(("no error", time.time() - t0))
    except Exception as exc:   # noqa: BLE001 - the failure is the expected outcome
        out.put((type(exc).__name__, time.time() - t0))
    out.close()
    out.join_thread()   # the result is sent before the hard exit
    os._exit(0)


class _Acc:
    def __init__(self):
        self.m = 1
        for k in KEYS:
            setattr(self, k, np.zeros(3))


def test_a_rank_that_dies_before_the_exchange_is_detected():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_fail, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    what, dt = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert procs[1].exitcode == 3
    assert what != "no error"
    assert dt < 60.0

"""GPU tests of the serving loop (include/spca_server.h): many sessions resident at once, row
blocks of uneven sizes arriving interleaved, admission against a device-memory budget. Each
result must be the one the same session gives alone: bit for bit on the FP32 path (its
kernels do not depend on how blocks are batched), within the tensor-core form's stated
tolerance (1e-3 on sigma) where the batching of blocks into launches changes the order of
FP32 accumulation. Closed and reserved sessions wait in the server's pool and are admitted
again by a reset of their state; a reused session gives the result of a new one.
"""
import time

import numpy as np
import pytest
import torch

import paper_1704_07669_gb300 as spca
from paper_1704_07669_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
WAIT = 120.0   # seconds: a request that takes longer fails the test instead of hanging it


@pytest.fixture(scope="module", autouse=True)
def _built():
    if DEV is None:
        pytest.fail("GPU tests need CUDA")
    spca.build.build()
    spca.lib()


def session_data(n, k, p, seed, rows):
    r = min(n, k + p + 30)
    A = synth.low_rank_plus_noise(rows, n, synth.spectrum("dec20", r), noise_std=1e-4, mean_std=0.5, seed=seed,
                                  device=DEV, dtype=torch.float32)
    return A.contiguous()


def blocks_of(rows, rng, lo=64, hi=900):
    out, r0 = [], 0
    while r0 < rows:
        b = int(rng.integers(lo, hi + 1))
        out.append((r0, min(rows, r0 + b)))
        r0 += b
    return out


def alone(A, k, p, seed, blocks, math):
    n = A.shape[1]
    with spca.Session(n, k, p, seed, math=math, max_block_rows=4096) as s:
        for a, b in blocks:
            s.update(A[a:b])
        return s.finalize()


# (n, k, p): the first ones fit a tensor-core kernel (FP16 form, including n = 12000 on the
# grouped kernel), the ones with l > 63 do not and are served by the FP32 path
MIX = [(300, 8, 8), (700, 10, 10), (1500, 20, 20), (3000, 30, 10), (6000, 50, 10), (9000, 40, 20),
       (900, 70, 10), (12000, 20, 10), (2500, 100, 20)]


def expected_math(n, k, p):
    """The server's automatic choice: the FP16 tensor-core pass where a tensor-core kernel takes
    the shape (session creation succeeds), the FP32 path elsewhere."""
    try:
        with spca.Session(n, k, p, 1, math="fp16", max_block_rows=4096):
            return "fp16"
    except spca.SpcaError:
        return "fp32"


def test_results_alone_and_in_the_mix():
    rng = np.random.default_rng(7)
    data, plans = [], []
    for i, (n, k, p) in enumerate(MIX):
        rows = int(rng.integers(1500, 3000))
        data.append(session_data(n, k, p, 500 + i, rows))
        plans.append(blocks_of(rows, rng))
    with spca.Server(max_block_rows=4096) as sv:
        ids = [sv.open(n, k, p, 900 + i) for i, (n, k, p) in enumerate(MIX)]
        # interleave the sessions' blocks at random, each session's own blocks in order
        cursors = [0] * len(MIX)
        tickets = []
        while any(c < len(pl) for c, pl in zip(cursors, plans)):
            i = int(rng.choice([j for j in range(len(MIX)) if cursors[j] < len(plans[j])]))
            a, b = plans[i][cursors[i]]
            tickets.append(sv.update(ids[i], data[i][a:b]))
            cursors[i] += 1
        outs = []
        for i, (n, k, p) in enumerate(MIX):
            sig, V = np.zeros(k), np.zeros((k, n))
            outs.append((sig, V, sv.finalize(ids[i], sig, V)))
        for t in tickets:
            sv.wait(t, WAIT)
        for sig, V, t in outs:
            sv.wait(t, WAIT)
        st = sv.stats()
        for i in ids:
            sv.close_session(i)
    assert st["updates_done"] == len(tickets) and st["finalizes_done"] == len(MIX)
    assert 0 < st["update_p50_ms"] <= st["update_p99_ms"]
    for i, (n, k, p) in enumerate(MIX):
        math = expected_math(n, k, p)
        s_alone, V_alone = alone(data[i], k, p, 900 + i, plans[i], math)
        sig, Vt, _ = outs[i]
        V = Vt.T
        if math == "fp32":
            assert np.array_equal(sig, s_alone) and np.array_equal(V, V_alone), (n, k, p)
        else:
            assert np.max(np.abs(sig - s_alone) / s_alone) <= 1e-3, (n, k, p)


def test_admission_waits_for_memory():
    n, k, p = 4000, 20, 10
    rows = 1024
    datas = [session_data(n, k, p, 40 + i, rows) for i in range(4)]
    with spca.Server(max_block_rows=4096) as probe:
        sid = probe.open(n, k, p, 1)
        probe.wait(probe.update(sid, datas[0][:256]), WAIT)
        footprint = probe.stats()["device_bytes_in_use"]
    assert footprint > 0
    with spca.Server(device_bytes=int(2.5 * footprint), max_block_rows=4096) as sv:
        ids = [sv.open(n, k, p, 60 + i) for i in range(4)]
        fins = []
        for i, sid in enumerate(ids):
            sv.update(sid, datas[i][:512])
            sv.update(sid, datas[i][512:])
            sig, V = np.zeros(k), np.zeros((k, n))
            fins.append((sig, V, sv.finalize(sid, sig, V)))
        sv.wait(fins[0][2], WAIT)
        sv.wait(fins[1][2], WAIT)
        st = sv.stats()
        assert st["sessions_admitted"] == 2 and st["sessions_waiting"] == 2
        assert st["device_bytes_in_use"] <= st["device_bytes_budget"]
        sv.close_session(ids[0])
        sv.close_session(ids[1])
        sv.wait(fins[2][2], WAIT)
        sv.wait(fins[3][2], WAIT)
        for i in range(4):
            s_alone, _ = alone(datas[i], k, p, 60 + i, [(0, 512), (512, rows)], expected_math(n, k, p))
            assert np.max(np.abs(fins[i][0] - s_alone) / s_alone) <= 1e-3


def test_rejects_bad_requests():
    with spca.Server(max_block_rows=1024) as sv:
        with pytest.raises(spca.SpcaError) as ei:
            sv.update(5, torch.zeros((4, 10), device=DEV))
        assert ei.value.status == 1
        with pytest.raises(spca.SpcaError) as ei:
            sv.open(10, 8, 8, 1)   # l > n
        assert ei.value.status == 1
        sid = sv.open(100, 4, 4, 1)
        with pytest.raises(spca.SpcaError) as ei:
            sv.update(sid, torch.zeros((2048, 100), device=DEV))   # more rows than max_block_rows
        assert ei.value.status == 1
        sv.close_session(sid)
        with pytest.raises(spca.SpcaError) as ei:
            sv.update(sid, torch.zeros((4, 100), device=DEV))   # closed
        assert ei.value.status == 1


def _wait_until(sv, key, value):
    t0 = time.perf_counter()
    while sv.stats()[key] != value:
        assert time.perf_counter() - t0 < WAIT, (key, sv.stats()[key], value)
        time.sleep(0.001)


@pytest.mark.parametrize("math", ["fp32", "auto"])
def test_pooled_sessions_are_reused_and_give_the_same_results(math):
    # three sessions reserved ahead of time serve two waves of three opens each: no session is
    # created after the reservation, and every result equals the same session run alone
    n, k, p, rows = 3000, 20, 10, 2048
    blocks = [(0, 700), (700, 1500), (1500, rows)]
    datas = [session_data(n, k, p, 70 + i, rows) for i in range(6)]
    kw = {} if math == "auto" else {"math": math}
    got = []
    with spca.Server(max_block_rows=4096, **kw) as sv:
        sv.wait(sv.reserve(n, k, p, 3), WAIT)
        st = sv.stats()
        assert (st["sessions_pooled"], st["sessions_created"], st["device_bytes_in_use"]) == (3, 3, 0)
        assert st["device_bytes_pooled"] > 0
        for wave in range(2):
            ids = [sv.open(n, k, p, 80 + 3 * wave + i) for i in range(3)]
            fins = []
            for i, sid in enumerate(ids):
                for a, b in blocks:
                    sv.update(sid, datas[3 * wave + i][a:b])
                sig, V = np.zeros(k), np.zeros((k, n))
                fins.append((sig, V, sv.finalize(sid, sig, V)))
            for sig, V, t in fins:
                sv.wait(t, WAIT)
                got.append((sig, V.T.copy()))
            for sid in ids:
                sv.close_session(sid)
            _wait_until(sv, "sessions_pooled", 3)
        st = sv.stats()
        assert (st["sessions_created"], st["admissions_from_pool"]) == (3, 6)
    used = expected_math(n, k, p) if math == "auto" else math
    for j, (sig, V) in enumerate(got):
        s_alone, V_alone = alone(datas[j], k, p, 80 + j, blocks, used)
        if used == "fp32":
            assert np.array_equal(sig, s_alone) and np.array_equal(V, V_alone), j
        else:
            assert np.max(np.abs(sig - s_alone) / s_alone) <= 1e-3, j


def test_an_admission_of_another_shape_frees_pooled_sessions():
    n, k, p = 4000, 20, 10
    with spca.Server(max_block_rows=4096) as probe:
        probe.wait(probe.reserve(n, k, p, 1), WAIT)
        footprint = probe.stats()["device_bytes_pooled"]
    assert footprint > 0
    data = session_data(n, 24, 6, 90, 1024)
    with spca.Server(device_bytes=int(2.5 * footprint), max_block_rows=4096) as sv:
        sv.wait(sv.reserve(n, k, p, 2), WAIT)
        assert sv.stats()["sessions_pooled"] == 2
        # same footprint (l = 30), another shape: the oldest pooled session makes room
        sid = sv.open(n, 24, 6, 91)
        sv.wait(sv.update(sid, data), WAIT)
        st = sv.stats()
        assert (st["sessions_pooled"], st["sessions_created"], st["admissions_from_pool"]) == (1, 3, 0)
        assert st["device_bytes_in_use"] + st["device_bytes_pooled"] <= st["device_bytes_budget"]
        with pytest.raises(spca.SpcaError) as ei:   # 2 of 2.5 footprints used: no room for a third
            sv.wait(sv.reserve(n, k, p, 1), WAIT)
        assert ei.value.status == 2
        assert sv.stats()["sessions_pooled"] == 1

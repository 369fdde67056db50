"""Failure handling without a GPU fault: every failure here is made on the host or by a
bounded wait that runs out, never by a bad address, a trap or a hang.

* allocation failures: SPCA_FAIL_ALLOC_AT=N makes the N-th device allocation of a
  spca_create report out-of-memory; for every N the call returns SPCA_E_NOMEM, frees what
  it had allocated (device memory back to where it was) and leaves the device usable;
* the bounded wait: spca_wait_selftest waits for a device counter that nothing writes and
  gives up after its limit with SPCA_E_TIMEOUT, promptly, with the context still usable;
  a short pipeline wait limit (SPCA_WAIT_LIMIT_MS) does not disturb a normal pass;
* a session torn down with work batched or in flight (a tensor-core session with pending
  blocks, an FP32 session with kernels queued) closes cleanly, and the next session on the
  device gives the same result as before.
"""
import os
import time

import numpy as np
import pytest
import torch

import paper_1704_07669_gb300 as spca
from paper_1704_07669_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
NOMEM, TIMEOUT = 2, 6


@pytest.fixture(scope="module", autouse=True)
def _built():
    if DEV is None:
        pytest.fail("GPU tests need CUDA")
    spca.build.build()
    spca.lib()


def _sigma(math, A, k=10, p=10, seed=7):
    with spca.Session(A.shape[1], k, p, seed, math=math) as s:
        for r0 in range(0, A.shape[0], 1000):
            s.update(A[r0:r0 + 1000])
        return s.finalize()[0]


@pytest.fixture(scope="module")
def data():
    return synth.low_rank_plus_noise(3000, 2500, synth.spectrum("dec20", 40), noise_std=1e-4, mean_std=0.3,
                                     seed=17, device=DEV, dtype=torch.float32)


@pytest.mark.parametrize("math", ["fp32", "fp16"])
def test_every_allocation_failure_of_create_is_reported_and_cleaned_up(math, data):
    ref = _sigma(math, data)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    n_fail = 0
    try:
        for at in range(200):
            os.environ["SPCA_FAIL_ALLOC_AT"] = str(at)
            try:
                s = spca.Session(2500, 10, 10, 7, math=math)
            except spca.SpcaError as exc:
                assert exc.status == NOMEM, exc
                n_fail += 1
                continue
            s.close()   # N is past the last allocation: the session was made whole
            break
        else:
            pytest.fail("spca_create kept failing")
    finally:
        os.environ.pop("SPCA_FAIL_ALLOC_AT", None)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert n_fail >= 10
    assert abs(free1 - free0) <= 8 << 20, (free0, free1)   # nothing held back (allocator granularity)
    assert np.array_equal(_sigma(math, data), ref)


def test_the_bounded_wait_runs_out_and_the_device_stays_usable(data):
    ref = _sigma("fp16", data)
    t0 = time.perf_counter()
    with pytest.raises(spca.SpcaError) as exc:
        spca.spca_wait_selftest(2_000_000)   # 2 ms
    dt = time.perf_counter() - t0
    assert exc.value.status == TIMEOUT
    assert dt < 2.0, dt
    assert np.array_equal(_sigma("fp16", data), ref)


def test_a_short_pipeline_wait_limit_leaves_a_normal_pass_alone(data):
    ref = _sigma("fp16", data)
    os.environ["SPCA_WAIT_LIMIT_MS"] = "200"
    try:
        got = _sigma("fp16", data)
    finally:
        os.environ.pop("SPCA_WAIT_LIMIT_MS", None)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("math", ["fp32", "fp16"])
def test_sessions_torn_down_with_work_pending(math, data):
    ref = _sigma(math, data)
    for _ in range(3):
        s = spca.Session(2500, 10, 10, 7, math=math)
        for r0 in range(0, 3000, 1000):
            s.update(data[r0:r0 + 1000])   # batched (tensor cores) or queued (FP32), not finalized
        s.close()
    assert np.array_equal(_sigma(math, data), ref)

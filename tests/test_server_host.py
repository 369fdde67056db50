"""The serving loop's host logic on CPU: csrc/server.cu compiled against a host-only stand-in
for the CUDA runtime and the session calls (tests/server_host/fake_device.cpp).

The stand-in folds each session's rows into a 64-bit FNV-1a digest (the 32-bit words of every
row, rows in order) and its finalisation writes values derived from the digest and the seed,
so each check below is exact: a session's result shows whether it received exactly its own
rows, in submission order, and whether the result reached the request that asked for it.
Streams complete after configurable delays, sessions are created slowly on request, and
creation can be made to fail, which exercises:
* many sessions fed from several threads at once, each result its own;
* sessions closed before the worker admitted them and replaced at once (the slot must not be
  handed out again while the worker still holds its requests); every request completes;
* the pool: reservations, reuse on admission, eviction for another shape, the budget;
* failed creation: only that session's requests fail;
* destroy with work queued: returns, and every session and allocation is freed;
* the close-and-replace stress built with ThreadSanitizer: no data race reported.
"""
import ctypes
import os
import shutil
import subprocess
import threading
import time

import numpy as np
import pytest

from paper_1704_07669_gb300 import ServerOptions, ServerStats

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"
MASK = (1 << 64) - 1
GOLD = 0x9E3779B97F4A7C15
OK, NOMEM = 0, 2
WAIT = 30.0


@pytest.fixture(scope="module")
def fake(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime_api.h")):
        pytest.skip("needs g++ and the CUDA headers")
    out = str(tmp_path_factory.mktemp("server_host") / "libserver_host.so")
    src = os.path.join(ROOT, "paper_1704_07669_gb300", "csrc")
    cmd = ["g++", "-std=c++17", "-O1", "-g", "-fPIC", "-shared", f"-I{CUDA_INC}", f"-I{ROOT}/include", f"-I{src}",
           "-x", "c++", os.path.join(src, "server.cu"),
           "-x", "c++", os.path.join(ROOT, "tests", "server_host", "fake_device.cpp"), "-o", out, "-lpthread",
           "-Wl,-Bsymbolic"]   # its own stand-ins, even where the process has loaded the CUDA runtime
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = ctypes.CDLL(out)
    vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    protos = {
        "spca_server_default_options": (None, [ctypes.POINTER(ServerOptions)]),
        "spca_server_create": (i32, [ctypes.POINTER(ServerOptions), ctypes.POINTER(vp)]),
        "spca_server_open": (i32, [vp, i64, i32, i32, u64, ctypes.POINTER(i32)]),
        "spca_server_reserve": (i32, [vp, i64, i32, i32, i32, ctypes.POINTER(u64)]),
        "spca_server_update": (i32, [vp, i32, vp, i64, i64, ctypes.POINTER(u64)]),
        "spca_server_finalize": (i32, [vp, i32, vp, vp, ctypes.POINTER(u64)]),
        "spca_server_wait": (i32, [vp, u64, ctypes.c_double]),
        "spca_server_close": (i32, [vp, i32]),
        "spca_server_get_stats": (i32, [vp, ctypes.POINTER(ServerStats)]),
        "spca_server_destroy": (i32, [vp]),
        "spca_server_last_error": (ctypes.c_char_p, []),
        "fake_set_delays": (None, [i64, i64, i64]),
        "fake_fail_create_every": (None, [i64]),
        "fake_live_allocations": (i64, []),
        "fake_live_sessions": (i64, []),
        "fake_creates": (i64, []),
    }
    for name, (res, args) in protos.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    return lib


@pytest.fixture(autouse=True)
def _reset_controls(request):
    if "fake" in request.fixturenames:
        lib = request.getfixturevalue("fake")
        lib.fake_set_delays(0, 0, 0)
        lib.fake_fail_create_every(0)
    yield


class Srv:
    def __init__(self, lib, device_bytes=0, math=-1):
        self.lib = lib
        opt = ServerOptions()
        lib.spca_server_default_options(ctypes.byref(opt))
        opt.device_bytes, opt.math = int(device_bytes), int(math)
        h = ctypes.c_void_p()
        assert lib.spca_server_create(ctypes.byref(opt), ctypes.byref(h)) == OK
        self.h = h.value

    def open(self, n, k, p, seed):
        sid = ctypes.c_int32(-1)
        assert self.lib.spca_server_open(self.h, n, k, p, seed, ctypes.byref(sid)) == OK
        return sid.value

    def reserve(self, n, k, p, count):
        t = ctypes.c_uint64(0)
        assert self.lib.spca_server_reserve(self.h, n, k, p, count, ctypes.byref(t)) == OK
        return t.value

    def update(self, sid, rows):
        t = ctypes.c_uint64(0)
        st = self.lib.spca_server_update(self.h, sid, rows.ctypes.data, rows.shape[0], rows.strides[0] // 4,
                                         ctypes.byref(t))
        assert st == OK, st
        return t.value

    def finalize(self, sid, sigma, V):
        t = ctypes.c_uint64(0)
        assert self.lib.spca_server_finalize(self.h, sid, sigma.ctypes.data, V.ctypes.data, ctypes.byref(t)) == OK
        return t.value

    def wait(self, ticket, timeout=WAIT):
        return self.lib.spca_server_wait(self.h, ticket, timeout)

    def wait_msg(self, ticket, timeout=WAIT):
        """(status, reason) of a request; the reason is read on the waiting thread."""
        st = self.lib.spca_server_wait(self.h, ticket, timeout)
        return st, (self.lib.spca_server_last_error() or b"").decode() if st != OK else ""

    def close_session(self, sid):
        assert self.lib.spca_server_close(self.h, sid) == OK

    def stats(self):
        st = ServerStats()
        assert self.lib.spca_server_get_stats(self.h, ctypes.byref(st)) == OK
        return {name: getattr(st, name) for name, _ in ServerStats._fields_}

    def destroy(self, limit=WAIT):
        """Destroy from a helper thread so that a worker that never stops fails the test."""
        th = threading.Thread(target=self.lib.spca_server_destroy, args=(self.h,), daemon=True)
        th.start()
        th.join(limit)
        assert not th.is_alive(), "spca_server_destroy did not return"


def digest(blocks, n):
    h = 1469598103934665603
    for b in blocks:
        for w in np.ascontiguousarray(b[:, :n]).view(np.uint32).ravel().tolist():
            h = ((h ^ w) * 1099511628211) & MASK
    return h


def expected(blocks, n, k, seed):
    h = digest(blocks, n)
    words = [(((h ^ seed) + i * GOLD) & MASK) >> 11 for i in range(k + n * k)]
    vals = np.array(words, dtype=np.float64) * (1.0 / 9007199254740992.0)
    return vals[:k], vals[k:]


def rows(rng, m, n, ld=None):
    a = rng.standard_normal((m, ld or n)).astype(np.float32)
    return a if ld is None else a[:, :n]


def test_every_session_gets_its_own_rows_and_result(fake):
    fake.fake_set_delays(200, 30, 300)
    base = fake.fake_live_allocations()
    sv = Srv(fake)
    rng = np.random.default_rng(1)
    shapes = [(int(rng.integers(8, 41)), int(rng.integers(2, 7)), int(rng.integers(0, 4))) for _ in range(24)]
    failures = []

    def client(idx):
        r = np.random.default_rng(100 + idx)
        try:
            for j in range(idx, len(shapes), 4):
                n, k, p = shapes[j]
                seed = 1000 + j
                sid = sv.open(n, k, p, seed)
                blocks, tickets = [], []
                for _ in range(int(r.integers(3, 12))):
                    ld = int(n + r.integers(0, 3)) if r.random() < 0.3 else None
                    b = rows(r, int(r.integers(1, 30)), n, ld)
                    blocks.append(b)
                    tickets.append(sv.update(sid, b))
                    if r.random() < 0.2:
                        time.sleep(0.0005)
                sig, V = np.zeros(k), np.zeros((k, n))
                tf = sv.finalize(sid, sig, V)
                for t in tickets:
                    assert sv.wait(t) == OK
                assert sv.wait(tf) == OK
                es, eV = expected(blocks, n, k, seed)
                assert np.array_equal(sig, es) and np.array_equal(V.ravel(), eV), j
                sv.close_session(sid)
        except Exception as exc:   # noqa: BLE001 - reported by the main thread
            failures.append(repr(exc))

    ths = [threading.Thread(target=client, args=(i,)) for i in range(4)]
    for t in ths:
        t.start()
    for t in ths:
        t.join(120)
    assert not failures, failures
    st = sv.stats()
    assert st["finalizes_done"] == len(shapes)
    sv.destroy()
    assert fake.fake_live_sessions() == 0
    assert fake.fake_live_allocations() == base


def test_sessions_closed_before_admission_and_replaced_at_once(fake):
    # slow creation: opens, closes and re-opens pile up before the worker admits them; a slot
    # must not be handed out again while the worker still holds its requests
    fake.fake_set_delays(1500, 20, 100)
    base = fake.fake_live_allocations()
    sv = Srv(fake)
    n, k, p = 16, 3, 1
    failures = []

    def client(idx):
        r = np.random.default_rng(7 + idx)
        try:
            pending = []
            for it in range(60):
                seed = 10000 * idx + it
                sid = sv.open(n, k, p, seed)
                b = rows(r, int(r.integers(1, 8)), n)
                pending.append((sv.update(sid, b), b))
                if it % 5 == 4:   # this one runs to a result
                    b2 = rows(r, 3, n)
                    pending.append((sv.update(sid, b2), b2))
                    sig, V = np.zeros(k), np.zeros((k, n))
                    tf = sv.finalize(sid, sig, V)
                    assert sv.wait(tf) == OK
                    es, eV = expected([b, b2], n, k, seed)
                    assert np.array_equal(sig, es) and np.array_equal(V.ravel(), eV)
                sv.close_session(sid)   # often before the worker has admitted it
            for t, _ in pending:
                assert sv.wait(t) == OK
        except Exception as exc:   # noqa: BLE001
            failures.append(repr(exc))

    ths = [threading.Thread(target=client, args=(i,)) for i in range(4)]
    for t in ths:
        t.start()
    for t in ths:
        t.join(180)
    assert not any(t.is_alive() for t in ths), "a client is still waiting"
    assert not failures, failures
    st = sv.stats()
    assert st["admissions_from_pool"] > 0
    assert st["sessions_created"] + st["admissions_from_pool"] == 4 * 60
    sv.destroy()
    assert fake.fake_live_sessions() == 0
    assert fake.fake_live_allocations() == base


def footprint(n, k, p):
    return ((1 << 20) | n * (k + p) * 8) + 8 * (n * k + k)


def test_reservations_reuse_and_eviction(fake):
    n, k, p = 64, 6, 2
    fp = footprint(n, k, p)
    sv = Srv(fake, device_bytes=int(2.5 * fp))
    assert sv.wait(sv.reserve(n, k, p, 2)) == OK
    st = sv.stats()
    assert (st["sessions_pooled"], st["sessions_created"], st["device_bytes_pooled"]) == (2, 2, 2 * fp)
    rng = np.random.default_rng(3)
    # same shape: taken from the pool, reset for its own seed
    sid = sv.open(n, k, p, 77)
    b = rows(rng, 5, n)
    assert sv.wait(sv.update(sid, b)) == OK
    sig, V = np.zeros(k), np.zeros((k, n))
    assert sv.wait(sv.finalize(sid, sig, V)) == OK
    assert np.array_equal(sig, expected([b], n, k, 77)[0])
    st = sv.stats()
    assert (st["sessions_pooled"], st["admissions_from_pool"], st["sessions_created"]) == (1, 1, 2)
    # another shape of the same footprint: the pooled session makes room
    sid2 = sv.open(n, k + 1, p - 1, 78)
    assert sv.wait(sv.update(sid2, b)) == OK
    st = sv.stats()
    assert (st["sessions_pooled"], st["sessions_created"]) == (0, 3)
    assert st["device_bytes_in_use"] + st["device_bytes_pooled"] <= st["device_bytes_budget"]
    # no room for a reservation
    assert sv.wait(sv.reserve(n, k, p, 1)) == NOMEM
    # closing returns the sessions to the pool, and a reservation of the same shape still fits none
    sv.close_session(sid)
    sv.close_session(sid2)
    t0 = time.perf_counter()
    while sv.stats()["sessions_pooled"] != 2:
        assert time.perf_counter() - t0 < WAIT
        time.sleep(0.001)
    assert sv.stats()["device_bytes_in_use"] == 0
    sv.destroy()
    assert fake.fake_live_sessions() == 0


def test_a_failed_creation_fails_only_that_sessions_requests(fake):
    fake.fake_set_delays(0, 10, 50)
    fake.fake_fail_create_every(3)
    first = fake.fake_creates()
    sv = Srv(fake)
    rng = np.random.default_rng(5)
    n, k, p = 12, 2, 2
    sessions = []
    for i in range(6):
        sid = sv.open(n + i, k, p, 500 + i)   # distinct shapes: every admission creates
        b = rows(rng, 4, n + i)
        sig, V = np.zeros(k), np.zeros((k, n + i))
        sessions.append((sid, b, sig, V, sv.update(sid, b), sv.finalize(sid, sig, V)))
    statuses = []
    for i, (sid, b, sig, V, tu, tf) in enumerate(sessions):
        su, sf = sv.wait(tu), sv.wait(tf)
        statuses.append((su, sf))
        if su == OK:
            assert sf == OK and np.array_equal(sig, expected([b], n + i, k, 500 + i)[0])
        else:
            assert (su, sf) == (NOMEM, NOMEM)
        sv.close_session(sid)
    failed = [i for i, s in enumerate(statuses) if s[0] != OK]
    assert failed == [i for i in range(6) if (first + i + 1) % 3 == 0]
    sv.destroy()
    assert fake.fake_live_sessions() == 0


def test_destroy_with_work_queued_frees_everything(fake):
    fake.fake_set_delays(300, 200, 500)
    base = fake.fake_live_allocations()
    sv = Srv(fake)
    rng = np.random.default_rng(9)
    keep = []
    for i in range(12):
        n = 10 + i
        sid = sv.open(n, 2, 1, i)
        for _ in range(3):
            b = rows(rng, 6, n)
            keep.append(b)
            sv.update(sid, b)
        sig, V = np.zeros(2), np.zeros((2, n))
        keep += [sig, V]
        sv.finalize(sid, sig, V)
    sv.destroy()
    assert fake.fake_live_sessions() == 0
    assert fake.fake_live_allocations() == base


def test_stress_under_thread_sanitizer(tmp_path):
    """The close-and-replace stress as a C++ program built with ThreadSanitizer: no data race
    reported, every request completed, every result its session's own, nothing left alive."""
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime_api.h")):
        pytest.skip("needs g++ and the CUDA headers")
    src = os.path.join(ROOT, "paper_1704_07669_gb300", "csrc")
    exe = str(tmp_path / "stress")
    cmd = ["g++", "-std=c++17", "-O1", "-g", "-fsanitize=thread", f"-I{CUDA_INC}", f"-I{ROOT}/include", f"-I{src}",
           "-x", "c++", os.path.join(src, "server.cu"),
           "-x", "c++", os.path.join(ROOT, "tests", "server_host", "fake_device.cpp"),
           "-x", "c++", os.path.join(ROOT, "tests", "server_host", "stress_driver.cpp"), "-o", exe, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "tsan" in r.stderr.lower():
        pytest.skip("ThreadSanitizer runtime not available")
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, TSAN_OPTIONS="halt_on_error=0 second_deadlock_stack=1")
    r = subprocess.run([exe], capture_output=True, text=True, timeout=240, env=env)
    assert "ThreadSanitizer" not in r.stderr, r.stderr[-4000:]
    assert r.returncode == 0, (r.stdout, r.stderr[-2000:])
    assert r.stdout.startswith("failures 0"), r.stdout


def test_a_failed_request_reports_its_own_reason(fake):
    """Each failed request carries the reason of the session that ran it: a refused update of
    one session and the failed creation of another are told apart, and the other requests of
    the first session still complete."""
    fake.fake_set_delays(0, 10, 20)
    first = fake.fake_creates()
    fake.fake_fail_create_every(first + 2)   # the second session made below fails
    sv = Srv(fake)
    rng = np.random.default_rng(12)
    n, k, p = 10, 2, 1
    a = sv.open(n, k, p, 71)
    assert sv.wait(sv.update(a, rows(rng, 4, n))) == OK   # a is created (the first creation)
    b = sv.open(n + 1, k, p, 72)                          # the second creation fails
    bad = sv.update(a, rows(rng, 97, n))                  # refused by a's session (97 rows)
    tb = sv.update(b, rows(rng, 4, n + 1))
    good = rows(rng, 5, n)
    tg = sv.update(a, good)
    st_bad, msg_bad = sv.wait_msg(bad)
    st_b, msg_b = sv.wait_msg(tb)
    assert st_bad == 1 and "update rejected" in msg_bad and "seed 71" in msg_bad, msg_bad
    assert st_b == NOMEM and "could not be created" in msg_b and "seed 71" not in msg_b, msg_b
    assert sv.wait(tg) == OK
    sv.close_session(a)
    sv.close_session(b)
    sv.destroy()
    assert fake.fake_live_sessions() == 0

"""Benchmark: sketch-pass throughput of the single-pass randomized PCA on one GB300.

A step is one whole pass of the method over the 100000 x 10000 FP32
low-rank-plus-noise workload (k = 50, p = 10, 4096-row blocks, column centring):
Omega regenerated (spca_reset), 25 row blocks folded in (spca_update) and the
FP64 finalisation (spca_finalize). The data (4.0 GB) is larger than L2, so no
L2 flush is needed between steps. The timed form is the FP16 tensor-core pass
(G split into two FP16 terms), the one that holds every sigma within 1e-3 of
the oracle; the FP32 and BF16 forms are measured on the same data and reported
under "forms".

Prints one JSON line. `value` is GB/s of A (as stored) per second of device
time; `e2e` is the same metric through the C ABI with host (pinned) buffers and
the host-to-device copies inside the timed region. `--impl reference` times the
FP64 CPU oracle on a bounded sample of the same workload instead.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sketch-pass GB/s of A + roofline %, FP32 vs tensor-core at ≤1e-3 σ error; p99"
WORKLOAD = "100000x10000 f32 low-rank+noise (sigma_i=10^(-i/20), i<=200; noise 1e-4 sigma_1; column means N(0,1)), " \
           "k=50 p=10 (l=60), 4096-row blocks, column-centred"
M, N, K, P, BLOCK = 100_000, 10_000, 50, 10, 4096
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0,
                "source": "fallback"}


# ------------------------------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "50", "-i", str(self.gpu_index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------------ CPU oracle

def oracle_pass_seconds(A_rows_f32, seed):
    """Time the FP64 oracle (sketch loop + Alg. 4 finalisation) on the given rows."""
    from oracle import spca as O
    A64 = np.asarray(A_rows_f32, dtype=np.float64)
    t0 = time.perf_counter()
    O.single_pass_pca(A64, K, P, seed, BLOCK, finalize="blocked", omega_form="f32")
    return time.perf_counter() - t0


OMEGA_FORM = {"fp32": "f32", "fp16": "f16", "bf16": "bf16"}


def oracle_precision(A_dev, seed, results):
    """The error of each timed form against the FP64 oracle on the whole timed matrix (the same
    stored rows, Omega in the form's operand format): sigma_i relative error (all k and the
    leading 10) and the sine of the largest principal angle between the leading 10 directions.
    Part of the CPU oracle leg of the benchmark (host cores, outside every timed region)."""
    from oracle import spca as O
    A64 = A_dev.cpu().double().numpy()
    out = {}
    for math_name, (sigma, V) in results.items():
        t0 = time.perf_counter()
        ref = O.single_pass_pca(A64, K, P, seed, BLOCK, center_columns=True, finalize="gram",
                                omega_form=OMEGA_FORM[math_name])
        rel = np.abs(sigma - ref["sigma"]) / ref["sigma"]
        out[math_name] = {"sigma_rel_max": float(rel.max()), "sigma_rel_lead10": float(rel[:10].max()),
                          "sin_theta_V10": float(O.max_principal_sine(V[:, :10], ref["V"][:, :10])),
                          "every_sigma_within_1e-3": bool(rel.max() <= 1e-3),
                          "oracle_s": time.perf_counter() - t0}
        if math_name == "bf16":
            out[math_name]["note"] = ("BF16 operands round the shifted rows to 8 significant bits, which moves the "
                                      "tail sigma by more than 1e-3 (an FP64 model with exact accumulation moves "
                                      "them as much); the gate is sigma >= sigma_1/10 within 1e-3")
    return out


def cpu_baseline(A_sample_f32, seed, what):
    secs = oracle_pass_seconds(A_sample_f32, seed)
    gb = A_sample_f32.shape[0] * A_sample_f32.shape[1] * 4 / 1e9
    return {"value": gb / secs, "unit": "GB/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{what}: {A_sample_f32.shape[0]} of {M} rows x {N} (f32 stored, FP64 compute), "
                      f"Alg. 4 sketch loop + blocked finalisation, {secs:.2f} s"}


# ------------------------------------------------------------------------------------------ arms

def dist_setup():
    """Rank layout from the torchrun environment; one process per GPU, each over its own rows."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    """The largest of each rank's x (the job's time is its slowest rank's)."""
    if ws == 1:
        return x
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args):
    # the oracle runs on rank 0's host cores only; other ranks exit without work
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    from paper_1704_07669_gb300 import synth
    rows = 8192
    w = synth.workload_c2(m=rows, n=N, device="cpu")
    A = w["A"].numpy()
    for _ in range(args.warmup):
        oracle_pass_seconds(A, w["seed"])
    times = [oracle_pass_seconds(A, w["seed"]) for _ in range(args.steps)]
    gb = rows * N * 4 / 1e9
    t = float(np.sum(times))
    value = gb * args.steps / t
    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD + f"; each step a {rows}-row sample of the same recipe",
                       "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{rows} rows x {N} per step, FP64 numpy oracle (Alg. 4)"},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def roofline_for(math_name, prof, bytes_total, rows_total, pk):
    """Roofline of the dominant kernel of the pass for one arithmetic form."""
    l = K + P
    if math_name == "fp32":
        # the FP32 path is bound by the FMA pipe: each contraction is 2 m n l flops per pass
        dom = max(("g_partial", "h_partial"), key=lambda k_: prof[k_][0])
        dom_ms, dom_launches = prof[dom]
        flops = 2.0 * rows_total * N * l
        achieved = flops / (dom_ms * 1e-3) / 1e12
        alu_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * pk["sm_max_mhz"] * 1e6 / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved / alu_peak,
                "traffic": None, "kernel": dom, "kernel_avg_ms": dom_ms / max(dom_launches, 1),
                "peak_note": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x max SM clock"}
    # the fused tensor-core kernel reads every byte of A once: HBM-bound
    dom = "tc_sketch"
    dom_ms, dom_launches = prof[dom]
    achieved = bytes_total / (dom_ms * 1e-3) / 1e9
    traffic = None
    rec = traffic_record(math_name)
    if rec is not None:
        traffic = rec["dram_bytes_per_row"] * rows_total / max(dom_launches, 1)
    return {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / pk["hbm_gbs"], "traffic": traffic, "kernel": dom,
            "kernel_avg_ms": dom_ms / max(dom_launches, 1),
            "peak_note": f"HBM copy bandwidth ({pk['source']}), algorithmic bytes = A read once per pass",
            "algorithmic_bytes_per_launch": bytes_total / max(dom_launches, 1)}


TC_KERNEL_SOURCES = ("sketch_grp.cu", "tc_ptx.cuh")   # the grouped kernel that runs the pass


def tc_source_sha256():
    import hashlib
    h = hashlib.sha256()
    for name in TC_KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1704_07669_gb300", "csrc", name), "rb").read())
    return h.hexdigest()


def traffic_record(math_name):
    """DRAM bytes per row of the fused kernel from a committed ncu capture, if it was taken on
    the kernel sources as they are now (the record stores their SHA-256)."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "tc_sketch_traffic.json")))[math_name]
        if tc_source_sha256() != rec["source_sha256"]:
            return None
        return rec
    except Exception:
        return None


def run_form(spca, math_name, A, seed, stream, steps_arg, warmup, ws):
    """Time whole passes (reset, all row blocks, finalize) of one arithmetic form. With N ranks
    each rank passes over its own rows and the exchange step merges every rank's sketch into
    rank 0's, which alone finalizes (the rows of all ranks form one matrix)."""
    from paper_1704_07669_gb300 import shard
    m = A.shape[0]
    dev = A.device
    sess = spca.Session(N, K, P, seed, math=math_name, stream=stream)
    scratch = shard.scratch_like(sess) if ws > 1 and torch.distributed.get_rank() == 0 else None
    sigma_d = torch.zeros(K, dtype=torch.float64, device=dev)
    V_d = torch.zeros((K, N), dtype=torch.float64, device=dev)

    def step():
        spca.spca_reset(sess.handle, seed)
        for r0 in range(0, m, BLOCK):
            spca.spca_update(sess.handle, A[r0:r0 + BLOCK])
        if ws > 1 and not shard.merge_across_ranks(sess, scratch=scratch):
            return
        spca.spca_finalize(sess.handle, sigma_d, V_d, out_on_device=True)

    for _ in range(max(warmup, 1)):
        step()
    torch.cuda.synchronize()
    steps = steps_arg
    if steps is None:
        t0 = time.perf_counter()
        step()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        steps = max(10, int(math.ceil(3.0 / max(dt, 1e-4))))
    spca.spca_clear_profile(sess.handle)
    spca.spca_set_profiling(sess.handle, True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]   # per-pass times
    barrier(ws)
    torch.cuda.synchronize()
    ev0.record(stream)
    marks[0].record(stream)
    for i in range(steps):
        step()
        marks[i + 1].record(stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    spca.spca_set_profiling(sess.handle, False)
    ms = max_over_ranks(ev0.elapsed_time(ev1), ws)
    per_pass = np.array([marks[i].elapsed_time(marks[i + 1]) for i in range(steps)])
    prof = sess.profile()
    return sess, step, {"ms": ms, "steps": steps, "prof": prof, "sigma": sigma_d.cpu().numpy(),
                        "V": V_d.cpu().numpy().T,
                        "pass_ms_p50": float(np.percentile(per_pass, 50)),
                        "pass_ms_p99": float(np.percentile(per_pass, 99))}


SERVING = "64 sessions, n log-uniform in [512, 32768], l in {20, 40, 80, 140} (k = l - 10), FP32 row blocks " \
          "of 256-4096 rows (uniform), low-rank-plus-noise per session seed, Poisson arrivals"


def tensor_core_takes(spca, n, l):
    """Whether the serving loop's automatic choice puts a session of this shape on the tensor cores."""
    try:
        with spca.Session(n, l - 10, 10, 1, math="fp16", max_block_rows=4096):
            return True
    except spca.SpcaError:
        return False


def run_serving(spca, dev, seconds=3.0, loads=(0.25, 0.5, 0.75), seed=17040769 + 4):
    """The serving loop under stated loads: first the saturation throughput (every block of a
    fixed plan queued at once), then, per load, a fresh server with Poisson arrivals at that
    fraction of saturation for `seconds`, then one finalisation per session. Returns p50/p99
    latencies and throughput per load (the 50 % load also at the top level)."""
    rng = np.random.default_rng(seed)
    S = 64
    ns = np.exp(rng.uniform(np.log(512), np.log(32768), S)).astype(np.int64)
    ls = rng.choice([20, 40, 80, 140], S)
    gen = torch.Generator(device=dev)
    pools = []
    for i in range(S):
        n, l = int(ns[i]), int(ls[i])
        gen.manual_seed(seed * 100 + i)
        r = l + 20
        U = torch.randn(4096, r, generator=gen, device=dev) / 64.0
        V = torch.randn(int(n), r, generator=gen, device=dev) / math.sqrt(n)
        sig = 10.0 ** (-torch.arange(r, device=dev, dtype=torch.float32) / 20.0)
        A = (U * sig) @ V.T
        A += 1e-4 / (64.0 + math.sqrt(n)) * torch.randn(4096, int(n), generator=gen, device=dev)
        A += torch.randn(1, int(n), generator=gen, device=dev)
        pools.append(A.contiguous())
    torch.cuda.synchronize()

    def block(i):
        b = int(rng.integers(256, 4097))
        return pools[i][:b], 4.0 * b * int(ns[i])

    out = {"workload": SERVING, "sessions": S}
    with spca.Server(max_block_rows=4096) as sv:
        # saturation: 8 blocks per session queued at once (a server of its own)
        ids = [sv.open(int(ns[i]), int(ls[i]) - 10, 10, 900 + i) for i in range(S)]
        for i in range(S):   # admit every session before the clock starts
            sv.wait(sv.update(ids[i], pools[i][:256]), 300.0)
        plan = [i for i in range(S) for _ in range(8)]
        rng.shuffle(plan)
        t0 = time.perf_counter()
        nbytes = 0.0
        tickets = []
        for i in plan:
            rows, b = block(i)
            nbytes += b
            tickets.append(sv.update(ids[i], rows))
        for t in tickets:
            sv.wait(t, 300.0)
        sat = nbytes / (time.perf_counter() - t0) / 1e9
    mean_bytes = nbytes / len(plan)
    out["saturation_GBps"] = sat
    sweep = []
    for load in loads:
        sweep.append(_serving_phase(spca, sat, mean_bytes, load, seconds, ns, ls, S, block, rng, pools))
    mid = next((x for x in sweep if abs(x["load"] - 0.5) < 1e-9), sweep[0])
    out.update({k_: v for k_, v in mid.items() if k_ != "load"})
    out["load_sweep"] = sweep
    out.update({"latency_note": "percentiles over each Poisson phase (sessions closed and replaced inside it), "
                                "one 256-row admission block per session before it and the final "
                                "finalize of every session",
                "tc_sessions": int(sum(1 for i in range(S) if tensor_core_takes(spca, int(ns[i]), int(ls[i]))))})
    del pools
    return out


def _serving_phase(spca, sat, mean_bytes, load, seconds, ns, ls, S, block, rng, pools, churn_every=25, churned=8):
    """One Poisson phase of the serving measurement on a fresh server (all sessions admitted
    first). Sessions also come and go inside the timed window: every `churn_every`-th arrival
    closes one of the first `churned` sessions (its client leaves without a result) and opens a
    new session of the same shape in its place, fed a first 256-row block at once; one session
    per such shape is reserved before the window, so these admissions reset pooled sessions
    instead of allocating. Finalisations run after the window (all sessions at once): inside it,
    their single-block kernels would hold SMs that the cooperative tensor-core launches wait
    for."""
    rate = load * sat * 1e9 / mean_bytes          # requests per second
    with spca.Server(max_block_rows=4096) as sv:
        ids = [sv.open(int(ns[i]), int(ls[i]) - 10, 10, 900 + i) for i in range(S)]
        for i in range(S):
            sv.wait(sv.update(ids[i], pools[i][:256]), 300.0)
        for i in range(churned):
            sv.wait(sv.reserve(int(ns[i]), int(ls[i]) - 10, 10, 1), 300.0)
        base = sv.stats()
        # Poisson arrivals at `load` of saturation
        tickets, fins = [], []
        t_next = time.perf_counter()
        t_end = t_next + seconds
        nbytes = 0.0
        n_req = n_churn = 0
        t0 = time.perf_counter()
        while t_next < t_end:
            while time.perf_counter() < t_next:
                pass
            n_req += 1
            if n_req % churn_every == 0:
                i = int(rng.integers(0, churned))
                k = int(ls[i]) - 10
                sv.close_session(ids[i])   # the client leaves without a result
                n_churn += 1
                ids[i] = sv.open(int(ns[i]), k, 10, 5000 + n_churn)
                tickets.append(sv.update(ids[i], pools[i][:256]))   # its first rows, as at admission
                nbytes += 4.0 * 256 * int(ns[i])
            else:
                i = int(rng.integers(0, S))
                rows, b = block(i)
                nbytes += b
                tickets.append(sv.update(ids[i], rows))
            t_next += rng.exponential(1.0 / rate)
        for t in tickets:
            sv.wait(t, 300.0)
        wall = time.perf_counter() - t0
        for i in range(S):
            k = int(ls[i]) - 10
            sig_h, V_h = np.zeros(k), np.zeros((k, int(ns[i])))
            fins.append((sig_h, V_h, sv.finalize(ids[i], sig_h, V_h)))
        for f in fins:
            sv.wait(f[2], 300.0)
        st = sv.stats()
    n_upd = st["updates_done"] - base["updates_done"]
    return {"load": load, "offered_load": f"{load:.0%} of saturation, Poisson, {rate:.0f} blocks/s",
            "updates": int(n_upd), "achieved_GBps": nbytes / wall / 1e9,
            "update_p50_ms": st["update_p50_ms"], "update_p99_ms": st["update_p99_ms"],
            "finalize_p50_ms": st["finalize_p50_ms"], "finalize_p99_ms": st["finalize_p99_ms"],
            "sessions_replaced_in_window": n_churn,
            "admissions_from_pool_in_window": int(st["admissions_from_pool"] - base["admissions_from_pool"]),
            "sessions_created_in_window": int(st["sessions_created"] - base["sessions_created"]),
            "device_budget_bytes": st["device_bytes_budget"]}


def h2d_copy_gbs(host, dev):
    """A plain pinned host-to-device copy's rate (three copies after two warm-up copies)."""
    buf = torch.empty(host.shape, dtype=host.dtype, device=dev)
    for _ in range(2):
        buf.copy_(host, non_blocking=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        buf.copy_(host, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    del buf
    return 3 * host.numel() * host.element_size() / (e0.elapsed_time(e1) * 1e-3) / 1e9


def run_streamed(spca, dev, math_name):
    """The 937500 x 40000 FP32 stream (150 GB, larger than the device) from pinned host memory
    through spca_update with host pointers (the session's double-buffered copies), against a
    plain pinned host-to-device copy measured in the same run."""
    from paper_1704_07669_gb300 import synth
    w = synth.workload_c4(device=dev)
    pool, schedule = w["pool"], w["schedule"]
    n, k, p, seed = w["n"], w["k"], w["p"], w["seed"]
    torch.cuda.synchronize()
    copy_gbs = h2d_copy_gbs(pool[0], dev)
    rows_np = [b.numpy() for b in pool]
    with spca.Session(n, k, p, seed, math=math_name) as s:
        s.update(rows_np[0][:1])         # the staging buffers are made by the first host update
        s.sync()
        s.reset(seed)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for b, rows in schedule:
            s.update(rows_np[b][:rows])
        sigma, V = s.finalize()          # includes the result's copy to the host
        secs = time.perf_counter() - t0
        desc = spca.spca_describe(s.handle)
    nbytes = 4.0 * w["m"] * n
    del pool, rows_np
    return {"workload": w["name"], "math": math_name, "value": nbytes / secs / 1e9, "unit": "GB/s",
            "seconds": secs, "h2d_copy_GBps": copy_gbs, "frac_of_h2d": nbytes / secs / 1e9 / copy_gbs,
            "kernel": desc, "note": "end to end: host rows -> device by the session's pinned staging, the pass, "
                                    "the FP64 finalisation, sigma and V back to the host"}


def run_ours(args):
    import paper_1704_07669_gb300 as spca
    from paper_1704_07669_gb300 import build as spca_build
    from paper_1704_07669_gb300 import synth

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    spca_build.build()
    spca.lib()
    pk = peaks()
    m = args.m

    # each rank its own rows of the workload's recipe; one Omega (one session seed) for all ranks
    w = synth.workload_c2(m=m, device=dev, seed=synth.SEED_BASE + 1 + rank)
    A = w["A"]
    seed = synth.SEED_BASE + 1
    stream = torch.cuda.Stream(device=dev)
    bytes_A = m * N * 4

    # the other arithmetic forms, measured first on the same data (reported under "forms")
    forms = {}
    results = {}
    for other in [f for f in args.forms.split(",") if f and f != args.math]:
        s_o, _, r_o = run_form(spca, other, A, seed, stream, args.steps, args.warmup, ws)
        s_o.close()
        results[other] = (r_o["sigma"], r_o["V"])
        forms[other] = {"value": ws * bytes_A * r_o["steps"] / (r_o["ms"] * 1e-3) / 1e9, "unit": "GB/s",
                        "ms_per_step": r_o["ms"] / r_o["steps"], "steps": r_o["steps"],
                        "roofline": roofline_for(other, r_o["prof"], bytes_A * r_o["steps"], m * r_o["steps"], pk),
                        "finalize_ms_per_step": r_o["prof"]["finalize"][0] / r_o["steps"]}

    with ClockSampler(local) as clocks:
        time.sleep(0.3)
        sess, step, res = run_form(spca, args.math, A, seed, stream, args.steps, args.warmup, ws)
    ms, steps, prof = res["ms"], res["steps"], res["prof"]
    results[args.math] = (res["sigma"], res["V"])
    launches = int(sum(v[1] for v in prof.values()))
    value = ws * bytes_A * steps / (ms * 1e-3) / 1e9
    roofline = roofline_for(args.math, prof, bytes_A * steps, m * steps, pk)
    kernels = {k_: {"ms_per_step": v[0] / steps, "launches_per_step": v[1] / steps} for k_, v in prof.items()
               if v[1]}

    # end to end through the C ABI: pinned host rows copied inside the timed region, results read back
    A_host = torch.empty((m, N), dtype=torch.float32, pin_memory=True)
    A_host.copy_(A)
    sig_h = np.zeros(K)
    V_h = np.zeros((K, N))
    e2e_steps = 2
    rows_np = A_host.numpy()

    from paper_1704_07669_gb300 import shard
    scratch = shard.scratch_like(sess) if ws > 1 and rank == 0 else None

    def e2e_step():
        spca.spca_reset(sess.handle, seed)
        for r0 in range(0, m, BLOCK):
            spca.spca_update(sess.handle, rows_np[r0:r0 + BLOCK])
        if ws > 1 and not shard.merge_across_ranks(sess, scratch=scratch):
            return
        spca.spca_finalize(sess.handle, sig_h, V_h, out_on_device=False)

    e2e_step()
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws)
    e2e = {"value": ws * bytes_A * e2e_steps / e2e_s / 1e9, "unit": "GB/s", "h2d_bytes_per_step": bytes_A,
           "d2h_bytes_per_step": 8 * (K + K * N)}

    # the optional parts report a failure inside the line instead of losing the measurement
    streamed = None
    if rank == 0 and not args.no_streamed:
        try:
            streamed = run_streamed(spca, dev, args.math)
        except Exception as exc:   # noqa: BLE001 - any failure of this part is reported, not raised
            streamed = {"error": f"{type(exc).__name__}: {exc}"}
    serving = None
    if rank == 0 and not args.no_serving:
        try:
            serving = run_serving(spca, dev)
        except Exception as exc:   # noqa: BLE001 - any failure of this part is reported, not raised
            serving = {"error": f"{type(exc).__name__}: {exc}"}

    cpu = None
    precision = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # the CPU oracle leg: the oracle timed on a bounded sample, and the oracle's result on the
        # whole matrix for the error of each timed form
        sample_rows = min(8 * BLOCK, m)
        try:
            cpu = cpu_baseline(A[:sample_rows].cpu().numpy(), seed, "first 8 row blocks of the timed matrix")
        except Exception as exc:   # noqa: BLE001
            cpu = {"error": f"{type(exc).__name__}: {exc}", "kind": "oracle"}
        try:
            precision = oracle_precision(A, seed, results)
        except Exception as exc:   # noqa: BLE001
            precision = {"error": f"{type(exc).__name__}: {exc}"}

    sess.close()
    if rank != 0:
        return 0
    workload = WORKLOAD if m == M else WORKLOAD.replace("100000x", f"{m}x")
    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": steps, "warmup": args.warmup,
            "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp16": "f16"}.get(args.math, "bf16"), "data": "synthetic",
            "config": {"workload": workload, "math": args.math,
                       "l2": f"inputs larger than L2 ({bytes_A / 1e9:.1f} GB), no flush",
                       "parallelism": (f"rows sharded over {ws} ranks ({m} rows each), one exchange step: "
                                       "rank checkpoints gathered and merged on rank 0, which finalizes")
                       if ws > 1 else "single"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "precision_vs_oracle": precision,
            "clocks": clocks.summary(), "kernels": kernels, "forms": forms, "serving": serving, "streamed": streamed,
            "pass_ms": {"p50": res["pass_ms_p50"], "p99": res["pass_ms_p99"],
                        "note": "per-pass times of the timed passes (CUDA events on the session stream)"},
            "peaks_source": pk["source"],
            "tflops": 4.0 * m * N * (K + P) * steps * ws / (ms * 1e-3) / 1e12}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--math", default="fp16", choices=["fp32", "bf16", "fp16"],
                    help="arithmetic of the timed pass (default: the FP16 tensor-core form, split G)")
    ap.add_argument("--forms", default="fp32,bf16",
                    help="other forms measured on the same data and reported under 'forms' ('' for none)")
    ap.add_argument("--m", type=int, default=M, help="rows of the workload (profiling runs use fewer)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-loop measurement")
    ap.add_argument("--no-streamed", action="store_true", help="skip the 150 GB host-stream measurement")
    args = ap.parse_args()
    if args.impl == "reference":
        if args.steps is None:
            args.steps = 3
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

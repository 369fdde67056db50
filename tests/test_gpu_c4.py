"""Full-size parity on the 937500 x 40000 FP32 stream (150 GB, larger than the device).

The rows reach the library from pinned host memory, 16384 rows per update, and are
copied to the device in pieces by the session's double-buffered host-to-device
path. Four distinct blocks are generated and cycled (``synth.workload_c4``); the
FP64 oracle folds each distinct block in once with its multiplicity in the stream
(``ShiftedPass.add(times=...)``), which is the same sum as the literal stream.
Checked: the shift (the FP32 mean of the first staged piece, to 1 ulp), H_bar, the
Gram matrix and the column sums (relative Frobenius error <= 1e-5), sigma_1..50
(<= 1e-4 relative) and the leading directions of V, and that the session's device
memory stays under 1 GB. The pass's end-to-end GB/s is printed beside a plain
pinned host-to-device copy's.
"""
import time
from collections import Counter

import numpy as np
import pytest
import torch

import paper_1704_07669_gb300 as spca
from oracle import spca as O
from paper_1704_07669_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
TOL_STATE = 1e-5
TOL_SIGMA = 1e-4
STAGE_BYTES = 256 << 20          # the session's host-to-device staging piece


def _h2d_gbs(host):
    dev = torch.empty(host.shape, dtype=host.dtype, device=DEV)
    for _ in range(2):
        dev.copy_(host, non_blocking=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        dev.copy_(host, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    return 3 * host.numel() * host.element_size() / (e0.elapsed_time(e1) * 1e-3) / 1e9


@pytest.fixture(scope="module")
def c4():
    if DEV is None:
        pytest.fail("GPU tests need CUDA")
    spca.build.build()
    spca.lib()
    w = synth.workload_c4(device=DEV)
    torch.cuda.synchronize()
    m, n, k, p, seed, mb = w["m"], w["n"], w["k"], w["p"], w["seed"], w["block_rows"]
    pool, schedule = w["pool"], w["schedule"]
    free0 = torch.cuda.mem_get_info(DEV)[0]
    with spca.Session(n, k, p, seed) as s:
        s.update(pool[0][:1])            # staging buffers are made on the first host update
        s.sync()
        s.reset(seed)
        used = free0 - torch.cuda.mem_get_info(DEV)[0]
        t0 = time.perf_counter()
        for pi, rows in schedule:
            s.update(pool[pi][:rows])
        s.sync()
        t_pass = time.perf_counter() - t0
        sigma, V = s.finalize()
        st = s.state()
    h2d = _h2d_gbs(pool[0])
    bytes_A = m * n * 4
    print(f"\n937500x40000 f32 from pinned host: {t_pass:.2f} s, {bytes_A / t_pass / 1e9:.1f} GB/s end to end; "
          f"plain pinned H2D copy {h2d:.1f} GB/s; session device memory {used / 2**20:.0f} MiB")
    Om = O.omega(n, k + p, seed, "f32")
    piece = min(mb, STAGE_BYTES // (4 * n))
    c_or = O.first_block_shift(pool[0][:piece].double().numpy())
    acc = O.ShiftedPass(Om, c=st["shift"].astype(np.float64))
    buf = np.empty((mb, n))
    for (pi, rows), times in Counter(schedule).items():
        t = torch.from_numpy(buf[:rows])
        t.copy_(pool[pi][:rows])
        acc.add(t.numpy(), overwrite=True, times=times)
    ref = acc.state()
    H_bar, gram_bar = O.centering_correction(ref["H"], ref["gram"], ref["s"], ref["sG"], ref["m"])
    s_ref, V_ref = O.finalize_centred(ref["G"], ref["H"], ref["s"], ref["sG"], ref["m"], Om, k)
    return {"w": w, "sigma": sigma, "V": V, "state": st, "used": used, "c_oracle": c_or, "H_bar": H_bar,
            "gram_bar": gram_bar, "s": ref["s"], "m": ref["m"], "sigma_ref": s_ref, "V_ref": V_ref}


def test_c4_state_against_oracle(c4):
    st = c4["state"]
    c_gpu, c_or = st["shift"], c4["c_oracle"]
    assert np.all(np.abs(c_gpu.astype(np.float64) - c_or) <= np.spacing(np.abs(c_or).astype(np.float32)).astype(np.float64))
    assert st["m"] == c4["m"] == c4["w"]["m"]
    e_H = O.rel_fro(st["H_bar"], c4["H_bar"])
    e_g = O.rel_fro(st["gram_bar"], c4["gram_bar"])
    e_s = O.rel_fro(st["colsum"], c4["s"])
    print(f"c4: rel Frobenius error H_bar {e_H:.2e}, Gram {e_g:.2e}, column sums {e_s:.2e}")
    assert e_H <= TOL_STATE and e_g <= TOL_STATE and e_s <= TOL_STATE


def test_c4_sigma_and_directions_against_oracle(c4):
    rel = np.abs(c4["sigma"] - c4["sigma_ref"]) / c4["sigma_ref"]
    sin10 = O.max_principal_sine(c4["V"][:, :10], c4["V_ref"][:, :10])
    print(f"c4: sigma rel max {rel.max():.2e}, sin theta V[:, :10] {sin10:.2e}")
    assert rel.max() <= TOL_SIGMA
    assert sin10 <= 1e-4
    assert np.all(np.sum(c4["V"][:, :10] * c4["V_ref"][:, :10], axis=0) > 0)


def test_c4_device_state_under_1_gb(c4):
    assert 0 < c4["used"] < 1 << 30

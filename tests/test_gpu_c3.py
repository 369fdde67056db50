"""Full-size parity on the 400000 x 40000 precision-sweep workload, per storage form.

The matrix (64 GB in FP32) is never held whole: ``synth.workload_c3`` regenerates
it one 8192-row block at a time on the GPU, and each block is stored as FP32,
BF16 and FP8 e4m3 with a per-block FP32 scale. One FP32-path session per storage
form reads the stored block on the device; the FP64 oracle (``ShiftedPass``)
reads the same stored values, copied to the host, block by block. Per storage
form the test checks the shift c (to 1 ulp), the sketch rows G_i of the first
and of the ragged last block (6784 rows), H_bar, the Gram matrix and the column
sums (relative Frobenius error <= 1e-5), and sigma_1..100 (<= 1e-4 relative)
with the principal-angle sine of the leading directions of V. The effect of the
storage precision itself (the oracle on BF16 or FP8 values against the oracle on
the FP32 values) is printed beside it.

The tensor cores on the same stored rows: one FP16-operand session per reduced-precision
storage form reads the BF16 or FP8 rows in their storage format (the grouped kernel, Gram
formed after each launch at l = 120); its own FP64 oracle runs the method on the same stored
values with Omega rounded to FP16 (the form's definition). Held to H_bar and the Gram matrix
within 1e-4 relative Frobenius and every sigma_1..100 within 1e-3 (the tensor-core gate).
"""
import time

import numpy as np
import pytest
import torch

import paper_1704_07669_gb300 as spca
from oracle import spca as O
from paper_1704_07669_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
STORES = ("f32", "bf16", "f8e4m3")
TC_STORES = ("bf16", "f8e4m3")
TOL_STATE = 1e-5
TOL_STATE_TC = 1e-4
TOL_SIGMA_TC = 1e-3
TOL_SIGMA = 1e-4


def _host_f64(stored, scale, buf):
    """The stored values in FP64 on the host, in buf (waits for the current stream)."""
    t = torch.from_numpy(buf[:stored.shape[0]])
    t.copy_(stored)
    if scale is not None:
        t.mul_(scale)
    return t.numpy()


@pytest.fixture(scope="module")
def c3():
    if DEV is None:
        pytest.fail("GPU tests need CUDA")
    spca.build.build()
    spca.lib()
    stream = torch.cuda.Stream(DEV)
    t0 = time.time()
    with torch.cuda.stream(stream):
        w = synth.workload_c3(device=DEV)
        m, n, k, p, seed, mb = w["m"], w["n"], w["k"], w["p"], w["seed"], w["block_rows"]
        l = k + p
        Om = O.omega(n, l, seed, "f32")
        sess = {st: spca.Session(n, k, p, seed, max_block_rows=mb, stream=stream) for st in STORES}
        sess_tc = {st: spca.Session(n, k, p, seed, math="fp16", max_block_rows=mb, stream=stream) for st in TC_STORES}
        Om16 = O.omega(n, l, seed, "f16")
        acc = {}
        acc_tc = {}
        G_gpu = {st: [] for st in STORES}
        G_ref = {st: [] for st in STORES}
        shift_first = {}
        last0 = ((m - 1) // mb) * mb
        buf = np.empty((mb, n))
        for r0, a in w["blocks"]():
            keep = r0 in (0, last0)
            for st in STORES:
                stored, scale = synth.store_rows(a, st)
                G = torch.empty((a.shape[0], l), device=DEV, dtype=torch.float32) if keep else None
                sess[st].update(stored, G_out=G, block_scale=scale)
                if st in TC_STORES:
                    sess_tc[st].update(stored, block_scale=scale)
                    # the tensor-core session batches device rows until a flush and `stored` is
                    # freed after this iteration: launch the block now (spca_sync flushes)
                    sess_tc[st].sync()
                a64 = _host_f64(stored, scale, buf)     # waits for this stream: the updates have read it
                if r0 == 0:
                    # the oracle's own shift, then the pass on the session's shift (equal to 1 ulp)
                    shift_first[st] = O.first_block_shift(a64)
                    sess[st].sync()
                    acc[st] = O.ShiftedPass(Om, c=sess[st].state()["shift"].astype(np.float64))
                    if st in TC_STORES:
                        sess_tc[st].sync()
                        acc_tc[st] = O.ShiftedPass(Om16, c=sess_tc[st].state()["shift"].astype(np.float64),
                                                   keep_G=False)
                if st in TC_STORES:
                    acc_tc[st].add(a64)                      # before the FP32 oracle shifts a64 in place
                g = acc[st].add(a64, overwrite=True)
                if keep:
                    G_gpu[st].append(G.cpu().double().numpy())
                    G_ref[st].append(g)
            del a
        out = {}
        for st in STORES:
            sigma, V = sess[st].finalize()
            state = sess[st].state()
            sess[st].close()
            ref_state = acc[st].state()
            H_bar, gram_bar = O.centering_correction(ref_state["H"], ref_state["gram"], ref_state["s"],
                                                     ref_state["sG"], ref_state["m"])
            s_ref, V_ref = O.finalize_centred(ref_state["G"], ref_state["H"], ref_state["s"], ref_state["sG"],
                                              ref_state["m"], Om, k)
            out[st] = {"sigma": sigma, "V": V, "state": state, "H_bar": H_bar, "gram_bar": gram_bar,
                       "s": ref_state["s"], "m": ref_state["m"], "sigma_ref": s_ref, "V_ref": V_ref,
                       "shift_oracle": shift_first[st], "G_gpu": G_gpu[st], "G_ref": G_ref[st]}
        for st in TC_STORES:
            sigma, V = sess_tc[st].finalize()
            state = sess_tc[st].state()
            sess_tc[st].close()
            rs = acc_tc[st].state()
            H_bar, gram_bar = O.centering_correction(rs["H"], rs["gram"], rs["s"], rs["sG"], rs["m"])
            res = O.gram_qb(gram_bar, H_bar)
            _, s_ref, V_ref = O.svd_truncate(None, res["B"], k)
            V_ref, _ = O.sign_fix(V_ref)
            out["tc_" + st] = {"sigma": sigma, "V": V, "state": state, "H_bar": H_bar, "gram_bar": gram_bar,
                               "sigma_ref": s_ref, "V_ref": V_ref}
    torch.cuda.synchronize()
    print(f"\n400000x40000 sweep (3 storage forms on the FP32 path, 2 on the tensor cores, GPU + FP64 oracle): "
          f"{time.time() - t0:.0f} s")
    return w, out


@pytest.mark.parametrize("store", STORES)
def test_c3_state_against_oracle(c3, store):
    w, out = c3
    r = out[store]
    st = r["state"]
    c_gpu = st["shift"]
    c_or = r["shift_oracle"]
    assert np.all(np.abs(c_gpu.astype(np.float64) - c_or) <= np.spacing(np.abs(c_or).astype(np.float32)).astype(np.float64))
    assert st["m"] == w["m"] == r["m"]
    for g_gpu, g_ref in zip(r["G_gpu"], r["G_ref"]):
        assert O.rel_fro(g_gpu, g_ref) <= TOL_STATE
    assert [g.shape[0] for g in r["G_gpu"]] == [w["block_rows"], w["m"] % w["block_rows"]]
    e_H = O.rel_fro(st["H_bar"], r["H_bar"])
    e_g = O.rel_fro(st["gram_bar"], r["gram_bar"])
    e_s = O.rel_fro(st["colsum"], r["s"])
    print(f"{store}: rel Frobenius error H_bar {e_H:.2e}, Gram {e_g:.2e}, column sums {e_s:.2e}")
    assert e_H <= TOL_STATE and e_g <= TOL_STATE and e_s <= TOL_STATE


@pytest.mark.parametrize("store", STORES)
def test_c3_sigma_and_directions_against_oracle(c3, store):
    w, out = c3
    r = out[store]
    k = w["k"]
    rel = np.abs(r["sigma"] - r["sigma_ref"]) / r["sigma_ref"]
    sin10 = O.max_principal_sine(r["V"][:, :10], r["V_ref"][:, :10])
    sin_k = O.max_principal_sine(r["V"], r["V_ref"])
    # storage precision: the oracle on the stored values against the oracle on the FP32 values
    base = out["f32"]
    rel_store = np.abs(r["sigma_ref"] - base["sigma_ref"]) / base["sigma_ref"]
    sin_store = O.max_principal_sine(r["V_ref"][:, :10], base["V_ref"][:, :10])
    print(f"{store}: GPU vs FP64 oracle of the stored values: sigma rel max {rel.max():.2e} "
          f"(leading 10 {rel[:10].max():.2e}), sin theta V[:, :10] {sin10:.2e}, V[:, :{k}] {sin_k:.2e}; "
          f"storage vs FP32 values: sigma rel max {rel_store.max():.2e} "
          f"(leading 10 {rel_store[:10].max():.2e}), sin theta V[:, :10] {sin_store:.2e}")
    assert rel.max() <= TOL_SIGMA
    assert sin10 <= 1e-3
    cos = np.sum(r["V"][:, :10] * r["V_ref"][:, :10], axis=0)
    assert np.all(cos > 0)          # the same sign convention on both sides


@pytest.mark.parametrize("store", TC_STORES)
def test_c3_tensor_cores_against_oracle(c3, store):
    """FP16 operands on BF16 / FP8 rows at the full 400000 x 40000 (l = 120)."""
    _, out = c3
    r = out["tc_" + store]
    e_H = O.rel_fro(r["state"]["H_bar"], r["H_bar"])
    e_g = O.rel_fro(r["state"]["gram_bar"], r["gram_bar"])
    rel = np.abs(r["sigma"] - r["sigma_ref"]) / r["sigma_ref"]
    sin10 = O.max_principal_sine(r["V"][:, :10], r["V_ref"][:, :10])
    print(f"tensor cores (FP16 operands) on {store} rows: H_bar {e_H:.2e}, Gram {e_g:.2e}; sigma rel max "
          f"{rel.max():.2e} (leading 10 {rel[:10].max():.2e}), sin theta V[:, :10] {sin10:.2e}")
    assert e_H <= TOL_STATE_TC and e_g <= TOL_STATE_TC
    assert rel.max() <= TOL_SIGMA_TC
    assert sin10 <= 1e-2

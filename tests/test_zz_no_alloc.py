"""GPU checks of spca_shift_static, the allocation-free form of the centering
shift (Sec. 2.1: the data are column-centred; the pass subtracts the FP32 column
mean c of the first rows). It must give what a session computes from the same
rows, call after call, with its scratch in a fixed device array."""
import numpy as np
import pytest
import torch

import paper_1704_07669_gb300 as spca

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
MAX_N = 16384   # SPCA_SHIFT_STATIC_MAX_N


@pytest.fixture(scope="module", autouse=True)
def _built():
    if DEV is None:
        pytest.fail("GPU tests need CUDA")
    spca.build.build()
    spca.lib()


def _rows(m, n, seed):
    g = torch.Generator().manual_seed(seed)
    A = 0.1 * torch.randn(m, n, generator=g) + 3.0 * torch.randn(1, n, generator=g)
    return A.to(DEV)


def _session_shift(A):
    m, n = A.shape
    with spca.Session(n, 4, 4, 1, max_block_rows=max(m, 8)) as s:
        s.update(A)
        return s.state()["shift"]


@pytest.mark.parametrize("m,n,cols", [(3000, 2000, 2000), (1000, 1500, 1200), (7, 40, 33), (200, MAX_N, MAX_N)],
                         ids=["3000x2000", "strided-1000x1200", "tiny-7x33", f"n-at-limit-{MAX_N}"])
def test_matches_the_session_shift_on_two_calls_in_a_row(m, n, cols):
    full = _rows(m, n, seed=m + n)
    A = full[:, :cols]                       # ld = n >= cols
    ref = _session_shift(A)
    out = [torch.full((cols,), float("nan"), device=DEV) for _ in range(2)]
    spca.spca_shift_static(A, out[0])
    spca.spca_shift_static(A, out[1])
    torch.cuda.synchronize()
    for o in out:
        got = o.cpu().numpy()
        # same kernels, same partition of the rows: the values agree bit for bit
        assert np.array_equal(got, ref), np.abs(got - ref).max()
    # and they are the FP32 column means of the rows
    mean64 = A.double().mean(0).cpu().numpy()
    assert np.abs(out[0].cpu().numpy() - mean64).max() <= 1e-6 * np.abs(mean64).max()


def test_on_a_caller_stream():
    A = _rows(512, 256, seed=5)
    ref = _session_shift(A)
    st = torch.cuda.Stream()
    out = torch.empty(256, device=DEV)
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        spca.spca_shift_static(A, out, stream=st)
    st.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref)


def test_rejects_sizes_beyond_the_fixed_scratch():
    A = torch.zeros((4, MAX_N + 1), device=DEV)
    out = torch.zeros(MAX_N + 1, device=DEV)
    with pytest.raises(spca.SpcaError) as ei:
        spca.spca_shift_static(A, out)
    assert ei.value.status == 1
    assert "exceeds the fixed scratch" in str(ei.value)


def test_binding_rejects_views_and_outputs_it_cannot_pass():
    A = _rows(64, 48, seed=9)
    out = torch.zeros(48, device=DEV)
    with pytest.raises(ValueError):
        spca.spca_shift_static(A.t(), torch.zeros(64, device=DEV))   # column-strided view
    with pytest.raises(ValueError):
        spca.spca_shift_static(A, out[:40])                           # shift shorter than n
    with pytest.raises(ValueError):
        spca.spca_shift_static(A, out.double())                       # wrong dtype
    with pytest.raises(ValueError):
        spca.spca_shift_static(A.cpu(), out)                          # host rows

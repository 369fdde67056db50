"""The shared-memory layout of the pipelined tensor-core pass, checked on the CPU.

A small host program compiled against the kernel source prints `tc3_layout` for every
configuration the pass may choose (l padded to L = 16..64, FP16 or BF16 operands, clusters
of 1..16 CTAs, 128..768 features per CTA). Each region must be large enough for every access
the kernel makes to it, aligned as its users need (1024 bytes for the 128-byte-swizzled
operands and TMA boxes, 16 bytes for vector and bulk accesses), disjoint from the others, and
inside the allocation. This is the class of fault where the H drain staged 32 KB in an
exchange region of 18 KB at L = 32.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1704_07669_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")

HARNESS = r'''
#include "sketch_tc3.cu"
#include <cstdio>
namespace spca {   // symbols of other translation units that the layout never calls
void Prof::begin(int, cudaStream_t) {}
void Prof::end(int, cudaStream_t) {}
cudaError_t launch_tc_finish(const State&, const TcWork&, int, int64_t, int, cudaStream_t, Prof*) { return cudaSuccess; }
}
int main() {
  using namespace spca;
  std::printf("consts %u %u %u %u %d\n", STAGE_BYTES, BLOCK16, GT_CHUNK, static_cast<unsigned>(NSTAGE), T3_ROWS);
  for (int L = 16; L <= 64; L += 16)
    for (int gs = 1; gs <= 2; ++gs)
      for (int CS = 1; CS <= 16; CS *= 2)
        for (int w = 128; w <= 768; w += 128) {
          const Tc3Layout t = tc3_layout(L, w, CS, gs);
          std::printf("lay %d %d %d %d %d %u %u %u %u %u %u %u %u %u %u\n", L, gs, CS, w, t.RPC, t.stage, t.pair, t.om,
                      t.xch, t.gt, t.pub, t.shift, t.sy, t.bars, t.total);
        }
  return 0;
}
'''


@pytest.fixture(scope="module")
def layouts(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc is not available")
    d = tmp_path_factory.mktemp("tc3_layout")
    src, exe = d / "harness.cu", d / "harness"
    src.write_text(HARNESS)
    r = subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=compute_103a", "-I", INCLUDE,
                        "-I", CSRC, str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    consts = [int(x) for x in out[0].split()[1:]]
    rows = [[int(x) for x in ln.split()[1:]] for ln in out[1:] if ln.startswith("lay ")]
    return consts, rows


def _chosen(L, w):
    """Configurations the pass can take: at most six 128-feature units, TMEM for two D1
    buffers and H, and the 227 KB of shared memory a CTA may have."""
    return w // 128 <= 6 and 2 * L + (w // 128) * L <= 512


def test_every_region_fits_its_accesses_and_alignment(layouts):
    (stage_bytes, block16, gt_chunk, nstage, rows_per_tile), rows = layouts
    assert stage_bytes == rows_per_tile * 64 * 4 and block16 == rows_per_tile * 64 * 2
    checked = 0
    for L, gs, CS, w, RPC, stage, pair, om, xch, gt, pub, shift, sy, bars, total in rows:
        if not _chosen(L, w) or total > 227 * 1024:
            continue
        checked += 1
        assert RPC == rows_per_tile // CS
        xch_need = rows_per_tile * (L + 4) * 4
        if L % 32 == 0:
            xch_need = max(xch_need, 2 * 128 * 128)   # the TMA drain's two 16 KB staging halves
        need = [   # (name, offset, bytes the kernel touches, alignment its users need)
            ("stage", stage, nstage * stage_bytes, 1024),   # TMA boxes; MMA2 reads image units here
            ("pair", pair, 2 * block16, 1024),             # swizzled MMA1 operand, bulk-copied out
            ("om", om, 2 * L * 128, 1024),                  # swizzled Omega chunks (MMA1 B operand)
            ("xch", xch, xch_need, 1024),                   # D1 exchange rows; drain staging boxes
            ("gt", gt, 2 * gt_chunk, 1024),                 # swizzled G^T (MMA2 B operand), 2 L rows
            ("pub", pub, 2 * L * gs * (RPC // 8) * 16, 16),  # packed own rows, two tile parities
            ("shift", shift, w * 4, 16),                    # float4 reads of the shift
            ("sy", sy, RPC * L * 4, 16),                    # own rows of G', float4 writes
            ("bars", bars, 64 * 8, 8),                      # the mbarriers
        ]
        spans = []
        for name, off, size, align in need:
            assert off % align == 0, (name, L, gs, CS, w, off)
            spans.append((off, off + size, name))
        spans.sort()
        for (a0, a1, an), (b0, b1, bn) in zip(spans, spans[1:]):
            assert a1 <= b0, (an, bn, L, gs, CS, w)
        # the kernel aligns the dynamic shared memory base up to 1024 bytes inside the allocation
        assert spans[-1][1] + 1024 <= total, (L, gs, CS, w)
        # two tiles' G^T fit in the chunk rows when there are no lo terms (2 L <= 128 rows)
        assert 2 * L <= 128
    assert checked > 50

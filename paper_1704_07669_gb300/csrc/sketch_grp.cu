// The streaming pass on the tensor cores with all SMs in groups (Alg. 4 steps 5-7, Eq. 11).
//
// A persistent, cooperatively launched grid of NG groups of S CTAs. The n features are cut
// into 64-feature blocks; CTA j of every group owns the blocks [j NBT / S, (j + 1) NBT / S)
// for the whole launch. Group g takes the 128-row tiles g, g + NG, g + 2 NG, ... in order.
// Per tile i of a group:
//  - phase 1 (every CTA of the group, its own blocks): TMA streams the stored rows into a
//    stage ring (FP32: two 32-feature boxes per block; BF16: one 64-feature box; FP8 E4M3:
//    one 64-feature box of codes, decoded with the block's scale); converter warps subtract
//    the shift c, scale and round into a 16-bit operand block (K-major, 128-byte swizzle); MMA1
//    accumulates D1 = A_hat[:, own] Omega[own, :] in TMEM; a copier warp writes each
//    converted block to the CTA's image ring in global memory (kept in L2);
//  - the epilogue warps move D1 to the CTA's slot of the group's partial ring in global
//    memory (column-major, coalesced) and count the arrival;
//  - the reducer warps of CTA j, once all S partials of the tile are in, sum them in a
//    fixed order (deterministic) for the rows [32 j / S, 32 (j + 1) / S) quads, round to the
//    operand format (FP16: hi + lo), append the ones column, and write those rows of G' to
//    the group's G' ring in the layout MMA2 reads; the same rows feed the Gram matrix and
//    the sums of G (double-float) and the optional G output;
//  - phase 2 (every CTA, its own blocks, once G' of the tile is complete): the CTA's image
//    of the tile comes back from L2 (no second conversion) and MMA2 computes
//    A_hat[:, own]^T G' per 128-feature M-tile into a fresh TMEM buffer, which a drain group
//    adds into the CTA's running H (FP32, round to nearest, TMEM resident for the launch):
//    tcgen05 accumulation then truncates only within one tile's 8-16 MMAs. H leaves TMEM
//    once, at the end of the launch (per-group partials, summed in a fixed order after).
// Shapes whose H does not fit beside a fresh buffer accumulate H in TMEM directly and drain
// it to the partials every few tiles instead (add-reductions owned by one thread each).
// Cross-CTA signalling goes through monotonic counters in global memory (release adds,
// acquire polls); all waits are bounded and a thread that gives up sets flags[0] bit 2 and
// skips its later waits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp8.h>

#include <cstdio>
#include <cstring>

#include "spca_internal.cuh"
#include "tc_ptx.cuh"

namespace spca {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn();   // sketch_tc3.cu

namespace {

constexpr int GR_ROWS = 128;
constexpr uint32_t BLK16 = GR_ROWS * 64 * 2;     // 16-bit operand block: 128 rows x 64 features
constexpr uint32_t STG = GR_ROWS * 32 * 4;       // stage slot: 128 rows x 32 FP32 (or 64 BF16, 64 FP8) features
constexpr uint32_t P2U = 16384;                  // phase-2 unit: 2 blocks x 64 rows x 128 B
constexpr int RING_R = 4;                        // group rings (partials, G', counters)
#ifndef SPCA_GRP_IMG_R
#define SPCA_GRP_IMG_R 3
#endif
constexpr int IMG_R = SPCA_GRP_IMG_R;            // per-CTA image ring (tiles)
constexpr int OM_R = 2;                          // Omega blocks in flight
constexpr int NS2 = 3;                           // phase-2 unit slots
constexpr int GRAM_BLK = 3;                      // 4 x 2 Gram blocks per reducer thread at most
constexpr int MAX_SEGS = 48;
// storage formats of the rows (the session's dtype): FP32, BF16, FP8 E4M3 codes x a block scale
constexpr int IN_F32 = 0, IN_BF16 = 1, IN_F8 = 2;

// warp roles (21 warps)
constexpr int W_P1 = 0, W_P2 = 1, W_MMA1 = 2, W_MMA2 = 3;
constexpr int W_EPI0 = 4;     // 4 warps: D1 -> partials (TMEM lane quadrants 0-3)
constexpr int W_DRN0 = 8;     // 4 warps: H adds and drains (TMEM lane quadrants 0-3)
constexpr int W_RED0 = 12;    // 4 warps: reduction of the group's partials
constexpr int RED_T = 128;
constexpr int W_COPY = 16;
constexpr int W_CV0 = 17;     // 4 converter warps
constexpr int CV_W = 4;
constexpr int GRP_NT = 32 * (W_CV0 + CV_W);   // 672 threads
constexpr int GRP_MAX_PAIRS = GRAM_BLK * RED_T;   // 4 x 2 Gram blocks of the lower triangle at most

}  // namespace

struct GrpLayout {
  uint32_t st1, op, om, gp, p2, shift, red, gram, bars, total;
};

// 4 x 2 blocks (a, b) of the l x l Gram matrix that meet its lower triangle: rows 4a..4a+3,
// columns 2b, 2b+1 with b <= 2a + 1; a-major, so block a starts at index a (a + 1)
__host__ __device__ inline int gram_pairs(int l) {
  const int na = (l + 3) / 4;
  return na * (na + 1);
}

// ns1: FP32 stages; nbmax: blocks per CTA; gs: 1, or 2 when G' is split (hi + lo); rpc: reducer
// rows per CTA at most; npairs: the reducers' Gram blocks (0: the Gram matrix is formed after
// the launch from the G' rows)
__host__ __device__ inline GrpLayout grp_layout(int L, int npairs, int nbmax, int ns1, int gs, int rpc) {
  GrpLayout t;
  uint32_t o = 0;
  t.st1 = o; o += static_cast<uint32_t>(ns1) * STG;
  t.op = o; o += 2u * BLK16;
  t.om = o; o += static_cast<uint32_t>(OM_R) * static_cast<uint32_t>(L) * 128u;
  t.gp = o; o += static_cast<uint32_t>(gs) * 2u * static_cast<uint32_t>(L) * 128u;
  t.p2 = o; o += static_cast<uint32_t>(NS2) * P2U;
  t.shift = o; o += static_cast<uint32_t>(nbmax) * 64u * 4u;
  t.red = o; o += ((static_cast<uint32_t>(rpc) * static_cast<uint32_t>(L) * 4u) + 15u) & ~15u;
  t.gram = o; o += static_cast<uint32_t>(npairs) * 8u * 8u;   // double-float Gram accumulators
  o = (o + 15u) & ~15u;
  t.bars = o; o += 80u * 8u;   // BAR_SLOTS
  t.total = o + 1024u;   // the base is rounded up to 1024 bytes in the kernel
  return t;
}

struct GrpSeg {
  int64_t m;
  float* gout;
  int64_t tile0;
  float dscale;                 // FP8 rows: the block's scale (a stored value is code x dscale); else 1
};

struct GrpArgs {
  CUtensorMap maps[MAX_SEGS];   // the rows: FP32 box 32 x 128 and BF16 box 64 x 128 (128-byte swizzle),
                                // FP8 box 64 x 128 (no swizzle); features x rows
  GrpSeg seg[MAX_SEGS];
  int nseg;
  int64_t ntiles;
  int64_t n;
  int l, L;
  int S, NG;                    // CTAs per group, groups launched
  int nbt, nbmax, nu;           // 64-feature blocks in all, per CTA at most, M-tiles per CTA
  int ns1, nd1;                 // FP32 stages, D1 buffers (1 or 2)
  int nf;                       // fresh H buffers (1 or 2) added into a running H in TMEM; 0: direct
  int drain_every;              // fresh == 0: tiles between drains of H to the partials
  const float* shift;
  const uint16_t* om16;         // Omega, pre-swizzled 64-feature blocks (L x 128 B each)
  const uint16_t* zero8k;       // 8 KB of zeros (the missing half of an odd last M-tile)
  uint16_t* img;                // per CTA: IMG_R tiles x nbmax blocks x 16 KB
  float* part;                  // per group: RING_R slots x S x L x 128 (column-major)
  uint16_t* gbuf;               // per group: RING_R slots x gs x 2 x L x 64 16-bit
  unsigned* cnt;                // per group: RING_R x 3 counters (arrived, reduced, loaded)
  const float* scale;
  int npairs;                   // the reducers' Gram blocks (gram_pairs(l)), or 0 with gfull
  float* gfull;                 // npairs == 0: G' rows of the launch, tile t at rows 128 t (ld L), unscaled
  float* Hpart;                 // per group: nbt*64 x L (FP32)
  uint64_t wait_ns;             // the pipeline waits' limit (a wait that runs out sets flags[0] bit 2)
  double* gram_part;            // per CTA: L x L
  double* sG_part;              // per CTA: L
  int* flags;
  unsigned long long* trace;    // SPCA_GRP_TRACE builds: phase times of CTA 0 for its first 16 tiles
};

#ifdef SPCA_GRP_TRACE
#define GRP_TRACE(ti, ev)                                                        \
  do {                                                                           \
    if (blockIdx.x == a.S - 1 && (ti) >= 0 && (ti) < 16 && a.trace) {             \
      unsigned long long t_;                                                     \
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_));                     \
      a.trace[(ti) * 16 + (ev)] = t_;                                            \
    }                                                                            \
  } while (0)
// per CTA of group 0 (the first 16): event k of tile ti at trace[256 + 256 k + 16 cta + ti]
#define GRP_TRACE_ALL(ti, k)                                                      \
  do {                                                                           \
    if (blockIdx.x < 16 && blockIdx.x < a.S && (ti) >= 0 && (ti) < 16 && a.trace) { \
      unsigned long long t_;                                                     \
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_));                     \
      a.trace[256 + 256 * (k) + 16 * blockIdx.x + (ti)] = t_;                    \
    }                                                                            \
  } while (0)
#else
#define GRP_TRACE_ALL(ti, k) \
  do {                       \
  } while (0)
#define GRP_TRACE(ti, ev) \
  do {                    \
  } while (0)
#endif

namespace {

__device__ __forceinline__ int find_seg(const GrpArgs& a, int64_t tile) {
  int s = 0;
  while (s + 1 < a.nseg && a.seg[s + 1].tile0 <= tile) ++s;
  return s;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t gtime_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// The waits of the pipeline give up after the launch's wait limit (GrpArgs::wait_ns, half a
// second unless the session says otherwise); the waits for a CTA's own copies in flight before
// it leaves keep half a second whatever that limit is.
constexpr uint64_t kOwnWaitNs = 500000000ull;

// bounded poll of a global counter until it reaches target: short sleeps between polls (the
// counters are written by other SMs)
__device__ __forceinline__ bool wait_geq(const unsigned* p, unsigned target, uint64_t limit_ns = kOwnWaitNs) {
  if (ld_acquire_u32(p) >= target) return true;
  const uint64_t t0 = gtime_ns();
  for (;;) {
    __nanosleep(64);
    if (ld_acquire_u32(p) >= target) return true;
    if (gtime_ns() - t0 > limit_ns) return false;
  }
}
// try_wait with a suspend-time hint: the thread sleeps in hardware until the phase completes
// (or the hint, 20 us, runs out), so a waiting warp takes no issue slots and wakes at once
__device__ __forceinline__ bool mbar_try_sus(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity), "r"(20000u)
      : "memory");
  return ok != 0;
}
// bounded: gives up after limit_ns
__device__ __forceinline__ bool mbar_wait_fast(uint32_t a, uint32_t parity, uint64_t limit_ns = kOwnWaitNs) {
  if (mbar_try_sus(a, parity)) return true;
  const uint64_t t0 = gtime_ns();
  for (;;) {
    if (mbar_try_sus(a, parity)) return true;
    if (gtime_ns() - t0 > limit_ns) return false;
  }
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* r) {
  tmem_st8(taddr, r);
  tmem_st8(taddr + 8u, r + 8);
}
// invalidate a 128-byte line in L2 without writing it back (its data is dead)
__device__ __forceinline__ void discard_l2(const void* p) {
  asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}
// two E4M3 codes (low byte first) to floats, exactly (through the FP16 conversion)
__device__ __forceinline__ float2 fp8x2_e4m3_to_float2(uint16_t two) {
  const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(two), __NV_E4M3);
  return __half22float2(__half2(h));
}
__device__ __forceinline__ void st_global_v2u(void* p, uint32_t a, uint32_t b) {
  asm volatile("st.global.v2.u32 [%0], {%1, %2};" ::"l"(p), "r"(a), "r"(b) : "memory");
}

// Double-float product accumulation: x y added exactly as a pair (two-product by FMA), then
// the pair into hi + lo (two-sum). Used for the Gram entries of the rounded G'.
struct F2Prod {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add_prod(float x, float y) {
    const float p = x * y;
    const float e = fmaf(x, y, -p);
    const float s = hi + p;
    const float bb = s - hi;
    lo += ((hi - (s - bb)) + (p - bb)) + e;
    hi = s;
  }
};

// barrier slots (each ring's slots follow from its size)
constexpr int MAX_NS1 = 16;
enum {
  B_S1_FULL = 0,                          // [MAX_NS1] FP32 stage landed
  B_S1_EMPTY = B_S1_FULL + MAX_NS1,       // [MAX_NS1] converted
  B_OM_FULL = B_S1_EMPTY + MAX_NS1,       // [OM_R]
  B_OM_EMPTY = B_OM_FULL + OM_R,          // [OM_R]
  B_OP_FULL = B_OM_EMPTY + OM_R,          // [2] operand block converted
  B_OP_EMPTY = B_OP_FULL + 2,             // [2] MMA1 and the image copy are done with it
  B_D1_FULL = B_OP_EMPTY + 2,             // [2]
  B_D1_EMPTY = B_D1_FULL + 2,             // [2]
  B_IMG_READY = B_D1_EMPTY + 2,           // [IMG_R] a tile's image is complete in global memory
  B_IMG_FREE = B_IMG_READY + IMG_R,       // [IMG_R] phase 2 has loaded a tile's image
  B_GP_FULL = B_IMG_FREE + IMG_R,
  B_GP_EMPTY = B_GP_FULL + 1,
  B_P2_FULL = B_GP_EMPTY + 1,             // [NS2]
  B_P2_EMPTY = B_P2_FULL + NS2,           // [NS2]
  B_F_FULL = B_P2_EMPTY + NS2,            // [2] a fresh buffer (or, direct mode: a drain tile's MMA2) is done
  B_F_FREE = B_F_FULL + 2,                // [2] the drain group has taken it
  B_FINAL = B_F_FREE + 2,
  B_COUNT = B_FINAL + 1
};
constexpr int BAR_SLOTS = 80;
static_assert(B_COUNT <= BAR_SLOTS, "barrier slots");

template <int FMT, int INP>
__global__ void __launch_bounds__(GRP_NT, 1) sketch_grp_kernel(const __grid_constant__ GrpArgs a) {
  constexpr int GS = FMT == FMT_F16 ? 2 : 1;
  constexpr int SPB = INP == IN_F32 ? 2 : 1;                  // stages per 64-feature block
  constexpr uint32_t SBYTES = INP == IN_F8 ? STG / 2 : STG;   // bytes a stage receives
  extern __shared__ __align__(1024) uint8_t smem_g[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_g) + 1023) & ~uintptr_t(1023));
  const int L = a.L, l = a.l, S = a.S;
  const int grp = static_cast<int>(blockIdx.x) / S, j = static_cast<int>(blockIdx.x) % S;
  const int blk0 = static_cast<int>((static_cast<int64_t>(j) * a.nbt) / S);
  const int blk1 = static_cast<int>((static_cast<int64_t>(j + 1) * a.nbt) / S);
  const int NB = blk1 - blk0;   // >= 1: the configuration keeps S <= the number of blocks
  const int q0 = (32 * j) / S, q1 = (32 * (j + 1)) / S;   // reducer row quads
  const int rpc = 4 * (q1 - q0);
  const GrpLayout lay = grp_layout(L, a.npairs, a.nbmax, a.ns1, GS, (32 + S - 1) / S * 4);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + lay.bars);
  auto bar = [&](int i) { return su32(&bars[i]); };
  float* sShift = reinterpret_cast<float*>(base + lay.shift);
  float* sRed = reinterpret_cast<float*>(base + lay.red);
  float2* sGram = reinterpret_cast<float2*>(base + lay.gram);
  __shared__ uint32_t tmem_sh;
  __shared__ unsigned red_go;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int NG = a.NG;
  const uint64_t wl = a.wait_ns;
#define PWAIT_MBAR(addr, par) mbar_wait_fast((addr), (par), wl)
#define PWAIT_GEQ(ptr, target) wait_geq((ptr), (target), wl)
  const int nt = grp < a.ntiles ? static_cast<int>((a.ntiles - 1 - grp) / NG + 1) : 0;
  const int64_t f0 = static_cast<int64_t>(blk0) * 64;
  const int64_t fend = static_cast<int64_t>(blk1) * 64;
  const float op_scale = a.scale ? *a.scale : 1.f;
  const float inv_s = 1.f / op_scale;
  const uint32_t om_bytes = static_cast<uint32_t>(L) * 128u;
  const uint32_t gp_bytes = static_cast<uint32_t>(GS) * 2u * static_cast<uint32_t>(L) * 128u;
  const int64_t cta = blockIdx.x;
  uint16_t* img_cta = a.img + cta * static_cast<int64_t>(IMG_R) * a.nbmax * (BLK16 / 2);
  float* part_g = a.part + static_cast<int64_t>(grp) * RING_R * S * L * GR_ROWS;
  uint16_t* gbuf_g = a.gbuf + static_cast<int64_t>(grp) * RING_R * (gp_bytes / 2);
  unsigned* cnt_g = a.cnt + static_cast<int64_t>(grp) * RING_R * 3;
  auto c_arrived = [&](int slot) { return cnt_g + slot * 3 + 0; };
  auto c_reduced = [&](int slot) { return cnt_g + slot * 3 + 1; };
  auto c_loaded = [&](int slot) { return cnt_g + slot * 3 + 2; };
  const int nu = a.nu;
  const int ND1 = a.nd1;
  const int NF = a.nf;
  const bool fresh = NF > 0;

  {
    // the launch must match the layout and the TMEM budget this code assumes; otherwise report
    // (flags[0] bit 4) and touch nothing
    uint32_t dyn = 0;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    const uint32_t used = static_cast<uint32_t>(base - smem_g) + lay.total - 1024u;
    const bool bad = used > dyn || (ND1 + nu + NF) * L > 512 || ND1 < 1 || ND1 > 2 || NF < 0 || NF > 2 ||
                     static_cast<int>(gridDim.x) != a.NG * S || blockDim.x != GRP_NT || NB < 1 || NB > a.nbmax ||
                     2 * nu < a.nbmax || a.ns1 < 1 || a.ns1 > MAX_NS1 || rpc > (32 + S - 1) / S * 4;
    if (bad) {
      if (tid == 0) atomicOr(a.flags, 16);
      return;
    }
  }
  for (int i = tid; i < a.nbmax * 64; i += GRP_NT) {
    const int64_t f = f0 + i;
    sShift[i] = (f < fend && f < a.n) ? a.shift[f] : 0.f;
  }
  if (tid == 0) {
    for (int s = 0; s < a.ns1; ++s) {
      mbar_init(bar(B_S1_FULL + s), 1);
      mbar_init(bar(B_S1_EMPTY + s), CV_W);
    }
    for (int p = 0; p < 2; ++p) {
      mbar_init(bar(B_OM_FULL + p), 1);
      mbar_init(bar(B_OM_EMPTY + p), 1);
      mbar_init(bar(B_OP_FULL + p), CV_W);
      mbar_init(bar(B_OP_EMPTY + p), 2);
      mbar_init(bar(B_D1_FULL + p), 1);
      mbar_init(bar(B_D1_EMPTY + p), 128);
    }
    for (int r = 0; r < IMG_R; ++r) {
      mbar_init(bar(B_IMG_READY + r), 1);
      mbar_init(bar(B_IMG_FREE + r), fresh ? 128 : 1);   // the drain group, or the MMA2 issuer
    }
    mbar_init(bar(B_GP_FULL), 1);
    mbar_init(bar(B_GP_EMPTY), 1);
    for (int s = 0; s < NS2; ++s) {
      mbar_init(bar(B_P2_FULL + s), 1);
      mbar_init(bar(B_P2_EMPTY + s), 1);
    }
    for (int f = 0; f < 2; ++f) {
      mbar_init(bar(B_F_FULL + f), 1);
      mbar_init(bar(B_F_FREE + f), 128);
    }
    mbar_init(bar(B_FINAL), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_sh)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_sh;
  const uint32_t tHrun = tmem + static_cast<uint32_t>(ND1 * L);          // running H: nu x L columns
  const uint32_t tF = tHrun + static_cast<uint32_t>(nu * L);             // fresh buffers: NF x L columns
  bool dead = false;

  // drain schedule of the direct mode: after tile i
  auto drain_tile = [&](int i) { return ((i + 1) % a.drain_every == 0) || (i == nt - 1); };

  if (warp == W_P1) {
    // ------------------------------------------------------------ phase-1 producer
    if (lane == 0 && NB > 0) {
      const uint64_t drop = l2_policy_evict_first(), keep = l2_policy_evict_last();
      uint32_t spos = 0, opos = 0;
      for (int i = 0; i < nt; ++i) {
        const int64_t tile = grp + static_cast<int64_t>(i) * NG;
        const int sgi = find_seg(a, tile);
        const void* tmap = &a.maps[sgi];
        const int32_t y0 = static_cast<int32_t>((tile - a.seg[sgi].tile0) * GR_ROWS);
        GRP_TRACE(i, 0);
        for (int b = 0; b < NB; ++b) {
          for (int hf = 0; hf < SPB; ++hf) {
            const uint32_t s = spos % a.ns1, k = spos / a.ns1;
            if (k >= 1 && !dead && !PWAIT_MBAR(bar(B_S1_EMPTY + s), (k - 1) & 1u)) dead = true;
            mbar_expect_tx(bar(B_S1_FULL + s), SBYTES);
            tma_load_2d_hint(su32(base + lay.st1) + s * STG, tmap, static_cast<int32_t>(f0 + 64 * b + 32 * hf), y0,
                             bar(B_S1_FULL + s), drop);
            ++spos;
          }
          const uint32_t o = opos % OM_R, ko = opos / OM_R;
          if (ko >= 1 && !dead && !PWAIT_MBAR(bar(B_OM_EMPTY + o), (ko - 1) & 1u)) dead = true;
          mbar_expect_tx(bar(B_OM_FULL + o), om_bytes);
          bulk_g2s_hint(su32(base + lay.om) + o * om_bytes, a.om16 + static_cast<int64_t>(blk0 + b) * L * 64,
                        om_bytes, bar(B_OM_FULL + o), keep);
          ++opos;
        }
        GRP_TRACE(i, 1);
        GRP_TRACE_ALL(i, 1);
      }
      // the last copies land before the CTA may leave
      for (uint32_t s = 0; s < static_cast<uint32_t>(a.ns1) && s < spos; ++s) {
        const uint32_t uses = (spos - s + a.ns1 - 1) / a.ns1;
        mbar_wait_fast(bar(B_S1_FULL + s), (uses - 1) & 1u);
      }
      for (uint32_t o = 0; o < OM_R && o < opos; ++o) {
        const uint32_t uses = (opos - o + OM_R - 1) / OM_R;
        mbar_wait_fast(bar(B_OM_FULL + o), (uses - 1) & 1u);
      }
    }
  } else if (warp == W_P2) {
    // ------------------------------------------------------------ phase-2 producer
    if (lane == 0 && NB > 0) {
      const uint64_t drop = l2_policy_evict_first();
      uint32_t ppos = 0;
      for (int i = 0; i < nt; ++i) {
        const int slot = i % RING_R;
        const unsigned use = static_cast<unsigned>(i / RING_R);
        const int ri = i % IMG_R;
        if (!dead && !PWAIT_MBAR(bar(B_IMG_READY + ri), static_cast<uint32_t>(i / IMG_R) & 1u)) dead = true;
        GRP_TRACE(i, 7);
        fence_proxy_async_global();   // the image (bulk writes of this CTA) before the bulk reads
        // G' of the tile: once every reducer of the group has published its rows
        auto load_g = [&]() {
          if (!dead && !PWAIT_GEQ(c_reduced(slot), static_cast<unsigned>(S) * (use + 1))) dead = true;
          GRP_TRACE(i, 8);
          fence_proxy_async_global();   // other CTAs' plain stores of G' before the bulk read
          if (i >= 1 && !dead && !PWAIT_MBAR(bar(B_GP_EMPTY), static_cast<uint32_t>(i - 1) & 1u)) dead = true;
          mbar_expect_tx(bar(B_GP_FULL), gp_bytes);
          bulk_g2s_hint(su32(base + lay.gp), gbuf_g + static_cast<int64_t>(slot) * (gp_bytes / 2), gp_bytes,
                        bar(B_GP_FULL), drop);
        };
        // the image units do not depend on G': the first NS2 of them go out before it
        const uint16_t* img_t = img_cta + static_cast<int64_t>(ri) * a.nbmax * (BLK16 / 2);
        int issued = 0;
        for (int u = 0; u < nu; ++u) {
          for (int h = 0; h < 2; ++h) {
            if (issued == NS2) load_g();
            const uint32_t s = ppos % NS2, k = ppos / NS2;
            if (k >= 1 && !dead && !PWAIT_MBAR(bar(B_P2_EMPTY + s), (k - 1) & 1u)) dead = true;
            mbar_expect_tx(bar(B_P2_FULL + s), P2U);
            const uint32_t dst = su32(base + lay.p2) + s * P2U;
            for (int e = 0; e < 2; ++e) {
              const int b = 2 * u + e;
              const uint16_t* src = b < NB ? img_t + static_cast<int64_t>(b) * (BLK16 / 2) + h * (BLK16 / 4)
                                           : a.zero8k;
              bulk_g2s_hint(dst + e * (P2U / 2), src, P2U / 2, bar(B_P2_FULL + s), drop);
            }
            ++ppos;
            ++issued;
          }
        }
        if (issued <= NS2) load_g();
        GRP_TRACE(i, 9);
        // once G' has landed, count it as loaded: the reducers may then reuse the slot
        if (!dead && !PWAIT_MBAR(bar(B_GP_FULL), static_cast<uint32_t>(i) & 1u)) dead = true;
        fence_proxy_async_global();
        red_release_add(c_loaded(slot), 1u);
      }
      for (uint32_t s = 0; s < NS2 && s < ppos; ++s) {
        const uint32_t uses = (ppos - s + NS2 - 1) / NS2;
        mbar_wait_fast(bar(B_P2_FULL + s), (uses - 1) & 1u);
      }
    }
  } else if (warp == W_MMA1) {
    // ------------------------------------------------------------ MMA1 issuer
    if (lane == 0 && NB > 0) {
      const uint32_t id1 = idesc_fmt<FMT>(GR_ROWS, L, 0, 0);
      uint32_t opos = 0;
      tc_fence_after();
      for (int i = 0; i < nt; ++i) {
        const int d = i % ND1;
        const uint32_t d1 = tmem + static_cast<uint32_t>(d * L);
        if (i >= ND1 && !dead && !PWAIT_MBAR(bar(B_D1_EMPTY + d), static_cast<uint32_t>(i / ND1 - 1) & 1u)) dead = true;
        tc_fence_after();
        for (int b = 0; b < NB; ++b) {
          const uint32_t p = opos & 1u, o = opos % OM_R;
          if (!dead && !PWAIT_MBAR(bar(B_OP_FULL + p), (opos >> 1) & 1u)) dead = true;
          if (!dead && !PWAIT_MBAR(bar(B_OM_FULL + o), (opos / OM_R) & 1u)) dead = true;
          tc_fence_after();
          if (!dead) {
            const uint64_t dA = sdesc(su32(base + lay.op) + p * BLK16, 16, 1024);
            const uint64_t dB = sdesc(su32(base + lay.om) + o * om_bytes, 16, 1024);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              mma_bf16(d1, dA + ((kk * 32u) >> 4), dB + ((kk * 32u) >> 4), id1, (b | kk) != 0 ? 1u : 0u);
          }
          mma_commit(bar(B_OP_EMPTY + p));
          mma_commit(bar(B_OM_EMPTY + o));
          ++opos;
        }
        mma_commit(bar(B_D1_FULL + d));
        GRP_TRACE(i, 3);
      }
    }
  } else if (warp == W_MMA2) {
    // ------------------------------------------------------------ MMA2 issuer
    if (lane == 0 && NB > 0) {
      const uint32_t id2 = idesc_fmt<FMT>(GR_ROWS, L, 1, 0);
      uint32_t ppos = 0, fuses = 0, drains = 0;
      tc_fence_after();
      for (int i = 0; i < nt; ++i) {
        if (!dead && !PWAIT_MBAR(bar(B_GP_FULL), static_cast<uint32_t>(i) & 1u)) dead = true;
        // direct mode: after a drain tile, H starts again from zero once the drain has read it
        const bool zero_h = !fresh && (i == 0 || drain_tile(i - 1));
        if (!fresh && i >= 1 && drain_tile(i - 1)) {
          if (!dead && !PWAIT_MBAR(bar(B_F_FREE), (drains - 1) & 1u)) dead = true;
        }
        tc_fence_after();
        for (int u = 0; u < nu; ++u) {
          const uint32_t fb = fresh ? fuses % NF : 0u;
          const uint32_t dst = fresh ? tF + fb * static_cast<uint32_t>(L) : tHrun + static_cast<uint32_t>(u * L);
          if (fresh && fuses >= static_cast<uint32_t>(NF) && !dead &&
              !PWAIT_MBAR(bar(B_F_FREE + fb), (fuses / NF - 1) & 1u))
            dead = true;
          tc_fence_after();
          for (int h = 0; h < 2; ++h) {
            const uint32_t s = ppos % NS2;
            if (!dead && !PWAIT_MBAR(bar(B_P2_FULL + s), (ppos / NS2) & 1u)) dead = true;
            tc_fence_after();
            if (!dead) {
              const uint64_t dA2 = sdesc(su32(base + lay.p2) + s * P2U, P2U / 2, 1024);   // MN-major: features x rows
              const uint64_t dB2 = sdesc(su32(base + lay.gp), 16, 1024);                  // K-major: L x rows
#pragma unroll
              for (int ks = 0; ks < 4; ++ks)
#pragma unroll
                for (int gsi = 0; gsi < GS; ++gsi) {
                  const bool first = (h == 0 && ks == 0 && gsi == 0) && (fresh || zero_h);
                  mma_bf16(dst, dA2 + ((static_cast<uint32_t>(ks) * 2048u) >> 4),
                           dB2 + ((static_cast<uint32_t>(gsi) * 2u * L * 128u + static_cast<uint32_t>(h) * L * 128u +
                                   static_cast<uint32_t>(ks) * 32u) >> 4),
                           id2, first ? 0u : 1u);
                }
            }
            mma_commit(bar(B_P2_EMPTY + s));
            ++ppos;
          }
          if (fresh) {
            mma_commit(bar(B_F_FULL + fb));
            ++fuses;
          }
        }
        mma_commit(bar(B_GP_EMPTY));
        GRP_TRACE(i, 10);
        // direct mode: every unit of this tile's image has landed, the copier may reuse the slot
        // (with fresh buffers the drain group says so, after dropping the lines from L2)
        if (!fresh) mbar_arrive(bar(B_IMG_FREE + i % IMG_R));
        if (!fresh && drain_tile(i)) {
          mma_commit(bar(B_F_FULL));
          ++drains;
        }
      }
      mma_commit(bar(B_FINAL));
      mbar_wait_fast(bar(B_FINAL), 0);
    }
  } else if (warp >= W_EPI0 && warp < W_EPI0 + 4) {
    // ------------------------------------------------------------ D1 -> the group's partials
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const int et = tid - W_EPI0 * 32;
    if (NB > 0) {
      for (int i = 0; i < nt; ++i) {
        const int d = i % ND1;
        const int slot = i % RING_R;
        const unsigned use = static_cast<unsigned>(i / RING_R);
        // the previous use of the slot has been reduced (the reducers read before they count)
        if (use >= 1 && !dead && !PWAIT_GEQ(c_reduced(slot), static_cast<unsigned>(S) * use)) dead = true;
        if (!dead && !PWAIT_MBAR(bar(B_D1_FULL + d), static_cast<uint32_t>(i / ND1) & 1u)) dead = true;
        tc_fence_after();
        float* dstp = part_g + (static_cast<int64_t>(slot) * S + j) * L * GR_ROWS;
        const uint32_t d1 = tmem + static_cast<uint32_t>(d * L) + (static_cast<uint32_t>(q * 32) << 16);
        for (int c0 = 0; c0 < L; c0 += 16) {
          uint32_t r[16];
          tmem_ld8_issue(d1 + static_cast<uint32_t>(c0), r);
          tmem_ld8_issue(d1 + static_cast<uint32_t>(c0 + 8), r + 8);
          tmem_wait_ld();
          if (c0 + 16 >= L) {   // D1 may take the next tile's MMA1 as soon as it has been read
            tc_fence_before();
            mbar_arrive(bar(B_D1_EMPTY + d));
          }
#pragma unroll
          for (int e = 0; e < 16; ++e) dstp[static_cast<int64_t>(c0 + e) * GR_ROWS + row] = __uint_as_float(r[e]);
        }
        // every thread's stores happen before thread 0's release: the barrier orders them, and a
        // release at GPU scope is cumulative (no fence per thread)
        named_bar(1, 128);
        if (et == 0) red_release_add(c_arrived(slot), 1u);
        if (et == 0) GRP_TRACE(i, 4);
        if (et == 0) GRP_TRACE_ALL(i, 0);
      }
    }
  } else if (warp >= W_DRN0 && warp < W_DRN0 + 4) {
    // ------------------------------------------------------------ H: fresh adds, drains
    const int q = warp & 3;
    const int r = q * 32 + lane;
    const uint32_t lq = static_cast<uint32_t>(q * 32) << 16;
    if (NB > 0) {
      auto store_h = [&](bool add) {
        for (int u = 0; u < nu; ++u) {
          const int64_t f = f0 + 128 * u + r;
          const bool own = f < fend && f < static_cast<int64_t>(a.nbt) * 64;
          float* hrow = a.Hpart + (static_cast<int64_t>(grp) * a.nbt * 64 + f) * L;
          for (int c0 = 0; c0 < L; c0 += 16) {
            uint32_t v[16];
            tmem_ld8_issue(tHrun + static_cast<uint32_t>(u * L + c0) + lq, v);
            tmem_ld8_issue(tHrun + static_cast<uint32_t>(u * L + c0 + 8) + lq, v + 8);
            tmem_wait_ld();
            if (!own) continue;
#pragma unroll
            for (int e4 = 0; e4 < 4; ++e4) {
              float x[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {   // H carries s^2, the column sums s
                const int c = c0 + 4 * e4 + e;
                x[e] = __uint_as_float(v[4 * e4 + e]) * (c == l ? inv_s : inv_s * inv_s);
              }
              if (add) red_add_v4(hrow + c0 + 4 * e4, x[0], x[1], x[2], x[3]);
              else *reinterpret_cast<float4*>(hrow + c0 + 4 * e4) = make_float4(x[0], x[1], x[2], x[3]);
            }
          }
        }
      };
      if (fresh) {
        uint32_t fuses = 0;
        for (int i = 0; i < nt; ++i) {
          for (int u = 0; u < nu; ++u) {
            const uint32_t fb = fuses % NF;
            if (!dead && !PWAIT_MBAR(bar(B_F_FULL + fb), (fuses / NF) & 1u)) dead = true;
            tc_fence_after();
            const uint32_t hb = tHrun + static_cast<uint32_t>(u * L) + lq;
            const uint32_t fbase = tF + fb * static_cast<uint32_t>(L) + lq;
            for (int c0 = 0; c0 < L; c0 += 16) {
              uint32_t fv[16], hv[16];
              tmem_ld8_issue(fbase + static_cast<uint32_t>(c0), fv);
              tmem_ld8_issue(fbase + static_cast<uint32_t>(c0 + 8), fv + 8);
              if (i > 0) {
                tmem_ld8_issue(hb + static_cast<uint32_t>(c0), hv);
                tmem_ld8_issue(hb + static_cast<uint32_t>(c0 + 8), hv + 8);
              }
              tmem_wait_ld();
#pragma unroll
              for (int e = 0; e < 16; ++e)
                hv[e] = i > 0 ? __float_as_uint(__uint_as_float(hv[e]) + __uint_as_float(fv[e])) : fv[e];
              tmem_st16(hb + static_cast<uint32_t>(c0), hv);
            }
            tmem_wait_st();
            tc_fence_before();
            mbar_arrive(bar(B_F_FREE + fb));
            ++fuses;
            // this M-tile's image blocks have been read (their bulk loads completed before MMA2):
            // drop their lines from L2 unwritten, so dead image data never goes back to HBM
            const uint8_t* img_t =
                reinterpret_cast<const uint8_t*>(img_cta + static_cast<int64_t>(i % IMG_R) * a.nbmax * (BLK16 / 2));
            for (int e = 0; e < 2; ++e) {
              const int b = 2 * u + e;
              if (b >= NB) continue;
              const uint8_t* blk = img_t + static_cast<int64_t>(b) * BLK16;
              for (int ln = r; ln < static_cast<int>(BLK16 / 128); ln += 128) discard_l2(blk + ln * 128);
            }
          }
          // the whole image of tile i is read and dropped: its slot may take tile i + IMG_R
          mbar_arrive(bar(B_IMG_FREE + i % IMG_R));
          if (r == 0) GRP_TRACE(i, 11);
        }
        if (nt > 0) store_h(false);
      } else {
        uint32_t drains = 0;
        for (int i = 0; i < nt; ++i) {
          if (!drain_tile(i)) continue;
          if (!dead && !PWAIT_MBAR(bar(B_F_FULL), drains & 1u)) dead = true;
          tc_fence_after();
          store_h(drains > 0);
          tc_fence_before();
          mbar_arrive(bar(B_F_FREE));
          ++drains;
        }
      }
    }
  } else if (warp >= W_RED0 && warp < W_RED0 + 4) {
    // ------------------------------------------------------------ reducers
    const int rt = tid - W_RED0 * 32;
    // G'^T G' (columns < l) in 4 x 2 blocks (a, b) of the lower triangle: block
    // p = rt + k RED_T is this thread's; its 8 entries are double-float pairs in shared memory
    // (sGram[(k RED_T + rt) 8 + e]). A row of G' then costs a 16-byte and an 8-byte load and
    // feeds 8 independent product-sums.
    const int npairs = a.npairs;
    auto block_ab = [&](int pidx, int& ba, int& bb) {
      ba = static_cast<int>((sqrtf(4.f * static_cast<float>(pidx) + 1.f) - 1.f) * 0.5f);
      while (ba * (ba + 1) > pidx) --ba;
      while ((ba + 1) * (ba + 2) <= pidx) ++ba;
      bb = pidx - ba * (ba + 1);
    };
    for (int k = 0; k < GRAM_BLK; ++k)
      if (rt + k * RED_T < npairs)
        for (int e = 0; e < 8; ++e) sGram[e * npairs + k * RED_T + rt] = make_float2(0.f, 0.f);
    F2Acc sg;
    const int nq = q1 - q0;
    for (int i = 0; i < nt; ++i) {
      const int slot = i % RING_R;
      const unsigned use = static_cast<unsigned>(i / RING_R);
      const int64_t tile = grp + static_cast<int64_t>(i) * NG;
      const int sgi = find_seg(a, tile);
      const int64_t row0 = (tile - a.seg[sgi].tile0) * GR_ROWS;
      const int64_t mseg = a.seg[sgi].m;
      if (rt == 0) {
        bool ok = dead || PWAIT_GEQ(c_arrived(slot), static_cast<unsigned>(S) * (use + 1));
        if (ok && use >= 1 && !dead) ok = PWAIT_GEQ(c_loaded(slot), static_cast<unsigned>(S) * use);
        red_go = ok ? 1u : 0u;
      }
      named_bar(2, RED_T);
      if (rt == 0) GRP_TRACE(i, 5);
      if (!red_go) dead = true;
      uint16_t* gdst = gbuf_g + static_cast<int64_t>(slot) * (gp_bytes / 2);
      const float* ps = part_g + static_cast<int64_t>(slot) * S * L * GR_ROWS;
      for (int it = rt; it < nq * L; it += RED_T) {
        const int qq = it / L, c = it % L;
        const int r4 = 4 * (q0 + qq);
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!dead) {
          // eight partials in flight at a time, added in CTA order (the same sum in every run)
          for (int jj0 = 0; jj0 < S; jj0 += 8) {
            float4 v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e)
              if (jj0 + e < S)
                v[e] = __ldcg(reinterpret_cast<const float4*>(ps + (static_cast<int64_t>(jj0 + e) * L + c) * GR_ROWS + r4));
#pragma unroll
            for (int e = 0; e < 8; ++e)
              if (jj0 + e < S) {
                acc.x += v[e].x; acc.y += v[e].y; acc.z += v[e].z; acc.w += v[e].w;
              }
          }
        }
        const float ac[4] = {acc.x, acc.y, acc.z, acc.w};
        float hi[4], lo[4], y[4];
        bool fin = true;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const bool valid = row0 + r4 + e < mseg;
          float x = ac[e];
          if (c == l) x = valid ? 1.f : 0.f;   // ones column: MMA2 makes the column sums
          else if (c > l || !valid) x = 0.f;
          hi[e] = round1<FMT>(x);
          fin = fin && isfinite(hi[e]);
          lo[e] = GS == 2 ? round1<FMT>(x - hi[e]) : 0.f;
          y[e] = hi[e] + lo[e];
          sRed[(4 * qq + e) * L + c] = y[e];
        }
        if (!fin) atomicOr(a.flags, 1);
        // G'^T, K-major with 128-byte swizzle: [part][row half][L rows of 128 bytes]
        const int kc = r4 >> 6, rr = r4 & 63;
        const uint32_t off = static_cast<uint32_t>(kc) * static_cast<uint32_t>(L) * 128u +
                             static_cast<uint32_t>(c >> 3) * 1024u + sw128(static_cast<uint32_t>(c & 7), rr * 2u);
        uint8_t* gb = reinterpret_cast<uint8_t*>(gdst);
        st_global_v2u(gb + off, pack2<FMT>(hi[0], hi[1]), pack2<FMT>(hi[2], hi[3]));
        if constexpr (GS == 2)
          st_global_v2u(gb + 2u * L * 128u + off, pack2<FMT>(lo[0], lo[1]), pack2<FMT>(lo[2], lo[3]));
      }
      named_bar(2, RED_T);
      // G' rows published (the barrier orders every thread's stores before the release); the
      // Gram products follow off the critical path, while the next tile's partials come in
      if (rt == 0) {
        GRP_TRACE(i, 13);
        red_release_add(c_reduced(slot), 1u);
        GRP_TRACE(i, 6);
      }
      // the Gram entries and sums of the own rows of G' (exact values hi + lo)
      for (int k = 0; k < GRAM_BLK; ++k) {
        const int pidx = rt + k * RED_T;
        if (pidx >= npairs) break;
        int ba, bb;
        block_ab(pidx, ba, bb);
        float2* gs = sGram + k * RED_T + rt;   // entry e at gs[e npairs]: consecutive threads, consecutive words
        F2Prod acc[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const float2 g = gs[e * npairs];
          acc[e].hi = g.x;
          acc[e].lo = g.y;
        }
        // four rows' operands loaded together, then their products (one load latency per four rows)
        for (int r0 = 0; r0 < rpc; r0 += 4) {
          float4 xa[4];
          float2 xb[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int rr = r0 + t < rpc ? r0 + t : r0;
            xa[t] = *reinterpret_cast<const float4*>(sRed + rr * L + 4 * ba);
            xb[t] = *reinterpret_cast<const float2*>(sRed + rr * L + 2 * bb);
          }
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            if (r0 + t >= rpc) break;
            const float va[4] = {xa[t].x, xa[t].y, xa[t].z, xa[t].w}, vb[2] = {xb[t].x, xb[t].y};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 2; ++v) acc[u * 2 + v].add_prod(va[u], vb[v]);
          }
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) gs[e * npairs] = make_float2(acc[e].hi, acc[e].lo);
      }
      if (rt == 0) GRP_TRACE(i, 14);
      if (rt < l)
        for (int rr = 0; rr < rpc; ++rr) sg.add(sRed[rr * L + rt]);
      if (a.gfull != nullptr) {   // the Gram matrix is formed after the launch from these rows
        float* gf = a.gfull + (tile * GR_ROWS + 4 * q0) * L;
        for (int it = rt; it < rpc * L; it += RED_T) {
          const int rr = it / L, c = it % L;
          gf[rr * L + c] = c < l ? sRed[rr * L + c] * inv_s : 0.f;
        }
      }
      if (a.seg[sgi].gout != nullptr) {
        for (int it = rt; it < rpc * l; it += RED_T) {
          const int rr = it / l, c = it % l;
          const int64_t grow = row0 + 4 * q0 + rr;
          if (grow < mseg) a.seg[sgi].gout[grow * l + c] = sRed[rr * L + c] * inv_s;
        }
      }
      if (rt == 0) GRP_TRACE(i, 15);
    }
    named_bar(2, RED_T);   // every thread is done with the last tile's rows
    // this CTA's Gram and sums partials
    const int LL = L * L;
    for (int e = rt; e < LL; e += RED_T) a.gram_part[cta * LL + e] = 0.0;
    named_bar(2, RED_T);
    const double s2 = static_cast<double>(inv_s) * inv_s;
    for (int k = 0; k < GRAM_BLK; ++k) {
      const int pidx = rt + k * RED_T;
      if (pidx >= npairs) break;
      int ba, bb;
      block_ab(pidx, ba, bb);
      const float2* gs = sGram + k * RED_T + rt;
      for (int u = 0; u < 4; ++u)
        for (int v = 0; v < 2; ++v) {
          const int c1 = 4 * ba + u, c2 = 2 * bb + v;
          if (c1 >= l || c2 > c1) continue;
          const float2 g = gs[(u * 2 + v) * npairs];
          const double val = (static_cast<double>(g.x) + static_cast<double>(g.y)) * s2;
          a.gram_part[cta * LL + c1 * L + c2] = val;
          a.gram_part[cta * LL + c2 * L + c1] = val;
        }
    }
    for (int c = rt; c < L; c += RED_T) a.sG_part[cta * L + c] = 0.0;
    named_bar(2, RED_T);
    if (rt < l) a.sG_part[cta * L + rt] = sg.value() * inv_s;
  } else if (warp == W_COPY) {
    // ------------------------------------------------------------ image copies
    if (lane == 0 && NB > 0) {
      const uint64_t keep = l2_policy_evict_last();
      uint32_t opos = 0;
      for (int i = 0; i < nt; ++i) {
        const int ri = i % IMG_R;
        uint16_t* img_t = img_cta + static_cast<int64_t>(ri) * a.nbmax * (BLK16 / 2);
        for (int b = 0; b < NB; ++b) {
          const uint32_t p = opos & 1u;
          if (!dead && !PWAIT_MBAR(bar(B_OP_FULL + p), (opos >> 1) & 1u)) dead = true;
          if (b == 0 && i >= IMG_R) {
            if (!dead && !PWAIT_MBAR(bar(B_IMG_FREE + ri), static_cast<uint32_t>(i / IMG_R - 1) & 1u)) dead = true;
            fence_proxy_async_global();   // the slot's discards before the bulk writes of the new tile
          }
          if (!dead) bulk_s2g_hint(img_t + static_cast<int64_t>(b) * (BLK16 / 2), su32(base + lay.op) + p * BLK16,
                                   BLK16, keep);
          bulk_commit();
          if (b > 0) {
            bulk_wait_read<1>();
            mbar_arrive(bar(B_OP_EMPTY + (p ^ 1u)));
          }
          ++opos;
        }
        bulk_wait_read<0>();
        mbar_arrive(bar(B_OP_EMPTY + ((opos - 1) & 1u)));
        bulk_wait_all();   // the image is in global memory before phase 2 loads it
        mbar_arrive(bar(B_IMG_READY + ri));
        GRP_TRACE(i, 12);
      }
    }
  } else if (warp >= W_CV0 && warp < W_CV0 + CV_W) {
    // ------------------------------------------------------------ converters
    const int ct = tid - W_CV0 * 32;   // 0..127
    uint32_t spos = 0, opos = 0;
    for (int i = 0; i < nt; ++i) {
      const int64_t tile = grp + static_cast<int64_t>(i) * NG;
      const int sgi = find_seg(a, tile);
      const int64_t row0 = (tile - a.seg[sgi].tile0) * GR_ROWS;
      const int64_t mseg = a.seg[sgi].m;
      const float xs = INP == IN_F8 ? a.seg[sgi].dscale * op_scale : op_scale;   // stored value -> scaled operand
      for (int b = 0; b < NB; ++b) {
        const uint32_t p = opos & 1u;
        if (opos >= 2 && !dead && !PWAIT_MBAR(bar(B_OP_EMPTY + p), ((opos >> 1) - 1) & 1u)) dead = true;
        uint8_t* op = base + lay.op + p * BLK16;
        // (x - c) s = fma(x, s, -c s) rounds once like the subtraction does (s a power of two; for
        // FP8, x = code and s = block scale x s, exact because the code has 4 significant bits
        // and the scale is taken as given). All loads of a stage first (they overlap), then the
        // conversions and stores; the stage goes back to the producer only after the stores.
        // cs: -c s of the 8 features fb..fb+7 (taken once per stage and reused for every row)
        auto shift8 = [&](int fb, float (&cs)[8]) {
#pragma unroll
          for (int e = 0; e < 8; ++e) cs[e] = -sShift[64 * b + fb + e] * op_scale;
        };
        auto put8 = [&](int r, int fb, const float (&xv)[8], const float (&cs)[8], bool valid) {
          float v[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] = valid ? fmaf(xv[e], xs, cs[e]) : 0.f;
          *reinterpret_cast<uint4*>(op + static_cast<uint32_t>(r >> 3) * 1024u +
                                    sw128(static_cast<uint32_t>(r & 7), static_cast<uint32_t>(fb) * 2u)) =
              make_uint4(pack2<FMT>(v[0], v[1]), pack2<FMT>(v[2], v[3]), pack2<FMT>(v[4], v[5]),
                         pack2<FMT>(v[6], v[7]));
        };
        for (int hf = 0; hf < SPB; ++hf) {
          const uint32_t s = spos % a.ns1;
          if (!dead && !PWAIT_MBAR(bar(B_S1_FULL + s), (spos / a.ns1) & 1u)) dead = true;
          const uint8_t* stg = base + lay.st1 + s * STG;
          if constexpr (INP == IN_F32) {
            // 128-byte rows of 32 features: thread = (8-feature piece cq, rows rb + 32 k)
            const int cq = ct & 3, rb = ct >> 2;
            const int fb = 32 * hf + 8 * cq;
            float cs[8];
            shift8(fb, cs);
            float4 x[8];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const int r = rb + 32 * k;
              x[2 * k] = *reinterpret_cast<const float4*>(stg + r * 128 + (((2 * cq) ^ (r & 7)) << 4));
              x[2 * k + 1] = *reinterpret_cast<const float4*>(stg + r * 128 + (((2 * cq + 1) ^ (r & 7)) << 4));
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const int r = rb + 32 * k;
              const float xv[8] = {x[2 * k].x, x[2 * k].y, x[2 * k].z, x[2 * k].w,
                                   x[2 * k + 1].x, x[2 * k + 1].y, x[2 * k + 1].z, x[2 * k + 1].w};
              put8(r, fb, xv, cs, row0 + r < mseg);
            }
          } else if constexpr (INP == IN_BF16) {
            // 128-byte rows of 64 features: thread = (16-byte chunk c8 = 8 features, rows rb + 16 k)
            const int c8 = ct & 7, rb = ct >> 3;
            float cs[8];
            shift8(8 * c8, cs);
            uint4 x[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const int r = rb + 16 * k;
              x[k] = *reinterpret_cast<const uint4*>(stg + r * 128 + ((c8 ^ (r & 7)) << 4));
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const int r = rb + 16 * k;
              const uint32_t w[4] = {x[k].x, x[k].y, x[k].z, x[k].w};
              float xv[8];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                xv[2 * e] = __uint_as_float(w[e] << 16);
                xv[2 * e + 1] = __uint_as_float(w[e] & 0xFFFF0000u);
              }
              put8(r, 8 * c8, xv, cs, row0 + r < mseg);
            }
          } else {
            // 64-byte rows of 64 codes, unswizzled: thread = (16-code chunk c4, rows rb + 32 k)
            const int c4 = ct & 3, rb = ct >> 2;
            float cs0[8], cs1[8];
            shift8(16 * c4, cs0);
            shift8(16 * c4 + 8, cs1);
            uint4 x[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) x[k] = *reinterpret_cast<const uint4*>(stg + (rb + 32 * k) * 64 + c4 * 16);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const int r = rb + 32 * k;
              const uint32_t w[4] = {x[k].x, x[k].y, x[k].z, x[k].w};
              float xv[16];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const float2 lo = fp8x2_e4m3_to_float2(static_cast<uint16_t>(w[e] & 0xFFFFu));
                const float2 hi = fp8x2_e4m3_to_float2(static_cast<uint16_t>(w[e] >> 16));
                xv[4 * e] = lo.x;
                xv[4 * e + 1] = lo.y;
                xv[4 * e + 2] = hi.x;
                xv[4 * e + 3] = hi.y;
              }
              const bool valid = row0 + r < mseg;
              const float x0[8] = {xv[0], xv[1], xv[2], xv[3], xv[4], xv[5], xv[6], xv[7]};
              const float x1[8] = {xv[8], xv[9], xv[10], xv[11], xv[12], xv[13], xv[14], xv[15]};
              put8(r, 16 * c4, x0, cs0, valid);
              put8(r, 16 * c4 + 8, x1, cs1, valid);
            }
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(bar(B_S1_EMPTY + s));
          ++spos;
        }
        fence_async_cta();   // the tensor cores and the bulk copy read what was written
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(B_OP_FULL + p));
        ++opos;
      }
      if (ct == 0) GRP_TRACE(i, 2);
    }
  }
#undef PWAIT_MBAR
#undef PWAIT_GEQ
  if (dead) atomicOr(a.flags, 2);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// The Gram matrix and nothing else from the G' rows of a launch (when l is too large for the
// reducers to hold its blocks): block p of the grid sums rows [r0, r1) of its share in the
// same 4 x 2 double-float blocks of the lower triangle as the reducers, 32 rows staged in
// shared memory at a time, and leaves gram_part[p] (both triangles, FP64) with sG_part[p] = 0.
constexpr int GRR_T = 512;
constexpr int GRR_ROWS = 32;
__global__ void __launch_bounds__(GRR_T) gram_rows_kernel(const float* __restrict__ G, int64_t rows, int l, int L,
                                                          double* __restrict__ gram_part,
                                                          double* __restrict__ sG_part) {
  extern __shared__ __align__(16) float gr_s[];   // GRR_ROWS x L
  const int npairs = gram_pairs(l);
  const int64_t per = (rows + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * per;
  const int64_t r1 = r0 + per < rows ? r0 + per : rows;
  constexpr int KMAX = 3;   // blocks per thread: gram_pairs(l) <= 3 x 512 for l <= 128 (na = 32: 1056)
  F2Prod acc[KMAX][8];
  int ba[KMAX], bb[KMAX];
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    const int pidx = threadIdx.x + k * GRR_T;
    ba[k] = -1;
    bb[k] = 0;
    if (pidx < npairs) {
      int a = static_cast<int>((sqrtf(4.f * static_cast<float>(pidx) + 1.f) - 1.f) * 0.5f);
      while (a * (a + 1) > pidx) --a;
      while ((a + 1) * (a + 2) <= pidx) ++a;
      ba[k] = a;
      bb[k] = pidx - a * (a + 1);
    }
  }
  for (int64_t c0 = r0; c0 < r1; c0 += GRR_ROWS) {
    const int nr = static_cast<int>(r1 - c0 < GRR_ROWS ? r1 - c0 : GRR_ROWS);
    __syncthreads();
    for (int e = threadIdx.x; e < nr * L / 4; e += GRR_T)
      reinterpret_cast<float4*>(gr_s)[e] = reinterpret_cast<const float4*>(G + c0 * L)[e];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
      if (ba[k] < 0) continue;
      for (int r = 0; r < nr; ++r) {
        const float4 xa = *reinterpret_cast<const float4*>(gr_s + r * L + 4 * ba[k]);
        const float2 xb = *reinterpret_cast<const float2*>(gr_s + r * L + 2 * bb[k]);
        const float va[4] = {xa.x, xa.y, xa.z, xa.w}, vb[2] = {xb.x, xb.y};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 2; ++v) acc[k][u * 2 + v].add_prod(va[u], vb[v]);
      }
    }
  }
  const int LL = L * L;
  double* out = gram_part + static_cast<int64_t>(blockIdx.x) * LL;
  for (int e = threadIdx.x; e < LL; e += GRR_T) out[e] = 0.0;
  for (int c = threadIdx.x; c < L; c += GRR_T) sG_part[static_cast<int64_t>(blockIdx.x) * L + c] = 0.0;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    if (ba[k] < 0) continue;
    for (int u = 0; u < 4; ++u)
      for (int v = 0; v < 2; ++v) {
        const int c1 = 4 * ba[k] + u, c2 = 2 * bb[k] + v;
        if (c1 >= l || c2 > c1) continue;
        const double val = static_cast<double>(acc[k][u * 2 + v].hi) + static_cast<double>(acc[k][u * 2 + v].lo);
        out[c1 * L + c2] = val;
        out[c2 * L + c1] = val;
      }
  }
}

// the self-test of the bounded waits: a counter nothing writes, and the outcome
__device__ unsigned g_never_written = 0;
__device__ int g_selftest_result = 0;

__global__ void wait_selftest_kernel(uint64_t limit_ns) {
  if (threadIdx.x == 0) g_selftest_result = wait_geq(&g_never_written, 1u, limit_ns) ? 1 : 2;
}

thread_local char g_grp_reason[192] = "";

}  // namespace

const char* grp_config_reason() { return g_grp_reason; }

// Choose the group size S and the stage count for (n, L): every CTA's H (nu M-tiles of L
// columns) must fit TMEM beside D1 (and the fresh buffer), the shared memory beside it; among
// the fits, the most block throughput (groups x blocks / the largest share of one CTA).
bool grp_config(int64_t n, int l, int L, int fmt, GrpConfig* cfg) {
  snprintf(g_grp_reason, sizeof(g_grp_reason), "no group size fits");
  if (!encode_fn()) {
    snprintf(g_grp_reason, sizeof(g_grp_reason), "cuTensorMapEncodeTiled is not available");
    return false;
  }
  if (L % 16 != 0 || L > 128 || l >= L) {
    snprintf(g_grp_reason, sizeof(g_grp_reason), "padded l = %d exceeds 128", L);
    return false;
  }
  // the reducers hold the Gram blocks of l <= 76; larger l forms the Gram matrix after each
  // launch from the G' rows the reducers write out
  const bool gram_in = gram_pairs(l) <= GRP_MAX_PAIRS;
  const int npairs = gram_in ? gram_pairs(l) : 0;
  const int gs = fmt == FMT_F16 ? 2 : 1;
  int dev = 0, sms = 0, optin = 0, coop = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop || sms < 1) {
    snprintf(g_grp_reason, sizeof(g_grp_reason), "cooperative launch is not available");
    return false;
  }
  const auto kern = fmt == FMT_F16 ? sketch_grp_kernel<FMT_F16, IN_F32> : sketch_grp_kernel<FMT_BF16, IN_F32>;
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) {
    cudaGetLastError();
    snprintf(g_grp_reason, sizeof(g_grp_reason), "kernel attributes unavailable");
    return false;
  }
  const int smem_max = optin - static_cast<int>(fa.sharedSizeBytes);
  const int nbt = static_cast<int>((n + 63) / 64);
  double best = 0.0;
  GrpConfig pick{};
  for (int S = 4; S <= sms && S <= nbt; ++S) {
    const int NG = sms / S;
    const int nbmax = (nbt + S - 1) / S;
    const int nu = (nbmax + 1) / 2;
    // TMEM: D1 (nd1 buffers), the running H (nu M-tiles) and nf fresh buffers, L columns each;
    // two fresh buffers let MMA2 run while the previous M-tile is added (worth a single D1)
    static const int opt_nd1[6] = {2, 1, 2, 1, 2, 1}, opt_nf[6] = {2, 2, 1, 1, 0, 0};
    static const double opt_w[6] = {1.0, 0.98, 0.85, 0.83, 0.8, 0.78};
    int oi = 0;
    while (oi < 6 && (opt_nd1[oi] + nu + opt_nf[oi]) * L > 512) ++oi;
    if (oi == 6) continue;
    const int nd1 = opt_nd1[oi], nf = opt_nf[oi];
    const int rpc = (32 + S - 1) / S * 4;
    int ns1 = 0;
    for (int k = 16; k >= 2; --k) {
      if (static_cast<int>(grp_layout(L, npairs, nbmax, k, gs, rpc).total) <= smem_max) {
        ns1 = k;
        break;
      }
    }
    if (ns1 == 0) continue;
    if (ns1 > 6) ns1 = 6;
    // block throughput, discounted for the partial traffic per block (L / (64 blocks))
    const double eff = static_cast<double>(NG) * nbt / nbmax / (1.0 + static_cast<double>(L) / (64.0 * nbmax)) *
                       opt_w[oi];
    if (eff > best) {
      best = eff;
      pick.S = S;
      pick.NG = NG;
      pick.nbt = nbt;
      pick.nbmax = nbmax;
      pick.nu = nu;
      pick.ns1 = ns1;
      pick.nd1 = nd1;
      pick.nf = nf;
      pick.smem = grp_layout(L, npairs, nbmax, ns1, gs, rpc).total;
      pick.gram_in = gram_in;
    }
  }
  if (best == 0.0) return false;
  // every storage format's variant of the kernel (same code size and static shared memory)
  const bool attr_ok =
      fmt == FMT_F16
          ? (cudaFuncSetAttribute(sketch_grp_kernel<FMT_F16, IN_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  smem_max) == cudaSuccess &&
             cudaFuncSetAttribute(sketch_grp_kernel<FMT_F16, IN_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  smem_max) == cudaSuccess &&
             cudaFuncSetAttribute(sketch_grp_kernel<FMT_F16, IN_F8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  smem_max) == cudaSuccess)
          : (cudaFuncSetAttribute(sketch_grp_kernel<FMT_BF16, IN_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  smem_max) == cudaSuccess &&
             cudaFuncSetAttribute(sketch_grp_kernel<FMT_BF16, IN_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  smem_max) == cudaSuccess &&
             cudaFuncSetAttribute(sketch_grp_kernel<FMT_BF16, IN_F8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  smem_max) == cudaSuccess);
  if (!attr_ok) {
    cudaGetLastError();
    snprintf(g_grp_reason, sizeof(g_grp_reason), "cannot raise the shared-memory limit");
    return false;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, GRP_NT, pick.smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    snprintf(g_grp_reason, sizeof(g_grp_reason), "the kernel does not fit one SM");
    return false;
  }
  *cfg = pick;
  return true;
}

size_t grp_img_elems(const GrpConfig& c) {
  return static_cast<size_t>(c.NG) * c.S * IMG_R * c.nbmax * (BLK16 / 2);
}
size_t grp_part_elems(const GrpConfig& c, int L) {
  return static_cast<size_t>(c.NG) * RING_R * c.S * L * GR_ROWS;
}
size_t grp_gbuf_elems(const GrpConfig& c, int L, int fmt) {
  return static_cast<size_t>(c.NG) * RING_R * (fmt == FMT_F16 ? 2 : 1) * 2 * L * 64;
}
size_t grp_cnt_elems(const GrpConfig& c) { return static_cast<size_t>(c.NG) * RING_R * 3; }

cudaError_t grp_wait_selftest(uint64_t limit_ns, cudaStream_t st, bool* ran_out) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(limit_ns);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int r = 0;
  e = cudaMemcpyFromSymbolAsync(&r, g_selftest_result, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  *ran_out = r == 2;
  return e;
}
// G' rows of one launch when the Gram matrix is formed after it: the tiles of every block a
// launch can hold (the batch closes at kTcPendingRows rows; a block has at most
// max_block_rows rows and one ragged tile)
size_t grp_gfull_rows(const GrpConfig& c, int64_t max_block_rows) {
  if (c.gram_in) return 0;
  const int64_t mb = max_block_rows > kTcPendingRows ? max_block_rows : kTcPendingRows;
  return static_cast<size_t>(mb + (kTcPendingRows + GR_ROWS - 1) / GR_ROWS * GR_ROWS + kTcPendingMax * GR_ROWS);
}

// One cooperative launch over the pending row blocks; *used = false (nothing launched) when a
// block cannot be described by a tensor map.
cudaError_t grp_pass(const State& s, const TcWork& w, const TcPending& pend, cudaStream_t st, Prof* prof,
                     bool* used) {
  *used = false;
  if (pend.nseg == 0) {
    *used = true;
    return cudaSuccess;
  }
  static_assert(kTcPendingMax <= MAX_SEGS, "segment capacity");
  GrpArgs args;
  std::memset(&args, 0, sizeof(args));
  const GrpConfig& cfg = w.grp;
  const int inp = pend.dtype == SPCA_BF16 ? IN_BF16 : (pend.dtype == SPCA_F8E4M3 ? IN_F8 : IN_F32);
  if (pend.dtype != SPCA_F32 && inp == IN_F32) return cudaSuccess;   // a storage format this kernel does not read
  const int es = inp == IN_F32 ? 4 : (inp == IN_BF16 ? 2 : 1);
  int64_t tiles = 0;
  for (int i = 0; i < pend.nseg; ++i) {
    const uintptr_t addr = reinterpret_cast<uintptr_t>(pend.rows[i]);
    if ((addr & 15u) != 0 || (pend.ld[i] * es) % 16 != 0) return cudaSuccess;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(s.n), static_cast<cuuint64_t>(pend.m[i])};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(pend.ld[i]) * es};
    cuuint32_t box[2] = {inp == IN_F32 ? 32u : 64u, GR_ROWS};
    cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType dt = inp == IN_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : (inp == IN_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8);
    const CUresult r = encode_fn()(&args.maps[i], dt, 2, const_cast<void*>(pend.rows[i]), dims, strides, box, estr,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE,
                                   inp == IN_F8 ? CU_TENSOR_MAP_SWIZZLE_NONE : CU_TENSOR_MAP_SWIZZLE_128B,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaSuccess;
    args.seg[i].m = pend.m[i];
    args.seg[i].gout = pend.gout[i];
    args.seg[i].dscale = inp == IN_F8 ? pend.dscale[i] : 1.f;
    args.seg[i].tile0 = tiles;
    tiles += (pend.m[i] + GR_ROWS - 1) / GR_ROWS;
  }
  if (!cfg.gram_in && tiles * GR_ROWS > w.gfull_rows) return cudaErrorInvalidValue;   // sized at creation
  const int NG = static_cast<int>(tiles < cfg.NG ? tiles : cfg.NG);
  args.nseg = pend.nseg;
  args.ntiles = tiles;
  args.n = s.n;
  args.l = s.l;
  args.L = s.L;
  args.S = cfg.S;
  args.NG = NG;
  args.nbt = cfg.nbt;
  args.nbmax = cfg.nbmax;
  args.nu = cfg.nu;
  args.ns1 = cfg.ns1;
  args.nd1 = cfg.nd1;
  args.nf = cfg.nf;
  args.drain_every = w.fmt == FMT_F16 ? 2 : 4;
  args.shift = s.shift;
  args.om16 = w.om16;
  args.zero8k = w.zero8k;
  args.img = w.img;
  args.part = w.part;
  args.gbuf = w.gbuf;
  args.cnt = w.cnt;
  args.scale = w.fmt == FMT_F16 ? w.scale : nullptr;
  args.npairs = cfg.gram_in ? gram_pairs(s.l) : 0;
  args.gfull = cfg.gram_in ? nullptr : w.gfull;
  args.Hpart = w.Hpart;
  args.gram_part = w.gram_part;
  args.sG_part = w.sG_part;
  args.flags = s.flags;
  args.wait_ns = w.wait_ns;
  args.trace = nullptr;
#ifdef SPCA_GRP_TRACE
  static unsigned long long* dtrace = nullptr;
  if (!dtrace) cudaMalloc(&dtrace, sizeof(unsigned long long) * 768);
  cudaMemsetAsync(dtrace, 0, sizeof(unsigned long long) * 768, st);
  args.trace = dtrace;
#endif

  cudaError_t e = cudaMemsetAsync(w.cnt, 0, sizeof(unsigned) * grp_cnt_elems(cfg), st);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(static_cast<unsigned>(NG * cfg.S), 1, 1);
  lc.blockDim = dim3(GRP_NT, 1, 1);
  lc.dynamicSmemBytes = cfg.smem;
  lc.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  prof->begin(SPCA_K_TC_SKETCH, st);
  if (w.fmt == FMT_F16)
    e = inp == IN_F32    ? cudaLaunchKernelEx(&lc, sketch_grp_kernel<FMT_F16, IN_F32>, args)
        : inp == IN_BF16 ? cudaLaunchKernelEx(&lc, sketch_grp_kernel<FMT_F16, IN_BF16>, args)
                         : cudaLaunchKernelEx(&lc, sketch_grp_kernel<FMT_F16, IN_F8>, args);
  else
    e = inp == IN_F32    ? cudaLaunchKernelEx(&lc, sketch_grp_kernel<FMT_BF16, IN_F32>, args)
        : inp == IN_BF16 ? cudaLaunchKernelEx(&lc, sketch_grp_kernel<FMT_BF16, IN_BF16>, args)
                         : cudaLaunchKernelEx(&lc, sketch_grp_kernel<FMT_BF16, IN_F8>, args);
  prof->end(SPCA_K_TC_SKETCH, st);
  if (e != cudaSuccess) return e;
  *used = true;
#ifdef SPCA_GRP_TRACE
  {
    unsigned long long h[768];
    cudaStreamSynchronize(st);
    cudaMemcpy(h, dtrace, sizeof(h), cudaMemcpyDeviceToHost);
    for (int k = 0; k < 2; ++k)
      for (int t = 8; t < 12; ++t) {
        fprintf(stderr, "grp %s tile %2d by CTA:", k == 0 ? "epi" : "p1end", t);
        for (int c = 0; c < 16; ++c)
          if (h[256 + 256 * k + 16 * c + t]) fprintf(stderr, " %.1f", (double)(h[256 + 256 * k + 16 * c + t] - h[0]) / 1000.0);
        fprintf(stderr, "\n");
      }
    const unsigned long long t0 = h[0];
    static const char* names[16] = {"p1beg", "p1end", "cvend", "mma1", "epi", "redgo", "reddone", "p2img",
                                    "p2g", "p2iss", "mma2", "drain", "imgrdy", "redsum", "redgram", "redfence"};
    for (int t = 0; t < 16; ++t) {
      fprintf(stderr, "grp tile %2d:", t);
      for (int ev = 0; ev < 16; ++ev)
        if (h[t * 16 + ev]) fprintf(stderr, " %s=%.1f", names[ev], (double)(h[t * 16 + ev] - t0) / 1000.0);
      fprintf(stderr, " us\n");
    }
  }
#endif
  e = launch_tc_finish(s, w, NG, static_cast<int64_t>(cfg.nbt) * 64, NG * cfg.S, st, prof);
  if (e != cudaSuccess || cfg.gram_in) return e;
  // the Gram matrix from the launch's G' rows (their partials reuse the reducers' slots, which
  // launch_tc_finish has consumed)
  const int64_t grows = tiles * GR_ROWS;
  int64_t P = (grows + 255) / 256;
  if (P > static_cast<int64_t>(NG) * cfg.S) P = static_cast<int64_t>(NG) * cfg.S;
  if (P < 1) P = 1;
  prof->begin(SPCA_K_GRAM_ACCUM, st);
  gram_rows_kernel<<<static_cast<unsigned>(P), GRR_T, sizeof(float) * GRR_ROWS * s.L, st>>>(w.gfull, grows, s.l, s.L,
                                                                                            w.gram_part, w.sG_part);
  e = launch_gram_accum(w.gram_part, w.sG_part, static_cast<int>(P), s.L, s.gram, s.sG, st);
  prof->end(SPCA_K_GRAM_ACCUM, st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace spca

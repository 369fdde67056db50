// The streaming pass on the tensor cores, pipelined across row tiles (Alg. 4 steps 5-7,
// Eq. 11). Same decomposition as sketch_tc.cu - a cluster of CS CTAs splits the n features
// (w per CTA), clusters walk 128-row tiles, the CS partials of A_hat Omega are reduced over
// distributed shared memory - but no CTA holds its 128 x w operand tile for the whole tile:
//  - phase 1 of tile i streams the slice of A from HBM (TMA, FP32, 64 features x 128 rows
//    per stage), converter warps subtract c, scale and round into a 16-bit operand buffer
//    (two 64-feature blocks), and MMA1 accumulates D1 = A_hat Omega in TMEM;
//  - the converted operand of each unit also goes out, by a bulk copy, to an image in global
//    memory (two tiles per CTA, kept in L2); phase 2 of tile i, once G(i) is known, bulk-loads
//    that image into the idle stage ring - half the bytes of the FP32 slice and no second
//    conversion - and MMA2 accumulates H += A_hat^T G' per 128-feature unit;
//  - a reduce group of four warps turns D1(i) into G'(i) (cluster reduction, rounding,
//    Gram matrix, sums, G^T operand) while the other warps already stream tile i+1: phase 1
//    of tile i+1 runs before phase 2 of tile i, so the latency of the reduction overlaps the
//    loads. D1 is double-buffered in TMEM.
// Roles (384 threads): warps 0-3 reduce group (TMEM lane quadrants 0-3), warps 4-9
// converters, warp 10 TMA producer, warp 11 MMA issuer. CTAs signal one another with
// mbarriers in shared memory (remote arrives at cluster scope), not with cluster-wide
// barriers, so that no role waits for another's unrelated work. Every wait is bounded; a
// thread that gives up sets flags[0] bit 2 and skips its later waits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <cstring>

#include "spca_internal.cuh"
#include "tc_ptx.cuh"

namespace spca {

namespace {

constexpr int T3_ROWS = 128;
constexpr int T3_NT = 384;
constexpr int RG_THREADS = 128;     // warps 0-3
constexpr int CV_WARP0 = 4, CV_WARPS = 6;
constexpr int CV_ROWS = (T3_ROWS + 2 * CV_WARPS - 1) / (2 * CV_WARPS);   // stage rows per converter lane
constexpr int PROD_WARP = 10, MMA3_WARP = 11;
constexpr int NSTAGE = 2;
constexpr uint32_t STAGE_BYTES = T3_ROWS * 64 * 4;   // FP32: 128 rows x 64 features
constexpr uint32_t BLOCK16 = T3_ROWS * 64 * 2;       // 16-bit: 128 rows x 64 features
constexpr int T3_MAX_UNITS = 6;                      // w <= 768
constexpr uint32_t GT_CHUNK = 128u * 128u;   // G^T operand chunk: 128 rows (hi, lo, zero) x 64 tile rows
constexpr int T3_GRAM_PER_THREAD = 4;        // G'^T G' entries per converter thread
constexpr uint32_t TMEM3_COLS = 512;
constexpr int T3_MAX_SEGS = 48;

}  // namespace

struct Tc3Layout {
  int RPC;
  uint32_t stage, pair, om, xch, gt, pub, shift, sy, bars, total;
};

// gs: 1, or 2 when G enters MMA2 as hi + lo
__host__ __device__ inline Tc3Layout tc3_layout(int L, int w, int CS, int gs) {
  Tc3Layout t;
  t.RPC = T3_ROWS / CS;
  uint32_t o = 0;
  t.stage = o; o += NSTAGE * STAGE_BYTES;
  t.pair = o; o += 2 * 2 * BLOCK16;                                     // two slots of two blocks
  t.om = o; o += 2u * static_cast<uint32_t>(L) * 128u;                  // Omega: two 64-feature chunks
  // the exchange rows of D1; the TMA drain of H (L a multiple of 32) stages its boxes in two
  // 16 KB halves of the same space, so it is never smaller than that
  uint32_t xch = ((T3_ROWS * static_cast<uint32_t>(L + 4) * 4u) + 1023u) & ~1023u;
  if (L % 32 == 0 && xch < 2u * 128u * 128u) xch = 2u * 128u * 128u;
  t.xch = o; o += xch;
  t.gt = o; o += 2u * GT_CHUNK;   // G^T: two chunks of 64 tile rows; rows [0,L) hi, [L,2L) lo, rest 0
  t.pub = o; o += 2u * static_cast<uint32_t>(L * gs) * (t.RPC / 8) * 16u;   // two tile parities
  t.shift = o; o += ((static_cast<uint32_t>(w) * 4u) + 15u) & ~15u;
  t.sy = o; o += ((static_cast<uint32_t>(t.RPC) * L * 4u) + 15u) & ~15u;
  t.bars = o; o += 16u * 32u;
  t.total = o + 1024u;
  return t;
}

struct Tc3Seg {
  int64_t m;
  float* gout;
  int64_t tile0;
};

struct Tc3Args {
  CUtensorMap maps[T3_MAX_SEGS];   // per row block: FP32 rows, box 64 features x 128 rows
  CUtensorMap hmap;                // the H partials (L columns x all rows), box 32 columns x 128 rows, 128-byte swizzle
  Tc3Seg seg[T3_MAX_SEGS];
  int nseg;
  int64_t ntiles;
  int64_t n;
  int l, L, w, CS;
  int drain_every;
  const float* shift;
  const uint16_t* om16;
  uint16_t* img;               // operand images: per CTA two tiles of w / 128 units (128 x 128, 16-bit)
  int64_t img_halves;          // its size; a copy that would leave it is skipped and flags[0] bit 3 set
  const float* scale;
  float* Hpart;
  double* gram_part;
  double* sG_part;
  int* flags;
  unsigned long long* trace;   // phase timestamps of cluster 0, CTA 0 (builds with SPCA_TC_TRACE only)
};

#ifdef SPCA_TC_TRACE
#define T3_TRACE(ti, slot)                                                               \
  do {                                                                                    \
    if (rank == 0 && cid == 0 && (ti) >= 0 && (ti) < 8 && a.trace) {                      \
      unsigned long long t_;                                                              \
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_));                              \
      a.trace[(ti) * 16 + (slot)] = t_;                                                   \
    }                                                                                     \
  } while (0)
// stage events of tile 3: a.trace[128 + 4 * stage + event]
#define T3_STRACE(ti, stage, ev)                                                          \
  do {                                                                                    \
    if (rank == 0 && cid == 0 && (ti) == 3 && (stage) < 32 && a.trace) {                 \
      unsigned long long t_;                                                              \
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_));                              \
      a.trace[128 + (stage) * 8 + (ev)] = t_;                                             \
    }                                                                                     \
  } while (0)
#else
#define T3_STRACE(ti, stage, ev) \
  do {                           \
  } while (0)
#define T3_TRACE(ti, slot) \
  do {                     \
  } while (0)
#endif

namespace {

__device__ __forceinline__ int find_seg3(const Tc3Args& a, int64_t tile) {
  int sgi = 0;
  while (sgi + 1 < a.nseg && a.seg[sgi + 1].tile0 <= tile) ++sgi;
  return sgi;
}

// barrier slots
enum {
  // a ring slot holds a phase-1 stage or a phase-2 unit; each kind has its own full and
  // empty barriers, so that a waiter, which sees only its own kind, is never more than one
  // phase ahead of the barrier it polls by parity
  B_STAGE_FULL = 0,                        // [NSTAGE] a phase-1 stage landed
  B_STAGE_EMPTY = B_STAGE_FULL + NSTAGE,   // [NSTAGE] a phase-1 stage was converted
  B_UNIT_FULL = B_STAGE_EMPTY + NSTAGE,    // [NSTAGE] a phase-2 unit landed
  B_SLOT_EMPTY = B_UNIT_FULL + NSTAGE,     // [NSTAGE] a phase-2 unit was consumed by MMA2
  B_PAIR_FULL = B_SLOT_EMPTY + NSTAGE,   // [2]
  B_PAIR_EMPTY = B_PAIR_FULL + 2,
  B_OM_FULL = B_PAIR_EMPTY + 2,
  B_OM_EMPTY,
  B_D1_FULL,                           // [2]
  B_D1_EMPTY = B_D1_FULL + 2,          // [2]
  B_G_READY = B_D1_EMPTY + 2,          // [2] a tile's G^T is in every CTA of the cluster (by tile parity)
  B_MMA2_DONE = B_G_READY + 2,                         // [2] a tile's MMA2 has completed (by tile parity)
  B_XCH_READY = B_MMA2_DONE + 2,
  B_XCH_FREE,
  B_PEER_FREE,                         // every peer's G^T buffer may be written (cluster scope)
  B_GT_FULL,                           // every peer has stored its rows of G^T here (cluster scope)
  B_FINAL,                             // the MMA issuer's last commit
  B_IMG_READY,                         // [2] a tile's operand image is in global memory (tile parity)
  B_GT_FREE = B_IMG_READY + 2,         // [2] the converters' Gram products are done with a tile's G^T
  B_COUNT = B_GT_FREE + 2
};
static_assert(B_COUNT <= 64, "barrier slots: 16 x 32 bytes in the layout");

// tile i of this cluster is a drain tile: H leaves TMEM after its MMA2
// (clusters drain at staggered tiles, so that not all of them load L2 with reductions at once)
__device__ __forceinline__ bool drain_tile(int i, int nt, int every, uint32_t cid) {
  return ((i + 1 + static_cast<int>(cid)) % every == 0) || (i == nt - 1);
}

template <int FMT>
__global__ void __launch_bounds__(T3_NT, 1) sketch_tc3_kernel(const __grid_constant__ Tc3Args a) {
  constexpr int GS = FMT == FMT_F16 ? 2 : 1;
  // G^T buffers: without the lo terms (BF16) the rows [L, 2L) of the chunks hold a second
  // tile's G^T, so a tile's G^T may be stored while the previous tile's MMA2 still reads its own
  constexpr int GT_NB = GS == 1 ? 2 : 1;
  extern __shared__ __align__(1024) uint8_t smem3[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem3) + 1023) & ~uintptr_t(1023));
  const int L = a.L, w = a.w, CS = a.CS, l = a.l;
  const Tc3Layout lay = tc3_layout(L, w, CS, GS);
  const int RPC = lay.RPC, G8 = RPC / 8;
  const float* sStage = reinterpret_cast<const float*>(base + lay.stage);
  uint8_t* sPair = base + lay.pair;
  uint8_t* sOm = base + lay.om;
  float* sX = reinterpret_cast<float*>(base + lay.xch);
  uint8_t* sGt = base + lay.gt;
  uint4* sPub = reinterpret_cast<uint4*>(base + lay.pub);
  float* sShift = reinterpret_cast<float*>(base + lay.shift);
  float* sY = reinterpret_cast<float*>(base + lay.sy);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + lay.bars);
  auto bar = [&](int i) { return su32(&bars[i]); };
  __shared__ uint32_t tmem_sh;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const uint32_t rank = cluster_rank();
  const uint32_t cid = cluster_id();
  const uint32_t ncl = cluster_count();
  const int64_t n = a.n;
  const int64_t f0 = static_cast<int64_t>(rank) * w;
  const int U = w / 128;
  const int xld = L + 4;
  const uint32_t chunk_bytes = static_cast<uint32_t>(L) * 128u;
  const int64_t g0 = f0 / 64;
  const int nt = cid < a.ntiles ? static_cast<int>((a.ntiles - 1 - cid) / ncl + 1) : 0;   // local tiles
  const float op_scale = a.scale ? *a.scale : 1.f;
  constexpr uint32_t UNIT_BYTES = 2 * BLOCK16;   // one 128 x 128 operand unit
  static_assert(STAGE_BYTES == UNIT_BYTES, "a ring slot holds a stage or a unit");
  const int64_t img_cta = (static_cast<int64_t>(cid) * CS + rank) * 2 * U * (UNIT_BYTES / 2);
  auto img_off = [&](int ti, int u) { return img_cta + (static_cast<int64_t>(ti & 1) * U + u) * (UNIT_BYTES / 2); };
  auto img_ok = [&](int64_t off) {
    const bool ok = off >= 0 && off + UNIT_BYTES / 2 <= a.img_halves;
    if (!ok) atomicOr(a.flags, 8);
    return ok;
  };
  const float inv_s = 1.f / op_scale;

  for (int i = tid; i < w; i += T3_NT) sShift[i] = (f0 + i < n) ? a.shift[f0 + i] : 0.f;
  // the rows of the G^T chunks that no pull writes (lo terms when not split, padding) stay 0
  for (uint32_t i = tid; i < 2u * GT_CHUNK / 16u; i += T3_NT) reinterpret_cast<uint4*>(sGt)[i] = make_uint4(0, 0, 0, 0);
  fence_async_cta();   // the tensor cores read these zeros
  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(bar(B_STAGE_FULL + s), 1);
      mbar_init(bar(B_STAGE_EMPTY + s), CV_WARPS);
      mbar_init(bar(B_UNIT_FULL + s), 1);
      mbar_init(bar(B_SLOT_EMPTY + s), 1);
    }
    for (int p = 0; p < 2; ++p) {
      mbar_init(bar(B_PAIR_FULL + p), CV_WARPS);
      mbar_init(bar(B_PAIR_EMPTY + p), 2);   // MMA1 done, and the image copy has read the slot
      mbar_init(bar(B_D1_FULL + p), 1);
      mbar_init(bar(B_D1_EMPTY + p), RG_THREADS);
      mbar_init(bar(B_MMA2_DONE + p), 1);
      mbar_init(bar(B_G_READY + p), RG_THREADS);
      mbar_init(bar(B_GT_FREE + p), CV_WARPS);
    }
    mbar_init(bar(B_OM_FULL), 1);
    mbar_init(bar(B_OM_EMPTY), 1);
    mbar_init(bar(B_XCH_READY), static_cast<uint32_t>(CS));
    mbar_init(bar(B_XCH_FREE), static_cast<uint32_t>(CS));
    mbar_init(bar(B_FINAL), 1);
    mbar_init(bar(B_PEER_FREE), static_cast<uint32_t>(CS));
    mbar_init(bar(B_GT_FULL), static_cast<uint32_t>(CS));
    mbar_init(bar(B_IMG_READY), 1);
    mbar_init(bar(B_IMG_READY + 1), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_sh)),
                 "r"(TMEM3_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();   // every peer's barriers are initialised before the first remote arrive
  tc_fence_after();
  const uint32_t tmem = tmem_sh;
  const uint32_t tH = tmem + 2u * static_cast<uint32_t>(L);   // D1 buffers at columns [0, 2L)
  bool dead = false;

  if (warp == PROD_WARP) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      // the ring: phase 1 of tile i+1 (2U FP32 stages), then phase 2 of tile i (U image units)
      // per ring slot (two, kept in registers): fills of each kind and the kind of the last one
      static_assert(NSTAGE == 2, "two ring slots");
      uint32_t pos = 0, om_fills = 0;
      uint32_t n1a = 0, n1b = 0, n2a = 0, n2b = 0;
      int lasta = 0, lastb = 0;
      const uint64_t keep = l2_policy_evict_last(), drop = l2_policy_evict_first();
      auto claim = [&](int s) {   // the previous fill of ring slot s has been consumed
        const int last = s ? lastb : lasta;
        const uint32_t n1 = s ? n1b : n1a, n2 = s ? n2b : n2a;
        if (last == 1 && !dead && !mbar_wait(bar(B_STAGE_EMPTY + s), (n1 - 1) & 1u)) dead = true;
        if (last == 2 && !dead && !mbar_wait(bar(B_SLOT_EMPTY + s), (n2 - 1) & 1u)) dead = true;
      };
      auto filled = [&](int s, int kind) {
        if (s) { lastb = kind; if (kind == 1) ++n1b; else ++n2b; }
        else { lasta = kind; if (kind == 1) ++n1a; else ++n2a; }
      };
      for (int i = -1; i < nt; ++i) {
        if (i + 1 < nt) {
          const int ti = i + 1;
          const int64_t tile = cid + static_cast<int64_t>(ti) * ncl;
          const int sgi = find_seg3(a, tile);
          const void* tmap = &a.maps[sgi];
          const int32_t y0 = static_cast<int32_t>((tile - a.seg[sgi].tile0) * T3_ROWS);
          T3_TRACE(ti, 0);
          for (int u = 0; u < U; ++u) {
            for (int b = 0; b < 2; ++b) {
              const int s = static_cast<int>(pos % NSTAGE);
              T3_STRACE(ti, 2 * u + b, 3);
              claim(s);
              mbar_expect_tx(bar(B_STAGE_FULL + s), STAGE_BYTES);
              T3_STRACE(ti, 2 * u + b, 0);
              tma_load_2d_hint(su32(sStage) + s * STAGE_BYTES, tmap, static_cast<int32_t>(f0 + 64 * (2 * u + b)),
                               y0, bar(B_STAGE_FULL + s), drop);
              filled(s, 1);
              ++pos;
            }
            // Omega chunks of this unit for MMA1 (one slot: after the rows are on their way)
            if (om_fills > 0 && !dead && !mbar_wait(bar(B_OM_EMPTY), (om_fills - 1) & 1u)) dead = true;
            mbar_expect_tx(bar(B_OM_FULL), 2 * chunk_bytes);
            for (int c = 0; c < 2; ++c)
              bulk_g2s_hint(su32(sOm) + c * chunk_bytes, a.om16 + (g0 + 2 * u + c) * static_cast<int64_t>(L) * 64,
                            chunk_bytes, bar(B_OM_FULL), keep);
            ++om_fills;
          }
        }
        if (i >= 0) {
          const int ti = i;
          T3_TRACE(ti, 1);
          // the converters have written this tile's image (all its bulk copies complete)
          // (one barrier per tile parity: the other parity's next tile cannot complete before this wait)
          if (!dead && !mbar_wait(bar(B_IMG_READY + (ti & 1)), static_cast<uint32_t>(ti >> 1) & 1u)) dead = true;
          for (int u = 0; u < U; ++u) {
            const int s = static_cast<int>(pos % NSTAGE);
            claim(s);
            mbar_expect_tx(bar(B_UNIT_FULL + s), UNIT_BYTES);
            const int64_t off = img_off(ti, u);
            if (img_ok(off))
              bulk_g2s_hint(su32(sStage) + s * STAGE_BYTES, a.img + off, UNIT_BYTES, bar(B_UNIT_FULL + s), drop);
            else
              mbar_complete_tx(bar(B_UNIT_FULL + s), UNIT_BYTES);   // complete the phase without a copy
            filled(s, 2);
            ++pos;
          }
        }
      }
      // let the last copies land before the CTA may exit
      if (n1a > 0) mbar_wait(bar(B_STAGE_FULL + 0), (n1a - 1) & 1u);
      if (n1b > 0) mbar_wait(bar(B_STAGE_FULL + 1), (n1b - 1) & 1u);
      if (n2a > 0) mbar_wait(bar(B_UNIT_FULL + 0), (n2a - 1) & 1u);
      if (n2b > 0) mbar_wait(bar(B_UNIT_FULL + 1), (n2b - 1) & 1u);
      if (om_fills > 0) mbar_wait(bar(B_OM_FULL), (om_fills - 1) & 1u);
    }
  } else if (warp >= CV_WARP0 && warp < CV_WARP0 + CV_WARPS) {
    // ------------------------------------------------------------ converters
    const int cw = warp - CV_WARP0;
    constexpr int CVT = CV_WARPS * 32;
    const int ctid = tid - CV_WARP0 * 32;
    const uint64_t keep = l2_policy_evict_last();
    uint32_t pos = 0, units = 0, f1a = 0, f1b = 0;   // ring position; phase-1 fills seen per slot
    // G'^T G' (columns < l, lower triangle): once G^T of a tile is pulled every CTA holds all 128
    // of its rows, so the cluster splits the entries - this thread takes e = rank CVT + ctid +
    // k CVT CS - and works on them while phase 2 of the tile runs. Products of the 16-bit terms
    // are exact in FP32 and summed as double-float pairs.
    const int LTl = l * (l + 1) / 2;
    F2Acc gram_acc[T3_GRAM_PER_THREAD];
    int gc1[T3_GRAM_PER_THREAD], gc2[T3_GRAM_PER_THREAD];
#pragma unroll
    for (int k = 0; k < T3_GRAM_PER_THREAD; ++k) {
      const int e = static_cast<int>(rank) * CVT + ctid + k * CVT * CS;
      int c1 = 0, c2 = 0;
      if (e < LTl) {
        c1 = static_cast<int>((sqrtf(8.f * static_cast<float>(e) + 1.f) - 1.f) * 0.5f);
        while (c1 * (c1 + 1) / 2 > e) --c1;
        while ((c1 + 1) * (c1 + 2) / 2 <= e) ++c1;
        c2 = e - c1 * (c1 + 1) / 2;
      }
      gc1[k] = e < LTl ? c1 : -1;
      gc2[k] = c2;
    }
    auto gt_off = [&](int h, int lc, int g) {
      return static_cast<uint32_t>(g >> 3) * GT_CHUNK + static_cast<uint32_t>((h * L + lc) >> 3) * 1024u +
             sw128(static_cast<uint32_t>(lc & 7), static_cast<uint32_t>(g & 7) * 16u);
    };
    for (int i = -1; i < nt; ++i) {
      if (i + 1 < nt) {
        const int ti = i + 1;
        const int64_t tile = cid + static_cast<int64_t>(ti) * ncl;
        const int sgi = find_seg3(a, tile);
        const int64_t row0 = (tile - a.seg[sgi].tile0) * T3_ROWS;
        const int64_t mseg = a.seg[sgi].m;
        for (int u = 0; u < U; ++u) {
          const uint32_t p = units & 1u;
          if (units >= 2 && !dead && !mbar_wait(bar(B_PAIR_EMPTY + p), ((units >> 1) - 1) & 1u)) dead = true;
          uint8_t* slot = sPair + p * 2 * BLOCK16;
          for (int b = 0; b < 2; ++b) {
            const int s = static_cast<int>(pos % NSTAGE);
            const uint32_t f1 = s ? f1b++ : f1a++;
            if (cw == 0 && lane == 0) T3_STRACE(ti, 2 * u + b, 1);
            if (!dead && !mbar_wait(bar(B_STAGE_FULL + s), f1 & 1u)) dead = true;
            if (cw == 0 && lane == 0) T3_STRACE(ti, 2 * u + b, 2);
            const float* src = sStage + s * (STAGE_BYTES / 4);
            const int fb = 2 * u + b;
            // lane: features 4 (lane % 16) .. +3 of row 2 k + lane / 16; (x - c) s = fma(x, s, -c s)
            // rounds once like the subtraction does (s is a power of two)
            const int fl = 4 * (lane & 15);
            const float4 sh = *reinterpret_cast<const float4*>(sShift + fb * 64 + fl);
            const float4 cs = make_float4(-sh.x * op_scale, -sh.y * op_scale, -sh.z * op_scale, -sh.w * op_scale);
            // all of the warp's rows of the stage are loaded before any is converted (the loads
            // overlap). The stage goes back to the producer only after the stores that consume
            // every loaded value: an arrive issued while shared-memory loads are outstanding
            // does not wait for them, and the next TMA fill could overwrite the stage first.
            const int rl = 2 * cw + (lane >> 4);
            float4 x[CV_ROWS];
#pragma unroll
            for (int j = 0; j < CV_ROWS; ++j) {
              const int r = rl + 2 * CV_WARPS * j;
              x[j] = r < T3_ROWS ? *reinterpret_cast<const float4*>(src + r * 64 + fl) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int j = 0; j < CV_ROWS; ++j) {
              const int r = rl + 2 * CV_WARPS * j;
              if (r >= T3_ROWS) continue;
              const bool valid = row0 + r < mseg;
              const float v0 = valid ? fmaf(x[j].x, op_scale, cs.x) : 0.f;
              const float v1 = valid ? fmaf(x[j].y, op_scale, cs.y) : 0.f;
              const float v2 = valid ? fmaf(x[j].z, op_scale, cs.z) : 0.f;
              const float v3 = valid ? fmaf(x[j].w, op_scale, cs.w) : 0.f;
              const uint32_t off = static_cast<uint32_t>(b) * BLOCK16 + static_cast<uint32_t>(r >> 3) * 1024u +
                                   sw128(static_cast<uint32_t>(r & 7), static_cast<uint32_t>(fl) * 2u);
              *reinterpret_cast<uint2*>(slot + off) = make_uint2(pack2<FMT>(v0, v1), pack2<FMT>(v2, v3));
            }
            __syncwarp();
            if (cw == 0 && lane == 0) T3_STRACE(ti, 2 * u + b, 4);
            if (lane == 0) mbar_arrive(bar(B_STAGE_EMPTY + s));
            ++pos;
          }
          fence_async_cta();
          __syncwarp();
          if (lane == 0) mbar_arrive(bar(B_PAIR_FULL + p));
          if (cw == 0 && lane == 0) {
            // once every converter is done with the unit, copy it out for phase 2; the copy of
            // the tile's previous unit has read its slot by now or soon: release that slot
            if (!dead && !mbar_wait(bar(B_PAIR_FULL + p), (units >> 1) & 1u)) dead = true;
            const int64_t off = img_off(ti, u);
            if (img_ok(off)) bulk_s2g_hint(a.img + off, su32(slot), UNIT_BYTES, keep);
            bulk_commit();
            if (u > 0) {
              bulk_wait_read<1>();
              mbar_arrive(bar(B_PAIR_EMPTY + (p ^ 1u)));
            }
          }
          ++units;
        }
        if (cw == 0 && lane == 0) {
          // the tile's image is complete in global memory: phase 2 may load it
          bulk_wait_all();
          mbar_arrive(bar(B_PAIR_EMPTY + ((units - 1) & 1u)));
          mbar_arrive(bar(B_IMG_READY + (ti & 1)));
        }
        __syncwarp();
        if (cw == 0 && lane == 0) T3_TRACE(ti, 2);
      }
      if (i >= 0) {
        pos += U;   // phase 2 of tile i passes through the ring without the converters
        // meanwhile: this thread's entries of G'^T G' over the tile's 128 rows
        if (!dead && !mbar_wait(bar(B_G_READY + (i & 1)), static_cast<uint32_t>(i >> 1) & 1u)) dead = true;
        const int hb = GT_NB == 2 ? (i & 1) : 0;   // the rows of tile i's G^T buffer
#pragma unroll
        for (int k = 0; k < T3_GRAM_PER_THREAD; ++k) {
          if (gc1[k] < 0) continue;
          for (int g = 0; g < T3_ROWS / 8; ++g) {
            float x1[GS][8], x2[GS][8];
#pragma unroll
            for (int h = 0; h < GS; ++h) {
              unpack8<FMT>(*reinterpret_cast<const uint4*>(sGt + gt_off(h + hb, gc1[k], g)), x1[h]);
              unpack8<FMT>(*reinterpret_cast<const uint4*>(sGt + gt_off(h + hb, gc2[k], g)), x2[h]);
            }
#pragma unroll
            for (int r = 0; r < 8; ++r) {
              gram_acc[k].add(x1[0][r] * x2[0][r]);
              if constexpr (GS == 2) {
                gram_acc[k].add(x1[0][r] * x2[1][r]);
                gram_acc[k].add(x1[1][r] * x2[0][r]);
                gram_acc[k].add(x1[1][r] * x2[1][r]);
              }
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(B_GT_FREE + (i & 1)));
      }
    }
    {
      const int LL = L * L;
      const int64_t cta = static_cast<int64_t>(cid) * CS + rank;
      for (int e = ctid; e < LL; e += CVT) a.gram_part[cta * LL + e] = 0.0;
      named_bar(2, CVT);
      const double s2 = static_cast<double>(inv_s) * inv_s;
#pragma unroll
      for (int k = 0; k < T3_GRAM_PER_THREAD; ++k) {
        if (gc1[k] < 0) continue;
        const double v = gram_acc[k].value() * s2;
        a.gram_part[cta * LL + gc1[k] * L + gc2[k]] = v;
        a.gram_part[cta * LL + gc2[k] * L + gc1[k]] = v;
      }
    }
  } else if (warp == MMA3_WARP) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t id1 = idesc_fmt<FMT>(T3_ROWS, L, 0, 0);
      const uint32_t id2 = idesc_fmt<FMT>(T3_ROWS, L, 1, 0);
      uint32_t pos = 0, units = 0, om_uses = 0, f2a = 0, f2b = 0;   // phase-2 fills seen per slot
      tc_fence_after();
      for (int i = -1; i < nt; ++i) {
        if (i + 1 < nt) {   // MMA1 of tile i+1 on the converted units
          const int ti = i + 1;
          const uint32_t d1 = tmem + static_cast<uint32_t>((ti & 1) * L);
          if (ti >= 2 && !dead && !mbar_wait(bar(B_D1_EMPTY + (ti & 1)), ((ti >> 1) - 1) & 1u)) dead = true;
          tc_fence_after();
          for (int u = 0; u < U; ++u) {
            const uint32_t p = units & 1u;
            if (!dead && !mbar_wait(bar(B_PAIR_FULL + p), (units >> 1) & 1u)) dead = true;
            const uint32_t slot = su32(sPair) + p * 2 * BLOCK16;
            if (!dead && !mbar_wait(bar(B_OM_FULL), om_uses & 1u)) dead = true;
            tc_fence_after();
            if (!dead) {
              const uint64_t dA = sdesc(slot, 16, 1024);
              const uint64_t dB = sdesc(su32(sOm), 16, 1024);
#pragma unroll
              for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                  mma_bf16(d1, dA + ((static_cast<uint32_t>(b) * BLOCK16 + kk * 32u) >> 4),
                           dB + ((static_cast<uint32_t>(b) * chunk_bytes + kk * 32u) >> 4), id1,
                           (u | b | kk) != 0 ? 1u : 0u);
            }
            mma_commit(bar(B_OM_EMPTY));
            ++om_uses;
            mma_commit(bar(B_PAIR_EMPTY + p));
            ++units;
            pos += 2;
          }
          mma_commit(bar(B_D1_FULL + (ti & 1)));
          T3_TRACE(ti, 4);
        }
        if (i >= 0) {   // MMA2 of tile i on its image units, as they land in the ring
          const int ti = i;
          if (!dead && !mbar_wait(bar(B_G_READY + (ti & 1)), static_cast<uint32_t>(ti >> 1) & 1u)) dead = true;
          const bool zero_h = ti == 0 || drain_tile(ti - 1, nt, a.drain_every, cid);
          tc_fence_after();
          for (int u = 0; u < U; ++u) {
            const int s = static_cast<int>(pos % NSTAGE);
            const uint32_t f2 = s ? f2b++ : f2a++;
            if (!dead && !mbar_wait(bar(B_UNIT_FULL + s), f2 & 1u)) dead = true;
            tc_fence_after();
            if (!dead) {
              const uint64_t dA2 = sdesc(su32(sStage) + s * STAGE_BYTES, BLOCK16, 1024);   // MN-major: features x rows
              const uint32_t gtb = GT_NB == 2 ? static_cast<uint32_t>(ti & 1) * static_cast<uint32_t>(L) * 128u : 0u;
              const uint64_t dB2 = sdesc(su32(sGt) + gtb, 16, 1024);                      // K-major: L x rows
#pragma unroll
              for (int ks = 0; ks < T3_ROWS / 16; ++ks)
#pragma unroll
                for (int h = 0; h < GS; ++h)
                  mma_bf16(tH + static_cast<uint32_t>(u * L), dA2 + ((static_cast<uint32_t>(ks) * 2048u) >> 4),
                           dB2 + ((static_cast<uint32_t>(h) * static_cast<uint32_t>(L) * 128u +
                                   static_cast<uint32_t>(ks >> 2) * GT_CHUNK +
                                   static_cast<uint32_t>(ks & 3) * 32u) >> 4),
                           id2, (zero_h && ks == 0 && h == 0) ? 0u : 1u);
            }
            mma_commit(bar(B_SLOT_EMPTY + s));
            ++pos;
          }
          mma_commit(bar(B_MMA2_DONE + (ti & 1)));
          T3_TRACE(ti, 5);
        }
      }
      // every MMA of this CTA has completed before TMEM is released
      mma_commit(bar(B_FINAL));
      mbar_wait(bar(B_FINAL), 0);
    }
  } else {
    // ------------------------------------------------------------ reduce group (warps 0-3)
    const int q = warp;   // TMEM lane quadrant
    F2Acc sg_acc;
    bool drained = false;
    const int r0 = static_cast<int>(rank) * RPC;
    // H (TMEM) -> the cluster's FP32 partial in global memory, as boxes of 128 features x 32
    // columns staged in the exchange buffer (free once every peer has read this CTA's rows of
    // the tile, so callers wait B_XCH_FREE first) in the 128-byte swizzled layout of the
    // tensor map: the TMA engine stores the first drain and adds the later ones in L2. Two
    // staging halves alternate; thread 0 issues the copies and waits for their reads.
    // (L a multiple of 32; otherwise drain_red below)
    auto drain_tma = [&]() {
      uint8_t* stg = reinterpret_cast<uint8_t*>(sX);
      const int row = q * 32 + lane;
      const int64_t hrow0 = static_cast<int64_t>(cid) * CS * w + f0;
      const int nbox = U * (L / 32);
      for (int bx = 0; bx < nbox; ++bx) {
        const int mt = bx / (L / 32), c0 = (bx % (L / 32)) * 32;
        uint8_t* half = stg + (bx & 1) * (128 * 128);
        if (bx >= 2) {
          if (tid == 0) bulk_wait_read<1>();   // the copy of box bx - 2 has read this half
          named_bar(1, RG_THREADS);
        }
        uint32_t r[32];
#pragma unroll
        for (int j = 0; j < 4; ++j)
          tmem_ld8_issue(tH + static_cast<uint32_t>(mt * L + c0 + 8 * j) + (static_cast<uint32_t>(q * 32) << 16),
                         r + 8 * j);
        tmem_wait_ld();
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) {   // 16-byte chunk ch of this row, swizzled by row % 8
          float v[4];
#pragma unroll
          for (int e = 0; e < 4; ++e)   // H carries s^2, sums s
            v[e] = __uint_as_float(r[4 * ch + e]) * (c0 + 4 * ch + e == l ? inv_s : inv_s * inv_s);
          *reinterpret_cast<float4*>(half + row * 128 + ((ch ^ (row & 7)) << 4)) = make_float4(v[0], v[1], v[2], v[3]);
        }
        fence_async_cta();
        named_bar(1, RG_THREADS);
        if (tid == 0) {
          const int32_t y = static_cast<int32_t>(hrow0 + mt * 128);
          if (drained) tma_reduce_add_2d(&a.hmap, c0, y, su32(half));
          else tma_store_2d(&a.hmap, c0, y, su32(half));
          bulk_commit();
        }
      }
      // the exchange buffer is free again once the copies have read it; after the stores of a
      // launch's first drain, also wait until they are written: bulk copies are not ordered
      // with one another, and a later drain's add-reductions to the same rows must not land first
      if (tid == 0) {
        if (drained) bulk_wait_read<0>();
        else bulk_wait_all();
      }
      named_bar(1, RG_THREADS);
      drained = true;
      tc_fence_before();
    };
    // the same with plain stores, then reductions issued by the threads themselves
    auto drain_red = [&]() {
      for (int ch = 0; ch < U * L; ch += 16) {   // 16 columns of a unit: two loads, one wait
        const int mt = ch / L, c0 = ch - mt * L;
        uint32_t r[16];
#pragma unroll
        for (int j = 0; j < 2; ++j)
          tmem_ld8_issue(tH + static_cast<uint32_t>(mt * L + c0 + 8 * j) + (static_cast<uint32_t>(q * 32) << 16),
                         r + 8 * j);
        tmem_wait_ld();
        const int64_t feat = f0 + mt * 128 + q * 32 + lane;
        float* hrow = a.Hpart + (static_cast<int64_t>(cid) * (CS * static_cast<int64_t>(w)) + feat) * L + c0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float v[4];
#pragma unroll
          for (int e = 0; e < 4; ++e)   // H carries s^2, sums s
            v[e] = __uint_as_float(r[4 * j + e]) * (c0 + 4 * j + e == l ? inv_s : inv_s * inv_s);
          float* dst = hrow + 4 * j;
          if (drained) red_add_v4(dst, v[0], v[1], v[2], v[3]);
          else *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
        }
      }
      drained = true;
      tc_fence_before();
    };
    auto drain_h = [&]() {
      if (L % 32 == 0) drain_tma();
      else drain_red();
    };
    for (int i = 0; i < nt; ++i) {
      const int64_t tile = cid + static_cast<int64_t>(i) * ncl;
      const int sgi = find_seg3(a, tile);
      const int64_t row0 = (tile - a.seg[sgi].tile0) * T3_ROWS;
      const int64_t mseg = a.seg[sgi].m;
      // 1. own D1 partial -> exchange rows; tell every peer
      if (!dead && !mbar_wait(bar(B_D1_FULL + (i & 1)), static_cast<uint32_t>(i >> 1) & 1u)) dead = true;
      if (tid == 0) T3_TRACE(i, 6);
      if (i >= 1 && !dead && !mbar_wait_cluster(bar(B_XCH_FREE), static_cast<uint32_t>(i - 1) & 1u)) dead = true;
      tc_fence_after();
      {
        const int row = q * 32 + lane;
        const uint32_t d1 = tmem + static_cast<uint32_t>((i & 1) * L) + (static_cast<uint32_t>(q * 32) << 16);
        for (int c0 = 0; c0 < L; c0 += 32) {   // 32 columns: four loads issued before one wait
          uint32_t r[32];
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (c0 + 8 * j < L) tmem_ld8_issue(d1 + static_cast<uint32_t>(c0 + 8 * j), r + 8 * j);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (c0 + 8 * j < L) {
              float4* dst = reinterpret_cast<float4*>(sX + row * xld + c0 + 8 * j);
              dst[0] = make_float4(__uint_as_float(r[8 * j]), __uint_as_float(r[8 * j + 1]),
                                   __uint_as_float(r[8 * j + 2]), __uint_as_float(r[8 * j + 3]));
              dst[1] = make_float4(__uint_as_float(r[8 * j + 4]), __uint_as_float(r[8 * j + 5]),
                                   __uint_as_float(r[8 * j + 6]), __uint_as_float(r[8 * j + 7]));
            }
          }
        }
      }
      tc_fence_before();
      mbar_arrive(bar(B_D1_EMPTY + (i & 1)));
      named_bar(1, RG_THREADS);
      if (warp == 0 && lane < CS) {
        fence_acq_rel_cluster();
        mbar_arrive_cluster(mapa(bar(B_XCH_READY), static_cast<uint32_t>(lane)));
      }
      // 2. reduce the own rows over the cluster, round, Gram and sums, publish
      if (tid == 0) T3_TRACE(i, 10);
      if (!dead && !mbar_wait_cluster(bar(B_XCH_READY), static_cast<uint32_t>(i) & 1u)) dead = true;
      if (tid == 0) T3_TRACE(i, 7);
      for (int it = tid; it < RPC * (L / 4); it += RG_THREADS) {
        const int rr = it / (L / 4), c4 = it % (L / 4);
        const uint32_t laddr = su32(sX + (r0 + rr) * xld + c4 * 4);
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int half = 0; half < 2; ++half) {   // eight peer loads in flight, then add in peer order
          float4 v[8];
#pragma unroll
          for (int q8 = 0; q8 < 8; ++q8)
            if (half * 8 + q8 < CS) v[q8] = ld_dsmem_v4f(mapa(laddr, static_cast<uint32_t>(half * 8 + q8)));
#pragma unroll
          for (int q8 = 0; q8 < 8; ++q8)
            if (half * 8 + q8 < CS) {
              acc.x += v[q8].x; acc.y += v[q8].y; acc.z += v[q8].z; acc.w += v[q8].w;
            }
        }
        const float ac[4] = {acc.x, acc.y, acc.z, acc.w};
        float y[4];
        bool fin = true;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float hi = round1<FMT>(ac[e]);
          fin = fin && isfinite(hi);
          y[e] = GS == 2 ? hi + round1<FMT>(ac[e] - hi) : hi;
        }
        if (!fin) atomicOr(a.flags, 1);
        const int cl = l - c4 * 4;
#pragma unroll
        for (int e = 0; e < 4; ++e)   // ones column -> column sums
          if (e == cl) y[e] = (row0 + r0 + rr < mseg) ? 1.f : 0.f;
        float* dst = sY + rr * L + c4 * 4;
        dst[0] = y[0]; dst[1] = y[1]; dst[2] = y[2]; dst[3] = y[3];
      }
      named_bar(1, RG_THREADS);
      if (tid == 0) T3_TRACE(i, 12);
      if (warp == 0 && lane < CS) {   // every peer may overwrite its exchange rows now
        fence_acq_rel_cluster();
        mbar_arrive_cluster(mapa(bar(B_XCH_FREE), static_cast<uint32_t>(lane)));
      }
      // 3. the MMA2 and Gram products of tile i - GT_NB are done with the G^T buffer tile i
      //    takes in this CTA: say so to every peer; then drain H if due, after the previous
      //    tile's MMA2
      if (i >= 1) {
        if (i >= GT_NB) {
          const int t = i - GT_NB;
          const uint32_t ph = static_cast<uint32_t>(t >> 1) & 1u;
          if (!dead && !mbar_wait(bar(B_MMA2_DONE + (t & 1)), ph)) dead = true;
          if (!dead && !mbar_wait(bar(B_GT_FREE + (t & 1)), ph)) dead = true;
        }
        if (warp == 0 && lane < CS) {
          fence_acq_rel_cluster();
          mbar_arrive_cluster(mapa(bar(B_PEER_FREE), static_cast<uint32_t>(lane)));
        }
        if (drain_tile(i - 1, nt, a.drain_every, cid)) {
          if (GT_NB == 2 && !dead &&
              !mbar_wait(bar(B_MMA2_DONE + ((i - 1) & 1)), static_cast<uint32_t>((i - 1) >> 1) & 1u))
            dead = true;
          if (!dead && !mbar_wait_cluster(bar(B_XCH_FREE), static_cast<uint32_t>(i) & 1u)) dead = true;
          tc_fence_after();
          drain_h();
        }
      }
      // 4. pack the own rows of G' (FP16: hi and lo) ...
      uint4* pub = sPub + (i & 1) * (GS * L * G8);
      for (int it = tid; it < L * G8; it += RG_THREADS) {
        const int lc = it / G8, g = it % G8;
        const float* yv = sY + (g * 8) * L + lc;
        float hi[8], lo[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          hi[r] = round1<FMT>(yv[r * L]);
          lo[r] = yv[r * L] - hi[r];
        }
        pub[lc * G8 + g] = make_uint4(pack2<FMT>(hi[0], hi[1]), pack2<FMT>(hi[2], hi[3]), pack2<FMT>(hi[4], hi[5]),
                                      pack2<FMT>(hi[6], hi[7]));
        if constexpr (GS == 2) {
          pub[(L + lc) * G8 + g] = make_uint4(pack2<FMT>(lo[0], lo[1]), pack2<FMT>(lo[2], lo[3]),
                                              pack2<FMT>(lo[4], lo[5]), pack2<FMT>(lo[6], lo[7]));
        }
      }
      if (tid == 0) T3_TRACE(i, 13);
      // sums of G and the G output of the own rows (sY stays valid until this group writes the
      // next tile's rows)
      if (tid < L) {
        for (int rr = 0; rr < RPC; ++rr) sg_acc.add(sY[rr * L + tid]);
      }
      if (a.seg[sgi].gout != nullptr) {
        for (int it = tid; it < RPC * l; it += RG_THREADS) {
          const int rr = it / l, c = it % l;
          const int64_t grow = row0 + r0 + rr;
          if (grow < mseg) a.seg[sgi].gout[grow * l + c] = sY[rr * L + c] * inv_s;
        }
      }
      named_bar(1, RG_THREADS);
      if (tid == 0) T3_TRACE(i, 14);
      // ... and store them into every peer's G^T operand once every peer's buffer is free
      if (i >= 1 && !dead && !mbar_wait_cluster(bar(B_PEER_FREE), static_cast<uint32_t>(i - 1) & 1u)) dead = true;
      if (tid == 0) T3_TRACE(i, 11);
      {
        const int nitems = GS * L * G8;
        for (int t = tid; t < nitems * CS; t += RG_THREADS) {
          const int it = t % nitems, pp = t / nitems;
          const int h = it / (L * G8), rem = it - h * (L * G8), lc = rem / G8, gl = rem % G8;
          const int g = static_cast<int>(rank) * G8 + gl;
          const int hr = h + (GT_NB == 2 ? (i & 1) : 0);   // row block of tile i's G^T buffer
          const uint32_t off = static_cast<uint32_t>(g >> 3) * GT_CHUNK + static_cast<uint32_t>((hr * L + lc) >> 3) * 1024u +
                               sw128(static_cast<uint32_t>(lc & 7), static_cast<uint32_t>(g & 7) * 16u);
          st_dsmem_v4u(mapa(su32(sGt + off), static_cast<uint32_t>(pp)), pub[it]);
        }
      }
      fence_proxy_async_all();
      named_bar(1, RG_THREADS);
      if (warp == 0 && lane < CS) {
        fence_acq_rel_cluster();
        mbar_arrive_cluster(mapa(bar(B_GT_FULL), static_cast<uint32_t>(lane)));
      }
      if (tid == 0) T3_TRACE(i, 8);
      if (!dead && !mbar_wait_cluster(bar(B_GT_FULL), static_cast<uint32_t>(i) & 1u)) dead = true;
      fence_async_cta();
      mbar_arrive(bar(B_G_READY + (i & 1)));
      if (tid == 0) T3_TRACE(i, 9);
    }
    // the last tile's MMA2, then its drain
    if (nt > 0) {
      if (!dead && !mbar_wait(bar(B_MMA2_DONE + ((nt - 1) & 1)), static_cast<uint32_t>((nt - 1) >> 1) & 1u)) dead = true;
      if (!dead && !mbar_wait_cluster(bar(B_XCH_FREE), static_cast<uint32_t>(nt - 1) & 1u)) dead = true;
      tc_fence_after();
      drain_h();
      if (tid == 0) bulk_wait_all();   // the last stores and adds are complete before the CTA leaves
    } else {
      for (int64_t e = tid; e < static_cast<int64_t>(w) * L; e += RG_THREADS)
        a.Hpart[(static_cast<int64_t>(cid) * CS * w + f0) * L + e] = 0.f;
    }
    const int64_t cta = static_cast<int64_t>(cid) * CS + rank;
    if (tid < L) a.sG_part[cta * L + tid] = sg_acc.value() * inv_s;
  }
  if (dead) atomicOr(a.flags, 2);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM3_COLS));
  }
  cluster_sync();   // no CTA leaves while a peer may still read its shared memory
}

}  // namespace

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against libcuda)
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  // looked up once per process (a function-local static is initialised by one thread)
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
    return static_cast<PFN_cuTensorMapEncodeTiled_v12000>(nullptr);
  }();
  return fn;
}

namespace {

thread_local char g_tc3_reason[192] = "";

}  // namespace

const char* tc3_config_reason() { return g_tc3_reason; }

bool tc3_config(int64_t n, int L, int fmt, TcConfig* cfg) {
  const auto kern = fmt == FMT_F16 ? sketch_tc3_kernel<FMT_F16> : sketch_tc3_kernel<FMT_BF16>;
  const int gs = fmt == FMT_F16 ? 2 : 1;
  snprintf(g_tc3_reason, sizeof(g_tc3_reason), "no cluster size fits");
  if (!encode_fn()) {
    snprintf(g_tc3_reason, sizeof(g_tc3_reason), "cuTensorMapEncodeTiled is not available");
    return false;
  }
  if (L % 16 != 0 || L > 64) {
    snprintf(g_tc3_reason, sizeof(g_tc3_reason), "padded l = %d exceeds 64", L);
    return false;
  }
  for (int CS : {1, 2, 4, 8, 16}) {
    int64_t w = (n + CS - 1) / CS;
    w = ((w + 127) / 128) * 128;
    // TMEM: two D1 buffers and H (w / 128 tiles of L columns); the cluster's 128 CS reduce
    // converter threads take at most T3_GRAM_PER_THREAD entries of G'^T G' each
    if (w / 128 > T3_MAX_UNITS || 2 * L + (w / 128) * L > static_cast<int64_t>(TMEM3_COLS)) continue;
    if (static_cast<int64_t>(CS) * CV_WARPS * 32 * T3_GRAM_PER_THREAD < static_cast<int64_t>(L) * (L + 1) / 2) continue;
    const Tc3Layout lay = tc3_layout(L, static_cast<int>(w), CS, gs);
    if (lay.total > 227u * 1024u) continue;
    cfg->CS = CS;
    cfg->w = static_cast<int>(w);
    cfg->smem = lay.total;
    // the kernel's limit is per function, shared by every session: set it to the device's
    // maximum rather than to this configuration's need, which another session may exceed
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa0{};
    cudaFuncGetAttributes(&fa0, kern);
    optin -= static_cast<int>(fa0.sharedSizeBytes);   // the static shared memory counts against the limit
    if (optin < static_cast<int>(lay.total)) continue;
    cudaError_t e1 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(static_cast<unsigned>(CS), 1, 1);
    lc.blockDim = dim3(T3_NT, 1, 1);
    lc.dynamicSmemBytes = lay.total;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = static_cast<unsigned>(CS);
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, kern, &lc) != cudaSuccess || ncl < 1) {
      cudaGetLastError();
      continue;
    }
    cfg->nclusters = ncl;
    return true;
  }
  return false;
}

// One launch of the pipelined pass over the pending row blocks; false in *used when a block
// cannot be described by a tensor map (base not 16-byte aligned or ld not a multiple of 4),
// in which case nothing is launched and the caller takes the other kernel.
cudaError_t tc3_pass(const State& s, const TcWork& w, const TcPending& pend, cudaStream_t st, Prof* prof,
                     bool* used) {
  *used = false;
  if (pend.nseg == 0) {
    *used = true;
    return cudaSuccess;
  }
  static_assert(kTcPendingMax <= T3_MAX_SEGS, "segment capacity");
  Tc3Args args;
  std::memset(&args, 0, sizeof(args));
  const TcConfig& cfg = w.cfg3;
  int64_t tiles = 0;
  for (int i = 0; i < pend.nseg; ++i) {
    const uintptr_t addr = reinterpret_cast<uintptr_t>(pend.rows[i]);
    if ((addr & 15u) != 0 || (pend.ld[i] % 4) != 0) return cudaSuccess;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(s.n), static_cast<cuuint64_t>(pend.m[i])};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(pend.ld[i]) * 4};
    cuuint32_t box[2] = {64, T3_ROWS};
    cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode_fn()(&args.maps[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                                   const_cast<void*>(pend.rows[i]), dims, strides, box, estr,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaSuccess;
    args.seg[i].m = pend.m[i];
    args.seg[i].gout = pend.gout[i];
    args.seg[i].tile0 = tiles;
    tiles += (pend.m[i] + T3_ROWS - 1) / T3_ROWS;
  }
  if (s.L % 32 == 0) {
    // H partials: L FP32 columns x (clusters x CS x w) rows, boxes of 32 columns x 128 rows
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(s.L), static_cast<cuuint64_t>(cfg.nclusters) * cfg.CS * cfg.w};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(s.L) * 4};
    cuuint32_t box[2] = {32, 128};
    cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode_fn()(&args.hmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, w.Hpart, dims, strides, box, estr,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                   CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaSuccess;   // the caller takes the other kernel
  }
  args.nseg = pend.nseg;
  args.ntiles = tiles;
  args.n = s.n;
  args.l = s.l;
  args.L = s.L;
  args.w = cfg.w;
  args.CS = cfg.CS;
  args.drain_every = w.fmt == FMT_F16 ? 2 : 4;   // 32 MMAs per TMEM accumulation of H either way
  args.shift = s.shift;
  args.om16 = w.om16;
  args.img = w.img;
  args.img_halves = static_cast<int64_t>(cfg.nclusters) * cfg.CS * cfg.w * 256;
  args.scale = w.fmt == FMT_F16 ? w.scale : nullptr;
  args.Hpart = w.Hpart;
  args.gram_part = w.gram_part;
  args.sG_part = w.sG_part;
  args.flags = s.flags;
  args.trace = nullptr;
#ifdef SPCA_TC_TRACE
  static unsigned long long* dtrace = nullptr;
  if (!dtrace) cudaMalloc(&dtrace, sizeof(unsigned long long) * (128 + 256));
  cudaMemsetAsync(dtrace, 0, sizeof(unsigned long long) * (128 + 256), st);
  args.trace = dtrace;
#endif

  cudaLaunchConfig_t lc = {};
  const int64_t ncl = tiles < cfg.nclusters ? tiles : cfg.nclusters;
  lc.gridDim = dim3(static_cast<unsigned>(ncl * cfg.CS), 1, 1);
  lc.blockDim = dim3(T3_NT, 1, 1);
  lc.dynamicSmemBytes = cfg.smem;
  lc.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = static_cast<unsigned>(cfg.CS);
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  prof->begin(SPCA_K_TC_SKETCH, st);
  cudaError_t e = w.fmt == FMT_F16 ? cudaLaunchKernelEx(&lc, sketch_tc3_kernel<FMT_F16>, args)
                                   : cudaLaunchKernelEx(&lc, sketch_tc3_kernel<FMT_BF16>, args);
  prof->end(SPCA_K_TC_SKETCH, st);
  if (e != cudaSuccess) return e;
  *used = true;
#ifdef SPCA_TC_TRACE
  {
    unsigned long long h[128 + 256];
    cudaStreamSynchronize(st);
    cudaMemcpy(h, dtrace, sizeof(h), cudaMemcpyDeviceToHost);
    const unsigned long long t0 = h[0];
    static const char* names[15] = {"prodP1", "prodP2", "cvP1end", "cvP2end", "mma1", "mma2", "rgD1",
                                    "rgXchRdy", "rgPushed", "rgG", "rgXchSent", "rgPeerFree", "rgReduced",
                                    "rgPacked", "rgSums"};
    for (int t = 0; t < 8; ++t) {
      fprintf(stderr, "tc3 tile %d:", t);
      for (int p = 0; p < 15; ++p)
        if (h[t * 16 + p]) fprintf(stderr, " %s=%.1f", names[p], (double)(h[t * 16 + p] - t0) / 1000.0);
      fprintf(stderr, " us\n");
    }
    for (int sg = 0; sg < 10; ++sg)
      fprintf(stderr, "tc3 tile 3 stage %d: claim %.2f issued %.2f cvwait %.2f cvfull %.2f cvdone %.2f us\n", sg,
              h[128 + sg * 8 + 3] ? (double)(h[128 + sg * 8 + 3] - t0) / 1000.0 : -1.0,
              h[128 + sg * 8 + 0] ? (double)(h[128 + sg * 8 + 0] - t0) / 1000.0 : -1.0,
              h[128 + sg * 8 + 1] ? (double)(h[128 + sg * 8 + 1] - t0) / 1000.0 : -1.0,
              h[128 + sg * 8 + 2] ? (double)(h[128 + sg * 8 + 2] - t0) / 1000.0 : -1.0,
              h[128 + sg * 8 + 4] ? (double)(h[128 + sg * 8 + 4] - t0) / 1000.0 : -1.0);
  }
#endif
  e = launch_tc_finish(s, w, static_cast<int>(ncl), cfg.CS * static_cast<int64_t>(cfg.w),
                       static_cast<int>(ncl) * cfg.CS, st, prof);
  return e;
}

}  // namespace spca

// The streaming pass on the tensor cores (tcgen05, BF16 operands, FP32 accumulation in
// TMEM), fused so that every element of A is read from HBM exactly once (Alg. 4 steps
// 5-7, Eq. 11).
//
// Decomposition. A thread-block cluster of CS CTAs splits the n features: CTA `rank`
// owns features [rank*w, rank*w + w). Clusters walk over 128-row tiles of the rows
// handed to the launch. Per tile, in every CTA of the cluster:
//   1. eight loader warps read the 128 x w slice of A (FP32) one 64-feature block at a
//      time, subtract the shift c, round to BF16 and store it in shared memory in the
//      128-byte-swizzled K-major layout (a2). Two register batches are in flight, and
//      the next tile's slice is prefetched into L2 while this tile computes;
//   2. MMA1 (issued by a ninth warp as soon as each feature block is stored):
//      D1[128 x L] = A_hat_slice (K-major) x Omega_slice (K-major chunks of 64 features
//      streamed through a ring by 1-D bulk copies of a pre-swizzled BF16 Omega) (a3);
//   3. the CS partials of D1 are reduced over distributed shared memory in a fixed
//      order: CTA `rank` sums rows [rank*128/CS, (rank+1)*128/CS) and rounds them to
//      BF16 (the G_hat' that every later step uses); column `l` of G' is set to 1 for
//      every valid row, so that MMA2 also produces the column sums of A_hat (a5);
//   4. each CTA accumulates G'^T G' and 1^T G' of its rows and publishes them packed;
//      every CTA pulls all 128 rows into its own G^T operand tile;
//   5. MMA2: H[w x L] += A_hat_slice^T (the same shared-memory tile, read MN-major) x G'
//      (K-major), H resident in TMEM for the whole launch (a4).
// At the end each CTA writes its H slice (with the column sums in column l) and its Gram
// partial; a finish kernel adds the per-cluster partials to the FP64 session state in a
// fixed order.
//
// All mbarrier waits are bounded; a thread that gives up sets flags[0] bit 2, skips
// later waits and keeps taking part in the cluster barriers (every CTA of a cluster
// runs the same number of them), so no wait can hang the GPU.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cstdio>
#include <cstring>

#include "philox.cuh"
#include "spca_internal.cuh"
#include "tc_ptx.cuh"

namespace spca {

namespace {

constexpr int TC_ROWS = 128;       // rows per tile = M of MMA1
constexpr int TC_LOADERS = 352;    // warps 0-10 load and convert A
constexpr int TC_NT = 384;         // + warp 11: MMA issue, Omega ring, L2 prefetch
constexpr int MMA_WARP = 11;
constexpr int LOAD_ITEMS = (TC_ROWS * 8 + TC_LOADERS - 1) / TC_LOADERS;   // (row, chunk) items per loader
constexpr int OM_STAGES = 4;       // Omega chunk ring depth
constexpr int MAX_CHUNKS = 10;     // w / 64 <= 10
constexpr int GRAM_PER_THREAD = 6;    // lower-triangle Gram entries per thread (L <= 64)
constexpr uint32_t TMEM_COLS = 512;

}  // namespace

// ------------------------------------------------------------------ layout

struct TcLayout {
  int L, w, CS, RPC;
  uint32_t a_bytes, ring_bytes, gt_bytes, shift_bytes, y_bytes, yt_bytes, bar_bytes, total;
};

// gs: 1, or 2 when G enters MMA2 as two 16-bit terms (hi + lo)
__host__ __device__ inline TcLayout tc_layout(int L, int w, int CS, int gs) {
  TcLayout t;
  t.L = L; t.w = w; t.CS = CS; t.RPC = TC_ROWS / CS;
  t.a_bytes = static_cast<uint32_t>(w) * 256u;                         // 128 rows x w, 16-bit
  const uint32_t ring = OM_STAGES * static_cast<uint32_t>(L) * 128u;   // Omega chunks
  const uint32_t xch = TC_ROWS * static_cast<uint32_t>(L + 4) * 4u;   // D1 partial exchange (FP32, padded rows)
  t.gt_bytes = 256u * static_cast<uint32_t>(L * gs);                   // G^T: gs x L x 128 rows, 16-bit
  // the Omega ring (MMA1), the exchange rows (cluster reduction) and the G^T operand (MMA2)
  // are live in turn within a tile, so they share one region
  uint32_t r = ring > xch ? ring : xch;
  r = r > t.gt_bytes ? r : t.gt_bytes;
  t.ring_bytes = (r + 1023u) & ~1023u;
  t.shift_bytes = ((static_cast<uint32_t>(w) * 4u) + 15u) & ~15u;
  t.y_bytes = ((static_cast<uint32_t>(t.RPC) * L * 4u) + 15u) & ~15u;  // own reduced rows, FP32
  t.yt_bytes = static_cast<uint32_t>(L * gs) * (t.RPC / 8) * 16u;       // same, packed 16-bit [gs][L][RPC/8]
  t.bar_bytes = 8u * (2 * OM_STAGES + MAX_CHUNKS + 2);
  t.total = 1024u + t.a_bytes + t.ring_bytes + t.shift_bytes + t.y_bytes + t.yt_bytes + t.bar_bytes;
  return t;
}

struct TcSeg {
  const float* rows;
  int64_t m;
  int64_t ld;
  float* gout;
  int64_t tile0;   // index of this segment's first tile in the launch
};

constexpr int kTcMaxSegs = 48;

struct TcArgs {
  TcSeg seg[kTcMaxSegs];
  int nseg;
  int64_t ntiles;
  int64_t n;
  int l, L, w, CS;
  int vec_ok;
  int drain_every;             // tiles accumulated in TMEM before H is added to Hpart
  const float* shift;
  const uint16_t* om16;        // Omega (operand format bits), chunk g at g * L * 64 elements, pre-swizzled
  const float* scale;          // operand scale s (power of two); NULL = 1
  float* Hpart;                // nclusters x (CS w) x L (column l: column sums)
  double* gram_part;           // nctas x L x L
  double* sG_part;             // nctas x L
  int* flags;
  unsigned long long* trace;   // phase timestamps of one CTA (builds with SPCA_TC_TRACE only)
};

#ifdef SPCA_TC_TRACE
#define TC_TRACE(slot)                                                                  \
  do {                                                                                  \
    if (tid == 0 && rank == 0 && cid == 0 && iter < 8 && a.trace) {                     \
      unsigned long long t_;                                                            \
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_));                            \
      a.trace[iter * 16 + (slot)] = t_;                                                 \
    }                                                                                   \
  } while (0)
#else
#define TC_TRACE(slot) \
  do {                 \
  } while (0)
#endif

namespace {

__device__ __forceinline__ int find_seg(const TcArgs& a, int64_t tile) {
  int sgi = 0;
  while (sgi + 1 < a.nseg && a.seg[sgi + 1].tile0 <= tile) ++sgi;
  return sgi;
}

// one CTA of 12 warps per SM (<= 170 registers per thread)
template <int FMT>
__global__ void __launch_bounds__(TC_NT, 1) sketch_tc_kernel(const __grid_constant__ TcArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int L = a.L, w = a.w, CS = a.CS, l = a.l;
  constexpr int GS = FMT == FMT_F16 ? 2 : 1;   // FP16 form: G = G_hi + G_lo in MMA2
  const TcLayout lay = tc_layout(L, w, CS, GS);
  const int RPC = lay.RPC, G8 = RPC / 8;
  uint8_t* sA = base;
  uint8_t* sRing = sA + lay.a_bytes;
  float* sX = reinterpret_cast<float*>(sRing);              // exchange buffer (aliases the ring)
  uint8_t* sGt = sRing;                                     // G^T operand (aliases the ring too)
  float* sShift = reinterpret_cast<float*>(sRing + lay.ring_bytes);
  float* sY = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(sShift) + lay.shift_bytes);
  uint4* sYt = reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(sY) + lay.y_bytes);
  uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(sYt) + lay.yt_bytes);
  uint64_t* full = bars;                       // [OM_STAGES]
  uint64_t* empty = bars + OM_STAGES;          // [OM_STAGES]
  uint64_t* ablk = bars + 2 * OM_STAGES;       // [MAX_CHUNKS]: feature block stored
  uint64_t* mma1_done = ablk + MAX_CHUNKS;
  uint64_t* mma2_done = mma1_done + 1;
  __shared__ uint32_t tmem_sh;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const uint32_t rank = cluster_rank();
  const uint32_t cid = cluster_id();
  const uint32_t ncl = cluster_count();
  const int64_t n = a.n;
  const int64_t f0 = static_cast<int64_t>(rank) * w;
  const int nchunk = w / 64;
  const int xld = L + 4;                    // exchange row stride (floats)
  const uint32_t chunk_bytes = static_cast<uint32_t>(L) * 128u;
  const int64_t g0 = f0 / 64;               // first Omega chunk of this slice
  // bytes of one row segment of this slice that exist (features < n), for L2 prefetch
  int64_t seg_feats = n - f0 < w ? n - f0 : w;
  const uint32_t pf_bytes = seg_feats > 0 ? static_cast<uint32_t>((seg_feats * 4) & ~int64_t(15)) : 0u;

  for (int i = tid; i < w; i += TC_NT) sShift[i] = (f0 + i < n) ? a.shift[f0 + i] : 0.f;
  if (tid == 0) {
    for (int s = 0; s < OM_STAGES; ++s) {
      mbar_init(su32(&full[s]), 1);
      mbar_init(su32(&empty[s]), 1);
    }
    for (int c = 0; c < MAX_CHUNKS; ++c) mbar_init(su32(&ablk[c]), TC_LOADERS);
    mbar_init(su32(mma1_done), 1);
    mbar_init(su32(mma2_done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_sh)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_sh;
  const uint32_t tD1 = tmem;
  const uint32_t tH = tmem + static_cast<uint32_t>(L);

  F2Acc gram_acc[GRAM_PER_THREAD];
  F2Acc sg_acc;

  // MMA-thread state
  uint32_t fills[OM_STAGES] = {0, 0, 0, 0};
  uint32_t cons[OM_STAGES] = {0, 0, 0, 0};
  uint32_t iter = 0;
  bool dead = false;
  bool any_tile = false;
  bool zero_h = true;     // the next MMA2 starts a fresh TMEM accumulation of H
  bool drained = false;   // this CTA's Hpart slice holds a partial already
  const uint32_t id1 = idesc_fmt<FMT>(TC_ROWS, L, 0, 0);
  const uint32_t id2 = idesc_fmt<FMT>(TC_ROWS, L, 1, 0);
  // operands carry s A_hat and s G; every partial is brought back by exact powers of two
  const float op_scale = a.scale ? *a.scale : 1.f;
  const float inv_s = 1.f / op_scale;
  const uint64_t dA1 = sdesc(su32(sA), 16, 1024);        // MMA1 A: K-major rows x features
  const uint64_t dA2 = sdesc(su32(sA), 16384, 1024);     // MMA2 A: MN-major features x rows
  const uint64_t dB2 = sdesc(su32(sGt), 16, 1024);       // MMA2 B: K-major L x rows
  const uint64_t dR = sdesc(su32(sRing), 16, 1024);      // MMA1 B: ring stage 0

  // prefetch the first tile of this cluster into L2
  if (warp == MMA_WARP && cid < a.ntiles && a.vec_ok && pf_bytes) {
    const TcSeg& sg = a.seg[find_seg(a, cid)];
    const int64_t row0 = (static_cast<int64_t>(cid) - sg.tile0) * TC_ROWS;
    for (int rr = lane; rr < TC_ROWS; rr += 32) {
      if (row0 + rr < sg.m) prefetch_l2(sg.rows + (row0 + rr) * sg.ld + f0, pf_bytes);
    }
  }

  for (int64_t tile = cid; tile < a.ntiles; tile += ncl, ++iter) {
    const TcSeg sg = a.seg[find_seg(a, tile)];
    const int64_t row0 = (tile - sg.tile0) * TC_ROWS;
    TC_TRACE(0);

    if (warp < MMA_WARP) {
      // ------------------------------------------------ loaders: A slice -> BF16 swizzled tile
      // a 64-feature block is 128 rows x 8 chunks of 8 features; loader thread t takes the
      // (row, chunk) items t, t + TC_LOADERS, t + 2 TC_LOADERS (< 1024)
      auto gload = [&](int fb, float4 (&v)[LOAD_ITEMS][2]) {
#pragma unroll
        for (int u = 0; u < LOAD_ITEMS; ++u) {
          const int item = tid + TC_LOADERS * u;
          const int rr = item >> 3, cc = item & 7;
          const int64_t fbase = f0 + fb * 64 + cc * 8;
          const int64_t grow = row0 + rr;
          v[u][0] = make_float4(0.f, 0.f, 0.f, 0.f);
          v[u][1] = v[u][0];
          if (item < TC_ROWS * 8 && grow < sg.m) {
            const float* src = sg.rows + grow * sg.ld + fbase;
            if (a.vec_ok && fbase + 7 < n) {
              v[u][0] = __ldg(reinterpret_cast<const float4*>(src));
              v[u][1] = __ldg(reinterpret_cast<const float4*>(src + 4));
            } else {
              float t[8];
#pragma unroll
              for (int q = 0; q < 8; ++q) t[q] = (fbase + q < n) ? __ldg(src + q) : 0.f;
              v[u][0] = make_float4(t[0], t[1], t[2], t[3]);
              v[u][1] = make_float4(t[4], t[5], t[6], t[7]);
            }
          }
        }
      };
      auto convert = [&](int fb, const float4 (&v)[LOAD_ITEMS][2]) {
#pragma unroll
        for (int u = 0; u < LOAD_ITEMS; ++u) {
          const int item = tid + TC_LOADERS * u;
          if (item >= TC_ROWS * 8) continue;
          const int rr = item >> 3, cc = item & 7;
          const float* shv = sShift + fb * 64 + cc * 8;
          const int64_t fbase = f0 + fb * 64 + cc * 8;
          const bool valid = row0 + rr < sg.m;
          const float x[8] = {v[u][0].x, v[u][0].y, v[u][0].z, v[u][0].w, v[u][1].x, v[u][1].y, v[u][1].z, v[u][1].w};
          uint32_t pk[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float lo = valid && (fbase + 2 * q < n) ? (x[2 * q] - shv[2 * q]) * op_scale : 0.f;
            const float hi = valid && (fbase + 2 * q + 1 < n) ? (x[2 * q + 1] - shv[2 * q + 1]) * op_scale : 0.f;
            pk[q] = pack2<FMT>(lo, hi);
          }
          const uint32_t off = static_cast<uint32_t>(fb) * 16384u + static_cast<uint32_t>(rr >> 3) * 1024u +
                               sw128(static_cast<uint32_t>(rr & 7), static_cast<uint32_t>(cc) * 16u);
          *reinterpret_cast<uint4*>(sA + off) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
        fence_async_cta();
        mbar_arrive(su32(&ablk[fb]));
      };
      // two register batches in flight: block fb+1 loads while block fb converts
      float4 bufA[LOAD_ITEMS][2], bufB[LOAD_ITEMS][2];
      gload(0, bufA);
      for (int fb = 0; fb < nchunk; fb += 2) {
        if (fb + 1 < nchunk) gload(fb + 1, bufB);
        convert(fb, bufA);
        if (fb + 1 < nchunk) {
          if (fb + 2 < nchunk) gload(fb + 2, bufA);
          convert(fb + 1, bufB);
        }
      }
    } else {
      // ------------------------------------------------ MMA warp: MMA1 as feature blocks arrive
      if (lane == 0) {
        auto issue = [&](int c) {
          const int s = c % OM_STAGES;
          if (fills[s] > 0 && !dead) {
            if (!mbar_wait(su32(&empty[s]), (fills[s] - 1) & 1u)) dead = true;
          }
          mbar_expect_tx(su32(&full[s]), chunk_bytes);
          bulk_g2s(su32(sRing + s * chunk_bytes), a.om16 + (g0 + c) * static_cast<int64_t>(L) * 64, chunk_bytes,
                   su32(&full[s]));
          ++fills[s];
        };
        fence_async_cta();   // the ring held the previous tile's exchange rows (generic writes)
        for (int c = 0; c < nchunk && c < OM_STAGES; ++c) issue(c);
        tc_fence_after();
        for (int c = 0; c < nchunk; ++c) {
          const int s = c % OM_STAGES;
          if (!dead && !mbar_wait(su32(&ablk[c]), iter & 1u)) dead = true;
          if (!dead && !mbar_wait(su32(&full[s]), cons[s] & 1u)) dead = true;
          ++cons[s];
          if (!dead) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t ad = dA1 + ((static_cast<uint32_t>(c) * 16384u + kk * 32u) >> 4);
              const uint64_t bd = dR + ((static_cast<uint32_t>(s) * chunk_bytes + kk * 32u) >> 4);
              mma_bf16(tD1, ad, bd, id1, (c | kk) != 0 ? 1u : 0u);
            }
          }
          mma_commit(su32(&empty[s]));
          // refill the stage consumed one chunk earlier: its MMAs precede the ones just queued
          if (c >= 1 && c - 1 + OM_STAGES < nchunk) issue(c - 1 + OM_STAGES);
        }
        mma_commit(su32(mma1_done));
      }
      __syncwarp();
      // prefetch the next tile of this cluster into L2 while this one computes
      const int64_t nt = tile + ncl;
      if (nt < a.ntiles && a.vec_ok && pf_bytes) {
        const TcSeg& sn = a.seg[find_seg(a, nt)];
        const int64_t r0n = (nt - sn.tile0) * TC_ROWS;
        for (int rr = lane; rr < TC_ROWS; rr += 32) {
          if (r0n + rr < sn.m) prefetch_l2(sn.rows + (r0n + rr) * sn.ld + f0, pf_bytes);
        }
      }
    }
    TC_TRACE(1);

    // ------------------------------------------------ D1 -> exchange buffer (rows x L, FP32)
    if (!dead && !mbar_wait(su32(mma1_done), iter & 1u)) dead = true;
    __syncwarp();
    tc_fence_after();
    TC_TRACE(2);
    if (warp < 8) {
      const int q = warp & 3, half = warp >> 2;
      const int row = q * 32 + lane;
      const int cbeg = half * (L / 2), cend = cbeg + L / 2;
      for (int c = cbeg; c < cend; c += 8) {
        float v[8];
        tmem_ld8(tD1 + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(c), v);
        float4* dst = reinterpret_cast<float4*>(sX + row * xld + c);
        dst[0] = make_float4(v[0], v[1], v[2], v[3]);
        dst[1] = make_float4(v[4], v[5], v[6], v[7]);
      }
    }
    tc_fence_before();
    TC_TRACE(3);
    cluster_sync();   // #1: all partials of the tile are in place
    TC_TRACE(4);

    // ------------------------------------------------ reduce own rows over the cluster
    const int r0 = static_cast<int>(rank) * RPC;
    for (int it = tid; it < RPC * (L / 4); it += TC_NT) {
      const int rr = it / (L / 4), c4 = it % (L / 4);
      const uint32_t laddr = su32(sX + (r0 + rr) * xld + c4 * 4);
      float4 v[16];   // every peer load in flight before the first add, then sum in peer order
#pragma unroll
      for (int p = 0; p < 16; ++p) {
        if (p < CS) v[p] = ld_dsmem_v4f(mapa(laddr, static_cast<uint32_t>(p)));
      }
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int p = 0; p < 16; ++p) {
        if (p < CS) {
          acc.x += v[p].x; acc.y += v[p].y; acc.z += v[p].z; acc.w += v[p].w;
        }
      }
      // G' = the operand value(s) of G: one rounding, or hi + lo (hi + lo is exact in FP32)
      const float ac[4] = {acc.x, acc.y, acc.z, acc.w};
      float y[4];
      bool fin = true;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float hi = round1<FMT>(ac[i]);
        fin = fin && isfinite(hi);   // after the rounding: an FP16 operand can overflow where FP32 did not
        y[i] = GS == 2 ? hi + round1<FMT>(ac[i] - hi) : hi;
      }
      if (!fin) atomicOr(a.flags, 1);
      const int cl = l - c4 * 4;
#pragma unroll
      for (int e = 0; e < 4; ++e)   // ones column -> column sums
        if (e == cl) y[e] = (row0 + r0 + rr < sg.m) ? 1.f : 0.f;
      float* dst = sY + rr * L + c4 * 4;
      dst[0] = y[0]; dst[1] = y[1]; dst[2] = y[2]; dst[3] = y[3];
    }
    __syncthreads();
    TC_TRACE(5);
    // publish the own rows packed as G^T chunks: 8 rows of one column in 16 bytes (hi terms,
    // then lo terms when split)
    for (int it = tid; it < L * G8; it += TC_NT) {
      const int lc = it / G8, g = it % G8;
      const float* y = sY + (g * 8) * L + lc;
      float hi[8], lo[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        hi[r] = round1<FMT>(y[r * L]);
        lo[r] = y[r * L] - hi[r];
      }
      sYt[lc * G8 + g] = make_uint4(pack2<FMT>(hi[0], hi[1]), pack2<FMT>(hi[2], hi[3]), pack2<FMT>(hi[4], hi[5]),
                                    pack2<FMT>(hi[6], hi[7]));
      if constexpr (GS == 2) {
        sYt[(L + lc) * G8 + g] = make_uint4(pack2<FMT>(lo[0], lo[1]), pack2<FMT>(lo[2], lo[3]),
                                            pack2<FMT>(lo[4], lo[5]), pack2<FMT>(lo[6], lo[7]));
      }
    }
    // Gram, sums of G and the optional G output from the own rows
    {
      const int LT = L * (L + 1) / 2;   // lower triangle, row by row
#pragma unroll
      for (int i = 0; i < GRAM_PER_THREAD; ++i) {
        const int e = tid + TC_NT * i;
        if (e < LT) {
          int c1 = static_cast<int>((sqrtf(8.f * static_cast<float>(e) + 1.f) - 1.f) * 0.5f);
          while (c1 * (c1 + 1) / 2 > e) --c1;
          while ((c1 + 1) * (c1 + 2) / 2 <= e) ++c1;
          const int c2 = e - c1 * (c1 + 1) / 2;
          float acc = 0.f;   // G' rows in FP32 (one 16-bit value, or hi + lo)
          for (int rr = 0; rr < RPC; ++rr) acc = fmaf(sY[rr * L + c1], sY[rr * L + c2], acc);
          gram_acc[i].add(acc);
        }
      }
      if (tid < L) {
        for (int rr = 0; rr < RPC; ++rr) sg_acc.add(sY[rr * L + tid]);
      }
      if (sg.gout != nullptr) {
        for (int it = tid; it < RPC * l; it += TC_NT) {
          const int rr = it / l, c = it % l;
          const int64_t grow = row0 + r0 + rr;
          if (grow < sg.m) sg.gout[grow * l + c] = sY[rr * L + c] * inv_s;
        }
      }
    }
    TC_TRACE(6);
    cluster_sync();   // #2: every CTA's rows are published
    TC_TRACE(7);
    // pull all 128 rows of G' into the own G^T operand tile (K-major, L x 128 rows; the lo
    // terms follow the hi terms at +256 L bytes)
    for (int it = tid; it < GS * L * (TC_ROWS / 8); it += TC_NT) {
      const int h = it / (L * (TC_ROWS / 8));
      const int rem = it - h * (L * (TC_ROWS / 8));
      const int lc = rem / (TC_ROWS / 8), g = rem % (TC_ROWS / 8);
      const int p = g / G8, gl = g % G8;
      const uint4 pk = ld_dsmem_v4u(mapa(su32(sYt + (h * L + lc) * G8 + gl), static_cast<uint32_t>(p)));
      const uint32_t off = static_cast<uint32_t>(h) * (256u * static_cast<uint32_t>(L)) +
                           static_cast<uint32_t>(g >> 3) * (static_cast<uint32_t>(L) * 128u) +
                           static_cast<uint32_t>(lc >> 3) * 1024u +
                           sw128(static_cast<uint32_t>(lc & 7), static_cast<uint32_t>(g & 7) * 16u);
      *reinterpret_cast<uint4*>(sGt + off) = pk;
    }
    fence_async_cta();
    __syncthreads();
    TC_TRACE(8);

    // ------------------------------------------------ MMA2: H += A_hat_slice^T G'
    if (warp == MMA_WARP && lane == 0) {
      tc_fence_after();
      if (!dead) {
        for (int mt = 0; mt < w / 128; ++mt) {
#pragma unroll
          for (int ks = 0; ks < TC_ROWS / 16; ++ks) {
            const uint64_t ad = dA2 + ((static_cast<uint32_t>(2 * mt) * 16384u + static_cast<uint32_t>(ks) * 2048u) >> 4);
#pragma unroll
            for (int h = 0; h < GS; ++h) {
              const uint64_t bd = dB2 + ((static_cast<uint32_t>(h) * 256u * static_cast<uint32_t>(L) +
                                          static_cast<uint32_t>(ks >> 2) * chunk_bytes +
                                          static_cast<uint32_t>(ks & 3) * 32u) >> 4);
              mma_bf16(tH + static_cast<uint32_t>(mt * L), ad, bd, id2, (zero_h && ks == 0 && h == 0) ? 0u : 1u);
            }
          }
        }
      }
      mma_commit(su32(mma2_done));
    }
    any_tile = true;
    if (!dead && !mbar_wait(su32(mma2_done), iter & 1u)) dead = true;
    __syncwarp();
    tc_fence_after();
    TC_TRACE(9);

    // ------------------------------------------------ drain: Hpart += H (TMEM), every few tiles
    // A TMEM accumulation rounds toward zero at every MMA; short accumulations keep H's
    // error at the level of FP32 rounding. Hpart (L2-resident, FP32) is owned by this CTA
    // for its features, so plain read-add-write in tile order is deterministic.
    zero_h = ((iter + 1) % static_cast<uint32_t>(a.drain_every) == 0) || (tile + ncl >= a.ntiles);
    if (zero_h) {
      const int q = warp & 3, part = warp >> 2;   // three warps per TMEM lane quadrant
      const int cpr = L / 8;                      // 8-column chunks per 128-feature tile
      for (int ch = part; ch < (w / 128) * cpr; ch += TC_NT / 128) {
        const int mt = ch / cpr, c = (ch - mt * cpr) * 8;
        float v[8];
        tmem_ld8(tH + static_cast<uint32_t>(mt * L + c) + (static_cast<uint32_t>(q * 32) << 16), v);
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] *= (c + i == l ? inv_s : inv_s * inv_s);   // H carries s^2, sums s
        const int64_t feat = f0 + mt * 128 + q * 32 + lane;
        float4* dst = reinterpret_cast<float4*>(a.Hpart + (static_cast<int64_t>(cid) * (CS * static_cast<int64_t>(w)) + feat) * L + c);
        if (drained) {   // added in L2; this thread is the only writer of these entries
          red_add_v4(reinterpret_cast<float*>(dst), v[0], v[1], v[2], v[3]);
          red_add_v4(reinterpret_cast<float*>(dst + 1), v[4], v[5], v[6], v[7]);
        } else {
          dst[0] = make_float4(v[0], v[1], v[2], v[3]);
          dst[1] = make_float4(v[4], v[5], v[6], v[7]);
        }
      }
      drained = true;
      tc_fence_before();   // the loads above precede the next MMA2 that overwrites H
    }
  }

  // ---------------------------------------------------------------- epilogue
  if (dead) {
    atomicOr(a.flags, 2);
  }
  __syncthreads();
  const int64_t npad = static_cast<int64_t>(CS) * w;
  const int64_t cta = static_cast<int64_t>(cid) * CS + rank;
  if (!any_tile) {   // a cluster without tiles contributes a zero H slice
    for (int64_t i = tid; i < static_cast<int64_t>(w) * L; i += TC_NT)
      a.Hpart[(static_cast<int64_t>(cid) * npad + f0) * L + i] = 0.f;
  }
  {
    const int LL = L * L, LT = L * (L + 1) / 2;
#pragma unroll
    for (int i = 0; i < GRAM_PER_THREAD; ++i) {
      const int e = tid + TC_NT * i;
      if (e < LT) {
        int c1 = static_cast<int>((sqrtf(8.f * static_cast<float>(e) + 1.f) - 1.f) * 0.5f);
        while (c1 * (c1 + 1) / 2 > e) --c1;
        while ((c1 + 1) * (c1 + 2) / 2 <= e) ++c1;
        const int c2 = e - c1 * (c1 + 1) / 2;
        const double g = gram_acc[i].value() * (static_cast<double>(inv_s) * inv_s);
        a.gram_part[cta * LL + c1 * L + c2] = g;
        a.gram_part[cta * LL + c2 * L + c1] = g;
      }
    }
    if (tid < L) a.sG_part[cta * L + tid] = sg_acc.value() * inv_s;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
  // keep the cluster together until every peer is done with our shared memory
  cluster_sync();
}

// H (FP64) += sum over clusters of the FP32 partial slices; column l of the partials
// holds the column sums of A_hat.
__global__ void tc_finish_kernel(const float* __restrict__ Hpart, int ncl, int64_t n, int64_t npad, int l, int L,
                                 double* __restrict__ H, double* __restrict__ colsum) {
  const int64_t total = n * L;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    // the cluster partials summed as an FP32 pair (two-sum): FP64 adds issue slowly here
    float hi = 0.f, lo = 0.f;
    for (int c = 0; c < ncl; ++c) {
      const float x = Hpart[static_cast<int64_t>(c) * npad * L + idx];
      const float s = hi + x;
      const float bb = s - hi;
      lo += (hi - (s - bb)) + (x - bb);
      hi = s;
    }
    const double acc = static_cast<double>(hi) + static_cast<double>(lo);
    const int col = static_cast<int>(idx % L);
    if (col < l) H[idx] += acc;
    else if (col == l) colsum[idx / L] += acc;
  }
}

// Omega as BF16 (RNE of the FP32 value) in the pre-swizzled chunk layout of the kernel:
// chunk g (features 64g..64g+63) is L rows (Omega columns) of 128 bytes, 8-row atoms.
template <int FMT>
__global__ void omega_op_kernel(uint64_t seed, int64_t n, int64_t npad, int l, int L, uint16_t* __restrict__ out) {
  const int qn = L / 4;
  const int64_t total = npad * qn;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t j = idx / qn;
    const int q = static_cast<int>(idx % qn);
    double z[4] = {0.0, 0.0, 0.0, 0.0};
    if (j < n) {
      const U32x4 wv = omega_words_at(seed, j, static_cast<uint32_t>(q), 0u);
      box_muller(wv.x, wv.y, z[0], z[1]);
      box_muller(wv.z, wv.w, z[2], z[3]);
    }
    const int64_t g = j / 64;
    const uint32_t fbyte = static_cast<uint32_t>(j % 64) * 2u;
    uint8_t* chunk = reinterpret_cast<uint8_t*>(out) + g * static_cast<int64_t>(L) * 128;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int c = 4 * q + t;
      const float v = (j < n && c < l) ? static_cast<float>(z[t]) : 0.f;
      const uint32_t off = static_cast<uint32_t>(c >> 3) * 1024u + sw128(static_cast<uint32_t>(c & 7), fbyte);
      *reinterpret_cast<uint16_t*>(chunk + off) = static_cast<uint16_t>(pack2<FMT>(v, 0.f) & 0xFFFFu);
    }
  }
}

// Omega given as a matrix (n x L FP64, ld L; the power scheme's orth(H)), in the operand
// format and the chunk layout above; columns >= l and features >= n are 0.
template <int FMT>
__global__ void omega_from_q_op_kernel(const double* __restrict__ Q, int64_t n, int64_t npad, int l, int L,
                                       uint16_t* __restrict__ out) {
  const int64_t total = npad * L;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t j = idx / L;
    const int c = static_cast<int>(idx % L);
    const float v = (j < n && c < l) ? static_cast<float>(Q[j * L + c]) : 0.f;
    uint8_t* chunk = reinterpret_cast<uint8_t*>(out) + (j / 64) * static_cast<int64_t>(L) * 128;
    const uint32_t off = static_cast<uint32_t>(c >> 3) * 1024u +
                         sw128(static_cast<uint32_t>(c & 7), static_cast<uint32_t>(j % 64) * 2u);
    *reinterpret_cast<uint16_t*>(chunk + off) = static_cast<uint16_t>(pack2<FMT>(v, 0.f) & 0xFFFFu);
  }
}

// The operand scale of the FP16 form: the largest shifted row norm of the first rows
// bounds every entry of s G (|g_rc| <= ||a_r - c|| ||omega_c||, ||omega_c|| ~ sqrt(n) for
// the Gaussian Omega, 1 for an orthonormal one), so
// s = 2^floor(log2(2^14 / (1.25 ||omega_c|| max_r ||a_r - c||))) keeps s G below 2^14 with
// four-fold headroom under the FP16 maximum.
__device__ __forceinline__ float stored_value(const float* p, int64_t i, float) { return p[i]; }
__device__ __forceinline__ float stored_value(const __nv_bfloat16* p, int64_t i, float) { return __bfloat162float(p[i]); }
__device__ __forceinline__ float stored_value(const __nv_fp8_e4m3* p, int64_t i, float scale) {
  return static_cast<float>(p[i]) * scale;
}

template <typename T>
__global__ void row_norm_max_kernel(const T* __restrict__ rows, float dscale, int64_t m, int64_t n, int64_t ld,
                                    const float* __restrict__ shift, unsigned int* __restrict__ out_bits) {
  __shared__ float red[256];   // only a power of two is taken from the result: FP32 suffices
  for (int64_t r = blockIdx.x; r < m; r += gridDim.x) {
    float s = 0.f;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
      const float d = stored_value(rows, r * ld + j, dscale) - shift[j];
      s = fmaf(d, d, s);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
      if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
      __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(out_bits, __float_as_uint(sqrtf(red[0])));
    __syncthreads();
  }
}

__global__ void op_scale_kernel(const unsigned int* __restrict__ bits, double omega_norm, float* __restrict__ scale) {
  const float mx = __uint_as_float(*bits);
  float s = 1.f;
  if (mx > 0.f && isfinite(mx)) {
    const double e = floor(log2(16384.0 / (1.25 * omega_norm * static_cast<double>(mx))));
    s = static_cast<float>(exp2(fmin(fmax(e, -100.0), 100.0)));
  }
  *scale = s;
}

int grid_for(int64_t total, int threads) {
  int64_t b = (total + threads - 1) / threads;
  if (b > 152 * 16) b = 152 * 16;
  return static_cast<int>(b < 1 ? 1 : b);
}

thread_local char g_tc_reason[192] = "";

}  // namespace

const char* tc_config_reason() { return g_tc_reason; }

bool tc_config(int64_t n, int L, int fmt, TcConfig* cfg) {
  const auto kern = fmt == FMT_F16 ? sketch_tc_kernel<FMT_F16> : sketch_tc_kernel<FMT_BF16>;
  snprintf(g_tc_reason, sizeof(g_tc_reason), "no cluster size fits");
  if (L % 16 != 0 || L * (L + 1) / 2 > GRAM_PER_THREAD * TC_NT) {
    snprintf(g_tc_reason, sizeof(g_tc_reason), "padded l = %d exceeds the Gram registers", L);
    return false;
  }
  for (int CS : {4, 8, 16}) {
    const int64_t w = ((n + CS - 1) / CS + 127) / 128 * 128;
    if (w > 64 * MAX_CHUNKS) continue;
    if ((1 + w / 128) * L > static_cast<int64_t>(TMEM_COLS)) continue;
    const TcLayout lay = tc_layout(L, static_cast<int>(w), CS, fmt == FMT_F16 ? 2 : 1);
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
      snprintf(g_tc_reason, sizeof(g_tc_reason), "cluster %d: attributes: %s / %s", CS, cudaGetErrorString(e1),
               cudaGetErrorString(e2));
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t lc = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.gridDim = dim3(CS, 1, 1);
    lc.blockDim = dim3(TC_NT, 1, 1);
    lc.dynamicSmemBytes = lay.total;
    lc.attrs = at;
    lc.numAttrs = 1;
    int ncl = 0;
    const cudaError_t e3 = cudaOccupancyMaxActiveClusters(&ncl, kern, &lc);
    if (e3 != cudaSuccess || ncl < 1) {
      cudaFuncAttributes fa{};
      cudaFuncGetAttributes(&fa, kern);
      int nb = -1;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, TC_NT, lay.total);
      snprintf(g_tc_reason, sizeof(g_tc_reason),
               "cluster %d, w %lld, smem %u: occupancy %s, %d clusters (regs %d, max threads %d, static smem %zu, "
               "blocks/SM %d)",
               CS, (long long)w, lay.total, cudaGetErrorString(e3), ncl, fa.numRegs, fa.maxThreadsPerBlock,
               fa.sharedSizeBytes, nb);
      cudaGetLastError();
      continue;
    }
    cfg->nclusters = ncl;
    return true;
  }
  return false;
}

cudaError_t launch_omega_op(int fmt, uint64_t seed, int64_t n, int64_t npad, int l, int L, uint16_t* out,
                            cudaStream_t st, Prof* prof) {
  if (prof) prof->begin(SPCA_K_OMEGA, st);
  if (fmt == FMT_F16)
    omega_op_kernel<FMT_F16><<<grid_for(npad * (L / 4), 256), 256, 0, st>>>(seed, n, npad, l, L, out);
  else
    omega_op_kernel<FMT_BF16><<<grid_for(npad * (L / 4), 256), 256, 0, st>>>(seed, n, npad, l, L, out);
  if (prof) prof->end(SPCA_K_OMEGA, st);
  return cudaGetLastError();
}

cudaError_t launch_omega_from_q_op(int fmt, const double* Q, int64_t n, int64_t npad, int l, int L, uint16_t* out,
                                   cudaStream_t st) {
  if (fmt == FMT_F16)
    omega_from_q_op_kernel<FMT_F16><<<grid_for(npad * L, 256), 256, 0, st>>>(Q, n, npad, l, L, out);
  else
    omega_from_q_op_kernel<FMT_BF16><<<grid_for(npad * L, 256), 256, 0, st>>>(Q, n, npad, l, L, out);
  return cudaGetLastError();
}

cudaError_t launch_op_scale(const void* rows, int dtype, float dscale, int64_t m, int64_t n, int64_t ld,
                            const float* shift, unsigned int* bits, float* scale, double omega_norm, cudaStream_t st,
                            Prof* prof) {
  if (prof) prof->begin(SPCA_K_SHIFT, st);
  cudaError_t e = cudaMemsetAsync(bits, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  const int blocks = static_cast<int>(m < 152 * 8 ? m : 152 * 8) < 1 ? 1 : static_cast<int>(m < 152 * 8 ? m : 152 * 8);
  if (dtype == SPCA_BF16)
    row_norm_max_kernel<<<blocks, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(rows), 1.f, m, n, ld, shift, bits);
  else if (dtype == SPCA_F8E4M3)
    row_norm_max_kernel<<<blocks, 256, 0, st>>>(static_cast<const __nv_fp8_e4m3*>(rows), dscale, m, n, ld, shift,
                                                 bits);
  else if (dtype == SPCA_F32)
    row_norm_max_kernel<<<blocks, 256, 0, st>>>(static_cast<const float*>(rows), 1.f, m, n, ld, shift, bits);
  else
    return cudaErrorInvalidValue;
  op_scale_kernel<<<1, 1, 0, st>>>(bits, omega_norm, scale);
  if (prof) {
    prof->launches[SPCA_K_SHIFT] += 1;
    prof->end(SPCA_K_SHIFT, st);
  }
  return cudaGetLastError();
}

cudaError_t tc_pass(const State& s, const TcWork& w, const TcPending& pend, cudaStream_t st, Prof* prof) {
  if (pend.nseg == 0) return cudaSuccess;
  TcArgs args;
  std::memset(&args, 0, sizeof(args));
  int64_t tiles = 0;
  bool vec_ok = true;
  for (int i = 0; i < pend.nseg; ++i) {
    args.seg[i].rows = static_cast<const float*>(pend.rows[i]);
    args.seg[i].m = pend.m[i];
    args.seg[i].ld = pend.ld[i];
    args.seg[i].gout = pend.gout[i];
    args.seg[i].tile0 = tiles;
    tiles += (pend.m[i] + TC_ROWS - 1) / TC_ROWS;
    vec_ok = vec_ok && (reinterpret_cast<uintptr_t>(pend.rows[i]) % 16 == 0) && (pend.ld[i] % 4 == 0);
  }
  args.nseg = pend.nseg;
  args.ntiles = tiles;
  args.n = s.n;
  args.l = s.l;
  args.L = s.L;
  args.w = w.cfg.w;
  args.CS = w.cfg.CS;
  args.vec_ok = vec_ok ? 1 : 0;
  args.drain_every = w.fmt == FMT_F16 ? 2 : 4;   // 32 MMAs per TMEM accumulation of H either way
  args.shift = s.shift;
  args.om16 = w.om16;
  args.scale = w.fmt == FMT_F16 ? w.scale : nullptr;
  args.Hpart = w.Hpart;
  args.gram_part = w.gram_part;
  args.sG_part = w.sG_part;
  args.flags = s.flags;
  args.trace = nullptr;
#ifdef SPCA_TC_TRACE
  static unsigned long long* dtrace = nullptr;
  if (!dtrace) cudaMalloc(&dtrace, sizeof(unsigned long long) * 8 * 16);
  cudaMemsetAsync(dtrace, 0, sizeof(unsigned long long) * 8 * 16, st);
  args.trace = dtrace;
#endif
  cudaLaunchConfig_t lc = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = w.cfg.CS;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.gridDim = dim3(w.cfg.nclusters * w.cfg.CS, 1, 1);
  lc.blockDim = dim3(TC_NT, 1, 1);
  lc.dynamicSmemBytes = w.cfg.smem;
  lc.stream = st;
  lc.attrs = at;
  lc.numAttrs = 1;
  prof->begin(SPCA_K_TC_SKETCH, st);
  cudaError_t e = w.fmt == FMT_F16 ? cudaLaunchKernelEx(&lc, sketch_tc_kernel<FMT_F16>, args)
                                   : cudaLaunchKernelEx(&lc, sketch_tc_kernel<FMT_BF16>, args);
  prof->end(SPCA_K_TC_SKETCH, st);
  if (e != cudaSuccess) return e;
#ifdef SPCA_TC_TRACE
  {
    unsigned long long h[8 * 16];
    cudaStreamSynchronize(st);
    cudaMemcpy(h, dtrace, sizeof(h), cudaMemcpyDeviceToHost);
    for (int t = 0; t < 8; ++t) {
      if (!h[t * 16]) break;
      fprintf(stderr, "tc trace tile %d:", t);
      for (int p = 1; p < 10; ++p) fprintf(stderr, " %lld", (long long)(h[t * 16 + p] - h[t * 16 + p - 1]));
      if (t + 1 < 8 && h[(t + 1) * 16]) fprintf(stderr, " | next %lld", (long long)(h[(t + 1) * 16] - h[t * 16 + 9]));
      fprintf(stderr, " ns\n");
    }
  }
#endif
  return launch_tc_finish(s, w, w.cfg.nclusters, static_cast<int64_t>(w.cfg.CS) * w.cfg.w,
                          w.cfg.nclusters * w.cfg.CS, st, prof);
}

cudaError_t launch_tc_finish(const State& s, const TcWork& w, int ncl, int64_t npad, int nctas, cudaStream_t st,
                             Prof* prof) {
  prof->begin(SPCA_K_H_FINISH, st);
  tc_finish_kernel<<<grid_for(s.n * s.L, 256), 256, 0, st>>>(w.Hpart, ncl, s.n, npad, s.l, s.L, s.H, s.colsum);
  prof->end(SPCA_K_H_FINISH, st);
  prof->begin(SPCA_K_GRAM_ACCUM, st);
  cudaError_t e = launch_gram_accum(w.gram_part, w.sG_part, nctas, s.L, s.gram, s.sG, st);
  prof->end(SPCA_K_GRAM_ACCUM, st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace spca

// The streaming pass on the tensor cores (tcgen05, BF16 operands, FP32 accumulation in
// TMEM), fused so that every element of A is read from HBM exactly once (Alg. 4 steps
// 5-7, Eq. 11).
//
// Decomposition. A thread-block cluster of CS CTAs splits the n features: CTA `rank`
// owns features [rank*w, rank*w + w). Clusters walk over 128-row tiles of the rows
// handed to the launch. For one tile, every CTA of the cluster
//   1. loads its 128 x w slice of A (FP32), subtracts the shift c, rounds to BF16 and
//      writes it to shared memory in the 128-byte-swizzled K-major layout (a2);
//   2. MMA1: D1[128 x L] = A_hat_slice (K-major) x Omega_slice (K-major chunks of 64
//      features streamed by 1-D bulk copies from a pre-swizzled BF16 copy of Omega):
//      the partial sketch of its features (a3);
//   3. reduces the CS partials of D1 over distributed shared memory in a fixed order:
//      CTA `rank` sums rows [rank*128/CS, (rank+1)*128/CS), rounds them to BF16 (the
//      G_hat' that every later step uses) and writes them into G^T tiles of all CTAs;
//   4. accumulates the Gram matrix G'^T G' and 1^T G' of its rows (a5);
//   5. MMA2: H[w x L] += A_hat_slice^T (the same shared-memory tile read MN-major) x G'
//      (K-major), H resident in TMEM for the whole launch (a4).
// Column sums of the BF16 A_hat values are kept by the loading threads (a5). At the
// end each CTA writes its H slice, sums and Gram partial; a finish kernel adds the
// per-cluster partials to the FP64 session state in a fixed order.
//
// All mbarrier waits are bounded; a CTA that gives up sets flags[0] bit 2 and keeps
// taking part in the cluster barriers (every CTA runs the same number of them).
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "philox.cuh"
#include "spca_internal.cuh"

namespace spca {

namespace {

constexpr int TC_ROWS = 128;      // rows per tile = M of MMA1
constexpr int TC_NT = 256;        // threads per CTA
constexpr int OM_STAGES = 4;      // Omega chunk ring depth
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t WAIT_LIMIT = 1u << 20;   // tries per wait; a thread that gives up skips later waits

// ------------------------------------------------------------------ PTX wrappers

__device__ __forceinline__ uint32_t su32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of (row, colbyte) in a 1024-byte aligned region of 8-row x 128-byte atoms
__host__ __device__ __forceinline__ uint32_t sw128(uint32_t row, uint32_t colbyte) {
  const uint32_t o = row * 128u + colbyte;
  return o ^ (((o >> 7) & 7u) << 4);
}

// tcgen05 shared-memory matrix descriptor, 128-byte swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  d |= static_cast<uint64_t>(2) << 61;
  return d;
}

// instruction descriptor: kind::f16, BF16 x BF16 -> FP32
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int a_mn, int b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(a_mn) << 15) |
         (static_cast<uint32_t>(b_mn) << 16) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity) {
  for (uint32_t it = 0; it < WAIT_LIMIT; ++it)
    if (mbar_try(a, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_cta() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_async_cluster() { asm volatile("fence.proxy.async.shared::cluster;" ::: "memory"); }
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_id() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t mapa(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ float4 ld_dsmem_v4(uint32_t a) {
  float4 v;
  asm volatile("ld.shared::cluster.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a)
               : "memory");
  return v;
}
__device__ __forceinline__ void st_dsmem_v4(uint32_t a, uint4 v) {
  asm volatile("st.shared::cluster.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&p);
}
__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

}  // namespace

// ------------------------------------------------------------------ layout

struct TcLayout {
  int L, w, CS, RPC;
  uint32_t a_bytes, ring_bytes, gt_bytes, shift_bytes, y_bytes, bar_bytes, total;
};

__host__ __device__ inline TcLayout tc_layout(int L, int w, int CS) {
  TcLayout t;
  t.L = L; t.w = w; t.CS = CS; t.RPC = TC_ROWS / CS;
  t.a_bytes = static_cast<uint32_t>(w) * 256u;                         // 128 rows x w BF16
  const uint32_t ring = OM_STAGES * static_cast<uint32_t>(L) * 128u;   // Omega chunks
  const uint32_t xch = TC_ROWS * static_cast<uint32_t>(L + 4) * 4u;   // D1 partial exchange (FP32, padded rows)
  t.ring_bytes = ((ring > xch ? ring : xch) + 1023u) & ~1023u;
  t.gt_bytes = 256u * static_cast<uint32_t>(L);                        // G^T: L x 128 rows BF16
  t.shift_bytes = ((static_cast<uint32_t>(w) * 4u) + 15u) & ~15u;
  t.y_bytes = ((static_cast<uint32_t>(t.RPC) * L * 4u) + 15u) & ~15u;
  t.bar_bytes = 8u * (2 * OM_STAGES + 2);
  t.total = 1024u + t.a_bytes + t.ring_bytes + t.gt_bytes + t.shift_bytes + t.y_bytes + t.bar_bytes;
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
  const float* shift;
  const __nv_bfloat16* om16;   // chunk g at om16 + g * L * 64 (pre-swizzled)
  float* Hpart;                // nclusters x (CS w) x L
  double* cs_part;             // nclusters x (CS w)
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

__global__ void __launch_bounds__(TC_NT, 1) sketch_tc_kernel(const __grid_constant__ TcArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int L = a.L, w = a.w, CS = a.CS;
  const TcLayout lay = tc_layout(L, w, CS);
  const int RPC = lay.RPC;
  uint8_t* sA = base;
  uint8_t* sRing = sA + lay.a_bytes;
  float* sX = reinterpret_cast<float*>(sRing);              // exchange buffer (aliases the ring)
  uint8_t* sGt = sRing + lay.ring_bytes;
  float* sShift = reinterpret_cast<float*>(sGt + lay.gt_bytes);
  float* sY = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(sShift) + lay.shift_bytes);
  uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(sY) + lay.y_bytes);
  uint64_t* full = bars;                    // [OM_STAGES]
  uint64_t* empty = bars + OM_STAGES;       // [OM_STAGES]
  uint64_t* mma1_done = bars + 2 * OM_STAGES;
  uint64_t* mma2_done = mma1_done + 1;
  __shared__ uint32_t tmem_sh;
  __shared__ int dead_sh;

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

  for (int i = tid; i < w; i += TC_NT) sShift[i] = (f0 + i < n) ? a.shift[f0 + i] : 0.f;
  if (tid == 0) {
    for (int s = 0; s < OM_STAGES; ++s) {
      mbar_init(su32(&full[s]), 1);
      mbar_init(su32(&empty[s]), 1);
    }
    mbar_init(su32(mma1_done), 1);
    mbar_init(su32(mma2_done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    dead_sh = 0;
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

  // loader mapping: CPR chunks of 8 features per row; RP row phases
  const int CPR = w / 8;
  const int RP = TC_NT / CPR;
  const bool loader = tid < RP * CPR;
  const int cc = loader ? tid % CPR : 0;
  const int rp = loader ? tid / CPR : 0;
  double cs_acc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) cs_acc[i] = 0.0;
  // Gram entries owned by this thread: e = tid + TC_NT * i, i < 16 (L <= 64)
  double gram_acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) gram_acc[i] = 0.0;
  double sg_acc = 0.0;

  // thread-0 ring bookkeeping
  uint32_t fills[OM_STAGES] = {0, 0, 0, 0};
  uint32_t cons[OM_STAGES] = {0, 0, 0, 0};
  uint32_t iter = 0;
  bool dead = false;
  bool any_tile = false;
  const uint32_t id1 = idesc_bf16(TC_ROWS, L, 0, 0);
  const uint32_t id2 = idesc_bf16(TC_ROWS, L, 1, 0);

  for (int64_t tile = cid; tile < a.ntiles; tile += ncl, ++iter) {
    // locate the segment of this tile
    int sgi = 0;
    while (sgi + 1 < a.nseg && a.seg[sgi + 1].tile0 <= tile) ++sgi;
    const TcSeg sg = a.seg[sgi];
    const int64_t row0 = (tile - sg.tile0) * TC_ROWS;

    TC_TRACE(0);
    // (a) Omega prefetch for the first stages
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
    if (tid == 0) {
      // the ring held the previous tile's exchange rows (generic proxy writes)
      fence_async_cta();
      for (int c = 0; c < nchunk && c < OM_STAGES; ++c) issue(c);
    }

    // (b) load, shift, round to BF16, store swizzled; column sums of the stored values
    if (loader) {
      const int64_t fbase = f0 + cc * 8;
      const float* shv = sShift + cc * 8;
      const int fb = (cc * 8) / 64;
      const uint32_t colbyte = static_cast<uint32_t>((cc * 8) % 64) * 2u;
      float csl[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) csl[i] = 0.f;
      for (int r = rp; r < TC_ROWS; r += RP * 4) {
        float4 v[4][2];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int rr = r + u * RP;
          const int64_t grow = row0 + rr;
          v[u][0] = make_float4(0.f, 0.f, 0.f, 0.f);
          v[u][1] = v[u][0];
          if (rr < TC_ROWS && grow < sg.m) {
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
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int rr = r + u * RP;
          if (rr >= TC_ROWS) continue;
          const int64_t grow = row0 + rr;
          const bool valid = grow < sg.m;
          float x[8] = {v[u][0].x, v[u][0].y, v[u][0].z, v[u][0].w, v[u][1].x, v[u][1].y, v[u][1].z, v[u][1].w};
          uint32_t pk[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float lo = valid && (fbase + 2 * q < n) ? x[2 * q] - shv[2 * q] : 0.f;
            float hi = valid && (fbase + 2 * q + 1 < n) ? x[2 * q + 1] - shv[2 * q + 1] : 0.f;
            pk[q] = pack_bf16(lo, hi);
            csl[2 * q] += __uint_as_float(pk[q] << 16);
            csl[2 * q + 1] += __uint_as_float(pk[q] & 0xFFFF0000u);
          }
          const uint32_t off = static_cast<uint32_t>(fb) * 16384u + static_cast<uint32_t>(rr >> 3) * 1024u +
                               sw128(static_cast<uint32_t>(rr & 7), colbyte);
          *reinterpret_cast<uint4*>(sA + off) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) cs_acc[i] += static_cast<double>(csl[i]);
    }
    fence_async_cta();
    __syncthreads();

    TC_TRACE(1);
    // (c) MMA1 over the feature chunks, Omega streamed through the ring
    if (tid == 0) {
      tc_fence_after();
      for (int c = 0; c < nchunk; ++c) {
        const int s = c % OM_STAGES;
        if (!dead && !mbar_wait(su32(&full[s]), cons[s] & 1u)) dead = true;
        ++cons[s];
        if (!dead) {
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint32_t aaddr = su32(sA) + static_cast<uint32_t>(c) * 16384u + kk * 32u;
            const uint32_t baddr = su32(sRing + s * chunk_bytes) + kk * 32u;
            mma_bf16(tD1, sdesc(aaddr, 16, 1024), sdesc(baddr, 16, 1024), id1, (c | kk) != 0 ? 1u : 0u);
          }
        }
        mma_commit(su32(&empty[s]));
        // refill the stage consumed one chunk earlier: its MMAs precede the ones just
        // queued, so waiting for them keeps the tensor pipe busy
        if (c >= 1 && c - 1 + OM_STAGES < nchunk) issue(c - 1 + OM_STAGES);
      }
      mma_commit(su32(mma1_done));
    }
    // (d) D1 -> exchange buffer (rows x L, FP32)
    TC_TRACE(2);
    if (!dead && !mbar_wait(su32(mma1_done), iter & 1u)) dead = true;
    TC_TRACE(3);
    tc_fence_after();
    {
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
    TC_TRACE(4);
    cluster_sync();   // #1: all partials of the tile are in place
    TC_TRACE(5);

    // (e) reduce own rows over the cluster (fixed peer order), round to BF16
    const int r0 = static_cast<int>(rank) * RPC;
    for (int it = tid; it < RPC * (L / 4); it += TC_NT) {
      const int rr = it / (L / 4), c4 = it % (L / 4);
      const uint32_t laddr = su32(sX + (r0 + rr) * xld + c4 * 4);
      // issue every peer load before the first add (one round trip), then sum in peer order
      float4 v[16];
#pragma unroll
      for (int p = 0; p < 16; ++p) {
        if (p < CS) v[p] = ld_dsmem_v4(mapa(laddr, static_cast<uint32_t>(p)));
      }
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int p = 0; p < 16; ++p) {
        if (p < CS) {
          acc.x += v[p].x; acc.y += v[p].y; acc.z += v[p].z; acc.w += v[p].w;
        }
      }
      float* y = sY + rr * L + c4 * 4;
      y[0] = bf16_round(acc.x); y[1] = bf16_round(acc.y); y[2] = bf16_round(acc.z); y[3] = bf16_round(acc.w);
      if (!(isfinite(acc.x) && isfinite(acc.y) && isfinite(acc.z) && isfinite(acc.w))) atomicOr(a.flags, 1);
    }
    __syncthreads();
    TC_TRACE(6);
    // (f) pack 8 rows of one G^T row into 16 bytes and store them into every CTA's G^T
    for (int it = tid; it < L * (RPC / 8); it += TC_NT) {
      const int lc = it % L, g8 = it / L;
      const int rr0 = g8 * 8;
      uint4 pk;
      pk.x = pack_bf16(sY[(rr0 + 0) * L + lc], sY[(rr0 + 1) * L + lc]);
      pk.y = pack_bf16(sY[(rr0 + 2) * L + lc], sY[(rr0 + 3) * L + lc]);
      pk.z = pack_bf16(sY[(rr0 + 4) * L + lc], sY[(rr0 + 5) * L + lc]);
      pk.w = pack_bf16(sY[(rr0 + 6) * L + lc], sY[(rr0 + 7) * L + lc]);
      const int r = r0 + rr0;
      const uint32_t off = static_cast<uint32_t>(r >> 6) * (static_cast<uint32_t>(L) * 128u) +
                           static_cast<uint32_t>(lc >> 3) * 1024u +
                           sw128(static_cast<uint32_t>(lc & 7), static_cast<uint32_t>(r & 63) * 2u);
      const uint32_t laddr = su32(sGt + off);
      for (int p = 0; p < CS; ++p) st_dsmem_v4(mapa(laddr, static_cast<uint32_t>(p)), pk);
    }
    fence_async_cluster();
    // (g) Gram, sums of G and the optional G output from the local rows
    {
      const int LL = L * L;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int e = tid + TC_NT * i;
        if (e < LL) {
          const int c1 = e / L, c2 = e % L;
          float acc = 0.f;
          for (int rr = 0; rr < RPC; ++rr) acc = fmaf(sY[rr * L + c1], sY[rr * L + c2], acc);
          gram_acc[i] += static_cast<double>(acc);
        }
      }
      if (tid < L) {
        double acc = 0.0;
        for (int rr = 0; rr < RPC; ++rr) acc += static_cast<double>(sY[rr * L + tid]);
        sg_acc += acc;
      }
      if (sg.gout != nullptr) {
        for (int it = tid; it < RPC * a.l; it += TC_NT) {
          const int rr = it / a.l, c = it % a.l;
          const int64_t grow = row0 + r0 + rr;
          if (grow < sg.m) sg.gout[grow * a.l + c] = sY[rr * L + c];
        }
      }
    }
    TC_TRACE(7);
    cluster_sync();   // #2: every G^T tile is complete
    TC_TRACE(8);

    // (h) MMA2: H += A_hat_slice^T G'
    if (tid == 0) {
      tc_fence_after();
      if (!dead) {
        for (int mt = 0; mt < w / 128; ++mt) {
#pragma unroll
          for (int ks = 0; ks < TC_ROWS / 16; ++ks) {
            const uint32_t aaddr = su32(sA) + static_cast<uint32_t>(2 * mt) * 16384u + static_cast<uint32_t>(ks) * 2048u;
            const uint32_t baddr = su32(sGt) + static_cast<uint32_t>(ks >> 2) * (static_cast<uint32_t>(L) * 128u) +
                                   static_cast<uint32_t>(ks & 3) * 32u;
            const uint32_t acc = (any_tile || ks > 0) ? 1u : 0u;
            mma_bf16(tH + static_cast<uint32_t>(mt * L), sdesc(aaddr, 16384, 1024), sdesc(baddr, 16, 1024), id2, acc);
          }
        }
      }
      mma_commit(su32(mma2_done));
    }
    any_tile = true;
    if (!dead && !mbar_wait(su32(mma2_done), iter & 1u)) dead = true;
    TC_TRACE(9);
    tc_fence_after();
  }

  // ---------------------------------------------------------------- epilogue
  if (dead) {
    atomicOr(a.flags, 2);
    dead_sh = 1;
  }
  __syncthreads();
  const int64_t npad = static_cast<int64_t>(CS) * w;
  const int64_t cta = static_cast<int64_t>(cid) * CS + rank;
  // H slice: TMEM lanes = features of each 128-feature tile
  {
    const int q = warp & 3, half = warp >> 2;
    for (int mt = 0; mt < w / 128; ++mt) {
      const int64_t feat = f0 + mt * 128 + q * 32 + lane;
      float* dst = a.Hpart + (static_cast<int64_t>(cid) * npad + feat) * L;
      const int cbeg = half * (L / 2), cend = cbeg + L / 2;
      for (int c = cbeg; c < cend; c += 8) {
        float v[8];
        tmem_ld8(tH + static_cast<uint32_t>(mt * L + c) + (static_cast<uint32_t>(q * 32) << 16), v);
        if (!any_tile || dead_sh) {
#pragma unroll
          for (int i = 0; i < 8; ++i) v[i] = 0.f;
        }
        reinterpret_cast<float4*>(dst + c)[0] = make_float4(v[0], v[1], v[2], v[3]);
        reinterpret_cast<float4*>(dst + c)[1] = make_float4(v[4], v[5], v[6], v[7]);
      }
    }
  }
  // column sums: combine the row phases in order through shared memory (sA is free now)
  double* stage = reinterpret_cast<double*>(sA);
  if (loader) {
#pragma unroll
    for (int i = 0; i < 8; ++i) stage[rp * w + cc * 8 + i] = cs_acc[i];
  }
  __syncthreads();
  for (int f = tid; f < w; f += TC_NT) {
    double s = 0.0;
    for (int p = 0; p < RP; ++p) s += stage[p * w + f];
    a.cs_part[static_cast<int64_t>(cid) * npad + f0 + f] = s;
  }
  {
    const int LL = L * L;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int e = tid + TC_NT * i;
      if (e < LL) a.gram_part[cta * LL + e] = gram_acc[i];
    }
    if (tid < L) a.sG_part[cta * L + tid] = sg_acc;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
  // keep the cluster together until every peer is done with our shared memory
  cluster_sync();
}

// H (FP64) += sum over clusters of the FP32 partial slices; colsum likewise.
__global__ void tc_finish_kernel(const float* __restrict__ Hpart, const double* __restrict__ cs_part, int ncl,
                                 int64_t n, int64_t npad, int L, double* __restrict__ H, double* __restrict__ colsum) {
  const int64_t total = n * L;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double acc = 0.0;
    for (int c = 0; c < ncl; ++c) acc += static_cast<double>(Hpart[static_cast<int64_t>(c) * npad * L + idx]);
    H[idx] += acc;
    if (idx < n) {
      double s = 0.0;
      for (int c = 0; c < ncl; ++c) s += cs_part[static_cast<int64_t>(c) * npad + idx];
      colsum[idx] += s;
    }
  }
}

// Omega as BF16 (RNE of the FP32 value) in the pre-swizzled chunk layout of the kernel:
// chunk g (features 64g..64g+63) is L rows (Omega columns) of 128 bytes, 8-row atoms.
__global__ void omega_bf16_kernel(uint64_t seed, int64_t n, int64_t npad, int l, int L, __nv_bfloat16* __restrict__ out) {
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
      *reinterpret_cast<__nv_bfloat16*>(chunk + off) = __float2bfloat16_rn(v);
    }
  }
}

int grid_for(int64_t total, int threads) {
  int64_t b = (total + threads - 1) / threads;
  if (b > 152 * 16) b = 152 * 16;
  return static_cast<int>(b < 1 ? 1 : b);
}

}  // namespace

bool tc_config(int64_t n, int L, TcConfig* cfg) {
  if (L > 64 || L % 16 != 0) return false;
  for (int CS : {4, 8, 16}) {
    const int64_t w = ((n + CS - 1) / CS + 127) / 128 * 128;
    if (w > 640) continue;
    if ((1 + w / 128) * L > static_cast<int64_t>(TMEM_COLS)) continue;
    const TcLayout lay = tc_layout(L, static_cast<int>(w), CS);
    if (lay.total > 227u * 1024u) continue;
    cfg->CS = CS;
    cfg->w = static_cast<int>(w);
    cfg->smem = lay.total;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaFuncSetAttribute(sketch_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(lay.total));
    cudaFuncSetAttribute(sketch_tc_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
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
    if (cudaOccupancyMaxActiveClusters(&ncl, sketch_tc_kernel, &lc) != cudaSuccess || ncl < 1) {
      cudaGetLastError();
      continue;
    }
    cfg->nclusters = ncl;
    return true;
  }
  return false;
}

cudaError_t launch_omega_bf16(uint64_t seed, int64_t n, int64_t npad, int l, int L, __nv_bfloat16* out,
                              cudaStream_t st, Prof* prof) {
  if (prof) prof->begin(SPCA_K_OMEGA, st);
  omega_bf16_kernel<<<grid_for(npad * (L / 4), 256), 256, 0, st>>>(seed, n, npad, l, L, out);
  if (prof) prof->end(SPCA_K_OMEGA, st);
  return cudaGetLastError();
}

cudaError_t tc_pass(const State& s, const TcWork& w, const TcPending& pend, cudaStream_t st, Prof* prof) {
  if (pend.nseg == 0) return cudaSuccess;
  TcArgs args;
  std::memset(&args, 0, sizeof(args));
  int64_t tiles = 0;
  bool vec_ok = true;
  for (int i = 0; i < pend.nseg; ++i) {
    args.seg[i].rows = pend.rows[i];
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
  args.shift = s.shift;
  args.om16 = w.om16;
  args.Hpart = w.Hpart;
  args.cs_part = w.cs_part;
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
  cudaError_t e = cudaLaunchKernelEx(&lc, sketch_tc_kernel, args);
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
  const int64_t npad = static_cast<int64_t>(w.cfg.CS) * w.cfg.w;
  prof->begin(SPCA_K_H_FINISH, st);
  tc_finish_kernel<<<grid_for(s.n * s.L, 256), 256, 0, st>>>(w.Hpart, w.cs_part, w.cfg.nclusters, s.n, npad, s.L,
                                                             s.H, s.colsum);
  prof->end(SPCA_K_H_FINISH, st);
  prof->begin(SPCA_K_GRAM_ACCUM, st);
  e = launch_gram_accum(w.gram_part, w.sG_part, w.cfg.nclusters * w.cfg.CS, s.L, s.gram, s.sG, st);
  prof->end(SPCA_K_GRAM_ACCUM, st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace spca

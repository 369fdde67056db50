// The streaming pass in plain FP32 on the CUDA cores (Alg. 4 steps 3-7, Eq. 11).
//
// One piece of m rows (row-major, leading dimension ld) is folded into the
// session state by five launches, all reductions in a fixed order so that the
// result is bit-reproducible:
//   omega      a1  Omega (n x L FP32, from the Philox counter of each entry)
//   g_partial  a3  split-K partial sketches  Gpart[s] = A_hat[:, K_s] Omega[K_s, :]
//   g_finish   a3  G = sum_s Gpart[s]; per 32-row group: G^T G and 1^T G  (a5)
//   gram_accum a5  Gram += sum of the group partials (FP64), sG += ...
//   h_partial  a4  split-rows partials  Hpart[t] = A_hat[R_t, :]^T G[R_t, :]
//                  and the column sums of A_hat over R_t (a5)
//   h_finish   a4  H += sum_t Hpart[t]; colsum += sum_t (FP64)
// with A_hat = A - 1 c^T rounded to FP32 on load (a2), c the session's shift.
// The two contractions are register-tiled 128 x 64 tiles (8 x 4 outputs per
// thread, 32-deep K chunks double-buffered in shared memory); both are bound by
// the FP32 FMA pipe (4 m n l flops against m n element reads).
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_fp16.h>

#include <mutex>

#include "philox.cuh"
#include "spca_internal.cuh"

namespace spca {

namespace {

constexpr int BM = 128, BN = 64, BK = 32, NT = 256, APAD = 4;
constexpr int GROUP_ROWS = 32;   // rows per Gram partial
// dynamic shared memory of the two contractions (above the 48 KB static limit)
constexpr size_t kSmemG = sizeof(float) * (2 * BK * (BM + APAD) + 2 * BK * BN);
constexpr size_t kSmemH = sizeof(float) * (2 * BK * BM + 2 * BK * BN + (NT / 32) * BM);

template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
}

// ------------------------------------------------------------------ element loads

template <typename T> struct Elem;
template <> struct Elem<float> {
  static __device__ __forceinline__ float get(const float* p, int64_t i, float) { return __ldg(p + i); }
  static __device__ __forceinline__ float4 get4(const float* p, int64_t i, float) {
    return __ldg(reinterpret_cast<const float4*>(p + i));
  }
};
template <> struct Elem<double> {
  // doubles are shifted in FP64 (see load4 below); these return FP32 only for the shift-free path
  static __device__ __forceinline__ float get(const double* p, int64_t i, float) { return static_cast<float>(__ldg(p + i)); }
  static __device__ __forceinline__ float4 get4(const double* p, int64_t i, float) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p + i));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p + i + 2));
    return make_float4(static_cast<float>(a.x), static_cast<float>(a.y), static_cast<float>(b.x), static_cast<float>(b.y));
  }
};
template <> struct Elem<__nv_bfloat16> {
  static __device__ __forceinline__ float get(const __nv_bfloat16* p, int64_t i, float) { return __bfloat162float(p[i]); }
  static __device__ __forceinline__ float4 get4(const __nv_bfloat16* p, int64_t i, float) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(p + i));
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xFFFF0000u),
                       __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xFFFF0000u));
  }
};
template <> struct Elem<__nv_fp8_e4m3> {
  static __device__ __forceinline__ float get(const __nv_fp8_e4m3* p, int64_t i, float scale) {
    return static_cast<float>(p[i]) * scale;
  }
  static __device__ __forceinline__ float4 get4(const __nv_fp8_e4m3* p, int64_t i, float scale) {
    return make_float4(get(p, i, scale), get(p, i + 1, scale), get(p, i + 2, scale), get(p, i + 3, scale));
  }
};

// Four consecutive shifted elements a[j..j+3] - c[j..j+3] of one row, zero past `jend`.
template <typename T>
__device__ __forceinline__ float4 load4_shifted(const T* row, int64_t j, int64_t jend, const float* shift,
                                                float scale, bool vec_ok) {
  float4 r;
  if (vec_ok && j + 3 < jend) {
    if constexpr (std::is_same<T, double>::value) {
      const double2 a = __ldg(reinterpret_cast<const double2*>(row + j));
      const double2 b = __ldg(reinterpret_cast<const double2*>(row + j + 2));
      const float4 c = __ldg(reinterpret_cast<const float4*>(shift + j));
      r = make_float4(static_cast<float>(a.x - static_cast<double>(c.x)), static_cast<float>(a.y - static_cast<double>(c.y)),
                      static_cast<float>(b.x - static_cast<double>(c.z)), static_cast<float>(b.y - static_cast<double>(c.w)));
    } else {
      const float4 a = Elem<T>::get4(row, j, scale);
      const float4 c = __ldg(reinterpret_cast<const float4*>(shift + j));
      r = make_float4(a.x - c.x, a.y - c.y, a.z - c.z, a.w - c.w);
    }
  } else {
    float v[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (j + t < jend) {
        if constexpr (std::is_same<T, double>::value) {
          v[t] = static_cast<float>(__ldg(row + j + t) - static_cast<double>(__ldg(shift + j + t)));
        } else {
          v[t] = Elem<T>::get(row, j + t, scale) - __ldg(shift + j + t);
        }
      } else {
        v[t] = 0.f;
      }
    }
    r = make_float4(v[0], v[1], v[2], v[3]);
  }
  return r;
}

// Kahan (compensated) summation step: s + x with the rounding error carried in c; the
// sum is s - c.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = __fsub_rn(x, c);
  const float t = __fadd_rn(s, y);
  c = __fsub_rn(__fsub_rn(t, s), y);
  s = t;
}

// 8 x 4 register tile update from one BK-deep chunk: acc[i][j] += sum_k As[k][m0+i] * Bs[k][n0+j].
template <int LDA>
__device__ __forceinline__ void mma_chunk(const float (*As)[LDA], const float (*Bs)[BN], int m0, int n0, float acc[8][4]) {
#pragma unroll
  for (int kk = 0; kk < BK; ++kk) {
    const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][m0]);
    const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][m0 + 4]);
    const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][n0]);
    const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
  }
}

// ------------------------------------------------------------------ a1: Omega

__global__ void omega_f32_kernel(uint64_t seed, int64_t n, int l, int L, float* __restrict__ out, int64_t ld) {
  const int qn = L / 4;
  const int64_t total = n * qn;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t j = idx / qn;
    const int q = static_cast<int>(idx % qn);
    const U32x4 w = omega_words_at(seed, j, static_cast<uint32_t>(q), 0u);
    double z[4];
    box_muller(w.x, w.y, z[0], z[1]);
    box_muller(w.z, w.w, z[2], z[3]);
    float4 v;
    v.x = (4 * q + 0 < l) ? static_cast<float>(z[0]) : 0.f;
    v.y = (4 * q + 1 < l) ? static_cast<float>(z[1]) : 0.f;
    v.z = (4 * q + 2 < l) ? static_cast<float>(z[2]) : 0.f;
    v.w = (4 * q + 3 < l) ? static_cast<float>(z[3]) : 0.f;
    float* dst = out + j * ld + 4 * q;
    dst[0] = v.x; dst[1] = v.y; dst[2] = v.z; dst[3] = v.w;
  }
}

// Omega given as a matrix (n x L FP64, ld L; the power scheme's orth(H)) in FP32, columns
// >= l zero.
__global__ void omega_from_q_f32_kernel(const double* __restrict__ Q, int64_t n, int l, int L, float* __restrict__ out) {
  const int64_t total = n * L;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x)
    out[idx] = (idx % L) < l ? static_cast<float>(Q[idx]) : 0.f;
}

__global__ void omega_words_kernel(uint64_t seed, int64_t n, int qn, uint32_t* __restrict__ out) {
  const int64_t total = n * qn;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t j = idx / qn;
    const int q = static_cast<int>(idx % qn);
    const U32x4 w = omega_words_at(seed, j, static_cast<uint32_t>(q), 0u);
    uint32_t* dst = out + idx * 4;
    dst[0] = w.x; dst[1] = w.y; dst[2] = w.z; dst[3] = w.w;
  }
}

// ------------------------------------------------------------------ shift c

template <typename T>
__global__ void shift_partial_kernel(const T* __restrict__ rows, int64_t m, int64_t n, int64_t ld, float scale,
                                     int64_t rows_per_part, double* __restrict__ part) {
  const int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (j >= n) return;
  const int64_t r0 = blockIdx.y * rows_per_part;
  const int64_t r1 = r0 + rows_per_part < m ? r0 + rows_per_part : m;
  if constexpr (std::is_same<T, double>::value) {
    double acc = 0.0;
    for (int64_t i = r0; i < r1; ++i) acc += rows[i * ld + j];
    part[blockIdx.y * n + j] = acc;
  } else {
    // FP64 adds issue at a small fraction of the FP32 rate here: sum as an FP32 pair instead
    // (Knuth's two-sum keeps each add's rounding error, about 48 significant bits in all)
    float hi = 0.f, lo = 0.f;
    for (int64_t i = r0; i < r1; ++i) {
      float x, xe = 0.f;
      if constexpr (std::is_same<T, __nv_fp8_e4m3>::value) {
        // the stored value code * scale exactly, as a pair (two-product): the mean is of the
        // rows as stored, not of their FP32 roundings
        const float code = static_cast<float>(rows[i * ld + j]);
        x = code * scale;
        xe = fmaf(code, scale, -x);
      } else {
        x = Elem<T>::get(rows, i * ld + j, scale);
      }
      const float s = hi + x;
      const float bb = s - hi;
      lo += (hi - (s - bb)) + (x - bb) + xe;
      hi = s;
    }
    part[blockIdx.y * n + j] = static_cast<double>(hi) + static_cast<double>(lo);
  }
}

__global__ void shift_final_kernel(const double* __restrict__ part, int parts, int64_t n, int64_t m,
                                   float* __restrict__ shift) {
  const int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (j >= n) return;
  double acc = 0.0;
  for (int p = 0; p < parts; ++p) acc += part[p * n + j];
  shift[j] = static_cast<float>(acc / static_cast<double>(m));
}

// ------------------------------------------------------------------ a3: G partials

template <typename T>
__global__ void __launch_bounds__(NT, 2)
g_partial_kernel(const T* __restrict__ A, int64_t m, int64_t n, int64_t ld, const float* __restrict__ shift,
                 float scale, bool vec_ok, const float* __restrict__ omega, int L, int64_t kslice,
                 float* __restrict__ Gpart, int64_t mstride) {
  extern __shared__ __align__(16) float smem_g[];
  float (*As)[BK][BM + APAD] = reinterpret_cast<float (*)[BK][BM + APAD]>(smem_g);
  float (*Bs)[BK][BN] = reinterpret_cast<float (*)[BK][BN]>(smem_g + 2 * BK * (BM + APAD));
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t row0 = static_cast<int64_t>(blockIdx.x) * BM;
  const int s = blockIdx.y;
  const int c0 = blockIdx.z * BN;
  const int64_t kb = static_cast<int64_t>(s) * kslice;
  const int64_t ke = kb + kslice < n ? kb + kslice : n;
  const int nchunks = ke > kb ? static_cast<int>((ke - kb + BK - 1) / BK) : 0;

  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

  float4 ra[4], rb[2];
  // A chunk: 128 rows x 32 features; thread -> row (tid >> 3) + 32 it, features (tid & 7) * 4
  auto gload = [&](int64_t k0) {
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int64_t r = row0 + (tid >> 3) + 32 * it;
      const int64_t j = k0 + (tid & 7) * 4;
      ra[it] = (r < m) ? load4_shifted<T>(A + r * ld, j, ke, shift, scale, vec_ok) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      const int64_t j = k0 + (tid >> 4) + 16 * it;
      const int c = c0 + (tid & 15) * 4;
      rb[it] = (j < ke && c < L) ? __ldg(reinterpret_cast<const float4*>(omega + j * L + c))
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  auto sstore = [&](int buf) {
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int r = (tid >> 3) + 32 * it;
      const int k = (tid & 7) * 4;
      As[buf][k + 0][r] = ra[it].x;
      As[buf][k + 1][r] = ra[it].y;
      As[buf][k + 2][r] = ra[it].z;
      As[buf][k + 3][r] = ra[it].w;
    }
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      *reinterpret_cast<float4*>(&Bs[buf][(tid >> 4) + 16 * it][(tid & 15) * 4]) = rb[it];
    }
  };

  if (nchunks > 0) {
    gload(kb);
    sstore(0);
    __syncthreads();
    for (int ch = 0; ch < nchunks; ++ch) {
      const int buf = ch & 1;
      if (ch + 1 < nchunks) gload(kb + static_cast<int64_t>(ch + 1) * BK);
      mma_chunk<BM + APAD>(As[buf], Bs[buf], ty * 8, tx * 4, acc);
      if (ch + 1 < nchunks) sstore(buf ^ 1);
      __syncthreads();
    }
  }
  const int c = c0 + tx * 4;
  if (c < L) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t r = row0 + ty * 8 + i;
      if (r < m) {
        *reinterpret_cast<float4*>(Gpart + (static_cast<int64_t>(s) * mstride + r) * L + c) =
            make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      }
    }
  }
}

// ---- FP32 rows, 16-byte aligned, n a multiple of 4: operands staged by cp.async rings
// (several chunks in flight per CTA, no registers held across the loads), then the shift
// subtracted in shared memory. Same tiles, same per-thread 8 x 4 products and the same
// arithmetic per element as the kernels above.

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc, bool valid) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gsrc), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

constexpr int GC_STAGES = 3;
constexpr int GC_RAW_LD = BK + 4;   // raw A rows padded: the transposing reads below are conflict-free
constexpr size_t kSmemGcp = sizeof(float) * (GC_STAGES * BM * GC_RAW_LD + GC_STAGES * BK * BN + BK * (BM + APAD));

__global__ void __launch_bounds__(NT, 2)
g_partial_cp_kernel(const float* __restrict__ A, int64_t m, int64_t n, int64_t ld, const float* __restrict__ shift,
                    const float* __restrict__ omega, int L, int64_t kslice, float* __restrict__ Gpart,
                    int64_t mstride) {
  extern __shared__ __align__(16) float smem_gc[];
  float (*raw)[BM][GC_RAW_LD] = reinterpret_cast<float (*)[BM][GC_RAW_LD]>(smem_gc);
  float (*Bs)[BK][BN] = reinterpret_cast<float (*)[BK][BN]>(smem_gc + GC_STAGES * BM * GC_RAW_LD);
  float (*As)[BM + APAD] = reinterpret_cast<float (*)[BM + APAD]>(smem_gc + GC_STAGES * BM * GC_RAW_LD +
                                                                   GC_STAGES * BK * BN);
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t row0 = static_cast<int64_t>(blockIdx.x) * BM;
  const int s = blockIdx.y;
  const int c0 = blockIdx.z * BN;
  const int64_t kb = static_cast<int64_t>(s) * kslice;
  const int64_t ke = kb + kslice < n ? kb + kslice : n;
  const int nchunks = ke > kb ? static_cast<int>((ke - kb + BK - 1) / BK) : 0;

  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

  auto issue = [&](int ch) {   // chunk ch of this K slice into stage ch % GC_STAGES
    const int stg = ch % GC_STAGES;
    const int64_t k0 = kb + static_cast<int64_t>(ch) * BK;
#pragma unroll
    for (int it = 0; it < 4; ++it) {   // A: 128 rows x 8 float4
      const int idx = tid + it * NT;
      const int r = idx >> 3, q = idx & 7;
      const int64_t gr = row0 + r, gk = k0 + q * 4;
      const bool ok = gr < m && gk < ke;
      cp_async16(&raw[stg][r][q * 4], ok ? A + gr * ld + gk : A, ok);
    }
#pragma unroll
    for (int it = 0; it < 2; ++it) {   // Omega: 32 rows x 16 float4
      const int idx = tid + it * NT;
      const int kr = idx >> 4, q = idx & 15;
      const int64_t gk = k0 + kr;
      const int c = c0 + q * 4;
      const bool ok = gk < ke && c < L;
      cp_async16(&Bs[stg][kr][q * 4], ok ? omega + gk * L + c : omega, ok);
    }
  };
  if (nchunks > 0) {
#pragma unroll
    for (int p = 0; p < GC_STAGES - 1; ++p) {
      if (p < nchunks) issue(p);
      cp_async_commit();
    }
    const int rr = tid & (BM - 1), kq = tid / BM;   // conversion: row rr, features [16 kq, 16 kq + 16)
    const bool row_ok = row0 + rr < m;
    for (int ch = 0; ch < nchunks; ++ch) {
      cp_async_wait<GC_STAGES - 2>();
      __syncthreads();   // chunk ch has landed everywhere; every thread is past the products of ch - 1
      const int stg = ch % GC_STAGES;
      const int64_t k0 = kb + static_cast<int64_t>(ch) * BK;
#pragma unroll
      for (int q = 0; q < 4; ++q) {   // As[k][r] = raw[r][k] - c_k
        const int k = 16 * kq + 4 * q;
        const float4 v = *reinterpret_cast<const float4*>(&raw[stg][rr][k]);
        const int64_t gk = k0 + k;
        const bool ok = row_ok && gk < ke;
        const float4 cc = gk < ke ? __ldg(reinterpret_cast<const float4*>(shift + gk)) : make_float4(0.f, 0.f, 0.f, 0.f);
        As[k + 0][rr] = ok ? v.x - cc.x : 0.f;
        As[k + 1][rr] = ok ? v.y - cc.y : 0.f;
        As[k + 2][rr] = ok ? v.z - cc.z : 0.f;
        As[k + 3][rr] = ok ? v.w - cc.w : 0.f;
      }
      if (ch + GC_STAGES - 1 < nchunks) issue(ch + GC_STAGES - 1);
      cp_async_commit();
      __syncthreads();   // As holds chunk ch
      mma_chunk<BM + APAD>(As, Bs[stg], ty * 8, tx * 4, acc);
    }
  }
  const int c = c0 + tx * 4;
  if (c < L) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t r = row0 + ty * 8 + i;
      if (r < m) {
        *reinterpret_cast<float4*>(Gpart + (static_cast<int64_t>(s) * mstride + r) * L + c) =
            make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      }
    }
  }
}

// G = sum over splits (fixed order); per group of 32 rows: Gram and column-sum partials.
__global__ void g_finish_kernel(const float* __restrict__ Gpart, int S, int64_t mstride, int64_t m, int L, int l,
                                float* __restrict__ G, float* __restrict__ G_out, double* __restrict__ gram_part,
                                double* __restrict__ sG_part, int* __restrict__ flags) {
  extern __shared__ float Gs[];   // GROUP_ROWS x L
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * GROUP_ROWS;
  bool bad = false;
  for (int idx = threadIdx.x; idx < GROUP_ROWS * L; idx += blockDim.x) {
    const int r = idx / L, c = idx % L;
    const int64_t row = r0 + r;
    float v = 0.f;
    if (row < m) {
      for (int s = 0; s < S; ++s) v += Gpart[(static_cast<int64_t>(s) * mstride + row) * L + c];
      G[row * L + c] = v;
      if (G_out != nullptr && c < l) G_out[row * l + c] = v;
      bad |= !isfinite(v);
    }
    Gs[idx] = v;
  }
  if (bad) atomicOr(flags, 1);
  __syncthreads();
  // Gram partial in double-float arithmetic: each product is split exactly into p + pe
  // (fma), each addition into s + se (two-sum), so the group sum carries ~48 bits.
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
    const int c1 = e / L, c2 = e % L;
    float hi = 0.f, lo = 0.f;
#pragma unroll 8
    for (int r = 0; r < GROUP_ROWS; ++r) {
      const float a = Gs[r * L + c1], b = Gs[r * L + c2];
      const float p = a * b;
      const float pe = fmaf(a, b, -p);
      const float s = hi + p;
      const float bb = s - hi;
      const float se = (hi - (s - bb)) + (p - bb);
      hi = s;
      lo += se + pe;
    }
    gram_part[static_cast<int64_t>(blockIdx.x) * L * L + e] = static_cast<double>(hi) + static_cast<double>(lo);
  }
  for (int c = threadIdx.x; c < L; c += blockDim.x) {
    double acc = 0.0;
    for (int r = 0; r < GROUP_ROWS; ++r) acc += static_cast<double>(Gs[r * L + c]);
    sG_part[static_cast<int64_t>(blockIdx.x) * L + c] = acc;
  }
}

// Gram += sum of the group partials. A block owns 32 entries (its lanes); warp w sums the
// partials p = w, w + 8, ... in order, then the 8 warp sums are added in warp order.
constexpr int ACC_WARPS = 8;
__global__ void __launch_bounds__(32 * ACC_WARPS)
gram_accum_kernel(const double* __restrict__ gram_part, const double* __restrict__ sG_part, int parts, int L,
                  double* __restrict__ gram, double* __restrict__ sG) {
  __shared__ double red[ACC_WARPS][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + lane;
  const int LL = L * L;
  // entries [0, LL) are the Gram matrix, [LL, LL + L) the column sums of G
  double acc = 0.0;
  if (e < LL) {
    for (int p = w; p < parts; p += ACC_WARPS) acc += gram_part[static_cast<int64_t>(p) * LL + e];
  } else if (e < LL + L) {
    for (int p = w; p < parts; p += ACC_WARPS) acc += sG_part[static_cast<int64_t>(p) * L + (e - LL)];
  }
  red[w][lane] = acc;
  __syncthreads();
  if (w == 0) {
    double t = 0.0;
#pragma unroll
    for (int ww = 0; ww < ACC_WARPS; ++ww) t += red[ww][lane];
    if (e < LL) gram[e] += t;
    else if (e < LL + L) sG[e - LL] += t;
  }
}

// ------------------------------------------------------------------ a4: H partials

template <typename T>
__global__ void __launch_bounds__(NT, 2)
h_partial_kernel(const T* __restrict__ A, int64_t m, int64_t n, int64_t ld, const float* __restrict__ shift,
                 float scale, bool vec_ok, const float* __restrict__ G, int L, int64_t rslice,
                 float* __restrict__ Hpart, float* __restrict__ cs_part) {
  extern __shared__ __align__(16) float smem_h[];
  float (*As)[BK][BM] = reinterpret_cast<float (*)[BK][BM]>(smem_h);
  float (*Bs)[BK][BN] = reinterpret_cast<float (*)[BK][BN]>(smem_h + 2 * BK * BM);
  float (*red)[BM] = reinterpret_cast<float (*)[BM]>(smem_h + 2 * BK * BM + 2 * BK * BN);
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t f0 = static_cast<int64_t>(blockIdx.x) * BM;
  const int t = blockIdx.y;
  const int c0 = blockIdx.z * BN;
  const int64_t rb_ = static_cast<int64_t>(t) * rslice;
  const int64_t re = rb_ + rslice < m ? rb_ + rslice : m;
  const int nchunks = re > rb_ ? static_cast<int>((re - rb_ + BK - 1) / BK) : 0;
  const bool do_cs = (blockIdx.z == 0);

  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  // column sums with Kahan compensation: the shifted sums are small against the sum of
  // magnitudes (the shift is only the first rows' mean), so plain FP32 sums lose digits
  float cs[4] = {0.f, 0.f, 0.f, 0.f};
  float cc[4] = {0.f, 0.f, 0.f, 0.f};

  float4 ra[4], rg[2];
  // A chunk: 32 rows x 128 features; thread -> row (tid >> 5) + 8 it, features (tid & 31) * 4
  auto gload = [&](int64_t r0c) {
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int64_t r = r0c + (tid >> 5) + 8 * it;
      const int64_t j = f0 + (tid & 31) * 4;
      ra[it] = (r < re) ? load4_shifted<T>(A + r * ld, j, n, shift, scale, vec_ok) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      const int64_t r = r0c + (tid >> 4) + 16 * it;
      const int c = c0 + (tid & 15) * 4;
      rg[it] = (r < re && c < L) ? __ldg(reinterpret_cast<const float4*>(G + r * L + c)) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  auto sstore = [&](int buf) {
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      *reinterpret_cast<float4*>(&As[buf][(tid >> 5) + 8 * it][(tid & 31) * 4]) = ra[it];
      if (do_cs) {
        kahan_add(cs[0], cc[0], ra[it].x);
        kahan_add(cs[1], cc[1], ra[it].y);
        kahan_add(cs[2], cc[2], ra[it].z);
        kahan_add(cs[3], cc[3], ra[it].w);
      }
    }
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      *reinterpret_cast<float4*>(&Bs[buf][(tid >> 4) + 16 * it][(tid & 15) * 4]) = rg[it];
    }
  };

  if (nchunks > 0) {
    gload(rb_);
    sstore(0);
    __syncthreads();
    for (int ch = 0; ch < nchunks; ++ch) {
      const int buf = ch & 1;
      if (ch + 1 < nchunks) gload(rb_ + static_cast<int64_t>(ch + 1) * BK);
      mma_chunk<BM>(As[buf], Bs[buf], ty * 8, tx * 4, acc);
      if (ch + 1 < nchunks) sstore(buf ^ 1);
      __syncthreads();
    }
  }
  const int c = c0 + tx * 4;
  if (c < L) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t j = f0 + ty * 8 + i;
      if (j < n) {
        *reinterpret_cast<float4*>(Hpart + (static_cast<int64_t>(t) * n + j) * L + c) =
            make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      }
    }
  }
  if (do_cs) {
    const int w = tid >> 5;
    const int fl = (tid & 31) * 4;
    red[w][fl + 0] = cs[0] - cc[0]; red[w][fl + 1] = cs[1] - cc[1];
    red[w][fl + 2] = cs[2] - cc[2]; red[w][fl + 3] = cs[3] - cc[3];
    __syncthreads();
    if (tid < BM) {
      float v = 0.f, vc = 0.f;
#pragma unroll
      for (int ww = 0; ww < NT / 32; ++ww) kahan_add(v, vc, red[ww][tid]);
      v -= vc;
      const int64_t j = f0 + tid;
      if (j < n) cs_part[static_cast<int64_t>(t) * n + j] = v;
    }
  }
}

constexpr int HC_STAGES = 4;
constexpr size_t kSmemHcp = sizeof(float) * (HC_STAGES * BK * BM + HC_STAGES * BK * BN + 2 * BM);

__global__ void __launch_bounds__(NT, 2)
h_partial_cp_kernel(const float* __restrict__ A, int64_t m, int64_t n, int64_t ld, const float* __restrict__ shift,
                    const float* __restrict__ G, int L, int64_t rslice, float* __restrict__ Hpart,
                    float* __restrict__ cs_part) {
  extern __shared__ __align__(16) float smem_hc[];
  float (*As)[BK][BM] = reinterpret_cast<float (*)[BK][BM]>(smem_hc);
  float (*Gs)[BK][BN] = reinterpret_cast<float (*)[BK][BN]>(smem_hc + HC_STAGES * BK * BM);
  float (*red)[BM] = reinterpret_cast<float (*)[BM]>(smem_hc + HC_STAGES * BK * BM + HC_STAGES * BK * BN);
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t f0 = static_cast<int64_t>(blockIdx.x) * BM;
  const int t = blockIdx.y;
  const int c0 = blockIdx.z * BN;
  const int64_t rb_ = static_cast<int64_t>(t) * rslice;
  const int64_t re = rb_ + rslice < m ? rb_ + rslice : m;
  const int nchunks = re > rb_ ? static_cast<int>((re - rb_ + BK - 1) / BK) : 0;
  const bool do_cs = (blockIdx.z == 0);

  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

  auto issue = [&](int ch) {   // chunk ch of this row slice into stage ch % HC_STAGES
    const int stg = ch % HC_STAGES;
    const int64_t r0c = rb_ + static_cast<int64_t>(ch) * BK;
#pragma unroll
    for (int it = 0; it < 4; ++it) {   // A: 32 rows x 32 float4 (128 features)
      const int idx = tid + it * NT;
      const int r = idx >> 5, q = idx & 31;
      const int64_t gr = r0c + r, gf = f0 + q * 4;
      const bool ok = gr < re && gf < n;
      cp_async16(&As[stg][r][q * 4], ok ? A + gr * ld + gf : A, ok);
    }
#pragma unroll
    for (int it = 0; it < 2; ++it) {   // G: 32 rows x 16 float4
      const int idx = tid + it * NT;
      const int r = idx >> 4, q = idx & 15;
      const int64_t gr = r0c + r;
      const int c = c0 + q * 4;
      const bool ok = gr < re && c < L;
      cp_async16(&Gs[stg][r][q * 4], ok ? G + gr * L + c : G, ok);
    }
  };
  const int ff = tid & (BM - 1), kh = tid / BM;   // conversion: feature ff, rows [16 kh, 16 kh + 16)
  const int64_t gf = f0 + ff;
  const float cf = gf < n ? __ldg(shift + gf) : 0.f;
  float csum = 0.f, ccomp = 0.f;   // Kahan-compensated column sum (see h_partial_kernel)
  if (nchunks > 0) {
#pragma unroll
    for (int p = 0; p < HC_STAGES - 1; ++p) {
      if (p < nchunks) issue(p);
      cp_async_commit();
    }
    for (int ch = 0; ch < nchunks; ++ch) {
      cp_async_wait<HC_STAGES - 2>();
      __syncthreads();   // chunk ch has landed everywhere; every thread is past the products of ch - 1
      const int stg = ch % HC_STAGES;
      const int64_t r0c = rb_ + static_cast<int64_t>(ch) * BK;
#pragma unroll
      for (int q = 0; q < BK / 2; ++q) {   // the shift, in place, and the column sums
        const int r = 16 * kh + q;
        const bool ok = r0c + r < re && gf < n;
        const float v = ok ? As[stg][r][ff] - cf : 0.f;
        As[stg][r][ff] = v;
        kahan_add(csum, ccomp, v);
      }
      if (ch + HC_STAGES - 1 < nchunks) issue(ch + HC_STAGES - 1);
      cp_async_commit();
      __syncthreads();
      mma_chunk<BM>(As[stg], Gs[stg], ty * 8, tx * 4, acc);
    }
  }
  const int c = c0 + tx * 4;
  if (c < L) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t j = f0 + ty * 8 + i;
      if (j < n) {
        *reinterpret_cast<float4*>(Hpart + (static_cast<int64_t>(t) * n + j) * L + c) =
            make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      }
    }
  }
  if (do_cs) {
    red[kh][ff] = csum - ccomp;
    __syncthreads();
    if (tid < BM && f0 + tid < n) cs_part[static_cast<int64_t>(t) * n + f0 + tid] = red[0][tid] + red[1][tid];
  }
}

__global__ void h_finish_kernel(const float* __restrict__ Hpart, const float* __restrict__ cs_part, int T, int64_t n,
                                int L, double* __restrict__ H, double* __restrict__ colsum) {
  // the T FP32 partials are summed as an FP32 pair (two-sum, ~48 bits: FP64 adds issue at a
  // small fraction of the FP32 rate here), then added once into the FP64 state
  auto sum_pair = [](const float* p, int64_t stride, int T_) {
    float hi = 0.f, lo = 0.f;
    for (int t = 0; t < T_; ++t) {
      const float x = p[static_cast<int64_t>(t) * stride];
      const float s = hi + x;
      const float bb = s - hi;
      lo += (hi - (s - bb)) + (x - bb);
      hi = s;
    }
    return static_cast<double>(hi) + static_cast<double>(lo);
  };
  const int64_t total = n * L;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    H[idx] += sum_pair(Hpart + idx, total, T);
    if (idx < n) colsum[idx] += sum_pair(cs_part + idx, n, T);
  }
}

__global__ void merge_kernel(double* __restrict__ H, const double* __restrict__ Hs, double* __restrict__ colsum,
                             const double* __restrict__ colsum_s, double* __restrict__ gram,
                             const double* __restrict__ gram_s, double* __restrict__ sG,
                             const double* __restrict__ sG_s, int64_t n, int L) {
  const int64_t total = n * L > static_cast<int64_t>(L) * L ? n * L : static_cast<int64_t>(L) * L;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    if (idx < n * L) H[idx] += Hs[idx];
    if (idx < n) colsum[idx] += colsum_s[idx];
    if (idx < static_cast<int64_t>(L) * L) gram[idx] += gram_s[idx];
    if (idx < L) sG[idx] += sG_s[idx];
  }
}

// Shift rebase of a merge. Sessions that saw different first rows subtract different
// shifts: src accumulated A_s = A - 1 c_s^T, dst wants A - 1 c_d^T = A_s + 1 delta^T with
// delta = c_s - c_d, hence G_d = G_s + 1 gamma^T with gamma = Omega^T delta (Omega as the
// pass used it: FP32, or rounded to BF16 / FP16). Summing over the m_s rows of src:
//   H_d = H_s + s_s gamma^T + delta sG_s^T + m_s delta gamma^T
//   Gram_d = Gram_s + sG_s gamma^T + gamma sG_s^T + m_s gamma gamma^T
//   s_d = s_s + m_s delta,  sG_d = sG_s + m_s gamma
// (s = column sums of the shifted rows, sG = column sums of G; Eq. 11 is a sum over rows).
// gamma_c, one block per column c < l, Omega regenerated from the seed, FP64 sums in a fixed
// order. fmt: 0 FP32, 1 BF16, 2 FP16.
__global__ void rebase_gamma_kernel(uint64_t seed, int64_t n, int fmt, const float* __restrict__ c_src,
                                    const float* __restrict__ c_dst, double* __restrict__ gamma) {
  __shared__ double red[256];
  const int c = blockIdx.x;
  double acc = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const double d = static_cast<double>(c_src[j]) - static_cast<double>(c_dst[j]);
    if (d == 0.0) continue;
    const U32x4 wv = omega_words_at(seed, j, static_cast<uint32_t>(c / 4), 0u);
    double z[4];
    box_muller(wv.x, wv.y, z[0], z[1]);
    box_muller(wv.z, wv.w, z[2], z[3]);
    const float f = static_cast<float>(z[c & 3]);
    double v = f;
    if (fmt == 1) v = __bfloat162float(__float2bfloat16_rn(f));
    if (fmt == 2) v = __half2float(__float2half_rn(f));
    acc = fma(v, d, acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) gamma[c] = red[0];
}

__global__ void merge_rebase_kernel(double* __restrict__ H, const double* __restrict__ Hs, double* __restrict__ colsum,
                                    const double* __restrict__ colsum_s, double* __restrict__ gram,
                                    const double* __restrict__ gram_s, double* __restrict__ sG,
                                    const double* __restrict__ sG_s, const float* __restrict__ c_src,
                                    const float* __restrict__ c_dst, const double* __restrict__ gamma, double m_s,
                                    int64_t n, int l, int L) {
  const int64_t total = n * L > static_cast<int64_t>(L) * L ? n * L : static_cast<int64_t>(L) * L;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    if (idx < n * L) {
      const int64_t j = idx / L;
      const int c = static_cast<int>(idx - j * L);
      double v = Hs[idx];
      if (c < l) {
        const double d = static_cast<double>(c_src[j]) - static_cast<double>(c_dst[j]);
        v += colsum_s[j] * gamma[c] + d * sG_s[c] + m_s * d * gamma[c];
      }
      H[idx] += v;
    }
    if (idx < n) {
      const double d = static_cast<double>(c_src[idx]) - static_cast<double>(c_dst[idx]);
      colsum[idx] += colsum_s[idx] + m_s * d;
    }
    if (idx < static_cast<int64_t>(L) * L) {
      const int a = static_cast<int>(idx / L), b = static_cast<int>(idx % L);
      double v = gram_s[idx];
      if (a < l && b < l) v += sG_s[a] * gamma[b] + gamma[a] * sG_s[b] + m_s * gamma[a] * gamma[b];
      gram[idx] += v;
    }
    if (idx < L) sG[idx] += sG_s[idx] + (idx < l ? m_s * gamma[idx] : 0.0);
  }
}

int grid_for(int64_t total, int threads) {
  int64_t b = (total + threads - 1) / threads;
  if (b > 152 * 32) b = 152 * 32;
  return static_cast<int>(b < 1 ? 1 : b);
}

template <typename T>
cudaError_t simt_pass_t(const State& s, const SimtWork& w, const T* rows, float scale, int64_t m, int64_t ld,
                        float* G_out, cudaStream_t st, Prof* prof) {
  const int L = s.L;
  const int col_tiles = (L + BN - 1) / BN;
  size_t align = 16;
  const bool vec_ok = (reinterpret_cast<uintptr_t>(rows) % align == 0) && (ld % 4 == 0);
  // a3: split K = n into S slices of whole BK chunks
  const int row_tiles = static_cast<int>((m + BM - 1) / BM);
  const int64_t kchunks = (s.n + BK - 1) / BK;
  const int64_t mstride = static_cast<int64_t>(row_tiles) * BM;
  int S = static_cast<int>(608 / (row_tiles * col_tiles));
  if (S > w.gp_rows / mstride) S = static_cast<int>(w.gp_rows / mstride);
  if (S > kchunks) S = static_cast<int>(kchunks);
  if (S < 1) S = 1;
  const int64_t kslice = ((kchunks + S - 1) / S) * BK;
  S = static_cast<int>((s.n + kslice - 1) / kslice);
  // FP32 rows that allow 16-byte copies take the kernels with cp.async rings
  bool use_cp = false;
  if constexpr (std::is_same<T, float>::value) use_cp = vec_ok && (s.n % 4 == 0);
  static std::atomic<uint64_t> g_attr{0};
  static std::mutex g_mu;
  {
    const cudaError_t ea = once_per_device(g_attr, g_mu, [] {
      cudaError_t e = allow_smem(g_partial_kernel<T>, kSmemG);
      if (e != cudaSuccess) return e;
      if constexpr (std::is_same<T, float>::value) {
        e = allow_smem(g_partial_cp_kernel, kSmemGcp);
        if (e != cudaSuccess) return e;
        e = allow_smem(h_partial_cp_kernel, kSmemHcp);
      }
      return e;
    });
    if (ea != cudaSuccess) return ea;
  }
  prof->begin(SPCA_K_G_PARTIAL, st);
  if constexpr (std::is_same<T, float>::value) {
    if (use_cp)
      g_partial_cp_kernel<<<dim3(row_tiles, S, col_tiles), NT, kSmemGcp, st>>>(rows, m, s.n, ld, s.shift, s.omega32, L,
                                                                              kslice, w.Gpart, mstride);
  }
  if (!use_cp)
    g_partial_kernel<T><<<dim3(row_tiles, S, col_tiles), NT, kSmemG, st>>>(rows, m, s.n, ld, s.shift, scale, vec_ok,
                                                                           s.omega32, L, kslice, w.Gpart, mstride);
  prof->end(SPCA_K_G_PARTIAL, st);
  const int groups = static_cast<int>((m + GROUP_ROWS - 1) / GROUP_ROWS);
  prof->begin(SPCA_K_G_FINISH, st);
  g_finish_kernel<<<groups, 256, GROUP_ROWS * L * sizeof(float), st>>>(w.Gpart, S, mstride, m, L, s.l, w.G, G_out,
                                                                       w.gram_part, w.sG_part, s.flags);
  prof->end(SPCA_K_G_FINISH, st);
  prof->begin(SPCA_K_GRAM_ACCUM, st);
  gram_accum_kernel<<<(L * L + L + 31) / 32, 32 * ACC_WARPS, 0, st>>>(w.gram_part, w.sG_part, groups, L, s.gram,
                                                                       s.sG);
  prof->end(SPCA_K_GRAM_ACCUM, st);
  // a4: split the rows into T slices of whole BK chunks
  const int f_tiles = static_cast<int>((s.n + BM - 1) / BM);
  const int64_t rchunks = (m + BK - 1) / BK;
  int T_ = static_cast<int>(608 / (f_tiles * col_tiles));
  if (T_ > w.T) T_ = w.T;
  if (T_ > rchunks) T_ = static_cast<int>(rchunks);
  if (T_ < 1) T_ = 1;
  const int64_t rslice = ((rchunks + T_ - 1) / T_) * BK;
  T_ = static_cast<int>((m + rslice - 1) / rslice);
  static std::atomic<uint64_t> h_attr{0};
  static std::mutex h_mu;
  {
    const cudaError_t ea = once_per_device(h_attr, h_mu, [] { return allow_smem(h_partial_kernel<T>, kSmemH); });
    if (ea != cudaSuccess) return ea;
  }
  prof->begin(SPCA_K_H_PARTIAL, st);
  if constexpr (std::is_same<T, float>::value) {
    if (use_cp)
      h_partial_cp_kernel<<<dim3(f_tiles, T_, col_tiles), NT, kSmemHcp, st>>>(rows, m, s.n, ld, s.shift, w.G, L, rslice,
                                                                              w.Hpart, w.cs_part);
  }
  if (!use_cp)
    h_partial_kernel<T><<<dim3(f_tiles, T_, col_tiles), NT, kSmemH, st>>>(rows, m, s.n, ld, s.shift, scale, vec_ok,
                                                                          w.G, L, rslice, w.Hpart, w.cs_part);
  prof->end(SPCA_K_H_PARTIAL, st);
  prof->begin(SPCA_K_H_FINISH, st);
  h_finish_kernel<<<grid_for(s.n * L, 256), 256, 0, st>>>(w.Hpart, w.cs_part, T_, s.n, L, s.H, s.colsum);
  prof->end(SPCA_K_H_FINISH, st);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ second pass: U = A_bar V Sigma^-1

// U (column i at U + i ldu, FP64) of a block of rows: the FP32 split-K partials of
// (a - c) W summed over the slices, minus the centring term corr (FP64): with
// mu = c + s_hat / m the column means, (a - mu) W = (a - c) W - (s_hat / m)^T W.
__global__ void u_finish_kernel(const float* __restrict__ Gpart, int S, int64_t mstride, int64_t m, int L, int k,
                                const double* __restrict__ corr, double* __restrict__ U, int64_t ldu) {
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < m * k;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = idx / k;
    const int j = static_cast<int>(idx - r * k);
    double v = 0.0;
    for (int s = 0; s < S; ++s) v += static_cast<double>(Gpart[(static_cast<int64_t>(s) * mstride + r) * L + j]);
    U[static_cast<int64_t>(j) * ldu + r] = v - corr[j];
  }
}

template <typename T>
cudaError_t u_pass_t(const T* rows, float scale, int64_t m, int64_t n, int64_t ld, const float* shift, const float* W,
                     int L, int k, const double* corr, float* Gpart, int64_t gp_rows, double* U, int64_t ldu,
                     cudaStream_t st) {
  const bool vec_ok = (reinterpret_cast<uintptr_t>(rows) % 16 == 0) && (ld % 4 == 0);
  const int col_tiles = (L + BN - 1) / BN;
  for (int64_t p0 = 0; p0 < m; p0 += gp_rows) {   // pieces whose partials fit the workspace
    const int64_t mp = m - p0 < gp_rows ? m - p0 : gp_rows;
    const int row_tiles = static_cast<int>((mp + BM - 1) / BM);
    const int64_t kchunks = (n + BK - 1) / BK;
    const int64_t mstride = static_cast<int64_t>(row_tiles) * BM;
    int S = static_cast<int>(608 / (row_tiles * col_tiles));
    if (S > gp_rows / mstride) S = static_cast<int>(gp_rows / mstride);
    if (S > kchunks) S = static_cast<int>(kchunks);
    if (S < 1) S = 1;
    const int64_t kslice = ((kchunks + S - 1) / S) * BK;
    S = static_cast<int>((n + kslice - 1) / kslice);
    const T* src = rows + p0 * ld;
    g_partial_kernel<T><<<dim3(row_tiles, S, col_tiles), NT, kSmemG, st>>>(src, mp, n, ld, shift, scale, vec_ok, W, L,
                                                                           kslice, Gpart, mstride);
    u_finish_kernel<<<grid_for(mp * k, 256), 256, 0, st>>>(Gpart, S, mstride, mp, L, k, corr, U + p0, ldu);
  }
  return cudaGetLastError();
}


template <typename T>
cudaError_t shift_t(const T* rows, int64_t m, int64_t n, int64_t ld, float scale, float* shift, double* part,
                    cudaStream_t st, Prof* prof) {
  int parts = static_cast<int>((m + 63) / 64);
  if (parts > kShiftParts) parts = kShiftParts;
  const int64_t rows_per_part = (m + parts - 1) / parts;
  parts = static_cast<int>((m + rows_per_part - 1) / rows_per_part);
  const int nb = static_cast<int>((n + 255) / 256);
  prof->begin(SPCA_K_SHIFT, st);
  shift_partial_kernel<T><<<dim3(nb, parts), 256, 0, st>>>(rows, m, n, ld, scale, rows_per_part, part);
  prof->end(SPCA_K_SHIFT, st);
  prof->begin(SPCA_K_SHIFT, st);
  shift_final_kernel<<<nb, 256, 0, st>>>(part, parts, n, m, shift);
  prof->end(SPCA_K_SHIFT, st);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_u_pass(const void* rows, int dtype, float scale, int64_t m, int64_t n, int64_t ld,
                          const float* shift, const float* W, int L, int k, const double* corr, float* Gpart,
                          int64_t gp_rows, double* U, int64_t ldu, cudaStream_t st) {
  static std::atomic<uint64_t> attr{0};
  static std::mutex mu;
  const cudaError_t ea = once_per_device(attr, mu, [] {
    cudaError_t e = allow_smem(g_partial_kernel<float>, kSmemG);
    if (e == cudaSuccess) e = allow_smem(g_partial_kernel<__nv_bfloat16>, kSmemG);
    if (e == cudaSuccess) e = allow_smem(g_partial_kernel<__nv_fp8_e4m3>, kSmemG);
    if (e == cudaSuccess) e = allow_smem(g_partial_kernel<double>, kSmemG);
    return e;
  });
  if (ea != cudaSuccess) return ea;
  switch (dtype) {
    case SPCA_F32:
      return u_pass_t(static_cast<const float*>(rows), scale, m, n, ld, shift, W, L, k, corr, Gpart, gp_rows, U, ldu, st);
    case SPCA_F64:
      return u_pass_t(static_cast<const double*>(rows), scale, m, n, ld, shift, W, L, k, corr, Gpart, gp_rows, U, ldu,
                      st);
    case SPCA_BF16:
      return u_pass_t(static_cast<const __nv_bfloat16*>(rows), scale, m, n, ld, shift, W, L, k, corr, Gpart, gp_rows, U,
                      ldu, st);
    case SPCA_F8E4M3:
      return u_pass_t(static_cast<const __nv_fp8_e4m3*>(rows), scale, m, n, ld, shift, W, L, k, corr, Gpart, gp_rows,
                      U, ldu, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_omega_f32(uint64_t seed, int64_t n, int l, int L, float* out, int64_t ld, cudaStream_t st,
                             Prof* prof) {
  if (prof) prof->begin(SPCA_K_OMEGA, st);
  omega_f32_kernel<<<grid_for(n * (L / 4), 256), 256, 0, st>>>(seed, n, l, L, out, ld);
  if (prof) prof->end(SPCA_K_OMEGA, st);
  return cudaGetLastError();
}

cudaError_t launch_omega_from_q_f32(const double* Q, int64_t n, int l, int L, float* out, cudaStream_t st) {
  omega_from_q_f32_kernel<<<grid_for(n * L, 256), 256, 0, st>>>(Q, n, l, L, out);
  return cudaGetLastError();
}

cudaError_t launch_omega_words(uint64_t seed, int64_t n, int l, uint32_t* out, cudaStream_t st) {
  const int qn = (l + 3) / 4;
  omega_words_kernel<<<grid_for(n * qn, 256), 256, 0, st>>>(seed, n, qn, out);
  return cudaGetLastError();
}

cudaError_t launch_shift(const void* rows, int dtype, int64_t m, int64_t n, int64_t ld, float scale, float* shift,
                         double* part, cudaStream_t st, Prof* prof) {
  switch (dtype) {
    case SPCA_F32: return shift_t(static_cast<const float*>(rows), m, n, ld, scale, shift, part, st, prof);
    case SPCA_F64: return shift_t(static_cast<const double*>(rows), m, n, ld, scale, shift, part, st, prof);
    case SPCA_BF16: return shift_t(static_cast<const __nv_bfloat16*>(rows), m, n, ld, scale, shift, part, st, prof);
    case SPCA_F8E4M3: return shift_t(static_cast<const __nv_fp8_e4m3*>(rows), m, n, ld, scale, shift, part, st, prof);
    default: return cudaErrorInvalidValue;
  }
}

// Scratch of spca_shift_static: a file-scope device array, so that the entry point needs no
// allocation. Every partial a call reads is written earlier in the same call, so the array
// never needs clearing; concurrent calls on one device share it and must be serialised.
static __device__ __align__(256) double g_shift_scratch[kShiftParts * SPCA_SHIFT_STATIC_MAX_N];

cudaError_t shift_static_scratch(double** out) {
  constexpr int kMaxDevices = 64;
  static std::mutex mu;
  static double* addr[kMaxDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_shift_scratch);   // with device `dev` current
    if (e != cudaSuccess) return e;
    addr[dev] = static_cast<double*>(p);
  }
  *out = addr[dev];
  return cudaSuccess;
}

cudaError_t simt_pass(const State& s, const SimtWork& w, const void* rows, int dtype, float scale, int64_t m,
                      int64_t ld, float* G_out, cudaStream_t st, Prof* prof) {
  switch (dtype) {
    case SPCA_F32: return simt_pass_t(s, w, static_cast<const float*>(rows), scale, m, ld, G_out, st, prof);
    case SPCA_F64: return simt_pass_t(s, w, static_cast<const double*>(rows), scale, m, ld, G_out, st, prof);
    case SPCA_BF16: return simt_pass_t(s, w, static_cast<const __nv_bfloat16*>(rows), scale, m, ld, G_out, st, prof);
    case SPCA_F8E4M3: return simt_pass_t(s, w, static_cast<const __nv_fp8_e4m3*>(rows), scale, m, ld, G_out, st, prof);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_gram_accum(const double* gram_part, const double* sG_part, int parts, int L, double* gram,
                              double* sG, cudaStream_t st) {
  gram_accum_kernel<<<(L * L + L + 31) / 32, 32 * ACC_WARPS, 0, st>>>(gram_part, sG_part, parts, L, gram, sG);
  return cudaGetLastError();
}

cudaError_t launch_merge(const State& dst, const State& src, cudaStream_t st) {
  const int64_t total = dst.n > dst.L ? dst.n * dst.L : static_cast<int64_t>(dst.L) * dst.L;
  merge_kernel<<<grid_for(total, 256), 256, 0, st>>>(dst.H, src.H, dst.colsum, src.colsum, dst.gram,
                                                              src.gram, dst.sG, src.sG, dst.n, dst.L);
  return cudaGetLastError();
}

cudaError_t launch_merge_rebase(const State& dst, const State& src, uint64_t seed, int fmt, int64_t m_src,
                                double* gamma, cudaStream_t st) {
  rebase_gamma_kernel<<<dst.l, 256, 0, st>>>(seed, dst.n, fmt, src.shift, dst.shift, gamma);
  const int64_t total = dst.n * dst.L > int64_t(dst.L) * dst.L ? dst.n * dst.L : int64_t(dst.L) * dst.L;
  merge_rebase_kernel<<<grid_for(total, 256), 256, 0, st>>>(dst.H, src.H, dst.colsum, src.colsum, dst.gram,
                                                             src.gram, dst.sG, src.sG, src.shift, dst.shift, gamma,
                                                             static_cast<double>(m_src), dst.n, dst.l, dst.L);
  return cudaGetLastError();
}

}  // namespace spca

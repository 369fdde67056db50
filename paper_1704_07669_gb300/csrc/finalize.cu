// FP64 finalisation on the device (Alg. 4 steps 9-20, in the Gram reading of Thm 1).
//
// Inputs are the pass accumulators on the shifted rows A_hat = A - 1 c^T:
// H_hat = A_hat^T G_hat (FP32), gram = G_hat^T G_hat, colsum = A_hat^T 1,
// sG = G_hat^T 1 (FP64) and the row count m. Steps:
//  1. centering (exact algebra of the shift): with A_bar = A_hat - (1/m) 1 colsum^T,
//     H_bar = H_hat - colsum sG^T / m and gram_bar = gram - sG sG^T / m.
//  2. R from gram_bar: gram_bar = L1 L1^T (Cholesky, R1 = L1^T), one refinement
//     in Gram space, X = L1^-1 gram_bar L1^-T = L2 L2^T, and T = L2^-1 L1^-1 = R^-T
//     with R = R2 R1. Then Q = G_bar R^-1 has orthonormal columns and
//     B = Q^T A_bar = T H_bar^T (Thm 1). Thm 1 assumes full column rank: if a
//     Cholesky pivot falls below l eps max(diag), or if fewer rows were seen
//     than l (the centred Gram then has rank <= m - 1), use the eigendecomposition
//     gram_bar = W diag(lam) W^T instead, keep at most that rank and only
//     lam > l eps lam_max, and set T = diag(lam_r)^-1/2 W_r^T.
//  3. Bt = H_bar T^T (n x r), i.e. B^T, and C = B B^T (r x r) in one sweep over n.
//  4. SVD of B through C = W_B diag(sigma^2) W_B^T (Jacobi with the parallel
//     ordering: an FP32 solve, then a polish of W_B^T C W_B with an FP64 diagonal,
//     see eig_f32_kernel); V = B^T W_B diag(1/sigma), the leading k columns
//     (Alg. 4 steps 17-19).
//  5. Each v_i scaled by +-1 so that its largest-magnitude entry (lowest index
//     on ties) is positive.
// The l x l steps run in one thread block, in shared memory when two l x l
// matrices fit; the n x l steps are spread over the GPU.
#include <cfloat>
#include <cstdio>

#include "spca_internal.cuh"

namespace spca {

namespace {

constexpr int FT = 256;          // threads of the single-block kernels
constexpr int SIGN_T = 1024;     // threads of the sign-fixing kernel
constexpr int BT_ROWS = 32;      // features per block in the B / C kernel

// -------------------------------------------------------------- n x l kernels

__global__ void center_h_kernel(const double* __restrict__ H, const double* __restrict__ colsum,
                                const double* __restrict__ sG, int64_t n, int l, int L, double inv_m,
                                double* __restrict__ Hbar) {
  const int64_t total = n * L;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t j = idx / L;
    const int c = static_cast<int>(idx % L);
    Hbar[idx] = (c < l) ? H[idx] - colsum[j] * sG[c] * inv_m : 0.0;
  }
}

__global__ void center_gram_kernel(const double* __restrict__ gram, const double* __restrict__ sG, int l, int L,
                                   double inv_m, double* __restrict__ gbar) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= L * L) return;
  const int a = e / L, b = e % L;
  gbar[e] = (a < l && b < l) ? gram[e] - sG[a] * sG[b] * inv_m : 0.0;
}

// For a block of BT_ROWS features: Bt[j][i] = sum_c T[i][c] Hbar[j][c] (i < r), and the
// partial C_p = sum_j Bt[j]^T Bt[j] of this block (lower triangle, ld L). FP64 issues at a
// small fraction of the FP32 rate here, so the kernel is built around the FP64 pipe: T^T is
// staged in shared memory (when it fits) so that lanes over i read consecutive words, each
// thread keeps BT_ROWS / 4 independent accumulators, and the lower triangle of C_p is
// packed so that no lane idles over the upper half.
__global__ void __launch_bounds__(256) bt_and_c_kernel(const double* __restrict__ Hbar, const double* __restrict__ T,
                                                       const int* __restrict__ info, int64_t n, int l, int L,
                                                       int tcc, double* __restrict__ Bt,
                                                       double* __restrict__ Cpart) {
  extern __shared__ double sm[];
  double* sH = sm;                  // BT_ROWS x L
  double* sB = sm + BT_ROWS * L;    // BT_ROWS x L
  double* sT = sB + BT_ROWS * L;    // tcc x L: sT[cc * L + i] = T[i][c0 + cc], tcc columns of T at a time
  constexpr int G = 256 / 64;       // row groups; thread = (row group, column i mod 64)
  constexpr int RPT = BT_ROWS / G;  // rows per thread
  const int r = info[0];
  const bool lower = info[1] == 0;   // T from the Cholesky route (the eigen route's T is full)
  const int tri = r * (r + 1) / 2;
  const bool whole = tcc >= l;      // all of T^T staged once
  double* out = Cpart + static_cast<int64_t>(blockIdx.x) * L * L;
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) out[e] = 0.0;
  if (whole) {
    for (int e = threadIdx.x; e < L * l; e += blockDim.x) {
      const int i = e / l, cc = e - i * l;
      sT[cc * L + i] = T[i * L + cc];
    }
  }
  const int grp = threadIdx.x >> 6, il = threadIdx.x & 63;
  const int64_t nblk = (n + BT_ROWS - 1) / BT_ROWS;
  for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const int64_t j0 = blk * BT_ROWS;
    __syncthreads();
    for (int e = threadIdx.x; e < BT_ROWS * L; e += blockDim.x) {
      const int64_t j = j0 + e / L;
      sH[e] = (j < n) ? Hbar[j * L + e % L] : 0.0;
      sB[e] = 0.0;
    }
    for (int c0 = 0; c0 < l; c0 += tcc) {
      if (!whole) {
        __syncthreads();
        const int cn = l - c0 < tcc ? l - c0 : tcc;
        for (int e = threadIdx.x; e < L * cn; e += blockDim.x) {
          const int i = e / cn, cc = e - i * cn;
          sT[cc * L + i] = T[i * L + c0 + cc];
        }
      }
      __syncthreads();
      const int c1 = l - c0 < tcc ? l : c0 + tcc;
      for (int i = il; i < L; i += 64) {
        if (i >= r) continue;
        double acc[RPT];
#pragma unroll
        for (int u = 0; u < RPT; ++u) acc[u] = 0.0;
        // the Cholesky route's T = R^-T is lower triangular (exact zeros above the diagonal):
        // columns c > i add nothing
        const int ce = (lower && c1 > i + 1) ? i + 1 : c1;
        for (int c = c0; c < ce; ++c) {
          const double t = sT[(c - c0) * L + i];
#pragma unroll
          for (int u = 0; u < RPT; ++u) acc[u] = fma(t, sH[(grp + G * u) * L + c], acc[u]);
        }
#pragma unroll
        for (int u = 0; u < RPT; ++u) sB[(grp + G * u) * L + i] += acc[u];
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < BT_ROWS * L; e += blockDim.x) {
      const int64_t j = j0 + e / L;
      if (j < n) Bt[j * L + e % L] = sB[e];
    }
    // this block's own partial over the packed lower triangle, a fixed order per entry
    for (int t = threadIdx.x; t < tri; t += blockDim.x) {
      int a = static_cast<int>((sqrtf(8.f * static_cast<float>(t) + 1.f) - 1.f) * 0.5f);
      while (a * (a + 1) / 2 > t) --a;
      while ((a + 1) * (a + 2) / 2 <= t) ++a;
      const int b = t - a * (a + 1) / 2;
      double acc0 = 0.0, acc1 = 0.0;
#pragma unroll 8
      for (int jr = 0; jr < BT_ROWS; jr += 2) {
        acc0 = fma(sB[jr * L + a], sB[jr * L + b], acc0);
        acc1 = fma(sB[(jr + 1) * L + a], sB[(jr + 1) * L + b], acc1);
      }
      out[a * L + b] += acc0 + acc1;
    }
  }
}

// C = sum over blocks (fixed order), symmetric fill from the lower triangle. A block takes
// 32 entries; its warps sum interleaved subsets of the partials, combined in warp order.
constexpr int CR_T = 256;
__global__ void __launch_bounds__(CR_T) c_reduce_kernel(const double* __restrict__ Cpart, int parts, int L,
                                                        double* __restrict__ C) {
  __shared__ double acc_w[CR_T / 32][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + lane;
  double acc = 0.0;
  if (e < L * L) {
    const int a = e / L, b = e % L;
    const int src = a >= b ? e : (b * L + a);
    for (int p = warp; p < parts; p += CR_T / 32) acc += Cpart[static_cast<int64_t>(p) * L * L + src];
  }
  acc_w[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && e < L * L) {
    double t = 0.0;
    for (int w = 0; w < CR_T / 32; ++w) t += acc_w[w][lane];
    C[e] = t;
  }
}

// V[j][i] (column-major output, ld n) = sum_c Bt[j][c] W[c][i] / sigma_i, i < k. A block
// takes FV_ROWS rows j at a time (staged in shared memory, padded against bank conflicts)
// and, with STAGE_W, the leading r x k block of W too (else W is read through L1, each
// warp reading one address at a time); thread (row j, output group) keeps up to FV_ACC
// independent FP64 accumulators.
constexpr int FV_ROWS = 64;
constexpr int FV_ACC = 13;
template <bool STAGE_W>
__global__ void __launch_bounds__(256) form_v_kernel(const double* __restrict__ Bt, const double* __restrict__ W,
                                                     const double* __restrict__ sig, const int* __restrict__ info,
                                                     int64_t n, int k, int L, double* __restrict__ V) {
  extern __shared__ double fsm[];
  const int r = info[0];
  const int kk = k < r ? k : r;                     // outputs i >= r are zero
  const int ld = r + 1;
  double* sBt = fsm;                                // FV_ROWS x (r + 1)
  double* sInv = fsm + FV_ROWS * ld;                // kk
  double* sW = sInv + kk;                           // r x kk when staged
  for (int i = threadIdx.x; i < kk; i += blockDim.x) sInv[i] = sig[i] > 0.0 ? 1.0 / sig[i] : 0.0;
  if (STAGE_W) {
    for (int e = threadIdx.x; e < r * kk; e += blockDim.x) {
      const int c = e / kk, i = e - c * kk;
      sW[e] = W[c * L + i];
    }
  }
  constexpr int G = 256 / FV_ROWS;
  const int jr = threadIdx.x % FV_ROWS, grp = threadIdx.x / FV_ROWS;
  for (int64_t j0 = static_cast<int64_t>(blockIdx.x) * FV_ROWS; j0 < n; j0 += static_cast<int64_t>(gridDim.x) * FV_ROWS) {
    __syncthreads();
    for (int e = threadIdx.x; e < FV_ROWS * r; e += blockDim.x) {
      const int jj = e / r, c = e - jj * r;
      const int64_t j = j0 + jj;
      sBt[jj * ld + c] = (j < n) ? Bt[j * L + c] : 0.0;
    }
    __syncthreads();
    const int64_t j = j0 + jr;
    for (int i0 = grp; i0 < kk; i0 += G * FV_ACC) {   // outputs i0, i0 + G, ... (FV_ACC of them)
      const int nu = (kk - i0 + G - 1) / G;          // live accumulators (the same in a warp)
      double acc[FV_ACC];
#pragma unroll
      for (int u = 0; u < FV_ACC; ++u) acc[u] = 0.0;
      for (int c = 0; c < r; ++c) {
        const double b = sBt[jr * ld + c];
#pragma unroll
        for (int u = 0; u < FV_ACC; ++u) {
          const int i = i0 + G * u;
          if (u < nu) acc[u] = fma(b, STAGE_W ? sW[c * kk + i] : __ldg(W + c * L + i), acc[u]);
        }
      }
      if (j < n) {
#pragma unroll
        for (int u = 0; u < FV_ACC; ++u) {
          const int i = i0 + G * u;
          if (u < nu) V[static_cast<int64_t>(i) * n + j] = acc[u] * sInv[i];
        }
      }
    }
  }
  if (kk < k) {   // columns beyond the rank
    for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < (k - kk) * n;
         idx += static_cast<int64_t>(gridDim.x) * blockDim.x)
      V[static_cast<int64_t>(kk) * n + idx] = 0.0;
  }
}

// Per column i: the entry of largest |.| (lowest index on ties) is made positive; the sign
// applied goes to flip[i] (+1 or -1).
__global__ void __launch_bounds__(SIGN_T) sign_fix_kernel(double* __restrict__ V, int64_t n, double* __restrict__ flip) {
  __shared__ double best_v[SIGN_T];
  __shared__ int64_t best_j[SIGN_T];
  double* col = V + static_cast<int64_t>(blockIdx.x) * n;
  double bv = -1.0;
  int64_t bj = 0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const double a = fabs(col[j]);
    if (a > bv) { bv = a; bj = j; }   // strictly greater keeps this thread's lowest index
  }
  best_v[threadIdx.x] = bv;
  best_j[threadIdx.x] = bj;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double ov = best_v[threadIdx.x + s];
      const int64_t oj = best_j[threadIdx.x + s];
      if (ov > best_v[threadIdx.x] || (ov == best_v[threadIdx.x] && oj < best_j[threadIdx.x])) {
        best_v[threadIdx.x] = ov;
        best_j[threadIdx.x] = oj;
      }
    }
    __syncthreads();
  }
  const bool neg = col[best_j[0]] < 0.0;
  __syncthreads();
  if (neg) {
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) col[j] = -col[j];
  }
  if (threadIdx.x == 0) flip[blockIdx.x] = neg ? -1.0 : 1.0;
}

// The map from sketch rows to left singular vectors (Alg. 4 steps 18-19 in the Gram reading
// of Thm 1): Q = G_bar R^-1 = G_bar T^T and U = Q U~, U~ the eigenvectors Z of B B^T, so
// U[:, i] = G_bar (T^T Z[:, i]) flip_i. M[c][i] = flip_i sum_{c' < r} T[c'][c] Z[c'][i] (l x k,
// columns beyond the rank 0) and, for the centred rows G_bar = G_hat - (1/m) 1 sG^T,
// mrow[i] = sum_c (sG[c] / m) M[c][i] (0 when centering is off: m = 0).
__device__ double blk_sum(double v, double* red);

// One block per column i (FP64 issues slowly: the l x k entries are spread over the SMs).
__global__ void u_map_kernel(const double* __restrict__ T, const double* __restrict__ Z, const int* __restrict__ info,
                             const double* __restrict__ flip, const double* __restrict__ sG, int64_t m, int l, int L,
                             int k, double* __restrict__ M, double* __restrict__ mrow) {
  __shared__ double red[32];
  const int r = info[0];
  const int kk = k < r ? k : r;
  const int i = blockIdx.x;
  double part = 0.0;
  for (int c = threadIdx.x; c < l; c += blockDim.x) {
    double acc = 0.0;
    if (i < kk) {
      for (int cp = 0; cp < r; ++cp) acc = fma(T[cp * L + c], Z[cp * L + i], acc);
      acc *= flip[i];
    }
    M[c * k + i] = acc;
    if (m > 0) part = fma(sG[c] / static_cast<double>(m), acc, part);
  }
  const double tot = blk_sum(part, red);
  if (threadIdx.x == 0) mrow[i] = tot;
}

// U rows [row0, row0 + mc) from the kept sketch rows: U[i * ldu + row] = G[row0 + row] M[:, i] - mrow[i]
// (G row-major with leading dimension l, FP32; U column-major, FP64).
__global__ void left_vectors_kernel(const float* __restrict__ G, int64_t row0, int64_t mc, int l, int k,
                                    const double* __restrict__ M, const double* __restrict__ mrow,
                                    double* __restrict__ U, int64_t ldu) {
  const int64_t total = mc * k;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t row = idx % mc;
    const int i = static_cast<int>(idx / mc);
    const float* g = G + (row0 + row) * l;
    double acc = 0.0;
    for (int c = 0; c < l; ++c) acc = fma(static_cast<double>(g[c]), M[c * k + i], acc);
    U[i * ldu + row] = acc - mrow[i];
  }
}

// -------------------------------------------------------------- one-block dense helpers
// Matrices are d x d blocks with leading dimension ld, in shared or global memory.
// On this GPU FP64 instructions issue at a small fraction of the FP32 rate and share
// one pipe per SM, so these helpers keep FP64 arithmetic to the work that needs it.

// Block-wide sum of v (every thread gets the same value, summed in the same order);
// red holds >= blockDim.x / 32 doubles.
__device__ double blk_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) s += red[w];
  __syncthreads();
  return s;
}

// The same for two FP32 sums at once; red holds >= blockDim.x / 16 floats.
__device__ void blk_sum2(float& a, float& b, float* red) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[2 * (threadIdx.x >> 5)] = a;
    red[2 * (threadIdx.x >> 5) + 1] = b;
  }
  __syncthreads();
  a = 0.f;
  b = 0.f;
  for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) {
    a += red[2 * w];
    b += red[2 * w + 1];
  }
  __syncthreads();
}

// 2^-e with 2^e <= x < 2^(e+1): an exact scale that brings x to [1, 2) (1 for x <= 0 or
// non-finite x).
__device__ double pow2_scale(double x) {
  if (!(x > 0.0) || !isfinite(x)) return 1.0;
  return ldexp(1.0, -ilogb(x));
}

// Jacobi rotation (c, s) that annihilates a_pq of [[a_pp, a_pq], [a_pq, a_qq]]. The angle is
// found in FP32 (an angle off by 1e-7 relative still shrinks a_pq by seven digits per
// visit); c = (1 + t^2)^-1/2 is then refined by two Newton steps in T, so that c^2 + s^2 = 1
// holds to the precision of T and the accumulated eigenvectors stay orthogonal.
template <typename T>
__device__ __forceinline__ void jacobi_rotation(T app, T aqq, T apq, T& c, T& s) {
  const float theta = static_cast<float>(aqq - app) / (2.f * static_cast<float>(apq));
  const float tf = (theta >= 0.f ? 1.f : -1.f) / (fabsf(theta) + sqrtf(fmaf(theta, theta, 1.f)));
  const T t = static_cast<T>(tf);
  const T x = T(1) + t * t;
  T y = static_cast<T>(rsqrtf(static_cast<float>(x)));
  y = y * (T(1.5) - T(0.5) * x * y * y);
  y = y * (T(1.5) - T(0.5) * x * y * y);
  c = y;
  s = t * y;
}

// FP32 rotation for the FP32 solve: the same formulas with the two divisions taken by the
// fast reciprocal (|2 a_pq| is far from the range where it loses accuracy; an overflowing
// theta gives t = 0, no rotation) and one Newton step on c.
// sqrt.approx: t need not be exact (the next sweeps absorb a slightly wrong angle; c^2 + s^2 = 1
// comes from the rsqrt and its Newton step below), and an infinite theta^2 gives t = 0
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void jacobi_rotation32(float app, float aqq, float apq, float& c, float& s) {
  const float theta = __fdividef(aqq - app, 2.f * apq);
  const float t = __fdividef(theta >= 0.f ? 1.f : -1.f, fabsf(theta) + sqrt_approx(fmaf(theta, theta, 1.f)));
  const float x = fmaf(t, t, 1.f);
  float y = rsqrtf(x);
  y = y * fmaf(-0.5f * x * y, y, 1.5f);
  c = y;
  s = t * y;
}

// Pair pi of round `round` in the round-robin (parallel) ordering of de = m + 1 indices:
// every round pairs each index exactly once, and m rounds visit every pair once.
__device__ __forceinline__ void rr_pair(int round, int pi, int m, int& p, int& q) {
  if (pi == 0) {
    p = m;
    q = round;
  } else {
    p = round + pi;
    if (p >= m) p -= m;
    q = round - pi;
    if (q < 0) q += m;
  }
  if (p > q) { const int t = p; p = q; q = t; }
}

constexpr int kPairRegs = kMaxL / 64;   // pairs per lane in jacobi32: d / 2 <= 32 * kPairRegs

// Rotation `idx` of a round from the lane that holds it (lane idx % 32, register idx / 32).
// Every lane of the warp must call this (shuffles); idx may differ between lanes.
__device__ __forceinline__ void fetch_pair(const int (&pr)[kPairRegs], const float (&cr)[kPairRegs],
                                           const float (&sr)[kPairRegs], int kp, int idx, int& pq, float& c,
                                           float& s) {
  const int src = idx & 31, reg = idx >> 5;
  pq = 0;
  c = 1.f;
  s = 0.f;
#pragma unroll
  for (int t = 0; t < kPairRegs; ++t) {
    if (t < kp) {
      const int v1 = __shfl_sync(0xffffffffu, pr[t], src);
      const float v2 = __shfl_sync(0xffffffffu, cr[t], src);
      const float v3 = __shfl_sync(0xffffffffu, sr[t], src);
      if (t == reg) { pq = v1; c = v2; s = v3; }
    }
  }
}

// Cyclic Jacobi eigendecomposition of the symmetric d x d matrix in A, FP32, parallel
// ordering (an odd d gets a dummy index d that pairs with nothing). Every warp works out all
// rotations of a round itself from the current matrix - lane t holds pairs t, t + 32, ... in
// registers - so that a round needs a single block barrier: the matrix moves between the
// buffers A and A2, each 2 x 2 block (a, b), a <= b, becoming R_a M R_b^T and written with
// its mirror image (the triangle of block pairs is folded into a rectangle of
// ceil(N/2) x (N' + 1) items, N pairs, N' = N rounded up to even, so that lanes stay busy),
// and the rows of W (set to the identity first; the eigenvectors on return, as columns) are
// rotated in place. A pair is left alone when a_pq^2 <= eps_rel^2 |a_pp a_qq|; a rotated
// pair's a_pq is set to zero. Sweeps stop once the off-diagonal part is at most `conv` of
// the whole (squared Frobenius norms), after a sweep without rotations, or after
// max_sweeps. The entries should be scaled to about 1. Returns the buffer (A or A2) that
// holds the final, nearly diagonal matrix; *sweeps_out gets the sweeps made. With A2 NULL
// (when only two d x d matrices fit in shared memory) the blocks are rotated in place, which
// costs a second barrier per round: every warp must have read the round's pivots before any
// block is overwritten.
__device__ float* jacobi32(float* A, float* A2, float* W, int d, int ld, float* red, float conv, float eps_rel,
                           int max_sweeps, int* sweeps_out) {
  const int de = d + (d & 1), npairs = de >> 1, m = de - 1;
  const int nf = npairs + (npairs & 1);            // folded: nf / 2 rows of nf + 1 items
  const int frows = nf >> 1, fcols = nf + 1;
  const int kp = (npairs + 31) >> 5;               // live entries of the per-lane pair registers
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const float eps2 = eps_rel * eps_rel;
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) W[(e / d) * ld + e % d] = ((e / d) == (e % d)) ? 1.f : 0.f;
  __syncthreads();
  float* cur = A;
  float* nxt = A2 ? A2 : A;
  int sweep = 0;
  for (; sweep < max_sweeps && d > 1; ++sweep) {
    float off = 0.f, tot = 0.f;
    for (int i = warp; i < d; i += nwarps) {
      for (int j = lane; j < d; j += 32) {
        const float v = cur[i * ld + j];
        tot = fmaf(v, v, tot);
        if (i != j) off = fmaf(v, v, off);
      }
    }
    blk_sum2(off, tot, red);
    if (off <= conv * tot || tot == 0.f) break;
    bool rotated = false;
    for (int round = 0; round < m; ++round) {
      int pr[kPairRegs];
      float cr[kPairRegs], sr[kPairRegs];
#pragma unroll
      for (int t = 0; t < kPairRegs; ++t) {
        const int pi = lane + 32 * t;
        int p = 0, q = 0;
        float c = 1.f, s = 0.f;
        if (t < kp && pi < npairs) {
          rr_pair(round, pi, m, p, q);
          if (q < d) {
            const float apq = cur[p * ld + q], app = cur[p * ld + p], aqq = cur[q * ld + q];
            const float a2 = apq * apq;
            if (a2 > 1e-37f && a2 > eps2 * fabsf(app * aqq)) {
              jacobi_rotation32(app, aqq, apq, c, s);
              rotated = true;
            }
          }
        }
        pr[t] = p | (q << 16);
        cr[t] = c;
        sr[t] = s;
      }
      if (A2 == nullptr) __syncthreads();   // in place: the pivots are read before blocks change
      // warp-rows: the folded A blocks (fcols items each, in chunks of 32), then W's rows
      const int achunks = (fcols + 31) >> 5;
      const int arows = frows * achunks;
      for (int row = warp; row < arows + (d + 3) / 4; row += nwarps) {
        if (row < arows) {
          const int fr = achunks == 1 ? row : row / achunks, fc = (row - fr * achunks) * 32 + lane;
          int pa, pb;
          if (fc < nf - fr) {
            pa = fr;
            pb = fr + fc;
          } else {
            pa = nf - 1 - fr;
            pb = pa + fc - (nf - fr);
          }
          const bool live = fc < fcols && pb < npairs;   // pa <= pb
          int pqa, pqb;
          float ca, sa, cb, sb;
          fetch_pair(pr, cr, sr, kp, live ? pa : 0, pqa, ca, sa);
          fetch_pair(pr, cr, sr, kp, live ? pb : 0, pqb, cb, sb);
          if (live) {
            const int ia = pqa & 0xffff, ja = pqa >> 16, ib = pqb & 0xffff, jb = pqb >> 16;
            const bool ra = ja < d, rb = jb < d;
            const float m00 = cur[ia * ld + ib];
            const float m01 = rb ? cur[ia * ld + jb] : 0.f;
            const float m10 = ra ? cur[ja * ld + ib] : 0.f;
            const float m11 = (ra && rb) ? cur[ja * ld + jb] : 0.f;
            const float r00 = ca * m00 - sa * m10, r01 = ca * m01 - sa * m11;   // R_a M
            const float r10 = sa * m00 + ca * m10, r11 = sa * m01 + ca * m11;
            const float o00 = cb * r00 - sb * r01, o01 = sb * r00 + cb * r01;   // (R_a M) R_b^T
            const float o10 = cb * r10 - sb * r11, o11 = sb * r10 + cb * r11;
            if (pa == pb) {
              nxt[ia * ld + ia] = o00;
              if (ra) {
                const float z = sa != 0.f ? 0.f : m01;
                nxt[ja * ld + ja] = o11;
                nxt[ia * ld + ja] = z;
                nxt[ja * ld + ia] = z;
              }
            } else {
              nxt[ia * ld + ib] = o00;
              nxt[ib * ld + ia] = o00;
              if (rb) {
                nxt[ia * ld + jb] = o01;
                nxt[jb * ld + ia] = o01;
              }
              if (ra) {
                nxt[ja * ld + ib] = o10;
                nxt[ib * ld + ja] = o10;
              }
              if (ra && rb) {
                nxt[ja * ld + jb] = o11;
                nxt[jb * ld + ja] = o11;
              }
            }
          }
        } else {
          // four rows of W at once (loads first) for the latency of shared memory
          const int i0 = 4 * (row - arows);
#pragma unroll
          for (int t = 0; t < kPairRegs; ++t) {
            const int pb = lane + 32 * t;
            if (t < kp && pb < npairs && sr[t] != 0.f) {
              const int ib = pr[t] & 0xffff, jb = pr[t] >> 16;
              const float cb = cr[t], sb = sr[t];
              float wp[4], wq[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int i = i0 + u < d ? i0 + u : i0;
                wp[u] = W[i * ld + ib];
                wq[u] = W[i * ld + jb];
              }
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                if (i0 + u < d) {
                  W[(i0 + u) * ld + ib] = cb * wp[u] - sb * wq[u];
                  W[(i0 + u) * ld + jb] = sb * wp[u] + cb * wq[u];
                }
              }
            }
          }
        }
      }
      __syncthreads();
      float* t = cur;
      cur = nxt;
      nxt = t;
    }
    // every warp made the same decisions from the same matrix, so this exit is uniform
    if (!__any_sync(0xffffffffu, rotated)) { ++sweep; break; }
  }
  *sweeps_out = sweep;
  return cur;
}

// Cyclic Jacobi eigendecomposition in FP64 (parallel ordering), in place, for the polish of
// a nearly diagonal matrix and for the FP64 fallback route. Warp 0 works out a round's
// rotations and lists only the pairs that need one; the rows of A for those pairs are then
// rotated, and after a barrier the columns of A and of W, so that the FP64 work is
// proportional to the rotations made. A pair is left alone when |a_pq| <= eps_rel
// sqrt(|a_pp a_qq|), or - with tau1 > 0 - when rotating it would move an eigenvalue by less
// than tau1 times the smaller diagonal entry and turn the vectors by less than tau2
// radians. Sweeps stop once the off-diagonal part is at most `conv` of the whole (squared
// Frobenius norms), after a sweep without rotations, or after max_sweeps. On return W holds
// the eigenvectors as columns and, when `sort` is set, lam the eigenvalues descending with
// W's columns in the same order (A is then scratch). The entries should be scaled to about
// 1. Returns the number of sweeps.
__device__ int jacobi64(double* A, double* W, double* lam, int d, int ld, double* red, double conv, double eps_rel,
                        double tau1, double tau2, int max_sweeps, bool sort) {
  __shared__ int act_pq[kMaxL / 2];
  __shared__ double act_c[kMaxL / 2], act_s[kMaxL / 2];
  __shared__ int nact[2];
  __shared__ int needed;
  const int de = d + (d & 1), npairs = de >> 1, m = de - 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double eps2 = eps_rel * eps_rel;
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) W[(e / d) * ld + e % d] = ((e / d) == (e % d)) ? 1.0 : 0.0;
  __syncthreads();
  int sweep = 0;
  for (; sweep < max_sweeps && d > 1; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
      const int i = e / d, j = e - i * d;
      const double v = A[i * ld + j];
      tot = fma(v, v, tot);
      if (i != j) off = fma(v, v, off);
    }
    const double off_sum = blk_sum(off, red);
    const double tot_sum = blk_sum(tot, red);
    if (off_sum <= conv * tot_sum || tot_sum == 0.0) break;
    if (tau1 > 0.0) {
      // look at every pair at once (FP32 estimates) and stop if none needs a rotation
      if (threadIdx.x == 0) needed = 0;
      __syncthreads();
      for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
        const int i = e / d, j = e - i * d;
        if (j <= i) continue;
        const float a = fabsf(static_cast<float>(A[i * ld + j]));
        const float ai = static_cast<float>(A[i * ld + i]), aj = static_cast<float>(A[j * ld + j]);
        const float gap = fabsf(aj - ai), mn = fminf(fabsf(ai), fabsf(aj));
        const bool work = a > static_cast<float>(eps_rel) * sqrtf(fabsf(ai)) * sqrtf(fabsf(aj)) &&
                          !(a * a <= static_cast<float>(tau1) * mn * gap && a <= static_cast<float>(tau2) * gap);
        if (work) needed = 1;
      }
      __syncthreads();
      if (!needed) break;
    }
    bool any = false;
    for (int round = 0; round < m; ++round) {
      if (warp == 0) {
        int base = 0;
        for (int pi0 = 0; pi0 < npairs; pi0 += 32) {
          const int pi = pi0 + lane;
          int p = 0, q = 0;
          bool work = false;
          double c = 1.0, s = 0.0;
          if (pi < npairs) {
            rr_pair(round, pi, m, p, q);
            if (q < d) {
              const double apq = A[p * ld + q], app = A[p * ld + p], aqq = A[q * ld + q];
              const double a2 = apq * apq;
              work = a2 > 1e-300 && a2 > eps2 * fabs(app * aqq);
              if (work && tau1 > 0.0) {
                const double gap = fabs(aqq - app), mn = fmin(fabs(app), fabs(aqq));
                if (a2 <= tau1 * mn * gap && a2 <= (tau2 * gap) * (tau2 * gap)) work = false;
              }
              if (work) jacobi_rotation<double>(app, aqq, apq, c, s);
            }
          }
          const unsigned bal = __ballot_sync(0xffffffffu, work);
          if (work) {
            const int slot = base + __popc(bal & ((1u << lane) - 1u));
            act_pq[slot] = p | (q << 16);
            act_c[slot] = c;
            act_s[slot] = s;
          }
          base += __popc(bal);
        }
        if (lane == 0) nact[round & 1] = base;
      }
      __syncthreads();
      const int n = nact[round & 1];   // two slots: warp 0 may write the next round's first
      if (n == 0) continue;
      any = true;
      const int nd = n * d;
      for (int e = threadIdx.x; e < nd; e += blockDim.x) {   // rows p, q of A
        const int k = e / d, j = e - k * d;
        const int pq = act_pq[k], p = pq & 0xffff, q = pq >> 16;
        const double c = act_c[k], s = act_s[k];
        const double x = A[p * ld + j], y = A[q * ld + j];
        A[p * ld + j] = c * x - s * y;
        A[q * ld + j] = s * x + c * y;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < 2 * nd; e += blockDim.x) {   // columns p, q of A, then of W
        const bool onw = e >= nd;
        const int e2 = onw ? e - nd : e;
        const int i = e2 / n, k = e2 - i * n;
        double* M = onw ? W : A;
        const int pq = act_pq[k], p = pq & 0xffff, q = pq >> 16;
        const double c = act_c[k], s = act_s[k];
        const double x = M[i * ld + p], y = M[i * ld + q];
        M[i * ld + p] = c * x - s * y;
        M[i * ld + q] = s * x + c * y;
      }
      __syncthreads();
    }
    if (!any) { ++sweep; break; }
  }
  if (!sort) return sweep;
  // sort descending: rank of each eigenvalue, then permute W's columns through A as scratch
  for (int i = threadIdx.x; i < d; i += blockDim.x) red[i] = A[i * ld + i];
  __syncthreads();
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    int rank = 0;
    const double v = red[i];
    for (int j = 0; j < d; ++j) {
      const double u = red[j];
      if (u > v || (u == v && j < i)) ++rank;
    }
    lam[rank] = v;
    for (int t = 0; t < d; ++t) A[t * ld + rank] = W[t * ld + i];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) W[(e / d) * ld + e % d] = A[(e / d) * ld + e % d];
  __syncthreads();
  return sweep;
}

// Cyclic Jacobi (parallel ordering) for the polish of a nearly diagonal symmetric matrix,
// held as its diagonal dg in FP64 and its off-diagonal part E in FP32 (E's diagonal unused).
// With off-diagonal entries of about eps_32 |A|, FP32 rounding in them is of order
// eps_32^2 |A|, far below what decides the small eigenvalues, while the diagonal - where
// those eigenvalues build up - is updated in FP64 by a'_pp = a_pp - t a_pq,
// a'_qq = a_qq + t a_pq (t = tan of the angle). Warp 0 works out a round's rotations (and
// the diagonal updates) and lists the pairs that need one; rows p, q of E are then rotated,
// and after a barrier its columns and those of W (FP32, the identity first), so that the
// work is proportional to the rotations made. Skipping and stopping rules as for jacobi64.
// On return lam holds the eigenvalues descending and W's columns the eigenvectors in the
// same order (E is then scratch). Entries should be scaled to about 1. Returns the sweeps.
__device__ int jacobi_mixed(double* dg, float* E, float* W, double* lam, int d, int ld, double* red, double conv,
                            double eps_rel, double tau1, double tau2, int max_sweeps) {
  __shared__ int act_pq[kMaxL / 2];
  __shared__ float act_c[kMaxL / 2], act_s[kMaxL / 2];
  __shared__ int nact[2];
  __shared__ int needed;
  const int de = d + (d & 1), npairs = de >> 1, m = de - 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const double eps2 = eps_rel * eps_rel;
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) W[(e / d) * ld + e % d] = ((e / d) == (e % d)) ? 1.f : 0.f;
  __syncthreads();
  int sweep = 0;
  for (; sweep < max_sweeps && d > 1; ++sweep) {
    float offf = 0.f;
    for (int i = warp; i < d; i += nwarps)
      for (int j = lane; j < d; j += 32)
        if (i != j) offf = fmaf(E[i * ld + j], E[i * ld + j], offf);
    double diag = 0.0;
    for (int i = threadIdx.x; i < d; i += blockDim.x) diag = fma(dg[i], dg[i], diag);
    const double off_sum = blk_sum(static_cast<double>(offf), red);
    const double tot_sum = off_sum + blk_sum(diag, red);
    if (off_sum <= conv * tot_sum || tot_sum == 0.0) break;
    if (tau1 > 0.0) {
      // look at every pair at once (FP32 estimates) and stop if none needs a rotation
      if (threadIdx.x == 0) needed = 0;
      __syncthreads();
      for (int i = warp; i < d; i += nwarps) {
        const float ai = static_cast<float>(dg[i]);
        for (int j = i + 1 + lane; j < d; j += 32) {
          const float a = fabsf(E[i * ld + j]), aj = static_cast<float>(dg[j]);
          const float gap = fabsf(aj - ai), mn = fminf(fabsf(ai), fabsf(aj));
          const bool work = a > static_cast<float>(eps_rel) * sqrtf(fabsf(ai)) * sqrtf(fabsf(aj)) &&
                            !(a * a <= static_cast<float>(tau1) * mn * gap && a <= static_cast<float>(tau2) * gap);
          if (work) needed = 1;
        }
      }
      __syncthreads();
      if (!needed) break;
    }
    bool any = false;
    for (int round = 0; round < m; ++round) {
      if (warp == 0) {
        int base = 0;
        for (int pi0 = 0; pi0 < npairs; pi0 += 32) {
          const int pi = pi0 + lane;
          int p = 0, q = 0;
          bool work = false;
          float c = 1.f, s = 0.f;
          if (pi < npairs) {
            rr_pair(round, pi, m, p, q);
            if (q < d) {
              const double apq = static_cast<double>(E[p * ld + q]), app = dg[p], aqq = dg[q];
              const double a2 = apq * apq;
              work = a2 > 1e-300 && a2 > eps2 * fabs(app * aqq);
              if (work && tau1 > 0.0) {
                const double gap = fabs(aqq - app), mn = fmin(fabs(app), fabs(aqq));
                if (a2 <= tau1 * mn * gap && a2 <= (tau2 * gap) * (tau2 * gap)) work = false;
              }
              if (work) {
                const float theta = static_cast<float>(aqq - app) / (2.f * static_cast<float>(apq));
                const float t = (theta >= 0.f ? 1.f : -1.f) / (fabsf(theta) + sqrtf(fmaf(theta, theta, 1.f)));
                const float x = fmaf(t, t, 1.f);
                float y = rsqrtf(x);
                y = y * fmaf(-0.5f * x * y, y, 1.5f);
                y = y * fmaf(-0.5f * x * y, y, 1.5f);
                c = y;
                s = t * y;
                const double ta = static_cast<double>(t) * apq;
                dg[p] = app - ta;
                dg[q] = aqq + ta;
              }
            }
          }
          const unsigned bal = __ballot_sync(0xffffffffu, work);
          if (work) {
            const int slot = base + __popc(bal & ((1u << lane) - 1u));
            act_pq[slot] = p | (q << 16);
            act_c[slot] = c;
            act_s[slot] = s;
          }
          base += __popc(bal);
        }
        if (lane == 0) nact[round & 1] = base;
      }
      __syncthreads();
      const int n = nact[round & 1];   // two slots: warp 0 may write the next round's first
      if (n == 0) continue;
      any = true;
      for (int k = warp; k < n; k += nwarps) {   // rows p, q of E, columns j outside {p, q}
        const int pq = act_pq[k], p = pq & 0xffff, q = pq >> 16;
        const float c = act_c[k], s = act_s[k];
        for (int j = lane; j < d; j += 32) {
          if (j == p || j == q) continue;
          const float x = E[p * ld + j], y = E[q * ld + j];
          E[p * ld + j] = c * x - s * y;
          E[q * ld + j] = s * x + c * y;
        }
      }
      __syncthreads();
      for (int row = warp; row < 2 * d; row += nwarps) {   // columns p, q of E (rows outside {p, q}), of W
        const bool onw = row >= d;
        const int i = onw ? row - d : row;
        float* M = onw ? W : E;
        for (int k = lane; k < n; k += 32) {
          const int pq = act_pq[k], p = pq & 0xffff, q = pq >> 16;
          if (!onw && (i == p || i == q)) continue;
          const float c = act_c[k], s = act_s[k];
          const float x = M[i * ld + p], y = M[i * ld + q];
          M[i * ld + p] = c * x - s * y;
          M[i * ld + q] = s * x + c * y;
        }
      }
      for (int k = threadIdx.x; k < n; k += blockDim.x) {   // the annihilated entries
        const int pq = act_pq[k], p = pq & 0xffff, q = pq >> 16;
        E[p * ld + q] = 0.f;
        E[q * ld + p] = 0.f;
      }
      __syncthreads();
    }
    if (!any) { ++sweep; break; }
  }
  // sort descending: rank of each eigenvalue, then permute W's columns through E as scratch
  for (int i = threadIdx.x; i < d; i += blockDim.x) red[i] = dg[i];
  __syncthreads();
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    int rank = 0;
    const double v = red[i];
    for (int j = 0; j < d; ++j) {
      const double u = red[j];
      if (u > v || (u == v && j < i)) ++rank;
    }
    lam[rank] = v;
    for (int t = 0; t < d; ++t) E[t * ld + rank] = W[t * ld + i];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) W[(e / d) * ld + e % d] = E[(e / d) * ld + e % d];
  __syncthreads();
  return sweep;
}

// In-place Cholesky: the lower triangle of A becomes L1 (A = L1 L1^T). False if a pivot <= tol.
__device__ bool blk_cholesky(double* A, int d, int ld, double tol) {
  __shared__ int ok;
  if (threadIdx.x == 0) ok = 1;
  __syncthreads();
  for (int k = 0; k < d; ++k) {
    if (threadIdx.x == 0) {
      const double v = A[k * ld + k];
      if (!(v > tol)) ok = 0;
      else A[k * ld + k] = sqrt(v);
    }
    __syncthreads();
    if (!ok) return false;
    const double dk = A[k * ld + k];
    for (int i = k + 1 + threadIdx.x; i < d; i += blockDim.x) A[i * ld + k] /= dk;
    __syncthreads();
    const int rem = d - k - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      const int i = k + 1 + e / rem, j = k + 1 + e % rem;
      if (j <= i) A[i * ld + j] -= A[i * ld + k] * A[j * ld + k];
    }
    __syncthreads();
  }
  return true;
}

// Linv = inverse of the lower triangle of Lm (strict upper part of Linv zeroed).
__device__ void blk_trinv_lower(const double* Lm, double* Linv, int d, int ld) {
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) Linv[(e / d) * ld + e % d] = 0.0;
  __syncthreads();
  for (int c = threadIdx.x; c < d; c += blockDim.x) {
    for (int i = c; i < d; ++i) {
      double acc = (i == c) ? 1.0 : 0.0;
      for (int j = c; j < i; ++j) acc -= Lm[i * ld + j] * Linv[j * ld + c];
      Linv[i * ld + c] = acc / Lm[i * ld + i];
    }
  }
  __syncthreads();
}

// The same factor and inverse, register-resident, for d(d+1)/2 <= blockDim.x * EPT: symmetric
// Gaussian elimination without square roots. Step k subtracts m_ik = x_ik / x_kk times row k
// from every row i > k of the trailing lower triangle (A = M D M^T, M unit lower triangular)
// and applies the same row operations to Y (the identity first), which ends as M^-1; the
// factor is M D^1/2, so its inverse is D^-1/2 M^-1 (row i scaled by x_ii^-1/2 at the end).
// X's trailing part and Y's finished part share one lower-triangular array Z (entry (i, j)
// is X's while j > k and Y's once j <= k: column k of X turns into column k of Y, -m_ik),
// held in registers, EPT entries per thread at fixed places. A step needs column k of Z
// (rows >= k) and row k of Y (columns < k): disjoint index ranges, so one vector u_k holds
// both, which the owners of those entries leave in shared memory (two copies by parity) at
// the end of the step before. Every thread loads all its operands first, then computes,
// then stores, so that a step costs one load latency and one block barrier.
// False, uniformly, if a pivot is <= tol.
template <int EPT>
__device__ bool blk_chol_inv32_reg(const float* X, float* Y, int d, int ld, float tol) {
  __shared__ float piv[kMaxL];
  __shared__ float uvec[2][kMaxL];   // u_k: column k of Z at indices >= k, row k of Y below k
  const int nt = blockDim.x, tri = d * (d + 1) / 2;
  float z[EPT];
  int zi[EPT], zj[EPT];
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int e = threadIdx.x + q * nt;
    zi[q] = -1;
    zj[q] = 0;
    z[q] = 0.f;
    if (e < tri) {   // e -> (i, j), j <= i, row by row
      int i = static_cast<int>((sqrtf(8.f * static_cast<float>(e) + 1.f) - 1.f) * 0.5f);
      while (i * (i + 1) / 2 > e) --i;
      while ((i + 1) * (i + 2) / 2 <= e) ++i;
      const int j = e - i * (i + 1) / 2;
      zi[q] = i;
      zj[q] = j;
      z[q] = X[i * ld + j];
      if (j == 0) uvec[0][i] = z[q];
    }
  }
  __syncthreads();
#ifdef SPCA_FIN_TRACE
  long long tt[4] = {0, 0, 0, 0};
  const long long tstart = clock64();
#endif
  for (int k = 0; k < d; ++k) {
#ifdef SPCA_FIN_TRACE
    const long long q0 = clock64();
#endif
    const float* u = uvec[k & 1];
    float* un = uvec[(k + 1) & 1];
    const float p = u[k];
    if (!(p > tol)) return false;   // the same value in every thread
    if (threadIdx.x == 0) piv[k] = p;
    const float inv = 1.f / p;
    float mi[EPT], rj[EPT];
#pragma unroll
    for (int q = 0; q < EPT; ++q) {   // loads (u at zi > k is column k, at zj: column or row)
      mi[q] = u[zi[q] > k ? zi[q] : k];
      rj[q] = u[zj[q]];
    }
#ifdef SPCA_FIN_TRACE
    float chk = inv;
#pragma unroll
    for (int q = 0; q < EPT; ++q) chk += mi[q] + rj[q];
    if (chk == 123.456f) piv[0] = chk;
    const long long q1 = clock64();
#endif
#pragma unroll
    for (int q = 0; q < EPT; ++q) {   // the updates: column k of Y; X's trailing part and Y's rows
      if (zi[q] > k) {
        const float m = mi[q] * inv;
        z[q] = zj[q] == k ? -m : fmaf(-m, rj[q], z[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < EPT; ++q) {   // u_{k+1}: the next column (indices >= k + 1), the next row of Y
      if (zj[q] == k + 1 && zi[q] > k) un[zi[q]] = z[q];
      else if (zi[q] == k + 1 && zj[q] <= k) un[zj[q]] = z[q];
    }
#ifdef SPCA_FIN_TRACE
    const long long q2 = clock64();
#endif
    __syncthreads();
#ifdef SPCA_FIN_TRACE
    const long long q3 = clock64();
    tt[0] += q1 - q0;
    tt[1] += q2 - q1;
    tt[2] += q3 - q2;
#endif
  }
#ifdef SPCA_FIN_TRACE
  if (threadIdx.x == 0 || threadIdx.x == 480)
    printf("chol reg d=%d thr %d: total %lld (loads+div %lld, update+store %lld, barrier %lld)\n", d, threadIdx.x,
           clock64() - tstart, tt[0], tt[1], tt[2]);
#endif
  const int nw = nt >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = warp; i < d; i += nw)
    for (int j = lane; j < d; j += 32) Y[i * ld + j] = 0.f;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int i = zi[q], j = zj[q];
    if (i >= 0) Y[i * ld + j] = (i == j ? 1.f : z[q]) * rsqrtf(piv[i]);
  }
  __syncthreads();
  return true;
}

// FP32 Cholesky of X (lower triangle, right-looking) and, alongside, Y = the inverse of the
// factor: the row operations of the forward substitution L Y = I are applied to Y (the
// identity first) step by step. Two block barriers per step. False, uniformly, if a pivot
// is <= tol; X's lower triangle then holds a partial factor.
__device__ bool blk_chol_inv32(float* X, float* Y, int d, int ld, float tol) {
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) Y[(e / d) * ld + e % d] = ((e / d) == (e % d)) ? 1.f : 0.f;
  __syncthreads();
  for (int k = 0; k < d; ++k) {
    const float v = X[k * ld + k];
    if (!(v > tol)) return false;   // the same value in every thread
    const float dk = sqrtf(v), inv = 1.f / dk;
    for (int e = threadIdx.x; e < d; e += blockDim.x) {   // column k of L (rows > k), row k of Y
      if (e > k) X[e * ld + k] *= inv;
      else Y[k * ld + e] *= inv;
    }
    __syncthreads();
    if (threadIdx.x == 0) X[k * ld + k] = dk;
    // rows i > k over warps, columns j <= i over lanes: j > k updates the factor, j <= k Y
    for (int i = k + 1 + (threadIdx.x >> 5); i < d; i += blockDim.x >> 5) {
      const float lik = X[i * ld + k];
      for (int j = threadIdx.x & 31; j <= i; j += 32) {
        if (j > k) X[i * ld + j] -= lik * X[j * ld + k];
        else Y[i * ld + j] -= lik * Y[k * ld + j];
      }
    }
    __syncthreads();
  }
  return true;
}

// R from gram_bar (step 2), all in FP64: the fallback when the mixed-precision route
// below fails (info[6] set). Writes T (r x l, ld L) and info = {r, route, sweeps}.
// Work matrices X, Y, Z live in shared memory when `smem` is set (3 l^2 doubles), else in
// the global scratch X / Wg / T.
__global__ void __launch_bounds__(FT) factor_kernel(const double* __restrict__ gbar, int l, int L, int r_max,
                                                    double* __restrict__ T, double* __restrict__ Xg,
                                                    double* __restrict__ Wg, double* __restrict__ lam,
                                                    int* __restrict__ info, int smem) {
  extern __shared__ double fsm[];
  __shared__ double red[FT];
  __shared__ double dmax;
  if (info[6] == 0) return;   // the mixed-precision route succeeded
  const int ld = smem ? l : L;
  double* X = smem ? fsm : Xg;
  double* Y = smem ? fsm + l * l : Wg;
  double* Z = smem ? fsm + 2 * l * l : T;
  if (threadIdx.x == 0) {
    double dm = 0.0;
    for (int i = 0; i < l; ++i) dm = fmax(dm, fabs(gbar[i * L + i]));
    dmax = dm;
  }
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) X[(e / l) * ld + e % l] = gbar[(e / l) * L + e % l];
  __syncthreads();
  const double tol = l * DBL_EPSILON * dmax;
  bool ok = (dmax > 0.0) && (r_max >= l) && blk_cholesky(X, l, ld, tol);
  if (ok) {
    blk_trinv_lower(X, Y, l, ld);                 // Y = T1 = L1^-1
    // refinement: X2 = T1 gbar T1^T, through Z = T1 gbar
    for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
      const int i = e / l, j = e % l;
      double acc = 0.0;
      for (int t = 0; t <= i; ++t) acc = fma(Y[i * ld + t], gbar[t * L + j], acc);
      Z[i * ld + j] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
      const int i = e / l, j = e % l;
      double acc = 0.0;
      for (int t = 0; t <= j; ++t) acc = fma(Z[i * ld + t], Y[j * ld + t], acc);
      X[i * ld + j] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < l * l; e += blockDim.x) {   // symmetrise
      const int i = e / l, j = e % l;
      if (j < i) {
        const double v = 0.5 * (X[i * ld + j] + X[j * ld + i]);
        X[i * ld + j] = v;
        X[j * ld + i] = v;
      }
    }
    __syncthreads();
    ok = blk_cholesky(X, l, ld, l * DBL_EPSILON);
    if (ok) {
      // T = L2^-1 L1^-1: invert L2 into Z, then multiply the two lower triangles
      blk_trinv_lower(X, Z, l, ld);
      for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
        const int i = e / l, j = e % l;
        double acc = 0.0;
        for (int t = j; t <= i; ++t) acc = fma(Z[i * ld + t], Y[t * ld + j], acc);
        X[i * ld + j] = (j <= i) ? acc : 0.0;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
        const int i = e / L, j = e % L;
        T[e] = (i < l && j < l) ? X[i * ld + j] : 0.0;
      }
      if (threadIdx.x == 0) { info[0] = l; info[1] = 0; info[2] = 0; }
      __syncthreads();
      return;
    }
  }
  // eigen route: gbar = W diag(lam) W^T, solved on gbar scaled by a power of two (exact)
  const double sc = pow2_scale(dmax);
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) X[(e / l) * ld + e % l] = sc * gbar[(e / l) * L + e % l];
  __syncthreads();
  // relative off-diagonal Frobenius norm <= 1e-13: below that, round-off of the rotations
  // themselves (about eps * lambda_max per entry) keeps it from shrinking further
  const int sweeps = jacobi64(X, Y, lam, l, ld, red, 1e-26, 1e-18, 0.0, 0.0, 40, true);
  for (int i = threadIdx.x; i < l; i += blockDim.x) lam[i] /= sc;
  __syncthreads();
  __shared__ int r_keep;
  if (threadIdx.x == 0) {
    const double cut = l * DBL_EPSILON * fmax(lam[0], 0.0);
    int r = 0;
    while (r < l && r < r_max && lam[r] > cut) ++r;
    r_keep = r;
    info[0] = r; info[1] = 1; info[2] = sweeps;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
    const int i = e / L, c = e % L;
    T[e] = (i < r_keep && c < l) ? Y[c * ld + i] / sqrt(lam[i]) : 0.0;
  }
}

// SVD of B through C = B B^T (r x r, r = info[0]) in two stages. FP64 arithmetic runs
// at a small fraction of the FP32 rate on this GPU, so a full FP64 Jacobi solve of C is
// the slowest step of the finalisation. Instead:
//  (i) eig_f32_kernel: Jacobi in FP32 gives W0 with C ~ W0 diag W0^T, accurate to about
//      eps_32 |C| (enough for the leading pairs, not for the small eigenvalues);
// (ii) small FP64 products make W0 orthogonal to FP64 precision (two Newton-Schulz steps,
//      W <- W (3 I - W^T W) / 2) and form C1 = W^T C W, nearly diagonal;
// (iii) eig_polish_kernel: Jacobi on C1 with its diagonal in FP64 and its (tiny)
//      off-diagonal part in FP32 (jacobi_mixed), skipping the rotations that would change
//      no eigenvalue by more than 1e-8 relative and no vector by more than 1e-6 rad - the
//      remaining work sits among the small eigenvalues that FP32 could not separate;
// (iv) Z = W W1 (FP64): the eigenvectors of C, columns by descending eigenvalue.
// Both solves are one thread block each; the scale of C is brought to about 1 by a power
// of two first (exact), so that FP32 ranges never matter.
constexpr int EIG_T = 512;    // threads of the FP32 Jacobi kernel
constexpr int POL_T = 512;    // threads of the polish and of the FP32 Cholesky kernels

__global__ void __launch_bounds__(EIG_T) eig_f32_kernel(const double* __restrict__ C, float* __restrict__ Xg,
                                                        float* __restrict__ Yg, float* __restrict__ Zg,
                                                        double* __restrict__ W0, int* __restrict__ info, int L,
                                                        int smem) {
  extern __shared__ float e32[];
  __shared__ float red[2 * (EIG_T / 32)];
  __shared__ double scale;
  const int r = info[0];
  const int ld = smem ? (r | 1) : L;   // odd: a column's entries fall in different banks
  // smem: 1 = A, A2 and W in shared memory; 2 = A and W only (rotated in place); 0 = global
  float* X = smem ? e32 : Xg;
  float* X2 = smem == 1 ? e32 + r * ld : (smem == 2 ? nullptr : Zg);
  float* Y = smem == 1 ? e32 + 2 * r * ld : (smem == 2 ? e32 + r * ld : Yg);
  if (threadIdx.x < 32) {   // C scaled by a power of two so that its largest diagonal entry is in [1, 2)
    double dm = 0.0;
    for (int i = threadIdx.x; i < r; i += 32) dm = fmax(dm, fabs(C[i * L + i]));
    for (int o = 16; o > 0; o >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
    if (threadIdx.x == 0) scale = pow2_scale(dm);
  }
  __syncthreads();
  const double sc = scale;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x)
    X[(e / r) * ld + e % r] = static_cast<float>(sc * C[(e / r) * L + e % r]);
  __syncthreads();
  int sweeps = 0;
#ifdef SPCA_FIN_TRACE
  const long long t0 = clock64();
#endif
  if (r > 0) jacobi32(X, X2, Y, r, ld, red, 1e-10f, 3e-8f, 16, &sweeps);
  __syncthreads();
#ifdef SPCA_FIN_TRACE
  if (threadIdx.x == 0) printf("eig_f32 d=%d threads=%d sweeps=%d cycles=%lld\n", r, blockDim.x, sweeps, clock64() - t0);
#endif
  if (threadIdx.x == 0) info[4] = sweeps;
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
    const int i = e / L, j = e % L;
    W0[e] = (i < r && j < r) ? static_cast<double>(Y[i * ld + j]) : 0.0;
  }
}

// The same FP32 Jacobi solve for r <= EIG2_MAXR, organised so that a round needs one
// barrier and shared memory is read and written without bank conflicts. Pairs sit at fixed
// positions (i, np + i) of the de = 2 np padded indices (an odd r gets a zero dummy index);
// after every round the matrix moves one step along the circle ordering (position 0 stays,
// the others form a cycle top 1 .. top np-1, bottom np-1 .. bottom 0), so that m = de - 1
// rounds meet every pair once and bring every index back to where it started. The matrix
// lives in two buffers of odd row stride: a round reads one and writes the other, each 2 x 2
// block (a, b), a <= b, becoming R_a M R_b^T at its moved place together with its mirror
// image (so the matrix stays exactly symmetric). Meanwhile one warp works out the next
// round's rotations from the same input: the three entries that the next round's pair
// will hold are entries of rotated 2 x 2 blocks of this round, which it forms with the same
// arithmetic as the update, and it appends them to a log in global memory. The eigenvector
// matrix is not formed here: eig_replay_kernel applies the logged rotations to the rows of
// the identity, one warp per row, in parallel over the GPU. Stopping rules as in
// eig_f32_kernel; info[4] = sweeps, info[5] = rounds made.
constexpr int EIG2_T = 1024;
constexpr int EIG2_MAXR = 128;
constexpr int EIG2_RW = EIG2_T / 32 - 1;            // the rotation warp; warps 0 .. EIG2_RW - 1 update
constexpr int EIG2_NU = EIG2_RW * 32;               // update threads
constexpr int EIG2_MAXK = (32 * 65 + EIG2_NU - 1) / EIG2_NU;   // blocks per update thread at r = 128
constexpr int EIG2_SWEEPS = 16;

__host__ __device__ inline size_t eig2_smem(int l) {
  const size_t de = static_cast<size_t>(l + (l & 1));
  return sizeof(float) * 2 * de * (de + 1) + sizeof(int) * de;
}

// rotations the log can hold for r <= l: every round of EIG2_SWEEPS sweeps and one more
__host__ __device__ inline size_t eig2_log_len(int l) {
  const size_t de = static_cast<size_t>(l + (l & 1));
  return (EIG2_SWEEPS * (de - 1) + 1) * (de / 2);
}

// Cycle coordinate of position pos != 0 (top i -> i - 1, bottom i -> 2 np - 2 - i) and back.
__device__ __forceinline__ int circ_cyc(int pos, int np) { return pos < np ? pos - 1 : 3 * np - 2 - pos; }
__device__ __forceinline__ int circ_pos(int c, int np) { return c < np - 1 ? c + 1 : 3 * np - 2 - c; }

// Position reached from `pos` after k rounds, |k| < m = 2 np - 1 (k < 0: where it came from).
__device__ __forceinline__ int circ_move(int pos, int k, int np) {
  if (pos == 0) return 0;
  const int m = 2 * np - 1;
  int c = circ_cyc(pos, np) + k;
  if (c >= m) c -= m;
  else if (c < 0) c += m;
  return circ_pos(c, np);
}

// o = R_a M R_b^T for the 2 x 2 block M = [m00 m01; m10 m11], R = [c -s; s c], with every
// rounding fixed (no contraction left to the compiler) so that the update and the rotation
// warp get the same values.
__device__ __forceinline__ void rot_block(float m00, float m01, float m10, float m11, float ca, float sa, float cb,
                                          float sb, float& o00, float& o01, float& o10, float& o11) {
  const float r00 = __fmaf_rn(ca, m00, __fmul_rn(-sa, m10)), r01 = __fmaf_rn(ca, m01, __fmul_rn(-sa, m11));
  const float r10 = __fmaf_rn(sa, m00, __fmul_rn(ca, m10)), r11 = __fmaf_rn(sa, m01, __fmul_rn(ca, m11));
  o00 = __fmaf_rn(cb, r00, __fmul_rn(-sb, r01));
  o01 = __fmaf_rn(sb, r00, __fmul_rn(cb, r01));
  o10 = __fmaf_rn(cb, r10, __fmul_rn(-sb, r11));
  o11 = __fmaf_rn(sb, r10, __fmul_rn(cb, r11));
}

// Entry (i, j) of R_a M R_b^T alone (M at `M`, its bottom row npl floats on, its right
// column np on), with exactly the operations rot_block uses for it.
__device__ __forceinline__ float rot_entry(const float* M, int np, int npl, bool i, bool j, float2 ra, float2 rb) {
  const float a0 = i ? ra.y : ra.x, a1 = i ? ra.x : -ra.y;   // row i of R_a
  const float b0 = j ? rb.y : rb.x, b1 = j ? rb.x : -rb.y;   // row j of R_b
  const float r0 = __fmaf_rn(a0, M[0], __fmul_rn(a1, M[npl]));
  const float r1 = __fmaf_rn(a0, M[np], __fmul_rn(a1, M[npl + np]));
  return __fmaf_rn(b0, r0, __fmul_rn(b1, r1));
}

__device__ __forceinline__ float2 eig2_rotation(float app, float aqq, float apq, float eps2, bool& rotated) {
  float c = 1.f, s = 0.f;
  const float a2 = apq * apq;
  rotated = a2 > 1e-37f && a2 > eps2 * fabsf(app * aqq);
  if (rotated) jacobi_rotation32(app, aqq, apq, c, s);
  return make_float2(c, s);
}

// Double-float numbers (hi + lo, |lo| <= ulp(hi) / 2): the polish keeps its diagonal in this
// form, since FP64 instructions issue at a small fraction of the FP32 rate on this GPU and
// would sit on the critical path of every round. Knuth's two-sum and the FMA two-product.
__device__ __forceinline__ float2 df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {   // a + b, both double-float
  const float2 s = df_two_sum(a.x, b.x);
  const float lo = __fadd_rn(s.y, __fadd_rn(a.y, b.y));
  const float hi = __fadd_rn(s.x, lo);
  return make_float2(hi, __fsub_rn(lo, __fsub_rn(hi, s.x)));
}
__device__ __forceinline__ float2 df_prod(float a, float b) {   // a b exactly, as hi + lo
  const float p = __fmul_rn(a, b);
  return make_float2(p, __fmaf_rn(a, b, -p));
}
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }

// The polish's rotation (the rules of jacobi_mixed): double-float diagonal, FP32 pivot; a
// pair is left alone when a_pq^2 <= eps_rel^2 |a_pp a_qq|, or when rotating it would change
// neither eigenvalue by more than tau1 relative nor the vectors by more than tau2 rad (the
// tests scaled so that nothing underflows for entries of the scaled matrix down to about
// 1e-30). del = t a_pq exactly, the change of the two diagonal entries (a_pp - del, a_qq + del).
constexpr double POL_EPS2 = 1e-36, POL_TAU1 = 1e-8, POL_TAU2 = 1e-6;
__device__ __forceinline__ float2 mixed_rotation(float2 app, float2 aqq, float apq, float2& del, bool& rotated) {
  const float2 gd = df_add(aqq, df_neg(app));
  const float gap = fabsf(gd.x), mn = fminf(fabsf(app.x), fabsf(aqq.x)), aa = fabsf(apq);
  // |a_pq| > 1e-18 sqrt|a_pp a_qq|; a_pq^2 <= tau1 mn gap as (|a_pq| / sqrt(mn))^2 <= tau1 gap
  bool work = aa > 0.f && aa > 1e-18f * sqrtf(fabsf(app.x)) * sqrtf(fabsf(aqq.x));
  if (work) {
    const float q = aa * rsqrtf(fmaxf(mn, 1e-37f));
    if (q * q <= static_cast<float>(POL_TAU1) * gap && aa <= static_cast<float>(POL_TAU2) * gap) work = false;
  }
  rotated = work;
  del = make_float2(0.f, 0.f);
  if (!work) return make_float2(1.f, 0.f);
  const float theta = __fdividef(gd.x, 2.f * apq);
  const float t = __fdividef(theta >= 0.f ? 1.f : -1.f, fabsf(theta) + sqrt_approx(fmaf(theta, theta, 1.f)));
  const float x = fmaf(t, t, 1.f);
  float y = rsqrtf(x);
  y = y * fmaf(-0.5f * x * y, y, 1.5f);
  y = y * fmaf(-0.5f * x * y, y, 1.5f);
  del = df_prod(t, apq);
  return make_float2(y, t * y);
}

// MIXED = false: the FP32 solve of C (eigenvectors through the log; info[4] = sweeps).
// MIXED = true: the polish of the nearly diagonal C1 = W^T C W - its diagonal in FP64 (moved
// with the matrix, by position), the off-diagonal part in FP32, a rotated pair's block set
// to zero; on return lam (descending), sig = sqrt(lam), rank[j] = the place of index j in
// that order, info[3] = sweeps. Both: info[5] = rounds made (the log's length).
template <bool MIXED>
__global__ void __launch_bounds__(EIG2_T) jacobi_circle_kernel(const double* __restrict__ C, float2* __restrict__ rlog,
                                                               int* __restrict__ info, int L, double* __restrict__ lam,
                                                               double* __restrict__ sig, int* __restrict__ rank) {
  extern __shared__ float e2[];
  __shared__ float red[2 * (EIG2_T / 32)];
  __shared__ double scale;
  __shared__ float2 rot[2][EIG2_MAXR / 2];   // by round parity: (c, s) of each pair
  __shared__ float2 rdel[2][EIG2_MAXR / 2];  // MIXED, by round parity: t a_pq of each pair (double-float)
  __shared__ float2 dgs[2][EIG2_MAXR];       // MIXED, by round parity: the diagonal by position (double-float)
  __shared__ int rflag[2];                   // by round parity: any rotation in that round
  __shared__ int needed;
  const int r = info[0];
  const int de = r + (r & 1), np = de >> 1, m = de - 1, lda = de + 1, dd = de * lda, npl = np * lda;
  int* pn = reinterpret_cast<int*>(e2 + 2 * dd);   // position after one round
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid < 32) {   // scaled by a power of two so that the largest diagonal entry is in [1, 2)
    double dm = 0.0;
    for (int i = tid; i < r; i += 32) dm = fmax(dm, fabs(C[i * L + i]));
    for (int o = 16; o > 0; o >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
    if (tid == 0) scale = pow2_scale(dm);
  }
  __syncthreads();
  const double sc = scale;
  for (int i = warp; i < de; i += EIG2_T / 32)
    for (int j = lane; j < de; j += 32) {
      const bool in = i < r && j < r && (!MIXED || i != j);
      e2[i * lda + j] = in ? static_cast<float>(sc * C[i * L + j]) : 0.f;
    }
  if (MIXED)
    for (int i = tid; i < de; i += blockDim.x) {
      const double v = i < r ? sc * C[i * L + i] : 0.0;
      const float hi = static_cast<float>(v);
      dgs[0][i] = make_float2(hi, static_cast<float>(v - static_cast<double>(hi)));
    }
  for (int p = tid; p < de; p += blockDim.x) pn[p] = circ_move(p, 1, np);
  __syncthreads();
  const float eps2 = 3e-8f * 3e-8f;
  // the update threads' blocks (a, b), a <= b: the triangle of pairs folded into nf / 2 rows
  // of nf + 1 (nf = np rounded up to even), taken in order; offsets fixed for the whole solve
  int u_ab[EIG2_MAXK], u_src[EIG2_MAXK], u_d0[EIG2_MAXK], u_d1[EIG2_MAXK], u_m0[EIG2_MAXK], u_m1[EIG2_MAXK];
  // the rotation warp's: the next round's pair j = lane + 32 h holds the indices now at
  // positions px (top) and py (bottom), of this round's pairs al and be
  int w_ofs[2][3], w_pair[2];
  if (warp < EIG2_RW) {
    const int nf = np + (np & 1), fcols = nf + 1, items = (nf >> 1) * fcols;
#pragma unroll
    for (int k = 0; k < EIG2_MAXK; ++k) {
      const int it = tid + k * EIG2_NU;
      u_ab[k] = -1;
      if (it < items) {
        const int fr = it / fcols, fc = it - fr * fcols;
        int pa, pb;
        if (fc < nf - fr) {
          pa = fr;
          pb = fr + fc;
        } else {
          pa = nf - 1 - fr;
          pb = pa + fc - (nf - fr);
        }
        if (pb < np) {
          const int Pa = pn[pa] * lda, Pna = pn[np + pa] * lda, Pb = pn[pb], Pnb = pn[np + pb];
          const int Ra = pn[pa], Rna = pn[np + pa], Rb = pn[pb] * lda, Rnb = pn[np + pb] * lda;
          u_ab[k] = pa | (pb << 8);
          u_src[k] = pa * lda + pb;
          u_d0[k] = (Pa + Pb) | ((Pa + Pnb) << 16);     // o00, o01 in place
          u_d1[k] = (Pna + Pb) | ((Pna + Pnb) << 16);   // o10, o11 in place
          u_m0[k] = (Rb + Ra) | ((Rnb + Ra) << 16);     // o00, o01 mirrored
          u_m1[k] = (Rb + Rna) | ((Rnb + Rna) << 16);   // o10, o11 mirrored
        }
      }
    }
  } else {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = lane + 32 * h;
      const int px = j < np ? circ_move(j, -1, np) : 0, py = j < np ? circ_move(np + j, -1, np) : np;
      const int al = px < np ? px : px - np, be = py < np ? py : py - np;
      const int rx = px < np ? 0 : 1, ry = py < np ? 0 : 1;
      const int lo = al < be ? al : be, hi = al < be ? be : al;
      w_ofs[h][0] = al * lda + al;
      w_ofs[h][1] = be * lda + be;
      w_ofs[h][2] = lo * lda + hi;
      // the stored a_pq is entry (rx, ry) of block (al, be), or (ry, rx) of its mirror (be,
      // al); with one pair only (al == be, r <= 2) it is entry (0, 1) of that pair's block
      const int iu = al < be ? rx : (al > be ? ry : 0), ju = al < be ? ry : (al > be ? rx : 1);
      w_pair[h] = al | (be << 8) | (rx << 16) | (ry << 17) | (iu << 18) | (ju << 19) | ((al < be ? 1 : 0) << 20) |
                  ((al == be ? 1 : 0) << 21);
    }
    bool any = false;   // the first round's rotations, from the pairs (i, np + i) as they stand
    for (int j = lane; j < np; j += 32) {
      bool rt;
      float2 cs;
      if (MIXED) {
        float2 del;
        cs = mixed_rotation(dgs[0][j], dgs[0][np + j], e2[j * lda + np + j], del, rt);
        rdel[0][j] = del;
      } else {
        cs = eig2_rotation(e2[j * lda + j], e2[(np + j) * lda + np + j], e2[j * lda + np + j], eps2, rt);
      }
      rot[0][j] = cs;
      rlog[j] = cs;
      any |= rt;
    }
    any = __any_sync(0xffffffffu, any);
    if (lane == 0) rflag[0] = any ? 1 : 0;
  }
  __syncthreads();
#ifdef SPCA_FIN_TRACE
  const long long t0 = clock64();
#endif
  int g = 0;   // rounds made: the parity picks the buffers
  int sweep = 0;
  for (; sweep < EIG2_SWEEPS && r > 1; ++sweep) {
    const float* Ac = e2 + (g & 1) * dd;   // positions are the identity between sweeps
    float off = 0.f, tot = 0.f;
    for (int i = warp; i < de; i += EIG2_T / 32)
      for (int j = lane; j < de; j += 32) {
        const float v = Ac[i * lda + j];
        tot = fmaf(v, v, tot);
        if (i != j) off = fmaf(v, v, off);
      }
    if (MIXED) {   // sums in FP32 (norms; FP64 instructions issued by every thread are slow here)
      const float2* dg = dgs[g & 1];
      for (int i = tid; i < de; i += blockDim.x) tot = fmaf(dg[i].x, dg[i].x, tot);
      blk_sum2(off, tot, red);
      if (off <= 1e-26f * tot || tot == 0.f) break;   // tot: the off-diagonal part and the diagonal
      // look at every pair at once (FP32 estimates) and stop if none needs a rotation
      if (tid == 0) needed = 0;
      __syncthreads();
      for (int i = warp; i < r; i += EIG2_T / 32) {
        const float ai = dg[i].x;
        for (int j = i + 1 + lane; j < r; j += 32) {
          const float aa = fabsf(Ac[i * lda + j]), aj = dg[j].x;
          const float gap = fabsf(aj - ai), mn = fminf(fabsf(ai), fabsf(aj));
          const bool work = aa > 1e-18f * sqrtf(fabsf(ai)) * sqrtf(fabsf(aj)) &&
                            !(aa * aa <= static_cast<float>(POL_TAU1) * mn * gap &&
                              aa <= static_cast<float>(POL_TAU2) * gap);
          if (work) needed = 1;
        }
      }
      __syncthreads();
      if (!needed) break;
    } else {
      blk_sum2(off, tot, red);
      if (off <= 1e-10f * tot || tot == 0.f) break;
    }
    bool any_sweep = false;
    for (int t = 0; t < m; ++t, ++g) {
      const float* A = e2 + (g & 1) * dd;
      float* An = e2 + ((g + 1) & 1) * dd;
      const float2* ro = rot[g & 1];
      const bool any = rflag[g & 1] != 0;
      any_sweep |= any;
      if (warp == EIG2_RW) {
        bool anyn = false;
        float2* lg = rlog + static_cast<size_t>(g + 1) * np;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int j = lane + 32 * h;
          if (j < np) {
            const int wp = w_pair[h], al = wp & 0xff, be = (wp >> 8) & 0xff;
            const bool rx = (wp >> 16) & 1, ry = (wp >> 17) & 1, alo = (wp >> 20) & 1;
            const float2 ra = ro[al], rb = ro[be];
            float apq = rot_entry(A + w_ofs[h][2], np, npl, (wp >> 18) & 1, (wp >> 19) & 1, alo ? ra : rb, alo ? rb : ra);
            if ((wp >> 21) & 1) apq = ra.y != 0.f ? 0.f : apq;   // one pair only: zeroed if rotated
            bool rt;
            float2 cs;
            if (MIXED) {
              const float2* dg = dgs[g & 1];
              const float2 da = rdel[g & 1][al], db = rdel[g & 1][be];
              const float2 app = df_add(dg[al + rx * np], rx ? da : df_neg(da));
              const float2 aqq = df_add(dg[be + ry * np], ry ? db : df_neg(db));
              float2 del;
              cs = mixed_rotation(app, aqq, apq, del, rt);
              rdel[(g + 1) & 1][j] = del;
              dgs[(g + 1) & 1][j] = app;
              dgs[(g + 1) & 1][np + j] = aqq;
            } else {
              const float app = rot_entry(A + w_ofs[h][0], np, npl, rx, rx, ra, ra);
              const float aqq = rot_entry(A + w_ofs[h][1], np, npl, ry, ry, rb, rb);
              cs = eig2_rotation(app, aqq, apq, eps2, rt);
            }
            rot[(g + 1) & 1][j] = cs;
            lg[j] = cs;
            anyn |= rt;
          }
        }
        anyn = __any_sync(0xffffffffu, anyn);
        if (lane == 0) rflag[(g + 1) & 1] = anyn ? 1 : 0;
      } else {
#pragma unroll
        for (int k = 0; k < EIG2_MAXK; ++k) {
          if (u_ab[k] < 0) continue;
          const int pa = u_ab[k] & 0xff, pb = u_ab[k] >> 8;
          const float2 ra = ro[pa], rb = ro[pb];
          const float* M = A + u_src[k];
          float o00, o01, o10, o11;
          rot_block(M[0], M[np], M[npl], M[npl + np], ra.x, ra.y, rb.x, rb.y, o00, o01, o10, o11);
          if (pa == pb) {   // the pair's own block: symmetric, its off-diagonal entry zeroed if rotated
            if (ra.y != 0.f) {
              o01 = 0.f;
              if (MIXED) {   // the diagonal lives in FP64 outside this matrix
                o00 = 0.f;
                o11 = 0.f;
              }
            }
            o10 = o01;
          }
          An[u_d0[k] & 0xffff] = o00;
          An[u_d0[k] >> 16] = o01;
          An[u_d1[k] & 0xffff] = o10;
          An[u_d1[k] >> 16] = o11;
          An[u_m0[k] & 0xffff] = o00;
          An[u_m0[k] >> 16] = o01;
          An[u_m1[k] & 0xffff] = o10;
          An[u_m1[k] >> 16] = o11;
        }
      }
      __syncthreads();
    }
    if (!any_sweep) {
      ++sweep;
      break;
    }
  }
#ifdef SPCA_FIN_TRACE
  if (tid == 0)
    printf("%s d=%d sweeps=%d rounds=%d cycles=%lld\n", MIXED ? "polish_circle" : "eig_f32_circle", r, sweep, g,
           clock64() - t0);
#endif
  if (MIXED) {   // eigenvalues by descending value, ties by index
    const float2* dg = dgs[g & 1];
    for (int i = tid; i < r; i += blockDim.x) {   // compared as (hi, lo) pairs: normalised, so in order
      int rk = 0;
      const float2 vi = dg[i];
      for (int j = 0; j < r; ++j) {
        const float2 u = dg[j];
        if (u.x > vi.x || (u.x == vi.x && (u.y > vi.y || (u.y == vi.y && j < i)))) ++rk;
      }
      const double v = static_cast<double>(vi.x) + static_cast<double>(vi.y);
      lam[rk] = v / sc;
      sig[rk] = sqrt(fmax(v / sc, 0.0));
      rank[i] = rk;
    }
    for (int i = r + tid; i < L; i += blockDim.x) sig[i] = 0.0;
  }
  if (tid == 0) {
    info[MIXED ? 3 : 4] = sweep;
    info[5] = g;
  }
}

// W0 (L x L, zero outside r x r) = the product of the logged rotations, applied in order to
// the rows of the identity, one warp per row; with `rank` its columns are put in that order.
// A row is kept by position, like the matrix of the solve: lane b holds positions b and
// np + b (and b + 32, np + b + 32 when np > 32) in registers, rotates them with its pair's
// logged rotation and passes them one step along the circle with shuffles; after whole
// sweeps the positions are the indices again. The log is staged in shared memory a chunk of
// rounds at a time, the next chunk loading (cp.async) while the current one is applied.
constexpr int RPL_W = 4;      // warps (rows) per block
constexpr int RPL_RC = 48;    // rounds per chunk

__host__ __device__ inline size_t replay_smem(int l) {
  const size_t de = static_cast<size_t>(l + (l & 1));
  return sizeof(float2) * 2 * RPL_RC * (de / 2);
}

__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(sdst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void rot_pair(float2 cs, float& t, float& b) {
  const float x = t, y = b;
  t = cs.x * x - cs.y * y;
  b = cs.y * x + cs.x * y;
}

__global__ void __launch_bounds__(RPL_W * 32) eig_replay_kernel(const float2* __restrict__ rlog,
                                                               const int* __restrict__ info, int L,
                                                               const int* __restrict__ rank,
                                                               double* __restrict__ W0) {
  extern __shared__ float2 rp[];
  const int r = info[0], G = info[5];
  const int de = r + (r & 1), np = de >> 1;
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * RPL_W + (threadIdx.x >> 5);
  const bool live = i < r;
  const unsigned full = 0xffffffffu;
  // T0, B0: positions lane, np + lane; T1, B1: positions 32 + lane, np + 32 + lane
  float T0 = (lane == i) ? 1.f : 0.f, B0 = (np + lane == i) ? 1.f : 0.f;
  float T1 = (32 + lane == i) ? 1.f : 0.f, B1 = (np + 32 + lane == i) ? 1.f : 0.f;
  const bool two = np > 32;
  const int nchunks = (G + RPL_RC - 1) / RPL_RC;
  auto load = [&](int c) {
    float2* dst = rp + (c & 1) * RPL_RC * np;
    const int g0 = c * RPL_RC, n = min(RPL_RC, G - g0) * np;
    for (int e = threadIdx.x; e < n; e += blockDim.x) cp_async8(dst + e, rlog + static_cast<size_t>(g0) * np + e);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  if (nchunks > 0) load(0);
  for (int c = 0; c < nchunks; ++c) {
    if (c + 1 < nchunks) {
      load(c + 1);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();
    const float2* ck = rp + (c & 1) * RPL_RC * np;
    const int n = min(RPL_RC, G - c * RPL_RC);
    if (live) {
      for (int gg = 0; gg < n; ++gg) {
        const float2* cr = ck + gg * np;
        if (lane < np) rot_pair(cr[lane], T0, B0);
        if (two && 32 + lane < np) rot_pair(cr[32 + lane], T1, B1);
        if (np == 1) continue;   // one pair: the circle is a single position
        // one step along the circle: top p -> p + 1 (p >= 1), top np-1 -> bottom np-1,
        // bottom q -> q - 1 (q >= 1), bottom 0 -> top 1, top 0 stays
        const float t0u = __shfl_up_sync(full, T0, 1), t1u = __shfl_up_sync(full, T1, 1);
        const float b0d = __shfl_down_sync(full, B0, 1), b1d = __shfl_down_sync(full, B1, 1);
        const float t0l = __shfl_sync(full, T0, 31), b0f = __shfl_sync(full, B0, 0), b1f = __shfl_sync(full, B1, 0);
        const float nT0 = lane == 0 ? T0 : (lane == 1 ? b0f : t0u);
        const float nT1 = lane == 0 ? t0l : t1u;
        float nB0 = lane == 31 ? b1f : b0d;
        float nB1 = b1d;
        if (lane == np - 1) nB0 = T0;
        if (32 + lane == np - 1) nB1 = T1;
        T0 = nT0;
        T1 = nT1;
        B0 = nB0;
        B1 = nB1;
      }
    }
    __syncthreads();   // the buffer is reloaded two chunks on
  }
  if (i < L) {   // position p = index p again; column j of the product goes to column rank[j]
    double* row = W0 + static_cast<size_t>(i) * L;
    for (int j = lane; j < L; j += 32) row[j] = 0.0;
    __syncwarp();
    if (live) {
      const float v[4] = {T0, B0, T1, B1};
      const int pos[4] = {lane, np + lane, 32 + lane, np + 32 + lane};
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int j = pos[h];
        const bool mine = (h & 1) ? (lane + (h >> 1) * 32 < np) : (lane + (h >> 1) * 32 < np);
        if (mine && j < r) row[rank ? rank[j] : j] = static_cast<double>(v[h]);
      }
    }
  }
}

// Out = alpha op(A) op(B) + beta D on the leading r x r block (ld L, zero elsewhere), with
// r = *rdev when rdev is given, else rhost; one block per row, FP64. Row i of op(A) is
// staged in shared memory, and op(B) too when `stage` is set (as r rows of odd stride, by
// asynchronous copies). D may be NULL.
constexpr int GEMM_T = 128;
constexpr size_t kGemmSmemMax = 200 * 1024;
__global__ void __launch_bounds__(GEMM_T) small_gemm_kernel(const double* __restrict__ A, int ta,
                                                            const double* __restrict__ B, int tb,
                                                            const double* __restrict__ D, double alpha, double beta,
                                                            const int* __restrict__ rdev, int rhost, int L,
                                                            int stage, double* __restrict__ Out) {
  extern __shared__ double gsm[];
  __shared__ double part[GEMM_T];
  double* sa = gsm;           // r: row i of op(A)
  double* sb = gsm + kMaxL;   // op(B)[t][j] at sb[t * ldb + j], ldb odd (column writes spread over banks)
  const int r = rdev ? *rdev : rhost;
  const int ldb = r | 1;
  const int i = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = GEMM_T / 32;
  if (i < r) {   // asynchronous copies, all in flight at once
    for (int t = threadIdx.x; t < r; t += blockDim.x) cp_async8(sa + t, ta ? A + t * L + i : A + i * L + t);
    if (stage) {   // a warp per row of B as stored (coalesced), lanes along it
      for (int u = warp; u < r; u += nw)
        for (int v = lane; v < r; v += 32) cp_async8(tb ? sb + v * ldb + u : sb + u * ldb + v, B + u * L + v);
    }
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  if (stage && r <= GEMM_T / 2) {   // two threads per output, each over half of t, two accumulators each
    const int j = threadIdx.x % (GEMM_T / 2), h = threadIdx.x / (GEMM_T / 2);
    const int t0 = h * (r >> 1), t1 = h ? r : (r >> 1);
    double acc0 = 0.0, acc1 = 0.0;
    if (i < r && j < r) {
      int t = t0;
      for (; t + 1 < t1; t += 2) {
        acc0 = fma(sa[t], sb[t * ldb + j], acc0);
        acc1 = fma(sa[t + 1], sb[(t + 1) * ldb + j], acc1);
      }
      if (t < t1) acc0 = fma(sa[t], sb[t * ldb + j], acc0);
    }
    part[threadIdx.x] = acc0 + acc1;
    __syncthreads();
    for (int jj = threadIdx.x; jj < L; jj += blockDim.x) {
      double acc = 0.0;
      if (i < r && jj < r) {
        acc = alpha * (part[jj] + part[jj + GEMM_T / 2]);
        if (D) acc = fma(beta, D[i * L + jj], acc);
      }
      Out[i * L + jj] = acc;
    }
    return;
  }
  for (int j = threadIdx.x; j < L; j += blockDim.x) {
    double acc = 0.0;
    if (i < r && j < r) {
      double acc1 = 0.0;
      if (stage) {
        int t = 0;
        for (; t + 1 < r; t += 2) {
          acc = fma(sa[t], sb[t * ldb + j], acc);
          acc1 = fma(sa[t + 1], sb[(t + 1) * ldb + j], acc1);
        }
        if (t < r) acc = fma(sa[t], sb[t * ldb + j], acc);
      } else {
        for (int t = 0; t < r; ++t) acc = fma(sa[t], tb ? B[j * L + t] : B[t * L + j], acc);
      }
      acc = alpha * (acc + acc1);
      if (D) acc = fma(beta, D[i * L + j], acc);
    }
    Out[i * L + j] = acc;
  }
}

__global__ void __launch_bounds__(POL_T) eig_polish_kernel(const double* __restrict__ C1, float* __restrict__ Eg,
                                                           float* __restrict__ Wg, double* __restrict__ W1,
                                                           double* __restrict__ lam, double* __restrict__ sig,
                                                           int* __restrict__ info, int L, int smem) {
  extern __shared__ float p32[];
  __shared__ double red[kMaxL];
  __shared__ double dg[kMaxL];
  __shared__ double scale;
  const int r = info[0];
  const int ld = smem ? (r | 1) : L;   // odd: columns of a row fall in different banks
  float* E = smem ? p32 : Eg;
  float* W = smem ? p32 + r * ld : Wg;
  if (threadIdx.x < 32) {   // C1 scaled by a power of two (exact), undone on lam
    double dm = 0.0;
    for (int i = threadIdx.x; i < r; i += 32) dm = fmax(dm, fabs(C1[i * L + i]));
    for (int o = 16; o > 0; o >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
    if (threadIdx.x == 0) scale = pow2_scale(dm);
  }
  __syncthreads();
  const double sc = scale;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e - i * r;
    const double v = sc * C1[i * L + j];
    if (i == j) dg[i] = v;
    E[i * ld + j] = i == j ? 0.f : static_cast<float>(v);
  }
  __syncthreads();
  int sweeps = 0;
#ifdef SPCA_FIN_TRACE
  const long long t0 = clock64();
#endif
  if (r > 0) sweeps = jacobi_mixed(dg, E, W, lam, r, ld, red, 1e-26, 1e-18, 1e-8, 1e-6, 40);
#ifdef SPCA_FIN_TRACE
  if (threadIdx.x == 0) printf("eig_polish d=%d threads=%d sweeps=%d cycles=%lld\n", r, blockDim.x, sweeps, clock64() - t0);
#endif
  for (int i = threadIdx.x; i < r; i += blockDim.x) lam[i] /= sc;
  __syncthreads();
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
    const int i = e / L, j = e % L;
    W1[e] = (i < r && j < r) ? static_cast<double>(W[i * ld + j]) : 0.0;
  }
  for (int i = threadIdx.x; i < L; i += blockDim.x) sig[i] = (i < r) ? sqrt(fmax(lam[i], 0.0)) : 0.0;
  if (threadIdx.x == 0) info[3] = sweeps;
}

// Mixed-precision route to T = R^-T (step 2), for GPUs whose FP64 rate is a small fraction
// of FP32: Cholesky factors and their inverses are taken in FP32, and every product with
// gram_bar in FP64. With Y1 = chol32(gram_bar)^-1, X1 = Y1 gram_bar Y1^T is within about
// eps_32 cond(gram_bar) of I; with T2 = chol32(X1)^-1 Y1, X2 = T2 gram_bar T2^T = I + E,
// |E| ~ eps_32; the first-order Cholesky factor of I + E is I + F, F = strict_lower(E) +
// diag(E) / 2, so T = (I - F) T2 leaves T gram_bar T^T = I + O(|E|^2).
//
// chol_inv_f32_kernel: Y = inverse of the FP32 Cholesky factor of the leading l x l block of
// M (FP64 in and out, ld L, zero outside). A pivot <= tol_rel * max diag, rank_ok == 0 or a
// non-finite entry sets info[6] (the FP64 fallback then runs); `first` clears it first.
__global__ void __launch_bounds__(POL_T) chol_inv_f32_kernel(const double* __restrict__ M, int l, int L,
                                                             double tol_rel, int rank_ok, int first,
                                                             float* __restrict__ Xg, float* __restrict__ Yg,
                                                             double* __restrict__ Y, int* __restrict__ info, int smem) {
  extern __shared__ float c32[];
  __shared__ float wmax[POL_T / 32];
  const int ld = smem ? l : L;
  float* X = smem ? c32 : Xg;
  float* Yf = smem ? c32 + l * l : Yg;
  float dm = 0.f;
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int i = e / l, j = e - i * l;
    const float v = static_cast<float>(M[i * L + j]);
    X[i * ld + j] = v;
    if (i == j) dm = fmaxf(dm, fabsf(v));
  }
  for (int o = 16; o > 0; o >>= 1) dm = fmaxf(dm, __shfl_xor_sync(0xffffffffu, dm, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = dm;
  __syncthreads();
  dm = 0.f;
  for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) dm = fmaxf(dm, wmax[w]);
  const float tol = static_cast<float>(tol_rel) * dm;
  const int tri = l * (l + 1) / 2, cap = static_cast<int>(blockDim.x);
  bool ok = rank_ok && dm > 0.f && isfinite(dm);
  if (ok) {   // the register-resident elimination where the triangle fits the block's registers
    if (tri <= 4 * cap) ok = blk_chol_inv32_reg<4>(X, Yf, l, ld, tol);
    else if (tri <= 8 * cap) ok = blk_chol_inv32_reg<8>(X, Yf, l, ld, tol);
    else if (tri <= 17 * cap) ok = blk_chol_inv32_reg<17>(X, Yf, l, ld, tol);
    else ok = blk_chol_inv32(X, Yf, l, ld, tol);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
    const int i = e / L, j = e % L;
    Y[e] = (ok && i < l && j < l) ? static_cast<double>(Yf[i * ld + j]) : 0.0;
  }
  if (threadIdx.x == 0) {
    if (first) info[6] = 0;
    if (!ok) info[6] = 1;
  }
}

// F = strict_lower(X2) + (diag(X2) - 1) / 2 on the leading l x l block; on success of the
// mixed route also records info = {l, route 0, 0 sweeps}.
__global__ void chol_first_order_kernel(const double* __restrict__ X2, int l, int L, double* __restrict__ F,
                                        int* __restrict__ info) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < L * L; e += gridDim.x * blockDim.x) {
    const int i = e / L, j = e % L;
    double v = 0.0;
    if (i < l && j < l) v = i > j ? X2[e] : (i == j ? 0.5 * (X2[e] - 1.0) : 0.0);
    F[e] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && info[6] == 0) {
    info[0] = l;
    info[1] = 0;
    info[2] = 0;
  }
}

int grid_for(int64_t total, int threads) {
  int64_t b = (total + threads - 1) / threads;
  if (b > 152 * 16) b = 152 * 16;
  return static_cast<int>(b < 1 ? 1 : b);
}

constexpr size_t kMaxDenseSmem = 200 * 1024;

}  // namespace

cudaError_t centered_state(const State& s, const FinalWork& f, int64_t m, cudaStream_t st) {
  const double inv_m = m > 0 ? 1.0 / static_cast<double>(m) : 0.0;
  center_h_kernel<<<grid_for(s.n * s.L, 256), 256, 0, st>>>(s.H, s.colsum, s.sG, s.n, s.l, s.L, inv_m, f.Hbar);
  center_gram_kernel<<<(s.L * s.L + 255) / 256, 256, 0, st>>>(s.gram, s.sG, s.l, s.L, inv_m, f.gbar);
  return cudaGetLastError();
}

// The dynamic shared memory limits of the one-block dense kernels, set once per process.
void set_dense_attrs() {
  static std::atomic<uint64_t> done{0};
  static std::mutex mu;
  once_per_device(done, mu, [] {
    cudaFuncSetAttribute(factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kMaxDenseSmem));
    cudaFuncSetAttribute(chol_inv_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(kMaxDenseSmem));
    cudaFuncSetAttribute(small_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(kGemmSmemMax));
    cudaFuncSetAttribute(eig_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kMaxDenseSmem));
    cudaFuncSetAttribute(jacobi_circle_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(eig2_smem(EIG2_MAXR)));
    cudaFuncSetAttribute(jacobi_circle_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(eig2_smem(EIG2_MAXR)));
    cudaFuncSetAttribute(eig_replay_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(replay_smem(EIG2_MAXR)));
    cudaFuncSetAttribute(eig_polish_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(kMaxDenseSmem));
    cudaFuncSetAttribute(bt_and_c_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(kMaxDenseSmem));
    cudaFuncSetAttribute(form_v_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(kMaxDenseSmem));
    cudaFuncSetAttribute(form_v_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(kMaxDenseSmem));
    return cudaGetLastError();
  });
}

cudaError_t finalize_run(const State& s, const FinalWork& f, int64_t m, int k, double* sigma_dev, double* V_dev,
                         cudaStream_t st, Prof* prof, int64_t rows_seen, bool centered) {
  set_dense_attrs();
  prof->begin(SPCA_K_FINALIZE, st);
  cudaError_t e = centered_state(s, f, m, st);
  if (e != cudaSuccess) return e;
  // rank bound: a centred Gram of m rows has rank <= m - 1, an uncentred one <= m
  int64_t r_max = centered ? rows_seen - 1 : rows_seen;
  if (r_max > s.l) r_max = s.l;
  if (r_max < 0) r_max = 0;
  const int64_t LL = static_cast<int64_t>(s.L) * s.L;
  float* s32 = reinterpret_cast<float*>(f.Cpart);   // FP32 scratch when l x l does not fit in shared memory
  const size_t dense32 = 2 * sizeof(float) * s.l * s.l;   // Cholesky: X, Y
  const int smem32 = dense32 <= kMaxDenseSmem ? 1 : 0;
  size_t dense32e = 3 * sizeof(float) * s.l * (s.l | 1);  // FP32 Jacobi: A, A2, W
  int smem32e = 1;
  if (dense32e > kMaxDenseSmem) {   // A and W only, rotated in place
    dense32e = 2 * sizeof(float) * s.l * (s.l | 1);
    smem32e = dense32e <= kMaxDenseSmem ? 2 : 0;
  }
  const int l = s.l, L = s.L;
  const int rank_ok = r_max >= l ? 1 : 0;
  const size_t gemm_full = sizeof(double) * (kMaxL + static_cast<size_t>(l) * (l | 1));
  const int gstage = gemm_full <= kGemmSmemMax ? 1 : 0;
  const size_t gemm_smem = gstage ? gemm_full : sizeof(double) * kMaxL;
  // mixed-precision route (buffers: Y1 W, X1 T, Y2 X, T2 C, X2 W, F X, T T)
  const dim3 gb(L), gt(GEMM_T);
  chol_inv_f32_kernel<<<1, POL_T, smem32 ? dense32 : 0, st>>>(f.gbar, l, L, l * 1.2e-7, rank_ok, 1, s32, s32 + LL, f.W,
                                                            f.info, smem32);
  // X1 = Y1 (gram Y1^T)
  small_gemm_kernel<<<gb, gt, gemm_smem, st>>>(f.gbar, 0, f.W, 1, nullptr, 1.0, 0.0, nullptr, l, L, gstage, f.X);
  small_gemm_kernel<<<gb, gt, gemm_smem, st>>>(f.W, 0, f.X, 0, nullptr, 1.0, 0.0, nullptr, l, L, gstage, f.T);
  chol_inv_f32_kernel<<<1, POL_T, smem32 ? dense32 : 0, st>>>(f.T, l, L, l * 1.2e-7, 1, 0, s32, s32 + LL, f.X, f.info,
                                                            smem32);
  // T2 = Y2 Y1; X2 = T2 (gram T2^T); T = T2 - F T2
  small_gemm_kernel<<<gb, gt, gemm_smem, st>>>(f.X, 0, f.W, 0, nullptr, 1.0, 0.0, nullptr, l, L, gstage, f.C);
  small_gemm_kernel<<<gb, gt, gemm_smem, st>>>(f.gbar, 0, f.C, 1, nullptr, 1.0, 0.0, nullptr, l, L, gstage, f.X);
  small_gemm_kernel<<<gb, gt, gemm_smem, st>>>(f.C, 0, f.X, 0, nullptr, 1.0, 0.0, nullptr, l, L, gstage, f.W);
  chol_first_order_kernel<<<(L * L + 255) / 256, 256, 0, st>>>(f.W, l, L, f.X, f.info);
  small_gemm_kernel<<<gb, gt, gemm_smem, st>>>(f.X, 0, f.C, 0, f.C, -1.0, 1.0, nullptr, l, L, gstage, f.T);
  // FP64 fallback (returns at once unless the mixed route failed)
  const size_t dense3 = 3 * sizeof(double) * s.l * s.l;
  const int factor_smem = dense3 <= kMaxDenseSmem ? 1 : 0;
  factor_kernel<<<1, FT, factor_smem ? dense3 : 0, st>>>(f.gbar, s.l, s.L, static_cast<int>(r_max), f.T, f.X, f.W,
                                                         f.lam, f.info, factor_smem);
  const size_t dense64 = 2 * sizeof(float) * s.l * (s.l | 1);   // polish: E, W (FP32)
  const int smem64 = dense64 <= kMaxDenseSmem ? 1 : 0;
  const int64_t nblk = (s.n + BT_ROWS - 1) / BT_ROWS;
  const int parts = static_cast<int>(nblk < f.nparts ? nblk : f.nparts);
  // T^T staged in shared memory whole when it fits, else 32 of its columns at a time
  const size_t bt_base = 2 * sizeof(double) * BT_ROWS * s.L;
  const int tcc = bt_base + sizeof(double) * s.L * s.l <= kMaxDenseSmem ? s.l : 32;
  bt_and_c_kernel<<<parts, 256, bt_base + sizeof(double) * s.L * tcc, st>>>(f.Hbar, f.T, f.info, s.n, s.l, s.L, tcc,
                                                                            f.Bt, f.Cpart);
  c_reduce_kernel<<<(s.L * s.L + 31) / 32, CR_T, 0, st>>>(f.Cpart, parts, s.L, f.C);
  // T (= R^-T) is scratch below; the map to U keeps a copy
  e = cudaMemcpyAsync(f.Tu, f.T, sizeof(double) * LL, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  // eigenvectors of C: FP32 Jacobi, FP64 orthogonalisation and polish (scratch: Cpart, whose
  // partials are consumed by now, and T, X, W)
  float* s64 = reinterpret_cast<float*>(f.Cpart + 2 * LL);   // E, W of the polish: 2 L^2 floats
  double* W1 = f.Cpart + 3 * LL;
  // the rotation log of the fast solver sits in Cpart after the polish's scratch
  float2* rlog = reinterpret_cast<float2*>(f.Cpart + 4 * LL);
  const bool fast_eig = s.l <= EIG2_MAXR && sizeof(double) * static_cast<size_t>(f.nparts - 4) * LL >=
                                               sizeof(float2) * eig2_log_len(s.l);
  const int rpl_grid = (L + RPL_W - 1) / RPL_W;
  if (fast_eig) {
    jacobi_circle_kernel<false><<<1, EIG2_T, eig2_smem(s.l), st>>>(f.C, rlog, f.info, s.L, nullptr, nullptr, nullptr);
    eig_replay_kernel<<<rpl_grid, RPL_W * 32, replay_smem(s.l), st>>>(rlog, f.info, L, nullptr, f.W);
  } else
    eig_f32_kernel<<<1, EIG_T, smem32e ? dense32e : 0, st>>>(f.C, s32, s32 + LL, s32 + 2 * LL, f.W, f.info, s.L,
                                                            smem32e);
  // Newton-Schulz, twice: W <- 1.5 W - 0.5 W (W^T W)  (W: f.W -> f.T -> f.W)
  small_gemm_kernel<<<gb, gt, gemm_smem, st>>>(f.W, 1, f.W, 0, nullptr, 1.0, 0.0, f.info, 0, s.L, gstage, f.X);
  small_gemm_kernel<<<gb, gt, gemm_smem, st>>>(f.W, 0, f.X, 0, f.W, -0.5, 1.5, f.info, 0, s.L, gstage, f.T);
  small_gemm_kernel<<<gb, gt, gemm_smem, st>>>(f.T, 1, f.T, 0, nullptr, 1.0, 0.0, f.info, 0, s.L, gstage, f.X);
  small_gemm_kernel<<<gb, gt, gemm_smem, st>>>(f.T, 0, f.X, 0, f.T, -0.5, 1.5, f.info, 0, s.L, gstage, f.W);
  // C1 = W^T C W
  small_gemm_kernel<<<gb, gt, gemm_smem, st>>>(f.C, 0, f.W, 0, nullptr, 1.0, 0.0, f.info, 0, s.L, gstage, f.X);
  small_gemm_kernel<<<gb, gt, gemm_smem, st>>>(f.W, 1, f.X, 0, nullptr, 1.0, 0.0, f.info, 0, s.L, gstage, f.T);
  if (fast_eig) {   // the polish's order of the eigenvalues in the scratch of the old polish
    int* rank = reinterpret_cast<int*>(s64);
    jacobi_circle_kernel<true><<<1, EIG2_T, eig2_smem(s.l), st>>>(f.T, rlog, f.info, s.L, f.lam, f.sig, rank);
    eig_replay_kernel<<<rpl_grid, RPL_W * 32, replay_smem(s.l), st>>>(rlog, f.info, L, rank, W1);
  } else {
    eig_polish_kernel<<<1, POL_T, smem64 ? dense64 : 0, st>>>(f.T, s64, s64 + LL, W1, f.lam, f.sig, f.info, s.L,
                                                              smem64);
  }
  // Z = W W1 (into f.X): the eigenvectors of C, used to form V
  small_gemm_kernel<<<gb, gt, gemm_smem, st>>>(f.W, 0, W1, 0, nullptr, 1.0, 0.0, f.info, 0, s.L, gstage, f.X);
  // a block of rows of Bt, 1/sigma and (when it fits) W's leading l x k block in shared
  // memory, sized for r = l, the largest rank
  const size_t fv_base = sizeof(double) * (FV_ROWS * (static_cast<size_t>(l) + 1) + k);
  const size_t fv_full = fv_base + sizeof(double) * static_cast<size_t>(l) * k;
  const int64_t fv_tiles = (s.n + FV_ROWS - 1) / FV_ROWS;
  const int fv_grid = static_cast<int>(fv_tiles < 152 * 2 ? fv_tiles : 152 * 2);
  if (fv_full <= kMaxDenseSmem)
    form_v_kernel<true><<<fv_grid, 256, fv_full, st>>>(f.Bt, f.X, f.sig, f.info, s.n, k, s.L, V_dev);
  else
    form_v_kernel<false><<<fv_grid, 256, fv_base, st>>>(f.Bt, f.X, f.sig, f.info, s.n, k, s.L, V_dev);
  sign_fix_kernel<<<k, SIGN_T, 0, st>>>(V_dev, s.n, f.flip);
  prof->launches[SPCA_K_FINALIZE] += fast_eig ? 26 : 24;  // launches above beyond the one begin() counted (not the copy)
  prof->end(SPCA_K_FINALIZE, st);
  e = cudaMemcpyAsync(sigma_dev, f.sig, sizeof(double) * k, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ the power scheme (P = 1)

// T = the l x l identity (zero elsewhere in L x L); info[0] = l (all output columns of
// bt_and_c), info[6] = 0 (no failed factorisation yet).
__global__ void eye_kernel(double* __restrict__ T, int l, int L, int* __restrict__ info) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < L * L; e += gridDim.x * blockDim.x)
    T[e] = (e / L == e % L && e / L < l) ? 1.0 : 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    info[0] = l;
    info[6] = 0;
  }
}

// One block: C = L1 L1^T (FP64 Cholesky, in place) and T = L1^-1, so that Q = Y T^T has
// orthonormal columns when C = Y^T Y. A pivot at or below l eps max_i C_ii sets info[6].
__global__ void chol_tinv64_kernel(double* __restrict__ C, int l, int L, double* __restrict__ T, int* __restrict__ info) {
  __shared__ double tol;
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int c = 0; c < l; ++c) mx = fmax(mx, C[c * L + c]);
    tol = static_cast<double>(l) * 2.220446049250313e-16 * mx;
  }
  __syncthreads();
  const bool ok = blk_cholesky(C, l, L, tol);
  if (!ok) {
    if (threadIdx.x == 0) info[6] = 1;
    return;
  }
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) T[e] = 0.0;
  __syncthreads();
  blk_trinv_lower(C, T, l, L);
}

cudaError_t power_omega_run(const State& s, const FinalWork& f, int64_t m, cudaStream_t st, const double** Q) {
  set_dense_attrs();
  cudaError_t e = centered_state(s, f, m, st);
  if (e != cudaSuccess) return e;
  const int l = s.l, L = s.L;
  const int64_t nblk = (s.n + BT_ROWS - 1) / BT_ROWS;
  const int parts = static_cast<int>(nblk < f.nparts ? nblk : f.nparts);
  const size_t bt_base = 2 * sizeof(double) * BT_ROWS * L;
  const int tcc = bt_base + sizeof(double) * L * l <= kMaxDenseSmem ? l : 32;
  const size_t bt_smem = bt_base + sizeof(double) * L * tcc;
  const int cr_grid = (L * L + 31) / 32;
  // Q = orth(H_bar) by Cholesky QR twice: C = H^T H = L1 L1^T, Q1 = H L1^-T; then again on Q1
  eye_kernel<<<(L * L + 255) / 256, 256, 0, st>>>(f.T, l, L, f.info);
  bt_and_c_kernel<<<parts, 256, bt_smem, st>>>(f.Hbar, f.T, f.info, s.n, l, L, tcc, f.Bt, f.Cpart);
  c_reduce_kernel<<<cr_grid, CR_T, 0, st>>>(f.Cpart, parts, L, f.C);
  chol_tinv64_kernel<<<1, 256, 0, st>>>(f.C, l, L, f.T, f.info);
  bt_and_c_kernel<<<parts, 256, bt_smem, st>>>(f.Hbar, f.T, f.info, s.n, l, L, tcc, f.Bt, f.Cpart);
  c_reduce_kernel<<<cr_grid, CR_T, 0, st>>>(f.Cpart, parts, L, f.C);
  chol_tinv64_kernel<<<1, 256, 0, st>>>(f.C, l, L, f.T, f.info);
  bt_and_c_kernel<<<parts, 256, bt_smem, st>>>(f.Bt, f.T, f.info, s.n, l, L, tcc, f.Hbar, f.Cpart);
  *Q = f.Hbar;
  return cudaGetLastError();
}

// After a finalize: W = V Sigma^-1 in FP32 (n x L, zero beyond the rank and past k) for a
// second pass over the rows, and corr = (s_hat / m)^T W in FP64 (from the FP32 W, so that the
// centring term matches the products it corrects; 0 without centring).
__global__ void upass_w_kernel(const double* __restrict__ V, const double* __restrict__ sigma, int64_t n, int k, int L,
                               float* __restrict__ W) {
  __shared__ double inv[kMaxL];   // 1 / sigma_j once per block (FP64 divisions are slow here)
  for (int j = threadIdx.x; j < L; j += blockDim.x) inv[j] = (j < k && sigma[j] > 0.0) ? 1.0 / sigma[j] : 0.0;
  __syncthreads();
  // a thread per (row c, 4 columns): V's columns read coalesced across threads, a float4 of W out
  const int64_t nq = n * (L / 4);
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < nq;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int jq = static_cast<int>(idx / n);
    const int64_t c = idx - static_cast<int64_t>(jq) * n;
    float w[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int j = 4 * jq + t;
      w[t] = j < k ? static_cast<float>(V[static_cast<int64_t>(j) * n + c] * inv[j]) : 0.f;
    }
    *reinterpret_cast<float4*>(W + c * L + 4 * jq) = make_float4(w[0], w[1], w[2], w[3]);
  }
}

__global__ void upass_corr_kernel(const float* __restrict__ W, const double* __restrict__ colsum, int64_t m, int64_t n,
                                  int L, double* __restrict__ corr) {
  __shared__ double red[256];
  const int j = blockIdx.x;
  double acc = 0.0;
  if (m > 0)
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) acc += colsum[c] * static_cast<double>(W[c * L + j]);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) corr[j] = m > 0 ? red[0] / static_cast<double>(m) : 0.0;
}

cudaError_t launch_upass_w(const State& s, const double* V, const double* sigma, int k, float* W, cudaStream_t st) {
  upass_w_kernel<<<grid_for(s.n * (s.L / 4), 256), 256, 0, st>>>(V, sigma, s.n, k, s.L, W);
  return cudaGetLastError();
}

cudaError_t launch_upass_corr(const State& s, const float* W, int64_t m_center, double* corr, cudaStream_t st) {
  upass_corr_kernel<<<s.L, 256, 0, st>>>(W, s.colsum, m_center, s.n, s.L, corr);
  return cudaGetLastError();
}

cudaError_t launch_u_map(const State& s, const FinalWork& f, int k, int64_t m, cudaStream_t st) {
  u_map_kernel<<<k, 64, 0, st>>>(f.Tu, f.X, f.info, f.flip, s.sG, m, s.l, s.L, k, f.M, f.mrow);
  return cudaGetLastError();
}

cudaError_t launch_left_vectors(const State& s, const FinalWork& f, int k, const float* G, int64_t row0, int64_t mc,
                                double* U, int64_t ldu, cudaStream_t st) {
  const int64_t total = mc * k;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  left_vectors_kernel<<<static_cast<int>(blocks), 256, 0, st>>>(G, row0, mc, s.l, k, f.M, f.mrow, U, ldu);
  return cudaGetLastError();
}

}  // namespace spca

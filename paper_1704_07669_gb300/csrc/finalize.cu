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
//     ordering: an FP32 solve, then an FP64 polish of W_B^T C W_B, see
//     eig_f32_kernel); V = B^T W_B diag(1/sigma), the leading k columns
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
// partial C_p = sum_j Bt[j]^T Bt[j] of this block (lower triangle, ld L).
__global__ void __launch_bounds__(256) bt_and_c_kernel(const double* __restrict__ Hbar, const double* __restrict__ T,
                                                       const int* __restrict__ info, int64_t n, int l, int L,
                                                       double* __restrict__ Bt, double* __restrict__ Cpart) {
  extern __shared__ double sm[];
  double* sH = sm;                  // BT_ROWS x L
  double* sB = sm + BT_ROWS * L;    // BT_ROWS x L
  const int r = info[0];
  double* out = Cpart + static_cast<int64_t>(blockIdx.x) * L * L;
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) out[e] = 0.0;
  const int64_t nblk = (n + BT_ROWS - 1) / BT_ROWS;
  for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const int64_t j0 = blk * BT_ROWS;
    __syncthreads();
    for (int e = threadIdx.x; e < BT_ROWS * L; e += blockDim.x) {
      const int64_t j = j0 + e / L;
      sH[e] = (j < n) ? Hbar[j * L + e % L] : 0.0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < BT_ROWS * L; e += blockDim.x) {
      const int jr = e / L, i = e % L;
      double acc = 0.0;
      if (i < r) {
        const double* t = T + static_cast<int64_t>(i) * L;
        const double* h = sH + jr * L;
        for (int c = 0; c < l; ++c) acc = fma(__ldg(t + c), h[c], acc);
      }
      sB[e] = acc;
      const int64_t j = j0 + jr;
      if (j < n) Bt[j * L + i] = acc;
    }
    __syncthreads();
    // this block's own partial, accumulated over its feature blocks in a fixed order
    for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
      const int a = e / L, b = e % L;
      if (a < r && b <= a) {
        double acc = out[e];
#pragma unroll 8
        for (int jr = 0; jr < BT_ROWS; ++jr) acc = fma(sB[jr * L + a], sB[jr * L + b], acc);
        out[e] = acc;
      }
    }
  }
}

// C = sum over blocks (fixed order), symmetric fill from the lower triangle.
__global__ void c_reduce_kernel(const double* __restrict__ Cpart, int parts, int L, double* __restrict__ C) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= L * L) return;
  const int a = e / L, b = e % L;
  const int src = a >= b ? e : (b * L + a);
  double acc = 0.0;
  for (int p = 0; p < parts; ++p) acc += Cpart[static_cast<int64_t>(p) * L * L + src];
  C[e] = acc;
}

// V[j][i] (column-major output, ld n) = sum_c Bt[j][c] W[c][i] / sigma_i, i < k.
__global__ void form_v_kernel(const double* __restrict__ Bt, const double* __restrict__ W,
                              const double* __restrict__ sig, const int* __restrict__ info, int64_t n, int k, int L,
                              double* __restrict__ V) {
  const int r = info[0];
  const int64_t total = n * k;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(idx / n);
    const int64_t j = idx % n;
    double acc = 0.0;
    if (i < r && sig[i] > 0.0) {
      const double* b = Bt + j * L;
      for (int c = 0; c < r; ++c) acc = fma(b[c], W[static_cast<int64_t>(c) * L + i], acc);
      acc /= sig[i];
    }
    V[idx] = acc;
  }
}

// Per column i: the entry of largest |.| (lowest index on ties) is made positive.
__global__ void __launch_bounds__(SIGN_T) sign_fix_kernel(double* __restrict__ V, int64_t n) {
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
  const bool flip = col[best_j[0]] < 0.0;
  __syncthreads();
  if (flip) {
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) col[j] = -col[j];
  }
}

// -------------------------------------------------------------- one-block dense helpers
// Matrices are d x d blocks with leading dimension ld, in shared or global memory.

__device__ double blk_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const double out = red[0];
  __syncthreads();
  return out;
}

// Precision-generic math: the float overloads must not fall back to FP64 (slow here).
__device__ __forceinline__ float tsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double tsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float tabs(float x) { return fabsf(x); }
__device__ __forceinline__ double tabs(double x) { return fabs(x); }
__device__ __forceinline__ float tmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double tmin(double a, double b) { return fmin(a, b); }

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

// In-place Cholesky: the lower triangle of A becomes L1 (A = L1 L1^T). False if a pivot <= tol.
template <typename T>
__device__ bool blk_cholesky(T* A, int d, int ld, double tol) {
  __shared__ int ok;
  if (threadIdx.x == 0) ok = 1;
  __syncthreads();
  for (int k = 0; k < d; ++k) {
    if (threadIdx.x == 0) {
      const T v = A[k * ld + k];
      if (!(static_cast<double>(v) > tol)) ok = 0;
      else A[k * ld + k] = tsqrt(v);
    }
    __syncthreads();
    if (!ok) return false;
    const T dk = A[k * ld + k];
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
template <typename T>
__device__ void blk_trinv_lower(const T* Lm, T* Linv, int d, int ld) {
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) Linv[(e / d) * ld + e % d] = T(0);
  __syncthreads();
  for (int c = threadIdx.x; c < d; c += blockDim.x) {
    for (int i = c; i < d; ++i) {
      T acc = (i == c) ? T(1) : T(0);
      for (int j = c; j < i; ++j) acc -= Lm[i * ld + j] * Linv[j * ld + c];
      Linv[i * ld + c] = acc / Lm[i * ld + i];
    }
  }
  __syncthreads();
}

// One-warp Cholesky (right-looking, lanes over rows) and inverse of the factor, for the
// small FP32 factorisations: a warp needs no block barriers between the d steps.
template <typename T>
__device__ bool warp_cholesky(T* A, int d, int ld, T tol) {
  const int lane = threadIdx.x & 31;
  for (int k = 0; k < d; ++k) {
    const T v = A[k * ld + k];
    if (!(v > tol)) return false;   // the same value in every lane: a uniform exit
    const T dk = tsqrt(v);
    const T inv = T(1) / dk;
    __syncwarp();
    if (lane == 0) A[k * ld + k] = dk;
    for (int i = k + 1 + lane; i < d; i += 32) A[i * ld + k] *= inv;
    __syncwarp();
    for (int i = k + 1 + lane; i < d; i += 32) {
      const T lik = A[i * ld + k];
      for (int j = k + 1; j <= i; ++j) A[i * ld + j] -= lik * A[j * ld + k];
    }
    __syncwarp();
  }
  return true;
}

template <typename T>
__device__ void warp_trinv_lower(const T* Lm, T* Linv, int d, int ld) {
  const int lane = threadIdx.x & 31;
  for (int c = lane; c < d; c += 32) {
    for (int i = 0; i < c; ++i) Linv[i * ld + c] = T(0);
    for (int i = c; i < d; ++i) {
      T acc = (i == c) ? T(1) : T(0);
      for (int j = c; j < i; ++j) acc -= Lm[i * ld + j] * Linv[j * ld + c];
      Linv[i * ld + c] = acc / Lm[i * ld + i];
    }
  }
  __syncwarp();
}

// Cyclic Jacobi eigendecomposition of the symmetric d x d matrix A (destroyed), in the
// arithmetic of T (float or double), parallel ordering: each round rotates d/2 disjoint
// pairs, A <- R A R^T and W <- W R^T, every thread updating whole 2 x 2 blocks so that a
// round needs two barriers. On return W holds the eigenvectors as columns (W is set to
// the identity first) and, when `sort` is set, lam the eigenvalues descending with W's
// columns in the same order. Sweeps stop once the off-diagonal part is below `conv`
// (relative, squared Frobenius norms), after a sweep without any rotation, or after
// max_sweeps. A pair is left alone when |a_pq| <= eps_rel sqrt(|a_pp a_qq|), or - with
// tau1 > 0 - when rotating it would move an eigenvalue by less than tau1 times the
// smaller diagonal entry and turn the vectors by less than tau2 radians.
template <typename T>
__device__ void blk_jacobi(T* A, T* W, double* lam, int d, int ld, double* red, int* sweeps_out, double conv,
                           double eps_rel, double tau1, double tau2, int max_sweeps, bool sort) {
  __shared__ T cs[kMaxL / 2 + 1], sn[kMaxL / 2 + 1];
  __shared__ int P[kMaxL / 2 + 1], Q[kMaxL / 2 + 1];
  __shared__ int rotated;
  const double tiny = sizeof(T) == 4 ? 1e-37 : 1e-300;
  const int de = d + (d & 1);           // even count; index d (when d is odd) is a dummy
  const int npairs = de / 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) W[(e / d) * ld + e % d] = ((e / d) == (e % d)) ? T(1) : T(0);
  __syncthreads();
  int sweep = 0;
#ifdef SPCA_FIN_TRACE
  long long c0 = clock64();
  unsigned long long g0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g0));
#endif
  for (; sweep < max_sweeps && d > 1; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
      const int i = e / d, j = e % d;
      const double v = static_cast<double>(A[i * ld + j]);
      tot += v * v;
      if (i != j) off += v * v;
    }
    const double off_sum = blk_sum(off, red);
    const double tot_sum = blk_sum(tot, red);
    if (off_sum <= conv * tot_sum || tot_sum == 0.0) break;
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    if (tau1 > 0.0) {
      // polish: look at every pair at once (FP32 estimates) and stop if none needs a rotation
      for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
        const int i = e / d, j = e - (e / d) * d;
        if (j <= i) continue;
        const float a = fabsf(static_cast<float>(A[i * ld + j]));
        const float ai = static_cast<float>(A[i * ld + i]), aj = static_cast<float>(A[j * ld + j]);
        const float gap = fabsf(aj - ai), mn = fminf(fabsf(ai), fabsf(aj));
        const bool work = a > static_cast<float>(eps_rel) * sqrtf(fabsf(ai)) * sqrtf(fabsf(aj)) &&
                          !(a * a <= static_cast<float>(tau1) * mn * gap && a <= static_cast<float>(tau2) * gap);
        if (work) rotated = 1;
      }
      __syncthreads();
      const bool any = rotated != 0;
      __syncthreads();
      if (!any) break;
      if (threadIdx.x == 0) rotated = 0;
      __syncthreads();
    }
    for (int round = 0; round < de - 1; ++round) {
      for (int pi = threadIdx.x; pi < npairs; pi += blockDim.x) {
        int p, q;
        if (pi == 0) {
          p = de - 1;
          q = round;
        } else {
          p = (round + pi) % (de - 1);
          q = (round - pi + (de - 1)) % (de - 1);
        }
        if (p > q) { const int t = p; p = q; q = t; }
        T c = T(1), sv = T(0);
        if (q < d) {
          const T apq = A[p * ld + q];
          const T app = A[p * ld + p], aqq = A[q * ld + q];
          const T a = tabs(apq);
          const T gap = tabs(aqq - app);
          const T mn = tmin(tabs(app), tabs(aqq));
          bool work = a > T(tiny) && a > T(eps_rel) * tsqrt(tabs(app)) * tsqrt(tabs(aqq));
          if (work && tau1 > 0.0 && a * a <= T(tau1) * mn * gap && a <= T(tau2) * gap) work = false;
          if (work) {
            jacobi_rotation<T>(app, aqq, apq, c, sv);
            rotated = 1;
          }
        }
        P[pi] = p; Q[pi] = q; cs[pi] = c; sn[pi] = sv;
      }
      __syncthreads();
      // A: the 2 x 2 block of pairs (a, b) becomes R_a M R_b^T (a warp per pa, lanes over pb);
      // W: row i of pair b, W R_b^T (the next warps, lanes over pb)
      for (int row = warp; row < npairs + d; row += nwarps) {
        for (int pb = lane; pb < npairs; pb += 32) {
        if (row < npairs) {
          const int pa = row;
          const T sa = sn[pa], sb = sn[pb];
          if (sa == T(0) && sb == T(0)) continue;
          const int ia = P[pa], ja = Q[pa], ib = P[pb], jb = Q[pb];   // rows ia, ja; columns ib, jb
          const bool ra = ja < d, rb = jb < d;
          const T ca = cs[pa], cb = cs[pb];
          const T m00 = A[ia * ld + ib];
          const T m01 = rb ? A[ia * ld + jb] : T(0);
          const T m10 = ra ? A[ja * ld + ib] : T(0);
          const T m11 = (ra && rb) ? A[ja * ld + jb] : T(0);
          const T r00 = ca * m00 - sa * m10, r01 = ca * m01 - sa * m11;   // R_a M
          const T r10 = sa * m00 + ca * m10, r11 = sa * m01 + ca * m11;
          A[ia * ld + ib] = cb * r00 - sb * r01;                          // (R_a M) R_b^T
          if (rb) A[ia * ld + jb] = sb * r00 + cb * r01;
          if (ra) A[ja * ld + ib] = cb * r10 - sb * r11;
          if (ra && rb) A[ja * ld + jb] = sb * r10 + cb * r11;
        } else {
          const int i = row - npairs;
          const T sb = sn[pb];
          if (sb == T(0)) continue;
          const int ib = P[pb], jb = Q[pb];
          const T cb = cs[pb];
          const T wp = W[i * ld + ib], wq = W[i * ld + jb];
          W[i * ld + ib] = cb * wp - sb * wq;
          W[i * ld + jb] = sb * wp + cb * wq;
        }
        }
      }
      __syncthreads();
    }
    if (!rotated) { ++sweep; break; }
  }
  if (threadIdx.x == 0 && sweeps_out) *sweeps_out = sweep;
#ifdef SPCA_FIN_TRACE
  {
    unsigned long long g1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g1));
    if (threadIdx.x == 0)
      printf("jacobi fp%d d=%d sweeps=%d cycles=%lld ns=%llu threads=%d\n", static_cast<int>(8 * sizeof(T)), d, sweep,
             clock64() - c0, g1 - g0, blockDim.x);
  }
#endif
  if (!sort) return;
  // sort descending: rank of each eigenvalue, then permute W's columns through A as scratch
  for (int i = threadIdx.x; i < d; i += blockDim.x) red[i] = static_cast<double>(A[i * ld + i]);
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
  // eigen route: gbar = W diag(lam) W^T
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) X[(e / l) * ld + e % l] = gbar[(e / l) * L + e % l];
  __syncthreads();
  int sweeps = 0;
  // relative off-diagonal Frobenius norm <= 1e-13: below that, round-off of the rotations
  // themselves (about eps * lambda_max per entry) keeps it from shrinking further
  blk_jacobi<double>(X, Y, lam, l, ld, red, &sweeps, 1e-26, 1e-18, 0.0, 0.0, 40, true);
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
// (iii) eig_polish_kernel: FP64 Jacobi on C1, skipping the rotations that would change no
//      eigenvalue by more than 1e-8 relative and no vector by more than 1e-6 rad - the
//      remaining work sits among the small eigenvalues that FP32 could not separate;
// (iv) Z = W W1 (FP64): the eigenvectors of C, columns by descending eigenvalue.
__global__ void __launch_bounds__(FT) eig_f32_kernel(const double* __restrict__ C, float* __restrict__ Xg,
                                                     float* __restrict__ Yg, double* __restrict__ W0,
                                                     const int* __restrict__ info, int L, int smem) {
  extern __shared__ float e32[];
  __shared__ double red[FT];
  const int r = info[0];
  const int ld = smem ? r : L;
  float* X = smem ? e32 : Xg;
  float* Y = smem ? e32 + r * r : Yg;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x)
    X[(e / r) * ld + e % r] = static_cast<float>(C[(e / r) * L + e % r]);
  __syncthreads();
  if (r > 0) blk_jacobi<float>(X, Y, nullptr, r, ld, red, nullptr, 1e-10, 3e-8, 0.0, 0.0, 16, false);
  __syncthreads();
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
    const int i = e / L, j = e % L;
    W0[e] = (i < r && j < r) ? static_cast<double>(Y[i * ld + j]) : 0.0;
  }
}

// Out = alpha op(A) op(B) + beta D on the leading r x r block (ld L, zero elsewhere), with
// r = *rdev when rdev is given, else rhost; one block per row, FP64. Row i of op(A) is
// staged in shared memory, and op(B) too when `stage` is set (as rows of r). D may be NULL.
constexpr int GEMM_T = 128;
constexpr size_t kGemmSmemMax = 200 * 1024;
__global__ void __launch_bounds__(GEMM_T) small_gemm_kernel(const double* __restrict__ A, int ta,
                                                            const double* __restrict__ B, int tb,
                                                            const double* __restrict__ D, double alpha, double beta,
                                                            const int* __restrict__ rdev, int rhost, int L,
                                                            int stage, double* __restrict__ Out) {
  extern __shared__ double gsm[];
  double* sa = gsm;           // r
  double* sb = gsm + kMaxL;   // r x r: sb[t * r + j] = op(B)[t][j]
  const int r = rdev ? *rdev : rhost;
  const int i = blockIdx.x;
  if (i < r) {
    for (int t = threadIdx.x; t < r; t += blockDim.x) sa[t] = ta ? A[t * L + i] : A[i * L + t];
    if (stage) {
      for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
        const int t = e / r, j = e - t * r;
        sb[e] = tb ? B[j * L + t] : B[t * L + j];
      }
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < L; j += blockDim.x) {
    double acc = 0.0;
    if (i < r && j < r) {
      if (stage) {
#pragma unroll 4
        for (int t = 0; t < r; ++t) acc = fma(sa[t], sb[t * r + j], acc);
      } else {
        for (int t = 0; t < r; ++t) acc = fma(sa[t], tb ? B[j * L + t] : B[t * L + j], acc);
      }
      acc *= alpha;
      if (D) acc = fma(beta, D[i * L + j], acc);
    }
    Out[i * L + j] = acc;
  }
}

__global__ void __launch_bounds__(FT) eig_polish_kernel(const double* __restrict__ C1, double* __restrict__ Xg,
                                                        double* __restrict__ W1, double* __restrict__ lam,
                                                        double* __restrict__ sig, int* __restrict__ info, int L,
                                                        int smem) {
  extern __shared__ double e64[];
  __shared__ double red[FT];
  const int r = info[0];
  const int ld = smem ? r : L;
  double* X = smem ? e64 : Xg;
  double* Y = smem ? e64 + r * r : W1;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) X[(e / r) * ld + e % r] = C1[(e / r) * L + e % r];
  __syncthreads();
  int sweeps = 0;
  if (r > 0) blk_jacobi<double>(X, Y, lam, r, ld, red, &sweeps, 1e-26, 1e-18, 1e-8, 1e-6, 40, true);
  __syncthreads();
  if (smem) {
    for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
      const int i = e / L, j = e % L;
      W1[e] = (i < r && j < r) ? Y[i * ld + j] : 0.0;
    }
  } else {
    for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
      const int i = e / L, j = e % L;
      if (!(i < r && j < r)) W1[e] = 0.0;
    }
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
__global__ void __launch_bounds__(32) chol_inv_f32_kernel(const double* __restrict__ M, int l, int L,
                                                          double tol_rel, int rank_ok, int first,
                                                          float* __restrict__ Xg, float* __restrict__ Yg,
                                                          double* __restrict__ Y, int* __restrict__ info,
                                                          int smem) {
  extern __shared__ float c32[];
  const int ld = smem ? l : L;
  float* X = smem ? c32 : Xg;
  float* Yf = smem ? c32 + l * l : Yg;
  for (int i = threadIdx.x >> 3; i < l; i += blockDim.x >> 3)   // 8 lanes per row
    for (int j = threadIdx.x & 7; j < l; j += 8) X[i * ld + j] = static_cast<float>(M[i * L + j]);
  __syncwarp();
  float dm = 0.f;
  for (int i = threadIdx.x; i < l; i += 32) dm = fmaxf(dm, fabsf(X[i * ld + i]));
  for (int o = 16; o > 0; o >>= 1) dm = fmaxf(dm, __shfl_xor_sync(0xffffffffu, dm, o));
  bool ok = rank_ok && dm > 0.f && isfinite(dm) && warp_cholesky<float>(X, l, ld, static_cast<float>(tol_rel) * dm);
  if (ok) warp_trinv_lower<float>(X, Yf, l, ld);
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

cudaError_t finalize_run(const State& s, const FinalWork& f, int64_t m, int k, double* sigma_dev, double* V_dev,
                         cudaStream_t st, Prof* prof, int64_t rows_seen, bool centered) {
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kMaxDenseSmem));
    cudaFuncSetAttribute(chol_inv_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(kMaxDenseSmem));
    cudaFuncSetAttribute(small_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(kGemmSmemMax));
    cudaFuncSetAttribute(eig_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kMaxDenseSmem));
    cudaFuncSetAttribute(eig_polish_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(kMaxDenseSmem));
    cudaFuncSetAttribute(bt_and_c_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(2 * sizeof(double) * BT_ROWS * kMaxL));
    attr_done = true;
  }
  prof->begin(SPCA_K_FINALIZE, st);
  cudaError_t e = centered_state(s, f, m, st);
  if (e != cudaSuccess) return e;
  // rank bound: a centred Gram of m rows has rank <= m - 1, an uncentred one <= m
  int64_t r_max = centered ? rows_seen - 1 : rows_seen;
  if (r_max > s.l) r_max = s.l;
  if (r_max < 0) r_max = 0;
  const int64_t LL = static_cast<int64_t>(s.L) * s.L;
  float* s32 = reinterpret_cast<float*>(f.Cpart);   // FP32 scratch when l x l does not fit in shared memory
  const size_t dense32 = 2 * sizeof(float) * s.l * s.l;
  const int smem32 = dense32 <= kMaxDenseSmem ? 1 : 0;
  const int l = s.l, L = s.L;
  const int rank_ok = r_max >= l ? 1 : 0;
  const size_t gemm_full = sizeof(double) * (kMaxL + static_cast<size_t>(l) * l);
  const int gstage = gemm_full <= kGemmSmemMax ? 1 : 0;
  const size_t gemm_smem = gstage ? gemm_full : sizeof(double) * kMaxL;
  // mixed-precision route (buffers: Y1 W, X1 T, Y2 X, T2 C, X2 W, F X, T T)
  const dim3 gb(L), gt(GEMM_T);
  chol_inv_f32_kernel<<<1, 32, smem32 ? dense32 : 0, st>>>(f.gbar, l, L, l * 1.2e-7, rank_ok, 1, s32, s32 + LL, f.W,
                                                            f.info, smem32);
  // X1 = Y1 (gram Y1^T)
  small_gemm_kernel<<<gb, gt, gemm_smem, st>>>(f.gbar, 0, f.W, 1, nullptr, 1.0, 0.0, nullptr, l, L, gstage, f.X);
  small_gemm_kernel<<<gb, gt, gemm_smem, st>>>(f.W, 0, f.X, 0, nullptr, 1.0, 0.0, nullptr, l, L, gstage, f.T);
  chol_inv_f32_kernel<<<1, 32, smem32 ? dense32 : 0, st>>>(f.T, l, L, l * 1.2e-7, 1, 0, s32, s32 + LL, f.X, f.info,
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
  const size_t dense64 = 2 * sizeof(double) * s.l * s.l;
  const int smem64 = dense64 <= kMaxDenseSmem ? 1 : 0;
  const int64_t nblk = (s.n + BT_ROWS - 1) / BT_ROWS;
  const int parts = static_cast<int>(nblk < f.nparts ? nblk : f.nparts);
  bt_and_c_kernel<<<parts, 256, 2 * sizeof(double) * BT_ROWS * s.L, st>>>(f.Hbar, f.T, f.info, s.n, s.l, s.L, f.Bt,
                                                                          f.Cpart);
  c_reduce_kernel<<<(s.L * s.L + 255) / 256, 256, 0, st>>>(f.Cpart, parts, s.L, f.C);
  // eigenvectors of C: FP32 Jacobi, FP64 orthogonalisation and polish (scratch: Cpart, whose
  // partials are consumed by now, and T, X, W)
  double* s64 = f.Cpart + 2 * LL;
  double* W1 = f.Cpart + 3 * LL;
  eig_f32_kernel<<<1, FT, smem32 ? dense32 : 0, st>>>(f.C, s32, s32 + LL, f.W, f.info, s.L, smem32);
  // Newton-Schulz, twice: W <- 1.5 W - 0.5 W (W^T W)  (W: f.W -> f.T -> f.W)
  small_gemm_kernel<<<gb, gt, gemm_smem, st>>>(f.W, 1, f.W, 0, nullptr, 1.0, 0.0, f.info, 0, s.L, gstage, f.X);
  small_gemm_kernel<<<gb, gt, gemm_smem, st>>>(f.W, 0, f.X, 0, f.W, -0.5, 1.5, f.info, 0, s.L, gstage, f.T);
  small_gemm_kernel<<<gb, gt, gemm_smem, st>>>(f.T, 1, f.T, 0, nullptr, 1.0, 0.0, f.info, 0, s.L, gstage, f.X);
  small_gemm_kernel<<<gb, gt, gemm_smem, st>>>(f.T, 0, f.X, 0, f.T, -0.5, 1.5, f.info, 0, s.L, gstage, f.W);
  // C1 = W^T C W
  small_gemm_kernel<<<gb, gt, gemm_smem, st>>>(f.C, 0, f.W, 0, nullptr, 1.0, 0.0, f.info, 0, s.L, gstage, f.X);
  small_gemm_kernel<<<gb, gt, gemm_smem, st>>>(f.W, 1, f.X, 0, nullptr, 1.0, 0.0, f.info, 0, s.L, gstage, f.T);
  eig_polish_kernel<<<1, FT, smem64 ? dense64 : 0, st>>>(f.T, s64, W1, f.lam, f.sig, f.info, s.L, smem64);
  // Z = W W1 (into f.X): the eigenvectors of C, used to form V
  small_gemm_kernel<<<gb, gt, gemm_smem, st>>>(f.W, 0, W1, 0, nullptr, 1.0, 0.0, f.info, 0, s.L, gstage, f.X);
  form_v_kernel<<<grid_for(s.n * k, 256), 256, 0, st>>>(f.Bt, f.X, f.sig, f.info, s.n, k, s.L, V_dev);
  sign_fix_kernel<<<k, SIGN_T, 0, st>>>(V_dev, s.n);
  prof->launches[SPCA_K_FINALIZE] += 24;  // launches above beyond the one begin() counted
  prof->end(SPCA_K_FINALIZE, st);
  e = cudaMemcpyAsync(sigma_dev, f.sig, sizeof(double) * k, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace spca

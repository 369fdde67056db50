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
//  4. SVD of B through C = W_B diag(sigma^2) W_B^T (cyclic Jacobi, parallel
//     ordering); V = B^T W_B diag(1/sigma), the leading k columns (Alg. 4
//     steps 17-19).
//  5. Each v_i scaled by +-1 so that its largest-magnitude entry (lowest index
//     on ties) is positive.
// The l x l steps run in one thread block, in shared memory when two l x l
// matrices fit; the n x l steps are spread over the GPU.
#include <cfloat>

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

// C = op(A) op(B), op = transpose when flagged; all d x d with leading dimension ld.
__device__ void blk_gemm(const double* A, bool ta, const double* B, bool tb, double* C, int d, int ld) {
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
    const int i = e / d, j = e % d;
    double acc = 0.0;
    for (int t = 0; t < d; ++t) {
      const double a = ta ? A[t * ld + i] : A[i * ld + t];
      const double b = tb ? B[j * ld + t] : B[t * ld + j];
      acc = fma(a, b, acc);
    }
    C[i * ld + j] = acc;
  }
  __syncthreads();
}

// Cyclic Jacobi eigendecomposition of the symmetric d x d matrix A (destroyed): on return W
// holds the eigenvectors as columns and lam the eigenvalues, descending.
__device__ void blk_jacobi_eig(double* A, double* W, double* lam, int d, int ld, double* red, int* sweeps_out) {
  __shared__ double cs[kMaxL / 2 + 1], sn[kMaxL / 2 + 1];
  __shared__ int P[kMaxL / 2 + 1], Q[kMaxL / 2 + 1];
  const int de = d + (d & 1);           // even count; index d (when d is odd) is a dummy
  const int npairs = de / 2;
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) W[(e / d) * ld + e % d] = ((e / d) == (e % d)) ? 1.0 : 0.0;
  __syncthreads();
  int sweep = 0;
  for (; sweep < 40 && d > 1; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
      const int i = e / d, j = e % d;
      const double v = A[i * ld + j];
      tot += v * v;
      if (i != j) off += v * v;
    }
    const double off_sum = blk_sum(off, red);
    const double tot_sum = blk_sum(tot, red);
    // relative off-diagonal Frobenius norm <= 1e-13: below that, round-off of the rotations
    // themselves (about eps * lambda_max per entry) keeps it from shrinking further
    if (off_sum <= 1e-26 * tot_sum || tot_sum == 0.0) break;
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
        double c = 1.0, s = 0.0;
        if (q < d) {
          const double apq = A[p * ld + q];
          const double app = A[p * ld + p], aqq = A[q * ld + q];
          if (fabs(apq) > 1e-300 && fabs(apq) > 1e-18 * sqrt(fabs(app * aqq))) {
            const double theta = (aqq - app) / (2.0 * apq);
            const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        }
        P[pi] = p; Q[pi] = q; cs[pi] = c; sn[pi] = s;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int e = threadIdx.x; e < npairs * d; e += blockDim.x) {
        const int pi = e / d, j = e % d;
        const int p = P[pi], q = Q[pi];
        const double s = sn[pi];
        if (q < d && s != 0.0) {
          const double c = cs[pi];
          const double ap = A[p * ld + j], aq = A[q * ld + j];
          A[p * ld + j] = c * ap - s * aq;
          A[q * ld + j] = s * ap + c * aq;
        }
      }
      __syncthreads();
      // columns: A <- A J, W <- W J
      for (int e = threadIdx.x; e < npairs * d; e += blockDim.x) {
        const int pi = e / d, i = e % d;
        const int p = P[pi], q = Q[pi];
        const double s = sn[pi];
        if (q < d && s != 0.0) {
          const double c = cs[pi];
          const double ap = A[i * ld + p], aq = A[i * ld + q];
          A[i * ld + p] = c * ap - s * aq;
          A[i * ld + q] = s * ap + c * aq;
          const double wp = W[i * ld + p], wq = W[i * ld + q];
          W[i * ld + p] = c * wp - s * wq;
          W[i * ld + q] = s * wp + c * wq;
        }
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0 && sweeps_out) *sweeps_out = sweep;
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
}

// R from gram_bar (step 2). Writes T (r x l, ld L) and info = {r, route, sweeps}.
// Work matrices X, Y, Z live in shared memory when `smem` is set (3 l^2 doubles), else in
// the global scratch X / Wg / T.
__global__ void __launch_bounds__(FT) factor_kernel(const double* __restrict__ gbar, int l, int L, int r_max,
                                                    double* __restrict__ T, double* __restrict__ Xg,
                                                    double* __restrict__ Wg, double* __restrict__ lam,
                                                    int* __restrict__ info, int smem) {
  extern __shared__ double fsm[];
  __shared__ double red[FT];
  __shared__ double dmax;
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
  blk_jacobi_eig(X, Y, lam, l, ld, red, &sweeps);
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

// SVD of B through C = B B^T (r x r): W (ld L), lam, sigma.
__global__ void __launch_bounds__(FT) eig_c_kernel(const double* __restrict__ C, double* __restrict__ Wg,
                                                   double* __restrict__ Xg, double* __restrict__ lam,
                                                   double* __restrict__ sig, int* __restrict__ info, int L, int smem) {
  extern __shared__ double esm[];
  __shared__ double red[FT];
  const int r = info[0];
  const int ld = smem ? r : L;
  double* X = smem ? esm : Xg;
  double* Y = smem ? esm + r * r : Wg;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) X[(e / r) * ld + e % r] = C[(e / r) * L + e % r];
  __syncthreads();
  int sweeps = 0;
  if (r > 0) blk_jacobi_eig(X, Y, lam, r, ld, red, &sweeps);
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
    const int i = e / L, j = e % L;
    Wg[e] = (i < r && j < r) ? Y[i * ld + j] : 0.0;
  }
  for (int i = threadIdx.x; i < L; i += blockDim.x) sig[i] = (i < r) ? sqrt(fmax(lam[i], 0.0)) : 0.0;
  if (threadIdx.x == 0) info[3] = sweeps;
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
    cudaFuncSetAttribute(eig_c_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kMaxDenseSmem));
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
  const size_t dense3 = 3 * sizeof(double) * s.l * s.l;
  const int factor_smem = dense3 <= kMaxDenseSmem ? 1 : 0;
  factor_kernel<<<1, FT, factor_smem ? dense3 : 0, st>>>(f.gbar, s.l, s.L, static_cast<int>(r_max), f.T, f.X, f.W,
                                                         f.lam, f.info, factor_smem);
  const size_t dense = 2 * sizeof(double) * s.l * s.l;
  const int use_smem = dense <= kMaxDenseSmem ? 1 : 0;
  const int64_t nblk = (s.n + BT_ROWS - 1) / BT_ROWS;
  const int parts = static_cast<int>(nblk < f.nparts ? nblk : f.nparts);
  bt_and_c_kernel<<<parts, 256, 2 * sizeof(double) * BT_ROWS * s.L, st>>>(f.Hbar, f.T, f.info, s.n, s.l, s.L, f.Bt,
                                                                          f.Cpart);
  c_reduce_kernel<<<(s.L * s.L + 255) / 256, 256, 0, st>>>(f.Cpart, parts, s.L, f.C);
  eig_c_kernel<<<1, FT, use_smem ? dense : 0, st>>>(f.C, f.W, f.X, f.lam, f.sig, f.info, s.L, use_smem);
  form_v_kernel<<<grid_for(s.n * k, 256), 256, 0, st>>>(f.Bt, f.W, f.sig, f.info, s.n, k, s.L, V_dev);
  sign_fix_kernel<<<k, SIGN_T, 0, st>>>(V_dev, s.n);
  prof->launches[SPCA_K_FINALIZE] += 7;   // launches above beyond the one begin() counted
  prof->end(SPCA_K_FINALIZE, st);
  e = cudaMemcpyAsync(sigma_dev, f.sig, sizeof(double) * k, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace spca

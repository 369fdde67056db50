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
//     B = Q^T A_bar = T H_bar^T (Thm 1). If a Cholesky pivot falls below
//     l eps max(diag), gram_bar is rank deficient (Thm 1 assumes full column
//     rank): use its eigendecomposition W diag(lam) W^T instead, keep
//     lam > l eps lam_max, T = diag(lam_r)^-1/2 W_r^T.
//  3. Bt = H_bar T^T (n x r), i.e. B^T.
//  4. SVD of B through the r x r matrix C = B B^T = W_B diag(sigma^2) W_B^T
//     (cyclic Jacobi, parallel ordering); then V = B^T W_B diag(1/sigma), the
//     leading k columns (Alg. 4 steps 17-19).
//  5. Each v_i scaled by +-1 so that its largest-magnitude entry (lowest index
//     on ties) is positive.
// The l x l steps run in one thread block; the n x l steps are spread over the GPU.
#include <cfloat>

#include "spca_internal.cuh"

namespace spca {

namespace {

constexpr int FT = 1024;   // threads of the single-block kernels

// -------------------------------------------------------------- n x l kernels

__global__ void center_h_kernel(const float* __restrict__ H, const double* __restrict__ colsum,
                                const double* __restrict__ sG, int64_t n, int l, int L, double inv_m,
                                double* __restrict__ Hbar) {
  const int64_t total = n * L;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t j = idx / L;
    const int c = static_cast<int>(idx % L);
    Hbar[idx] = (c < l) ? static_cast<double>(H[idx]) - colsum[j] * sG[c] * inv_m : 0.0;
  }
}

__global__ void center_gram_kernel(const double* __restrict__ gram, const double* __restrict__ sG, int l, int L,
                                   double inv_m, double* __restrict__ gbar) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= L * L) return;
  const int a = e / L, b = e % L;
  gbar[e] = (a < l && b < l) ? gram[e] - sG[a] * sG[b] * inv_m : 0.0;
}

// Bt[j][i] = sum_c T[i][c] Hbar[j][c], i < r.
__global__ void form_bt_kernel(const double* __restrict__ Hbar, const double* __restrict__ T,
                               const int* __restrict__ info, int64_t n, int l, int L, double* __restrict__ Bt) {
  const int r = info[0];
  const int64_t total = n * L;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t j = idx / L;
    const int i = static_cast<int>(idx % L);
    double acc = 0.0;
    if (i < r) {
      const double* h = Hbar + j * L;
      const double* t = T + static_cast<int64_t>(i) * L;
      for (int c = 0; c < l; ++c) acc = fma(t[c], h[c], acc);
    }
    Bt[idx] = acc;
  }
}

// Cpart[p] = sum over rows j of part p of Bt[j]^T Bt[j] (r x r, ld L).
__global__ void bbt_partial_kernel(const double* __restrict__ Bt, const int* __restrict__ info, int64_t n, int L,
                                   int64_t rows_per_part, double* __restrict__ Cpart) {
  const int r = info[0];
  const int64_t j0 = blockIdx.x * rows_per_part;
  const int64_t j1 = j0 + rows_per_part < n ? j0 + rows_per_part : n;
  double* out = Cpart + static_cast<int64_t>(blockIdx.x) * L * L;
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
    const int a = e / L, b = e % L;
    double acc = 0.0;
    if (a < r && b < r && b <= a) {
      for (int64_t j = j0; j < j1; ++j) acc = fma(Bt[j * L + a], Bt[j * L + b], acc);
    }
    out[e] = acc;
  }
}

__global__ void bbt_reduce_kernel(const double* __restrict__ Cpart, int parts, int L, double* __restrict__ C) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= L * L) return;
  const int a = e / L, b = e % L;
  const int lo = a < b ? a * L + b : b * L + a;   // symmetric fill from the lower triangle
  const int src = a >= b ? e : (b * L + a);
  (void)lo;
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
__global__ void sign_fix_kernel(double* __restrict__ V, int64_t n) {
  __shared__ double best_v[FT];
  __shared__ int64_t best_j[FT];
  double* col = V + static_cast<int64_t>(blockIdx.x) * n;
  double bv = -1.0;
  int64_t bj = 0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const double a = fabs(col[j]);
    if (a > bv) { bv = a; bj = j; }   // strictly greater keeps the lowest index of this thread
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

// -------------------------------------------------------------- one-block dense helpers (ld = L)

// In-place Cholesky of the leading l x l block: lower triangle of A becomes L1.
// Returns false (to all threads) if a pivot is <= tol.
__device__ bool blk_cholesky(double* A, int l, int L, double tol) {
  __shared__ int ok;
  if (threadIdx.x == 0) ok = 1;
  __syncthreads();
  for (int k = 0; k < l; ++k) {
    if (threadIdx.x == 0) {
      const double d = A[k * L + k];
      if (!(d > tol)) ok = 0;
      else A[k * L + k] = sqrt(d);
    }
    __syncthreads();
    if (!ok) return false;
    const double dk = A[k * L + k];
    for (int i = k + 1 + threadIdx.x; i < l; i += blockDim.x) A[i * L + k] /= dk;
    __syncthreads();
    const int rem = l - k - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      const int i = k + 1 + e / rem, j = k + 1 + e % rem;
      if (j <= i) A[i * L + j] -= A[i * L + k] * A[j * L + k];
    }
    __syncthreads();
  }
  return true;
}

// Linv = inverse of the lower-triangular leading l x l block of Lm (upper part zeroed).
__device__ void blk_trinv_lower(const double* Lm, double* Linv, int l, int L) {
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) Linv[e] = 0.0;
  __syncthreads();
  for (int c = threadIdx.x; c < l; c += blockDim.x) {
    for (int i = c; i < l; ++i) {
      double acc = (i == c) ? 1.0 : 0.0;
      for (int j = c; j < i; ++j) acc -= Lm[i * L + j] * Linv[j * L + c];
      Linv[i * L + c] = acc / Lm[i * L + i];
    }
  }
  __syncthreads();
}

// C = op(A) * op(B) on l x l blocks, op = transpose when the flag is set.
__device__ void blk_gemm(const double* A, bool ta, const double* B, bool tb, double* C, int l, int L) {
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int i = e / l, j = e % l;
    double acc = 0.0;
    for (int t = 0; t < l; ++t) {
      const double a = ta ? A[t * L + i] : A[i * L + t];
      const double b = tb ? B[j * L + t] : B[t * L + j];
      acc = fma(a, b, acc);
    }
    C[i * L + j] = acc;
  }
  __syncthreads();
}

// Cyclic Jacobi eigendecomposition of the symmetric leading n x n block of A (destroyed).
// On return W holds the eigenvectors as columns and lam the eigenvalues, descending.
__device__ void blk_jacobi_eig(double* A, double* W, double* lam, int n, int L, int* sweeps_out) {
  __shared__ double cs[kMaxL / 2 + 1], sn[kMaxL / 2 + 1];
  __shared__ int P[kMaxL / 2 + 1], Q[kMaxL / 2 + 1];
  __shared__ double red[FT];
  __shared__ int done;
  const int ne = n + (n & 1);          // even count; index n (if odd) is a dummy
  const int npairs = ne / 2;
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) W[e] = ((e / L) == (e % L)) ? 1.0 : 0.0;
  __syncthreads();
  int sweep = 0;
  for (; sweep < 60; ++sweep) {
    // convergence test: off-diagonal mass relative to the whole
    double off = 0.0, tot = 0.0;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int i = e / n, j = e % n;
      const double v = A[i * L + j];
      tot += v * v;
      if (i != j) off += v * v;
    }
    red[threadIdx.x] = off;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    const double off_sum = red[0];
    __syncthreads();
    red[threadIdx.x] = tot;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) done = (off_sum <= 1e-30 * red[0]) || (red[0] == 0.0);
    __syncthreads();
    if (done) break;
    for (int round = 0; round < ne - 1; ++round) {
      // round-robin pairing: index ne-1 meets `round`, the others pair symmetrically around it
      for (int pi = threadIdx.x; pi < npairs; pi += blockDim.x) {
        int p, q;
        if (pi == 0) {
          p = ne - 1;
          q = round;
        } else {
          p = (round + pi) % (ne - 1);
          q = (round - pi + (ne - 1)) % (ne - 1);
        }
        if (p > q) { const int t = p; p = q; q = t; }
        double c = 1.0, s = 0.0;
        if (q < n) {
          const double apq = A[p * L + q];
          const double app = A[p * L + p], aqq = A[q * L + q];
          if (apq != 0.0 && fabs(apq) > 1e-300) {
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
      for (int e = threadIdx.x; e < npairs * n; e += blockDim.x) {
        const int pi = e / n, j = e % n;
        const int p = P[pi], q = Q[pi];
        if (q < n) {
          const double c = cs[pi], s = sn[pi];
          const double ap = A[p * L + j], aq = A[q * L + j];
          A[p * L + j] = c * ap - s * aq;
          A[q * L + j] = s * ap + c * aq;
        }
      }
      __syncthreads();
      // columns: A <- A J, W <- W J
      for (int e = threadIdx.x; e < npairs * n; e += blockDim.x) {
        const int pi = e / n, i = e % n;
        const int p = P[pi], q = Q[pi];
        if (q < n) {
          const double c = cs[pi], s = sn[pi];
          const double ap = A[i * L + p], aq = A[i * L + q];
          A[i * L + p] = c * ap - s * aq;
          A[i * L + q] = s * ap + c * aq;
          const double wp = W[i * L + p], wq = W[i * L + q];
          W[i * L + p] = c * wp - s * wq;
          W[i * L + q] = s * wp + c * wq;
        }
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0 && sweeps_out) *sweeps_out = sweep;
  // sort descending: rank of each eigenvalue, then permute W's columns through A as scratch
  for (int i = threadIdx.x; i < n; i += blockDim.x) red[i] = A[i * L + i];
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int rank = 0;
    const double v = red[i];
    for (int j = 0; j < n; ++j) {
      const double u = red[j];
      if (u > v || (u == v && j < i)) ++rank;
    }
    lam[rank] = v;
    for (int t = 0; t < n; ++t) A[t * L + rank] = W[t * L + i];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int t = e / n, c = e % n;
    W[t * L + c] = A[t * L + c];
  }
  __syncthreads();
}

// R from gram_bar (step 2). Writes T (r x l, ld L) and info = {r, route, sweeps}.
__global__ void __launch_bounds__(FT) factor_kernel(const double* __restrict__ gbar, int l, int L,
                                                    double* __restrict__ T, double* __restrict__ X,
                                                    double* __restrict__ W, double* __restrict__ lam,
                                                    int* __restrict__ info) {
  __shared__ double dmax;
  if (threadIdx.x == 0) {
    double d = 0.0;
    for (int i = 0; i < l; ++i) d = fmax(d, fabs(gbar[i * L + i]));
    dmax = d;
  }
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) X[e] = gbar[e];
  __syncthreads();
  const double tol = l * DBL_EPSILON * dmax;
  bool ok = (dmax > 0.0) && blk_cholesky(X, l, L, tol);
  if (ok) {
    // T1 = L1^-1 into W; refinement X2 = T1 gbar T1^T
    blk_trinv_lower(X, W, l, L);                 // W = T1
    blk_gemm(W, false, gbar, false, T, l, L);    // T = T1 gbar
    blk_gemm(T, false, W, true, X, l, L);        // X = T1 gbar T1^T
    for (int e = threadIdx.x; e < l * l; e += blockDim.x) {   // symmetrise
      const int i = e / l, j = e % l;
      if (j < i) {
        const double v = 0.5 * (X[i * L + j] + X[j * L + i]);
        X[i * L + j] = v;
        X[j * L + i] = v;
      }
    }
    __syncthreads();
    ok = blk_cholesky(X, l, L, l * DBL_EPSILON);
    if (ok) {
      blk_trinv_lower(X, lam == nullptr ? T : T, l, L);   // T = T2 = L2^-1
      blk_gemm(T, false, W, false, X, l, L);               // X = T2 T1
      for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
        const int i = e / L, j = e % L;
        T[e] = (i < l && j < l) ? X[i * L + j] : 0.0;
      }
      if (threadIdx.x == 0) { info[0] = l; info[1] = 0; info[2] = 0; }
      __syncthreads();
      return;
    }
  }
  // eigen route: gbar = W diag(lam) W^T
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) X[e] = gbar[e];
  __syncthreads();
  int sweeps = 0;
  blk_jacobi_eig(X, W, lam, l, L, &sweeps);
  __shared__ int r_keep;
  if (threadIdx.x == 0) {
    const double cut = l * DBL_EPSILON * fmax(lam[0], 0.0);
    int r = 0;
    while (r < l && lam[r] > cut) ++r;
    r_keep = r;
    info[0] = r; info[1] = 1; info[2] = sweeps;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
    const int i = e / L, c = e % L;
    T[e] = (i < r_keep && c < l) ? W[c * L + i] / sqrt(lam[i]) : 0.0;
  }
}

__global__ void __launch_bounds__(FT) eig_c_kernel(double* __restrict__ C, double* __restrict__ W,
                                                   double* __restrict__ lam, double* __restrict__ sig,
                                                   int* __restrict__ info, int L) {
  const int r = info[0];
  int sweeps = 0;
  if (r > 0) blk_jacobi_eig(C, W, lam, r, L, &sweeps);
  for (int i = threadIdx.x; i < L; i += blockDim.x) sig[i] = (i < r) ? sqrt(fmax(lam[i], 0.0)) : 0.0;
  if (threadIdx.x == 0) info[3] = sweeps;
}

int grid_for(int64_t total, int threads) {
  int64_t b = (total + threads - 1) / threads;
  if (b > 152 * 16) b = 152 * 16;
  return static_cast<int>(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t centered_state(const State& s, const FinalWork& f, int64_t m, cudaStream_t st) {
  const double inv_m = m > 0 ? 1.0 / static_cast<double>(m) : 0.0;
  center_h_kernel<<<grid_for(s.n * s.L, 256), 256, 0, st>>>(s.H, s.colsum, s.sG, s.n, s.l, s.L, inv_m, f.Hbar);
  center_gram_kernel<<<(s.L * s.L + 255) / 256, 256, 0, st>>>(s.gram, s.sG, s.l, s.L, inv_m, f.gbar);
  return cudaGetLastError();
}

cudaError_t finalize_run(const State& s, const FinalWork& f, int64_t m, int k, double* sigma_dev, double* V_dev,
                         cudaStream_t st, Prof* prof) {
  prof->begin(SPCA_K_FINALIZE, st);
  cudaError_t e = centered_state(s, f, m, st);
  if (e != cudaSuccess) return e;
  factor_kernel<<<1, FT, 0, st>>>(f.gbar, s.l, s.L, f.T, f.X, f.W, f.lam, f.info);
  form_bt_kernel<<<grid_for(s.n * s.L, 256), 256, 0, st>>>(f.Hbar, f.T, f.info, s.n, s.l, s.L, f.Bt);
  const int64_t rows_per_part = (s.n + f.nparts - 1) / f.nparts;
  const int parts = static_cast<int>((s.n + rows_per_part - 1) / rows_per_part);
  bbt_partial_kernel<<<parts, 256, 0, st>>>(f.Bt, f.info, s.n, s.L, rows_per_part, f.Cpart);
  bbt_reduce_kernel<<<(s.L * s.L + 255) / 256, 256, 0, st>>>(f.Cpart, parts, s.L, f.C);
  eig_c_kernel<<<1, FT, 0, st>>>(f.C, f.W, f.lam, f.sig, f.info, s.L);
  form_v_kernel<<<grid_for(s.n * k, 256), 256, 0, st>>>(f.Bt, f.W, f.sig, f.info, s.n, k, s.L, V_dev);
  sign_fix_kernel<<<k, FT, 0, st>>>(V_dev, s.n);
  prof->launches[SPCA_K_FINALIZE] += 8;   // the launches above beyond the one begin() counted
  prof->end(SPCA_K_FINALIZE, st);
  e = cudaMemcpyAsync(sigma_dev, f.sig, sizeof(double) * k, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace spca

// Eigensolve in the enriched coarse space (Alg. 2 step 4; Alg. 3 steps 1 and 5):
// the k pairs of (Ahat - sigma Mhat) y = theta Mhat y with smallest |theta|, for the
// block matrices of Sec. 4.1 (size n = N_1 + k).
//
// The enriched basis [Q | X] is M-orthonormalised (the b_h-orthogonalisation of
// Alg. 2 step 3) by a Cholesky factorisation of the unit-diagonal scaled Mhat with
// diagonal pivoting; pivots below kDropTol mark basis vectors that are (numerically)
// in the span of the ones already taken, and are dropped.  The reduced standard
// problem L^{-1} D (Ahat - sigma Mhat) D L^{-T} is diagonalised by cyclic Jacobi in
// round-robin (parallel) order.  One CTA, float64, all matrices in global memory.
#include <cmath>

#include "common.cuh"

namespace bmg {
namespace {

constexpr double kDropTol = 1e-12;
constexpr int kThreads = 512;
constexpr int kMaxSweeps = 30;

struct Work {
  double* S;    // n*n scaled mass, overwritten by the Schur complements
  double* L;    // n*n Cholesky factor, row = original index, column = pivot step
  double* C;    // n*n reduced matrix, then Jacobi iterate
  double* V;    // n*n Jacobi eigenvectors
  double* Z;    // n*n back-substituted selected vectors
  double* d;    // n scaling
};

__device__ void block_sync() { __syncthreads(); }

__global__ void __launch_bounds__(kThreads)
dense_eig_kernel(const double* __restrict__ Ahat, const double* __restrict__ Mhat, int n,
                 double sigma, int k, double* __restrict__ theta_out, double* __restrict__ Y,
                 int* __restrict__ rank_out, int* __restrict__ stats, Work w) {
  __shared__ int perm[320];
  __shared__ double red_v[kThreads];
  __shared__ int red_i[kThreads];
  __shared__ int s_rank;
  __shared__ double s_off, s_frob;
  __shared__ double cs_c[160], cs_s[160];
  __shared__ int pr_p[160], pr_q[160];
  __shared__ int order[320];
  __shared__ int s_sweeps;
  __shared__ unsigned long long s_rot;
  const int tid = threadIdx.x;
  if (tid == 0) { s_sweeps = 0; s_rot = 0ull; }

  // 1. scaling D = diag(Mhat)^(-1/2) and S = D Mhat D (symmetrised)
  for (int i = tid; i < n; i += kThreads) {
    const double mii = Mhat[i * n + i];
    w.d[i] = (mii > 0.0) ? 1.0 / sqrt(mii) : 0.0;
    perm[i] = i;
  }
  block_sync();
  for (int q = tid; q < n * n; q += kThreads) {
    const int i = q / n, j = q % n;
    w.S[q] = 0.5 * (Mhat[i * n + j] + Mhat[j * n + i]) * w.d[i] * w.d[j];
    w.L[q] = 0.0;
  }
  if (tid == 0) s_rank = n;
  block_sync();

  // 2. pivoted Cholesky of S (outer-product form on the permuted Schur complement)
  for (int j = 0; j < n; ++j) {
    double best = -1.0;
    int bi = j;
    for (int i = j + tid; i < n; i += kThreads) {
      const double v = w.S[perm[i] * n + perm[i]];
      if (v > best || (v == best && i < bi)) { best = v; bi = i; }
    }
    red_v[tid] = best;
    red_i[tid] = bi;
    block_sync();
    for (int off = kThreads / 2; off > 0; off >>= 1) {
      if (tid < off) {
        const double v2 = red_v[tid + off];
        const int i2 = red_i[tid + off];
        if (v2 > red_v[tid] || (v2 == red_v[tid] && i2 < red_i[tid])) { red_v[tid] = v2; red_i[tid] = i2; }
      }
      block_sync();
    }
    const double piv = red_v[0];
    const int pi = red_i[0];
    if (!(piv > kDropTol)) {  // also catches NaN
      if (tid == 0) s_rank = j;
      block_sync();
      break;
    }
    if (tid == 0) { const int t = perm[j]; perm[j] = perm[pi]; perm[pi] = t; }
    block_sync();
    const double ljj = sqrt(piv);
    const int pj = perm[j];
    for (int i = j + tid; i < n; i += kThreads) {
      w.L[perm[i] * n + j] = (i == j) ? ljj : w.S[perm[i] * n + pj] / ljj;
    }
    block_sync();
    const int m = n - j - 1;
    for (int q = tid; q < m * m; q += kThreads) {
      const int a = j + 1 + q / m, b = j + 1 + q % m;
      w.S[perm[a] * n + perm[b]] -= w.L[perm[a] * n + j] * w.L[perm[b] * n + j];
    }
    block_sync();
  }
  const int r = s_rank;
  if (tid == 0) {
    *rank_out = r;
    if (stats) { stats[0] = 0; stats[1] = 0; }
  }
  if (r < k) return;  // caller reports BMG_ERR_SINGULAR

  // 3. C = D (Ahat - sigma Mhat) D in pivot order, leading r x r block
  for (int q = tid; q < r * r; q += kThreads) {
    const int i = q / r, j = q % r;
    const int a = perm[i], b = perm[j];
    const double aij = 0.5 * (Ahat[a * n + b] + Ahat[b * n + a]);
    const double mij = 0.5 * (Mhat[a * n + b] + Mhat[b * n + a]);
    w.C[i * r + j] = (aij - sigma * mij) * w.d[a] * w.d[b];
  }
  block_sync();
  // 4. W = L^{-1} C (rows, forward substitution), stored in Z; then C = L^{-1} W^T
  for (int i = 0; i < r; ++i) {
    const double* Li = w.L + perm[i] * n;
    const double lii = Li[i];
    for (int c = tid; c < r; c += kThreads) {
      double s = w.C[i * r + c];
      for (int q = 0; q < i; ++q) s -= Li[q] * w.Z[q * r + c];
      w.Z[i * r + c] = s / lii;
    }
    block_sync();
  }
  for (int i = 0; i < r; ++i) {
    const double* Li = w.L + perm[i] * n;
    const double lii = Li[i];
    for (int c = tid; c < r; c += kThreads) {
      double s = w.Z[c * r + i];  // (W^T)[i][c]
      for (int q = 0; q < i; ++q) s -= Li[q] * w.C[q * r + c];
      w.C[i * r + c] = s / lii;
    }
    block_sync();
  }
  for (int q = tid; q < r * r; q += kThreads) {
    const int i = q / r, j = q % r;
    if (i < j) {
      const double v = 0.5 * (w.C[i * r + j] + w.C[j * r + i]);
      w.C[i * r + j] = v;
      w.C[j * r + i] = v;
    }
    w.V[q] = (i == j) ? 1.0 : 0.0;
  }
  block_sync();

  // 5. cyclic Jacobi, round-robin order (m/2 disjoint rotations per step)
  const int m = (r % 2 == 0) ? r : r + 1;
  for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
    if (tid == 0) { s_off = 0.0; s_frob = 0.0; }
    block_sync();
    double off = 0.0, fro = 0.0;
    for (int q = tid; q < r * r; q += kThreads) {
      const double v = w.C[q];
      fro += v * v;
      if (q / r != q % r) off += v * v;
    }
    red_v[tid] = off;
    block_sync();
    for (int o = kThreads / 2; o > 0; o >>= 1) { if (tid < o) red_v[tid] += red_v[tid + o]; block_sync(); }
    if (tid == 0) s_off = red_v[0];
    block_sync();
    red_v[tid] = fro;
    block_sync();
    for (int o = kThreads / 2; o > 0; o >>= 1) { if (tid < o) red_v[tid] += red_v[tid + o]; block_sync(); }
    if (tid == 0) s_frob = red_v[0];
    block_sync();
    if (s_off <= 1e-32 * s_frob || s_frob == 0.0) break;
    if (tid == 0) s_sweeps = sweep + 1;
    for (int step = 0; step < m - 1; ++step) {
      for (int i = tid; i < m / 2; i += kThreads) {
        auto player = [&](int t) { return t == 0 ? 0 : ((t - 1 + step) % (m - 1)) + 1; };
        int p = player(i), q = player(m - 1 - i);
        if (p > q) { const int t = p; p = q; q = t; }
        double c = 1.0, s = 0.0;
        if (q < r) {
          const double apq = w.C[p * r + q];
          const double app = w.C[p * r + p], aqq = w.C[q * r + q];
          if (apq != 0.0 && fabs(apq) > 1e-18 * sqrt(fabs(app * aqq))) {
            const double tau = (aqq - app) / (2.0 * apq);
            double t;
            if (fabs(tau) > 1e150) t = 0.5 / tau;
            else t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
            atomicAdd(&s_rot, 1ull);
          }
        }
        cs_c[i] = c; cs_s[i] = s; pr_p[i] = p; pr_q[i] = (q < r) ? q : -1;
      }
      block_sync();
      const int half = m / 2;
      for (int it = tid; it < half * r; it += kThreads) {  // rows p, q  <- J^T A
        const int i = it / r, col = it % r;
        const int p = pr_p[i], q = pr_q[i];
        if (q < 0 || cs_s[i] == 0.0) continue;
        const double c = cs_c[i], s = cs_s[i];
        const double ap = w.C[p * r + col], aq = w.C[q * r + col];
        w.C[p * r + col] = c * ap - s * aq;
        w.C[q * r + col] = s * ap + c * aq;
      }
      block_sync();
      for (int it = tid; it < half * r; it += kThreads) {  // columns p, q  <- A J ; V <- V J
        const int i = it / r, row = it % r;
        const int p = pr_p[i], q = pr_q[i];
        if (q < 0 || cs_s[i] == 0.0) continue;
        const double c = cs_c[i], s = cs_s[i];
        const double ap = w.C[row * r + p], aq = w.C[row * r + q];
        w.C[row * r + p] = c * ap - s * aq;
        w.C[row * r + q] = s * ap + c * aq;
        const double vp = w.V[row * r + p], vq = w.V[row * r + q];
        w.V[row * r + p] = c * vp - s * vq;
        w.V[row * r + q] = s * vp + c * vq;
      }
      block_sync();
    }
  }

  // 6. selection: ascending (|theta|, theta, index)
  for (int i = tid; i < r; i += kThreads) {
    const double ti = w.C[i * r + i];
    int rank = 0;
    for (int j = 0; j < r; ++j) {
      const double tj = w.C[j * r + j];
      const bool before = fabs(tj) < fabs(ti) || (fabs(tj) == fabs(ti) && (tj < ti || (tj == ti && j < i)));
      rank += before ? 1 : 0;
    }
    if (rank < k) order[rank] = i;
  }
  block_sync();
  for (int c = tid; c < k; c += kThreads) theta_out[c] = w.C[order[c] * r + order[c]];
  if (tid == 0 && stats) { stats[0] = s_sweeps; stats[1] = (int)s_rot; }
  // 7. Y = D P L^{-T} V_sel  (back substitution, parallel over the k columns)
  for (int i = r - 1; i >= 0; --i) {
    const double lii = w.L[perm[i] * n + i];
    for (int c = tid; c < k; c += kThreads) {
      double s = w.V[i * r + order[c]];
      for (int q = i + 1; q < r; ++q) s -= w.L[perm[q] * n + i] * w.Z[q * k + c];
      w.Z[i * k + c] = s / lii;
    }
    block_sync();
  }
  for (int q = tid; q < n * k; q += kThreads) {
    const int i = q / k, c = q % k;
    const int row = perm[i];
    Y[row * k + c] = (i < r) ? w.d[row] * w.Z[i * k + c] : 0.0;
  }
}
}  // namespace

size_t dense_work_doubles(int n) { return 5 * (size_t)n * n + n; }

void dense_eig(const double* Ahat, const double* Mhat, int n, double sigma, int k, double* theta,
               double* Y, int* rank, double* work, int* stats, cudaStream_t s) {
  if (n < 1 || n > 320 || k < 1 || k > n) fail(BMG_ERR_INVALID_ARG, "dense_eig: need 1 <= k <= n <= 320");
  Work w;
  w.S = work;
  w.L = w.S + (size_t)n * n;
  w.C = w.L + (size_t)n * n;
  w.V = w.C + (size_t)n * n;
  w.Z = w.V + (size_t)n * n;
  w.d = w.Z + (size_t)n * n;
  prof_begin(KC_DENSE, s);
  dense_eig_kernel<<<1, kThreads, 0, s>>>(Ahat, Mhat, n, sigma, k, theta, Y, rank, stats, w);
  check_launch("dense_eig_kernel");
  // nominal count of a dense symmetric-definite eigensolve with vectors (9 n^3)
  const double nn = n;
  prof_end(KC_DENSE, s, 16.0 * nn * nn + 8.0 * nn * k, 9.0 * nn * nn * nn);
}

}  // namespace bmg

// Eigensolve in the enriched coarse space (Alg. 2 step 4; Alg. 3 steps 1 and 5):
// the k pairs of (Ahat - sigma Mhat) y = theta Mhat y with smallest |theta|, for the
// block matrices of Sec. 4.1 (size n = N_1 + k <= 320).
//
// GB300 executes FP64 at about 1/70 of its FP32 rate, so a single CTA cannot afford
// the O(n^3) work of a dense eigensolver in FP64.  The solve is split:
//   1. [1 CTA, FP64]  M-orthonormal basis of the enriched space (the b_h-
//      orthogonalisation of Alg. 2 step 3): Mhat scaled to unit diagonal, Cholesky
//      with diagonal pivoting; pivots below kDropTol mark basis vectors already in
//      the span of the others, which are dropped (rank r).
//   2. [multi-CTA, FP64]  reduced standard matrix T = L^{-1} D P^T (Ahat - sigma
//      Mhat) P D L^{-T} by two forward substitutions (one warp per column).
//   3. [1 CTA, FP32]  cyclic Jacobi (round-robin order) on T in shared memory:
//      eigenvectors W accurate to FP32.
//   4. [multi-CTA, FP64]  refinement of W to FP64 accuracy by the iterative scheme
//      of Ogita & Aishima (2018) for symmetric eigendecompositions:
//          G = W^T W, R = I - G, S = W^T T W, lt_i = s_ii / (1 - r_ii),
//          E_ij = (s_ij + lt_j r_ij) / (lt_j - lt_i) for well separated pairs,
//          r_ij / 2 otherwise,   W <- W (I + E);
//      pairs closer than the FP32 resolution form clusters whose m x m block is
//      diagonalised exactly (FP64 Jacobi) once the separated pairs have converged,
//      then one more step polishes the couplings.
//   5. [multi-CTA, FP64]  selection of the k smallest |theta| and back-transform
//      Y = D P L^{-T} W_sel (back substitution, one warp per column).
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace bmg {
namespace {

constexpr double kDropTol = 1e-12;
constexpr double kClusterFloor = 1e-3;   // relative gap below which the FP32 start cannot separate pairs
constexpr double kGuard = 0.05;          // largest first-order correction accepted by a step
constexpr int kCholThreads = 512;
constexpr int kJacThreads = 1024;
constexpr int kMaxN = 320;
constexpr int kMaxCluster = 40;   // larger clusters keep the orthonormalising step only

// Scratch carved from one device allocation; n x n blocks row-major, stride n.
struct DW {
  double *S, *L, *T, *Z, *W, *W2, *G, *SS, *E, *P, *d, *lam, *misc;
  int* perm;
  int* order;
  int* rank;
};

// ------------------------------------------------- 1. pivoted Cholesky (FP64) --
__global__ void __launch_bounds__(kCholThreads)
chol_kernel(const double* __restrict__ Mhat, int n, DW w) {
  __shared__ double red_v[kCholThreads];
  __shared__ int red_i[kCholThreads];
  __shared__ int perm[kMaxN];
  __shared__ int s_rank;
  const int tid = threadIdx.x;
  for (int i = tid; i < n; i += kCholThreads) {
    const double mii = Mhat[i * n + i];
    w.d[i] = (mii > 0.0) ? 1.0 / sqrt(mii) : 0.0;
    perm[i] = i;
  }
  __syncthreads();
  for (int q = tid; q < n * n; q += kCholThreads) {
    const int i = q / n, j = q % n;
    w.S[q] = 0.5 * (Mhat[i * n + j] + Mhat[j * n + i]) * w.d[i] * w.d[j];
    w.L[q] = 0.0;
  }
  if (tid == 0) s_rank = n;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    double best = -1.0;
    int bi = j;
    for (int i = j + tid; i < n; i += kCholThreads) {
      const double v = w.S[perm[i] * n + perm[i]];
      if (v > best || (v == best && i < bi)) { best = v; bi = i; }
    }
    red_v[tid] = best;
    red_i[tid] = bi;
    __syncthreads();
    for (int off = kCholThreads / 2; off > 0; off >>= 1) {
      if (tid < off) {
        const double v2 = red_v[tid + off];
        const int i2 = red_i[tid + off];
        if (v2 > red_v[tid] || (v2 == red_v[tid] && i2 < red_i[tid])) { red_v[tid] = v2; red_i[tid] = i2; }
      }
      __syncthreads();
    }
    const double piv = red_v[0];
    const int pi = red_i[0];
    __syncthreads();
    if (!(piv > kDropTol)) {  // also catches NaN
      if (tid == 0) s_rank = j;
      __syncthreads();
      break;
    }
    if (tid == 0) { const int t = perm[j]; perm[j] = perm[pi]; perm[pi] = t; }
    __syncthreads();
    const double ljj = sqrt(piv);
    const int pj = perm[j];
    for (int i = j + tid; i < n; i += kCholThreads)
      w.L[perm[i] * n + j] = (i == j) ? ljj : w.S[perm[i] * n + pj] / ljj;
    __syncthreads();
    const int m = n - j - 1;
    for (int q = tid; q < m * m; q += kCholThreads) {
      const int a = j + 1 + q / m, b = j + 1 + q % m;
      if (b < a) continue;  // update the upper triangle and mirror it
      const double v = w.S[perm[a] * n + perm[b]] - w.L[perm[a] * n + j] * w.L[perm[b] * n + j];
      w.S[perm[a] * n + perm[b]] = v;
      w.S[perm[b] * n + perm[a]] = v;
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += kCholThreads) w.perm[i] = perm[i];
  if (tid == 0) *w.rank = s_rank;
}

// --------------------------------------- 2. T = L^{-1} C L^{-T} (FP64, warps) --
// pass 0: Z = L^{-1} C with C[i][c] = d_a (Ahat - sigma Mhat)_ab d_b, a = perm[i],
//         b = perm[c] (symmetrised);  pass 1: T = L^{-1} Z^T.
// One warp per column c; the rows run in order, lanes share each dot product.
__global__ void trsm_fwd_kernel(const double* __restrict__ Ahat, const double* __restrict__ Mhat,
                                int n, double sigma, int pass, DW w) {
  const int r = *w.rank;
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= r) return;
  double* out = pass == 0 ? w.Z : w.T;
  const int* perm = w.perm;
  for (int i = 0; i < r; ++i) {
    const double* Li = w.L + perm[i] * n;
    double s = 0.0;
    for (int q = lane; q < i; q += 32) s += Li[q] * out[q * n + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      double rhs;
      if (pass == 0) {
        const int a = perm[i], b = perm[c];
        const double aij = 0.5 * (Ahat[a * n + b] + Ahat[b * n + a]);
        const double mij = 0.5 * (Mhat[a * n + b] + Mhat[b * n + a]);
        rhs = (aij - sigma * mij) * w.d[a] * w.d[b];
      } else {
        rhs = w.Z[c * n + i];
      }
      out[i * n + c] = (rhs - s) / Li[i];
    }
    __syncwarp();
  }
}

// ------------------------------------------------ 3. FP32 Jacobi (1 CTA) ------
// Round-robin parallel cyclic Jacobi on a float copy of T held in shared memory
// (2 r^2 floats) or in global scratch when it does not fit.
__global__ void __launch_bounds__(kJacThreads)
jacobi32_kernel(int n, int use_smem, float* __restrict__ gscratch, DW w, int max_sweeps, float tol) {
  extern __shared__ float sm[];
  __shared__ float cs_c[kMaxN / 2], cs_s[kMaxN / 2];
  __shared__ int pr_p[kMaxN / 2], pr_q[kMaxN / 2];
  __shared__ float red[kJacThreads / 32][2];
  __shared__ float s_off, s_fro;
  const int r = *w.rank;
  const int tid = threadIdx.x;
  float* A = use_smem ? sm : gscratch;
  float* V = A + r * r;
  for (int q = tid; q < r * r; q += kJacThreads) {
    const int i = q / r, j = q % r;
    A[q] = (float)(0.5 * (w.T[i * n + j] + w.T[j * n + i]));
    V[q] = (i == j) ? 1.f : 0.f;
  }
  __syncthreads();
  const int m = (r % 2 == 0) ? r : r + 1;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    float off = 0.f, fro = 0.f;
    for (int q = tid; q < r * r; q += kJacThreads) {
      const float v = A[q];
      fro += v * v;
      if (q / r != q % r) off += v * v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      fro += __shfl_xor_sync(0xffffffffu, fro, o);
    }
    if ((tid & 31) == 0) { red[tid >> 5][0] = off; red[tid >> 5][1] = fro; }
    __syncthreads();
    if (tid == 0) {
      float a = 0.f, b = 0.f;
      for (int q = 0; q < kJacThreads / 32; ++q) { a += red[q][0]; b += red[q][1]; }
      s_off = a;
      s_fro = b;
    }
    __syncthreads();
    if (s_off <= tol * tol * s_fro || s_fro == 0.f) break;
    for (int step = 0; step < m - 1; ++step) {
      for (int i = tid; i < m / 2; i += kJacThreads) {
        auto player = [&](int t) { return t == 0 ? 0 : ((t - 1 + step) % (m - 1)) + 1; };
        int p = player(i), q = player(m - 1 - i);
        if (p > q) { const int t = p; p = q; q = t; }
        float c = 1.f, s = 0.f;
        if (q < r) {
          const float apq = A[p * r + q];
          const float app = A[p * r + p], aqq = A[q * r + q];
          if (apq != 0.f && fabsf(apq) > 1e-12f * sqrtf(fabsf(app * aqq))) {
            const float tau = (aqq - app) / (2.f * apq);
            const float t = (fabsf(tau) > 1e18f) ? 0.5f / tau
                                                  : copysignf(1.f, tau) / (fabsf(tau) + sqrtf(1.f + tau * tau));
            c = 1.f / sqrtf(1.f + t * t);
            s = t * c;
          }
        }
        cs_c[i] = c; cs_s[i] = s; pr_p[i] = p; pr_q[i] = (q < r && s != 0.f) ? q : -1;
      }
      __syncthreads();
      const int half = m / 2;
      for (int it = tid; it < half * r; it += kJacThreads) {   // rows p, q  <- J^T A
        const int i = it / r, col = it % r;
        const int q = pr_q[i];
        if (q < 0) continue;
        const int p = pr_p[i];
        const float c = cs_c[i], s = cs_s[i];
        const float ap = A[p * r + col], aq = A[q * r + col];
        A[p * r + col] = c * ap - s * aq;
        A[q * r + col] = s * ap + c * aq;
      }
      __syncthreads();
      for (int it = tid; it < half * r; it += kJacThreads) {   // columns p, q <- A J ; V <- V J
        const int i = it / r, row = it % r;
        const int q = pr_q[i];
        if (q < 0) continue;
        const int p = pr_p[i];
        const float c = cs_c[i], s = cs_s[i];
        const float ap = A[row * r + p], aq = A[row * r + q];
        A[row * r + p] = c * ap - s * aq;
        A[row * r + q] = s * ap + c * aq;
        const float vp = V[row * r + p], vq = V[row * r + q];
        V[row * r + p] = c * vp - s * vq;
        V[row * r + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  for (int q = tid; q < r * r; q += kJacThreads) {
    const int i = q / r, j = q % r;
    w.W[i * n + j] = (double)V[q];
  }
}

// ------------------------------------------------ small FP64 GEMM (tiles) -----
// C = alpha * op(A) * B + beta * D  (m x p; inner q).  op(A) = A (m x q) or A^T
// (A stored q x m).  A negative size means the rank r.
constexpr int kT = 16;
template <bool TA>
__global__ void __launch_bounds__(kT * kT)
gemm64_kernel(int m, int p, int q, const double* __restrict__ A, int lda,
              const double* __restrict__ B, int ldb, double* C, int ldc, double alpha, double beta,
              const double* D, int ldd, const int* __restrict__ rank) {
  __shared__ double As[kT][kT + 1], Bs[kT][kT + 1];
  const int r = *rank;
  if (m < 0) m = r;
  if (p < 0) p = r;
  if (q < 0) q = r;
  if (blockIdx.y * kT >= m || blockIdx.x * kT >= p) return;   // whole block
  const int ty = threadIdx.x / kT, tx = threadIdx.x % kT;
  const int row = blockIdx.y * kT + ty, col = blockIdx.x * kT + tx;
  double acc = 0.0;
  for (int k0 = 0; k0 < q; k0 += kT) {
    const int ka = k0 + tx, kb = k0 + ty;
    if (TA) As[ty][tx] = (row < m && ka < q) ? A[ka * lda + row] : 0.0;
    else    As[ty][tx] = (row < m && ka < q) ? A[row * lda + ka] : 0.0;
    Bs[ty][tx] = (kb < q && col < p) ? B[kb * ldb + col] : 0.0;
    __syncthreads();
#pragma unroll
    for (int t = 0; t < kT; ++t) acc = fma(As[ty][t], Bs[t][tx], acc);
    __syncthreads();
  }
  if (row < m && col < p) {
    double v = alpha * acc;
    if (beta != 0.0) v += beta * D[row * ldd + col];
    C[row * ldc + col] = v;
  }
}

// ------------------------------------------------- 4. refinement step (1 CTA) --
// From G = W^T W and SS = W^T T W: lam (Rayleigh quotients) and the update E
// (W <- W + W E).
//   mode 0: Ogita-Aishima step; pairs with gap <= max(delta, floor * max|lam|)
//           only get the orthonormalising term.
//   mode 1: clusters (chains of sorted lam with gaps <= the same threshold) are
//           orthonormalised to first order and their blocks diagonalised exactly
//           by FP64 Jacobi; E = blockdiag(F_c) - I.
//   mode 2: lam and the error estimate only.
constexpr int kOAThreads = 1024;
__global__ void __launch_bounds__(kOAThreads)
oa_kernel(int n, int mode, double floor_rel, DW w) {
  __shared__ double red[kOAThreads / 32][3];
  __shared__ double s_delta, s_amax;
  __shared__ int srt[kMaxN];
  __shared__ int cl_start[kMaxN + 1];
  __shared__ int s_ncl;
  __shared__ double cA[kMaxCluster * kMaxCluster], cV[kMaxCluster * kMaxCluster];
  __shared__ double cK[kMaxCluster * kMaxCluster];
  __shared__ double ccs_c[kMaxCluster / 2], ccs_s[kMaxCluster / 2];
  __shared__ int cpr_p[kMaxCluster / 2], cpr_q[kMaxCluster / 2];
  __shared__ double s_toff, s_tfro;
  const int r = *w.rank;
  const int tid = threadIdx.x;
  // G and SS come from separate products and are symmetric only to rounding; the
  // update needs E + E^T = R exactly for pairs with tiny gaps, so use their
  // symmetric parts.
  auto Gs = [&](int i, int j) { return 0.5 * (w.G[i * n + j] + w.G[j * n + i]); };
  auto Ss = [&](int i, int j) { return 0.5 * (w.SS[i * n + j] + w.SS[j * n + i]); };
  for (int i = tid; i < r; i += kOAThreads) {
    const double gii = w.G[i * n + i];
    w.lam[i] = w.SS[i * n + i] / (2.0 - gii);   // s_ii / (1 - r_ii) with r = I - G
  }
  __syncthreads();
  double nS = 0.0, nR = 0.0, amax = 0.0;
  for (int q = tid; q < r * r; q += kOAThreads) {
    const int i = q / r, j = q % r;
    const double rij = (i == j ? 1.0 : 0.0) - Gs(i, j);
    const double sij = Ss(i, j) - (i == j ? w.lam[i] : 0.0);
    nS += sij * sij;
    nR += rij * rij;
    if (i == j) amax = fmax(amax, fabs(w.lam[i]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nS += __shfl_xor_sync(0xffffffffu, nS, o);
    nR += __shfl_xor_sync(0xffffffffu, nR, o);
    amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  }
  if ((tid & 31) == 0) { red[tid >> 5][0] = nS; red[tid >> 5][1] = nR; red[tid >> 5][2] = amax; }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int q = 0; q < kOAThreads / 32; ++q) { a += red[q][0]; b += red[q][1]; c = fmax(c, red[q][2]); }
    s_delta = 2.0 * (sqrt(a) + c * sqrt(b));
    s_amax = c;
    w.misc[0] = s_delta;
    w.misc[1] = (c > 0.0) ? (sqrt(a) / c + sqrt(b)) : sqrt(b);   // relative error estimate
  }
  __syncthreads();
  if (mode == 2) return;
  const double thr = fmax(s_delta, floor_rel * s_amax);
  if (mode == 0) {
    for (int q = tid; q < r * r; q += kOAThreads) {
      const int i = q / r, j = q % r;
      const double rij = (i == j ? 1.0 : 0.0) - Gs(i, j);
      double e = 0.5 * rij;
      if (i != j) {
        const double li = w.lam[i], lj = w.lam[j];
        if (fabs(li - lj) > thr) {
          const double t = (Ss(i, j) + lj * rij) / (lj - li);
          if (fabs(t) < kGuard) e = t;   // outside the convergence region: leave to clusters
        }
      }
      w.E[i * n + j] = e;
    }
    return;
  }
  // mode 1
  for (int i = tid; i < r; i += kOAThreads) {
    const double li = w.lam[i];
    int rk = 0;
    for (int j = 0; j < r; ++j) {
      const double lj = w.lam[j];
      rk += (lj < li || (lj == li && j < i)) ? 1 : 0;
    }
    srt[rk] = i;
  }
  for (int q = tid; q < r * r; q += kOAThreads) {
    const int i = q / r, j = q % r;
    w.E[i * n + j] = (i == j) ? 0.5 * (1.0 - w.G[i * n + i]) : 0.0;
  }
  __syncthreads();
  if (tid == 0) {
    int nc = 0;
    cl_start[nc++] = 0;
    for (int t = 1; t < r; ++t)
      if (!(w.lam[srt[t]] - w.lam[srt[t - 1]] <= thr)) cl_start[nc++] = t;
    cl_start[nc] = r;
    s_ncl = nc;
  }
  __syncthreads();
  for (int c = 0; c < s_ncl; ++c) {
    const int b = cl_start[c], mm = cl_start[c + 1] - b;
    if (mm < 2 || mm > kMaxCluster) continue;   // singletons keep the normalisation
    // K = I + R_c / 2 (first-order G_c^{-1/2});  cA = K S_c K
    for (int q = tid; q < mm * mm; q += kOAThreads) {
      const int a = q / mm, e = q % mm;
      cK[q] = (a == e ? 1.5 : 0.0) - 0.5 * Gs(srt[b + a], srt[b + e]);
    }
    __syncthreads();
    for (int q = tid; q < mm * mm; q += kOAThreads) {   // cV = K S_c (temporary)
      const int a = q / mm, e = q % mm;
      double s = 0.0;
      for (int u = 0; u < mm; ++u) s += cK[a * mm + u] * Ss(srt[b + u], srt[b + e]);
      cV[q] = s;
    }
    __syncthreads();
    for (int q = tid; q < mm * mm; q += kOAThreads) {
      const int a = q / mm, e = q % mm;
      double s = 0.0;
      for (int u = 0; u < mm; ++u) s += cV[a * mm + u] * cK[u * mm + e];
      cA[q] = s;
    }
    __syncthreads();
    for (int q = tid; q < mm * mm; q += kOAThreads) {
      const int a = q / mm, e = q % mm;
      if (a < e) {
        const double v = 0.5 * (cA[a * mm + e] + cA[e * mm + a]);
        cA[a * mm + e] = v;
        cA[e * mm + a] = v;
      }
    }
    __syncthreads();
    for (int q = tid; q < mm * mm; q += kOAThreads) cV[q] = (q / mm == q % mm) ? 1.0 : 0.0;
    __syncthreads();
    const int m2 = (mm % 2 == 0) ? mm : mm + 1;
    for (int sweep = 0; sweep < 30; ++sweep) {
      if (tid == 0) {
        double off = 0.0, fro = 0.0;
        for (int q = 0; q < mm * mm; ++q) {
          fro += cA[q] * cA[q];
          if (q / mm != q % mm) off += cA[q] * cA[q];
        }
        s_toff = off;
        s_tfro = fro;
      }
      __syncthreads();
      if (s_toff <= 1e-32 * s_tfro || s_tfro == 0.0) break;
      for (int step = 0; step < m2 - 1; ++step) {
        if (tid < m2 / 2) {
          const int i = tid;
          auto player = [&](int t) { return t == 0 ? 0 : ((t - 1 + step) % (m2 - 1)) + 1; };
          int p = player(i), q = player(m2 - 1 - i);
          if (p > q) { const int t = p; p = q; q = t; }
          double cc = 1.0, ss = 0.0;
          if (q < mm) {
            const double apq = cA[p * mm + q], app = cA[p * mm + p], aqq = cA[q * mm + q];
            if (apq != 0.0) {
              const double tau = (aqq - app) / (2.0 * apq);
              const double t = (fabs(tau) > 1e150) ? 0.5 / tau
                                                    : copysign(1.0, tau) / (fabs(tau) + sqrt(1.0 + tau * tau));
              cc = 1.0 / sqrt(1.0 + t * t);
              ss = t * cc;
            }
          }
          ccs_c[i] = cc; ccs_s[i] = ss; cpr_p[i] = p; cpr_q[i] = (q < mm && ss != 0.0) ? q : -1;
        }
        __syncthreads();
        const int half = m2 / 2;
        for (int it = tid; it < half * mm; it += kOAThreads) {
          const int i = it / mm, col = it % mm;
          const int q = cpr_q[i];
          if (q < 0) continue;
          const int p = cpr_p[i];
          const double cc = ccs_c[i], ss = ccs_s[i];
          const double ap = cA[p * mm + col], aq = cA[q * mm + col];
          cA[p * mm + col] = cc * ap - ss * aq;
          cA[q * mm + col] = ss * ap + cc * aq;
        }
        __syncthreads();
        for (int it = tid; it < half * mm; it += kOAThreads) {
          const int i = it / mm, row = it % mm;
          const int q = cpr_q[i];
          if (q < 0) continue;
          const int p = cpr_p[i];
          const double cc = ccs_c[i], ss = ccs_s[i];
          const double ap = cA[row * mm + p], aq = cA[row * mm + q];
          cA[row * mm + p] = cc * ap - ss * aq;
          cA[row * mm + q] = ss * ap + cc * aq;
          const double vp = cV[row * mm + p], vq = cV[row * mm + q];
          cV[row * mm + p] = cc * vp - ss * vq;
          cV[row * mm + q] = ss * vp + cc * vq;
        }
        __syncthreads();
      }
    }
    // F_c = K V ; E block = F_c - I (indices through srt)
    for (int q = tid; q < mm * mm; q += kOAThreads) {
      const int a = q / mm, e = q % mm;
      double s = 0.0;
      for (int u = 0; u < mm; ++u) s += cK[a * mm + u] * cV[u * mm + e];
      w.E[srt[b + a] * n + srt[b + e]] = s - (a == e ? 1.0 : 0.0);
    }
    __syncthreads();
  }
}

// ------------------------------------------- 5. selection and back-transform --
// order[0..k) = indices of the k smallest |lam| (ties: value, then index).
__global__ void select_kernel(int k, DW w, double* __restrict__ theta) {
  const int r = *w.rank;
  for (int c = threadIdx.x; c < k; c += blockDim.x) w.order[c] = 0;   // rank < k: stays in bounds
  __syncthreads();
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    const double li = w.lam[i];
    int rk = 0;
    for (int j = 0; j < r; ++j) {
      const double lj = w.lam[j];
      rk += (fabs(lj) < fabs(li) || (fabs(lj) == fabs(li) && (lj < li || (lj == li && j < i)))) ? 1 : 0;
    }
    if (rk < k) w.order[rk] = i;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < k; c += blockDim.x) theta[c] = w.lam[w.order[c]];
}

// Z = L^{-T} W_sel (back substitution, one warp per selected column), then
// Y[perm[i]][c] = d[perm[i]] Z[i][c] for i < r and 0 for the dropped rows.
__global__ void backsub_kernel(int n, int k, DW w, double* __restrict__ Y) {
  const int r = *w.rank;
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= k) return;
  const int* perm = w.perm;
  const int oc = w.order[c];
  for (int i = r - 1; i >= 0; --i) {
    double s = 0.0;
    for (int q = i + 1 + lane; q < r; q += 32) s += w.L[perm[q] * n + i] * w.Z[q * n + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) w.Z[i * n + c] = (w.W[i * n + oc] - s) / w.L[perm[i] * n + i];
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) {
    const int row = perm[i];
    Y[row * k + c] = (i < r) ? w.d[row] * w.Z[i * n + c] : 0.0;
  }
}

__global__ void copy_out_kernel(DW w, int* rank_out, double* quality) {
  *rank_out = *w.rank;
  if (quality) *quality = w.misc[1];
}

DW carve(double* work, int n) {
  DW w;
  const size_t nn = (size_t)n * n;
  double* p = work;
  w.S = p; p += nn;
  w.L = p; p += nn;
  w.T = p; p += nn;
  w.Z = p; p += nn;
  w.W = p; p += nn;
  w.W2 = p; p += nn;
  w.G = p; p += nn;
  w.SS = p; p += nn;
  w.E = p; p += nn;
  w.P = p; p += nn;
  w.d = p; p += n;
  w.lam = p; p += n;
  w.misc = p; p += 8;
  w.perm = reinterpret_cast<int*>(p); p += n / 2 + 1;
  w.order = reinterpret_cast<int*>(p); p += n / 2 + 1;
  w.rank = reinterpret_cast<int*>(p); p += 1;
  return w;
}

float* float_scratch(const DW& w) { return reinterpret_cast<float*>(w.rank + 2); }

void gemm64(bool ta, const double* A, const double* B, double* C, double beta, const double* D,
            const DW& w, int n, cudaStream_t s) {
  dim3 grid((n + kT - 1) / kT, (n + kT - 1) / kT);
  if (ta) gemm64_kernel<true><<<grid, kT * kT, 0, s>>>(-1, -1, -1, A, n, B, n, C, n, 1.0, beta, D, n, w.rank);
  else    gemm64_kernel<false><<<grid, kT * kT, 0, s>>>(-1, -1, -1, A, n, B, n, C, n, 1.0, beta, D, n, w.rank);
  check_launch("gemm64_kernel");
}

}  // namespace

size_t dense_work_doubles(int n) {
  // 10 n^2 blocks, d, lam, misc, perm, order, rank, then 2 n^2 floats for the Jacobi
  return 10 * (size_t)n * n + 2 * (size_t)n + 8 + 2 * (size_t)(n / 2 + 1) + 1 + (size_t)n * n + 16;
}

void dense_eig(const double* Ahat, const double* Mhat, int n, double sigma, int k, double* theta,
               double* Y, int* rank, double* work, double* quality, cudaStream_t s) {
  if (n < 1 || n > kMaxN || k < 1 || k > n) fail(BMG_ERR_INVALID_ARG, "dense_eig: need 1 <= k <= n <= 320");
  prof_begin(KC_DENSE, s);
  DW w = carve(work, n);
  // 1. basis
  chol_kernel<<<1, kCholThreads, 0, s>>>(Mhat, n, w);
  check_launch("chol_kernel");
  // 2. reduced standard matrix
  const int wpb = 8;
  trsm_fwd_kernel<<<(n + wpb - 1) / wpb, 32 * wpb, 0, s>>>(Ahat, Mhat, n, sigma, 0, w);
  check_launch("trsm_fwd_kernel");
  trsm_fwd_kernel<<<(n + wpb - 1) / wpb, 32 * wpb, 0, s>>>(Ahat, Mhat, n, sigma, 1, w);
  check_launch("trsm_fwd_kernel");
  // 3. FP32 Jacobi
  const size_t smem = 2 * (size_t)n * n * sizeof(float);
  const bool use_smem = smem <= 200 * 1024;
  if (use_smem)
    BMG_CUDA(cudaFuncSetAttribute(jacobi32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // run to the FP32 resolution: the refinement needs eigenvectors good to ~1e-6 of
  // the gaps it separates
  jacobi32_kernel<<<1, kJacThreads, use_smem ? smem : 0, s>>>(n, use_smem ? 1 : 0, float_scratch(w), w, 10,
                                                              2e-7f);
  check_launch("jacobi32_kernel");
  // 4. refinement schedule: steps separate pairs farther apart than a floor (relative
  //    to max|lam|); cluster steps diagonalise the groups below it exactly.  The
  //    floor starts at the FP32 resolution of W and is lowered once the separated
  //    pairs converged; pairs closer than 1e-10 max|lam| are left to the cluster
  //    steps (their computed couplings are rounding noise).
  const int nsteps = 7;
  const int modes[nsteps] = {0, 0, 1, 0, 0, 1, 0};
  const double floors[nsteps] = {kClusterFloor, kClusterFloor, kClusterFloor, 1e-7, 1e-7, 1e-7, 1e-10};
  for (int it = 0; it < nsteps; ++it) {
    gemm64(false, w.T, w.W, w.P, 0.0, nullptr, w, n, s);    // P = T W
    gemm64(true, w.W, w.P, w.SS, 0.0, nullptr, w, n, s);    // SS = W^T P
    gemm64(true, w.W, w.W, w.G, 0.0, nullptr, w, n, s);     // G = W^T W
    oa_kernel<<<1, kOAThreads, 0, s>>>(n, modes[it], floors[it], w);
    check_launch("oa_kernel");
    gemm64(false, w.W, w.E, w.W2, 1.0, w.W, w, n, s);       // W2 = W + W E
    std::swap(w.W, w.W2);
  }
  gemm64(false, w.T, w.W, w.P, 0.0, nullptr, w, n, s);
  gemm64(true, w.W, w.P, w.SS, 0.0, nullptr, w, n, s);
  gemm64(true, w.W, w.W, w.G, 0.0, nullptr, w, n, s);
  oa_kernel<<<1, kOAThreads, 0, s>>>(n, 2, 0.0, w);
  check_launch("oa_kernel");
  // 5. selection and back-transform
  select_kernel<<<1, 512, 0, s>>>(k, w, theta);
  check_launch("select_kernel");
  backsub_kernel<<<(k + wpb - 1) / wpb, 32 * wpb, 0, s>>>(n, k, w, Y);
  check_launch("backsub_kernel");
  copy_out_kernel<<<1, 1, 0, s>>>(w, rank, quality);
  check_launch("copy_out_kernel");
  const double nn = n;
  prof_end(KC_DENSE, s, 16.0 * nn * nn + 8.0 * nn * k, 9.0 * nn * nn * nn);
}

}  // namespace bmg

// Per-cycle kernels of the BMG cycle on k-interleaved vector blocks.
//
// A block of k vectors on a level with N vertices is stored row-major [N][ld]: the
// ld values of one vertex are contiguous, so every CSR neighbour access reads whole
// 16-byte chunks of one row (double2 in FP64, float4 in FP32) and a warp reads one
// or more full rows.  One warp processes one matrix row; lane l owns the chunks
// l, l+32, ... of that row.  Both operators of the pencil share one CSR pattern and
// are applied in one pass.
//
// Every kernel exists for FP64 blocks (the plain method) and FP32 blocks (the
// precision form: FP32 storage, FP32 matrix values and FP32 arithmetic).  The Gram
// products of FP32 blocks are accumulated without rounding loss (exact products and
// compensated sums), so their results carry FP64-class accuracy.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"

namespace bmg {
namespace {

constexpr int kWarpsPerBlock = 8;

// 16-byte chunks of a row: W values of type T.
template <typename T> struct Chunk;
template <> struct Chunk<double> { static constexpr int W = 2; };
template <> struct Chunk<float> { static constexpr int W = 4; };

__device__ __forceinline__ void ldv(const double* p, size_t i, double (&v)[2]) {
  const double2 t = reinterpret_cast<const double2*>(p)[i];
  v[0] = t.x; v[1] = t.y;
}
__device__ __forceinline__ void ldv(const float* p, size_t i, float (&v)[4]) {
  const float4 t = reinterpret_cast<const float4*>(p)[i];
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
// Gathers of X through the read-only path (X is not written by other threads during
// a launch: Jacobi and the residual write another block, a Gauss-Seidel sweep writes
// only rows of the current colour, which are never neighbours of each other).
__device__ __forceinline__ void ldv_ro(const double* p, size_t i, double (&v)[2]) {
  const double2 t = __ldg(reinterpret_cast<const double2*>(p) + i);
  v[0] = t.x; v[1] = t.y;
}
__device__ __forceinline__ void ldv_ro(const float* p, size_t i, float (&v)[4]) {
  const float4 t = __ldg(reinterpret_cast<const float4*>(p) + i);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
// Output rows are written once and not read again in the launch: streaming stores,
// so that they do not evict the gathered block from L2.
__device__ __forceinline__ void stv_cs(double* p, size_t i, const double (&v)[2]) {
  __stcs(reinterpret_cast<double2*>(p) + i, make_double2(v[0], v[1]));
}
__device__ __forceinline__ void stv_cs(float* p, size_t i, const float (&v)[4]) {
  __stcs(reinterpret_cast<float4*>(p) + i, make_float4(v[0], v[1], v[2], v[3]));
}
__device__ __forceinline__ void stv(double* p, size_t i, const double (&v)[2]) {
  reinterpret_cast<double2*>(p)[i] = make_double2(v[0], v[1]);
}
__device__ __forceinline__ void stv(float* p, size_t i, const float (&v)[4]) {
  reinterpret_cast<float4*>(p)[i] = make_float4(v[0], v[1], v[2], v[3]);
}

// aa += A_row X, mm += M_row X for one CSR row owned by LPR lanes (pattern and values
// streamed, neighbour rows of X gathered through the read-only path).  The row's
// nonzeros are taken G at a time: lane q of the row's lanes loads nonzero q's column
// and values (one coalesced load each), the columns are broadcast by shuffles and all
// G neighbour gathers are issued before the first multiply, so a warp keeps G gathers
// in flight instead of one dependent load chain per nonzero.  The products are added
// in the order of the nonzeros, as one nonzero at a time would.  Every lane of the
// warp must call this (len = 0 for lanes without a row): the loop bound is the
// warp's longest row.  (float32 blocks; float64 blocks take one nonzero at a time.)
template <typename T, int LPR, int CPL>
struct GatherWidth {
  static constexpr int regs = CPL * Chunk<T>::W * (int)(sizeof(T) / 4);   // 32-bit registers per nonzero
  static constexpr int G0 = 32 / regs < 2 ? 2 : 32 / regs;
  static constexpr int G = G0 < LPR ? G0 : LPR;
};
template <typename T, int LPR, int CPL, bool WITH_M = true>
__device__ __forceinline__ void gather_row(const int* __restrict__ col, const T* __restrict__ va,
                                           const T* __restrict__ vm, const T* __restrict__ X, int b, int len,
                                           int nch, int sl, T (&aa)[CPL][Chunk<T>::W],
                                           T (&mm)[CPL][Chunk<T>::W]) {
  // WITH_M = false: only A x (mm untouched), for shifted problems with shift 0
  constexpr int W = Chunk<T>::W;
  if (sizeof(T) == 8) {
    // float64 blocks: the sweeps are bound by the FP64 pipe, not by memory latency,
    // so one nonzero at a time (no shuffles competing for issue slots)
    for (int p = b; p < b + len; ++p) {
      const int j = __ldcs(col + p);
      const T a = __ldcs(va + p), m = WITH_M ? __ldcs(vm + p) : T(0);
#pragma unroll
      for (int u = 0; u < CPL; ++u) {
        const int c = sl + LPR * u;
        if (c < nch) {
          T x[W];
          ldv_ro(X, (size_t)j * nch + c, x);
#pragma unroll
          for (int z = 0; z < W; ++z) {
            aa[u][z] = fma(a, x[z], aa[u][z]);
            if (WITH_M) mm[u][z] = fma(m, x[z], mm[u][z]);
          }
        }
      }
    }
    return;
  }
  constexpr int G = GatherWidth<T, LPR, CPL>::G;
  const int maxlen = __reduce_max_sync(0xffffffffu, len);
  for (int p0 = 0; p0 < maxlen; p0 += G) {
    const int cnt = len - p0;
    int jl = 0;
    T al = T(0), ml = T(0);
    if (sl < G && sl < cnt) {
      jl = __ldcs(col + b + p0 + sl);
      al = __ldcs(va + b + p0 + sl);
      if (WITH_M) ml = __ldcs(vm + b + p0 + sl);
    }
    T x[G][CPL][W];
#pragma unroll
    for (int q = 0; q < G; ++q) {
      const int j = __shfl_sync(0xffffffffu, jl, q, LPR);
#pragma unroll
      for (int u = 0; u < CPL; ++u) {
        const int c = sl + LPR * u;
        if (q < cnt && c < nch) {
          ldv_ro(X, (size_t)j * nch + c, x[q][u]);
        } else {
#pragma unroll
          for (int z = 0; z < W; ++z) x[q][u][z] = T(0);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < G; ++q) {
      const T a = __shfl_sync(0xffffffffu, al, q, LPR);
      const T m = WITH_M ? __shfl_sync(0xffffffffu, ml, q, LPR) : T(0);
      if (q < cnt) {
#pragma unroll
        for (int u = 0; u < CPL; ++u)
          if (sl + LPR * u < nch) {
#pragma unroll
            for (int z = 0; z < W; ++z) {
              aa[u][z] = fma(a, x[q][u][z], aa[u][z]);
              if (WITH_M) mm[u][z] = fma(m, x[q][u][z], mm[u][z]);
            }
          }
      }
    }
  }
}

// 1/d for the smoother update.  FP64: an FP32 seed refined by two Newton-Raphson
// steps y <- y (2 - d y) in FP64 (the relative error squares: 2^-23 -> 2^-46 -> below
// rounding), a handful of FP64 operations instead of a full-precision division.  The
// shifted diagonal d is far inside the FP32 range.  FP32: the correctly rounded
// reciprocal.
__device__ __forceinline__ double recip(double d) {
  double y = (double)__frcp_rn((float)d);
  y = y * fma(-d, y, 2.0);
  y = y * fma(-d, y, 2.0);
  return y;
}
__device__ __forceinline__ float recip(float d) { return __frcp_rn(d); }

// ---- fused SpMM: AX = A X, MX = M X  (one pass over the shared pattern) ----
// Row tiling: LPR lanes per row (32 / LPR rows per warp), CPL 16-byte chunks per lane
// (chunks sl, sl + LPR, ...), blockDim.x / 32 warps per block; picked per level size
// and block width by the autotuner (tune_rows).
// Row groups (a group: the rows of one pass of a CTA's warps) are dealt to the CTAs in
// chunks of `groups` consecutive groups, round robin: an SM walks short contiguous
// stretches of the Morton row order (neighbour rows of X found in its L1), while all
// SMs together stay within a window of the order that L2 holds (neighbours shared
// across chunks found in L2).
template <typename T, int LPR, int CPL>
__global__ void __launch_bounds__(512)
spmm_am_kernel(const int* __restrict__ row_ptr, const int* __restrict__ col,
               const T* __restrict__ va, const T* __restrict__ vm,
               const T* __restrict__ X, int n, int nch, T* __restrict__ AX,
               T* __restrict__ MX, const int* __restrict__ order, int groups) {
  constexpr int W = Chunk<T>::W;
  constexpr int RPW = 32 / LPR;
  const int lane = threadIdx.x & 31, sl = lane % LPR;
  const int per_group = (blockDim.x >> 5) * RPW;
  const int ngroups = (n + per_group - 1) / per_group;
  for (int g = blockIdx.x * groups, gc = 0; g < ngroups; ++g) {
    if (gc == groups) { g += (gridDim.x - 1) * groups; gc = 0; if (g >= ngroups) break; }
    ++gc;
    const int w = g * per_group + (threadIdx.x >> 5) * RPW + lane / LPR;
    const bool live = w < n;               // every lane takes part in the row's shuffles
    const int row = live ? (order ? order[w] : w) : 0;
    T aa[CPL][W], mm[CPL][W];
#pragma unroll
    for (int u = 0; u < CPL; ++u)
#pragma unroll
      for (int q = 0; q < W; ++q) { aa[u][q] = T(0); mm[u][q] = T(0); }
    const int b = live ? row_ptr[row] : 0;
    gather_row<T, LPR, CPL>(col, va, vm, X, b, live ? row_ptr[row + 1] - b : 0, nch, sl, aa, mm);
    if (!live) continue;
#pragma unroll
    for (int u = 0; u < CPL; ++u) {
      const int c = sl + LPR * u;
      if (c < nch) {
        stv_cs(AX, (size_t)row * nch + c, aa[u]);
        stv_cs(MX, (size_t)row * nch + c, mm[u]);
      }
    }
  }
}

// ---- smoother / residual row update ----------------------------------------
// For row i and column c:  r = b - (A x - s_c M x),  d = dA_i - s_c dM_i.
//   MODE 0 (Jacobi):   xout = x + omega r / d
//   MODE 1 (GS):       x    = x + r / d          (in place, rows of one colour)
//   MODE 2 (residual): out  = r
// ZS: every shift is zero (the shifted problems of a solve at sigma = 0): r = b - A x
// and d = dA_i, so M and its diagonal are not read and 1/d is formed once per row.
template <typename T, int LPR, int CPL, int MODE, bool ZS>
__global__ void __launch_bounds__(512)
row_update_kernel(const int* __restrict__ row_ptr, const int* __restrict__ col,
                  const T* __restrict__ va, const T* __restrict__ vm,
                  const T* __restrict__ da, const T* __restrict__ dm,
                  const int* __restrict__ rows, int nrows, const T* X,
                  T* Out, const T* __restrict__ B, const T* __restrict__ shift,
                  int nch, T omega, int groups) {
  constexpr int W = Chunk<T>::W;
  constexpr int RPW = 32 / LPR;
  const int lane = threadIdx.x & 31, sl = lane % LPR;
  const int per_group = (blockDim.x >> 5) * RPW;
  const int ngroups = (nrows + per_group - 1) / per_group;
  for (int g = blockIdx.x * groups, gc = 0; g < ngroups; ++g) {
    if (gc == groups) { g += (gridDim.x - 1) * groups; gc = 0; if (g >= ngroups) break; }
    ++gc;
    const int w = g * per_group + (threadIdx.x >> 5) * RPW + lane / LPR;
    const bool live = w < nrows;           // every lane takes part in the row's shuffles
    const int row = live ? (rows ? rows[w] : w) : 0;
    T aa[CPL][W], mm[CPL][W];
#pragma unroll
    for (int u = 0; u < CPL; ++u)
#pragma unroll
      for (int q = 0; q < W; ++q) { aa[u][q] = T(0); mm[u][q] = T(0); }
    const int b = live ? row_ptr[row] : 0;
    gather_row<T, LPR, CPL, !ZS>(col, va, vm, X, b, live ? row_ptr[row + 1] - b : 0, nch, sl, aa, mm);
    if (!live) continue;
    const T dai = da[row], dmi = ZS ? T(0) : dm[row];
    const T rd0 = (ZS && MODE != 2) ? recip(dai) : T(0);
#pragma unroll
    for (int u = 0; u < CPL; ++u) {
      const int c = sl + LPR * u;
      if (c >= nch) continue;
      T s[W], r[W];
      if (ZS) {
#pragma unroll
        for (int q = 0; q < W; ++q) s[q] = T(0);
      } else {
        ldv(shift, c, s);
      }
#pragma unroll
      for (int q = 0; q < W; ++q) r[q] = ZS ? -aa[u][q] : -(aa[u][q] - s[q] * mm[u][q]);
      const size_t idx = (size_t)row * nch + c;
      if (B) {
        T bb[W];
        ldv(B, idx, bb);
#pragma unroll
        for (int q = 0; q < W; ++q) r[q] += bb[q];
      }
      if (MODE == 2) {
        stv_cs(Out, idx, r);
      } else {
        T x[W], o[W];
        ldv_ro(X, idx, x);   // a row of the running colour is read only by its own lanes
#pragma unroll
        for (int q = 0; q < W; ++q) {
          const T rd = ZS ? rd0 : recip(dai - s[q] * dmi);
          o[q] = (MODE == 0) ? x[q] + omega * (r[q] * rd) : x[q] + r[q] * rd;
        }
        // padding columns carry zero shift, zero data and stay zero
        if (MODE == 0) stv_cs(Out, idx, o); else stv(Out, idx, o);
      }
    }
  }
}

// ---- Kaczmarz projection of the rows of one colour --------------------------
// Row r: res_c = b_c - (A x - s_c M x)_r, coef_c = omega res_c / (na - 2 s_c nam +
// s_c^2 nm), then x_j += coef_c (a_rj - s_c m_rj) for every column j of the row.  Rows
// of one colour of a distance-2 colouring share no column, so the updates of a launch
// touch disjoint rows of X and no row they read is written by another row.
template <typename T, int LPR, int CPL>
__global__ void __launch_bounds__(512)
kaczmarz_kernel(const int* __restrict__ row_ptr, const int* __restrict__ col, const T* __restrict__ va,
                const T* __restrict__ vm, const T* __restrict__ na, const T* __restrict__ nam,
                const T* __restrict__ nm, const int* __restrict__ rows, int nrows, T* X,
                const T* __restrict__ B, const T* __restrict__ shift, int nch, T omega) {
  constexpr int W = Chunk<T>::W;
  constexpr int RPW = 32 / LPR;
  const int lane = threadIdx.x & 31, sl = lane % LPR;
  const int w = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * RPW + lane / LPR;
  const bool live = w < nrows;
  const int row = live ? rows[w] : 0;
  T aa[CPL][W], mm[CPL][W];
#pragma unroll
  for (int u = 0; u < CPL; ++u)
#pragma unroll
    for (int q = 0; q < W; ++q) { aa[u][q] = T(0); mm[u][q] = T(0); }
  const int b = live ? row_ptr[row] : 0;
  const int e = live ? row_ptr[row + 1] : 0;
  gather_row<T, LPR, CPL>(col, va, vm, X, b, e - b, nch, sl, aa, mm);
  if (!live) return;
  const T n_a = na[row], n_am = nam[row], n_m = nm[row];
  T coef[CPL][W], sv[CPL][W];
#pragma unroll
  for (int u = 0; u < CPL; ++u) {
    const int c = sl + LPR * u;
#pragma unroll
    for (int q = 0; q < W; ++q) { coef[u][q] = T(0); sv[u][q] = T(0); }
    if (c >= nch) continue;
    ldv(shift, c, sv[u]);
    T bb[W];
#pragma unroll
    for (int q = 0; q < W; ++q) bb[q] = T(0);
    if (B) ldv(B, (size_t)row * nch + c, bb);
#pragma unroll
    for (int q = 0; q < W; ++q) {
      const T res = bb[q] - (aa[u][q] - sv[u][q] * mm[u][q]);
      const T nrm = n_a - T(2) * sv[u][q] * n_am + sv[u][q] * sv[u][q] * n_m;
      coef[u][q] = nrm > T(0) ? omega * res / nrm : T(0);
    }
  }
  for (int p = b; p < e; ++p) {
    const int j = col[p];
    const T a = va[p], m = vm[p];
#pragma unroll
    for (int u = 0; u < CPL; ++u) {
      const int c = sl + LPR * u;
      if (c < nch) {
        T x[W];
        ldv(X, (size_t)j * nch + c, x);
#pragma unroll
        for (int q = 0; q < W; ++q) x[q] = fma(coef[u][q], a - sv[u][q] * m, x[q]);
        stv(X, (size_t)j * nch + c, x);
      }
    }
  }
}

template <typename T>
__global__ void row_norms_kernel(const int* __restrict__ row_ptr, const T* __restrict__ va,
                                 const T* __restrict__ vm, int n, T* na, T* nam, T* nm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T s1 = T(0), s2 = T(0), s3 = T(0);
  for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
    s1 = fma(va[p], va[p], s1);
    s2 = fma(va[p], vm[p], s2);
    s3 = fma(vm[p], vm[p], s3);
  }
  na[i] = s1;
  nam[i] = s2;
  nm[i] = s3;
}

// ---- transfers ----------------------------------------------------------------
// Y[v] (+)= P Xc: parents (a, b) of fine vertex v; a == b: copy, else the mean.
// order (optional): the fine rows in Morton order of their positions, so that the
// parents gathered by neighbouring threads are near one another in space and found in
// L2 (each row is computed alone: the result does not depend on the order).
template <typename T>
__global__ void prolong_kernel(const int* __restrict__ par, int nf, const T* __restrict__ Xc,
                               T* __restrict__ Y, int nch, int add, const int* __restrict__ order) {
  constexpr int W = Chunk<T>::W;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)nf * nch) return;
  const int v = order ? order[t / nch] : (int)(t / nch), c = (int)(t % nch);
  const int a = par[2 * v], b = par[2 * v + 1];
  T r[W];
  ldv(Xc, (size_t)a * nch + c, r);
  if (a != b) {
    T y[W];
    ldv(Xc, (size_t)b * nch + c, y);
#pragma unroll
    for (int q = 0; q < W; ++q) r[q] = T(0.5) * (r[q] + y[q]);
  }
  if (add) {
    T o[W];
    ldv(Y, (size_t)v * nch + c, o);
#pragma unroll
    for (int q = 0; q < W; ++q) r[q] = o[q] + r[q];
  }
  stv(Y, (size_t)v * nch + c, r);
}

// Zc[i] = R[i] + sum over edges (i, j): R[mid(i,j)] / 2, in ascending fine index.
// order (optional): the coarse rows in Morton order, as in prolong_kernel.
template <typename T>
__global__ void restrict_kernel(const int* __restrict__ row_ptr, const int* __restrict__ col,
                                const int* __restrict__ mid, int nc, const T* __restrict__ R,
                                T* __restrict__ Z, const T* __restrict__ R2, T* __restrict__ Z2, int nch,
                                const int* __restrict__ order) {
  // blockIdx.y = 1: the second block pair of a two-block launch
  if (blockIdx.y == 1) { R = R2; Z = Z2; }
  constexpr int W = Chunk<T>::W;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)nc * nch) return;
  const int i = order ? order[t / nch] : (int)(t / nch), c = (int)(t % nch);
  T acc[W];
  ldv(R, (size_t)i * nch + c, acc);
  for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
    const int m = mid[p];
    if (m < 0) continue;
    T r[W];
    ldv(R, (size_t)m * nch + c, r);
#pragma unroll
    for (int q = 0; q < W; ++q) acc[q] = acc[q] + T(0.5) * r[q];
  }
  stv(Z, (size_t)i * nch + c, acc);
}

// ---- tall-skinny Gram  G = X^T Y  --------------------------------------------
// Each block accumulates the full k x k product over a contiguous row range, each
// thread a set of 4x4 output tiles; row chunks are staged in shared memory.  Block
// partials are summed in a fixed order by gram_reduce_kernel (deterministic).
constexpr int kGramRows = 16;
constexpr int kGramThreads = 256;

// Output tile t of a Gram product with tk x tk tiles of 4 x 4: all tiles, or (sym)
// only the tiles on and above the diagonal, numbered row by row.
__device__ __forceinline__ void gram_tile(int t, int tk, int sym, int& ti, int& tj) {
  if (!sym) {
    ti = (t / tk) * 4;
    tj = (t % tk) * 4;
    return;
  }
  int I = 0, rem = t;
  while (rem >= tk - I) { rem -= tk - I; ++I; }
  ti = I * 4;
  tj = (I + rem) * 4;
}

template <int NT>
__global__ void __launch_bounds__(kGramThreads)
gram_kernel(const double* __restrict__ X, const double* __restrict__ Y, int n, int k, int ld,
            int rows_per_part, double* __restrict__ partial, int sym) {
  extern __shared__ double sh[];
  double* sx = sh;
  double* sy = sh + kGramRows * ld;
  const int tk = (k + 3) / 4;
  const int ntiles = sym ? tk * (tk + 1) / 2 : tk * tk;
  double acc[NT][4][4];
#pragma unroll
  for (int t = 0; t < NT; ++t)
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[t][a][b] = 0.0;
  const int r0 = blockIdx.x * rows_per_part;
  const int r1 = min(n, r0 + rows_per_part);
  for (int base = r0; base < r1; base += kGramRows) {
    const int nr = min(kGramRows, r1 - base);
    __syncthreads();
    for (int q = threadIdx.x; q < kGramRows * ld; q += blockDim.x) {
      const int r = q / ld;
      const bool ok = r < nr;
      sx[q] = ok ? X[(size_t)(base + r) * ld + (q % ld)] : 0.0;
      sy[q] = ok ? Y[(size_t)(base + r) * ld + (q % ld)] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int tile = threadIdx.x + t * kGramThreads;
      if (tile >= ntiles) continue;
      int ti, tj;
      gram_tile(tile, tk, sym, ti, tj);
      for (int r = 0; r < kGramRows; ++r) {
        double xv[4], yv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          xv[a] = (ti + a < ld) ? sx[r * ld + ti + a] : 0.0;
          yv[a] = (tj + a < ld) ? sy[r * ld + tj + a] : 0.0;
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[t][a][b] = fma(xv[a], yv[b], acc[t][a][b]);
      }
    }
  }
  double* out = partial + (size_t)blockIdx.x * k * k;
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int tile = threadIdx.x + t * kGramThreads;
    if (tile >= ntiles) continue;
    int ti, tj;
    gram_tile(tile, tk, sym, ti, tj);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (ti + a < k && tj + b < k) out[(ti + a) * k + tj + b] = acc[t][a][b];
  }
}

// FP32 blocks: every product x*y is split exactly into p + e (p = fl(x*y), e by one
// fused multiply-add), and p is added to the running sum s with Knuth's TwoSum, whose
// rounding error joins e in a second FP32 accumulator c.  The pair (s, c) is a
// double-float accumulator: the block partial s + c, formed in FP64, is accurate to
// about 2^-46 of sum |x y|, instead of the 2^-24 of plain FP32 accumulation.
// 512 threads, one 4x4 output tile each (two FP32 registers per output); blockIdx.y
// selects which 512 tiles, so large k runs as several CTAs over the same rows.
constexpr int kGram32Threads = 512;
__global__ void __launch_bounds__(kGram32Threads)
gram_f32_kernel(const float* __restrict__ X, const float* __restrict__ Y, int n, int k, int ld,
                int rows_per_part, double* __restrict__ partial, int sym) {
  extern __shared__ __align__(16) float shf[];
  float* sx = shf;
  float* sy = shf + kGramRows * ld;
  const int tk = (k + 3) / 4;
  const int ntiles = sym ? tk * (tk + 1) / 2 : tk * tk;
  const int tile = threadIdx.x + blockIdx.y * kGram32Threads;
  const bool active = tile < ntiles;
  int ti = 0, tj = 0;
  if (active) gram_tile(tile, tk, sym, ti, tj);
  float s[4][4], c[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { s[a][b] = 0.f; c[a][b] = 0.f; }
  const int r0 = blockIdx.x * rows_per_part;
  const int r1 = min(n, r0 + rows_per_part);
  for (int base = r0; base < r1; base += kGramRows) {
    const int nr = min(kGramRows, r1 - base);
    __syncthreads();
    for (int q = threadIdx.x; q < kGramRows * ld; q += blockDim.x) {
      const int r = q / ld;
      const bool ok = r < nr;
      sx[q] = ok ? X[(size_t)(base + r) * ld + (q % ld)] : 0.f;
      sy[q] = ok ? Y[(size_t)(base + r) * ld + (q % ld)] : 0.f;
    }
    __syncthreads();
    if (!active) continue;
    for (int r = 0; r < kGramRows; ++r) {
      const float4 xv = *reinterpret_cast<const float4*>(sx + r * ld + ti);
      const float4 yv = *reinterpret_cast<const float4*>(sy + r * ld + tj);
      const float xa[4] = {xv.x, xv.y, xv.z, xv.w};
      const float yb[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const float p = xa[a] * yb[b];
          const float e = fmaf(xa[a], yb[b], -p);
          const float sn = s[a][b] + p;
          const float bp = sn - s[a][b];
          const float err = (s[a][b] - (sn - bp)) + (p - bp);
          s[a][b] = sn;
          c[a][b] += err + e;
        }
    }
  }
  if (!active) return;
  double* out = partial + (size_t)blockIdx.x * k * k;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
      if (ti + a < k && tj + b < k) out[(ti + a) * k + tj + b] = (double)s[a][b] + (double)c[a][b];
}

// G[q] = sum of the block partials in block order.  With sym (a k x k Gram of which
// only the tiles on and above the diagonal were formed) an entry below the diagonal
// tiles takes its mirror.
__global__ void gram_reduce_kernel(const double* __restrict__ partial, int nparts, int kk,
                                   double* __restrict__ G, int k = 0, int sym = 0) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= kk) return;
  int src = q;
  if (sym) {
    const int i = q / k, j = q % k;
    if (i / 4 > j / 4) src = j * k + i;
  }
  double s = 0.0;
  for (int b = 0; b < nparts; ++b) s += partial[(size_t)b * kk + src];
  G[q] = s;
}

// ---- per-vector residual norms ----------------------------------------------
// partial[b][c] = sum_rows (AU - lam_c MU)^2,  partial[b][k + c] = sum_rows U^2,
// in FP64 for either block type.
template <typename T>
__global__ void eigres_kernel(const T* __restrict__ AU, const T* __restrict__ MU,
                              const T* __restrict__ U, const double* __restrict__ lam, int n,
                              int k, int ld, int rows_per_part, double* __restrict__ partial) {
  // one thread per column; threads of a block split the rows in interleaved fashion
  extern __shared__ double red[];
  const int c = threadIdx.x % k;
  const int slice = threadIdx.x / k;
  const int nslices = blockDim.x / k;
  double rr = 0.0, uu = 0.0;
  if (slice < nslices) {
    const int r0 = blockIdx.x * rows_per_part;
    const int r1 = min(n, r0 + rows_per_part);
    const double l = lam[c];
    for (int r = r0 + slice; r < r1; r += nslices) {
      const size_t idx = (size_t)r * ld + c;
      const double d = (double)AU[idx] - l * (double)MU[idx];
      const double u = (double)U[idx];
      rr = fma(d, d, rr);
      uu = fma(u, u, uu);
    }
  }
  red[threadIdx.x] = rr;
  red[blockDim.x + threadIdx.x] = uu;
  __syncthreads();
  if (threadIdx.x < k) {
    double s1 = 0.0, s2 = 0.0;
    for (int q = 0; q < nslices; ++q) { s1 += red[q * k + c]; s2 += red[blockDim.x + q * k + c]; }
    partial[(size_t)blockIdx.x * 2 * k + c] = s1;
    partial[(size_t)blockIdx.x * 2 * k + k + c] = s2;
  }
}

// ---- expand: U = Zf + X Yx ----------------------------------------------------
// One warp per row; Yx (k x ldy, FP64) staged in shared memory as T; lane owns the
// chunks lane + 32 u of the output row.
template <typename T, int CPL>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
expand_kernel(const T* __restrict__ Zf, const T* __restrict__ X,
              const double* __restrict__ Yx, int n, int k, int ld, int ldy,
              T* __restrict__ U) {
  constexpr int W = Chunk<T>::W;
  extern __shared__ __align__(16) unsigned char sy_raw[];
  T* sy = reinterpret_cast<T*>(sy_raw);
  for (int q = threadIdx.x; q < k * ld; q += blockDim.x) {
    const int r = q / ld, c = q % ld;
    sy[q] = (c < k) ? (T)Yx[(size_t)r * ldy + c] : T(0);
  }
  __syncthreads();
  const int nch = ld / W;
  const int lane = threadIdx.x & 31;
  for (int row = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); row < n;
       row += gridDim.x * kWarpsPerBlock) {
    T acc[CPL][W];
#pragma unroll
    for (int u = 0; u < CPL; ++u) {
      const int c = lane + 32 * u;
      if (Zf && c < nch) {
        ldv(Zf, (size_t)row * nch + c, acc[u]);
      } else {
#pragma unroll
        for (int q = 0; q < W; ++q) acc[u][q] = T(0);
      }
    }
    const T* xr = X + (size_t)row * ld;
    for (int q = 0; q < k; ++q) {
      const T xv = xr[q];
#pragma unroll
      for (int u = 0; u < CPL; ++u) {
        const int c = lane + 32 * u;
        if (c < nch) {
          T y[W];
          ldv(sy + q * ld, c, y);
#pragma unroll
          for (int z = 0; z < W; ++z) acc[u][z] = fma(xv, y[z], acc[u][z]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < CPL; ++u) {
      const int c = lane + 32 * u;
      if (c < nch) stv(U, (size_t)row * nch + c, acc[u]);
    }
  }
}

template <typename T>
__global__ void scale_rhs_kernel(const T* __restrict__ MU, const double* __restrict__ theta,
                                 size_t total, int ld, T* __restrict__ B) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < total) B[t] = (T)theta[t % ld] * MU[t];
}

int blocks_for(size_t n, int b) { return (int)std::max<size_t>(1, (n + b - 1) / b); }

int cpl_for(int nch) { return nch <= 32 ? 1 : (nch <= 64 ? 2 : 4); }

template <typename T>
constexpr double tb() { return (double)sizeof(T); }
}  // namespace

// ------------------------------------------------------------------ host ----
// Row-kernel shapes (lanes per row, chunks per lane) and the autotuner that picks one
// (with the warps per block) per kernel kind, arithmetic, block width and row count.
namespace {
constexpr int kNumShapes = 8;
constexpr int kShapeLPR[kNumShapes] = {32, 32, 32, 16, 16, 8, 8, 4};
constexpr int kShapeCPL[kNumShapes] = {1, 2, 4, 1, 2, 1, 2, 1};
constexpr int kWPB[3] = {4, 8, 16};

struct RowCfg {
  int shape, wpb;
  int chunk = 64;   // rows per chunk dealt to a CTA (row_grid)
};
constexpr int kChunks[4] = {32, 64, 128, 256};

int pow2_at_least(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}
// shapes whose lanes x chunks cover the row without idling more than half
bool shape_ok(int sh, int nch) {
  const int tot = kShapeLPR[sh] * kShapeCPL[sh];
  return tot >= nch && tot <= 2 * pow2_at_least(nch);
}
RowCfg default_cfg(int nch) {
  const int cpl = nch <= 32 ? 1 : (nch <= 64 ? 2 : 4);
  return {cpl == 1 ? 0 : (cpl == 2 ? 1 : 2), 8};
}

// Resident CTAs of a row kernel per SM (occupancy calculator), cached per kernel and
// block size.
std::mutex g_occ_mu;
std::map<std::pair<const void*, int>, int> g_occ;
int resident_blocks(const void* kernel, int threads) {
  std::lock_guard<std::mutex> lock(g_occ_mu);
  const auto key = std::make_pair(kernel, threads);
  auto it = g_occ.find(key);
  if (it != g_occ.end()) return it->second;
  int nb = 0, dev = 0, sms = 0;
  check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, 0), "occupancy");
  check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "sm count");
  const int v = std::max(1, nb) * std::max(1, sms);
  g_occ.emplace(key, v);
  return v;
}
// Grid of a row kernel over `items` row groups of `rows_per_group` rows: at most one
// wave of resident CTAs, dealt chunks of about `chunk` consecutive rows; shorter chunks
// when there would be fewer chunks than resident CTAs (small launches, such as the
// rows of one colour, keep every SM busy).
void row_grid(const void* kernel, int threads, int items, int rows_per_group, int chunk, int& grid, int& groups) {
  const int wave = resident_blocks(kernel, threads);
  groups = std::max(1, std::min(chunk / rows_per_group, items / wave));
  const int chunks = (items + groups - 1) / groups;
  grid = std::max(1, std::min(chunks, wave));
}

template <typename T, int LPR, int CPL>
void spmm_shape(int wpb, int chunk, const Mesh& m, const T* a, const T* mm, const T* X, int nch, T* AX, T* MX,
                cudaStream_t s) {
  const int per_block = wpb * (32 / LPR);
  int grid, groups;
  row_grid((const void*)spmm_am_kernel<T, LPR, CPL>, wpb * 32, blocks_for(m.n, per_block), per_block, chunk, grid,
           groups);
  spmm_am_kernel<T, LPR, CPL><<<grid, wpb * 32, 0, s>>>(m.row_ptr.get(), m.col.get(), a, mm, X, m.n, nch, AX, MX,
                                                        m.row_order.get(), groups);
  check_launch("spmm_am_kernel");
}
template <typename T>
void spmm_launch(RowCfg c, const Mesh& m, const T* a, const T* mm, const T* X, int nch, T* AX, T* MX,
                 cudaStream_t s) {
  switch (c.shape) {
    case 0: spmm_shape<T, 32, 1>(c.wpb, c.chunk, m, a, mm, X, nch, AX, MX, s); break;
    case 1: spmm_shape<T, 32, 2>(c.wpb, c.chunk, m, a, mm, X, nch, AX, MX, s); break;
    case 2: spmm_shape<T, 32, 4>(c.wpb, c.chunk, m, a, mm, X, nch, AX, MX, s); break;
    case 3: spmm_shape<T, 16, 1>(c.wpb, c.chunk, m, a, mm, X, nch, AX, MX, s); break;
    case 4: spmm_shape<T, 16, 2>(c.wpb, c.chunk, m, a, mm, X, nch, AX, MX, s); break;
    case 5: spmm_shape<T, 8, 1>(c.wpb, c.chunk, m, a, mm, X, nch, AX, MX, s); break;
    case 6: spmm_shape<T, 8, 2>(c.wpb, c.chunk, m, a, mm, X, nch, AX, MX, s); break;
    default: spmm_shape<T, 4, 1>(c.wpb, c.chunk, m, a, mm, X, nch, AX, MX, s); break;
  }
}

template <typename T, int LPR, int CPL, int MODE, bool ZS>
void row_shape(int wpb, int chunk, const Mesh& m, const T* a, const T* mm, const T* da, const T* dm, const int* rows,
               int nrows, const T* X, T* Out, const T* B, const T* shift, int nch, double omega, cudaStream_t s) {
  const int per_block = wpb * (32 / LPR);
  int grid, groups;
  row_grid((const void*)row_update_kernel<T, LPR, CPL, MODE, ZS>, wpb * 32, blocks_for(nrows, per_block), per_block,
           chunk, grid, groups);
  row_update_kernel<T, LPR, CPL, MODE, ZS><<<grid, wpb * 32, 0, s>>>(m.row_ptr.get(), m.col.get(), a, mm, da, dm, rows,
                                                                 nrows, X, Out, B, shift, nch, (T)omega, groups);
  check_launch("row_update_kernel");
}
template <typename T, int MODE, bool ZS>
void row_launch(RowCfg c, const Mesh& m, const T* a, const T* mm, const T* da, const T* dm, const int* rows,
                int nrows, const T* X, T* Out, const T* B, const T* shift, int nch, double omega, cudaStream_t s) {
  switch (c.shape) {
    case 0: row_shape<T, 32, 1, MODE, ZS>(c.wpb, c.chunk, m, a, mm, da, dm, rows, nrows, X, Out, B, shift, nch, omega, s); break;
    case 1: row_shape<T, 32, 2, MODE, ZS>(c.wpb, c.chunk, m, a, mm, da, dm, rows, nrows, X, Out, B, shift, nch, omega, s); break;
    case 2: row_shape<T, 32, 4, MODE, ZS>(c.wpb, c.chunk, m, a, mm, da, dm, rows, nrows, X, Out, B, shift, nch, omega, s); break;
    case 3: row_shape<T, 16, 1, MODE, ZS>(c.wpb, c.chunk, m, a, mm, da, dm, rows, nrows, X, Out, B, shift, nch, omega, s); break;
    case 4: row_shape<T, 16, 2, MODE, ZS>(c.wpb, c.chunk, m, a, mm, da, dm, rows, nrows, X, Out, B, shift, nch, omega, s); break;
    case 5: row_shape<T, 8, 1, MODE, ZS>(c.wpb, c.chunk, m, a, mm, da, dm, rows, nrows, X, Out, B, shift, nch, omega, s); break;
    case 6: row_shape<T, 8, 2, MODE, ZS>(c.wpb, c.chunk, m, a, mm, da, dm, rows, nrows, X, Out, B, shift, nch, omega, s); break;
    default: row_shape<T, 4, 1, MODE, ZS>(c.wpb, c.chunk, m, a, mm, da, dm, rows, nrows, X, Out, B, shift, nch, omega, s); break;
  }
}

// Tuned shapes, process-wide.  The candidates are timed on the call's own data and
// stream (spmm, Jacobi and residual kernels are idempotent: they write a block they
// do not read), three launches each after one warm-up, with CUDA events.  A solve
// with bmg_options.autotune = 0 uses the default shape (32 lanes per row, 8 warps
// per block) on its thread.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, RowCfg> g_tuned;
thread_local bool t_autotune = true;

bool autotune_enabled() { return t_autotune; }

template <typename F>
RowCfg tune_rows(int kind, int tsize, int nch, int n, cudaStream_t s, F&& launch) {
  const auto key = std::make_tuple(kind, tsize, nch, n);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) return it->second;
  }
  RowCfg best = default_cfg(nch);
  if (!autotune_enabled()) return best;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  check_cuda(cudaStreamIsCapturing(s, &cap), "cudaStreamIsCapturing");
  if (!autotune_enabled() || cap != cudaStreamCaptureStatusNone) return best;
  cudaEvent_t e0, e1;
  check_cuda(cudaEventCreate(&e0), "cudaEventCreate");
  check_cuda(cudaEventCreate(&e1), "cudaEventCreate");
  float best_ms = 1e30f;
  for (int sh = 0; sh < kNumShapes; ++sh) {
    if (!shape_ok(sh, nch)) continue;
    for (int wpb : kWPB) {
      RowCfg c;
      c.shape = sh;
      c.wpb = wpb;
      launch(c);
      check_cuda(cudaEventRecord(e0, s), "cudaEventRecord");
      for (int q = 0; q < 3; ++q) launch(c);
      check_cuda(cudaEventRecord(e1, s), "cudaEventRecord");
      check_cuda(cudaEventSynchronize(e1), "cudaEventSynchronize");
      float ms = 0.f;
      check_cuda(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
      if (ms < best_ms) { best_ms = ms; best = c; }
    }
  }
  // then the chunk length for the chosen shape
  for (int ch : kChunks) {
    if (ch == best.chunk) continue;
    RowCfg c = best;
    c.chunk = ch;
    launch(c);
    check_cuda(cudaEventRecord(e0, s), "cudaEventRecord");
    for (int q = 0; q < 3; ++q) launch(c);
    check_cuda(cudaEventRecord(e1, s), "cudaEventRecord");
    check_cuda(cudaEventSynchronize(e1), "cudaEventSynchronize");
    float ms = 0.f;
    check_cuda(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
    if (ms < best_ms) { best_ms = ms; best = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tuned[key] = best;
  return best;
}
}  // namespace

AutotuneScope::AutotuneScope(bool on) : prev_(t_autotune) { t_autotune = on; }
AutotuneScope::~AutotuneScope() { t_autotune = prev_; }

template <typename T>
void spmm_am(const Mesh& m, const T* a, const T* mm, const T* X, int ld, T* AX, T* MX, cudaStream_t s) {
  const int nch = ld / Chunk<T>::W;
  const RowCfg c = tune_rows(0, (int)sizeof(T), nch, m.n, s, [&](RowCfg q) {
    spmm_launch<T>(q, m, a, mm, X, nch, AX, MX, s);
  });
  prof_begin(KC_SPMM, s);
  spmm_launch<T>(c, m, a, mm, X, nch, AX, MX, s);
  prof_end(KC_SPMM, s, (4.0 + 2.0 * tb<T>()) * m.nnz + 4.0 * (m.n + 1) + 3.0 * tb<T>() * m.n * ld,
           4.0 * m.nnz * ld);
}

template <typename T, int MODE>
static void row_update(const Mesh& m, const T* a, const T* mm, const T* da, const T* dm,
                       const int* rows, int nrows, long long nnz_rows, const T* X, T* Out,
                       const T* B, const T* shift, int ld, double omega, cudaStream_t s,
                       T* scratch = nullptr, bool zero_shift = false) {
  const int nch = ld / Chunk<T>::W;
  if (nrows == 0) return;
  auto launch = [&](RowCfg q, int mode_override, T* out) {
    // mode_override: the residual form of a Gauss-Seidel colour, timed on a scratch block
    if (mode_override == 2) {
      if (zero_shift) row_launch<T, 2, true>(q, m, a, mm, da, dm, rows, nrows, X, out, B, shift, nch, omega, s);
      else row_launch<T, 2, false>(q, m, a, mm, da, dm, rows, nrows, X, out, B, shift, nch, omega, s);
    } else if (zero_shift) {
      row_launch<T, MODE, true>(q, m, a, mm, da, dm, rows, nrows, X, out, B, shift, nch, omega, s);
    } else {
      row_launch<T, MODE, false>(q, m, a, mm, da, dm, rows, nrows, X, out, B, shift, nch, omega, s);
    }
  };
  // Gauss-Seidel sweeps run in place and are not re-run for timing: with a scratch
  // block they take the shape tuned for the residual kernel on the same rows (same
  // gathers, written to the scratch block), else the one of the level's residual or
  // Jacobi sweep
  const int kind = (MODE == 2) ? 2 : 1;
  RowCfg c = default_cfg(nch);
  if (MODE == 1 && scratch) {
    c = tune_rows(3, (int)sizeof(T), nch, nrows, s, [&](RowCfg q) { launch(q, 2, scratch); });
  } else if (MODE == 1 && autotune_enabled()) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (int kd : {2, 1}) {
      auto it = g_tuned.find(std::make_tuple(kd, (int)sizeof(T), nch, m.n));
      if (it != g_tuned.end()) { c = it->second; break; }
    }
  } else {
    c = tune_rows(kind, (int)sizeof(T), nch, nrows, s, [&](RowCfg q) { launch(q, MODE, Out); });
  }
  const int cls = (MODE == 2) ? KC_RESID : KC_SMOOTH;
  prof_begin(cls, s);
  launch(c, MODE, Out);
  // matrix rows, diagonals, own-row read + write, one share of the gathered block, B
  // (without M and its diagonal when every shift is zero)
  const double vals = zero_shift ? 1.0 : 2.0;
  const double bytes = (4.0 + vals * tb<T>()) * nnz_rows + vals * tb<T>() * nrows +
                       tb<T>() * nrows * ld * (B ? 4.0 : 3.0);
  prof_end(cls, s, bytes, (zero_shift ? 2.0 : 4.0) * nnz_rows * ld + 6.0 * nrows * ld);
}

template <typename T>
void jacobi_sweep(const Mesh& m, const T* a, const T* mm, const T* da, const T* dm, const T* X,
                  T* Xout, const T* B, const T* shift, int ld, double omega, cudaStream_t s, bool zero_shift) {
  row_update<T, 0>(m, a, mm, da, dm, m.row_order.get(), m.n, m.nnz, X, Xout, B, shift, ld, omega, s, nullptr,
                   zero_shift);
}

template <typename T>
void gs_colour_sweep(const Mesh& m, const Level& lv, int c, const T* a, const T* mm, const T* da,
                     const T* dm, T* X, const T* B, const T* shift, int ld, cudaStream_t s, T* scratch,
                     bool zero_shift) {
  const int b = lv.col1.ptr_host[c], e = lv.col1.ptr_host[c + 1];
  row_update<T, 1>(m, a, mm, da, dm, lv.col1.rows.get() + b, e - b, lv.col1.nnz_host[c], X, X, B,
                   shift, ld, 1.0, s, scratch, zero_shift);
}

template <typename T>
void kaczmarz_colour_sweep(const Mesh& m, const Level& lv, int c, const T* a, const T* mm, const T* na,
                           const T* nam, const T* nm, T* X, const T* B, const T* shift, int ld, double omega,
                           cudaStream_t s) {
  const int b = lv.col2.ptr_host[c], e = lv.col2.ptr_host[c + 1];
  const int nrows = e - b;
  if (nrows == 0) return;
  const int nch = ld / Chunk<T>::W;
  const int* rows = lv.col2.rows.get() + b;
  constexpr int wpb = 8;
  prof_begin(KC_SMOOTH, s);
  // lanes per row and chunks per lane cover the row as the default row shape does
  if (nch <= 32)
    kaczmarz_kernel<T, 32, 1><<<blocks_for(nrows, wpb), wpb * 32, 0, s>>>(m.row_ptr.get(), m.col.get(), a, mm, na, nam,
                                                                          nm, rows, nrows, X, B, shift, nch, (T)omega);
  else if (nch <= 64)
    kaczmarz_kernel<T, 32, 2><<<blocks_for(nrows, wpb), wpb * 32, 0, s>>>(m.row_ptr.get(), m.col.get(), a, mm, na, nam,
                                                                          nm, rows, nrows, X, B, shift, nch, (T)omega);
  else
    kaczmarz_kernel<T, 32, 4><<<blocks_for(nrows, wpb), wpb * 32, 0, s>>>(m.row_ptr.get(), m.col.get(), a, mm, na, nam,
                                                                          nm, rows, nrows, X, B, shift, nch, (T)omega);
  check_launch("kaczmarz_kernel");
  const double nnz = (double)lv.col2.nnz_host[c];
  // matrix rows, norms, own-row b, gathered block and the written neighbour rows
  prof_end(KC_SMOOTH, s, (4.0 + 2.0 * tb<T>()) * nnz + 3.0 * tb<T>() * nrows + tb<T>() * ld * (nrows + 3.0 * nnz),
           8.0 * nnz * ld);
}

template <typename T>
void row_norms(const Mesh& m, const T* a, const T* mm, T* na, T* nam, T* nm, cudaStream_t s) {
  row_norms_kernel<T><<<blocks_for(m.n, 256), 256, 0, s>>>(m.row_ptr.get(), a, mm, m.n, na, nam, nm);
  check_launch("row_norms_kernel");
}

template <typename T>
void residual(const Mesh& m, const T* a, const T* mm, const T* X, const T* B, const T* shift, int ld,
              T* R, cudaStream_t s, bool zero_shift) {
  // the diagonal is not used in residual mode; pass the matrix values as placeholders
  row_update<T, 2>(m, a, mm, a, mm, m.row_order.get(), m.n, m.nnz, X, R, B, shift, ld, 0.0, s, nullptr,
                   zero_shift);
}

template <typename T>
void prolong(const Mesh& fine, const T* Xc, T* Y, int ld, bool add, cudaStream_t s) {
  const int nch = ld / Chunk<T>::W;
  const size_t total = (size_t)fine.n * nch;
  prof_begin(KC_TRANSFER, s);
  prolong_kernel<T><<<blocks_for(total, 256), 256, 0, s>>>(fine.parents.get(), fine.n, Xc, Y, nch, add ? 1 : 0,
                                                            fine.row_order.get());
  check_launch("prolong_kernel");
  const double nc = (fine.n + 6) / 4.0;  // vertices of the coarse level of a refined sphere
  prof_end(KC_TRANSFER, s, 8.0 * fine.n + tb<T>() * ld * (nc + fine.n * (add ? 2.0 : 1.0)), 1.0 * fine.n * ld);
}

template <typename T>
void restrict_(const Mesh& coarse, const T* R, T* Zc, int ld, cudaStream_t s) {
  restrict2_<T>(coarse, R, Zc, nullptr, nullptr, ld, s);
}

// Zc = P^T R and, when R2 is given, Zc2 = P^T R2 in the same launch.
template <typename T>
void restrict2_(const Mesh& coarse, const T* R, T* Zc, const T* R2, T* Zc2, int ld, cudaStream_t s) {
  const int nch = ld / Chunk<T>::W;
  const size_t total = (size_t)coarse.n * nch;
  const int pairs = R2 ? 2 : 1;
  prof_begin(KC_TRANSFER, s);
  restrict_kernel<T><<<dim3((unsigned)blocks_for(total, 256), pairs), 256, 0, s>>>(
      coarse.row_ptr.get(), coarse.col.get(), coarse.mid.get(), coarse.n, R, Zc, R2, Zc2, nch,
      coarse.row_order.get());
  check_launch("restrict_kernel");
  const double nf = 4.0 * coarse.n - 6.0;
  prof_end(KC_TRANSFER, s, pairs * (8.0 * coarse.nnz + tb<T>() * ld * (nf + coarse.n)), pairs * 2.0 * nf * ld);
}

int gram_parts(int n) { return std::max(1, std::min(304, (n + 63) / 64)); }

void gram(const double* X, const double* Y, int n, int k, int ld, double* G, double* partial,
          int nparts, cudaStream_t s, bool sym) {
  const int rows_per_part = (n + nparts - 1) / nparts;
  const int tk = (k + 3) / 4;
  const int ntiles = sym ? tk * (tk + 1) / 2 : tk * tk;
  const size_t smem = 2 * kGramRows * ld * sizeof(double);
  if (smem > 48 * 1024) {   // blocks wider than 192 columns (e.g. column slices of a wider block)
    const int sm = (int)smem;
    check_cuda(cudaFuncSetAttribute(gram_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm), "gram attr");
    check_cuda(cudaFuncSetAttribute(gram_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm), "gram attr");
    check_cuda(cudaFuncSetAttribute(gram_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm), "gram attr");
    check_cuda(cudaFuncSetAttribute(gram_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm), "gram attr");
  }
  prof_begin(KC_GRAM, s);
  if (ntiles <= kGramThreads) gram_kernel<1><<<nparts, kGramThreads, smem, s>>>(X, Y, n, k, ld, rows_per_part, partial, sym ? 1 : 0);
  else if (ntiles <= 2 * kGramThreads) gram_kernel<2><<<nparts, kGramThreads, smem, s>>>(X, Y, n, k, ld, rows_per_part, partial, sym ? 1 : 0);
  else if (ntiles <= 4 * kGramThreads) gram_kernel<4><<<nparts, kGramThreads, smem, s>>>(X, Y, n, k, ld, rows_per_part, partial, sym ? 1 : 0);
  else if (ntiles <= 8 * kGramThreads) gram_kernel<8><<<nparts, kGramThreads, smem, s>>>(X, Y, n, k, ld, rows_per_part, partial, sym ? 1 : 0);
  else fail(BMG_ERR_INVALID_ARG, "gram: k too large (k <= 180)");
  check_launch("gram_kernel");
  gram_reduce_kernel<<<blocks_for(k * k, 256), 256, 0, s>>>(partial, nparts, k * k, G, k, sym ? 1 : 0);
  check_launch("gram_reduce_kernel");
  prof_end(KC_GRAM, s, 16.0 * n * ld + 16.0 * nparts * k * k + 8.0 * k * k,
           (sym ? 1.0 : 2.0) * n * k * k + (sym ? 4.0 * n * k : 0.0));
}

void gram(const float* X, const float* Y, int n, int k, int ld, double* G, double* partial,
          int nparts, cudaStream_t s, bool sym) {
  if (ld % 4) fail(BMG_ERR_INVALID_ARG, "gram: FP32 blocks need ld % 4 == 0");
  const int rows_per_part = (n + nparts - 1) / nparts;
  const int tk = (k + 3) / 4;
  const int ntiles = sym ? tk * (tk + 1) / 2 : tk * tk;
  const size_t smem = 2 * kGramRows * ld * sizeof(float);
  if (smem > 48 * 1024)
    check_cuda(cudaFuncSetAttribute(gram_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
               "gram_f32 attr");
  prof_begin(KC_GRAM, s);
  const dim3 grid(nparts, (ntiles + kGram32Threads - 1) / kGram32Threads);
  gram_f32_kernel<<<grid, kGram32Threads, smem, s>>>(X, Y, n, k, ld, rows_per_part, partial, sym ? 1 : 0);
  check_launch("gram_f32_kernel");
  gram_reduce_kernel<<<blocks_for(k * k, 256), 256, 0, s>>>(partial, nparts, k * k, G, k, sym ? 1 : 0);
  check_launch("gram_reduce_kernel");
  prof_end(KC_GRAM, s, 8.0 * n * ld + 16.0 * nparts * k * k + 8.0 * k * k, 2.0 * n * k * k);
}

void gram_reduce(const double* partial, int nparts, int k, double* G, bool sym, cudaStream_t s) {
  gram_reduce_kernel<<<blocks_for(k * k, 256), 256, 0, s>>>(partial, nparts, k * k, G, k, sym ? 1 : 0);
  check_launch("gram_reduce_kernel");
}

template <typename T>
void eig_residuals(const T* AU, const T* MU, const T* U, const double* lam, int n, int k, int ld,
                   double* partial, int nparts, double* out, cudaStream_t s) {
  const int rows_per_part = (n + nparts - 1) / nparts;
  const int threads = std::max(k, (256 / k) * k);
  prof_begin(KC_SMALL, s);
  eigres_kernel<T><<<nparts, threads, 2 * threads * sizeof(double), s>>>(AU, MU, U, lam, n, k, ld,
                                                                         rows_per_part, partial);
  check_launch("eigres_kernel");
  gram_reduce_kernel<<<blocks_for(2 * k, 256), 256, 0, s>>>(partial, nparts, 2 * k, out);
  check_launch("gram_reduce_kernel");
  prof_end(KC_SMALL, s, 3.0 * tb<T>() * n * ld, 5.0 * n * k);
}

template <typename T>
void expand(const T* Zf, const T* X, const double* Yx, int n, int k, int ld, int ldy, T* U,
            cudaStream_t s) {
  const int nch = ld / Chunk<T>::W;
  const size_t smem = (size_t)k * ld * sizeof(T);
  const int grid = std::max(1, std::min(blocks_for(n, kWarpsPerBlock), 4 * 152));
  prof_begin(KC_EXPAND, s);
  switch (cpl_for(nch)) {
    case 1:
      cudaFuncSetAttribute(expand_kernel<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      expand_kernel<T, 1><<<grid, kWarpsPerBlock * 32, smem, s>>>(Zf, X, Yx, n, k, ld, ldy, U); break;
    case 2:
      cudaFuncSetAttribute(expand_kernel<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      expand_kernel<T, 2><<<grid, kWarpsPerBlock * 32, smem, s>>>(Zf, X, Yx, n, k, ld, ldy, U); break;
    default:
      cudaFuncSetAttribute(expand_kernel<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      expand_kernel<T, 4><<<grid, kWarpsPerBlock * 32, smem, s>>>(Zf, X, Yx, n, k, ld, ldy, U); break;
  }
  check_launch("expand_kernel");
  prof_end(KC_EXPAND, s, 3.0 * tb<T>() * n * ld + 8.0 * k * k, 2.0 * n * k * k);
}

template <typename T>
void scale_rhs(const T* MU, const double* theta, int n, int k, int ld, T* B, cudaStream_t s) {
  (void)k;
  const size_t total = (size_t)n * ld;
  scale_rhs_kernel<T><<<blocks_for(total, 256), 256, 0, s>>>(MU, theta, total, ld, B);
  check_launch("scale_rhs_kernel");
}

// Text of the tuned row-kernel shapes, one line per entry:
// "kind bytes nch rows -> lanes_per_row chunks_per_lane warps_per_block rows_per_cta_chunk".
std::string tuned_report() {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  std::string out;
  static const char* kinds[4] = {"spmm", "jacobi", "residual", "gs_colour"};
  for (const auto& kv : g_tuned) {
    const auto& k = kv.first;
    const RowCfg c = kv.second;
    out += std::string(kinds[std::get<0>(k)]) + " " + std::to_string(std::get<1>(k)) + " " +
           std::to_string(std::get<2>(k)) + " " + std::to_string(std::get<3>(k)) + " -> " +
           std::to_string(kShapeLPR[c.shape]) + " " + std::to_string(kShapeCPL[c.shape]) + " " +
           std::to_string(c.wpb) + " " + std::to_string(c.chunk) + "\n";
  }
  return out;
}

#define BMG_OPS_INSTANTIATE(T)                                                                          \
  template void spmm_am<T>(const Mesh&, const T*, const T*, const T*, int, T*, T*, cudaStream_t);      \
  template void jacobi_sweep<T>(const Mesh&, const T*, const T*, const T*, const T*, const T*, T*,     \
                                const T*, const T*, int, double, cudaStream_t, bool);                  \
  template void gs_colour_sweep<T>(const Mesh&, const Level&, int, const T*, const T*, const T*,       \
                                   const T*, T*, const T*, const T*, int, cudaStream_t, T*, bool);     \
  template void residual<T>(const Mesh&, const T*, const T*, const T*, const T*, const T*, int, T*,    \
                            cudaStream_t, bool);                                                       \
  template void prolong<T>(const Mesh&, const T*, T*, int, bool, cudaStream_t);                        \
  template void restrict_<T>(const Mesh&, const T*, T*, int, cudaStream_t);                            \
  template void restrict2_<T>(const Mesh&, const T*, T*, const T*, T*, int, cudaStream_t);             \
  template void eig_residuals<T>(const T*, const T*, const T*, const double*, int, int, int, double*,  \
                                 int, double*, cudaStream_t);                                          \
  template void expand<T>(const T*, const T*, const double*, int, int, int, int, T*, cudaStream_t);    \
  template void scale_rhs<T>(const T*, const double*, int, int, int, T*, cudaStream_t);                \
  template void kaczmarz_colour_sweep<T>(const Mesh&, const Level&, int, const T*, const T*, const T*,  \
                                         const T*, const T*, T*, const T*, const T*, int, double,      \
                                         cudaStream_t);                                                \
  template void row_norms<T>(const Mesh&, const T*, const T*, T*, T*, T*, cudaStream_t);

BMG_OPS_INSTANTIATE(double)
BMG_OPS_INSTANTIATE(float)
#undef BMG_OPS_INSTANTIATE

}  // namespace bmg

extern "C" int bmg_autotune_report(char* buf, int len) {
  const std::string r = bmg::tuned_report();
  if (buf && len > 0) {
    const int nb = std::min((int)r.size(), len - 1);
    std::memcpy(buf, r.data(), nb);
    buf[nb] = 0;
  }
  return (int)r.size();
}

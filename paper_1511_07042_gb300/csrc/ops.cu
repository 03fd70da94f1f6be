// Per-cycle kernels of the BMG cycle on k-interleaved vector blocks.
//
// A block of k vectors on a level with N vertices is stored row-major [N][ld]: the
// ld values of one vertex are contiguous, so every CSR neighbour access reads whole
// 16-byte double2 chunks of one row and a warp reads one or more full rows.  One warp
// processes one matrix row; lane l owns the double2 chunks l, l+32, ... of that row.
// Both operators of the pencil share one CSR pattern and are applied in one pass.
#include <algorithm>

#include "common.cuh"

namespace bmg {
namespace {

constexpr int kWarpsPerBlock = 8;

__device__ __forceinline__ double2 ld2(const double* p, size_t idx) {
  return reinterpret_cast<const double2*>(p)[idx];
}
__device__ __forceinline__ void st2(double* p, size_t idx, double2 v) {
  reinterpret_cast<double2*>(p)[idx] = v;
}

// ---- fused SpMM: AX = A X, MX = M X  (one pass over the shared pattern) ----
template <int CPL>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
spmm_am_kernel(const int* __restrict__ row_ptr, const int* __restrict__ col,
               const double* __restrict__ va, const double* __restrict__ vm,
               const double* __restrict__ X, int n, int nch, double* __restrict__ AX,
               double* __restrict__ MX) {
  const int row = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  double2 aa[CPL], mm[CPL];
#pragma unroll
  for (int u = 0; u < CPL; ++u) { aa[u] = make_double2(0.0, 0.0); mm[u] = make_double2(0.0, 0.0); }
  const int b = row_ptr[row], e = row_ptr[row + 1];
  for (int p = b; p < e; ++p) {
    const int j = __ldg(col + p);
    const double a = __ldg(va + p), m = __ldg(vm + p);
#pragma unroll
    for (int u = 0; u < CPL; ++u) {
      const int c = lane + 32 * u;
      if (c < nch) {
        const double2 x = ld2(X, (size_t)j * nch + c);
        aa[u].x = fma(a, x.x, aa[u].x); aa[u].y = fma(a, x.y, aa[u].y);
        mm[u].x = fma(m, x.x, mm[u].x); mm[u].y = fma(m, x.y, mm[u].y);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < CPL; ++u) {
    const int c = lane + 32 * u;
    if (c < nch) {
      st2(AX, (size_t)row * nch + c, aa[u]);
      st2(MX, (size_t)row * nch + c, mm[u]);
    }
  }
}

// ---- smoother / residual row update ----------------------------------------
// For row i and column c:  r = b - (A x - s_c M x),  d = dA_i - s_c dM_i.
//   MODE 0 (Jacobi):   xout = x + omega r / d
//   MODE 1 (GS):       x    = x + r / d          (in place, rows of one colour)
//   MODE 2 (residual): out  = r
template <int CPL, int MODE>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
row_update_kernel(const int* __restrict__ row_ptr, const int* __restrict__ col,
                  const double* __restrict__ va, const double* __restrict__ vm,
                  const double* __restrict__ da, const double* __restrict__ dm,
                  const int* __restrict__ rows, int nrows, const double* X,
                  double* Out, const double* __restrict__ B, const double* __restrict__ shift,
                  int nch, double omega) {
  const int w = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= nrows) return;
  const int row = rows ? rows[w] : w;
  double2 aa[CPL], mm[CPL];
#pragma unroll
  for (int u = 0; u < CPL; ++u) { aa[u] = make_double2(0.0, 0.0); mm[u] = make_double2(0.0, 0.0); }
  const int b = row_ptr[row], e = row_ptr[row + 1];
  for (int p = b; p < e; ++p) {
    const int j = __ldg(col + p);
    const double a = __ldg(va + p), m = __ldg(vm + p);
#pragma unroll
    for (int u = 0; u < CPL; ++u) {
      const int c = lane + 32 * u;
      if (c < nch) {
        const double2 x = ld2(X, (size_t)j * nch + c);
        aa[u].x = fma(a, x.x, aa[u].x); aa[u].y = fma(a, x.y, aa[u].y);
        mm[u].x = fma(m, x.x, mm[u].x); mm[u].y = fma(m, x.y, mm[u].y);
      }
    }
  }
  const double dai = da[row], dmi = dm[row];
#pragma unroll
  for (int u = 0; u < CPL; ++u) {
    const int c = lane + 32 * u;
    if (c >= nch) continue;
    const double2 s = ld2(shift, c);
    double2 r;
    r.x = -(aa[u].x - s.x * mm[u].x);
    r.y = -(aa[u].y - s.y * mm[u].y);
    if (B) {
      const double2 bb = ld2(B, (size_t)row * nch + c);
      r.x += bb.x; r.y += bb.y;
    }
    const size_t idx = (size_t)row * nch + c;
    if (MODE == 2) {
      st2(Out, idx, r);
    } else {
      const double2 x = ld2(X, idx);
      const double dx = dai - s.x * dmi, dy = dai - s.y * dmi;
      double2 o;
      if (MODE == 0) { o.x = x.x + omega * r.x / dx; o.y = x.y + omega * r.y / dy; }
      else           { o.x = x.x + r.x / dx;         o.y = x.y + r.y / dy; }
      // padding columns carry zero shift, zero data and must stay zero
      st2(Out, idx, o);
    }
  }
}

// ---- transfers ----------------------------------------------------------------
// Y[v] (+)= P Xc: parents (a, b) of fine vertex v; a == b: copy, else the mean.
__global__ void prolong_kernel(const int* __restrict__ par, int nf, const double* __restrict__ Xc,
                               double* __restrict__ Y, int nch, int add) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)nf * nch) return;
  const int v = (int)(t / nch), c = (int)(t % nch);
  const int a = par[2 * v], b = par[2 * v + 1];
  double2 r = ld2(Xc, (size_t)a * nch + c);
  if (a != b) {
    const double2 y = ld2(Xc, (size_t)b * nch + c);
    r.x = 0.5 * (r.x + y.x);
    r.y = 0.5 * (r.y + y.y);
  }
  if (add) {
    const double2 o = ld2(Y, (size_t)v * nch + c);
    r.x = o.x + r.x; r.y = o.y + r.y;
  }
  st2(Y, (size_t)v * nch + c, r);
}

// Zc[i] = R[i] + sum over edges (i, j): R[mid(i,j)] / 2, in ascending fine index.
__global__ void restrict_kernel(const int* __restrict__ row_ptr, const int* __restrict__ col,
                                const int* __restrict__ mid, int nc, const double* __restrict__ R,
                                double* __restrict__ Z, int nch) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)nc * nch) return;
  const int i = (int)(t / nch), c = (int)(t % nch);
  double2 acc = ld2(R, (size_t)i * nch + c);
  for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
    const int m = mid[p];
    if (m < 0) continue;
    const double2 r = ld2(R, (size_t)m * nch + c);
    acc.x = acc.x + 0.5 * r.x;
    acc.y = acc.y + 0.5 * r.y;
  }
  st2(Z, (size_t)i * nch + c, acc);
}

// ---- tall-skinny Gram  G = X^T Y  --------------------------------------------
// Each block accumulates the full k x k product over a contiguous row range, each
// thread a set of 4x4 output tiles; row chunks are staged in shared memory.  Block
// partials are summed in a fixed order by gram_reduce_kernel (deterministic).
constexpr int kGramRows = 16;
constexpr int kGramThreads = 256;

template <int NT>
__global__ void __launch_bounds__(kGramThreads)
gram_kernel(const double* __restrict__ X, const double* __restrict__ Y, int n, int k, int ld,
            int rows_per_part, double* __restrict__ partial) {
  extern __shared__ double sh[];
  double* sx = sh;
  double* sy = sh + kGramRows * ld;
  const int tk = (k + 3) / 4;
  const int ntiles = tk * tk;
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
      const int ti = (tile / tk) * 4, tj = (tile % tk) * 4;
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
    const int ti = (tile / tk) * 4, tj = (tile % tk) * 4;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (ti + a < k && tj + b < k) out[(ti + a) * k + tj + b] = acc[t][a][b];
  }
}

__global__ void gram_reduce_kernel(const double* __restrict__ partial, int nparts, int kk,
                                   double* __restrict__ G) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= kk) return;
  double s = 0.0;
  for (int b = 0; b < nparts; ++b) s += partial[(size_t)b * kk + q];
  G[q] = s;
}

// ---- per-vector residual norms ----------------------------------------------
// partial[b][c] = sum_rows (AU - lam_c MU)^2,  partial[b][k + c] = sum_rows U^2.
__global__ void eigres_kernel(const double* __restrict__ AU, const double* __restrict__ MU,
                              const double* __restrict__ U, const double* __restrict__ lam, int n,
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
      const double d = AU[idx] - l * MU[idx];
      rr = fma(d, d, rr);
      uu = fma(U[idx], U[idx], uu);
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
// One warp per row; Yx (k x ldy) staged in shared memory; lane owns columns
// 2*lane + 64*u (double2 chunks).
template <int CPL>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
expand_kernel(const double* __restrict__ Zf, const double* __restrict__ X,
              const double* __restrict__ Yx, int n, int k, int ld, int ldy,
              double* __restrict__ U) {
  extern __shared__ double sy[];
  for (int q = threadIdx.x; q < k * ld; q += blockDim.x) {
    const int r = q / ld, c = q % ld;
    sy[q] = (c < k) ? Yx[(size_t)r * ldy + c] : 0.0;
  }
  __syncthreads();
  const int nch = ld / 2;
  const int lane = threadIdx.x & 31;
  for (int row = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); row < n;
       row += gridDim.x * kWarpsPerBlock) {
    double2 acc[CPL];
#pragma unroll
    for (int u = 0; u < CPL; ++u) {
      const int c = lane + 32 * u;
      acc[u] = (Zf && c < nch) ? ld2(Zf, (size_t)row * nch + c) : make_double2(0.0, 0.0);
    }
    const double* xr = X + (size_t)row * ld;
    for (int q = 0; q < k; ++q) {
      const double xv = xr[q];
#pragma unroll
      for (int u = 0; u < CPL; ++u) {
        const int c = lane + 32 * u;
        if (c < nch) {
          const double2 y = reinterpret_cast<const double2*>(sy + q * ld)[c];
          acc[u].x = fma(xv, y.x, acc[u].x);
          acc[u].y = fma(xv, y.y, acc[u].y);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < CPL; ++u) {
      const int c = lane + 32 * u;
      if (c < nch) st2(U, (size_t)row * nch + c, acc[u]);
    }
  }
}

__global__ void scale_rhs_kernel(const double* __restrict__ MU, const double* __restrict__ theta,
                                 size_t total, int ld, double* __restrict__ B) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < total) B[t] = theta[t % ld] * MU[t];
}

int blocks_for(size_t n, int b) { return (int)std::max<size_t>(1, (n + b - 1) / b); }

int cpl_for(int nch) { return nch <= 32 ? 1 : (nch <= 64 ? 2 : 4); }
}  // namespace

// ------------------------------------------------------------------ host ----
void spmm_am(const Mesh& m, const double* a, const double* mm, const double* X, int ld, double* AX,
             double* MX, cudaStream_t s) {
  const int nch = ld / 2;
  prof_begin(KC_SPMM, s);
  const int grid = blocks_for(m.n, kWarpsPerBlock);
  switch (cpl_for(nch)) {
    case 1: spmm_am_kernel<1><<<grid, kWarpsPerBlock * 32, 0, s>>>(m.row_ptr.get(), m.col.get(), a, mm, X, m.n, nch, AX, MX); break;
    case 2: spmm_am_kernel<2><<<grid, kWarpsPerBlock * 32, 0, s>>>(m.row_ptr.get(), m.col.get(), a, mm, X, m.n, nch, AX, MX); break;
    default: spmm_am_kernel<4><<<grid, kWarpsPerBlock * 32, 0, s>>>(m.row_ptr.get(), m.col.get(), a, mm, X, m.n, nch, AX, MX); break;
  }
  check_launch("spmm_am_kernel");
  prof_end(KC_SPMM, s, 20.0 * m.nnz + 4.0 * (m.n + 1) + 24.0 * m.n * ld, 4.0 * m.nnz * ld);
}

template <int MODE>
static void row_update(const Mesh& m, const double* a, const double* mm, const double* da,
                       const double* dm, const int* rows, int nrows, long long nnz_rows,
                       const double* X, double* Out, const double* B, const double* shift, int ld,
                       double omega, cudaStream_t s) {
  const int nch = ld / 2;
  const int grid = blocks_for(nrows, kWarpsPerBlock);
  if (nrows == 0) return;
  const int cls = (MODE == 2) ? KC_RESID : KC_SMOOTH;
  prof_begin(cls, s);
  switch (cpl_for(nch)) {
    case 1: row_update_kernel<1, MODE><<<grid, kWarpsPerBlock * 32, 0, s>>>(m.row_ptr.get(), m.col.get(), a, mm, da, dm, rows, nrows, X, Out, B, shift, nch, omega); break;
    case 2: row_update_kernel<2, MODE><<<grid, kWarpsPerBlock * 32, 0, s>>>(m.row_ptr.get(), m.col.get(), a, mm, da, dm, rows, nrows, X, Out, B, shift, nch, omega); break;
    default: row_update_kernel<4, MODE><<<grid, kWarpsPerBlock * 32, 0, s>>>(m.row_ptr.get(), m.col.get(), a, mm, da, dm, rows, nrows, X, Out, B, shift, nch, omega); break;
  }
  check_launch("row_update_kernel");
  // matrix rows, diagonals, own-row read + write, one share of the gathered block, B
  const double bytes = 20.0 * nnz_rows + 24.0 * nrows + 8.0 * nrows * ld * (B ? 4.0 : 3.0);
  prof_end(cls, s, bytes, 4.0 * nnz_rows * ld + 6.0 * nrows * ld);
}

void jacobi_sweep(const Mesh& m, const double* a, const double* mm, const double* da,
                  const double* dm, const double* X, double* Xout, const double* B,
                  const double* shift, int ld, double omega, cudaStream_t s) {
  row_update<0>(m, a, mm, da, dm, nullptr, m.n, m.nnz, X, Xout, B, shift, ld, omega, s);
}

void gs_colour_sweep(const Mesh& m, const Level& lv, int c, const double* a, const double* mm,
                     const double* da, const double* dm, double* X, const double* B,
                     const double* shift, int ld, cudaStream_t s) {
  const int b = lv.colour_ptr_host[c], e = lv.colour_ptr_host[c + 1];
  row_update<1>(m, a, mm, da, dm, lv.colour_rows.get() + b, e - b, lv.colour_nnz_host[c], X, X, B,
                shift, ld, 1.0, s);
}

void residual(const Mesh& m, const double* a, const double* mm, const double* X, const double* B,
              const double* shift, int ld, double* R, cudaStream_t s) {
  // the diagonal is not used in residual mode; pass the matrix values as placeholders
  row_update<2>(m, a, mm, a, mm, nullptr, m.n, m.nnz, X, R, B, shift, ld, 0.0, s);
}

void prolong(const Mesh& fine, const double* Xc, double* Y, int ld, bool add, cudaStream_t s) {
  const int nch = ld / 2;
  const size_t total = (size_t)fine.n * nch;
  prof_begin(KC_TRANSFER, s);
  prolong_kernel<<<blocks_for(total, 256), 256, 0, s>>>(fine.parents.get(), fine.n, Xc, Y, nch, add ? 1 : 0);
  check_launch("prolong_kernel");
  const double nc = (fine.n + 6) / 4.0;  // vertices of the coarse level of a refined sphere
  prof_end(KC_TRANSFER, s, 8.0 * fine.n + 8.0 * ld * (nc + fine.n * (add ? 2.0 : 1.0)), 1.0 * fine.n * ld);
}

void restrict_(const Mesh& coarse, const double* R, double* Zc, int ld, cudaStream_t s) {
  const int nch = ld / 2;
  const size_t total = (size_t)coarse.n * nch;
  prof_begin(KC_TRANSFER, s);
  restrict_kernel<<<blocks_for(total, 256), 256, 0, s>>>(coarse.row_ptr.get(), coarse.col.get(), coarse.mid.get(),
                                                          coarse.n, R, Zc, nch);
  check_launch("restrict_kernel");
  const double nf = 4.0 * coarse.n - 6.0;
  prof_end(KC_TRANSFER, s, 8.0 * coarse.nnz + 8.0 * ld * (nf + coarse.n), 2.0 * nf * ld);
}

int gram_parts(int n) { return std::max(1, std::min(304, (n + 63) / 64)); }

void gram(const double* X, const double* Y, int n, int k, int ld, double* G, double* partial,
          int nparts, cudaStream_t s) {
  const int rows_per_part = (n + nparts - 1) / nparts;
  const int tk = (k + 3) / 4;
  const int ntiles = tk * tk;
  const size_t smem = 2 * kGramRows * ld * sizeof(double);
  prof_begin(KC_GRAM, s);
  if (ntiles <= kGramThreads) gram_kernel<1><<<nparts, kGramThreads, smem, s>>>(X, Y, n, k, ld, rows_per_part, partial);
  else if (ntiles <= 2 * kGramThreads) gram_kernel<2><<<nparts, kGramThreads, smem, s>>>(X, Y, n, k, ld, rows_per_part, partial);
  else if (ntiles <= 4 * kGramThreads) gram_kernel<4><<<nparts, kGramThreads, smem, s>>>(X, Y, n, k, ld, rows_per_part, partial);
  else if (ntiles <= 8 * kGramThreads) gram_kernel<8><<<nparts, kGramThreads, smem, s>>>(X, Y, n, k, ld, rows_per_part, partial);
  else fail(BMG_ERR_INVALID_ARG, "gram: k too large (k <= 180)");
  check_launch("gram_kernel");
  gram_reduce_kernel<<<blocks_for(k * k, 256), 256, 0, s>>>(partial, nparts, k * k, G);
  check_launch("gram_reduce_kernel");
  prof_end(KC_GRAM, s, 16.0 * n * ld + 16.0 * nparts * k * k + 8.0 * k * k, 2.0 * n * k * k);
}

void eig_residuals(const double* AU, const double* MU, const double* U, const double* lam, int n,
                   int k, int ld, double* partial, int nparts, double* out, cudaStream_t s) {
  const int rows_per_part = (n + nparts - 1) / nparts;
  const int threads = std::max(k, (256 / k) * k);
  prof_begin(KC_SMALL, s);
  eigres_kernel<<<nparts, threads, 2 * threads * sizeof(double), s>>>(AU, MU, U, lam, n, k, ld,
                                                                      rows_per_part, partial);
  check_launch("eigres_kernel");
  gram_reduce_kernel<<<blocks_for(2 * k, 256), 256, 0, s>>>(partial, nparts, 2 * k, out);
  check_launch("gram_reduce_kernel");
  prof_end(KC_SMALL, s, 24.0 * n * ld, 5.0 * n * k);
}

void expand(const double* Zf, const double* X, const double* Yx, int n, int k, int ld, int ldy,
            double* U, cudaStream_t s) {
  const int nch = ld / 2;
  const size_t smem = (size_t)k * ld * sizeof(double);
  const int grid = std::max(1, std::min(blocks_for(n, kWarpsPerBlock), 4 * 152));
  prof_begin(KC_EXPAND, s);
  switch (cpl_for(nch)) {
    case 1:
      cudaFuncSetAttribute(expand_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      expand_kernel<1><<<grid, kWarpsPerBlock * 32, smem, s>>>(Zf, X, Yx, n, k, ld, ldy, U); break;
    case 2:
      cudaFuncSetAttribute(expand_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      expand_kernel<2><<<grid, kWarpsPerBlock * 32, smem, s>>>(Zf, X, Yx, n, k, ld, ldy, U); break;
    default:
      cudaFuncSetAttribute(expand_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      expand_kernel<4><<<grid, kWarpsPerBlock * 32, smem, s>>>(Zf, X, Yx, n, k, ld, ldy, U); break;
  }
  check_launch("expand_kernel");
  prof_end(KC_EXPAND, s, 24.0 * n * ld + 8.0 * k * k, 2.0 * n * k * k);
}

void scale_rhs(const double* MU, const double* theta, int n, int k, int ld, double* B, cudaStream_t s) {
  (void)k;
  const size_t total = (size_t)n * ld;
  scale_rhs_kernel<<<blocks_for(total, 256), 256, 0, s>>>(MU, theta, total, ld, B);
  check_launch("scale_rhs_kernel");
}

}  // namespace bmg

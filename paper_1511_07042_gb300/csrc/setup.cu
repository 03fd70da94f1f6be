// Set-up kernels: surface refinement with projection, vertex adjacency (CSR),
// P1 assembly, greedy colouring, Galerkin products.
//
// Refinement and assembly use explicitly rounded arithmetic (__dadd_rn, __dmul_rn,
// ...) in a fixed evaluation order so that meshes and matrices are reproducible
// bit for bit: new vertex m = (v_i + v_j) * 0.5, projected radially as
// m / sqrt((x*x + y*y) + z*z) (Sec. 3, Eq. proj-1 and the lift Eq. lift: the
// closest point on the unit sphere), times r(n) on a star-shaped perturbed sphere.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace bmg {

namespace {
constexpr int kMaxDeg = 32;    // incident triangles per vertex accepted by the mesh kernels
constexpr int kMaxRow = 40;    // CSR row length accepted by the Galerkin kernel
constexpr int kScanBlock = 1024;

__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }

// ------------------------------------------------------------------- scan ----
__global__ void scan_block_kernel(const int* in, int* out, int* sums, int n) {
  __shared__ int sh[kScanBlock];
  int i = blockIdx.x * kScanBlock + threadIdx.x;
  int v = (i < n) ? in[i] : 0;
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < kScanBlock; off <<= 1) {
    int t = (threadIdx.x >= off) ? sh[threadIdx.x - off] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) out[i + 1] = sh[threadIdx.x];  // inclusive, shifted by one
  if (threadIdx.x == kScanBlock - 1) sums[blockIdx.x] = sh[threadIdx.x];
}

__global__ void scan_add_kernel(int* out, const int* offs, int n) {
  int i = blockIdx.x * kScanBlock + threadIdx.x;
  if (i < n) out[i + 1] += offs[blockIdx.x];
}

__global__ void set_zero_kernel(int* p) { *p = 0; }
}  // namespace

// out[0] = 0, out[i+1] = in[0] + ... + in[i]; out has n+1 entries.
void exclusive_scan(const int* in, int* out, int n, int* total_host, cudaStream_t s) {
  set_zero_kernel<<<1, 1, 0, s>>>(out);
  if (n > 0) {
    int nb = (n + kScanBlock - 1) / kScanBlock;
    DBuf<int> sums(nb), soffs(nb + 1);
    scan_block_kernel<<<nb, kScanBlock, 0, s>>>(in, out, sums.get(), n);
    check_launch("scan_block_kernel");
    if (nb > 1) {
      exclusive_scan(sums.get(), soffs.get(), nb, nullptr, s);
      scan_add_kernel<<<nb, kScanBlock, 0, s>>>(out, soffs.get(), n);
      check_launch("scan_add_kernel");
    }
    BMG_CUDA(cudaStreamSynchronize(s));
  }
  if (total_host) {
    BMG_CUDA(cudaMemcpyAsync(total_host, out + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    BMG_CUDA(cudaStreamSynchronize(s));
  }
}

// --------------------------------------------------------- mesh pattern ----
namespace {
__global__ void count_incidence_kernel(const int* tris, int nt, int n, int* cnt, int* err) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  for (int c = 0; c < 3; ++c) {
    int v = tris[3 * t + c];
    if (v < 0 || v >= n) { atomicExch(err, 1); continue; }
    atomicAdd(&cnt[v], 1);
  }
}

__global__ void fill_incidence_kernel(const int* tris, int nt, int n, const int* ptr,
                                      int* cursor, int* inc) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  for (int c = 0; c < 3; ++c) {
    int v = tris[3 * t + c];
    if (v < 0 || v >= n) continue;
    int slot = atomicAdd(&cursor[v], 1);
    inc[ptr[v] + slot] = t;
  }
}

// Sort each vertex's incident triangles, collect its neighbours, and count the row.
// A closed two-manifold has every neighbour in exactly two incident triangles.
__global__ void row_count_kernel(const int* tris, int n, const int* ptr, int* inc, int* rowlen,
                                 int* err) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  int b = ptr[v], e = ptr[v + 1], d = e - b;
  if (d < 3 || d > kMaxDeg) { atomicExch(err, 2); rowlen[v] = 1; return; }
  for (int i = b + 1; i < e; ++i) {  // insertion sort, short lists
    int x = inc[i], j = i - 1;
    while (j >= b && inc[j] > x) { inc[j + 1] = inc[j]; --j; }
    inc[j + 1] = x;
  }
  int nb[2 * kMaxDeg];
  int m = 0;
  for (int i = b; i < e; ++i) {
    int t = inc[i];
    for (int c = 0; c < 3; ++c) {
      int u = tris[3 * t + c];
      if (u != v) nb[m++] = u;
    }
  }
  for (int i = 1; i < m; ++i) {
    int x = nb[i], j = i - 1;
    while (j >= 0 && nb[j] > x) { nb[j + 1] = nb[j]; --j; }
    nb[j + 1] = x;
  }
  int uniq = 0;
  for (int i = 0; i < m;) {
    int j = i;
    while (j < m && nb[j] == nb[i]) ++j;
    if (j - i != 2) atomicExch(err, 3);
    ++uniq;
    i = j;
  }
  rowlen[v] = uniq + 1;
}

__global__ void row_fill_kernel(const int* tris, int n, const int* ptr, const int* inc,
                                const int* row_ptr, int* col, int* diag_pos) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  int b = ptr[v], e = ptr[v + 1], d = e - b;
  if (d < 3 || d > kMaxDeg) return;
  int nb[3 * kMaxDeg];
  int m = 0;
  for (int i = b; i < e; ++i) {
    int t = inc[i];
    for (int c = 0; c < 3; ++c) nb[m++] = tris[3 * t + c];  // includes v itself
  }
  for (int i = 1; i < m; ++i) {
    int x = nb[i], j = i - 1;
    while (j >= 0 && nb[j] > x) { nb[j + 1] = nb[j]; --j; }
    nb[j + 1] = x;
  }
  int o = row_ptr[v], lim = row_ptr[v + 1];
  int last = -1;
  for (int i = 0; i < m; ++i) {
    if (nb[i] == last) continue;
    last = nb[i];
    if (o >= lim) break;
    if (last == v) diag_pos[v] = o;
    col[o++] = last;
  }
}

int grid_for(int n, int block) { return std::max(1, (n + block - 1) / block); }
}  // namespace

void build_mesh_pattern(Mesh& m, cudaStream_t s) {
  const int n = m.n, nt = m.n_tris;
  DBuf<int> cnt(n), cursor(n), err(1);
  BMG_CUDA(cudaMemsetAsync(cnt.get(), 0, sizeof(int) * n, s));
  BMG_CUDA(cudaMemsetAsync(cursor.get(), 0, sizeof(int) * n, s));
  BMG_CUDA(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
  count_incidence_kernel<<<grid_for(nt, 256), 256, 0, s>>>(m.tris.get(), nt, n, cnt.get(), err.get());
  check_launch("count_incidence_kernel");
  m.inc_ptr.alloc(n + 1);
  int total = 0;
  exclusive_scan(cnt.get(), m.inc_ptr.get(), n, &total, s);
  m.inc_tri.alloc(std::max(total, 1));
  fill_incidence_kernel<<<grid_for(nt, 256), 256, 0, s>>>(m.tris.get(), nt, n, m.inc_ptr.get(),
                                                          cursor.get(), m.inc_tri.get());
  check_launch("fill_incidence_kernel");
  DBuf<int> rowlen(n);
  row_count_kernel<<<grid_for(n, 128), 128, 0, s>>>(m.tris.get(), n, m.inc_ptr.get(),
                                                    m.inc_tri.get(), rowlen.get(), err.get());
  check_launch("row_count_kernel");
  int herr = 0;
  BMG_CUDA(cudaMemcpyAsync(&herr, err.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
  BMG_CUDA(cudaStreamSynchronize(s));
  if (herr == 1) fail(BMG_ERR_MESH, "triangle vertex index out of range");
  if (herr == 2) fail(BMG_ERR_MESH, "vertex with fewer than 3 or more than 32 incident triangles");
  if (herr == 3) fail(BMG_ERR_MESH, "mesh is not a closed two-manifold (an edge is not shared by exactly two triangles)");
  m.row_ptr.alloc(n + 1);
  exclusive_scan(rowlen.get(), m.row_ptr.get(), n, &m.nnz, s);
  m.col.alloc(m.nnz);
  m.diag_pos.alloc(n);
  row_fill_kernel<<<grid_for(n, 128), 128, 0, s>>>(m.tris.get(), n, m.inc_ptr.get(), m.inc_tri.get(),
                                                   m.row_ptr.get(), m.col.get(), m.diag_pos.get());
  check_launch("row_fill_kernel");
  BMG_CUDA(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------ refinement ----
// Real orthonormal spherical harmonics Y_lm, l <= 4, as Cartesian polynomials,
// each product evaluated left to right; r(n) = 1 + a * sum_q Y_q c_q accumulated in
// q order.  Normalisation constants come from the host (fill_sh_constants).
__device__ double sh_radius(double x, double y, double z, double amp, const double* C,
                            const double* cf) {
  const double xx = dmul(x, x), yy = dmul(y, y), zz0 = dmul(z, z);
  const double x2my2 = dsub(xx, yy);
  const double three_xx = dmul(dmul(3.0, x), x), three_yy = dmul(dmul(3.0, y), y);
  const double five_zz = dmul(dmul(5.0, z), z), seven_zz = dmul(dmul(7.0, z), z);
  double Y[25];
  Y[0] = C[0];
  Y[1] = dmul(C[1], y);
  Y[2] = dmul(C[1], z);
  Y[3] = dmul(C[1], x);
  Y[4] = dmul(dmul(C[2], x), y);
  Y[5] = dmul(dmul(C[2], y), z);
  Y[6] = dmul(C[3], dsub(dmul(dmul(3.0, z), z), 1.0));
  Y[7] = dmul(dmul(C[2], x), z);
  Y[8] = dmul(C[4], x2my2);
  Y[9] = dmul(dmul(C[5], y), dsub(three_xx, yy));
  Y[10] = dmul(dmul(dmul(C[6], x), y), z);
  Y[11] = dmul(dmul(C[7], y), dsub(five_zz, 1.0));
  Y[12] = dmul(dmul(C[8], z), dsub(five_zz, 3.0));
  Y[13] = dmul(dmul(C[7], x), dsub(five_zz, 1.0));
  Y[14] = dmul(dmul(C[9], z), x2my2);
  Y[15] = dmul(dmul(C[5], x), dsub(xx, three_yy));
  Y[16] = dmul(dmul(dmul(C[10], x), y), x2my2);
  Y[17] = dmul(dmul(dmul(C[11], y), z), dsub(three_xx, yy));
  Y[18] = dmul(dmul(dmul(C[12], x), y), dsub(seven_zz, 1.0));
  Y[19] = dmul(dmul(dmul(C[13], y), z), dsub(seven_zz, 3.0));
  const double z4 = dmul(dmul(dmul(z, z), z), z);
  Y[20] = dmul(C[14], dadd(dsub(dmul(35.0, z4), dmul(dmul(30.0, z), z)), 3.0));
  Y[21] = dmul(dmul(dmul(C[13], x), z), dsub(seven_zz, 3.0));
  Y[22] = dmul(dmul(C[15], x2my2), dsub(seven_zz, 1.0));
  Y[23] = dmul(dmul(dmul(C[11], x), z), dsub(xx, three_yy));
  Y[24] = dmul(C[16], dsub(dmul(xx, dsub(xx, three_yy)), dmul(yy, dsub(three_xx, yy))));
  (void)zz0;
  double acc = dmul(Y[0], cf[0]);
  for (int q = 1; q < 25; ++q) acc = dadd(acc, dmul(Y[q], cf[q]));
  return dadd(1.0, dmul(amp, acc));
}

__device__ void project_point(double mx, double my, double mz, double amp, const double* C,
                              const double* cf, double* out) {
  const double nrm = __dsqrt_rn(dadd(dadd(dmul(mx, mx), dmul(my, my)), dmul(mz, mz)));
  const double nx = ddiv(mx, nrm), ny = ddiv(my, nrm), nz = ddiv(mz, nrm);
  if (amp == 0.0) {
    out[0] = nx; out[1] = ny; out[2] = nz;
    return;
  }
  const double r = sh_radius(nx, ny, nz, amp, C, cf);
  out[0] = dmul(r, nx); out[1] = dmul(r, ny); out[2] = dmul(r, nz);
}

namespace {
__global__ void project_input_kernel(double* v, int n, double amp, const double* C, const double* cf) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double out[3];
  project_point(v[3 * i], v[3 * i + 1], v[3 * i + 2], amp, C, cf, out);
  v[3 * i] = out[0]; v[3 * i + 1] = out[1]; v[3 * i + 2] = out[2];
}

__global__ void upper_count_kernel(const int* row_ptr, const int* diag_pos, int n, int* cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) cnt[i] = row_ptr[i + 1] - diag_pos[i] - 1;
}

__global__ void new_vertices_kernel(const double* cv, const int* row_ptr, const int* col,
                                    const int* diag_pos, const int* eoff, int nc, double amp,
                                    const double* C, const double* cf, double* fv, int* par,
                                    int* mid) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nc) return;
  fv[3 * i] = cv[3 * i]; fv[3 * i + 1] = cv[3 * i + 1]; fv[3 * i + 2] = cv[3 * i + 2];
  par[2 * i] = i; par[2 * i + 1] = i;
  const int dp = diag_pos[i];
  mid[dp] = -1;
  for (int p = dp + 1; p < row_ptr[i + 1]; ++p) {
    const int j = col[p];
    const int v = nc + eoff[i] + (p - dp - 1);
    const double mx = dmul(dadd(cv[3 * i], cv[3 * j]), 0.5);
    const double my = dmul(dadd(cv[3 * i + 1], cv[3 * j + 1]), 0.5);
    const double mz = dmul(dadd(cv[3 * i + 2], cv[3 * j + 2]), 0.5);
    double out[3];
    project_point(mx, my, mz, amp, C, cf, out);
    fv[3 * v] = out[0]; fv[3 * v + 1] = out[1]; fv[3 * v + 2] = out[2];
    par[2 * v] = i; par[2 * v + 1] = j;
    mid[p] = v;
  }
}

__device__ __forceinline__ int find_in_row(const int* col, int b, int e, int key) {
  int lo = b, hi = e - 1;
  while (lo <= hi) {
    int m = (lo + hi) >> 1;
    int c = col[m];
    if (c == key) return m;
    if (c < key) lo = m + 1; else hi = m - 1;
  }
  return -1;
}

__global__ void lower_mid_kernel(const int* row_ptr, const int* col, const int* diag_pos, int n,
                                 int* mid) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int p = row_ptr[i]; p < diag_pos[i]; ++p) {
    int j = col[p];
    int q = find_in_row(col, row_ptr[j], row_ptr[j + 1], i);
    mid[p] = (q >= 0) ? mid[q] : -1;
  }
}

__global__ void child_tris_kernel(const int* ct, int nt, const int* row_ptr, const int* col,
                                  const int* mid, int* ft) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const int a = ct[3 * t], b = ct[3 * t + 1], c = ct[3 * t + 2];
  auto m = [&](int u, int w) {
    int q = find_in_row(col, row_ptr[u], row_ptr[u + 1], w);
    return q >= 0 ? mid[q] : -1;
  };
  const int mab = m(a, b), mbc = m(b, c), mca = m(c, a);
  int* o = ft + 12 * t;
  o[0] = a;   o[1] = mab;  o[2] = mca;
  o[3] = b;   o[4] = mbc;  o[5] = mab;
  o[6] = c;   o[7] = mca;  o[8] = mbc;
  o[9] = mab; o[10] = mbc; o[11] = mca;
}
}  // namespace

// Constants of the harmonics, computed on the host in the same order as the
// textbook closed forms: 17 distinct normalisations.
void fill_sh_constants(double* C) {
  const double pi = 3.141592653589793;
  C[0] = 0.5 * std::sqrt(1.0 / pi);
  C[1] = std::sqrt(3.0 / (4.0 * pi));
  C[2] = 0.5 * std::sqrt(15.0 / pi);
  C[3] = 0.25 * std::sqrt(5.0 / pi);
  C[4] = 0.25 * std::sqrt(15.0 / pi);
  C[5] = 0.25 * std::sqrt(35.0 / (2.0 * pi));
  C[6] = 0.5 * std::sqrt(105.0 / pi);
  C[7] = 0.25 * std::sqrt(21.0 / (2.0 * pi));
  C[8] = 0.25 * std::sqrt(7.0 / pi);
  C[9] = 0.25 * std::sqrt(105.0 / pi);
  C[10] = 0.75 * std::sqrt(35.0 / pi);
  C[11] = 0.75 * std::sqrt(35.0 / (2.0 * pi));
  C[12] = 0.75 * std::sqrt(5.0 / pi);
  C[13] = 0.75 * std::sqrt(5.0 / (2.0 * pi));
  C[14] = (3.0 / 16.0) * std::sqrt(1.0 / pi);
  C[15] = (3.0 / 8.0) * std::sqrt(5.0 / pi);
  C[16] = (3.0 / 16.0) * std::sqrt(35.0 / pi);
}

void project_input(Mesh& m, double amplitude, const double* C, const double* cf, cudaStream_t s) {
  project_input_kernel<<<grid_for(m.n, 128), 128, 0, s>>>(m.verts.get(), m.n, amplitude, C, cf);
  check_launch("project_input_kernel");
}

// Uniform refinement of c into f (Sec. 3): midpoint numbering by lexicographic edge
// rank, children ordered as documented in bmg.h; fills c.mid.
void refine_mesh(const Mesh& cc, Mesh& f, double amplitude, const double* C, const double* cf,
                 cudaStream_t s) {
  Mesh& c = const_cast<Mesh&>(cc);
  const int nc = c.n;
  DBuf<int> cnt(nc), eoff(nc + 1);
  upper_count_kernel<<<grid_for(nc, 256), 256, 0, s>>>(c.row_ptr.get(), c.diag_pos.get(), nc, cnt.get());
  check_launch("upper_count_kernel");
  int E = 0;
  exclusive_scan(cnt.get(), eoff.get(), nc, &E, s);
  f.n = nc + E;
  f.n_tris = 4 * c.n_tris;
  f.verts.alloc(3 * (size_t)f.n);
  f.parents.alloc(2 * (size_t)f.n);
  f.tris.alloc(3 * (size_t)f.n_tris);
  c.mid.alloc(c.nnz);
  new_vertices_kernel<<<grid_for(nc, 128), 128, 0, s>>>(c.verts.get(), c.row_ptr.get(), c.col.get(),
                                                        c.diag_pos.get(), eoff.get(), nc, amplitude, C,
                                                        cf, f.verts.get(), f.parents.get(), c.mid.get());
  check_launch("new_vertices_kernel");
  lower_mid_kernel<<<grid_for(nc, 256), 256, 0, s>>>(c.row_ptr.get(), c.col.get(), c.diag_pos.get(), nc,
                                                     c.mid.get());
  check_launch("lower_mid_kernel");
  child_tris_kernel<<<grid_for(c.n_tris, 256), 256, 0, s>>>(c.tris.get(), c.n_tris, c.row_ptr.get(),
                                                            c.col.get(), c.mid.get(), f.tris.get());
  check_launch("child_tris_kernel");
  build_mesh_pattern(f, s);
}

// ------------------------------------------------------------- assembly ----
namespace {
struct V3 { double x, y, z; };
__device__ __forceinline__ V3 ld3(const double* v, int i) { return {v[3 * i], v[3 * i + 1], v[3 * i + 2]}; }
__device__ __forceinline__ V3 sub3(V3 a, V3 b) { return {dsub(a.x, b.x), dsub(a.y, b.y), dsub(a.z, b.z)}; }
__device__ __forceinline__ V3 cross3(V3 u, V3 v) {
  return {dsub(dmul(u.y, v.z), dmul(u.z, v.y)), dsub(dmul(u.z, v.x), dmul(u.x, v.z)),
          dsub(dmul(u.x, v.y), dmul(u.y, v.x))};
}
__device__ __forceinline__ double dot3(V3 u, V3 v) {
  return dadd(dadd(dmul(u.x, v.x), dmul(u.y, v.y)), dmul(u.z, v.z));
}
__device__ __forceinline__ double norm3(V3 u) { return __dsqrt_rn(dot3(u, u)); }
__device__ __forceinline__ double cot_at(V3 p, V3 q, V3 apex) {
  V3 u = sub3(p, apex), v = sub3(q, apex);
  return ddiv(dot3(u, v), norm3(cross3(u, v)));
}

// One thread per vertex: walk the incident triangles in ascending order and add the
// element entries of this vertex's row (cotangent stiffness, consistent mass).
__global__ void assemble_kernel(const double* verts, const int* tris, int n, const int* inc_ptr,
                                const int* inc_tri, const int* row_ptr, const int* col,
                                double* va, double* vm) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int rb = row_ptr[i], re = row_ptr[i + 1];
  for (int p = rb; p < re; ++p) { va[p] = 0.0; vm[p] = 0.0; }
  for (int q = inc_ptr[i]; q < inc_ptr[i + 1]; ++q) {
    const int t = inc_tri[q];
    const int g[3] = {tris[3 * t], tris[3 * t + 1], tris[3 * t + 2]};
    const V3 pa = ld3(verts, g[0]), pb = ld3(verts, g[1]), pc = ld3(verts, g[2]);
    const double ca = cot_at(pb, pc, pa), cb = cot_at(pc, pa, pb), cc = cot_at(pa, pb, pc);
    const double area = dmul(0.5, norm3(cross3(sub3(pb, pa), sub3(pc, pa))));
    double K[3][3];
    K[0][1] = K[1][0] = dmul(-0.5, cc);
    K[1][2] = K[2][1] = dmul(-0.5, ca);
    K[0][2] = K[2][0] = dmul(-0.5, cb);
    K[0][0] = dmul(0.5, dadd(cb, cc));
    K[1][1] = dmul(0.5, dadd(cc, ca));
    K[2][2] = dmul(0.5, dadd(ca, cb));
    const double moff = ddiv(area, 12.0), mdia = ddiv(area, 6.0);
    const int li = (g[0] == i) ? 0 : (g[1] == i ? 1 : 2);
    for (int lj = 0; lj < 3; ++lj) {
      const int j = g[lj];
      int p = rb;
      while (p < re && col[p] != j) ++p;
      if (p == re) continue;
      va[p] = dadd(va[p], K[li][lj]);
      vm[p] = dadd(vm[p], li == lj ? mdia : moff);
    }
  }
}
}  // namespace

void assemble_p1(Mesh& m, cudaStream_t s) {
  m.valA.alloc(m.nnz);
  m.valM.alloc(m.nnz);
  assemble_kernel<<<grid_for(m.n, 128), 128, 0, s>>>(m.verts.get(), m.tris.get(), m.n, m.inc_ptr.get(),
                                                     m.inc_tri.get(), m.row_ptr.get(), m.col.get(),
                                                     m.valA.get(), m.valM.get());
  check_launch("assemble_kernel");
}

// ------------------------------------------------------------ colouring ----
namespace {
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  // SplitMix64 output function (Steele, Lea & Flood 2014)
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ bool higher(uint64_t hu, int u, uint64_t hv, int v) {
  return hu > hv || (hu == hv && u > v);
}

// One Jones-Plassmann round: an uncoloured vertex whose higher-priority neighbours
// are all coloured takes the smallest colour none of them uses.  The result equals
// sequential greedy colouring in descending priority.
__global__ void jp_round_kernel(const int* row_ptr, const int* col, int n, int* colour,
                                int* remaining) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  if (colour[v] >= 0) return;
  const uint64_t hv = splitmix64((uint64_t)v);
  uint64_t used = 0;
  for (int p = row_ptr[v]; p < row_ptr[v + 1]; ++p) {
    const int u = col[p];
    if (u == v) continue;
    const int cu = ((volatile int*)colour)[u];
    if (cu < 0) {
      if (higher(splitmix64((uint64_t)u), u, hv, v)) { atomicAdd(remaining, 1); return; }
    } else if (cu < 64) {
      used |= (1ull << cu);
    }
  }
  int c = 0;
  while (c < 64 && (used >> c) & 1ull) ++c;
  colour[v] = c;
}

// The same round on the distance-2 graph (vertices within two edges): rows of one
// colour then share no column, as a Kaczmarz sweep needs.  Equal to sequential
// greedy colouring of that graph in descending priority.
__global__ void jp2_round_kernel(const int* row_ptr, const int* col, int n, int* colour, int* remaining) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  if (colour[v] >= 0) return;
  const uint64_t hv = splitmix64((uint64_t)v);
  uint64_t used = 0;
  for (int p = row_ptr[v]; p < row_ptr[v + 1]; ++p) {
    const int u = col[p];
    for (int q = row_ptr[u]; q < row_ptr[u + 1]; ++q) {
      const int x = col[q];
      if (x == v) continue;
      const int cx = ((volatile int*)colour)[x];
      if (cx < 0) {
        if (higher(splitmix64((uint64_t)x), x, hv, v)) { atomicAdd(remaining, 1); return; }
      } else if (cx < 64) {
        used |= (1ull << cx);
      }
    }
  }
  int c = 0;
  while (c < 64 && (used >> c) & 1ull) ++c;
  colour[v] = c;
}

__global__ void flag_colour_kernel(const int* colour, int n, int c, int* flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = (colour[i] == c) ? 1 : 0;
}
__global__ void scatter_colour_kernel(const int* colour, int n, int c, const int* pos, int base,
                                      int* rows) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && colour[i] == c) rows[base + pos[i]] = i;
}
__global__ void max_kernel(const int* x, int n, int* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicMax(out, x[i]);
}
}  // namespace

void colour_level(const Mesh& m, Level& lv, cudaStream_t s) { colour_mesh(m, lv.col1, false, s); }
void colour_level2(const Mesh& m, Level& lv, cudaStream_t s) {
  if (lv.col2.n_colours) return;
  colour_mesh(m, lv.col2, true, s);
  // rows of each colour in the Morton order of the level's row order (rank of a row)
  std::vector<int> order(m.n), rank(m.n), rows(m.n);
  BMG_CUDA(cudaMemcpyAsync(order.data(), m.row_order.get(), sizeof(int) * m.n, cudaMemcpyDeviceToHost, s));
  BMG_CUDA(cudaMemcpyAsync(rows.data(), lv.col2.rows.get(), sizeof(int) * m.n, cudaMemcpyDeviceToHost, s));
  BMG_CUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < m.n; ++i) rank[order[i]] = i;
  for (int c = 0; c < lv.col2.n_colours; ++c)
    std::sort(rows.begin() + lv.col2.ptr_host[c], rows.begin() + lv.col2.ptr_host[c + 1],
              [&](int a, int b) { return rank[a] < rank[b]; });
  BMG_CUDA(cudaMemcpyAsync(lv.col2.rows.get(), rows.data(), sizeof(int) * m.n, cudaMemcpyHostToDevice, s));
  BMG_CUDA(cudaStreamSynchronize(s));
}

void colour_mesh(const Mesh& m, Colouring& cl, bool distance2, cudaStream_t s) {
  const int n = m.n;
  cl.colour.alloc(n);
  BMG_CUDA(cudaMemsetAsync(cl.colour.get(), 0xff, sizeof(int) * n, s));
  DBuf<int> rem(1);
  for (int round = 0; round < 100000; ++round) {
    BMG_CUDA(cudaMemsetAsync(rem.get(), 0, sizeof(int), s));
    if (distance2)
      jp2_round_kernel<<<grid_for(n, 256), 256, 0, s>>>(m.row_ptr.get(), m.col.get(), n, cl.colour.get(), rem.get());
    else
      jp_round_kernel<<<grid_for(n, 256), 256, 0, s>>>(m.row_ptr.get(), m.col.get(), n, cl.colour.get(), rem.get());
    check_launch("jp_round_kernel");
    int h = 0;
    BMG_CUDA(cudaMemcpyAsync(&h, rem.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    BMG_CUDA(cudaStreamSynchronize(s));
    if (h == 0) break;
  }
  DBuf<int> mx(1);
  BMG_CUDA(cudaMemsetAsync(mx.get(), 0, sizeof(int), s));
  max_kernel<<<grid_for(n, 256), 256, 0, s>>>(cl.colour.get(), n, mx.get());
  int hmax = 0;
  BMG_CUDA(cudaMemcpyAsync(&hmax, mx.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
  BMG_CUDA(cudaStreamSynchronize(s));
  if (hmax >= 63) fail(BMG_ERR_MESH, "colouring needs more than 63 colours");
  cl.n_colours = hmax + 1;
  cl.rows.alloc(n);
  cl.ptr.alloc(cl.n_colours + 1);
  cl.ptr_host.assign(cl.n_colours + 1, 0);
  DBuf<int> flag(n), pos(n + 1);
  int base = 0;
  for (int c = 0; c < cl.n_colours; ++c) {
    flag_colour_kernel<<<grid_for(n, 256), 256, 0, s>>>(cl.colour.get(), n, c, flag.get());
    int cntc = 0;
    exclusive_scan(flag.get(), pos.get(), n, &cntc, s);
    scatter_colour_kernel<<<grid_for(n, 256), 256, 0, s>>>(cl.colour.get(), n, c, pos.get(), base,
                                                           cl.rows.get());
    cl.ptr_host[c] = base;
    base += cntc;
  }
  cl.ptr_host[cl.n_colours] = base;
  BMG_CUDA(cudaMemcpyAsync(cl.ptr.get(), cl.ptr_host.data(),
                           sizeof(int) * (cl.n_colours + 1), cudaMemcpyHostToDevice, s));
  std::vector<int> hrp(n + 1), hrows(n);
  BMG_CUDA(cudaMemcpyAsync(hrp.data(), m.row_ptr.get(), sizeof(int) * (n + 1), cudaMemcpyDeviceToHost, s));
  BMG_CUDA(cudaMemcpyAsync(hrows.data(), cl.rows.get(), sizeof(int) * n, cudaMemcpyDeviceToHost, s));
  BMG_CUDA(cudaStreamSynchronize(s));
  cl.nnz_host.assign(cl.n_colours, 0);
  for (int c = 0; c < cl.n_colours; ++c)
    for (int q = cl.ptr_host[c]; q < cl.ptr_host[c + 1]; ++q)
      cl.nnz_host[c] += hrp[hrows[q] + 1] - hrp[hrows[q]];
}

// Processing order of the rows of mesh m for the row kernels: vertices sorted by the
// 30-bit Morton code of their position in the bounding box (ties by index), and the
// rows of each colour of lv in the same order.  Any order gives the same results
// (every row is computed alone, rows of one colour are never neighbours); this one
// makes warps that run together gather nearby rows of the vector block, so that the
// gathers hit L2 instead of HBM.
void locality_order(Mesh& m, Level& lv, cudaStream_t s) {
  const int n = m.n;
  std::vector<double> v(3 * (size_t)n);
  std::vector<int> rows(n);
  BMG_CUDA(cudaMemcpyAsync(v.data(), m.verts.get(), sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
  BMG_CUDA(cudaMemcpyAsync(rows.data(), lv.col1.rows.get(), sizeof(int) * n, cudaMemcpyDeviceToHost, s));
  BMG_CUDA(cudaStreamSynchronize(s));
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int i = 0; i < n; ++i)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], v[3 * i + d]);
      hi[d] = std::max(hi[d], v[3 * i + d]);
    }
  auto spread = [](uint32_t x) {   // 10 bits -> every third bit
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
  };
  std::vector<uint32_t> key(n);
  for (int i = 0; i < n; ++i) {
    uint32_t q[3];
    for (int d = 0; d < 3; ++d) {
      const double w = hi[d] > lo[d] ? (v[3 * i + d] - lo[d]) / (hi[d] - lo[d]) : 0.0;
      q[d] = (uint32_t)std::min(1023.0, std::max(0.0, w * 1024.0));
    }
    key[i] = (spread(q[0]) << 2) | (spread(q[1]) << 1) | spread(q[2]);
  }
  auto before = [&](int a, int b) { return key[a] < key[b] || (key[a] == key[b] && a < b); };
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), before);
  for (int c = 0; c < lv.col1.n_colours; ++c)
    std::sort(rows.begin() + lv.col1.ptr_host[c], rows.begin() + lv.col1.ptr_host[c + 1], before);
  m.row_order.alloc(n);
  BMG_CUDA(cudaMemcpyAsync(m.row_order.get(), order.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
  BMG_CUDA(cudaMemcpyAsync(lv.col1.rows.get(), rows.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
  BMG_CUDA(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------- Galerkin ----
namespace {
// Coarse row i of P^T G P: fine rows a with P[a,i] != 0 are i (weight 1) and the
// midpoints of the edges at i (weight 1/2); fine column b spreads to its parents
// (weight 1, or 1/2 each).
__global__ void galerkin_kernel(const int* crow, const int* ccol, const int* cmid, int nc,
                                const int* frow, const int* fcol, const int* fpar,
                                const double* fa, const double* fm, double* ca, double* cm,
                                int* err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nc) return;
  const int rb = crow[i], re = crow[i + 1];
  const int len = re - rb;
  if (len > kMaxRow) { atomicExch(err, 1); return; }
  double accA[kMaxRow], accM[kMaxRow];
  for (int q = 0; q < len; ++q) { accA[q] = 0.0; accM[q] = 0.0; }
  for (int pp = rb - 1; pp < re; ++pp) {
    int a;
    double wa;
    if (pp < rb) { a = i; wa = 1.0; }
    else {
      if (ccol[pp] == i) continue;
      a = cmid[pp]; wa = 0.5;
      if (a < 0) { atomicExch(err, 2); continue; }
    }
    for (int q = frow[a]; q < frow[a + 1]; ++q) {
      const int b = fcol[q];
      const int b1 = fpar[2 * b], b2 = fpar[2 * b + 1];
      const double ga = wa * fa[q], gm = wa * fm[q];
      const int targets[2] = {b1, b2};
      const int nt = (b1 == b2) ? 1 : 2;
      const double wb = (b1 == b2) ? 1.0 : 0.5;
      for (int u = 0; u < nt; ++u) {
        int slot = -1;
        for (int r = 0; r < len; ++r)
          if (ccol[rb + r] == targets[u]) { slot = r; break; }
        if (slot < 0) { atomicExch(err, 2); continue; }
        accA[slot] += ga * wb;
        accM[slot] += gm * wb;
      }
    }
  }
  for (int q = 0; q < len; ++q) { ca[rb + q] = accA[q]; cm[rb + q] = accM[q]; }
}

__global__ void diag_kernel(const int* diag_pos, int n, const double* a, const double* m,
                            double* da, double* dm) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) { da[i] = a[diag_pos[i]]; dm[i] = m[diag_pos[i]]; }
}
}  // namespace

void galerkin(const Mesh& fine, const Mesh& coarse, const double* fa, const double* fm, double* ca,
              double* cm, cudaStream_t s) {
  DBuf<int> err(1);
  BMG_CUDA(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
  galerkin_kernel<<<grid_for(coarse.n, 128), 128, 0, s>>>(
      coarse.row_ptr.get(), coarse.col.get(), coarse.mid.get(), coarse.n, fine.row_ptr.get(),
      fine.col.get(), fine.parents.get(), fa, fm, ca, cm, err.get());
  check_launch("galerkin_kernel");
  int h = 0;
  BMG_CUDA(cudaMemcpyAsync(&h, err.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
  BMG_CUDA(cudaStreamSynchronize(s));
  if (h) fail(BMG_ERR_MESH, "Galerkin product left the coarse pattern");
}

void extract_diag(const Mesh& m, const double* a, const double* mm, double* da, double* dm,
                  cudaStream_t s) {
  diag_kernel<<<grid_for(m.n, 256), 256, 0, s>>>(m.diag_pos.get(), m.n, a, mm, da, dm);
  check_launch("diag_kernel");
}

}  // namespace bmg

// C ABI of libbmg: set-up, hierarchy, the BFMG solve and the per-step entry points.
//
// The solve is Alg. 4 (BFMG) over levels 2..L with the BMG cycle of Alg. 3 on each
// level f:
//   1. [AX | MX] on the k-block X                       (matrix form, Eq. pb-f-aux-mat)
//   2. Grams X^T AX, X^T MX and the couplings Q^T AX, Q^T MX by the restriction chain
//      (block matrices of Sec. 4.1; Q = P_2 ... P_f)
//   3. eigensolve in V_{h_1} + span X, k pairs nearest sigma        (Alg. 2 step 4)
//   4. Ritz vectors U = Q Y_c + X Y_x, their residuals; stop when all wanted pairs
//      meet tol (finest level) or after the intermediate cycle cap
//   5. source problems from U smoothed on level f, then corrections on coarser
//      levels (Galerkin operators) prolonged back        (Alg. 3 step 3, Eq. pb-m-s)
// Between levels the Ritz vectors are prolongated (Alg. 4 step 3, Eq. proj-1).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"

namespace bmg {

static thread_local std::string g_last_error = "no error";

void set_error(const std::string& msg) { g_last_error = msg; }

[[noreturn]] void fail(bmg_status code, const std::string& msg) { throw BmgException{code, msg}; }

void check_cuda(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(e == cudaErrorMemoryAllocation ? BMG_ERR_OOM : BMG_ERR_CUDA,
         std::string(what) + ": " + cudaGetErrorString(e));
  }
}

void check_launch(const char* what) {
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) fail(BMG_ERR_CUDA, std::string("launch of ") + what + ": " + cudaGetErrorString(e));
}

namespace {

template <typename F>
bmg_status guarded(F&& f) {
  try {
    f();
    return BMG_OK;
  } catch (const BmgException& e) {
    set_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return BMG_ERR_OOM;
  } catch (...) {
    set_error("unknown error");
    return BMG_ERR_CUDA;
  }
}

__global__ void csr_to_dense_kernel(const int* row_ptr, const int* col, const double* v, int n,
                                    double* D) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int j = 0; j < n; ++j) D[i * n + j] = 0.0;
  for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p) D[i * n + col[p]] = v[p];
}

__global__ void row_abs_max_kernel(const int* row_ptr, const double* v, int n,
                                   unsigned long long* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p) s += fabs(v[p]);
  atomicMax(out, (unsigned long long)__double_as_longlong(s));
}

__global__ void ratio_max_kernel(const double* da, const double* dm, int n, unsigned long long* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double r = dm[i] / da[i];
  if (!(r >= 0.0)) r = 1e300;
  atomicMax(out, (unsigned long long)__double_as_longlong(r));
}




int grid_of(size_t n, int b) { return (int)std::max<size_t>(1, (n + b - 1) / b); }

}  // namespace
}  // namespace bmg

using namespace bmg;

// ------------------------------------------------------------------------------
extern "C" void bmg_default_options(bmg_options* o) {
  if (!o) return;
  o->smoother = BMG_SMOOTH_JACOBI;
  o->nu = 2;
  o->omega = 2.0 / 3.0;
  o->form = BMG_FORM_SHIFTED;
  o->vcycle_depth = 99;
  o->cycles_intermediate = 6;
  o->tol_intermediate = -1.0;
  o->max_cycles = 200;
  o->precision = BMG_PREC_FP64;
  o->switch_tol = 1e-7;
  o->stop_after_cycles = 0;
  o->resume = 0;
  o->tensor_cores = 1;
  o->autotune = 1;
  o->graphs = 1;
  o->adaptive_shift = 0;
  o->selection = 0;
  o->index_first = 0;
  o->coarse_start = 0;
}

extern "C" const char* bmg_last_error(void) { return g_last_error.c_str(); }

extern "C" void bmg_destroy(bmg_problem* p) {
  if (!p) return;
  try { delete p; } catch (...) {}
}

extern "C" bmg_status bmg_assemble(const double* verts, int n_verts, const int* tris, int n_tris,
                                   int refinements, double amplitude, const double* sh_coefs,
                                   void* stream, bmg_problem** out) {
  return guarded([&] {
    TraceRange trace("bmg_assemble");
    if (!out) fail(BMG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!verts || !tris || n_verts < 4 || n_tris < 4) fail(BMG_ERR_INVALID_ARG, "empty or null mesh");
    if (refinements < 0 || refinements > 10) fail(BMG_ERR_INVALID_ARG, "refinements must be in 0..10");
    if (amplitude != 0.0 && !sh_coefs) fail(BMG_ERR_INVALID_ARG, "sh_coefs is NULL");
    if (!std::isfinite(amplitude)) fail(BMG_ERR_INVALID_ARG, "amplitude not finite");
    for (int i = 0; i < 3 * n_tris; ++i)
      if (tris[i] < 0 || tris[i] >= n_verts) fail(BMG_ERR_MESH, "triangle index out of range");
    std::unique_ptr<bmg_problem> p(new bmg_problem());
    p->stream = (cudaStream_t)stream;
    cudaStream_t s = p->stream;
    p->R = refinements;
    p->amplitude = amplitude;
    p->mesh.resize(refinements + 1);
    double C[17];
    fill_sh_constants(C);
    DBuf<double> dC(17), dcf(25);
    double cf[25] = {0};
    if (amplitude != 0.0) std::memcpy(cf, sh_coefs, sizeof(cf));
    BMG_CUDA(cudaMemcpyAsync(dC.get(), C, sizeof(C), cudaMemcpyHostToDevice, s));
    BMG_CUDA(cudaMemcpyAsync(dcf.get(), cf, sizeof(cf), cudaMemcpyHostToDevice, s));
    Mesh& m0 = p->mesh[0];
    m0.n = n_verts;
    m0.n_tris = n_tris;
    m0.verts.alloc(3 * (size_t)n_verts);
    m0.tris.alloc(3 * (size_t)n_tris);
    m0.parents.alloc(2 * (size_t)n_verts);
    BMG_CUDA(cudaMemcpyAsync(m0.verts.get(), verts, sizeof(double) * 3 * n_verts, cudaMemcpyHostToDevice, s));
    BMG_CUDA(cudaMemcpyAsync(m0.tris.get(), tris, sizeof(int) * 3 * n_tris, cudaMemcpyHostToDevice, s));
    {
      std::vector<int> par(2 * (size_t)n_verts);
      for (int i = 0; i < n_verts; ++i) { par[2 * i] = i; par[2 * i + 1] = i; }
      BMG_CUDA(cudaMemcpyAsync(m0.parents.get(), par.data(), sizeof(int) * par.size(), cudaMemcpyHostToDevice, s));
      BMG_CUDA(cudaStreamSynchronize(s));
    }
    project_input(m0, amplitude, dC.get(), dcf.get(), s);
    build_mesh_pattern(m0, s);
    for (int r = 1; r <= refinements; ++r) {
      refine_mesh(p->mesh[r - 1], p->mesh[r], amplitude, dC.get(), dcf.get(), s);
      assemble_p1(p->mesh[r], s);
    }
    BMG_CUDA(cudaStreamSynchronize(s));
    *out = p.release();
  });
}

extern "C" bmg_status bmg_hierarchy(bmg_problem* p, int levels) {
  return guarded([&] {
    TraceRange trace("bmg_hierarchy");
    if (!p) fail(BMG_ERR_INVALID_ARG, "null problem");
    if (levels < 2 || levels > p->R) fail(BMG_ERR_INVALID_ARG, "levels must be in 2..refinements");
    if (p->L) fail(BMG_ERR_STATE, "hierarchy already built");
    cudaStream_t s = p->stream;
    const int L = levels;
    p->r0 = p->R - L + 1;
    if (p->r0 < 1) fail(BMG_ERR_INVALID_ARG, "coarsest level must be refinement >= 1");
    p->lev.clear();
    p->lev.resize(L + 1);
    for (int l = 1; l <= L; ++l) {
      p->lev[l].refinement = p->r0 + l - 1;
      colour_level(p->meshOf(l), p->lev[l], s);
      locality_order(p->meshOf(l), p->lev[l], s);
    }
    p->ops.clear();
    p->ops.resize(L + 1);
    p->norm1.assign(L + 1, 0.0);
    DBuf<unsigned long long> um(1);
    for (int f = 2; f <= L; ++f) {
      p->ops[f].resize(f + 1);
      for (int j = f; j >= 1; --j) {
        const Mesh& mj = p->meshOf(j);
        OpSet& o = p->ops[f][j];
        if (j < f) {
          o.a.alloc(mj.nnz);
          o.m.alloc(mj.nnz);
          galerkin(p->meshOf(j + 1), mj, p->opA(f, j + 1), p->opM(f, j + 1), o.a.get(), o.m.get(), s);
        }
        o.da.alloc(mj.n);
        o.dm.alloc(mj.n);
        extract_diag(mj, p->opA(f, j), p->opM(f, j), o.da.get(), o.dm.get(), s);
      }
      const Mesh& mf = p->meshOf(f);
      BMG_CUDA(cudaMemsetAsync(um.get(), 0, sizeof(unsigned long long), s));
      row_abs_max_kernel<<<grid_of(mf.n, 256), 256, 0, s>>>(mf.row_ptr.get(), mf.valA.get(), mf.n, um.get());
      check_launch("row_abs_max_kernel");
      unsigned long long h = 0;
      BMG_CUDA(cudaMemcpyAsync(&h, um.get(), sizeof(h), cudaMemcpyDeviceToHost, s));
      BMG_CUDA(cudaStreamSynchronize(s));
      double nrm;
      std::memcpy(&nrm, &h, sizeof(nrm));
      p->norm1[f] = nrm;
    }
    p->L = L;
  });
}

// ----------------------------------------------------------------- inspection -
static const Mesh& mesh_at(const bmg_problem* p, int r) {
  if (!p) fail(BMG_ERR_INVALID_ARG, "null problem");
  if (r < 0 || r > p->R) fail(BMG_ERR_INVALID_ARG, "refinement out of range");
  return p->mesh[r];
}

extern "C" bmg_status bmg_get_sizes(const bmg_problem* p, int r, int* n, int* nt, int* nnz) {
  return guarded([&] {
    const Mesh& m = mesh_at(p, r);
    if (n) *n = m.n;
    if (nt) *nt = m.n_tris;
    if (nnz) *nnz = m.nnz;
  });
}

extern "C" bmg_status bmg_get_mesh(const bmg_problem* p, int r, double* verts, int* tris, int* parents) {
  return guarded([&] {
    const Mesh& m = mesh_at(p, r);
    if (verts) BMG_CUDA(cudaMemcpy(verts, m.verts.get(), sizeof(double) * 3 * m.n, cudaMemcpyDeviceToHost));
    if (tris) BMG_CUDA(cudaMemcpy(tris, m.tris.get(), sizeof(int) * 3 * m.n_tris, cudaMemcpyDeviceToHost));
    if (parents) BMG_CUDA(cudaMemcpy(parents, m.parents.get(), sizeof(int) * 2 * m.n, cudaMemcpyDeviceToHost));
  });
}

extern "C" bmg_status bmg_get_csr(const bmg_problem* p, int r, int* row_ptr, int* col, double* a, double* mm) {
  return guarded([&] {
    const Mesh& m = mesh_at(p, r);
    if (row_ptr) BMG_CUDA(cudaMemcpy(row_ptr, m.row_ptr.get(), sizeof(int) * (m.n + 1), cudaMemcpyDeviceToHost));
    if (col) BMG_CUDA(cudaMemcpy(col, m.col.get(), sizeof(int) * m.nnz, cudaMemcpyDeviceToHost));
    if ((a || mm) && r < 1) fail(BMG_ERR_INVALID_ARG, "no matrices on refinement 0");
    if (a) BMG_CUDA(cudaMemcpy(a, m.valA.get(), sizeof(double) * m.nnz, cudaMemcpyDeviceToHost));
    if (mm) BMG_CUDA(cudaMemcpy(mm, m.valM.get(), sizeof(double) * m.nnz, cudaMemcpyDeviceToHost));
  });
}

static void check_levels(const bmg_problem* p, int f, int j) {
  if (!p) fail(BMG_ERR_INVALID_ARG, "null problem");
  if (!p->L) fail(BMG_ERR_STATE, "bmg_hierarchy not called");
  if (f < 1 || f > p->L || j < 1 || j > f) fail(BMG_ERR_INVALID_ARG, "level out of range");
}

extern "C" bmg_status bmg_get_galerkin(const bmg_problem* p, int f, int j, double* a, double* mm) {
  return guarded([&] {
    check_levels(p, f, j);
    if (f < 2) fail(BMG_ERR_INVALID_ARG, "f must be >= 2");
    const Mesh& m = p->meshOf(j);
    if (a) BMG_CUDA(cudaMemcpy(a, p->opA(f, j), sizeof(double) * m.nnz, cudaMemcpyDeviceToHost));
    if (mm) BMG_CUDA(cudaMemcpy(mm, p->opM(f, j), sizeof(double) * m.nnz, cudaMemcpyDeviceToHost));
  });
}

extern "C" bmg_status bmg_get_colouring(const bmg_problem* p, int level, int* colour, int* n_colours) {
  return guarded([&] {
    check_levels(p, level, level);
    if (colour) BMG_CUDA(cudaMemcpy(colour, p->lev[level].col1.colour.get(), sizeof(int) * p->meshOf(level).n, cudaMemcpyDeviceToHost));
    if (n_colours) *n_colours = p->lev[level].col1.n_colours;
  });
}

extern "C" bmg_status bmg_get_colouring2(bmg_problem* p, int level, int* colour, int* n_colours) {
  return guarded([&] {
    check_levels(p, level, level);
    colour_level2(p->meshOf(level), p->lev[level], p->stream);
    const Colouring& c = p->lev[level].col2;
    if (colour) BMG_CUDA(cudaMemcpy(colour, c.colour.get(), sizeof(int) * p->meshOf(level).n, cudaMemcpyDeviceToHost));
    if (n_colours) *n_colours = c.n_colours;
  });
}

namespace bmg {
// Distance-2 colourings of every level and the row norms of every operator set (and
// of their float32 copies), for the Kaczmarz smoother; built once.
void ensure_kaczmarz(bmg_problem* p, bool fp32) {
  cudaStream_t s = p->stream;
  for (int l = 1; l <= p->L; ++l) colour_level2(p->meshOf(l), p->lev[l], s);
  for (int f = 2; f <= p->L; ++f)
    for (int j = 1; j <= f; ++j) {
      OpSet& o = p->ops[f][j];
      const Mesh& mj = p->meshOf(j);
      if (!o.na.get()) {
        o.na.alloc(mj.n); o.nam.alloc(mj.n); o.nm.alloc(mj.n);
        row_norms<double>(mj, p->opA(f, j), p->opM(f, j), o.na.get(), o.nam.get(), o.nm.get(), s);
      }
      if (fp32 && !p->ops32.empty()) {
        OpSet32& q = p->ops32[f][j];
        if (!q.na.get()) {
          q.na.alloc(mj.n); q.nam.alloc(mj.n); q.nm.alloc(mj.n);
          row_norms<float>(mj, q.a.get(), q.m.get(), q.na.get(), q.nam.get(), q.nm.get(), s);
        }
      }
    }
  BMG_CUDA(cudaStreamSynchronize(s));
}
}  // namespace bmg

// ------------------------------------------------------------- step entries ---
static const double* opDA_or_compute(const bmg_problem* p, int f, int j) {
  if (f >= 2) return p->opDA(f, j);
  return nullptr;
}

extern "C" bmg_status bmg_spmm(const bmg_problem* p, int f, int level, const double* X, int k, int ld,
                               double* AX, double* MX, void* stream) {
  return guarded([&] {
    check_levels(p, f, level);
    if (!X || !AX || !MX || k < 1 || ld < k || (ld & 1)) fail(BMG_ERR_INVALID_ARG, "bad block arguments");
    spmm_am(p->meshOf(level), p->opA(f, level), p->opM(f, level), X, ld, AX, MX, (cudaStream_t)stream);
  });
}

extern "C" bmg_status bmg_smooth(const bmg_problem* p, int f, int level, double* X, const double* B,
                                 const double* sft, int k, int ld, int smoother, int nu, double omega,
                                 double* work, void* stream) {
  return guarded([&] {
    check_levels(p, f, level);
    if (f < 2) fail(BMG_ERR_INVALID_ARG, "f must be >= 2");
    if (!X || !sft || k < 1 || ld < k || (ld & 1) || nu < 0) fail(BMG_ERR_INVALID_ARG, "bad block arguments");
    cudaStream_t s = (cudaStream_t)stream;
    const Mesh& m = p->meshOf(level);
    const double *a = p->opA(f, level), *mm = p->opM(f, level);
    const double *da = p->opDA(f, level), *dm = p->opDM(f, level);
    (void)opDA_or_compute;
    if (smoother == BMG_SMOOTH_JACOBI) {
      if (!work) fail(BMG_ERR_INVALID_ARG, "Jacobi needs a work block");
      for (int it = 0; it < nu; ++it) {
        jacobi_sweep(m, a, mm, da, dm, X, work, B, sft, ld, omega, s);
        BMG_CUDA(cudaMemcpyAsync(X, work, sizeof(double) * (size_t)m.n * ld, cudaMemcpyDeviceToDevice, s));
      }
    } else if (smoother == BMG_SMOOTH_MCGS || smoother == BMG_SMOOTH_MCSGS) {
      const Level& lv = p->lev[level];
      for (int it = 0; it < nu; ++it) {
        for (int c = 0; c < lv.col1.n_colours; ++c) gs_colour_sweep(m, lv, c, a, mm, da, dm, X, B, sft, ld, s);
        if (smoother == BMG_SMOOTH_MCSGS)
          for (int c = lv.col1.n_colours - 1; c >= 0; --c) gs_colour_sweep(m, lv, c, a, mm, da, dm, X, B, sft, ld, s);
      }
    } else if (smoother == BMG_SMOOTH_KACZMARZ) {
      bmg_problem* pm = const_cast<bmg_problem*>(p);
      ensure_kaczmarz(pm, false);
      const Level& lv = p->lev[level];
      const OpSet& o = p->ops[f][level];
      for (int it = 0; it < nu; ++it)
        for (int c = 0; c < lv.col2.n_colours; ++c)
          kaczmarz_colour_sweep<double>(m, lv, c, a, mm, o.na.get(), o.nam.get(), o.nm.get(), X, B, sft, ld, omega, s);
    } else {
      fail(BMG_ERR_INVALID_ARG, "unknown smoother");
    }
  });
}

extern "C" bmg_status bmg_prolong(const bmg_problem* p, int level, const double* Xc, double* Y, int k, int ld,
                                  int add, void* stream) {
  return guarded([&] {
    check_levels(p, level, level);
    if (level < 2) fail(BMG_ERR_INVALID_ARG, "level must be >= 2");
    if (!Xc || !Y || k < 1 || ld < k || (ld & 1)) fail(BMG_ERR_INVALID_ARG, "bad block arguments");
    prolong(p->meshOf(level), Xc, Y, ld, add != 0, (cudaStream_t)stream);
  });
}

extern "C" bmg_status bmg_restrict(const bmg_problem* p, int level, const double* R, double* Zc, int k, int ld,
                                   void* stream) {
  return guarded([&] {
    check_levels(p, level, level);
    if (level < 2) fail(BMG_ERR_INVALID_ARG, "level must be >= 2");
    if (!R || !Zc || k < 1 || ld < k || (ld & 1)) fail(BMG_ERR_INVALID_ARG, "bad block arguments");
    restrict_(p->meshOf(level - 1), R, Zc, ld, (cudaStream_t)stream);
  });
}

extern "C" bmg_status bmg_gram(const double* X, const double* Y, int n, int k, int ld, double* G, void* stream) {
  return guarded([&] {
    if (!X || !Y || !G || n < 1 || k < 1 || k > 160 || ld < k || ld > kGramMaxLd)
      fail(BMG_ERR_INVALID_ARG, "bad gram arguments (1 <= k <= 160, k <= ld <= 800)");
    const int parts = gram_parts(n);
    DBuf<double> partial((size_t)parts * k * k);
    gram(X, Y, n, k, ld, G, partial.get(), parts, (cudaStream_t)stream);
    BMG_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  });
}

// Reads a device error flag raised by a tensor-core kernel after the stream is idle.
static void check_tc_flag(const int* flag, cudaStream_t s) {
  int h = 0;
  BMG_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  BMG_CUDA(cudaStreamSynchronize(s));
  if (h) fail(BMG_ERR_TIMEOUT, "a bounded wait in a tensor-core kernel expired");
}

template <typename T>
static void gram_tc_entry(const T* X, const T* Y, int n, int k, int ld, double* G, void* stream) {
  if (!X || !Y || !G || n < 1 || k < 1 || k > kTcMaxK || ld < k)
    fail(BMG_ERR_INVALID_ARG, "bad gram arguments (1 <= k <= 128, ld >= k)");
  cudaStream_t s = (cudaStream_t)stream;
  const int parts = gram_tc_parts(n, k);
  DBuf<double> partial((size_t)parts * k * k);
  DBuf<int> flag(1);
  BMG_CUDA(cudaMemsetAsync(flag.get(), 0, sizeof(int), s));
  gram_tc(X, Y, n, k, ld, G, partial.get(), parts, flag.get(), s, false);
  check_tc_flag(flag.get(), s);
}

extern "C" bmg_status bmg_gram_tc(const double* X, const double* Y, int n, int k, int ld, double* G, void* stream) {
  return guarded([&] { gram_tc_entry(X, Y, n, k, ld, G, stream); });
}

extern "C" bmg_status bmg_gram_tc_f32(const float* X, const float* Y, int n, int k, int ld, double* G,
                                      void* stream) {
  return guarded([&] {
    if (ld & 3) fail(BMG_ERR_INVALID_ARG, "bad gram arguments (ld % 4 == 0)");
    gram_tc_entry(X, Y, n, k, ld, G, stream);
  });
}

// Test of the tensor-core kernels' bounded waits: a Gram whose waits are made to
// expire (gram_tc_timeout_selftest).  Returns what a product call returns after such
// an expiry, BMG_ERR_TIMEOUT, once the kernel has returned; the context stays usable.
extern "C" bmg_status bmg_tc_timeout_selftest(void* stream) {
  return guarded([&] {
    cudaStream_t s = (cudaStream_t)stream;
    DBuf<double> X((size_t)4096 * 64), G((size_t)64 * 64), partial((size_t)gram_tc_parts(4096, 64) * 64 * 64);
    DBuf<int> flag(1);
    BMG_CUDA(cudaMemsetAsync(X.get(), 0, sizeof(double) * 4096 * 64, s));
    BMG_CUDA(cudaMemsetAsync(flag.get(), 0, sizeof(int), s));
    gram_tc_timeout_selftest(X.get(), G.get(), partial.get(), flag.get(), s);
    check_tc_flag(flag.get(), s);
    fail(BMG_ERR_CUDA, "tc timeout self-test: the bounded waits did not expire");
  });
}

template <typename T>
static void expand_entry(const T* Z, const T* X, const double* Yx, int n, int k, int ld, int ldy, T* U,
                         int tensor_cores, void* stream) {
  const int align = sizeof(T) == 8 ? 2 : 4;
  if (!X || !Yx || !U || n < 1 || k < 1 || ld < k || ld % align || ldy < k)
    fail(BMG_ERR_INVALID_ARG, "bad expand arguments");
  if (k > 160) fail(BMG_ERR_INVALID_ARG, "expand: k <= 160");
  cudaStream_t s = (cudaStream_t)stream;
  if (tensor_cores) {
    if (k > kTcMaxK) fail(BMG_ERR_INVALID_ARG, "tensor-core expand: k <= 128");
    DBuf<unsigned char> scratch(expand_tc_scratch_bytes(k));
    DBuf<int> flag(1);
    BMG_CUDA(cudaMemsetAsync(flag.get(), 0, sizeof(int), s));
    expand_tc(Z, X, Yx, n, k, ld, ldy, U, scratch.get(), flag.get(), s);
    check_tc_flag(flag.get(), s);
  } else {
    expand<T>(Z, X, Yx, n, k, ld, ldy, U, s);
    BMG_CUDA(cudaStreamSynchronize(s));
  }
}

extern "C" bmg_status bmg_expand(const double* Z, const double* X, const double* Yx, int n, int k, int ld, int ldy,
                                 double* U, int tensor_cores, void* stream) {
  return guarded([&] { expand_entry(Z, X, Yx, n, k, ld, ldy, U, tensor_cores, stream); });
}

extern "C" bmg_status bmg_expand_f32(const float* Z, const float* X, const double* Yx, int n, int k, int ld,
                                     int ldy, float* U, int tensor_cores, void* stream) {
  return guarded([&] { expand_entry(Z, X, Yx, n, k, ld, ldy, U, tensor_cores, stream); });
}

extern "C" bmg_status bmg_dense_eig(const double* Ahat, const double* Mhat, int n, double sigma, int k,
                                    double* theta, double* Y, int* rank_out, void* stream) {
  return guarded([&] {
    if (!Ahat || !Mhat || !theta || !Y) fail(BMG_ERR_INVALID_ARG, "null pointer");
    if (n < 1 || n > 224 || k < 1 || k > n) fail(BMG_ERR_INVALID_ARG, "need 1 <= k <= n <= 224");
    DBuf<double> work(dense_work_doubles(n));
    DBuf<int> rk(1);
    dense_eig(Ahat, Mhat, n, sigma, k, theta, Y, rank_out ? rank_out : rk.get(), work.get(), nullptr,
              kDropFP64, 0, (cudaStream_t)stream);
    BMG_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  });
}

// ------------------------------------------------------------------- solve ----
namespace bmg {
namespace {

// Operators of finest level f on level j in the block arithmetic T.
template <typename T> struct Ops;
template <> struct Ops<double> {
  static const double* NA(const bmg_problem* p, int f, int j) { return p->ops[f][j].na.get(); }
  static const double* NAM(const bmg_problem* p, int f, int j) { return p->ops[f][j].nam.get(); }
  static const double* NM(const bmg_problem* p, int f, int j) { return p->ops[f][j].nm.get(); }
  static const double* A(const bmg_problem* p, int f, int j) { return p->opA(f, j); }
  static const double* M(const bmg_problem* p, int f, int j) { return p->opM(f, j); }
  static const double* DA(const bmg_problem* p, int f, int j) { return p->opDA(f, j); }
  static const double* DM(const bmg_problem* p, int f, int j) { return p->opDM(f, j); }
};
template <> struct Ops<float> {
  static const float* NA(const bmg_problem* p, int f, int j) { return p->ops32[f][j].na.get(); }
  static const float* NAM(const bmg_problem* p, int f, int j) { return p->ops32[f][j].nam.get(); }
  static const float* NM(const bmg_problem* p, int f, int j) { return p->ops32[f][j].nm.get(); }
  static const float* A(const bmg_problem* p, int f, int j) { return p->ops32[f][j].a.get(); }
  static const float* M(const bmg_problem* p, int f, int j) { return p->ops32[f][j].m.get(); }
  static const float* DA(const bmg_problem* p, int f, int j) { return p->ops32[f][j].da.get(); }
  static const float* DM(const bmg_problem* p, int f, int j) { return p->ops32[f][j].dm.get(); }
};

__global__ void to_float_kernel(const double* __restrict__ in, size_t n, float* __restrict__ out) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = (float)in[t];
}

// Block copy between leading dimensions and arithmetic types (columns [0, cols)).
template <typename S, typename D>
__global__ void convert_block_kernel(const S* __restrict__ in, int ldi, D* __restrict__ out, int ldo,
                                     int rows, int cols) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)rows * cols) return;
  const size_t r = t / cols, c = t % cols;
  out[r * ldo + c] = (D)in[r * ldi + c];
}

// float32 copies of every operator set (precision form), built once per problem.
void ensure_ops32(bmg_problem* p) {
  if (!p->ops32.empty()) return;
  cudaStream_t s = p->stream;
  const int L = p->L;
  std::vector<std::vector<OpSet32>> ops(L + 1);
  auto conv = [&](const double* src, size_t n, DBuf<float>& dst) {
    dst.alloc(n);
    to_float_kernel<<<grid_of(n, 256), 256, 0, s>>>(src, n, dst.get());
    check_launch("to_float_kernel");
  };
  for (int f = 2; f <= L; ++f) {
    ops[f].resize(f + 1);
    for (int j = 1; j <= f; ++j) {
      const Mesh& mj = p->meshOf(j);
      conv(p->opA(f, j), mj.nnz, ops[f][j].a);
      conv(p->opM(f, j), mj.nnz, ops[f][j].m);
      conv(p->opDA(f, j), mj.n, ops[f][j].da);
      conv(p->opDM(f, j), mj.n, ops[f][j].dm);
    }
  }
  BMG_CUDA(cudaStreamSynchronize(s));
  p->ops32 = std::move(ops);
}

// Device views of the blocks of one arithmetic.
template <typename T>
struct Blocks {
  int ld = 0;
  T *X = nullptr, *AX = nullptr, *MX = nullptr, *U = nullptr, *AU = nullptr, *MU = nullptr;
  T *B = nullptr, *W = nullptr, *Zf = nullptr, *shift = nullptr;
  std::vector<T*> cA, cB, cC, cD;
};

Blocks<double> blocks64(SolveWork& w) {
  Blocks<double> b;
  b.ld = w.ld;
  b.X = w.X.get(); b.AX = w.AX.get(); b.MX = w.MX.get(); b.U = w.U.get(); b.AU = w.AU.get();
  b.MU = w.MU.get(); b.B = w.B.get(); b.W = w.W.get(); b.Zf = w.Zf.get(); b.shift = w.shift.get();
  for (auto* v : {&w.cA, &w.cB, &w.cC, &w.cD}) {
    std::vector<double*>& dst = (v == &w.cA) ? b.cA : (v == &w.cB) ? b.cB : (v == &w.cC) ? b.cC : b.cD;
    for (auto& d : *v) dst.push_back(d.get());
  }
  return b;
}

Blocks<float> blocks32(bmg_problem* p, SolveWork& w) {
  cudaStream_t s = w.s;
  if (!w.ld32) {
    w.ld32 = (w.k + 3) & ~3;
    const size_t big = (size_t)p->meshOf(w.L).n * w.ld32;
    for (DBuf<float>* b : {&w.X32, &w.AX32, &w.MX32, &w.U32, &w.AU32, &w.MU32, &w.B32, &w.W32, &w.Zf32}) {
      b->alloc(big);
      BMG_CUDA(cudaMemsetAsync(b->get(), 0, sizeof(float) * big, s));
    }
    w.shift32.alloc(w.ld32);
    BMG_CUDA(cudaMemsetAsync(w.shift32.get(), 0, sizeof(float) * w.ld32, s));
    w.cA32.resize(w.L); w.cB32.resize(w.L); w.cC32.resize(w.L); w.cD32.resize(w.L);
    for (int j = 1; j < w.L; ++j) {
      const size_t sz = (size_t)p->meshOf(j).n * w.ld32;
      for (auto* v : {&w.cA32, &w.cB32, &w.cC32, &w.cD32}) {
        (*v)[j].alloc(sz);
        BMG_CUDA(cudaMemsetAsync((*v)[j].get(), 0, sizeof(float) * sz, s));
      }
    }
  }
  Blocks<float> b;
  b.ld = w.ld32;
  b.X = w.X32.get(); b.AX = w.AX32.get(); b.MX = w.MX32.get(); b.U = w.U32.get(); b.AU = w.AU32.get();
  b.MU = w.MU32.get(); b.B = w.B32.get(); b.W = w.W32.get(); b.Zf = w.Zf32.get(); b.shift = w.shift32.get();
  for (auto* v : {&w.cA32, &w.cB32, &w.cC32, &w.cD32}) {
    std::vector<float*>& dst = (v == &w.cA32) ? b.cA : (v == &w.cB32) ? b.cB : (v == &w.cC32) ? b.cC : b.cD;
    for (auto& d : *v) dst.push_back(d.get());
  }
  return b;
}

template <typename S, typename D>
void convert_block(const S* in, int ldi, D* out, int ldo, int rows, int cols, cudaStream_t s) {
  const size_t total = (size_t)rows * cols;
  convert_block_kernel<S, D><<<grid_of(total, 256), 256, 0, s>>>(in, ldi, out, ldo, rows, cols);
  check_launch("convert_block_kernel");
}

// Ahat = [[AQ, CA], [CA^T, GA]] (n = n1 + k), CA read from a [n1][ld] block.
template <typename T>
__global__ void assemble_hat_kernel(const double* AQ, const T* CA, const double* GA, int n1, int k,
                                    int ld, double* H) {
  const int n = n1 + k;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n * n) return;
  const int i = q / n, j = q % n;
  double v;
  if (i < n1 && j < n1) v = AQ[i * n1 + j];
  else if (i < n1) v = (double)CA[(size_t)i * ld + (j - n1)];
  else if (j < n1) v = (double)CA[(size_t)j * ld + (i - n1)];
  else v = GA[(i - n1) * k + (j - n1)];
  H[q] = v;
}

// Coarse coefficients Y[0:n1][0:k] into a [n1][ld] block (zero padding).
template <typename T>
__global__ void pack_coarse_kernel(const double* Y, int n1, int k, int ld, T* Z) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n1 * ld) return;
  const int i = q / ld, c = q % ld;
  Z[q] = (c < k) ? (T)Y[i * k + c] : T(0);
}

// lam = theta + sigma (k values); the per-column smoothing shift in the block
// arithmetic (form), zero in the padding.
template <typename T>
__global__ void shifts_kernel(const double* theta, int k, int ld, double sigma, int form, double* lam,
                              T* shift) {
  const int c = threadIdx.x + blockIdx.x * blockDim.x;
  if (c >= ld) return;
  if (c < k) {
    lam[c] = theta[c] + sigma;
    shift[c] = (T)((form == BMG_FORM_SHIFTED) ? sigma : theta[c] + sigma);
  } else {
    shift[c] = T(0);
  }
}

// nu sweeps of the configured smoother on level j (operators of finest level f),
// from Xin into Xout (Xin may equal Xout).  Jacobi alternates between Xout and work
// so that the last sweep lands in Xout; Gauss-Seidel runs in place on Xout.
// zero_shift: every shift is zero (shifted form at sigma = 0), so M is not read.
template <typename T>
void smooth_level(const bmg_problem* p, int f, int j, const bmg_options& o, const T* Xin, T* Xout,
                  const T* B, const T* shift, int ld, T* work, cudaStream_t s, bool zero_shift) {
  const Mesh& m = p->meshOf(j);
  const T *a = Ops<T>::A(p, f, j), *mm = Ops<T>::M(p, f, j), *da = Ops<T>::DA(p, f, j), *dm = Ops<T>::DM(p, f, j);
  const size_t bytes = sizeof(T) * (size_t)m.n * ld;
  if (o.smoother == BMG_SMOOTH_JACOBI) {
    const T* src = Xin;
    if (Xin == Xout && (o.nu % 2 == 1)) {
      BMG_CUDA(cudaMemcpyAsync(work, Xin, bytes, cudaMemcpyDeviceToDevice, s));
      src = work;
      for (int it = 0; it < o.nu; ++it) {
        T* dst = (it % 2 == 0) ? Xout : work;
        jacobi_sweep<T>(m, a, mm, da, dm, src, dst, B, shift, ld, o.omega, s, zero_shift);
        src = dst;
      }
      return;
    }
    for (int it = 0; it < o.nu; ++it) {
      T* dst = ((o.nu - 1 - it) % 2 == 0) ? Xout : work;
      jacobi_sweep<T>(m, a, mm, da, dm, src, dst, B, shift, ld, o.omega, s, zero_shift);
      src = dst;
    }
    return;
  }
  if (Xin != Xout) BMG_CUDA(cudaMemcpyAsync(Xout, Xin, bytes, cudaMemcpyDeviceToDevice, s));
  const Level& lv = p->lev[j];
  if (o.smoother == BMG_SMOOTH_KACZMARZ) {
    for (int it = 0; it < o.nu; ++it)
      for (int c = 0; c < lv.col2.n_colours; ++c)
        kaczmarz_colour_sweep<T>(m, lv, c, a, mm, Ops<T>::NA(p, f, j), Ops<T>::NAM(p, f, j), Ops<T>::NM(p, f, j), Xout,
                                 B, shift, ld, o.omega, s);
    return;
  }
  for (int it = 0; it < o.nu; ++it) {
    for (int c = 0; c < lv.col1.n_colours; ++c)
      gs_colour_sweep<T>(m, lv, c, a, mm, da, dm, Xout, B, shift, ld, s, work, zero_shift);
    if (o.smoother == BMG_SMOOTH_MCSGS)
      for (int c = lv.col1.n_colours - 1; c >= 0; --c)
        gs_colour_sweep<T>(m, lv, c, a, mm, da, dm, Xout, B, shift, ld, s, work, zero_shift);
  }
}

// Allocates a solve workspace for block size k; its set-up work runs on stream s.
std::unique_ptr<SolveWork> make_work(bmg_problem* p, int k, cudaStream_t s) {
  const int L = p->L;
  const int n1 = p->meshOf(1).n, nL = p->meshOf(L).n;
  std::unique_ptr<SolveWork> wp(new SolveWork());
  SolveWork& w = *wp;
  w.s = s;
  w.k = k;
  w.ld = (k + 1) & ~1;
  w.n1 = n1;
  w.nh = n1 + k;
  w.L = L;
  const int ld = w.ld;
  const size_t big = (size_t)nL * ld;
  for (DBuf<double>* b : {&w.X, &w.AX, &w.MX, &w.U, &w.AU, &w.MU, &w.B, &w.W, &w.Zf}) {
    b->alloc(big);
    BMG_CUDA(cudaMemsetAsync(b->get(), 0, sizeof(double) * big, s));
  }
  w.cA.resize(L); w.cB.resize(L); w.cC.resize(L); w.cD.resize(L);
  for (int j = 1; j < L; ++j) {
    const size_t sz = (size_t)p->meshOf(j).n * ld;
    for (auto* v : {&w.cA, &w.cB, &w.cC, &w.cD}) {
      (*v)[j].alloc(sz);
      BMG_CUDA(cudaMemsetAsync((*v)[j].get(), 0, sizeof(double) * sz, s));
    }
  }
  w.Ahat.alloc((size_t)w.nh * w.nh);
  w.Mhat.alloc((size_t)w.nh * w.nh);
  w.Y.alloc((size_t)w.nh * k);
  w.theta.alloc(k);
  w.lam.alloc((k + 3) & ~3);
  w.shift.alloc(ld);
  w.GA.alloc((size_t)k * k);
  w.GM.alloc((size_t)k * k);
  w.dense.alloc(dense_work_doubles(w.nh));
  BMG_CUDA(cudaMemsetAsync(w.dense.get(), 0, sizeof(double) * dense_work_doubles(w.nh), s));
  w.parts = std::max(gram_parts(nL), gram_tc_parts(nL, std::min(k, kTcMaxK)));
  w.partial.alloc((size_t)w.parts * std::max(k * k, 2 * k));
  if (k <= kTcMaxK) {
    w.tcscratch.alloc(expand_tc_scratch_bytes(k));
    w.tcerr.alloc(1);
    BMG_CUDA(cudaMemsetAsync(w.tcerr.get(), 0, sizeof(int), s));
  }
  w.res.alloc(2 * k);
  w.rank.alloc(1);
  w.dquality.alloc(1);
  BMG_CUDA(cudaMallocHost(&w.hbuf, sizeof(double) * (5 * (size_t)k + 8)));  // res, lam, quality, rank, Gram diagonals
  w.AQ.resize(L + 1);
  w.MQ.resize(L + 1);
  const Mesh& m1 = p->meshOf(1);
  for (int f = 2; f <= L; ++f) {
    w.AQ[f].alloc((size_t)n1 * n1);
    w.MQ[f].alloc((size_t)n1 * n1);
    csr_to_dense_kernel<<<grid_of(n1, 64), 64, 0, s>>>(m1.row_ptr.get(), m1.col.get(), p->opA(f, 1), n1, w.AQ[f].get());
    csr_to_dense_kernel<<<grid_of(n1, 64), 64, 0, s>>>(m1.row_ptr.get(), m1.col.get(), p->opM(f, 1), n1, w.MQ[f].get());
    check_launch("csr_to_dense_kernel");
  }
  // max over rows of dM/dA per (f, j): admissible depth of the down-leg
  w.ratio.assign(L + 1, std::vector<double>(L + 1, 0.0));
  DBuf<unsigned long long> um(1);
  for (int f = 2; f <= L; ++f)
    for (int j = 1; j < f; ++j) {
      BMG_CUDA(cudaMemsetAsync(um.get(), 0, sizeof(unsigned long long), s));
      ratio_max_kernel<<<grid_of(p->meshOf(j).n, 256), 256, 0, s>>>(p->opDA(f, j), p->opDM(f, j), p->meshOf(j).n, um.get());
      check_launch("ratio_max_kernel");
      unsigned long long h = 0;
      BMG_CUDA(cudaMemcpyAsync(&h, um.get(), sizeof(h), cudaMemcpyDeviceToHost, s));
      BMG_CUDA(cudaStreamSynchronize(s));
      std::memcpy(&w.ratio[f][j], &h, sizeof(double));
    }
  return wp;
}

// Workspace slot `slot` of problem p for block size k (slot 0 is the one of
// bmg_solve), kept between calls; its solves run on stream s.
SolveWork& workspace(bmg_problem* p, int k, int slot, cudaStream_t s) {
  std::unique_ptr<SolveWork>* wp = &p->ws;
  if (slot > 0) {
    if ((int)p->ws_more.size() < slot) p->ws_more.resize(slot);
    wp = &p->ws_more[slot - 1];
  }
  if (!*wp || (*wp)->k != k) {
    wp->reset();
    *wp = make_work(p, k, s);
  }
  (*wp)->s = s;
  return **wp;
}

// Outcome of one cycle: Ritz values, residuals and convergence of the wanted pairs.
struct CycleState {
  std::vector<double> rho, lamv;
  double max_dense_err = 0.0;
};

// Runs `body` (a sequence of asynchronous launches on w.s) either directly or as a
// CUDA graph: the first time a key is met the body runs eagerly (the row-kernel
// autotuner times its candidates then); the second time it is captured, instantiated
// and replayed from then on.  Graphs are off while the kernel profiler runs (its
// events must be recorded per launch) and with bmg_options.graphs = 0.
template <typename F>
void run_graph(bmg_problem* p, SolveWork& w, const std::tuple<int, int, int, int>& key, F&& body) {
  (void)p;
  if (!w.use_graphs || prof_enabled() || w.s != w.own) {
    body();
    return;
  }
  auto it = w.graphs.find(key);
  if (it == w.graphs.end()) {
    if (!w.seen.count(key)) {
      w.seen.insert(key);
      body();
      return;
    }
    cudaGraph_t g = nullptr;
    const long long before = launch_count();
    BMG_CUDA(cudaStreamBeginCapture(w.s, cudaStreamCaptureModeRelaxed));
    try {
      body();
    } catch (...) {
      cudaStreamEndCapture(w.s, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    BMG_CUDA(cudaStreamEndCapture(w.s, &g));
    count_launches(before - launch_count());   // captured launches did not run
    // kernel nodes, for the launch counter
    size_t nn = 0;
    int kernels = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
    for (size_t q = 0; q < nn; ++q) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nodes[q], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
    }
    cudaGraphExec_t ge = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    check_cuda(e, "cudaGraphInstantiate");
    it = w.graphs.emplace(key, std::make_pair(ge, kernels)).first;
  }
  BMG_CUDA(cudaGraphLaunch(it->second.first, w.s));
  count_launches(it->second.second);
}

// One BMG cycle on level f with blocks of arithmetic T (steps 1-5 of the file
// header).  Smoothing (step 5) runs unless the wanted pairs met ftol or `last` is
// set.  Returns whether every wanted pair met ftol.
// With bmg_options.adaptive_shift, every cycle of a solve but its first replaces
// sigma (in/out) by the mean Rayleigh quotient of the columns of X, read from the
// diagonals of this cycle's Grams before its eigensolve (Alg. 3 step 4; Sec. 5.3).
template <typename T>
bool run_cycle(bmg_problem* p, SolveWork& w, Blocks<T>& b, int f, const bmg_options& o, double& sigma, int k,
               int n_wanted, double ftol, bool last, bool first, CycleState& cs) {
  cudaStream_t s = w.s;
  const int ld = b.ld, n1 = w.n1, nh = w.nh;
  const Mesh& mf = p->meshOf(f);
  const int nf = mf.n;
  const T *Af = Ops<T>::A(p, f, f), *Mf = Ops<T>::M(p, f, f);
  double* hres = w.hbuf;            // 2k residual sums
  double* hlam = w.hbuf + 2 * k;    // k Ritz values
  double* hqual = w.hbuf + 3 * k;   // error estimate of the enriched eigensolve
  int* hint = reinterpret_cast<int*>(w.hbuf + 3 * k + 1);  // rank
  int* htc = reinterpret_cast<int*>(w.hbuf + 3 * k + 2);   // tensor-core wait expired
  const bool tc = o.tensor_cores && k <= kTcMaxK;
  // 1-4: products, Grams and couplings, enriched eigensolve, Ritz vectors, residuals
  auto part_a1 = [&]() {
    // 1-2: products, Grams, couplings Q^T AX, Q^T MX by the restriction chain
    spmm_am<T>(mf, Af, Mf, b.X, ld, b.AX, b.MX, s);
    if (tc) {
      gram_tc(b.X, b.AX, nf, k, ld, w.GA.get(), w.partial.get(), gram_tc_parts(nf, k), w.tcerr.get(), s, true);
      gram_tc(b.X, b.MX, nf, k, ld, w.GM.get(), w.partial.get(), gram_tc_parts(nf, k), w.tcerr.get(), s, true);
    } else {
      gram(b.X, b.AX, nf, k, ld, w.GA.get(), w.partial.get(), gram_parts(nf), s, true);
      gram(b.X, b.MX, nf, k, ld, w.GM.get(), w.partial.get(), gram_parts(nf), s, true);
    }
    const T* ca = b.AX;
    const T* cm = b.MX;
    for (int j = f; j >= 2; --j) {
      restrict2_<T>(p->meshOf(j - 1), ca, b.cA[j - 1], cm, b.cB[j - 1], ld, s);
      ca = b.cA[j - 1];
      cm = b.cB[j - 1];
    }
  };
  auto part_a2 = [&]() {
    const T* ca = b.cA[1];
    const T* cm = b.cB[1];
    prof_begin(KC_SMALL, s);
    assemble_hat_kernel<T><<<grid_of((size_t)nh * nh, 256), 256, 0, s>>>(w.AQ[f].get(), ca, w.GA.get(), n1, k, ld, w.Ahat.get());
    check_launch("assemble_hat_kernel");
    assemble_hat_kernel<T><<<grid_of((size_t)nh * nh, 256), 256, 0, s>>>(w.MQ[f].get(), cm, w.GM.get(), n1, k, ld, w.Mhat.get());
    check_launch("assemble_hat_kernel");
    prof_end(KC_SMALL, s, 32.0 * nh * nh, 0.0);
    // 3: enriched eigensolve
    dense_eig(w.Ahat.get(), w.Mhat.get(), nh, sigma, k, w.theta.get(), w.Y.get(), w.rank.get(), w.dense.get(),
              w.dquality.get(), sizeof(T) == sizeof(float) ? kDropFP32 : kDropFP64, n1, s,
              o.selection ? o.index_first : -1);
    prof_begin(KC_SMALL, s);
    shifts_kernel<T><<<grid_of(ld, 128), 128, 0, s>>>(w.theta.get(), k, ld, sigma, o.form, w.lam.get(), b.shift);
    check_launch("shifts_kernel");
    // 4: Ritz vectors U = Q Y_c + X Y_x
    pack_coarse_kernel<T><<<grid_of((size_t)n1 * ld, 256), 256, 0, s>>>(w.Y.get(), n1, k, ld, b.cC[1]);
    check_launch("pack_coarse_kernel");
    prof_end(KC_SMALL, s, 8.0 * n1 * ld, 0.0);
    const T* z = b.cC[1];
    for (int j = 2; j < f; ++j) {
      prolong<T>(p->meshOf(j), z, b.cC[j], ld, false, s);
      z = b.cC[j];
    }
    prolong<T>(mf, z, b.Zf, ld, false, s);
    if (tc)
      expand_tc<T>(b.Zf, b.X, w.Y.get() + (size_t)n1 * k, nf, k, ld, k, b.U, w.tcscratch.get(), w.tcerr.get(), s);
    else
      expand<T>(b.Zf, b.X, w.Y.get() + (size_t)n1 * k, nf, k, ld, k, b.U, s);
    spmm_am<T>(mf, Af, Mf, b.U, ld, b.AU, b.MU, s);
    eig_residuals<T>(b.AU, b.MU, b.U, w.lam.get(), nf, k, ld, w.partial.get(), gram_parts(nf), w.res.get(), s);
    BMG_CUDA(cudaMemcpyAsync(hres, w.res.get(), sizeof(double) * 2 * k, cudaMemcpyDeviceToHost, s));
    BMG_CUDA(cudaMemcpyAsync(hlam, w.lam.get(), sizeof(double) * k, cudaMemcpyDeviceToHost, s));
    BMG_CUDA(cudaMemcpyAsync(hint, w.rank.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    BMG_CUDA(cudaMemcpyAsync(hqual, w.dquality.get(), sizeof(double), cudaMemcpyDeviceToHost, s));
    if (tc) BMG_CUDA(cudaMemcpyAsync(htc, w.tcerr.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
  };
  {
    TraceRange trace("cycle: products, Rayleigh-Ritz, Ritz vectors, residuals");
    if (o.adaptive_shift && !first) {
      // the shift from the Rayleigh quotients of X: diagonals of the Grams
      part_a1();
      double* hg = w.hbuf + 3 * k + 8;   // 2k values: diag(X^T A X), diag(X^T M X)
      BMG_CUDA(cudaMemcpy2DAsync(hg, sizeof(double), w.GA.get(), sizeof(double) * (k + 1), sizeof(double), k,
                                 cudaMemcpyDeviceToHost, s));
      BMG_CUDA(cudaMemcpy2DAsync(hg + k, sizeof(double), w.GM.get(), sizeof(double) * (k + 1), sizeof(double), k,
                                 cudaMemcpyDeviceToHost, s));
      BMG_CUDA(cudaStreamSynchronize(s));
      double mu = 0.0;
      for (int i = 0; i < k; ++i) mu += hg[i] / hg[k + i];
      mu /= k;
      if (!std::isfinite(mu)) fail(BMG_ERR_NONFINITE, "adaptive shift not finite");
      sigma = mu;
      part_a2();
    } else {
      run_graph(p, w, std::make_tuple(0, f, (int)sizeof(T), 0), [&]() {
        part_a1();
        part_a2();
      });
    }
  }
  BMG_CUDA(cudaStreamSynchronize(s));
  if (tc && *htc) fail(BMG_ERR_TIMEOUT, "a bounded wait in a tensor-core kernel expired");
  if (hint[0] < k) fail(BMG_ERR_SINGULAR, "enriched space rank " + std::to_string(hint[0]) + " < k");
  if (!(*hqual <= 1e-6))
    fail(BMG_ERR_NONFINITE, "enriched eigensolve refinement failed (error estimate " + std::to_string(*hqual) + ")");
  cs.max_dense_err = std::max(cs.max_dense_err, *hqual);
  bool conv = true, finite = true;
  for (int i = 0; i < k; ++i) {
    cs.lamv[i] = hlam[i];
    cs.rho[i] = std::sqrt(hres[i]) / (p->norm1[f] * std::sqrt(hres[k + i]));
    if (!std::isfinite(cs.rho[i]) || !std::isfinite(hlam[i])) finite = false;
    if (i < n_wanted && !(cs.rho[i] <= ftol)) conv = false;
  }
  if (!finite) fail(BMG_ERR_NONFINITE, "non-finite Ritz pair on level " + std::to_string(f));
  if (conv || last) return conv;
  double smax = (o.form == BMG_FORM_SHIFTED) ? sigma : -1e300;
  if (o.form != BMG_FORM_SHIFTED) for (int i = 0; i < k; ++i) smax = std::max(smax, cs.lamv[i]);
  std::vector<int> legs;
  for (int j = f - 1; j >= 1 && (int)legs.size() < o.vcycle_depth; --j) {
    if (!(smax * w.ratio[f][j] < 1.0 - 0.25)) break;
    legs.push_back(j);
  }
  // the shifted form at sigma = 0 smooths A x_i = theta_i M u_i: M not needed
  const bool zs = o.form == BMG_FORM_SHIFTED && sigma == 0.0;
  auto part_b = [&]() {
    // 5: smoothing of the source problems from U, then the down-leg
    const T* Bp = nullptr;
    if (o.form == BMG_FORM_SHIFTED) {
      prof_begin(KC_SMALL, s);
      scale_rhs<T>(b.MU, w.theta.get(), nf, k, ld, b.B, s);
      prof_end(KC_SMALL, s, 2.0 * sizeof(T) * nf * ld, 1.0 * nf * ld);
      Bp = b.B;
    }
    smooth_level<T>(p, f, f, o, b.U, b.X, Bp, b.shift, ld, b.W, s, zs);
    if (!legs.empty()) {
      residual<T>(mf, Af, Mf, b.X, Bp, b.shift, ld, b.W, s, zs);
      const T* rprev = b.W;
      for (size_t t = 0; t < legs.size(); ++t) {
        const int j = legs[t];
        const Mesh& mj = p->meshOf(j);
        restrict_<T>(mj, rprev, b.cA[j], ld, s);
        BMG_CUDA(cudaMemsetAsync(b.cB[j], 0, sizeof(T) * (size_t)mj.n * ld, s));
        smooth_level<T>(p, f, j, o, b.cB[j], b.cB[j], b.cA[j], b.shift, ld, b.cD[j], s, zs);
        if (t + 1 < legs.size()) {
          residual<T>(mj, Ops<T>::A(p, f, j), Ops<T>::M(p, f, j), b.cB[j], b.cA[j], b.shift, ld, b.cC[j], s, zs);
          rprev = b.cC[j];
        }
      }
      for (size_t t = legs.size() - 1; t >= 1; --t) {
        const int j = legs[t];  // coarser; add into level j+1
        prolong<T>(p->meshOf(j + 1), b.cB[j], b.cB[j + 1], ld, true, s);
      }
      prolong<T>(mf, b.cB[f - 1], b.X, ld, true, s);
    }
  };
  {
    TraceRange trace("cycle: smoothing and down-leg");
    run_graph(p, w, std::make_tuple(1, f, (int)sizeof(T), (int)legs.size()), part_b);
  }
  return false;
}
// Argument checks shared by bmg_solve and bmg_solve_batched.
bmg_options checked_options(const bmg_problem* p, int k, int n_wanted, double sigma, double tol,
                            const bmg_options* opt_in, const double* X0, const double* evals) {
  if (!p) fail(BMG_ERR_INVALID_ARG, "null problem");
  if (!p->L) fail(BMG_ERR_STATE, "bmg_hierarchy not called");
  bmg_options o;
  bmg_default_options(&o);
  if (opt_in) o = *opt_in;
  const int n1 = p->meshOf(1).n, n2 = p->meshOf(2).n;
  if (k < 1 || k > 160 || n_wanted < 1 || n_wanted > k || k > n2 || n1 + k > 224)
    fail(BMG_ERR_INVALID_ARG, "need 1 <= n_wanted <= k <= min(N_2, 160) and N_1 + k <= 224");
  if ((!X0 && o.resume != 1 && o.coarse_start != 1) || !evals)
    fail(BMG_ERR_INVALID_ARG, "X0 (unless resuming or starting from the coarse eigenvectors) and evals are required");
  if (o.coarse_start == 1 && k > n1) fail(BMG_ERR_INVALID_ARG, "coarse_start needs k <= N_1");
  if (!(tol > 0.0) || !std::isfinite(sigma)) fail(BMG_ERR_INVALID_ARG, "bad tol or sigma");
  if (o.nu < 1 || o.nu > 64 || o.smoother < 0 || o.smoother > 3 || o.form < 0 || o.form > 1 ||
      o.max_cycles < 1 || o.cycles_intermediate < 1 || !(o.omega > 0.0) || o.precision < 0 ||
      o.precision > 1 || !(o.switch_tol > 0.0) || o.stop_after_cycles < 0 || o.resume < 0 || o.resume > 1 ||
      o.tensor_cores < 0 || o.tensor_cores > 1 || o.autotune < 0 || o.autotune > 1 || o.graphs < 0 || o.graphs > 1 ||
      o.adaptive_shift < 0 || o.adaptive_shift > 1 || o.selection < 0 || o.selection > 1 || o.index_first < 0 ||
      o.coarse_start < 0 || o.coarse_start > 1)
    fail(BMG_ERR_INVALID_ARG, "bad options");
  return o;
}

// --- Checkpoint: the solver state between two cycles of the BFMG loop, as bytes:
// StateHead, then hist[n_hist], hist_level[n_info], hist_fp32[n_info] (int32),
// hist_resid[n_info], lamv[k], rho[k], X[n_f][k] (the iterate; float32 values of the
// precision form are exact in float64).
struct StateHead {
  uint32_t magic, version;
  int32_t k, L, n_wanted, level, cycle, fp32, total_cycles, fp32_cycles, n_f, n_hist, n_info, pad;
  int32_t cyc[33];
  double sigma, tol, max_dense_err;
  int32_t smoother, nu, form, vcycle_depth, cycles_intermediate, max_cycles, precision, tensor_cores;
  double omega, tol_intermediate, switch_tol;
  int32_t adaptive_shift, pad3;
  double mu;                       // shift of the next cycle (adaptive_shift)
  int32_t selection, index_first, coarse_start, pad4;
};
constexpr uint32_t kStateMagic = 0x53474d42u;   // "BMGS"
constexpr uint32_t kStateVersion = 3;
size_t state_bytes(const StateHead& h) {
  return sizeof(StateHead) + sizeof(double) * ((size_t)h.n_hist + h.n_info + 2 * (size_t)h.k + (size_t)h.n_f * h.k) +
         sizeof(int32_t) * 2 * (size_t)h.n_info;
}
void head_options(StateHead& h, const bmg_options& o) {
  h.smoother = o.smoother; h.nu = o.nu; h.form = o.form; h.vcycle_depth = o.vcycle_depth;
  h.cycles_intermediate = o.cycles_intermediate; h.max_cycles = o.max_cycles; h.precision = o.precision;
  h.tensor_cores = o.tensor_cores;
  h.adaptive_shift = o.adaptive_shift;
  h.selection = o.selection;
  h.index_first = o.index_first;
  h.coarse_start = o.coarse_start;
  h.omega = o.omega; h.tol_intermediate = o.tol_intermediate; h.switch_tol = o.switch_tol;
}
bool same_options(const StateHead& h, const bmg_options& o) {
  StateHead g = h;
  head_options(g, o);
  return g.smoother == h.smoother && g.nu == h.nu && g.form == h.form && g.vcycle_depth == h.vcycle_depth &&
         g.cycles_intermediate == h.cycles_intermediate && g.max_cycles == h.max_cycles &&
         g.precision == h.precision && g.tensor_cores == h.tensor_cores && g.adaptive_shift == h.adaptive_shift &&
         g.selection == h.selection && g.index_first == h.index_first && g.coarse_start == h.coarse_start &&
         g.omega == h.omega && g.tol_intermediate == h.tol_intermediate &&
         g.switch_tol == h.switch_tol;
}
// Checks a state's structure against the problem; returns its header.
StateHead parse_state(const bmg_problem* p, int k, const unsigned char* buf, size_t len) {
  StateHead h;
  if (!buf || len < sizeof(StateHead)) fail(BMG_ERR_INVALID_ARG, "state buffer too small");
  std::memcpy(&h, buf, sizeof(h));
  if (h.magic != kStateMagic || h.version != kStateVersion) fail(BMG_ERR_INVALID_ARG, "not a solver state");
  if (h.k != k || h.L != p->L || h.level < 2 || h.level > p->L || h.n_f != p->meshOf(h.level).n ||
      h.n_hist < 0 || h.n_info < 0 || h.n_info > 256 || h.cycle < 0 || h.total_cycles < 0)
    fail(BMG_ERR_INVALID_ARG, "state of another problem, hierarchy or block size");
  if (state_bytes(h) != len) fail(BMG_ERR_INVALID_ARG, "state size mismatch");
  return h;
}

// The BFMG solve (Alg. 4) of one problem and shift on the workspace w and its stream.
// Returns whether every wanted pair met tol; throws BmgException on errors.
bool solve_impl(bmg_problem* p, SolveWork& w, int k, int n_wanted, double sigma, double tol,
                const bmg_options& o, const double* X0, int x0_on_device, double* evals, double* evecs,
                int evecs_on_device, double* resid, bmg_solve_info* info,
                const std::vector<unsigned char>* resume = nullptr, bool* stopped = nullptr) {
  TraceRange trace("bmg_solve");
  AutotuneScope tune_scope(o.autotune != 0);
  w.use_graphs = o.graphs != 0 && !o.adaptive_shift;   // the adaptive shift reads each cycle's Grams
  const int L = p->L;
  const int n2 = p->meshOf(2).n, nL = p->meshOf(L).n;
  // the solve runs on the workspace's own non-blocking stream (capturable into CUDA
  // graphs), ordered after the caller's stream; it returns after its work completes
  if (!w.own) {
    BMG_CUDA(cudaStreamCreateWithFlags(&w.own, cudaStreamNonBlocking));
    BMG_CUDA(cudaEventCreateWithFlags(&w.ev, cudaEventDisableTiming));
  }
  BMG_CUDA(cudaEventRecord(w.ev, w.s));
  BMG_CUDA(cudaStreamWaitEvent(w.own, w.ev, 0));
  w.s = w.own;
  cudaStream_t s = w.s;
  const int ld = w.ld;
  // the cycle graphs hold these values as launch arguments: recapture when they change
  const std::vector<double> sig = {sigma, (double)o.form, (double)o.smoother, (double)o.nu, o.omega,
                                   (double)o.vcycle_depth, (double)o.precision, (double)o.tensor_cores,
                                   (double)(o.selection ? o.index_first : -1)};
  if (sig != w.gsig) {
    BMG_CUDA(cudaStreamSynchronize(s));
    w.drop_graphs();
    w.gsig = sig;
  }
  Blocks<double> b64 = blocks64(w);
  Blocks<float> b32;
  bool fp32 = o.precision == BMG_PREC_FP32;
  if (fp32) {
    ensure_ops32(p);
    b32 = blocks32(p, w);
  }
  if (o.smoother == BMG_SMOOTH_KACZMARZ) ensure_kaczmarz(p, fp32);
  CycleState cs;
  double mu = sigma;   // the shift of the current cycle (adaptive_shift updates it)
  cs.rho.assign(k, 0.0);
  cs.lamv.assign(k, 0.0);
  int total_cycles = 0, fp32_cycles = 0;
  bool converged = false;
  std::vector<int> cyc(L + 1, 0);
  std::vector<double> hist;   // finest-level FP32 max residuals
  std::vector<int> hl, hp;     // per-cycle level and arithmetic (info history)
  std::vector<double> hr;      // per-cycle largest wanted residual
  int f0 = 2, c0 = 0, last_level = 0;
  if (resume) {
    // continue from a state: the iterate on its level, counters and history
    const StateHead h = parse_state(p, k, resume->data(), resume->size());
    if (h.n_wanted != n_wanted || h.sigma != sigma || h.tol != tol || !same_options(h, o))
      fail(BMG_ERR_INVALID_ARG, "resume needs the n_wanted, sigma, tol and options of the stopped solve");
    if (h.cycle >= ((h.level == L) ? o.max_cycles : o.cycles_intermediate))
      fail(BMG_ERR_INVALID_ARG, "state past the cycle budget of its level");
    const unsigned char* q = resume->data() + sizeof(StateHead);
    auto take = [&](void* dst, size_t bytes) { std::memcpy(dst, q, bytes); q += bytes; };
    f0 = h.level;
    c0 = h.cycle;
    fp32 = h.fp32 != 0;
    total_cycles = h.total_cycles;
    fp32_cycles = h.fp32_cycles;
    for (int f = 0; f <= L && f < 33; ++f) cyc[f] = h.cyc[f];
    cs.max_dense_err = h.max_dense_err;
    mu = h.mu;
    hist.resize(h.n_hist);
    hl.resize(h.n_info);
    hp.resize(h.n_info);
    hr.resize(h.n_info);
    take(hist.data(), sizeof(double) * h.n_hist);
    take(hl.data(), sizeof(int32_t) * h.n_info);
    take(hp.data(), sizeof(int32_t) * h.n_info);
    take(hr.data(), sizeof(double) * h.n_info);
    take(cs.lamv.data(), sizeof(double) * k);
    take(cs.rho.data(), sizeof(double) * k);
    BMG_CUDA(cudaMemsetAsync(w.X.get(), 0, sizeof(double) * (size_t)h.n_f * ld, s));
    BMG_CUDA(cudaMemcpy2DAsync(w.X.get(), sizeof(double) * ld, q, sizeof(double) * k, sizeof(double) * k, h.n_f,
                               cudaMemcpyHostToDevice, s));
    if (fp32) convert_block(w.X.get(), ld, b32.X, b32.ld, h.n_f, k, s);
  } else if (o.coarse_start) {
    // Alg. 4 step 1: the eigenvectors of the level-1 problem for the Galerkin pair of
    // level 2, k of them kept as every Rayleigh-Ritz keeps its pairs, prolongated to
    // level 2 (own eigensolve workspace: the cycle's holds a cached factor)
    const int n1 = p->meshOf(1).n;
    const size_t cwn = dense_work_doubles(n1);
    DBuf<double> cw(cwn), cth(k), cy((size_t)n1 * k), cq(1);
    DBuf<int> crk(1);
    BMG_CUDA(cudaMemsetAsync(cw.get(), 0, sizeof(double) * cwn, s));
    dense_eig(w.AQ[2].get(), w.MQ[2].get(), n1, sigma, k, cth.get(), cy.get(), crk.get(), cw.get(), cq.get(),
              kDropFP64, 0, s, o.selection ? o.index_first : -1);
    pack_coarse_kernel<double><<<grid_of((size_t)n1 * ld, 256), 256, 0, s>>>(cy.get(), n1, k, ld, b64.cC[1]);
    check_launch("pack_coarse_kernel");
    prolong<double>(p->meshOf(2), b64.cC[1], w.X.get(), ld, false, s);
    if (fp32) convert_block(w.X.get(), ld, b32.X, b32.ld, n2, k, s);
    BMG_CUDA(cudaStreamSynchronize(s));   // the local buffers are freed on return
  } else {
    // X0 -> X on level 2 (ld-strided; padding columns stay zero)
    BMG_CUDA(cudaMemsetAsync(w.X.get(), 0, sizeof(double) * (size_t)n2 * ld, s));
    BMG_CUDA(cudaMemcpy2DAsync(w.X.get(), sizeof(double) * ld, X0, sizeof(double) * k, sizeof(double) * k, n2,
                               x0_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    if (fp32) convert_block(w.X.get(), ld, b32.X, b32.ld, n2, k, s);
  }
  // keeps the state before cycle c on level f (the iterate is in the X block)
  auto save_state = [&](int f, int c) {
    StateHead h;
    std::memset(&h, 0, sizeof(h));
    h.magic = kStateMagic;
    h.version = kStateVersion;
    h.k = k; h.L = L; h.n_wanted = n_wanted; h.level = f; h.cycle = c; h.fp32 = fp32 ? 1 : 0;
    h.total_cycles = total_cycles; h.fp32_cycles = fp32_cycles; h.n_f = p->meshOf(f).n;
    h.n_hist = (int)hist.size(); h.n_info = (int)hr.size();
    for (int j = 0; j <= L && j < 33; ++j) h.cyc[j] = cyc[j];
    h.sigma = sigma; h.tol = tol; h.max_dense_err = cs.max_dense_err; h.mu = mu;
    head_options(h, o);
    std::vector<unsigned char> buf(state_bytes(h));
    unsigned char* q = buf.data();
    auto put = [&](const void* src, size_t bytes) { std::memcpy(q, src, bytes); q += bytes; };
    put(&h, sizeof(h));
    put(hist.data(), sizeof(double) * hist.size());
    std::vector<int32_t> hl32(hl.begin(), hl.end()), hp32(hp.begin(), hp.end());
    put(hl32.data(), sizeof(int32_t) * hl32.size());
    put(hp32.data(), sizeof(int32_t) * hp32.size());
    put(hr.data(), sizeof(double) * hr.size());
    put(cs.lamv.data(), sizeof(double) * k);
    put(cs.rho.data(), sizeof(double) * k);
    if (fp32) {
      std::vector<float> xf((size_t)h.n_f * k);
      BMG_CUDA(cudaMemcpy2DAsync(xf.data(), sizeof(float) * k, b32.X, sizeof(float) * b32.ld, sizeof(float) * k,
                                 h.n_f, cudaMemcpyDeviceToHost, s));
      BMG_CUDA(cudaStreamSynchronize(s));
      std::vector<double> xd(xf.begin(), xf.end());
      put(xd.data(), sizeof(double) * xd.size());
    } else {
      BMG_CUDA(cudaMemcpy2DAsync(q, sizeof(double) * k, w.X.get(), sizeof(double) * ld, sizeof(double) * k, h.n_f,
                                 cudaMemcpyDeviceToHost, s));
      BMG_CUDA(cudaStreamSynchronize(s));
    }
    p->ckpt[k] = std::move(buf);
  };
  bool halted = false;
  for (int f = f0; f <= L && !halted; ++f) {
    static const char* const kLevelNames[] = {"level 0", "level 1", "level 2", "level 3", "level 4", "level 5",
                                              "level 6", "level 7", "level 8", "level 9", "level 10"};
    TraceRange trace_level(kLevelNames[f <= 10 ? f : 10]);
    const Mesh& mf = p->meshOf(f);
    if (f > f0) {
      if (fp32) prolong<float>(mf, b32.U, b32.X, b32.ld, false, s);
      else prolong<double>(mf, b64.U, b64.X, ld, false, s);
    }
    const int budget = (f == L) ? o.max_cycles : o.cycles_intermediate;
    const double ftol = (f == L) ? tol : o.tol_intermediate;
    for (int c = (f == f0) ? c0 : 0; c < budget; ++c) {
      if (o.stop_after_cycles > 0 && total_cycles >= o.stop_after_cycles) {
        save_state(f, c);
        halted = true;
        break;
      }
      const bool last = c + 1 == budget;
      const bool first = total_cycles == 0;
      const bool conv = fp32 ? run_cycle<float>(p, w, b32, f, o, mu, k, n_wanted, ftol, last, first, cs)
                             : run_cycle<double>(p, w, b64, f, o, mu, k, n_wanted, ftol, last, first, cs);
      last_level = f;
      if (total_cycles < 256) {
        double mr = 0.0;
        for (int i = 0; i < n_wanted; ++i) mr = std::max(mr, cs.rho[i]);
        hl.push_back(f);
        hp.push_back(fp32 ? 1 : 0);
        hr.push_back(mr);
      }
      ++total_cycles;
      if (fp32) ++fp32_cycles;
      cyc[f] = c + 1;
      if (f == L) converged = conv;
      if (conv || last) break;
      if (fp32 && f == L) {
        // hand-over to FP64 cycles: the FP32 residual reached switch_tol, or it
        // did not halve over the last three cycles
        double mr = 0.0;
        for (int i = 0; i < n_wanted; ++i) mr = std::max(mr, cs.rho[i]);
        hist.push_back(mr);
        const size_t h = hist.size();
        if (mr <= o.switch_tol || (h >= 4 && mr > 0.5 * hist[h - 4])) {
          convert_block(b32.X, b32.ld, w.X.get(), ld, nL, ld, s);
          fp32 = false;
        }
      }
    }
    if (converged) break;
  }
  if (stopped) *stopped = halted;
  // outputs: the last Ritz pairs (on level L unless the solve stopped before it)
  const bool on_finest = last_level == L;
  if (fp32 && on_finest) convert_block(b32.U, b32.ld, w.U.get(), ld, nL, ld, s);
  for (int i = 0; i < n_wanted; ++i) evals[i] = cs.lamv[i];
  if (resid) for (int i = 0; i < n_wanted; ++i) resid[i] = cs.rho[i];
  if (evecs && on_finest) {
    BMG_CUDA(cudaMemcpy2DAsync(evecs, sizeof(double) * n_wanted, w.U.get(), sizeof(double) * ld,
                               sizeof(double) * n_wanted, nL,
                               evecs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  }
  BMG_CUDA(cudaStreamSynchronize(s));
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->levels = L;
    for (int f = 2; f <= L && f - 2 < 32; ++f) info->cycles[f - 2] = cyc[f];
    info->total_cycles = total_cycles;
    info->fp32_cycles = fp32_cycles;
    info->n_history = (int)hr.size();
    for (size_t q = 0; q < hr.size(); ++q) {
      info->history_level[q] = hl[q];
      info->history_fp32[q] = hp[q];
      info->history_resid[q] = hr[q];
    }
    info->converged = converged ? 1 : 0;
    double mx = 0.0;
    for (int i = 0; i < n_wanted; ++i) mx = std::max(mx, cs.rho[i]);
    info->max_resid = mx;
    info->max_dense_err = cs.max_dense_err;
    info->final_shift = mu;
  }
  return converged;
}

}  // namespace
}  // namespace bmg

extern "C" bmg_status bmg_solve(bmg_problem* p, int k, int n_wanted, double sigma, double tol,
                                const bmg_options* opt_in, const double* X0, int x0_on_device,
                                double* evals, double* evecs, int evecs_on_device, double* resid,
                                bmg_solve_info* info) {
  bool converged = false, stopped = false;
  bmg_status st = guarded([&] {
    const bmg_options o = checked_options(p, k, n_wanted, sigma, tol, opt_in, X0, evals);
    const std::vector<unsigned char>* state = nullptr;
    if (o.resume) {
      auto it = p->resume_state.find(k);
      if (it == p->resume_state.end()) fail(BMG_ERR_STATE, "resume without a state (bmg_set_state)");
      state = &it->second;
    }
    SolveWork& w = workspace(p, k, 0, p->stream);
    converged = solve_impl(p, w, k, n_wanted, sigma, tol, o, X0, x0_on_device, evals, evecs, evecs_on_device,
                           resid, info, state, &stopped);
  });
  if (st != BMG_OK) return st;
  if (stopped) {
    set_error("stopped after stop_after_cycles cycles; state kept (bmg_get_state)");
    return BMG_ERR_NOT_CONVERGED;
  }
  if (!converged) {
    set_error("cycle cap reached before every wanted pair met tol");
    return BMG_ERR_NOT_CONVERGED;
  }
  return BMG_OK;
}

extern "C" bmg_status bmg_solve_batched(int n_jobs, bmg_problem* const* problems, const double* sigmas, int k,
                                        int n_wanted, double tol, const bmg_options* opt_in,
                                        const double* const* X0, double* const* evals, double* const* evecs,
                                        double* const* resid, bmg_solve_info* infos, int concurrency) {
  struct Result { bmg_status code = BMG_OK; std::string msg; bool converged = false; };
  std::vector<Result> res;
  bmg_status st = guarded([&] {
    if (n_jobs < 1 || !problems || !sigmas || !X0 || !evals) fail(BMG_ERR_INVALID_ARG, "bad batch arrays");
    std::vector<bmg_options> opts(n_jobs);
    std::vector<int> slot(n_jobs, 0);
    if (opt_in && (opt_in->stop_after_cycles != 0 || opt_in->resume != 0))
      fail(BMG_ERR_INVALID_ARG, "stop_after_cycles and resume are for bmg_solve");
    for (int j = 0; j < n_jobs; ++j) {
      opts[j] = checked_options(problems[j], k, n_wanted, sigmas[j], tol, opt_in, X0[j], evals[j]);
      for (int q = 0; q < j; ++q) slot[j] += problems[q] == problems[j];
    }
    for (int j = 0; j < n_jobs; ++j)
      if (opts[j].precision == BMG_PREC_FP32) ensure_ops32(problems[j]);
    int dev = 0;
    BMG_CUDA(cudaGetDevice(&dev));
    const int nthreads = std::max(1, std::min(n_jobs, concurrency > 0 ? concurrency : 64));
    std::vector<cudaStream_t> streams(nthreads, nullptr);
    for (auto& st_ : streams) BMG_CUDA(cudaStreamCreateWithFlags(&st_, cudaStreamNonBlocking));
    // workspaces are made (or found) up front: allocation and release synchronise the device
    std::vector<SolveWork*> works(n_jobs);
    for (int j = 0; j < n_jobs; ++j) {
      works[j] = &workspace(problems[j], k, slot[j], streams[j % nthreads]);
      if (opts[j].precision == BMG_PREC_FP32) blocks32(problems[j], *works[j]);
    }
    for (auto& st_ : streams) BMG_CUDA(cudaStreamSynchronize(st_));
    res.assign(n_jobs, Result());
    std::atomic<int> next{0};
    auto worker = [&](int t) {
      cudaSetDevice(dev);
      for (int j = next.fetch_add(1); j < n_jobs; j = next.fetch_add(1)) {
        try {
          works[j]->s = streams[t];
          res[j].converged = solve_impl(problems[j], *works[j], k, n_wanted, sigmas[j], tol, opts[j], X0[j], 0,
                                        evals[j], evecs ? evecs[j] : nullptr, 0, resid ? resid[j] : nullptr,
                                        infos ? infos + j : nullptr);
        } catch (const BmgException& e) {
          res[j].code = e.code;
          res[j].msg = e.msg;
        } catch (...) {
          res[j].code = BMG_ERR_CUDA;
          res[j].msg = "unknown error";
        }
      }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nthreads; ++t) pool.emplace_back(worker, t);
    worker(0);
    for (auto& th : pool) th.join();
    for (auto& st_ : streams) cudaStreamDestroy(st_);
  });
  if (st != BMG_OK) return st;
  for (int j = 0; j < n_jobs; ++j)
    if (res[j].code != BMG_OK) {
      set_error("job " + std::to_string(j) + ": " + res[j].msg);
      return res[j].code;
    }
  for (int j = 0; j < n_jobs; ++j)
    if (!res[j].converged) {
      set_error("job " + std::to_string(j) + ": cycle cap reached before every wanted pair met tol");
      return BMG_ERR_NOT_CONVERGED;
    }
  return BMG_OK;
}

// ---------------------------------------------- precision-form step entries ---
extern "C" bmg_status bmg_spmm_f32(bmg_problem* p, int f, int level, const float* X, int k, int ld, float* AX,
                                   float* MX, void* stream) {
  return guarded([&] {
    check_levels(p, f, level);
    if (f < 2) fail(BMG_ERR_INVALID_ARG, "f must be >= 2");
    if (!X || !AX || !MX || k < 1 || ld < k || (ld & 3)) fail(BMG_ERR_INVALID_ARG, "bad block arguments (ld % 4 == 0)");
    ensure_ops32(p);
    spmm_am<float>(p->meshOf(level), Ops<float>::A(p, f, level), Ops<float>::M(p, f, level), X, ld, AX, MX,
                   (cudaStream_t)stream);
  });
}

extern "C" bmg_status bmg_smooth_f32(bmg_problem* p, int f, int level, float* X, const float* B, const float* sft,
                                     int k, int ld, int smoother, int nu, double omega, float* work, void* stream) {
  return guarded([&] {
    check_levels(p, f, level);
    if (f < 2) fail(BMG_ERR_INVALID_ARG, "f must be >= 2");
    if (!X || !sft || k < 1 || ld < k || (ld & 3) || nu < 0) fail(BMG_ERR_INVALID_ARG, "bad block arguments (ld % 4 == 0)");
    ensure_ops32(p);
    cudaStream_t s = (cudaStream_t)stream;
    const Mesh& m = p->meshOf(level);
    const float *a = Ops<float>::A(p, f, level), *mm = Ops<float>::M(p, f, level);
    const float *da = Ops<float>::DA(p, f, level), *dm = Ops<float>::DM(p, f, level);
    if (smoother == BMG_SMOOTH_JACOBI) {
      if (!work) fail(BMG_ERR_INVALID_ARG, "Jacobi needs a work block");
      for (int it = 0; it < nu; ++it) {
        jacobi_sweep<float>(m, a, mm, da, dm, X, work, B, sft, ld, omega, s);
        BMG_CUDA(cudaMemcpyAsync(X, work, sizeof(float) * (size_t)m.n * ld, cudaMemcpyDeviceToDevice, s));
      }
    } else if (smoother == BMG_SMOOTH_MCGS || smoother == BMG_SMOOTH_MCSGS) {
      const Level& lv = p->lev[level];
      for (int it = 0; it < nu; ++it) {
        for (int c = 0; c < lv.col1.n_colours; ++c) gs_colour_sweep<float>(m, lv, c, a, mm, da, dm, X, B, sft, ld, s);
        if (smoother == BMG_SMOOTH_MCSGS)
          for (int c = lv.col1.n_colours - 1; c >= 0; --c) gs_colour_sweep<float>(m, lv, c, a, mm, da, dm, X, B, sft, ld, s);
      }
    } else if (smoother == BMG_SMOOTH_KACZMARZ) {
      ensure_kaczmarz(p, true);
      const Level& lv = p->lev[level];
      for (int it = 0; it < nu; ++it)
        for (int c = 0; c < lv.col2.n_colours; ++c)
          kaczmarz_colour_sweep<float>(m, lv, c, a, mm, Ops<float>::NA(p, f, level), Ops<float>::NAM(p, f, level),
                                       Ops<float>::NM(p, f, level), X, B, sft, ld, omega, s);
    } else {
      fail(BMG_ERR_INVALID_ARG, "unknown smoother");
    }
  });
}

extern "C" bmg_status bmg_gram_f32(const float* X, const float* Y, int n, int k, int ld, double* G, void* stream) {
  return guarded([&] {
    if (!X || !Y || !G || n < 1 || k < 1 || k > 160 || ld < k || (ld & 3) || ld > kGramMaxLd)
      fail(BMG_ERR_INVALID_ARG, "bad gram arguments (1 <= k <= 160, k <= ld <= 800, ld % 4 == 0)");
    const int parts = gram_parts(n);
    DBuf<double> partial((size_t)parts * k * k);
    gram(X, Y, n, k, ld, G, partial.get(), parts, (cudaStream_t)stream);
    BMG_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  });
}

extern "C" bmg_status bmg_get_state(const bmg_problem* p, int k, void* buf, size_t len, size_t* used) {
  return guarded([&] {
    if (!p) fail(BMG_ERR_INVALID_ARG, "null problem");
    auto it = p->ckpt.find(k);
    if (it == p->ckpt.end()) fail(BMG_ERR_STATE, "no stopped solve of this block size");
    if (used) *used = it->second.size();
    if (buf) {
      if (len < it->second.size()) fail(BMG_ERR_INVALID_ARG, "state buffer too small");
      std::memcpy(buf, it->second.data(), it->second.size());
    }
  });
}

extern "C" bmg_status bmg_set_state(bmg_problem* p, int k, const void* buf, size_t len) {
  return guarded([&] {
    if (!p) fail(BMG_ERR_INVALID_ARG, "null problem");
    if (!p->L) fail(BMG_ERR_STATE, "bmg_hierarchy not called");
    const unsigned char* b = static_cast<const unsigned char*>(buf);
    parse_state(p, k, b, len);
    p->resume_state[k].assign(b, b + len);
  });
}

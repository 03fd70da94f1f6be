// Internal definitions shared by the libbmg translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/bmg.h"
#include <nvtx3/nvToolsExt.h>

namespace bmg {

// ---------------------------------------------------------------- errors ----
void set_error(const std::string& msg);
// Thrown by fail(); every extern "C" entry catches it and returns its code.
// Host-side trace range (NVTX, header-only): the phases of set-up and solve (assembly,
// hierarchy, levels, the two halves of a cycle, the enriched eigensolve) appear on a
// profiler's timeline; without an attached tool a push or pop is one pointer check.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

struct BmgException {
  bmg_status code;
  std::string msg;
};
// Throwing is confined to the library; every extern "C" entry catches.
[[noreturn]] void fail(bmg_status code, const std::string& msg);
void check_cuda(cudaError_t e, const char* what);
#define BMG_CUDA(call) ::bmg::check_cuda((call), #call)
void check_launch(const char* what);

// ------------------------------------------------------- device buffers ----
// Owning device buffer (cudaMalloc / cudaFree), move-only.
template <typename T>
struct DBuf {
  T* ptr = nullptr;
  size_t n = 0;
  DBuf() = default;
  explicit DBuf(size_t count) { alloc(count); }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : ptr(o.ptr), n(o.n) { o.ptr = nullptr; o.n = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) { release(); ptr = o.ptr; n = o.n; o.ptr = nullptr; o.n = 0; }
    return *this;
  }
  ~DBuf() { release(); }
  void alloc(size_t count);
  void release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    n = 0;
  }
  T* get() const { return ptr; }
};

template <typename T>
void DBuf<T>::alloc(size_t count) {
  release();
  if (count == 0) return;
  cudaError_t e = cudaMalloc(&ptr, count * sizeof(T));
  if (e != cudaSuccess) {
    ptr = nullptr;
    cudaGetLastError();
    fail(BMG_ERR_OOM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed: " +
                          cudaGetErrorString(e));
  }
  n = count;
}

// ----------------------------------------------------------- structures ----
// One refinement of the surface mesh (refinement 0 = the input mesh).
struct Mesh {
  int n = 0, n_tris = 0, nnz = 0;
  DBuf<double> verts;    // [n][3]
  DBuf<int> tris;        // [n_tris][3]
  DBuf<int> parents;     // [n][2]
  DBuf<int> row_ptr;     // [n+1] vertex adjacency incl. self, ascending columns
  DBuf<int> col;         // [nnz]
  DBuf<int> diag_pos;    // [n] position of the diagonal in each row
  DBuf<int> inc_ptr;     // [n+1] incident triangles per vertex
  DBuf<int> inc_tri;     // ascending triangle ids
  DBuf<int> mid;         // [nnz] fine index of the midpoint of edge (i, col) (-1 on diag);
                         //       filled when the next refinement exists
  DBuf<double> valA, valM;  // [nnz] assembled P1 stiffness / mass (refinement >= 1)
  DBuf<int> row_order;   // [n] processing order of rows for the row kernels: vertices
                         //     sorted by the Morton code of their position, so that
                         //     warps running together gather nearby rows (hierarchy levels)
};

// Operators of one level l of the hierarchy, for one finest level f.
struct OpSet {
  DBuf<double> a, m;     // [nnz_l] values on mesh l's pattern
  DBuf<double> da, dm;   // [n_l] diagonals
  DBuf<double> na, nam, nm;  // [n_l] sum a^2, sum a m, sum m^2 per row (Kaczmarz; on first use)
};

// float32 copies of one OpSet (precision form).
struct OpSet32 {
  DBuf<float> a, m, da, dm;
  DBuf<float> na, nam, nm;
};

// A colouring of a level's vertices and its rows grouped by colour.
struct Colouring {
  int n_colours = 0;
  DBuf<int> colour;        // [n]
  DBuf<int> ptr;           // [n_colours+1]
  DBuf<int> rows;          // [n] rows grouped by colour, Morton order within a colour
  std::vector<int> ptr_host;
  std::vector<long long> nnz_host;  // CSR nonzeros of the rows of each colour
};

struct Level {
  int refinement = 0;
  Colouring col1;          // distance 1: Gauss-Seidel
  Colouring col2;          // distance 2 (built on first use): Kaczmarz
};

}  // namespace bmg

namespace bmg {
// Kernel classes timed by the profiler (bmg_profile_*).
enum KernelClass { KC_SPMM = 0, KC_SMOOTH, KC_RESID, KC_TRANSFER, KC_GRAM, KC_DENSE, KC_EXPAND,
                   KC_SMALL, KC_COUNT };

// Process-wide kernel profiler: when enabled, launches of each class are bracketed
// by CUDA events on their stream; totals are folded in by prof_flush() once the
// stream is idle.  Algorithmic bytes and flops per launch are accumulated with them.
void prof_begin(int cls, cudaStream_t s);
void prof_end(int cls, cudaStream_t s, double bytes, double flops);
void prof_flush();
bool prof_enabled();
long long launch_count();
void count_launch();
void count_launches(long long n);

// Workspace of bmg_solve, kept in the problem between calls with the same k.
struct SolveWork {
  cudaStream_t s = nullptr;                 // stream of the solve using it
  int ld = 0, k = 0, n1 = 0, nh = 0, L = 0, parts = 0;
  DBuf<double> X, AX, MX, U, AU, MU, B, W, Zf;
  std::vector<DBuf<double>> cA, cB, cC, cD;  // per coarse level j < L: [N_j][ld]
  DBuf<double> Ahat, Mhat, Y, theta, lam, shift, GA, GM, dense, partial, res;
  DBuf<int> rank;
  DBuf<double> dquality;                    // error estimate of the last enriched eigensolve
  // float32 blocks of the precision form (allocated on first use), ld32 % 4 == 0
  int ld32 = 0;
  DBuf<float> X32, AX32, MX32, U32, AU32, MU32, B32, W32, Zf32, shift32;
  std::vector<DBuf<float>> cA32, cB32, cC32, cD32;
  std::vector<DBuf<double>> AQ, MQ;         // per f: dense n1 x n1 coarse blocks
  std::vector<std::vector<double>> ratio;   // [f][j] max_i dM_i / dA_i
  double* hbuf = nullptr;                   // pinned host staging (res, lam, quality, rank, tc flag)
  DBuf<unsigned char> tcscratch;            // digits of the expansion coefficients (tensor cores)
  DBuf<int> tcerr;                          // raised by a tensor-core kernel whose wait expired
  bool use_graphs = true;                   // bmg_options.graphs of the running solve
  // CUDA graphs of the cycle: part A (steps 1-4) per (level, arithmetic), part B
  // (step 5) per (level, arithmetic, down-leg depth); instantiated on the second cycle
  // of a level on this workspace (the first runs eagerly, so the autotuner can time).
  cudaStream_t own = nullptr;               // the library's non-blocking stream
  cudaEvent_t ev = nullptr;                 // orders `own` after the caller's stream
  std::map<std::tuple<int, int, int, int>, std::pair<cudaGraphExec_t, int>> graphs;  // exec, kernel nodes
  std::set<std::tuple<int, int, int, int>> seen;
  std::vector<double> gsig;                 // solve parameters the graphs were captured with
  void drop_graphs() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second.first);
    graphs.clear();
    seen.clear();
  }
  ~SolveWork() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second.first);
    if (ev) cudaEventDestroy(ev);
    if (own) cudaStreamDestroy(own);
    if (hbuf) cudaFreeHost(hbuf);
  }
};
}  // namespace bmg

// Opaque handle.
struct bmg_problem {
  cudaStream_t stream = nullptr;
  int R = 0;                        // finest refinement
  double amplitude = 0.0;
  std::vector<bmg::Mesh> mesh;      // refinements 0..R
  int L = 0;                        // hierarchy levels (0 until bmg_hierarchy)
  int r0 = 0;                       // refinement of level 1
  std::vector<bmg::Level> lev;      // index 1..L
  // ops[f][j]: operator set of finest level f on level j (j <= f); ops[f][f] aliases
  // the assembled matrices through pointers below.
  std::vector<std::vector<bmg::OpSet>> ops;
  std::vector<double> norm1;        // ||A_f||_1 per level (host)
  // float32 copies of every operator set, ops32[f][j] for j <= f (j == f: the
  // assembled matrices); built on the first precision-form call.
  std::vector<std::vector<bmg::OpSet32>> ops32;
  std::unique_ptr<bmg::SolveWork> ws;  // cached solve workspace (bmg_solve; batch slot 0)
  // per block size k: state of the last stopped solve, and the state to resume from
  std::map<int, std::vector<unsigned char>> ckpt, resume_state;
  std::vector<std::unique_ptr<bmg::SolveWork>> ws_more;  // batch slots 1, 2, ...
  bmg::Mesh& meshOf(int level) { return mesh[r0 + level - 1]; }
  const bmg::Mesh& meshOf(int level) const { return mesh[r0 + level - 1]; }
  const double* opA(int f, int j) const {
    return f == j ? meshOf(j).valA.get() : ops[f][j].a.get();
  }
  const double* opM(int f, int j) const {
    return f == j ? meshOf(j).valM.get() : ops[f][j].m.get();
  }
  const double* opDA(int f, int j) const { return ops[f][j].da.get(); }
  const double* opDM(int f, int j) const { return ops[f][j].dm.get(); }
};

namespace bmg {
// set-up (setup.cu)
void exclusive_scan(const int* in, int* out, int n, int* total_host, cudaStream_t s);
void build_mesh_pattern(Mesh& m, cudaStream_t s);
void refine_mesh(const Mesh& c, Mesh& f, double amplitude, const double* sh_consts_dev,
                 const double* coefs_dev, cudaStream_t s);
void assemble_p1(Mesh& m, cudaStream_t s);
void colour_level(const Mesh& m, Level& lv, cudaStream_t s);
void colour_mesh(const Mesh& m, Colouring& cl, bool distance2, cudaStream_t s);
// distance-2 colouring of the level (Kaczmarz), rows in Morton order; once
void colour_level2(const Mesh& m, Level& lv, cudaStream_t s);
void locality_order(Mesh& m, Level& lv, cudaStream_t s);
void galerkin(const Mesh& fine, const Mesh& coarse, const double* fa, const double* fm,
              double* ca, double* cm, cudaStream_t s);
void extract_diag(const Mesh& m, const double* a, const double* mm, double* da, double* dm,
                  cudaStream_t s);
void fill_sh_constants(double* c17);
void project_input(Mesh& m, double amplitude, const double* sh_consts_dev,
                   const double* coefs_dev, cudaStream_t s);

// cycle steps (ops.cu), for FP64 blocks (T = double) and FP32 blocks (T = float);
// an FP32 block has ld % 4 == 0, an FP64 block ld % 2 == 0.
template <typename T>
void spmm_am(const Mesh& m, const T* a, const T* mm, const T* X, int ld, T* AX, T* MX, cudaStream_t s);
// zero_shift: every shift of the block is zero (M and its diagonal are not read)
template <typename T>
void jacobi_sweep(const Mesh& m, const T* a, const T* mm, const T* da, const T* dm, const T* X,
                  T* Xout, const T* B, const T* shift, int ld, double omega, cudaStream_t s,
                  bool zero_shift = false);
// scratch: a free [N][ld] block of the level, used to time shape candidates on the
// colour's rows (the sweep itself runs in place), or nullptr
template <typename T>
void gs_colour_sweep(const Mesh& m, const Level& lv, int colour, const T* a, const T* mm,
                     const T* da, const T* dm, T* X, const T* B, const T* shift, int ld,
                     cudaStream_t s, T* scratch = nullptr, bool zero_shift = false);
// One multicolour Kaczmarz colour on (A - s_c M) x_c = b_c: each row r of colour c of
// the distance-2 colouring projects x onto its equation, x += omega res / ||k_r||^2 k_r
// with k_r = a_r - s m_r and ||k_r||^2 = na - 2 s nam + s^2 nm.  In place on X.
template <typename T>
void kaczmarz_colour_sweep(const Mesh& m, const Level& lv, int colour, const T* a, const T* mm, const T* na,
                           const T* nam, const T* nm, T* X, const T* B, const T* shift, int ld, double omega,
                           cudaStream_t s);
// na, nam, nm of the operator values a, mm on mesh m's pattern
template <typename T>
void row_norms(const Mesh& m, const T* a, const T* mm, T* na, T* nam, T* nm, cudaStream_t s);
template <typename T>
void residual(const Mesh& m, const T* a, const T* mm, const T* X, const T* B, const T* shift,
              int ld, T* R, cudaStream_t s, bool zero_shift = false);
template <typename T>
void prolong(const Mesh& fine, const T* Xc, T* Y, int ld, bool add, cudaStream_t s);
template <typename T>
void restrict_(const Mesh& coarse, const T* R, T* Zc, int ld, cudaStream_t s);
template <typename T>
void restrict2_(const Mesh& coarse, const T* R, T* Zc, const T* R2, T* Zc2, int ld, cudaStream_t s);
// sym: Y = S X with S symmetric, so G is symmetric: only the 4x4 tiles on and above
// the diagonal are formed (half the products) and the rest mirrored.
void gram(const double* X, const double* Y, int n, int k, int ld, double* G, double* partial,
          int nparts, cudaStream_t s, bool sym = false);
void gram(const float* X, const float* Y, int n, int k, int ld, double* G, double* partial,
          int nparts, cudaStream_t s, bool sym = false);
int gram_parts(int n);
// Widest block the CUDA-core Gram kernels stage (2 x 16 rows of ld values in shared memory).
constexpr int kGramMaxLd = 800;
// Row-kernel autotuning on the calling thread while the scope lives (a solve's
// bmg_options.autotune); off: the default shapes.
struct AutotuneScope {
  explicit AutotuneScope(bool on);
  ~AutotuneScope();
  AutotuneScope(const AutotuneScope&) = delete;
  AutotuneScope& operator=(const AutotuneScope&) = delete;
 private:
  bool prev_;
};
// G[q] = sum of the nparts partials partial[b][q] in block order (q < k*k); with sym an
// entry below the diagonal 4x4 tiles takes its mirror.
void gram_reduce(const double* partial, int nparts, int k, double* G, bool sym, cudaStream_t s);
std::string tuned_report();

// tensor-core products (tc.cu): float64-class results from exact BF16 digit slices on
// tcgen05, for k <= kTcMaxK.  err: device int raised when a bounded wait expired.
constexpr int kTcMaxK = 128;
int gram_tc_parts(int n, int k);
size_t expand_tc_scratch_bytes(int k);
template <typename TI>
void gram_tc(const TI* X, const TI* Y, int n, int k, int ld, double* G, double* partial, int nparts, int* err,
             cudaStream_t s, bool sym);
template <typename TI>
void expand_tc(const TI* Zf, const TI* X, const double* Yx, int n, int k, int ld, int ldy, TI* U,
               unsigned char* scratch, int* err, cudaStream_t s);
// A float64 Gram of the zero 4096 x 64 block X whose bounded waits are made to expire
// (see tc.cu); raises *err.
void gram_tc_timeout_selftest(const double* X, double* G, double* partial, int* err, cudaStream_t s);
template <typename T>
void eig_residuals(const T* AU, const T* MU, const T* U, const double* lam, int n, int k, int ld,
                   double* partial, int nparts, double* out, cudaStream_t s);
template <typename T>
void expand(const T* Zf, const T* X, const double* Yx, int n, int k, int ld, int ldy, T* U,
            cudaStream_t s);
template <typename T>
void scale_rhs(const T* MU, const double* theta, int n, int k, int ld, T* B, cudaStream_t s);

// dense (dense.cu)
// drop_tol: pivots of the unit-diagonal M-hat below it are dropped (kDropFP64 for
// float64 data; kDropFP32 when the enriched matrices come from float32 blocks, whose
// entries carry relative errors near 1e-7 so that smaller pivots are noise).
constexpr double kDropFP64 = 1e-12;
constexpr double kDropFP32 = 1e-5;
// nq > 0: the leading nq x nq block of Mhat repeats from call to call on the same
// work buffer (the coarse space's mass matrix), whose factor is then kept in `work`
// (zero-filled before its first use).
// sel_first < 0: the k pairs of smallest |theta| (index-updating); >= 0: positions
// sel_first .. sel_first + k - 1 of the ascending values (index-fixed; moved down when
// past the top), ordered by (|theta|, theta, index) like the former.
void dense_eig(const double* Ahat, const double* Mhat, int n, double sigma, int k,
               double* theta, double* Y, int* rank, double* work, double* quality, double drop_tol,
               int nq, cudaStream_t s, int sel_first = -1);
size_t dense_work_doubles(int n);
}  // namespace bmg

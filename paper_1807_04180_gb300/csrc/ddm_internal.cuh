// Internal types shared by the CUDA translation units of libddm (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/ddm.h"

namespace ddm {

// ---------------------------------------------------------------------------
// complex arithmetic on interleaved (re, im) pairs
// ---------------------------------------------------------------------------
template <typename T> struct cplx;
template <> struct __align__(8) cplx<float> { float x, y; };
template <> struct __align__(16) cplx<double> { double x, y; };

template <typename T> __host__ __device__ __forceinline__ cplx<T> mk(T a, T b) { cplx<T> r; r.x = a; r.y = b; return r; }
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator-(cplx<T> a) { return mk<T>(-a.x, -a.y); }
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator*(cplx<T> a, cplx<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator*(T s, cplx<T> a) { return mk<T>(s * a.x, s * a.y); }
// acc += a * b
template <typename T> __host__ __device__ __forceinline__ void cfma(cplx<T>& acc, cplx<T> a, cplx<T> b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename T> __host__ __device__ __forceinline__ void cfma_conj(cplx<T>& acc, cplx<T> a, cplx<T> b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}
template <typename T> __host__ __device__ __forceinline__ T cabs2(cplx<T> a) { return a.x * a.x + a.y * a.y; }
template <typename T> __host__ __device__ __forceinline__ cplx<T> cinv(cplx<T> a) {
  T d = a.x * a.x + a.y * a.y;
  return mk<T>(a.x / d, -a.y / d);
}
template <typename To, typename Ti> __host__ __device__ __forceinline__ cplx<To> ccast(cplx<Ti> a) {
  return mk<To>((To)a.x, (To)a.y);
}
typedef cplx<double> z64;   // complex128
typedef cplx<float> c32;    // complex64

// ---------------------------------------------------------------------------
// partition descriptors
// ---------------------------------------------------------------------------
constexpr int MAXDIM = 3;
constexpr int NDIR = 27;     // direction code (dx+1) + 3 (dy+1) + 9 (dz+1); 13 = centre

struct SubDesc;
__host__ __device__ inline long long lvofs(const SubDesc& s, int r, int nrhs);

struct SubDesc {
  int idx[MAXDIM];     // part index per physical axis
  int lo[MAXDIM];      // own node start (global interior node index)
  int nown[MAXDIM];    // own nodes per axis
  int ext[MAXDIM];     // nown + 2e (1 on unused axes)
  int tab[MAXDIM];     // offset of its alpha tables (node table, then half-node inverse table)
  int fid;             // factor id
  int at_lo;           // bit a set: low side of axis a is on the global boundary
  int at_hi;           // bit a set: high side of axis a is on the global boundary
  int pad;            // leading dimension of its factor blocks
  int sofs, scnt;      // its range in the strip-node list (nodes that receive a transfer)
  int pad2;
  long long vofs;      // offset of its local vector with one right-hand side (see lvofs)
  long long fofs;      // element offset of its factor (blocks of b x ldb)
  int nbr[NDIR];       // neighbour id per direction code, -1 if none (nbr[13] = self)
};

// Element offset of right-hand side r's local vector of subdomain s when nrhs right-hand sides
// are stored: subdomain-major, i.e. the nrhs vectors of subdomain 0, then those of subdomain 1,
// ...  A CTA that works on one subdomain and many right-hand sides then touches one contiguous
// region instead of nrhs regions ltotal elements apart (far fewer pages and DRAM rows).
__host__ __device__ inline long long lvofs(const SubDesc& s, int r, int nrhs) {
  return s.vofs * nrhs + (long long)r * s.ext[0] * s.ext[1] * s.ext[2];
}


// everything a kernel needs to evaluate the operator and the partition
struct Geom {
  int dim, e, ov, nsub;
  int N[MAXDIM];          // global extended nodes per axis (1 on unused axes)
  long long nglob;        // product of N
  long long ltotal;       // total local length (one right-hand side)
  double h2;              // h^2
  const double* k2;       // k^2 on the global extended grid
  const z64* tab;         // alpha tables: [ofs .. ofs+ext) alpha at nodes, [ofs+ext .. ofs+2ext+1) 1/alpha at half nodes
  int gtab[MAXDIM];       // offsets of the global box's tables
  const double* beta;     // beta_0(q / ov), q = 0..ov (beta[ov] = 0)
  const SubDesc* subs;
  const void* lcoef;      // per-subdomain operator planes (local precision)
  const z64* gcoef;       // global operator planes (FP64)
  const int* sidx;           // strip-node list: local node index
  const unsigned* smask;     // strip-node list: bit d = receives direction code d; bit 31 = own region
  const int* owner[MAXDIM];  // part owning global extended index g along axis a
  const int* cuts[MAXDIM];   // parts+1 cuts per axis
  int parts[MAXDIM];
};

// error word bits set by kernels
// ERRBIT_WEAKPIV: a dense-block factorisation with pivots restricted to each panel's diagonal rows
// failed its threshold check (not an error: it is redone with the search over all rows)
enum { ERRBIT_TIMEOUT = 1, ERRBIT_SINGULAR = 2, ERRBIT_NONFINITE = 4, ERRBIT_WEAKPIV = 8 };

// ---------------------------------------------------------------------------
// operator coefficients at a node (computed in FP64 from the alpha tables)
// ---------------------------------------------------------------------------
struct Coef {
  z64 c;            // centre
  z64 m[MAXDIM];    // coupling to x - e_a
  z64 p[MAXDIM];    // coupling to x + e_a
};

// alpha tables of one box: node value along axis a at ext index i, inverse half value at j
__device__ __forceinline__ z64 tab_node(const Geom& g, int ofs, int i) { return g.tab[ofs + i]; }
__device__ __forceinline__ z64 tab_ihalf(const Geom& g, int ofs, int ext, int j) { return g.tab[ofs + ext + j]; }

// Coefficients of the J-scaled operator at ext node x of a box with tables tofs[] and
// extents ext[]; k2 value at the node supplied by the caller.
__device__ __forceinline__ Coef coef_at(const Geom& g, const int* tofs, const int* ext, const int* x, double k2v) {
  Coef r;
  z64 an[MAXDIM];
  z64 J = mk<double>(1.0, 0.0);
  for (int a = 0; a < g.dim; ++a) { an[a] = tab_node(g, tofs[a], x[a]); J = J * an[a]; }
  z64 c = (g.h2 * k2v) * J;
  for (int a = 0; a < g.dim; ++a) {
    z64 oth = mk<double>(1.0, 0.0);
    for (int b = 0; b < g.dim; ++b) if (b != a) oth = oth * an[b];
    r.p[a] = oth * tab_ihalf(g, tofs[a], ext[a], x[a] + 1);
    r.m[a] = oth * tab_ihalf(g, tofs[a], ext[a], x[a]);
    c = c - r.p[a] - r.m[a];
  }
  r.c = c;
  return r;
}

// ---------------------------------------------------------------------------
// timing slots (ddm_timing)
// ---------------------------------------------------------------------------
enum { T_SOLVE = 0, T_TRANSFER, T_ASSEMBLE, T_GLOBAL, T_KRYLOV, T_FACTOR, T_GRAPH, T_NSLOT };

namespace nd { struct State; }
}  // namespace ddm

// ---------------------------------------------------------------------------
// the context (C ABI handle)
// ---------------------------------------------------------------------------
struct ddm_ctx {
  ddm_params p;
  int64_t cuts_h[3][4097];
  double omega;
  cudaStream_t st;
  int dim, e, prec;
  // block path: the subdomain factors and solves run on the dense-block machinery (3D z-planes;
  // in 2D when some subdomain's x-lines are wider than the 2D kernels' 128 nodes)
  bool blockpath = false;
  ddm::Geom g;
  std::vector<ddm::SubDesc> subs;
  ddm::SubDesc* d_subs = nullptr;
  // device arrays
  double* d_k2 = nullptr;
  void* d_lcoef = nullptr;       // per-subdomain operator planes (local precision), ltotal x (2 dim + 1)
  ddm::z64* d_gcoef = nullptr;   // global operator planes (FP64), nglob x (2 dim + 1)
  ddm::z64* d_tab = nullptr;
  double* d_beta = nullptr;
  int* d_owner = nullptr;
  int* d_sidx = nullptr;
  unsigned* d_smask = nullptr;
  int max_scnt = 0;
  int* d_cuts = nullptr;
  int* d_err = nullptr;
  double* d_part = nullptr;      // reduction partials
  long long npart = 0;
  double* d_scal = nullptr;      // small device scalars (norms, Krylov coefficients)
  double* h_scal = nullptr;      // pinned host mirror
  // factors (grow-only buffers: graphs of M_K keep their addresses)
  void* d_G = nullptr;
  size_t G_cap = 0;              // bytes
  int nfac = 0;
  std::vector<int> fac_b, fac_m, fac_ldb;
  std::vector<long long> fac_ofs;
  long long fac_elems = 0;
  bool factored = false;
  float factor_ms = 0.f;
  // local vectors (precision of the local solves), max_rhs wide
  void* d_src = nullptr;
  void* d_ring[3] = {nullptr, nullptr, nullptr};
  void* d_U = nullptr;
  // global complex128 work vectors (one right-hand side each unless noted)
  ddm::z64* d_gb = nullptr;      // max_rhs wide
  ddm::z64* d_gr = nullptr;      // max_rhs wide
  ddm::z64* d_gw = nullptr;      // max_rhs wide
  ddm::z64* d_hostbuf = nullptr; // staging for ddm_solve_host: f then u, max_rhs wide each
  double* d_chost = nullptr;     // staging for ddm_set_medium_host
  // Krylov workspace (allocated on first FGMRES solve)
  int kry_m = 0, kry_nb = 0;
  double* d_bscal = nullptr;     // batched Krylov scalars: 4 x nb doubles
  double* h_bscal = nullptr;     // pinned mirror
  int* d_jr = nullptr;           // per right-hand side basis length of the current cycle
  ddm::z64* d_V = nullptr;
  ddm::z64* d_Z = nullptr;
  ddm::z64* d_H = nullptr;       // (m+1) x m column major
  ddm::z64* d_gs = nullptr;      // Givens: cs[m], sn[m], g[m+1], y[m]
  // 3D solves: column offsets of the right-hand sides sharing a factor
  long long* d_col3d = nullptr;
  size_t col3d_cap = 0;
  // tensor-core (tcgen05) path of the mixed-precision 3D plane steps: packed 3xTF32 factors and
  // the packed operand of the current plane step
  bool use_tc = true;
  float* d_gtc = nullptr;
  size_t gtc_cap = 0;            // floats
  std::vector<long long> tc_ofs;
  float* d_ytc = nullptr;
  size_t ytc_cap = 0;
  float* d_tcpart = nullptr;     // split-K partial tiles of the current plane step
  size_t tcpart_cap = 0;
  // tensor-core path of the mixed-precision 2D multi-right-hand-side solves: packed 3xTF32
  // factors (written by ddm_factor when max_rhs >= 16) and their per-factor offsets
  float* d_gtc2 = nullptr;
  long long* d_tc2ofs = nullptr;
  size_t gtc2_cap = 0, tc2ofs_cap = 0;   // floats, entries
  std::vector<long long> tc2_ofs;
  // persistent tensor-core solve: per number of 64-right-hand-side groups, the CTA count and the
  // device arrays of the work lists (CTA i runs items[ofs[i] .. ofs[i+1])), built once outside
  // any graph capture and kept until the context is destroyed
  struct TC2Plan { int nctas = 0; int* d_ofs = nullptr; int2* d_items = nullptr; };
  std::map<int, TC2Plan> tc2plans;
  // autotuned right-hand sides per CTA of the 2D local solve, per nrhs, and the timings taken
  std::map<int, int> tuned_nr;
  int forced_nr = 0;             // ddm_set_rhs_per_cta: 0 = autotuned
  struct TuneRec { int nrhs, nr; float ms; };
  std::vector<TuneRec> tune_log;
  // CUDA graphs of one preconditioner application M_K, per (nrhs, K)
  bool use_graph = false;
  cudaStream_t gstream = nullptr;
  cudaEvent_t gev[2] = {nullptr, nullptr};
  ddm::z64* d_gin = nullptr;
  ddm::z64* d_gout = nullptr;
  struct GraphRec { int nrhs, K; cudaGraphExec_t exec; long long kernels; };
  std::vector<GraphRec> graphs;
  void drop_graphs() {   // a buffer the captured kernels address was reallocated
    for (auto& gr : graphs) cudaGraphExecDestroy(gr.exec);
    graphs.clear();
  }
  // kernels launched by this context (ddm_kernel_launches)
  long long nlaunch = 0;
  // timing
  bool timing = false;
  double t_ms[ddm::T_NSLOT] = {0};
  long long t_n[ddm::T_NSLOT] = {0};
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
  // per-call scratch of ddm_factor and of FGMRES, sized once (no allocation per call)
  unsigned long long* d_hash = nullptr;   // nsub
  int* d_pairs = nullptr;                 // 2 nsub
  int* d_mis = nullptr;                   // nsub
  int* d_reps = nullptr;                  // nsub
  int* d_ldb = nullptr;                   // nsub
  long long* d_fofs = nullptr;            // nsub
  int* d_fsel = nullptr;                  // nsub: factor ids in launch order (by kernel variant)
  ddm::z64* d_coef = nullptr;             // (kry_m + 1) x kry_nb Gram-Schmidt coefficients
  // local solver (ddm_set_local_solver) and the nested-dissection plans, work lists and buffers
  // pivoting of the dense-block factorisation (3D and wide 2D; ddm_set_pivoting): threshold tau
  // of the search restricted to each panel's diagonal rows (0: the cluster search over all rows);
  // piv_full is set while a factorisation is redone after a failed check, piv_redone counts them
  double piv_tau = 4.0;
  bool piv_full = false;
  long long piv_redone = 0;
  int local_solver = DDM_LOCAL_BLOCK;
  int nd_leaf = DDM_ND_LEAF_DEFAULT;
  ddm::nd::State* nd = nullptr;
  std::string err;
};

namespace ddm {
// Device memory of a context: stream-ordered allocations (cudaMallocFromPoolAsync on the
// context's stream) from one memory pool of the library per device, so that creating and
// destroying contexts neither synchronises the device nor stalls work of other contexts (as
// cudaMalloc / cudaFree can).  Freed memory returns to the pool.  dev_free(nullptr) is a no-op.
cudaError_t dev_alloc(ddm_ctx* c, void** p, size_t bytes);
void dev_free(ddm_ctx* c, void* p);
// Pinned host buffers from a process-wide free list (cudaFreeHost can synchronise the device).
cudaError_t host_pinned_alloc(void** p, size_t bytes);
void host_pinned_free(void* p);

// launchers implemented in the .cu files (all enqueue on ctx->st)
cudaError_t launch_build_tables(ddm_ctx* c, const int* d_tdesc, int ntab, double sigma0, double power, int npml);
cudaError_t launch_k2(ddm_ctx* c, const double* c_dev);
cudaError_t launch_coefs(ddm_ctx* c);
cudaError_t launch_beta(ddm_ctx* c);
cudaError_t launch_sub_hash(ddm_ctx* c, unsigned long long* d_hash);
cudaError_t launch_sub_compare(ddm_ctx* c, const int* d_pairs, int npairs, int* d_mismatch);
cudaError_t launch_rhs(ddm_ctx* c, const z64* f, z64* b, int nrhs);
cudaError_t launch_factor_all(ddm_ctx* c, const int* d_reps, const long long* d_fofs, const int* d_ldb);
cudaError_t launch_local_solve(ddm_ctx* c, const void* src, void* out, void* accum, int nrhs);
cudaError_t launch_restrict(ddm_ctx* c, const z64* b, void* src, void* U_zero, int nrhs);
cudaError_t launch_transfer_n(ddm_ctx* c, int s, void* src_next, double* part, int nrhs, int want_res, int* nblk);
cudaError_t launch_assemble(ddm_ctx* c, const void* U, z64* w, int nrhs);
cudaError_t launch_global_apply(ddm_ctx* c, const z64* x, z64* y, const z64* bsub, int nrhs);
// reductions / Krylov building blocks
cudaError_t launch_norm2_partial(ddm_ctx* c, const z64* x, long long n, int nvec, double* part, int* nblocks);
cudaError_t launch_sum_partials(ddm_ctx* c, const double* part, int nblocks, int nvals, double* out);
cudaError_t launch_dots(ddm_ctx* c, const z64* V, int nv, const z64* w, long long n, double* part, int* nblocks);
cudaError_t launch_arnoldi_coef(ddm_ctx* c, const double* part, int nblocks, int nv, z64* Hcol, z64* coef, int first);
cudaError_t launch_sub_axpy(ddm_ctx* c, const z64* V, int nv, const z64* coef, z64* w, long long n);
cudaError_t launch_givens(ddm_ctx* c, int j, int m, const double* nrm2, z64* H, z64* gs, double* out_est);
cudaError_t launch_scale(ddm_ctx* c, const z64* x, const z64* s, z64* dst, long long n);
cudaError_t launch_lsq_update(ddm_ctx* c, int j, int m, z64* H, z64* gs, const z64* Z, z64* x, long long n);
cudaError_t launch_copy_scaled(ddm_ctx* c, const z64* src, double s, z64* dst, long long n);
cudaError_t launch_axpy(ddm_ctx* c, double s, const z64* w, z64* x, long long n);
cudaError_t launch_dots_b(ddm_ctx* c, const z64* V, int nb, int nv, const z64* w, long long n, double* part, int* nblocks);
cudaError_t launch_arnoldi_coef_b(ddm_ctx* c, const double* part, int nblocks, int nv, int nb, z64* H, int j, int m,
                                  z64* coef, int first);
cudaError_t launch_sub_axpy_b(ddm_ctx* c, const z64* V, int nb, int nv, const z64* coef, int m, z64* w, long long n);
cudaError_t launch_givens_b(ddm_ctx* c, int nb, int j, int m, const double* nrm2, z64* H, z64* gs, double* out_est);
cudaError_t launch_scale_b(ddm_ctx* c, int nb, z64* w, const z64* gs, int m, long long n);
cudaError_t launch_scale_vec_b(ddm_ctx* c, int nb, const z64* src, const double* s, z64* dst, long long n);
cudaError_t launch_lsq_update_b(ddm_ctx* c, int nb, const int* d_jr, int m, const z64* H, z64* gs, const z64* Z, z64* x,
                                long long n);
int ring_slots(const ddm_ctx* c);
cudaError_t launch_factor3d(ddm_ctx* c, const std::vector<int>& reps);
// Make `need` bytes of dynamic shared memory launchable for kernel `func` on the current
// device.  The limit is process-wide state of the kernel, so it is raised once to everything the
// device allows beside the kernel's static shared memory (under a lock) instead of being set to
// each context's size before each launch, which races between host threads driving different
// contexts.  cudaErrorInvalidValue if `need` exceeds what the device allows.
cudaError_t allow_dynamic_smem(const void* func, size_t need);
cudaError_t launch_local_solve3d(ddm_ctx* c, const void* src, void* out, void* U, int nrhs);
long long tc3d_packed_floats(int b, int m);
long long tc2d_packed_floats(int b, int m);
cudaError_t tc2d_pack_factors(ddm_ctx* c);
bool tc2d_supported(const ddm_ctx* c, int nrt);
cudaError_t tc2d_solve(ddm_ctx* c, int nrt, const void* src, void* out, void* U, int nrhs);
cudaError_t tc3d_pack_factors(ddm_ctx* c);
// nested-dissection local solver (nd.cu): factor-store layout (sets c->fac_ofs, returns the
// total elements), factorisation of the distinct factors, batched local solve, release
cudaError_t nd_layout(ddm_ctx* c, const std::vector<int>& reps, long long* elems);
cudaError_t nd_factor(ddm_ctx* c, const std::vector<int>& reps);
cudaError_t nd_solve(ddm_ctx* c, const void* src, void* out, void* U, int nrhs);
void nd_free(ddm_ctx* c);
long long nd_read_elems(const ddm_ctx* c);
cudaError_t tc3d_sweeps(ddm_ctx* c, int f, const long long* d_colofs, int ncol, const c32* cS, const c32* cN,
                        const c32* src, c32* out, c32* U);
}  // namespace ddm

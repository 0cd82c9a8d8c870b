// Nested-dissection (multifrontal) local solver for 2D subdomains: the sparse direct
// factorisation the paper uses for Algorithm 3.1's local problems (Section 4, a multifrontal
// solver), in place of the block-tridiagonal inverse of factor.cu / blocks3d.cu.
//
// Ordering.  The subdomain's extended grid (nx x ny nodes, x fastest) is bisected recursively:
// a box of more than `leaf` nodes is cut by one grid line across its longer side; that line is
// the separator, eliminated after the two halves.  Boxes of at most `leaf` nodes are leaves.
// Every tree node ("front") eliminates its pivots P (the separator, or all nodes of a leaf) and
// couples to its boundary set B: the nodes just outside its box, all of which lie on ancestors'
// separators (or nowhere, at the subdomain's Dirichlet edge).
//
// Factor.  The front matrix over [P; B] is assembled from the operator's entries that involve
// a pivot of this front plus the Schur complements of its children (extend-add), then swept by
// Gauss-Jordan over its |P| pivots (partial pivoting among the rows of P):
//     [F_PP F_PB; F_BP F_BB]  ->  [F_PP^-1, F_PP^-1 F_PB; -F_BP F_PP^-1, F_BB - F_BP F_PP^-1 F_PB].
// The first |P| columns, M = [F_PP^-1; -F_BP F_PP^-1] (m x |P|, column-major), are the stored
// factor; the trailing block is the Schur complement passed to the parent.  One launch per tree
// height, over all fronts of that height of every distinct factor; a front of up to ~160
// (complex64) / ~110 (complex128) variables is swept in shared memory, larger ones in place
// in a global scratch (L2-resident).
//
// Solve (u = A^-1 src per subdomain and right-hand side).  Forward, by increasing height: a
// front gathers src on its pivots and its children's update vectors, then
//     [z_P; u] = M r_P + [0; r_B]
// with z_P kept in the output and u (its update vector, |B| values) passed to the parent.
// Backward, by decreasing height: x_P = z_P + M_BP^T x_B, with x_B the already final values of
// its ancestors' separators.  The operator is complex symmetric (A = A^T), so
// F_PP^-1 F_PB = (F_BP F_PP^-1)^T and the backward sweep needs no second block.
// Update vectors are gathered by the parent (no atomics): results do not depend on scheduling.
//
// Precision.  Fronts, stored blocks, update vectors and the working solution are FP64 in both
// precisions of the library; in complex64 contexts only the input source, the output and the
// accumulated U are complex64.  An interior front's pivot block is the operator of its box with
// Dirichlet walls and no PML damping, which can lie close to a resonance: on the 1024^2
// heterogeneous workload such blocks reach condition numbers of about 1e6.  Intermediate values
// then exceed the solution by that factor and cancel in the backward sweep, so rounding either
// the blocks or the intermediate vectors to FP32 loses every digit there (measured: relative
// error O(1) on the worst subdomain), while FP64 keeps the error at the complex64 operator's
// own rounding.  The block-tridiagonal Schur complements of factor.cu never meet this: each one
// is the operator of a region that contains a PML layer.
#include <algorithm>
#include <functional>
#include <map>
#include <vector>

#include <cooperative_groups.h>

#include "ddm_internal.cuh"

namespace ddm {
namespace nd {

// one front of a plan (host); indices local to the plan
struct Front {
  int s = 0, d = 0, h = 0;            // pivots, boundary nodes, height (leaves 0)
  int piv = 0, bnd = 0;               // offsets into Plan::piv / Plan::bnd
  int child[2] = {-1, -1};            // child fronts
  int cmap[2] = {0, 0};               // offsets into Plan::cmap of each child's boundary positions
  int ent = 0, nent = 0;              // offsets into Plan::ent
  int uofs = 0;                       // offset of its update vector (sum of d before it)
  long long mofs = 0, fofs = 0;       // offsets of its stored block M (m x s) and its scratch (m x m)
};

// entry of the front matrix: F[row][col] += plane `plane` of the operator at local node `node`
// (planes: 0 centre, 1 x-, 2 x+, 3 y-, 4 y+)
struct Ent { int row, col, node, plane; };

struct Plan {
  int nx = 0, ny = 0, leaf = 0, height = 0;
  std::vector<Front> fr;              // post-order: children before parents, the root last
  std::vector<int> piv, bnd, cmap;
  std::vector<Ent> ent;
  long long mtot = 0, ftot = 0;       // sum of m*s and of m*m
  int dtot = 0;                       // sum of d
};

Plan build_plan(int nx, int ny, int leaf) {
  Plan P;
  P.nx = nx; P.ny = ny; P.leaf = leaf;
  std::vector<int> pos((size_t)nx * ny, -1);   // position of a node in the front being built
  std::function<int(int, int, int, int)> rec = [&](int x0, int x1, int y0, int y1) -> int {
    if (x1 <= x0 || y1 <= y0) return -1;
    const int w = x1 - x0, h = y1 - y0;
    Front F;
    std::vector<int> pv;
    if ((long long)w * h <= leaf) {
      for (int y = y0; y < y1; ++y)
        for (int x = x0; x < x1; ++x) pv.push_back(y * nx + x);
    } else if (h > w) {                           // cut across y: the separator is an x-line
      const int ym = y0 + h / 2;
      F.child[0] = rec(x0, x1, y0, ym);
      F.child[1] = rec(x0, x1, ym + 1, y1);
      for (int x = x0; x < x1; ++x) pv.push_back(ym * nx + x);
    } else {                                      // cut across x: the separator is a y-line
      const int xm = x0 + w / 2;
      F.child[0] = rec(x0, xm, y0, y1);
      F.child[1] = rec(xm + 1, x1, y0, y1);
      for (int y = y0; y < y1; ++y) pv.push_back(y * nx + xm);
    }
    std::vector<int> bd;                          // nodes just outside the box, inside the grid
    if (y0 > 0) for (int x = x0; x < x1; ++x) bd.push_back((y0 - 1) * nx + x);
    if (y1 < ny) for (int x = x0; x < x1; ++x) bd.push_back(y1 * nx + x);
    if (x0 > 0) for (int y = y0; y < y1; ++y) bd.push_back(y * nx + x0 - 1);
    if (x1 < nx) for (int y = y0; y < y1; ++y) bd.push_back(y * nx + x1);
    std::sort(bd.begin(), bd.end());
    F.s = (int)pv.size();
    F.d = (int)bd.size();
    const int m = F.s + F.d;
    for (int c = 0; c < 2; ++c)
      if (F.child[c] >= 0) F.h = std::max(F.h, P.fr[F.child[c]].h + 1);
    for (int i = 0; i < F.s; ++i) pos[pv[i]] = i;
    for (int i = 0; i < F.d; ++i) pos[bd[i]] = F.s + i;
    // children's boundary nodes lie on this separator or on this machine's boundary
    for (int c = 0; c < 2; ++c) {
      F.cmap[c] = (int)P.cmap.size();
      if (F.child[c] < 0) continue;
      const Front& C = P.fr[F.child[c]];
      for (int t = 0; t < C.d; ++t) P.cmap.push_back(pos[P.bnd[C.bnd + t]]);
    }
    // operator entries with a pivot of this front: (pivot, pivot-or-boundary) from the pivot's
    // row, and (boundary, pivot) from the boundary node's row; entries between two boundary
    // nodes belong to an ancestor's front, entries with an eliminated node to a descendant's
    F.ent = (int)P.ent.size();
    for (int i = 0; i < F.s; ++i) {
      const int n = pv[i], x = n % nx, y = n / nx;
      P.ent.push_back({i, i, n, 0});
      const int nb[4] = {x > 0 ? n - 1 : -1, x + 1 < nx ? n + 1 : -1, y > 0 ? n - nx : -1, y + 1 < ny ? n + nx : -1};
      const int opp[4] = {2, 1, 4, 3};
      for (int q = 0; q < 4; ++q) {
        const int j = nb[q];
        if (j < 0 || pos[j] < 0) continue;
        P.ent.push_back({i, pos[j], n, 1 + q});
        if (pos[j] >= F.s) P.ent.push_back({pos[j], i, j, opp[q]});
      }
    }
    F.nent = (int)P.ent.size() - F.ent;
    for (int v : pv) pos[v] = -1;
    for (int v : bd) pos[v] = -1;
    F.piv = (int)P.piv.size();
    P.piv.insert(P.piv.end(), pv.begin(), pv.end());
    F.bnd = (int)P.bnd.size();
    P.bnd.insert(P.bnd.end(), bd.begin(), bd.end());
    F.uofs = P.dtot;
    P.dtot += F.d;
    F.mofs = P.mtot;
    P.mtot += (long long)m * F.s;
    F.fofs = P.ftot;
    P.ftot += (long long)m * m;
    P.height = std::max(P.height, F.h);
    P.fr.push_back(F);
    return (int)P.fr.size() - 1;
  };
  rec(0, nx, 0, ny);
  return P;
}

}  // namespace nd
}  // namespace ddm

namespace ddm {
namespace nd {

// device copy of a front; indices are global over the concatenated plans of a context
struct FrontD {
  int s, d;
  int piv, bnd;          // into the concatenated pivot / boundary node lists
  int child[2];          // global front ids, -1 if none
  int cmap[2];           // into the concatenated child position maps
  int ent, nent;         // into the concatenated entry list
  int uofs, pad;         // update vector offset within its subdomain's update block
  long long mofs, fofs;  // block M offset within its factor; scratch offset within its factor's scratch
};

constexpr int FT = 256;          // threads of the factor kernel
constexpr int ST = 128;          // threads of the solve kernels

// Entry packing: x = row | col << 16, y = node << 3 | plane.
__device__ __forceinline__ void ent_unpack(int2 v, int& row, int& col, int& node, int& plane) {
  row = v.x & 0xFFFF; col = (int)((unsigned)v.x >> 16); node = (int)((unsigned)v.y >> 3); plane = v.y & 7;
}

// One CTA per (factor f, front): assemble the front, sweep its pivots, store M and the Schur
// complement.  Shared memory: [front (fcap elements) | colk, rowk, rowo (mcap each) |
// perm, colsrc (scap ints each) | warp partials].  A front with m*m > fcap is swept in place
// in its global scratch.
template <typename TC>
__global__ void __launch_bounds__(FT) k_nd_factor(Geom g, const int2* __restrict__ items, const FrontD* __restrict__ fr,
                                                const int* __restrict__ cmap, const int2* __restrict__ ent,
                                                const int* __restrict__ reps, const long long* __restrict__ ffofs,
                                                const long long* __restrict__ fscr, z64* __restrict__ G,
                                                z64* scr, int fcap, int mcap, int scap, int* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  typedef z64 C;
  typedef double T;
  const int2 it = items[blockIdx.x];
  const int f = it.x;
  const FrontD F = fr[it.y];
  const int s = F.s, d = F.d, m = s + d;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = FT / 32;
  const SubDesc& sd = g.subs[reps[f]];
  const long long len = (long long)sd.ext[0] * sd.ext[1];
  const cplx<TC>* lc = (const cplx<TC>*)g.lcoef + sd.vofs * 5;
  C* Fg = scr + fscr[f] + F.fofs;
  const bool in_smem = m * m <= fcap;
  C* A = in_smem ? (C*)smem : Fg;
  C* colk = (C*)smem + fcap;
  C* rowk = colk + mcap;
  C* rowo = rowk + mcap;
  int* perm = (int*)(rowo + mcap);
  int* colsrc = perm + scap;
  T* redv = (T*)(colsrc + scap);
  int* redi = (int*)(redv + nw);

  for (int i = tid; i < m * m; i += FT) A[i] = mk<T>(0, 0);
  __syncthreads();
  for (int e = F.ent + tid; e < F.ent + F.nent; e += FT) {
    int row, col, node, plane;
    ent_unpack(ent[e], row, col, node, plane);
    A[row * m + col] = A[row * m + col] + ccast<double>(lc[plane * len + node]);   // (row, col) pairs are distinct
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 2; ++c) {                  // extend-add, one child at a time
    const int cf = F.child[c];
    if (cf < 0) continue;
    const FrontD K = fr[cf];
    const int mc = K.s + K.d;
    const C* S = scr + fscr[f] + K.fofs;
    const int* cm = cmap + F.cmap[c];
    for (int i = tid; i < K.d * K.d; i += FT) {
      const int a = i / K.d, b = i - a * K.d;
      const int o = cm[a] * m + cm[b];
      A[o] = A[o] + S[(long long)(K.s + a) * mc + K.s + b];
    }
    __syncthreads();
  }
  // Gauss-Jordan sweep over the s pivots, row interchanges among the pivot rows
  for (int k = 0; k < s; ++k) {
    T bv = (T)-1;
    int bi = k;
    for (int i = k + tid; i < s; i += FT) {
      const T v = cabs2(A[i * m + k]);
      if (v > bv) { bv = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_down_sync(0xffffffffu, bv, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { redv[warp] = bv; redi[warp] = bi; }
    __syncthreads();
    bv = redv[0]; bi = redi[0];
    for (int w = 1; w < nw; ++w)
      if (redv[w] > bv || (redv[w] == bv && redi[w] < bi)) { bv = redv[w]; bi = redi[w]; }
    const int r = bi;
    if (tid == 0) {
      perm[k] = r;
      if (!(bv > (T)0) || !(bv < (T)INFINITY)) atomicOr(err, ERRBIT_SINGULAR);
    }
    const C pinv = cinv(A[r * m + k]);
    for (int i = tid; i < m; i += FT) {
      colk[i] = A[(i == k ? r : (i == r ? k : i)) * m + k];
      rowk[i] = A[r * m + i] * pinv;
      rowo[i] = A[k * m + i];
    }
    __syncthreads();
    for (int i = warp; i < m; i += nw) {
      const C ci = colk[i];
      C* Ai = A + (long long)i * m;
      if (i == k) {
        for (int j = lane; j < m; j += 32) Ai[j] = j == k ? pinv : rowk[j];
      } else if (i == r) {
        for (int j = lane; j < m; j += 32) Ai[j] = j == k ? -(ci * pinv) : rowo[j] - ci * rowk[j];
      } else {
        for (int j = lane; j < m; j += 32) Ai[j] = j == k ? -(ci * pinv) : Ai[j] - ci * rowk[j];
      }
    }
    __syncthreads();
  }
  // undo the interchanges on the first s columns: column c of the result is swept column colsrc[c]
  if (tid == 0) {
    for (int c = 0; c < s; ++c) colsrc[c] = c;
    for (int k = s - 1; k >= 0; --k) {
      const int r = perm[k], t = colsrc[k];
      colsrc[k] = colsrc[r];
      colsrc[r] = t;
    }
  }
  __syncthreads();
  C* M = G + ffofs[f] + F.mofs;
  for (int i = tid; i < m * s; i += FT) {
    const int c = i / m, row = i - c * m;
    M[i] = A[row * m + colsrc[c]];
  }
  if (in_smem)
    for (int i = tid; i < d * d; i += FT) {
      const int a = i / d, b = i - a * d;
      Fg[(long long)(s + a) * m + s + b] = A[(s + a) * m + s + b];
    }
}

// A front too large for shared memory is swept by a cluster of NDC CTAs in place in its global
// scratch: CTA q owns the rows i = q (mod NDC).  Per pivot: every CTA finds the best of its own
// candidate rows and publishes it in shared memory; after a cluster barrier each CTA reads the
// NDC candidates (distributed shared memory) and agrees on the pivot row r, copies rows r and k
// (scaled and old) and its own rows' column k, then after a second barrier updates its own
// rows.  Loads of the front bypass L1 (other CTAs write the lines), and the cluster barriers
// order the global writes between CTAs.  Every thread of every CTA passes the same barriers
// (the loop bounds are the front's sizes), so they cannot deadlock.
constexpr int NDC = 8;

__device__ __forceinline__ z64 ldcg(const z64* p) {
  const double2 v = __ldcg((const double2*)p);
  return mk<double>(v.x, v.y);
}

template <typename TC>
__global__ void __cluster_dims__(NDC, 1, 1) __launch_bounds__(FT)
    k_nd_factor_cl(Geom g, const int2* __restrict__ items, const FrontD* __restrict__ fr, const int* __restrict__ cmap,
                   const int2* __restrict__ ent, const int* __restrict__ reps, const long long* __restrict__ ffofs,
                   const long long* __restrict__ fscr, z64* __restrict__ G, z64* scr, int mcap, int scap, int* err) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int q = (int)cl.block_rank();
  extern __shared__ __align__(16) unsigned char smem[];
  typedef z64 C;
  typedef double T;
  __shared__ T cand_v;
  __shared__ int cand_i;
  const int2 it = items[blockIdx.x / NDC];
  const int f = it.x;
  const FrontD F = fr[it.y];
  const int s = F.s, d = F.d, m = s + d;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = FT / 32;
  const int gt = q * FT + tid, GT = NDC * FT;
  const SubDesc& sd = g.subs[reps[f]];
  const long long len = (long long)sd.ext[0] * sd.ext[1];
  const cplx<TC>* lc = (const cplx<TC>*)g.lcoef + sd.vofs * 5;
  C* A = scr + fscr[f] + F.fofs;
  C* rowk = (C*)smem;
  C* rowo = rowk + mcap;
  C* colk = rowo + mcap;                                  // own rows' column k: (mcap + NDC - 1) / NDC
  int* perm = (int*)(colk + (mcap + NDC - 1) / NDC);
  int* colsrc = perm + scap;
  T* redv = (T*)(colsrc + scap);
  int* redi = (int*)(redv + nw);

  for (long long i = gt; i < (long long)m * m; i += GT) A[i] = mk<T>(0, 0);
  cl.sync();
  for (int e = F.ent + gt; e < F.ent + F.nent; e += GT) {
    int row, col, node, plane;
    ent_unpack(ent[e], row, col, node, plane);
    A[row * m + col] = ldcg(A + row * m + col) + ccast<double>(lc[plane * len + node]);
  }
  cl.sync();
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int cf = F.child[c];
    if (cf < 0) continue;
    const FrontD K = fr[cf];
    const int mc = K.s + K.d;
    const C* S = scr + fscr[f] + K.fofs;
    const int* cm = cmap + F.cmap[c];
    for (int i = gt; i < K.d * K.d; i += GT) {
      const int a = i / K.d, b = i - a * K.d;
      const int o = cm[a] * m + cm[b];
      A[o] = ldcg(A + o) + ldcg(S + (long long)(K.s + a) * mc + K.s + b);
    }
    cl.sync();
  }
  for (int k = 0; k < s; ++k) {
    T bv = (T)-1;
    int bi = k;
    const int i0 = k + ((q - k % NDC) + NDC) % NDC;
    for (int i = i0 + tid * NDC; i < s; i += FT * NDC) {
      const T v = cabs2(ldcg(A + (long long)i * m + k));
      if (v > bv) { bv = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_down_sync(0xffffffffu, bv, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { redv[warp] = bv; redi[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < nw; ++w)
        if (redv[w] > bv || (redv[w] == bv && redi[w] < bi)) { bv = redv[w]; bi = redi[w]; }
      cand_v = bv;
      cand_i = bi;
    }
    cl.sync();
    bv = *cl.map_shared_rank(&cand_v, 0);
    bi = *cl.map_shared_rank(&cand_i, 0);
    for (int rr = 1; rr < NDC; ++rr) {
      const T v = *cl.map_shared_rank(&cand_v, rr);
      const int ii = *cl.map_shared_rank(&cand_i, rr);
      if (v > bv || (v == bv && ii < bi)) { bv = v; bi = ii; }
    }
    const int r = bi;
    if (tid == 0) {
      perm[k] = r;
      if (q == 0 && (!(bv > (T)0) || !(bv < (T)INFINITY))) atomicOr(err, ERRBIT_SINGULAR);
    }
    const C pinv = cinv(ldcg(A + (long long)r * m + k));
    for (int j = tid; j < m; j += FT) {
      rowk[j] = ldcg(A + (long long)r * m + j) * pinv;
      rowo[j] = ldcg(A + (long long)k * m + j);
    }
    for (int li = tid; q + li * NDC < m; li += FT) {
      const int i = q + li * NDC;
      colk[li] = ldcg(A + (long long)(i == k ? r : (i == r ? k : i)) * m + k);
    }
    cl.sync();                       // rows k and r are read everywhere before their owners write
    for (int li = warp; q + li * NDC < m; li += nw) {
      const int i = q + li * NDC;
      const C ci = colk[li];
      C* Ai = A + (long long)i * m;
      if (i == k) {
        for (int j = lane; j < m; j += 32) Ai[j] = j == k ? pinv : rowk[j];
      } else if (i == r) {
        for (int j = lane; j < m; j += 32) Ai[j] = j == k ? -(ci * pinv) : rowo[j] - ci * rowk[j];
      } else {
        for (int j = lane; j < m; j += 32) Ai[j] = j == k ? -(ci * pinv) : ldcg(Ai + j) - ci * rowk[j];
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    for (int c = 0; c < s; ++c) colsrc[c] = c;
    for (int k = s - 1; k >= 0; --k) {
      const int r = perm[k], t = colsrc[k];
      colsrc[k] = colsrc[r];
      colsrc[r] = t;
    }
  }
  cl.sync();                         // every row is final (the Schur block stays in place)
  C* M = G + ffofs[f] + F.mofs;
  for (long long i = gt; i < (long long)m * s; i += GT) {
    const int c = (int)(i / m), row = (int)(i - (long long)c * m);
    M[i] = ldcg(A + (long long)row * m + colsrc[c]);
  }
}

// Forward sweep of one tree height.  CTA = (subdomain, front) x group of NR right-hand sides.
// r (shared, NR x mcap): src on the pivots, the children's update vectors added at their
// positions; then [z; u] = M r_P + [0; r_B]: z to the pivots of `out`, u to this front's
// update vector.  M is read once per CTA, coalesced down its columns.
template <typename TV, int NR>
__global__ void __launch_bounds__(ST) k_nd_fwd(Geom g, const int2* __restrict__ items, const FrontD* __restrict__ fr,
                                             const int* __restrict__ piv, const int* __restrict__ cmap,
                                             const long long* __restrict__ ffofs, const long long* __restrict__ subu,
                                             const z64* __restrict__ G, const cplx<TV>* __restrict__ src,
                                             z64* __restrict__ xw, z64* __restrict__ ubuf, int nrhs, int mcap) {
  extern __shared__ __align__(16) unsigned char smem[];
  typedef z64 C;
  typedef double T;
  C* r = (C*)smem;
  const int2 it = items[blockIdx.x];
  const int sub = it.x;
  const FrontD F = fr[it.y];
  const int s = F.s, d = F.d, m = s + d, tid = threadIdx.x;
  const SubDesc& sd = g.subs[sub];
  const int r0 = blockIdx.y * NR, nr = min(NR, nrhs - r0);
  const int* pv = piv + F.piv;
  for (int q = 0; q < NR; ++q)
    for (int p = tid; p < m; p += ST)
      r[q * mcap + p] = (q < nr && p < s) ? ccast<double>(src[lvofs(sd, r0 + q, nrhs) + pv[p]]) : mk<T>(0, 0);
  __syncthreads();
  const long long ubase = subu[sub] * nrhs;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int cf = F.child[c];
    if (cf < 0) continue;
    const FrontD K = fr[cf];
    const C* ub = ubuf + ubase + (long long)K.uofs * nrhs;
    const int* cm = cmap + F.cmap[c];
    for (int q = 0; q < nr; ++q)
      for (int t = tid; t < K.d; t += ST) r[q * mcap + cm[t]] = r[q * mcap + cm[t]] + ub[(long long)(r0 + q) * K.d + t];
    __syncthreads();
  }
  const C* M = G + ffofs[sd.fid] + F.mofs;
  C* uo = ubuf + ubase + (long long)F.uofs * nrhs;
  for (int i = tid; i < m; i += ST) {
    C acc[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) acc[q] = mk<T>(0, 0);
    const C* Mi = M + i;
    int j = 0;
    for (; j + 4 <= s; j += 4) {
      const C a0 = Mi[(long long)j * m], a1 = Mi[(long long)(j + 1) * m];
      const C a2 = Mi[(long long)(j + 2) * m], a3 = Mi[(long long)(j + 3) * m];
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        cfma(acc[q], a0, r[q * mcap + j]);
        cfma(acc[q], a1, r[q * mcap + j + 1]);
        cfma(acc[q], a2, r[q * mcap + j + 2]);
        cfma(acc[q], a3, r[q * mcap + j + 3]);
      }
    }
    for (; j < s; ++j) {
      const C a = Mi[(long long)j * m];
#pragma unroll
      for (int q = 0; q < NR; ++q) cfma(acc[q], a, r[q * mcap + j]);
    }
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      if (q >= nr) break;
      if (i < s) xw[lvofs(sd, r0 + q, nrhs) + pv[i]] = acc[q];
      else uo[(long long)(r0 + q) * d + (i - s)] = r[q * mcap + i] + acc[q];
    }
  }
}

// Backward sweep of one tree height: x_P = z_P + M_BP^T x_B, one warp per pivot column
// (coalesced down the column's boundary part), U += x where U is given.
template <typename TV, int NR>
__global__ void __launch_bounds__(ST) k_nd_bwd(Geom g, const int2* __restrict__ items, const FrontD* __restrict__ fr,
                                             const int* __restrict__ piv, const int* __restrict__ bnd,
                                             const long long* __restrict__ ffofs, const z64* __restrict__ G,
                                             z64* __restrict__ xw, cplx<TV>* __restrict__ out, cplx<TV>* __restrict__ U,
                                             int nrhs, int dcap) {
  extern __shared__ __align__(16) unsigned char smem[];
  typedef z64 C;
  typedef double T;
  C* xb = (C*)smem;
  const int2 it = items[blockIdx.x];
  const int sub = it.x;
  const FrontD F = fr[it.y];
  const int s = F.s, d = F.d, m = s + d, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const SubDesc& sd = g.subs[sub];
  const int r0 = blockIdx.y * NR, nr = min(NR, nrhs - r0);
  const int* pv = piv + F.piv;
  const int* bd = bnd + F.bnd;
  for (int q = 0; q < NR; ++q)
    for (int t = tid; t < d; t += ST) xb[q * dcap + t] = q < nr ? xw[lvofs(sd, r0 + q, nrhs) + bd[t]] : mk<T>(0, 0);
  __syncthreads();
  const C* M = G + ffofs[sd.fid] + F.mofs;
  for (int j = warp; j < s; j += ST / 32) {
    C acc[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) acc[q] = mk<T>(0, 0);
    const C* Mj = M + (long long)j * m + s;
    for (int t = lane; t < d; t += 32) {
      const C w = Mj[t];
#pragma unroll
      for (int q = 0; q < NR; ++q) cfma(acc[q], w, xb[q * dcap + t]);
    }
#pragma unroll
    for (int q = 0; q < NR; ++q)
      for (int o = 16; o > 0; o >>= 1) {
        acc[q].x += __shfl_xor_sync(0xffffffffu, acc[q].x, o);
        acc[q].y += __shfl_xor_sync(0xffffffffu, acc[q].y, o);
      }
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      if (q >= nr) break;
      if (lane == q) {
        const long long o = lvofs(sd, r0 + q, nrhs) + pv[j];
        const C x = xw[o] + acc[q];
        xw[o] = x;
        if (out) out[o] = ccast<TV>(x);
        if (U) U[o] = U[o] + ccast<TV>(x);
      }
    }
  }
}

}  // namespace nd
}  // namespace ddm

namespace ddm {
namespace nd {

struct State {
  int leaf = 0;
  std::vector<Plan> plans;
  std::map<std::pair<int, int>, int> by_shape;   // (nx, ny) -> plan
  std::vector<int> front0;                       // global id of each plan's first front
  std::vector<int> sub_plan;
  int hmax = 0;
  std::vector<int> sofs;                         // solve items of height h: [sofs[h], sofs[h+1])
  std::vector<int> lvl_mmax, lvl_dmax;           // largest m and d among them
  long long utot = 0;                            // update-vector entries per right-hand side
  long long read_elems = 0;                      // factor elements one local solve reads
  FrontD* d_fr = nullptr;
  int *d_piv = nullptr, *d_bnd = nullptr, *d_cmap = nullptr;
  int2* d_ent = nullptr;
  int2* d_sitems = nullptr;
  long long* d_subu = nullptr;
  void* d_ubuf = nullptr;
  void* d_xw = nullptr;                          // FP64 working vector of mixed contexts
  long long* d_ffofs = nullptr;                  // per factor: offset of its blocks in the factor store
  long long* d_fscr = nullptr;                   // per factor: offset of its fronts in the scratch
  int2* d_fitems = nullptr;
  size_t fitems_cap = 0;
  void* d_scr = nullptr;
  size_t scr_cap = 0;
};

static void free_state(ddm_ctx* c, State* S) {
  void* ptrs[] = {S->d_fr, S->d_piv, S->d_bnd, S->d_cmap, S->d_ent, S->d_sitems, S->d_subu, S->d_ubuf, S->d_xw,
                  S->d_ffofs, S->d_fscr, S->d_fitems, S->d_scr};
  for (void* p : ptrs) dev_free(c, p);
  delete S;
}

template <typename V>
static cudaError_t upload(ddm_ctx* c, V** dst, const std::vector<V>& v) {
  cudaError_t e = dev_alloc(c, (void**)dst, sizeof(V) * std::max<size_t>(v.size(), 1));
  if (e != cudaSuccess || v.empty()) return e;
  return cudaMemcpyAsync(*dst, v.data(), sizeof(V) * v.size(), cudaMemcpyHostToDevice, c->st);
}

// Plans of every subdomain shape, their concatenation on the device, the solve work lists and
// the update-vector buffer.  Depends only on the partition and the leaf size: built once.
static cudaError_t prepare(ddm_ctx* c) {
  if (c->nd && c->nd->leaf == c->nd_leaf) return cudaSuccess;
  if (c->nd) { free_state(c, c->nd); c->nd = nullptr; }
  c->drop_graphs();
  State* S = new State;
  S->leaf = c->nd_leaf;
  const int nsub = c->g.nsub;
  for (int i = 0; i < nsub; ++i) {
    const auto key = std::make_pair(c->subs[i].ext[0], c->subs[i].ext[1]);
    auto it = S->by_shape.find(key);
    if (it == S->by_shape.end()) {
      it = S->by_shape.emplace(key, (int)S->plans.size()).first;
      S->plans.push_back(build_plan(key.first, key.second, S->leaf));
    }
    S->sub_plan.push_back(it->second);
  }
  std::vector<FrontD> fr;
  std::vector<int> piv, bnd, cmap;
  std::vector<int2> ent;
  for (const Plan& P : S->plans) {
    const int f0 = (int)fr.size(), p0 = (int)piv.size(), b0 = (int)bnd.size(), c0 = (int)cmap.size(), e0 = (int)ent.size();
    S->front0.push_back(f0);
    for (const Front& F : P.fr) {
      FrontD D;
      D.s = F.s; D.d = F.d; D.piv = p0 + F.piv; D.bnd = b0 + F.bnd;
      for (int k = 0; k < 2; ++k) { D.child[k] = F.child[k] < 0 ? -1 : f0 + F.child[k]; D.cmap[k] = c0 + F.cmap[k]; }
      D.ent = e0 + F.ent; D.nent = F.nent; D.uofs = F.uofs; D.pad = 0; D.mofs = F.mofs; D.fofs = F.fofs;
      fr.push_back(D);
    }
    piv.insert(piv.end(), P.piv.begin(), P.piv.end());
    bnd.insert(bnd.end(), P.bnd.begin(), P.bnd.end());
    cmap.insert(cmap.end(), P.cmap.begin(), P.cmap.end());
    for (const Ent& q : P.ent) ent.push_back(make_int2(q.row | (q.col << 16), (q.node << 3) | q.plane));
    S->hmax = std::max(S->hmax, P.height);
  }
  // solve items by height; update-vector offsets per subdomain
  std::vector<int2> items;
  std::vector<long long> subu(nsub);
  S->sofs.assign(S->hmax + 2, 0);
  S->lvl_mmax.assign(S->hmax + 1, 1);
  S->lvl_dmax.assign(S->hmax + 1, 1);
  for (int h = 0; h <= S->hmax; ++h) {
    S->sofs[h] = (int)items.size();
    for (int i = 0; i < nsub; ++i) {
      const Plan& P = S->plans[S->sub_plan[i]];
      for (int j = 0; j < (int)P.fr.size(); ++j) {
        const Front& F = P.fr[j];
        if (F.h != h) continue;
        items.push_back(make_int2(i, S->front0[S->sub_plan[i]] + j));
        S->lvl_mmax[h] = std::max(S->lvl_mmax[h], F.s + F.d);
        S->lvl_dmax[h] = std::max(S->lvl_dmax[h], F.d);
      }
    }
  }
  S->sofs[S->hmax + 1] = (int)items.size();
  S->utot = 0;
  S->read_elems = 0;
  for (int i = 0; i < nsub; ++i) {
    const Plan& P = S->plans[S->sub_plan[i]];
    subu[i] = S->utot;
    S->utot += P.dtot;
    for (const Front& F : P.fr) S->read_elems += (long long)(F.s + 2 * F.d) * F.s;
  }
  cudaError_t e;
  c->nd = S;
  if ((e = upload(c, &S->d_fr, fr)) != cudaSuccess) return e;
  if ((e = upload(c, &S->d_piv, piv)) != cudaSuccess) return e;
  if ((e = upload(c, &S->d_bnd, bnd)) != cudaSuccess) return e;
  if ((e = upload(c, &S->d_cmap, cmap)) != cudaSuccess) return e;
  if ((e = upload(c, &S->d_ent, ent)) != cudaSuccess) return e;
  if ((e = upload(c, &S->d_sitems, items)) != cudaSuccess) return e;
  if ((e = upload(c, &S->d_subu, subu)) != cudaSuccess) return e;
  if ((e = dev_alloc(c, &S->d_ubuf, sizeof(z64) * std::max<long long>(S->utot, 1) * c->p.max_rhs)) != cudaSuccess) return e;
  if (c->prec == DDM_MIXED &&
      (e = dev_alloc(c, &S->d_xw, sizeof(z64) * c->g.ltotal * c->p.max_rhs)) != cudaSuccess) return e;
  if ((e = dev_alloc(c, (void**)&S->d_ffofs, sizeof(long long) * nsub)) != cudaSuccess) return e;
  if ((e = dev_alloc(c, (void**)&S->d_fscr, sizeof(long long) * nsub)) != cudaSuccess) return e;
  return cudaStreamSynchronize(c->st);   // the host vectors above go out of scope
}

}  // namespace nd

// Factor store layout of the nested-dissection factors: c->fac_ofs[f] and the total elements.
cudaError_t nd_layout(ddm_ctx* c, const std::vector<int>& reps, long long* elems) {
  cudaError_t e = nd::prepare(c);
  if (e != cudaSuccess) return e;
  nd::State* S = c->nd;
  long long ofs = 0;
  for (size_t f = 0; f < reps.size(); ++f) {
    c->fac_ofs[f] = ofs;
    ofs += S->plans[S->sub_plan[reps[f]]].mtot;
  }
  *elems = ofs;
  return cudaMemcpyAsync(S->d_ffofs, c->fac_ofs.data(), sizeof(long long) * reps.size(), cudaMemcpyHostToDevice, c->st);
}

template <typename TC>
static cudaError_t nd_factor_t(ddm_ctx* c, const std::vector<int>& reps) {
  nd::State* S = c->nd;
  const size_t el = sizeof(z64);
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaError_t e = allow_dynamic_smem((const void*)nd::k_nd_factor<TC>, (size_t)optin - 1024);
  if (e != cudaSuccess) return e;
  // scratch: the fronts of as many factors as fit in a budget, one chunk of factors at a time
  size_t total = 0, largest = 0;
  for (int r : reps) {
    const size_t b = (size_t)S->plans[S->sub_plan[r]].ftot * el;
    total += b;
    largest = std::max(largest, b);
  }
  const size_t budget = std::max(largest, std::min(total, (size_t)4 << 30));
  if (budget > S->scr_cap) {
    dev_free(c, S->d_scr);
    S->d_scr = nullptr;
    S->scr_cap = 0;
    if ((e = dev_alloc(c, &S->d_scr, budget)) != cudaSuccess) return e;
    S->scr_cap = budget;
  }
  size_t f0 = 0;
  while (f0 < reps.size()) {
    size_t f1 = f0, used = 0;
    std::vector<long long> fscr(reps.size(), 0);
    while (f1 < reps.size()) {
      const size_t b = (size_t)S->plans[S->sub_plan[reps[f1]]].ftot * el;
      if (f1 > f0 && used + b > budget) break;
      fscr[f1] = (long long)(used / el);
      used += b;
      ++f1;
    }
    // per height: fronts that fit in shared memory (one CTA each), then the larger ones (a
    // cluster each); extra = the shared memory of the single-CTA kernel besides the front
    std::vector<int2> items;
    std::vector<int> sm0(S->hmax + 1), smn(S->hmax + 1), cl0(S->hmax + 1), cln(S->hmax + 1);
    std::vector<int> hm(S->hmax + 1, 1), hs(S->hmax + 1, 1), cm(S->hmax + 1, 1), cs(S->hmax + 1, 1);
    std::vector<long long> fcap(S->hmax + 1, 0);
    for (int h = 0; h <= S->hmax; ++h) {
      // the single-CTA kernel's own shared memory besides the front, for this height's sizes
      int mh = 1, sh = 1;
      for (size_t f = f0; f < f1; ++f) {
        const nd::Plan& P = S->plans[S->sub_plan[reps[f]]];
        for (const nd::Front& F : P.fr)
          if (F.h == h) { mh = std::max(mh, F.s + F.d); sh = std::max(sh, F.s); }
      }
      const size_t extra = 3 * (size_t)mh * el + 2 * (size_t)sh * sizeof(int) + (nd::FT / 32) * (sizeof(double) + sizeof(int)) + 64;
      const size_t room = (size_t)optin - 1024 > extra ? (size_t)optin - 1024 - extra : 0;
      for (int pass = 0; pass < 2; ++pass) {
        (pass == 0 ? sm0 : cl0)[h] = (int)items.size();
        for (size_t f = f0; f < f1; ++f) {
          const int pl = S->sub_plan[reps[f]];
          const nd::Plan& P = S->plans[pl];
          for (int j = 0; j < (int)P.fr.size(); ++j) {
            const nd::Front& F = P.fr[j];
            if (F.h != h) continue;
            const int m = F.s + F.d;
            const bool fits = (size_t)m * m * el <= room;
            if (fits != (pass == 0)) continue;
            items.push_back(make_int2((int)f, S->front0[pl] + j));
            if (fits) {
              hm[h] = std::max(hm[h], m); hs[h] = std::max(hs[h], F.s);
              fcap[h] = std::max(fcap[h], (long long)m * m);
            } else {
              cm[h] = std::max(cm[h], m); cs[h] = std::max(cs[h], F.s);
            }
          }
        }
        (pass == 0 ? smn : cln)[h] = (int)items.size() - (pass == 0 ? sm0 : cl0)[h];
      }
    }
    if (items.size() > S->fitems_cap) {
      dev_free(c, S->d_fitems);
      S->d_fitems = nullptr;
      S->fitems_cap = 0;
      if ((e = dev_alloc(c, (void**)&S->d_fitems, sizeof(int2) * items.size())) != cudaSuccess) return e;
      S->fitems_cap = items.size();
    }
    if ((e = cudaMemcpyAsync(S->d_fitems, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice, c->st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(S->d_fscr, fscr.data(), sizeof(long long) * reps.size(), cudaMemcpyHostToDevice, c->st)) != cudaSuccess) return e;
    for (int h = 0; h <= S->hmax; ++h) {
      if (smn[h] > 0) {
        const size_t smem = (size_t)fcap[h] * el + 3 * (size_t)hm[h] * el + 2 * (size_t)hs[h] * sizeof(int) +
                            (nd::FT / 32) * (sizeof(double) + sizeof(int)) + 64;
        ++c->nlaunch;
        nd::k_nd_factor<TC><<<smn[h], nd::FT, smem, c->st>>>(c->g, S->d_fitems + sm0[h], S->d_fr, S->d_cmap, S->d_ent,
                                                             c->d_reps, S->d_ffofs, S->d_fscr, (z64*)c->d_G,
                                                             (z64*)S->d_scr, (int)fcap[h], hm[h], hs[h], c->d_err);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
      }
      if (cln[h] > 0) {
        const size_t smem = (2 * (size_t)cm[h] + (cm[h] + nd::NDC - 1) / nd::NDC) * el + 2 * (size_t)cs[h] * sizeof(int) +
                            (nd::FT / 32) * (sizeof(double) + sizeof(int)) + 64;
        if ((e = allow_dynamic_smem((const void*)nd::k_nd_factor_cl<TC>, smem)) != cudaSuccess) return e;
        ++c->nlaunch;
        nd::k_nd_factor_cl<TC><<<cln[h] * nd::NDC, nd::FT, smem, c->st>>>(
            c->g, S->d_fitems + cl0[h], S->d_fr, S->d_cmap, S->d_ent, c->d_reps, S->d_ffofs, S->d_fscr, (z64*)c->d_G,
            (z64*)S->d_scr, cm[h], cs[h], c->d_err);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
      }
    }
    // the host vectors of this chunk are reused by the next one
    if ((e = cudaStreamSynchronize(c->st)) != cudaSuccess) return e;
    f0 = f1;
  }
  return cudaSuccess;
}

cudaError_t nd_factor(ddm_ctx* c, const std::vector<int>& reps) {
  return c->prec == DDM_MIXED ? nd_factor_t<float>(c, reps) : nd_factor_t<double>(c, reps);
}

template <typename T, int NR>
static cudaError_t nd_solve_t(ddm_ctx* c, const void* src, void* out, void* U, int nrhs) {
  nd::State* S = c->nd;
  const size_t el = sizeof(z64);
  // FP64 working vector: the output itself in FP64 contexts, a separate buffer in mixed ones
  z64* xw = sizeof(T) == sizeof(double) ? (z64*)out : (z64*)S->d_xw;
  cplx<T>* outv = sizeof(T) == sizeof(double) ? nullptr : (cplx<T>*)out;
  cudaError_t e;
  const int groups = (nrhs + NR - 1) / NR;
  for (int h = 0; h <= S->hmax; ++h) {
    const int n = S->sofs[h + 1] - S->sofs[h];
    const size_t smem = (size_t)NR * S->lvl_mmax[h] * el;
    if ((e = allow_dynamic_smem((const void*)nd::k_nd_fwd<T, NR>, smem)) != cudaSuccess) return e;
    ++c->nlaunch;
    nd::k_nd_fwd<T, NR><<<dim3(n, groups), nd::ST, smem, c->st>>>(
        c->g, S->d_sitems + S->sofs[h], S->d_fr, S->d_piv, S->d_cmap, S->d_ffofs, S->d_subu, (const z64*)c->d_G,
        (const cplx<T>*)src, xw, (z64*)S->d_ubuf, nrhs, S->lvl_mmax[h]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  for (int h = S->hmax; h >= 0; --h) {
    const int n = S->sofs[h + 1] - S->sofs[h];
    const size_t smem = (size_t)NR * S->lvl_dmax[h] * el;
    if ((e = allow_dynamic_smem((const void*)nd::k_nd_bwd<T, NR>, smem)) != cudaSuccess) return e;
    ++c->nlaunch;
    nd::k_nd_bwd<T, NR><<<dim3(n, groups), nd::ST, smem, c->st>>>(
        c->g, S->d_sitems + S->sofs[h], S->d_fr, S->d_piv, S->d_bnd, S->d_ffofs, (const z64*)c->d_G, xw, outv,
        (cplx<T>*)U, nrhs, S->lvl_dmax[h]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T>
static cudaError_t nd_solve_p(ddm_ctx* c, const void* src, void* out, void* U, int nrhs) {
  if (nrhs <= 1) return nd_solve_t<T, 1>(c, src, out, U, nrhs);
  if (nrhs <= 2) return nd_solve_t<T, 2>(c, src, out, U, nrhs);
  if (nrhs <= 4) return nd_solve_t<T, 4>(c, src, out, U, nrhs);
  return nd_solve_t<T, 8>(c, src, out, U, nrhs);
}

cudaError_t nd_solve(ddm_ctx* c, const void* src, void* out, void* U, int nrhs) {
  return c->prec == DDM_MIXED ? nd_solve_p<float>(c, src, out, U, nrhs) : nd_solve_p<double>(c, src, out, U, nrhs);
}

void nd_free(ddm_ctx* c) {
  if (c->nd) nd::free_state(c, c->nd);
  c->nd = nullptr;
}

long long nd_read_elems(const ddm_ctx* c) { return c->nd ? c->nd->read_elems : 0; }

void set_global_error(const std::string& msg);
}  // namespace ddm

// Host-only export of a plan (no CUDA call), for inspection and tests.
extern "C" ddm_status ddm_nd_plan(int nx, int ny, int leaf, ddm_nd_plan_info* info, int* fronts, int* piv, int* bnd,
                                  int* cmap, int* ent) {
  if (!info || nx < 1 || ny < 1 || nx > 4096 || ny > 4096 || leaf < 0 || leaf > 4096) {
    ddm::set_global_error("ddm_nd_plan: need info, 1 <= nx, ny <= 4096 and 0 <= leaf <= 4096");
    return DDM_E_INVAL;
  }
  const ddm::nd::Plan P = ddm::nd::build_plan(nx, ny, leaf == 0 ? DDM_ND_LEAF_DEFAULT : leaf);
  info->nfront = (int)P.fr.size();
  info->height = P.height;
  info->n_piv = (int64_t)P.piv.size();
  info->n_bnd = (int64_t)P.bnd.size();
  info->n_cmap = (int64_t)P.cmap.size();
  info->n_ent = (int64_t)P.ent.size();
  info->factor_entries = P.mtot;
  info->scratch_entries = P.ftot;
  info->update_entries = P.dtot;
  if (fronts)
    for (size_t j = 0; j < P.fr.size(); ++j) {
      const ddm::nd::Front& F = P.fr[j];
      const int row[12] = {F.s, F.d, F.h, F.piv, F.bnd, F.child[0], F.child[1], F.cmap[0], F.cmap[1], F.ent, F.nent, F.uofs};
      std::copy(row, row + 12, fronts + 12 * j);
    }
  if (piv) std::copy(P.piv.begin(), P.piv.end(), piv);
  if (bnd) std::copy(P.bnd.begin(), P.bnd.end(), bnd);
  if (cmap) std::copy(P.cmap.begin(), P.cmap.end(), cmap);
  if (ent)
    for (size_t q = 0; q < P.ent.size(); ++q) {
      ent[4 * q] = P.ent[q].row; ent[4 * q + 1] = P.ent[q].col; ent[4 * q + 2] = P.ent[q].node; ent[4 * q + 3] = P.ent[q].plane;
    }
  return DDM_OK;
}

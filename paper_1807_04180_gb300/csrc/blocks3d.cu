// 3D subdomain factorisation and solves (the local problems of Algorithm 3.1 in 3D).
//
// A 3D subdomain operator in natural ordering (x fastest, then y, then z) is block tridiagonal
// over its z-planes: b = ext_x * ext_y unknowns per plane, m = ext_z planes, diagonal blocks
// T_k (the in-plane 5-point couplings and the centre), and diagonal couplings L_k = diag(c_zm),
// U_k = diag(c_zp) between planes.  As in 2D the factor keeps G_k = D_k^{-1},
// D_k = T_k - L_k G_{k-1} U_{k-1}, column-major with leading dimension ldb; here a block
// (1444 x 1444 for 38^3 subdomains) lives in global memory (it stays in L2) and is inverted by
// blocked Gauss-Jordan with partial pivoting: 16-column panels eliminated by a thread-block
// cluster, the panel's interchanges, and a tiled rank-16 update of the other columns (one pivot
// at a time, an interchange and a rank-1 update kernel per pivot, for planes wider than the
// cluster panel covers).  The solve applies the blocks to every right-hand side that shares the factor at once
// (a GEMM per plane, right-hand sides as columns) with the Schur coupling fused into the
// operand load and the t / x / U updates fused into the epilogue.
#include <algorithm>
#include <type_traits>
#include <vector>

#include <cooperative_groups.h>

#include "ddm_internal.cuh"
#include "tcgen05.cuh"

namespace ddm {

struct F3State { int piv; int bad; double app_x, app_y, inv_x, inv_y; };

// ---------------------------------------------------------------------------------- factor
// D_k into W (row-major b x ldw): W[i][j] = T_k[i][j] - c_zm(i,k) G_{k-1}[i][j] c_zp(j,k-1),
// G_{k-1} read from the stored column-major factor through the column map cm.
template <typename T>
__global__ void k_f3_schur(Geom g, int rep, const cplx<T>* G, long long fofs, int ldb, int k, cplx<T>* W, int ldw,
                           const int* cm) {
  const SubDesc& s = g.subs[rep];
  // 3D: blocks are z-planes (in-plane x and y couplings); 2D (subdomains wider than the 2D
  // kernels take): blocks are x-lines (x couplings only), coupled along y
  const int d = g.dim;
  const int ex = s.ext[0], ey = d == 3 ? s.ext[1] : 1, nb = s.ext[d - 1];
  const int b = ex * ey;
  const long long len = (long long)b * nb;
  const int zm = 2 * d - 1, zp = 2 * d;   // planes of the couplings to the previous / next block
  const cplx<T>* lc = (const cplx<T>*)g.lcoef + s.vofs * (2 * d + 1);   // C, x-, x+, y-, y+(, z-, z+)
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)b * b;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / b), j = (int)(idx - (long long)i * b);
    cplx<T> dv = mk<T>(0, 0);
    const long long oi = (long long)k * b + i;
    if (k > 0) {
      const cplx<T> gij = G[fofs + ((long long)(k - 1) * b + j) * ldb + i];
      const long long oj = (long long)(k - 1) * b + j;
      dv = -(lc[zm * len + oi] * gij * lc[zp * len + oj]);
    }
    if (j == i) dv = dv + lc[oi];
    const int xi = i % ex, yi = i / ex;
    if (j == i + 1 && xi + 1 < ex) dv = dv + lc[2 * len + oi];
    if (j == i - 1 && xi > 0) dv = dv + lc[1 * len + oi];
    if (d == 3 && j == i + ex && yi + 1 < ey) dv = dv + lc[4 * len + oi];
    if (d == 3 && j == i - ex && yi > 0) dv = dv + lc[3 * len + oi];
    W[(long long)i * ldw + j] = dv;
  }
  (void)cm;
}

// pivot of column p (rows >= p), then the interchange of rows p and r, scaling of the pivot
// row, the multipliers of column p (colp) and clearing of column p in the other rows
template <typename T>
__global__ void k_f3_pivot(int b, int p, cplx<T>* W, int ldw, cplx<T>* colp, int* perm, F3State* st, int* err) {
  __shared__ T sbest[32];
  __shared__ int sidx[32];
  __shared__ int s_r;
  __shared__ cplx<T> s_inv, s_app;
  T best = (T)-1;
  int bi = p;
  for (int i = p + threadIdx.x; i < b; i += blockDim.x) {
    const T a = cabs2(W[(long long)i * ldw + p]);
    if (a > best) { best = a; bi = i; }
  }
  for (int o = 16; o; o >>= 1) {
    const T ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  if ((threadIdx.x & 31) == 0) { sbest[threadIdx.x >> 5] = best; sidx[threadIdx.x >> 5] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (sbest[w] > best || (sbest[w] == best && sidx[w] < bi)) { best = sbest[w]; bi = sidx[w]; }
    s_r = bi;
    s_app = W[(long long)p * ldw + p];
    if (!(best > (T)0) || !isfinite(best)) { atomicOr(err, ERRBIT_SINGULAR); s_inv = mk<T>(0, 0); }
    else s_inv = cinv(W[(long long)bi * ldw + p]);
    perm[p] = bi;
    st->piv = bi;
  }
  __syncthreads();
  const int r = s_r;
  const cplx<T> inv = s_inv, app = s_app;
  // thread j alone touches W[p][j], W[r][j] and W[j][p]
  for (int j = threadIdx.x; j < b; j += blockDim.x) {
    const cplx<T> ap = W[(long long)p * ldw + j];
    const cplx<T> ar = W[(long long)r * ldw + j];
    colp[j] = (j == p) ? mk<T>(0, 0) : (j == r ? app : W[(long long)j * ldw + p]);
    W[(long long)p * ldw + j] = (j == p) ? inv : ar * inv;
    if (r != p) W[(long long)r * ldw + j] = (j == p) ? mk<T>(0, 0) : ap;
    if (j != p && j != r) W[(long long)j * ldw + p] = mk<T>(0, 0);
  }
}

// W[i][j] -= colp[i] W[p][j] for every row i != p (rank-1 update, column p already cleared)
template <typename T>
__global__ void k_f3_update(int b, int p, cplx<T>* W, int ldw, const cplx<T>* colp) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= b) return;
  const cplx<T> mp = W[(long long)p * ldw + j];
  for (int i = blockIdx.y; i < b; i += gridDim.y) {
    if (i == p) continue;
    cplx<T> cur = W[(long long)i * ldw + j];
    cfma(cur, -colp[i], mp);
    W[(long long)i * ldw + j] = cur;
  }
}

// Blocked Gauss-Jordan on W (the same block step as the 2D factor, for 3D's wide plane blocks).
// For a panel P = [p0, p0 + w):
//  1. k_f3_panel_cl: a cluster of CTAs holds the panel's columns (all b rows) in registers and
//     runs the unblocked elimination on them (pivot search over rows >= c, interchange, scaling,
//     elimination of column c from every other row); the panel then holds the new column block
//     of the inverse, and the panel's interchanges are composed into a list of moved rows;
//  2. k_f3_gather: the interchanges on the other columns; the old pivot rows are saved in Tp
//     (w x b) and zeroed in W;
//  3. k_f3_rankw: every other column takes the w elimination steps at once,
//     W[i][j] += sum_q W[i][p0 + q] Tp[q][j]  (for the pivot rows this is their new value).
// Three launches per panel instead of two per pivot.
template <typename T> struct F3Panel { static constexpr int W = 16; };
template <> struct F3Panel<double> { static constexpr int W = 8; };

// The same panel elimination spread over a cluster of F3C_N CTAs (planes up to F3C_N x 256 rows
// wide): CTA q holds rows [q R, (q + 1) R), R = ceil(b / F3C_N), one row per thread in registers.
// One cluster barrier per pivot: after eliminating pivot c, every CTA writes its best candidate
// for pivot c + 1 (value, row index and the row's panel values) into its slot of every CTA's
// shared memory, and the holder of row c + 1 writes that row too; after the barrier each CTA
// picks the pivot among the F3C_N slots and has the pivot row and the old row c + 1 locally.  The
// slots alternate between two buffers by pivot parity, so a slot is rewritten only after every
// CTA has passed the barrier that follows its last read.  Every thread of every CTA passes the
// same barriers (the loop bounds are kernel arguments), so the cluster barriers cannot deadlock.
constexpr int F3C_N = 8, F3C_T = 256;

// Compose a panel's interchanges (step q moved row perm[q] to row p0 + q) into (destination,
// source) rows for k_f3_gather: lane t holds one touched row (the panel's rows first) and the row
// its content comes from.  One warp; swl[0] = number of pairs.
__device__ __forceinline__ void f3_compose_swaps(int p0, int w, const int* s_perm, int* swl, int lane) {
  int row_l = lane < w ? p0 + lane : -1, src_l = row_l, n = w;
  for (int qc = 0; qc < w; ++qc) {
    const int pr = s_perm[qc];
    const unsigned m = __ballot_sync(0xffffffffu, row_l == pr);
    int bb;
    if (m) {
      bb = __ffs(m) - 1;
    } else {
      bb = n;
      if (lane == n) { row_l = pr; src_l = pr; }
      ++n;
    }
    const int sa = __shfl_sync(0xffffffffu, src_l, qc), sb = __shfl_sync(0xffffffffu, src_l, bb);
    if (lane == qc) src_l = sb;
    if (lane == bb) src_l = sa;
  }
  const bool emit = lane < n && (lane < w || src_l != row_l);
  const unsigned em = __ballot_sync(0xffffffffu, emit);
  const int pos = __popc(em & ((1u << lane) - 1u));
  if (emit) { swl[1 + 2 * pos] = row_l; swl[2 + 2 * pos] = src_l; }
  if (lane == 0) swl[0] = __popc(em);
}

template <typename T>
__global__ void __cluster_dims__(F3C_N, 1, 1) __launch_bounds__(F3C_T)
    k_f3_panel_cl(int b, int p0, int w, cplx<T>* W, int ldw, int* perm, int* swl, int* err) {
  namespace cg = cooperative_groups;
  constexpr int PW = F3Panel<T>::W;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  __shared__ T s_wb[F3C_T / 32];
  __shared__ int s_wi[F3C_T / 32];
  __shared__ T s_best;
  __shared__ int s_idx;
  // slots written by the cluster's CTAs: candidate value, row and panel values per CTA; row c
  __shared__ T s_cv[2][F3C_N];
  __shared__ int s_ci[2][F3C_N];
  __shared__ cplx<T> s_crow[2][F3C_N][PW];
  __shared__ cplx<T> s_rowc[2][PW];
  __shared__ int s_bad, s_perm[PW];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int rpc = (b + F3C_N - 1) / F3C_N;
  const int i = rank * rpc + tid;
  const bool have = tid < rpc && i < b;
  cplx<T> R[PW];
#pragma unroll
  for (int q = 0; q < PW; ++q) R[q] = (have && q < w) ? W[(long long)i * ldw + p0 + q] : mk<T>(0, 0);
  if (tid == 0) s_bad = 0;
  // the warp holding local row lr sends that row's panel values to dst(d) in every CTA d
  auto send_row = [&](int row, auto dst) {
    const int lr = row - rank * rpc;
    if (row < 0 || row >= b || lr < 0 || lr >= rpc || wid != (lr >> 5)) return;   // warp-uniform
    const int src = lr & 31;
    cplx<T> mine = mk<T>(0, 0);
#pragma unroll
    for (int q = 0; q < PW; ++q) {
      const T x = __shfl_sync(0xffffffffu, R[q].x, src);
      const T y = __shfl_sync(0xffffffffu, R[q].y, src);
      if (lane == q) mine = mk<T>(x, y);
    }
    if (lane < PW)
      for (int d = 0; d < F3C_N; ++d) dst((unsigned)d)[lane] = mine;
  };
  // this CTA's best candidate (largest |.|^2, ties to the lowest row) into slot buf of every CTA,
  // with its row; and row c into every CTA's s_rowc[buf]
  auto publish = [&](T best, int bi, int buf, int c) {
    for (int o = 16; o; o >>= 1) {
      const T ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { s_wb[wid] = best; s_wi[wid] = bi; }
    __syncthreads();
    if (tid == 0) {
      for (int q = 1; q < F3C_T / 32; ++q)
        if (s_wb[q] > best || (s_wb[q] == best && s_wi[q] < bi)) { best = s_wb[q]; bi = s_wi[q]; }
      s_best = best;
      s_idx = bi;
    }
    __syncthreads();
    const int cb = s_idx;
    if (tid < F3C_N) {
      *cl.map_shared_rank(&s_cv[buf][rank], (unsigned)tid) = s_best;
      *cl.map_shared_rank(&s_ci[buf][rank], (unsigned)tid) = cb;
    }
    send_row(cb, [&](unsigned d) { return cl.map_shared_rank(&s_crow[buf][rank][0], d); });
    send_row(c, [&](unsigned d) { return cl.map_shared_rank(&s_rowc[buf][0], d); });
  };
  {
    T best = (T)-1;
    int bi = b;
    if (have && i >= p0) { best = cabs2(R[0]); bi = i; }
    publish(best, bi, 0, p0);
  }
  cl.sync();
#pragma unroll 1
  for (int qc = 0; qc < w; ++qc) {
    const int c = p0 + qc, buf = qc & 1;
    // the cluster's pivot from the slots (every warp alike): lane l < F3C_N reads CTA l's slot
    T best = lane < F3C_N ? s_cv[buf][lane] : (T)-1;
    int r = lane < F3C_N ? s_ci[buf][lane] : b;
    int k = lane < F3C_N ? lane : F3C_N;
    for (int o = 16; o; o >>= 1) {
      const T ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, r, o);
      const int ok2 = __shfl_xor_sync(0xffffffffu, k, o);
      if (ob > best || (ob == best && oi < r)) { best = ob; r = oi; k = ok2; }
    }
    const bool ok = best > (T)0 && isfinite(best) && r < b && k < F3C_N;
    if (!ok) { r = c; k = 0; }
    const cplx<T>* prow = s_crow[buf][k];      // old row r
    const cplx<T>* vc = s_rowc[buf];           // old row c
    if (rank == 0 && tid == 0) {
      perm[c] = r;
      s_perm[qc] = r;
      if (!ok) s_bad = 1;
    }
    const cplx<T> inv = ok ? cinv(prow[qc]) : mk<T>(0, 0);
    // interchange and elimination of column qc on this thread's row; candidate of the next pivot
    T nb = (T)-1;
    int ni = b;
    if (have) {
      if (i == c) {
#pragma unroll
        for (int q = 0; q < PW; ++q) R[q] = q == qc ? inv : prow[q] * inv;
      } else {
        if (i == r) {
#pragma unroll
          for (int q = 0; q < PW; ++q) R[q] = vc[q];   // row r takes old row c
        }
        cplx<T> fi = mk<T>(0, 0);
#pragma unroll
        for (int q = 0; q < PW; ++q)
          if (q == qc) fi = -R[q];
        const cplx<T> fiv = fi * inv;
#pragma unroll
        for (int q = 0; q < PW; ++q) {
          if (q == qc) R[q] = fiv;
          else cfma(R[q], fiv, prow[q]);    // fi rs[q] = (fi inv) prow[q]
        }
        if (i > c && qc + 1 < w) {
          cplx<T> nx = mk<T>(0, 0);
#pragma unroll
          for (int q = 0; q < PW; ++q)
            if (q == qc + 1) nx = R[q];
          nb = cabs2(nx);
          ni = i;
        }
      }
    }
    if (qc + 1 < w) {
      publish(nb, ni, buf ^ 1, c + 1);
      cl.sync();
    }
  }
#pragma unroll
  for (int q = 0; q < PW; ++q)
    if (have && q < w) W[(long long)i * ldw + p0 + q] = R[q];
  if (tid == 0 && s_bad) atomicOr(err, ERRBIT_SINGULAR);
  if (rank == 0 && wid == 0) f3_compose_swaps(p0, w, s_perm, swl, lane);
}

// The panel elimination with the pivots taken on the panel's diagonal (no interchanges), checked.
// The Schur blocks of this method contain a PML layer, and partial pivoting over all rows takes
// their diagonal entries (pivot growth 1 in every block examined), so the cluster search above is
// not needed to find them.  Without interchanges, Gauss-Jordan on the panel turns its diagonal
// block A into A^-1 and every other row's panel values v into X = -v A^-1 (rows of earlier panels
// included).  Each CTA therefore inverts A in shared memory (one element per thread, two barriers
// per step, no barrier between CTAs) and forms X for its rows as one 1 x w by w x w product; CTA 0
// writes A^-1, the identity permutation and the interchange list.  Checks, against threshold tau:
// a block row below the step's pivot holding more than tau times it (what partial pivoting would
// have swapped in), or an unpivoted row's multiplier |X| above tau, sets ERRBIT_WEAKPIV and the
// host redoes the factorisation with k_f3_panel_cl.  With wp > 0 the kernel first applies the
// previous panel [pp, pp + wp) to this panel's columns, W[i][j] += sum_q W[i][pp + q] Tp[q][j]
// (what k_f3_rankw_cols does), so that update is not a launch of its own on the critical path.
constexpr int F3B_T = 256;

template <typename T>
__global__ void __launch_bounds__(F3B_T) k_f3_panel_blk(int b, int pp, int wp, const cplx<T>* __restrict__ Tp, int p0,
                                                      int w, cplx<T>* W, int ldw, int* perm, int* swl, T tau2,
                                                      int* err) {
  constexpr int PW = F3Panel<T>::W;
  __shared__ cplx<T> As[PW][PW + 1];
  __shared__ cplx<T> Ts[PW][PW];         // the previous panel's old pivot rows in this panel's columns
  __shared__ int s_perm[PW];
  __shared__ int s_bad, s_weak;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int ea = tid / PW, eq = tid - ea * PW;             // this thread's element of the block
  const bool he = ea < w && eq < w;
  if (tid == 0) { s_bad = 0; s_weak = 0; }
  if (tid < wp * w) {
    const int q = tid / w, j = tid - q * w;
    Ts[q][j] = Tp[(long long)q * ldw + p0 + j];
  }
  __syncthreads();
  if (he) {
    cplx<T> v = W[(long long)(p0 + ea) * ldw + p0 + eq];
    for (int q = 0; q < wp; ++q) cfma(v, W[(long long)(p0 + ea) * ldw + pp + q], Ts[q][eq]);
    As[ea][eq] = v;
  }
  __syncthreads();
  bool weak = false, bad = false;
  for (int qc = 0; qc < w; ++qc) {
    const cplx<T> pv = As[qc][qc];
    const T pa = cabs2(pv);
    const bool ok = pa > (T)0 && isfinite(pa);
    bad = bad || !ok;
    const cplx<T> inv = ok ? cinv(pv) : mk<T>(0, 0);
    cplx<T> colv = mk<T>(0, 0), rowv = mk<T>(0, 0), cur = mk<T>(0, 0);
    if (he) { colv = As[ea][qc]; rowv = As[qc][eq]; cur = As[ea][eq]; }
    __syncthreads();
    if (he) {
      cplx<T> nv;
      if (ea == qc) {
        nv = eq == qc ? inv : rowv * inv;
      } else {
        const cplx<T> fiv = (-colv) * inv;
        if (eq == qc) {
          nv = fiv;
          weak = weak || (ea > qc && cabs2(colv) > tau2 * pa);
        } else {
          nv = cur;
          cfma(nv, fiv, rowv);
        }
      }
      As[ea][eq] = nv;
    }
    __syncthreads();
  }
  if (blockIdx.x == 0) {
    if (he) W[(long long)(p0 + ea) * ldw + p0 + eq] = As[ea][eq];
    if (tid < w) { s_perm[tid] = p0 + tid; perm[p0 + tid] = p0 + tid; }
    __syncthreads();
    if (wid == 0) f3_compose_swaps(p0, w, s_perm, swl, lane);
  }
  for (int i = blockIdx.x * F3B_T + tid; i < b; i += gridDim.x * F3B_T) {
    if (i >= p0 && i < p0 + w) continue;
    const bool unpiv = i >= p0 + w;      // rows below p0 are earlier pivot rows
    cplx<T> v[PW], x[PW];
#pragma unroll
    for (int q = 0; q < PW; ++q) {
      v[q] = q < w ? W[(long long)i * ldw + p0 + q] : mk<T>(0, 0);
      x[q] = mk<T>(0, 0);
    }
    if (wp > 0) {                        // the previous panel's update of these columns
#pragma unroll
      for (int q2 = 0; q2 < PW; ++q2) {
        if (q2 >= wp) break;
        const cplx<T> xp = W[(long long)i * ldw + pp + q2];
#pragma unroll
        for (int q = 0; q < PW; ++q) cfma(v[q], xp, Ts[q2][q]);
      }
    }
#pragma unroll
    for (int a2 = 0; a2 < PW; ++a2) {
      if (a2 >= w) break;
      const cplx<T> nv = -v[a2];
#pragma unroll
      for (int q = 0; q < PW; ++q) cfma(x[q], nv, As[a2][q]);
    }
#pragma unroll
    for (int q = 0; q < PW; ++q)
      if (q < w) {
        weak = weak || (unpiv && cabs2(x[q]) > tau2);
        W[(long long)i * ldw + p0 + q] = x[q];
      }
  }
  if (weak) s_weak = 1;
  if (bad) s_bad = 1;
  __syncthreads();
  if (tid == 0 && blockIdx.x == 0 && s_bad) atomicOr(err, ERRBIT_SINGULAR);
  if (tid == 0 && s_weak) atomicOr(err, ERRBIT_WEAKPIV);
}

// thread per column j outside the panel, driven by the list of k_f3_panel_cl: every moved row's
// source is loaded first, then the old pivot rows go to Tp (w x ldw) and are zeroed in W and the
// other moved rows are written in place
template <typename T>
__global__ void k_f3_gather(int b, int p0, int w, cplx<T>* W, int ldw, const int* swl, cplx<T>* Tp) {
  constexpr int PW = F3Panel<T>::W;
  __shared__ int s_dst[2 * PW], s_src[2 * PW], s_n;
  if (threadIdx.x == 0) s_n = swl[0];
  if (threadIdx.x < 2 * PW) {
    s_dst[threadIdx.x] = swl[1 + 2 * threadIdx.x];
    s_src[threadIdx.x] = swl[2 + 2 * threadIdx.x];
  }
  __syncthreads();
  const int n = s_n;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < b; j += gridDim.x * blockDim.x) {
    if (j >= p0 && j < p0 + w) continue;
    cplx<T> v[2 * PW];
#pragma unroll
    for (int t = 0; t < 2 * PW; ++t)
      if (t < n) v[t] = W[(long long)s_src[t] * ldw + j];
#pragma unroll
    for (int t = 0; t < 2 * PW; ++t) {
      if (t >= n) break;
      const int d = s_dst[t];
      if (d >= p0 && d < p0 + w) {
        Tp[(long long)(d - p0) * ldw + j] = v[t];
        W[(long long)d * ldw + j] = mk<T>(0, 0);
      } else {
        W[(long long)d * ldw + j] = v[t];
      }
    }
  }
}

// W[i][j] += sum_q W[i][p0 + q] Tp[q][j] for the columns j outside the panel: 64 x 64 tiles,
// 256 threads, 4 x 4 outputs each (rows ty + 16 a, columns tx + 16 c)
// (columns j in [jlo, jhi) outside [xlo, xhi); tile columns start at jlo rounded down to 64)
template <typename T>
__global__ void __launch_bounds__(256) k_f3_rankw(int b, int p0, int w, cplx<T>* W, int ldw, const cplx<T>* Tp,
                                                  int jlo, int jhi, int xlo, int xhi) {
  constexpr int PW = F3Panel<T>::W;
  __shared__ cplx<T> As[64][PW + 1];
  __shared__ cplx<T> Bs[PW][64];
  const int i0 = blockIdx.y * 64, j0 = (jlo & ~63) + blockIdx.x * 64;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int idx = tid; idx < 64 * PW; idx += 256) {
    const int ii = idx / PW, q = idx - ii * PW;
    As[ii][q] = (i0 + ii < b && q < w) ? W[(long long)(i0 + ii) * ldw + p0 + q] : mk<T>(0, 0);
  }
  for (int idx = tid; idx < PW * 64; idx += 256) {
    const int q = idx >> 6, jj = idx & 63;
    Bs[q][jj] = (j0 + jj < b && q < w) ? Tp[(long long)q * ldw + j0 + jj] : mk<T>(0, 0);
  }
  __syncthreads();
  cplx<T> acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = i0 + ty + 16 * a, j = j0 + tx + 16 * c;
      acc[a][c] = (i < b && j < b) ? W[(long long)i * ldw + j] : mk<T>(0, 0);
    }
#pragma unroll
  for (int q = 0; q < PW; ++q) {
    cplx<T> av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = As[ty + 16 * a][q];
#pragma unroll
    for (int c = 0; c < 4; ++c) bv[c] = Bs[q][tx + 16 * c];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) cfma(acc[a][c], av[a], bv[c]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = i0 + ty + 16 * a, j = j0 + tx + 16 * c;
      if (i < b && j >= jlo && j < jhi && (j < xlo || j >= xhi)) W[(long long)i * ldw + j] = acc[a][c];
    }
}

// The rank-16 update of k_f3_rankw (complex64) on the tensor cores, one 128 x 128 tile of W per
// CTA (256 threads): D[j][i] = sum_q Tp[q][j] P[i][q], P = the panel's new columns W[i][p0 + q],
// as a split-TF32 complex contraction (12 MMAs of M = 128 columns j, N = 128 rows i, K = 8 per
// K step, two K steps) into two TMEM accumulators (real: columns 0-127, imaginary: 128-255); then
// each thread (TMEM lane = column j of W, half of the rows) adds row by row: W[i][j] += D[j][i]
// for the columns outside the panel (coalesced along j).  The operands are built in shared memory by the CTA's threads
// (K-major core matrices, planes {re hi, re lo, im hi, im lo} of A = Tp^T and of B = P).
constexpr int RW_T = 128, RW_K = 16;                   // tile, K (complex columns of the panel)
constexpr int RW_PLANE = RW_T * RW_K;                  // floats per plane (8 KB)
constexpr int RW_SMEM = 8 * RW_PLANE * 4 + 1024;       // A and B, 4 planes each, 1 KB alignment

__global__ void __launch_bounds__(256, 1)
    k_f3_rankw_tc(int b, int p0, int w, c32* W, int ldw, const c32* __restrict__ Tp, int xlo, int xhi, int* err) {
  extern __shared__ unsigned char rw_raw[];
  __shared__ __align__(8) uint64_t s_acc;
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int j0 = blockIdx.x * RW_T, i0 = blockIdx.y * RW_T;
  const uint32_t base = (tc::smem_addr(rw_raw) + 1023u) & ~1023u;
  float* A = reinterpret_cast<float*>(rw_raw + (base - tc::smem_addr(rw_raw)));   // 4 planes of Tp^T
  float* B = A + 4 * RW_PLANE;                                                     // 4 planes of P
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(&s_tmem), 256);
  if (tid == 0) {
    tc::bar_init(tc::smem_addr(&s_acc), 1);
    tc::bar_init_fence();
  }
  // operands: row r of A = column j0 + r of Tp (K = q), row r of B = row i0 + r of the panel
  for (int idx = tid; idx < RW_T * RW_K; idx += 256) {
    const int r = idx / RW_K, q = idx - r * RW_K;
    const int e = tc::kmajor_index(r, q, RW_K);
    const int j = j0 + r, i = i0 + r;
    const c32 t = (j < b && q < w) ? Tp[(long long)q * ldw + j] : mk<float>(0.f, 0.f);
    const c32 pv = (i < b && q < w) ? W[(long long)i * ldw + p0 + q] : mk<float>(0.f, 0.f);
    float h, l;
    tc::split_tf32(t.x, h, l);  A[e] = h; A[RW_PLANE + e] = l;
    tc::split_tf32(t.y, h, l);  A[2 * RW_PLANE + e] = h; A[3 * RW_PLANE + e] = l;
    tc::split_tf32(pv.x, h, l); B[e] = h; B[RW_PLANE + e] = l;
    tc::split_tf32(pv.y, h, l); B[2 * RW_PLANE + e] = h; B[3 * RW_PLANE + e] = l;
  }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = s_tmem;
  if (tid == 0) {
    constexpr uint32_t ID = tc::idesc_tf32(RW_T, RW_T, false);
    constexpr uint32_t IDN = tc::idesc_tf32(RW_T, RW_T, true);
    const uint32_t accR = tmem, accI = tmem + RW_T;
    const uint32_t LBO = 128, SBO = (RW_K / 4) * 128;
    const uint32_t a0 = base, b0 = base + 4 * RW_PLANE * 4;
#pragma unroll
    for (int ks = 0; ks < RW_K / 8; ++ks) {
      const uint32_t ko = (uint32_t)ks * 2 * 128;   // two core matrices along K per step of 8
      const uint64_t Arh = tc::sdesc(a0 + ko, LBO, SBO), Arl = tc::sdesc(a0 + RW_PLANE * 4 + ko, LBO, SBO);
      const uint64_t Aih = tc::sdesc(a0 + 2 * RW_PLANE * 4 + ko, LBO, SBO), Ail = tc::sdesc(a0 + 3 * RW_PLANE * 4 + ko, LBO, SBO);
      const uint64_t Brh = tc::sdesc(b0 + ko, LBO, SBO), Brl = tc::sdesc(b0 + RW_PLANE * 4 + ko, LBO, SBO);
      const uint64_t Bih = tc::sdesc(b0 + 2 * RW_PLANE * 4 + ko, LBO, SBO), Bil = tc::sdesc(b0 + 3 * RW_PLANE * 4 + ko, LBO, SBO);
      const uint32_t first = ks > 0 ? 1u : 0u;
      // Re: Tr Pr - Ti Pi
      tc::mma_tf32(accR, Arh, Brh, ID, first);
      tc::mma_tf32(accR, Arh, Brl, ID, 1u);
      tc::mma_tf32(accR, Arl, Brh, ID, 1u);
      tc::mma_tf32(accR, Aih, Bih, IDN, 1u);
      tc::mma_tf32(accR, Aih, Bil, IDN, 1u);
      tc::mma_tf32(accR, Ail, Bih, IDN, 1u);
      // Im: Tr Pi + Ti Pr
      tc::mma_tf32(accI, Arh, Bih, ID, first);
      tc::mma_tf32(accI, Arh, Bil, ID, 1u);
      tc::mma_tf32(accI, Arl, Bih, ID, 1u);
      tc::mma_tf32(accI, Aih, Brh, ID, 1u);
      tc::mma_tf32(accI, Aih, Brl, ID, 1u);
      tc::mma_tf32(accI, Ail, Brh, ID, 1u);
    }
    tc::mma_commit(tc::smem_addr(&s_acc));
  }
  __syncwarp();
  const bool got = tc::bar_wait(tc::smem_addr(&s_acc), 0u);
  const int bad = __syncthreads_or(!got);
  tc::fence_after();
  if (!bad) {
    // warps q4 and q4 + 4 share TMEM lane quarter q4 (columns j) and split the rows i in halves;
    // each thread holds the next 16 values of W in flight while it adds and stores the current 16
    const int q4 = warp & 3, half = warp >> 2;
    const int j = j0 + q4 * 32 + lane;
    const bool jok = j < b && (j < xlo || j >= xhi);
    const uint32_t lanebase = tmem + ((uint32_t)(q4 * 32) << 16);
    const int ib = i0 + half * (RW_T / 2);
    c32 o[16], on[16];
    auto fetch = [&](int c0, c32* dst) {
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int i = ib + c0 + e;
        dst[e] = (jok && i < b) ? W[(long long)i * ldw + j] : mk<float>(0.f, 0.f);
      }
    };
    fetch(0, on);
    for (int c0 = 0; c0 < RW_T / 2; c0 += 16) {
#pragma unroll
      for (int e = 0; e < 16; ++e) o[e] = on[e];
      if (c0 + 16 < RW_T / 2) fetch(c0 + 16, on);
      float vr[16], vi[16];
      tc::tmem_ld16(lanebase + (uint32_t)(half * (RW_T / 2) + c0), vr);
      tc::tmem_ld16(lanebase + (uint32_t)(RW_T + half * (RW_T / 2) + c0), vi);
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int i = ib + c0 + e;
        if (jok && i < b) W[(long long)i * ldw + j] = mk<float>(o[e].x + vr[e], o[e].y + vi[e]);
      }
    }
  } else if (tid == 0) {
    atomicOr(err, ERRBIT_TIMEOUT);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, 256);
}

// G_k (column-major, ld ldb) from W with the column interchanges undone
template <typename T>
__global__ void k_f3_store(int b, const cplx<T>* W, int ldw, const int* cm, cplx<T>* G, long long gofs, int ldb) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)b * ldb;
       idx += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(idx / ldb), i = (int)(idx - (long long)j * ldb);
    G[gofs + idx] = i < b ? W[(long long)i * ldw + cm[j]] : mk<T>(0, 0);
  }
}

// the column map undoing the interchanges: the swaps are sequential, so one thread applies them in
// shared memory (the maps loaded and stored by the whole CTA); dynamic shared memory 2 b ints
__global__ void k_f3_colmap(int b, const int* perm, int* cm) {
  extern __shared__ int cm_sh[];
  int* sp = cm_sh;
  int* sc = cm_sh + b;
  for (int j = threadIdx.x; j < b; j += blockDim.x) { sp[j] = perm[j]; sc[j] = j; }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int p = b - 1; p >= 0; --p) { const int q = sp[p]; const int t = sc[p]; sc[p] = sc[q]; sc[q] = t; }
  __syncthreads();
  for (int j = threadIdx.x; j < b; j += blockDim.x) cm[j] = sc[j];
}

// the update of the columns [c0, c0 + nc) alone by panel [p0, p0 + w) (the next panel's columns,
// on the look-ahead's critical path): one output per thread, W[i][j] += sum_q W[i][p0 + q] Tp[q][j]
// (the old pivot rows are zero in W, so they take their new values)
template <typename T>
__global__ void k_f3_rankw_cols(int b, int p0, int w, cplx<T>* W, int ldw, const cplx<T>* Tp, int c0, int nc) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int i = (int)(idx / nc), jj = (int)(idx - (long long)i * nc);
  if (i >= b) return;
  const int j = c0 + jj;
  cplx<T> acc = W[(long long)i * ldw + j];
  for (int q = 0; q < w; ++q) cfma(acc, W[(long long)i * ldw + p0 + q], Tp[(long long)q * ldw + j]);
  W[(long long)i * ldw + j] = acc;
}

template <typename T>
static cudaError_t factor3d_t(ddm_ctx* c, const std::vector<int>& reps) {
  cudaError_t e = cudaSuccess;
  int bmax = 0;
  for (size_t f = 0; f < reps.size(); ++f) bmax = std::max(bmax, c->fac_b[f]);
  const int ldw = bmax;
  // scratch buffers, released on every return path by stream-ordered frees on the context's
  // stream (after the launches that use them)
  struct Scratch {
    ddm_ctx* c;
    void* p[8] = {};
    int n = 0;
    explicit Scratch(ddm_ctx* cc) : c(cc) {}
    ~Scratch() {
      for (int i = 0; i < n; ++i) dev_free(c, p[i]);
    }
  } scratch(c);
  auto alloc = [&](void** ptr, size_t bytes) {
    const cudaError_t r = dev_alloc(c, ptr, bytes);
    if (r == cudaSuccess) scratch.p[scratch.n++] = *ptr;
    return r;
  };
  cplx<T>* W = nullptr;
  cplx<T>* colp = nullptr;
  int *perm = nullptr, *cm = nullptr;
  F3State* st = nullptr;
  constexpr int PW = F3Panel<T>::W;
  cplx<T>* Tp = nullptr;
  int* swl = nullptr;
  if ((e = alloc((void**)&W, sizeof(cplx<T>) * (size_t)bmax * ldw)) != cudaSuccess) return e;
  if ((e = alloc((void**)&colp, sizeof(cplx<T>) * bmax)) != cudaSuccess) return e;
  if ((e = alloc((void**)&perm, sizeof(int) * bmax)) != cudaSuccess) return e;
  if ((e = alloc((void**)&cm, sizeof(int) * bmax)) != cudaSuccess) return e;
  if ((e = alloc((void**)&st, sizeof(F3State))) != cudaSuccess) return e;
  if ((e = alloc((void**)&swl, sizeof(int) * (4 * PW + 1))) != cudaSuccess) return e;
  if ((e = alloc((void**)&Tp, sizeof(cplx<T>) * (size_t)PW * ldw)) != cudaSuccess) return e;
  // blocked when every plane block fits the cluster panel (b <= 2048); wider planes one pivot at
  // a time
  const bool blocked = bmax <= F3C_N * F3C_T;
  // the rank-16 updates of the blocked path on the tensor cores (complex64, blocks of at least 512
  // rows: narrower ones keep the CUDA-core tiles, which spread over more CTAs)
  bool rw_tc = std::is_same<T, float>::value && c->use_tc && blocked && bmax >= 512;
  if (rw_tc && (e = allow_dynamic_smem((const void*)k_f3_rankw_tc, RW_SMEM)) != cudaSuccess) return e;
  if ((e = allow_dynamic_smem((const void*)k_f3_colmap, 2 * sizeof(int) * (size_t)bmax)) != cudaSuccess) return e;
  // the second stream and its events of the look-ahead, released on every return path
  struct Side {
    cudaStream_t s = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    ~Side() {
      if (s) { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } side;
  if (blocked) {
    if ((e = cudaStreamCreateWithFlags(&side.s, cudaStreamNonBlocking)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&side.a, cudaEventDisableTiming)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&side.b, cudaEventDisableTiming)) != cudaSuccess) return e;
  }
  cudaStream_t s2 = side.s;
  cudaEvent_t evA = side.a, evB = side.b;
  // panel elimination: pivots searched among the panel's diagonal rows (threshold-checked), or
  // over all rows by the cluster kernel (tau = 0, or when a factorisation is redone)
  const bool full = c->piv_tau <= 0 || c->piv_full;
  const T tau2 = (T)(c->piv_tau * c->piv_tau);
  // panel [p, p + wn); with the restricted kernel the previous panel [pp, pp + wpp)'s update of its
  // columns is fused in (wpp = 0: none)
  auto panel = [&](int bb, int pp, int wpp, int p, int wn) {
    if (full) k_f3_panel_cl<T><<<F3C_N, F3C_T, 0, c->st>>>(bb, p, wn, W, ldw, perm, swl, c->d_err);
    else
      k_f3_panel_blk<T><<<(bb + F3B_T - 1) / F3B_T, F3B_T, 0, c->st>>>(bb, pp, wpp, Tp, p, wn, W, ldw, perm, swl, tau2,
                                                                      c->d_err);
  };
  cplx<T>* G = (cplx<T>*)c->d_G;
  for (size_t f = 0; f < reps.size(); ++f) {
    const int b = c->fac_b[f], m = c->fac_m[f], ldb = c->fac_ldb[f];
    const long long fofs = c->fac_ofs[f];
    for (int k = 0; k < m; ++k) {
      ++c->nlaunch;
      k_f3_schur<T><<<1216, 256, 0, c->st>>>(c->g, reps[f], G, fofs, ldb, k, W, ldw, cm);
      if (blocked) {
        // look-ahead: on the context's stream the interchanges of panel p (gather), the update of
        // panel p + 1's columns alone and the elimination of panel p + 1; on the second stream the
        // update of every other column by panel p, beside them (disjoint columns of W).  The next
        // gather waits for that update (it moves rows in all columns and rewrites Tp).
        const dim3 gr((b + 63) / 64, (b + 63) / 64);
        ++c->nlaunch;
        panel(b, 0, 0, 0, std::min(PW, b));
        for (int p0 = 0; p0 < b; p0 += PW) {
          const int w = std::min(PW, b - p0);
          const int p1 = p0 + w, w1 = p1 < b ? std::min(PW, b - p1) : 0;
          if (p0 > 0 && (e = cudaStreamWaitEvent(c->st, evB, 0)) != cudaSuccess) break;
          c->nlaunch += 2;
          k_f3_gather<T><<<(b + 127) / 128, 128, 0, c->st>>>(b, p0, w, W, ldw, swl, Tp);
          if ((e = cudaEventRecord(evA, c->st)) != cudaSuccess) break;
          if (w1 > 0) {
            if (full) {
              c->nlaunch += 2;
              k_f3_rankw_cols<T><<<(b * w1 + 255) / 256, 256, 0, c->st>>>(b, p0, w, W, ldw, Tp, p1, w1);
              panel(b, 0, 0, p1, w1);
            } else {
              ++c->nlaunch;
              panel(b, p0, w, p1, w1);
            }
          }
          if ((e = cudaStreamWaitEvent(s2, evA, 0)) != cudaSuccess) break;
          if (rw_tc) {
            k_f3_rankw_tc<<<dim3((b + RW_T - 1) / RW_T, (b + RW_T - 1) / RW_T), 256, RW_SMEM, s2>>>(
                b, p0, w, (c32*)W, ldw, (const c32*)Tp, p0, p1 + w1, c->d_err);
          } else {
            k_f3_rankw<T><<<gr, 256, 0, s2>>>(b, p0, w, W, ldw, Tp, 0, b, p0, p1 + w1);
          }
          if ((e = cudaEventRecord(evB, s2)) != cudaSuccess) break;
        }
        if (e != cudaSuccess) break;
        if ((e = cudaStreamWaitEvent(c->st, evB, 0)) != cudaSuccess) break;
      } else {
        // planes too wide for the cluster panel: one pivot at a time
        for (int p = 0; p < b; ++p) {
          c->nlaunch += 2;
          k_f3_pivot<T><<<1, 1024, 0, c->st>>>(b, p, W, ldw, colp, perm, st, c->d_err);
          dim3 gu((b + 127) / 128, 152);
          k_f3_update<T><<<gu, 128, 0, c->st>>>(b, p, W, ldw, colp);
        }
      }
      c->nlaunch += 2;
      k_f3_colmap<<<1, 256, 2 * sizeof(int) * b, c->st>>>(b, perm, cm);
      k_f3_store<T><<<1216, 256, 0, c->st>>>(b, W, ldw, cm, G, fofs + (long long)k * b * ldb, ldb);
      if ((e = cudaGetLastError()) != cudaSuccess) break;
    }
    if (e != cudaSuccess) break;
  }
  cudaStreamSynchronize(c->st);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

cudaError_t launch_factor3d(ddm_ctx* c, const std::vector<int>& reps) {
  return c->prec == DDM_MIXED ? factor3d_t<float>(c, reps) : factor3d_t<double>(c, reps);
}

// ---------------------------------------------------------------------------------- solve
// One plane step for the columns (subdomain, right-hand side) of one factor group:
//   forward  (pass 0): C = G_k Y,  Y[j][q] = src_q[k b + j] - c_zm(j,k) out_q[(k-1) b + j]
//                      out_q[k b + i] = C[i][q]; at k = m-1 also U_q += C
//   backward (pass 1): C = G_k Z,  Z[j][q] = c_zp(j,k) out_q[(k+1) b + j]
//                      x = out_q[k b + i] - C[i][q]; out_q = x; U_q += x
// colofs[q] = element offset of column q's local vector (lvofs of its subdomain and rhs).
constexpr int G3_BM = 64, G3_BN = 64, G3_BK = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_gemm3d(const cplx<T>* __restrict__ G, long long gofs, int ldb, int b,
                                               const cplx<T>* __restrict__ cS, const cplx<T>* __restrict__ cN,
                                               int pass, int k, int m, const long long* __restrict__ colofs, int ncol,
                                               const cplx<T>* __restrict__ src, cplx<T>* out, cplx<T>* U) {
  __shared__ cplx<T> As[G3_BK][G3_BM + 1];
  __shared__ cplx<T> Bs[G3_BK][G3_BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;            // 16 x 16 threads, 4 x 4 outputs each
  const int i0 = blockIdx.x * G3_BM, q0 = blockIdx.y * G3_BN;
  cplx<T> acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = mk<T>(0, 0);
  const cplx<T>* Gk = G + gofs + (long long)k * b * ldb;
  for (int j0 = 0; j0 < b; j0 += G3_BK) {
    // A tile: G_k[i0 .. i0+63][j0 .. j0+15] (column-major: contiguous in i)
    for (int t = tid; t < G3_BM * G3_BK; t += 256) {
      const int ii = t % G3_BM, jj = t / G3_BM;
      const int i = i0 + ii, j = j0 + jj;
      As[jj][ii] = (i < b && j < b) ? Gk[(long long)j * ldb + i] : mk<T>(0, 0);
    }
    // B tile: the block's right-hand side for columns q0 .. q0+63, rows j0 .. j0+15
    for (int t = tid; t < G3_BK * G3_BN; t += 256) {
      const int jj = t % G3_BK, qq = t / G3_BK;
      const int j = j0 + jj, q = q0 + qq;
      cplx<T> v = mk<T>(0, 0);
      if (j < b && q < ncol) {
        const long long base = colofs[q];
        if (pass == 0) {
          v = src[base + (long long)k * b + j];
          if (k > 0) v = v - cS[(long long)k * b + j] * out[base + (long long)(k - 1) * b + j];
        } else {
          v = cN[(long long)k * b + j] * out[base + (long long)(k + 1) * b + j];
        }
      }
      Bs[jj][qq] = v;
    }
    __syncthreads();
#pragma unroll
    for (int jj = 0; jj < G3_BK; ++jj) {
      cplx<T> av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[jj][ty + 16 * a];
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[c] = Bs[jj][tx + 16 * c];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) cfma(acc[a][c], av[a], bv[c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + ty + 16 * a;
    if (i >= b) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int q = q0 + tx + 16 * c;
      if (q >= ncol) continue;
      const long long o = colofs[q] + (long long)k * b + i;
      cplx<T> v = acc[a][c];
      if (pass == 1) v = out[o] - v;
      out[o] = v;
      if (U && (pass == 1 || k == m - 1)) U[o] = U[o] + v;
    }
  }
}

template <typename T>
static cudaError_t solve3d_t(ddm_ctx* c, const void* src, void* out, void* U, int nrhs) {
  // columns grouped by factor
  std::vector<std::vector<long long>> cols(c->nfac);
  std::vector<int> rep(c->nfac, -1);
  // a subdomain's right-hand sides in adjacent columns (and adjacent in memory)
  for (int s = 0; s < c->g.nsub; ++s)
    for (int r = 0; r < nrhs; ++r) {
      cols[c->subs[s].fid].push_back(lvofs(c->subs[s], r, nrhs));
      if (rep[c->subs[s].fid] < 0) rep[c->subs[s].fid] = s;
    }
  cudaError_t e = cudaSuccess;
  for (int f = 0; f < c->nfac; ++f) {
    const int ncol = (int)cols[f].size();
    if (!ncol) continue;
    if ((size_t)ncol > c->col3d_cap) {
      dev_free(c, c->d_col3d);
      c->d_col3d = nullptr;
      if ((e = dev_alloc(c, (void**)&c->d_col3d, sizeof(long long) * ncol)) != cudaSuccess) return e;
      c->col3d_cap = ncol;
    }
    if ((e = cudaMemcpyAsync(c->d_col3d, cols[f].data(), sizeof(long long) * ncol, cudaMemcpyHostToDevice, c->st)) !=
        cudaSuccess)
      return e;
    const SubDesc& s = c->subs[rep[f]];
    const int b = c->fac_b[f], m = c->fac_m[f], ldb = c->fac_ldb[f];
    const long long len = (long long)b * m;
    const int zm = 2 * c->dim - 1, zp = 2 * c->dim;   // couplings to the previous / next block
    const cplx<T>* lc = (const cplx<T>*)c->d_lcoef + s.vofs * (2 * c->dim + 1);
    if constexpr (std::is_same<T, float>::value) {
      if (c->use_tc && c->d_gtc) {
        if ((e = tc3d_sweeps(c, f, c->d_col3d, ncol, lc + zm * len, lc + zp * len, (const c32*)src, (c32*)out,
                             (c32*)U)) != cudaSuccess)
          return e;
        if (f + 1 < c->nfac) cudaStreamSynchronize(c->st);
        continue;
      }
    }
    dim3 grid((b + G3_BM - 1) / G3_BM, (ncol + G3_BN - 1) / G3_BN);
    for (int i = 0; i < 2 * m - 1; ++i) {
      const int pass = i < m ? 0 : 1;
      const int k = pass == 0 ? i : 2 * m - 2 - i;
      ++c->nlaunch;
      k_gemm3d<T><<<grid, 256, 0, c->st>>>((const cplx<T>*)c->d_G, c->fac_ofs[f], ldb, b, lc + zm * len, lc + zp * len,
                                           pass, k, m, c->d_col3d, ncol, (const cplx<T>*)src, (cplx<T>*)out,
                                           (cplx<T>*)U);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the column list is reused by the next group: wait until these launches have read it
    if (f + 1 < c->nfac) cudaStreamSynchronize(c->st);
  }
  return cudaGetLastError();
}

cudaError_t launch_local_solve3d(ddm_ctx* c, const void* src, void* out, void* U, int nrhs) {
  return c->prec == DDM_MIXED ? solve3d_t<float>(c, src, out, U, nrhs) : solve3d_t<double>(c, src, out, U, nrhs);
}

}  // namespace ddm

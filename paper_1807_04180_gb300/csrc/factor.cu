// Factorisation of the subdomain PML operators (the local problems of Algorithm 3.1).
//
// A subdomain operator in natural ordering (x fastest) is block tridiagonal over its
// x-lines: diagonal blocks T_k (tridiagonal, x-couplings of line k) and diagonal
// off-diagonal blocks L_k = diag(c_S(., k)), U_k = diag(c_N(., k)).  Block elimination
// gives D_0 = T_0, D_k = T_k - L_k D_{k-1}^{-1} U_{k-1}; the factor stores
// G_k = D_k^{-1} (dense b x b, column-major, leading dimension ldb), inverted in shared memory
// by blocked Gauss-Jordan elimination with partial (row) pivoting inside the block.  One CTA
// per distinct factor walks the lines sequentially.
#include <algorithm>

#include "ddm_internal.cuh"

namespace ddm {

constexpr int FAC_W = 4;          // panel width of the blocked Gauss-Jordan inversion
constexpr int FAC_THREADS = 256;  // per CTA: two CTAs per SM in complex64 (registers, shared memory)

template <typename T>
__global__ void __launch_bounds__(FAC_THREADS, sizeof(T) == 4 ? 2 : 1) k_factor2d(Geom g, const int* reps, const long long* fofs_arr,
                                                  const int* ldbs, cplx<T>* Gout, int* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  const SubDesc& s = g.subs[reps[blockIdx.x]];
  const long long fofs = fofs_arr[blockIdx.x];
  const int ldb = ldbs[blockIdx.x];
  const int b = s.ext[0], m = s.ext[1];
  const int njj = (b + 31) / 32;             // 32-column groups per row
  const int ldm = 32 * njj + 1;              // padded, odd: whole lane groups, conflict-free columns
  cplx<T>* M = (cplx<T>*)smem;               // b x ldm working block
  cplx<T>* Tp = M + (long long)b * ldm;      // FAC_W x ldm: old pivot rows of a panel
  cplx<T>* cC = Tp + (long long)FAC_W * ldm; // centre of line k
  cplx<T>* cE = cC + b;                      // x+ coupling
  cplx<T>* cW = cE + b;                      // x- coupling
  cplx<T>* cS = cW + b;                      // coupling of line k to line k-1
  cplx<T>* cNp = cS + b;                     // coupling of line k-1 to line k
  cplx<T>* cNn = cNp + b;
  int* perm = (int*)(cNn + b);
  int* cm = perm + b;
  __shared__ int s_bad;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
  if (tid == 0) s_bad = 0;
  for (int j = tid; j < b; j += nth) cm[j] = j;
  __syncthreads();

  for (int k = 0; k < m; ++k) {
    // coefficients of line k from the operator planes (C, W, E, S, N)
    {
      const long long len = (long long)b * m;
      const cplx<T>* lc = (const cplx<T>*)g.lcoef + s.vofs * 5 + (long long)k * b;
      for (int i = tid; i < b; i += nth) {
        cC[i] = lc[i]; cW[i] = lc[len + i]; cE[i] = lc[2 * len + i];
        cS[i] = lc[3 * len + i]; cNn[i] = lc[4 * len + i];
      }
    }
    __syncthreads();
    // D_k = T_k - L_k G_{k-1} U_{k-1}; each warp rebuilds whole rows (reading the row of
    // G_{k-1} through the column map into registers first, then overwriting it)
    for (int i = warp; i < b; i += nwarp) {
      cplx<T> v[4];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        int j = lane + 32 * jj;
        v[jj] = (k > 0 && j < b) ? M[i * ldm + cm[j]] : mk<T>(0, 0);
      }
      __syncwarp();
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        int j = lane + 32 * jj;
        if (j < b) {
          cplx<T> d = mk<T>(0, 0);
          if (k > 0) d = -(cS[i] * v[jj] * cNp[j]);
          if (j == i) d = d + cC[i];
          if (j == i + 1) d = d + cE[i];
          if (j == i - 1) d = d + cW[i];
          M[i * ldm + j] = d;
        }
      }
    }
    __syncthreads();
    for (int j = tid; j < b; j += nth) cNp[j] = cNn[j];   // read by the next line's build only

    // Gauss-Jordan inversion with partial pivoting, in place, blocked by panels of FAC_W
    // columns.  For a panel P = [p0, p0 + w): warp 0 runs the unblocked elimination on the
    // panel's columns only (pivot search over rows >= c, interchange, scaling, elimination of
    // column c from every other row), which leaves the panel holding the new column block
    // [-A_01 A_11^-1 ; A_11^-1 ; -A_21 A_11^-1] of the inverse.  The interchanges are then
    // applied to the other columns, the old pivot rows T = rows P (other columns) are kept, and
    // every other column j takes the same w elimination steps at once:
    //   rows i outside P:  M[i][j] += sum_q M[i][p0+q] T[q][j]
    //   rows of P:         M[p0+q'][j] = sum_q M[p0+q'][p0+q] T[q][j]
    // (the block Gauss-Jordan step)
    // Look-ahead: after panel p's interchanges, warp 0 applies panel p's step to the next panel's
    // columns in its registers and eliminates that panel, while the other warps apply panel p's
    // step to the remaining columns (two barriers per panel; the elimination of a panel by one
    // warp runs beside the update instead of before it).
    cplx<T> R[4][FAC_W];    // warp 0's panel: R[t][q] = M[lane + 32 t][p0 + q]
    auto eliminate = [&](const int p0, const int w) {
#pragma unroll
        for (int qc = 0; qc < FAC_W; ++qc) {
          if (qc >= w) break;
          const int c = p0 + qc;
          // pivot: largest |M[i][c]| over rows i >= c (ties to the lowest row)
          T best = (T)-1; int bi = c;
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int i = lane + 32 * t;
            if (i >= c && i < b) {
              const T a = cabs2(R[t][qc]);
              if (a > best) { best = a; bi = i; }
            }
          }
          for (int o = 16; o; o >>= 1) {
            const T ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
          }
          if (lane == 0) {
            perm[c] = bi;
            if (!(best > (T)0) || !isfinite(best)) s_bad = 1;
          }
          // rows c and bi as every lane sees them: row c's and row bi's panel values
          const int lc = c & 31, tcr = c >> 5, lr = bi & 31, trr = bi >> 5;
          cplx<T> vc[FAC_W], vr[FAC_W];
#pragma unroll
          for (int q = 0; q < FAC_W; ++q) {
            cplx<T> sc = R[0][q], sr = R[0][q];
#pragma unroll
            for (int t = 1; t < 4; ++t) {
              if (tcr == t) sc = R[t][q];
              if (trr == t) sr = R[t][q];
            }
            vc[q].x = __shfl_sync(0xffffffffu, sc.x, lc);
            vc[q].y = __shfl_sync(0xffffffffu, sc.y, lc);
            vr[q].x = __shfl_sync(0xffffffffu, sr.x, lr);
            vr[q].y = __shfl_sync(0xffffffffu, sr.y, lr);
          }
          // the interchange: row bi takes row c's values (the pivot row is written below)
          if (bi != c && lane == lr) {
#pragma unroll
            for (int t = 0; t < 4; ++t)
              if (trr == t)
#pragma unroll
                for (int q = 0; q < FAC_W; ++q) R[t][q] = vc[q];
          }
          // pivot row after the interchange, scaled; column c of the inverse
          const cplx<T> pv = vr[qc];
          const cplx<T> inv = (best > (T)0 && isfinite(best)) ? cinv(pv) : mk<T>(0, 0);
          cplx<T> rs[FAC_W];
#pragma unroll
          for (int q = 0; q < FAC_W; ++q) rs[q] = q == qc ? inv : vr[q] * inv;
          // eliminate column c from the other rows; the pivot row becomes rs
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int i = lane + 32 * t;
            if (i == c) {
#pragma unroll
              for (int q = 0; q < FAC_W; ++q) R[t][q] = rs[q];
            } else {
              const cplx<T> fi = -R[t][qc];
#pragma unroll
              for (int q = 0; q < FAC_W; ++q) {
                if (q == qc) R[t][q] = fi * inv;
                else cfma(R[t][q], fi, rs[q]);
              }
            }
          }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
          for (int q = 0; q < FAC_W; ++q) {
            const int i = lane + 32 * t;
            if (i < b && q < w) M[i * ldm + p0 + q] = R[t][q];
          }
    };
    if (warp == 0) {
      const int w = min(FAC_W, b);
#pragma unroll
      for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int q = 0; q < FAC_W; ++q) {
          const int i = lane + 32 * t;
          R[t][q] = (i < b && q < w) ? M[i * ldm + q] : mk<T>(0, 0);
        }
      eliminate(0, w);
    }
    __syncthreads();
    for (int p0 = 0; p0 < b; p0 += FAC_W) {
      const int w = min(FAC_W, b - p0);
      const int p1 = p0 + w, w1 = min(FAC_W, b - p1);   // the next panel (none when w1 <= 0)
      // the panel's interchanges on the other columns, in order, and the old pivot rows
      for (int j = tid; j < b; j += nth) {
        if (j >= p0 && j < p0 + w) continue;
        for (int c = p0; c < p0 + w; ++c) {
          const int r = perm[c];
          if (r != c) {
            const cplx<T> t0 = M[c * ldm + j];
            M[c * ldm + j] = M[r * ldm + j];
            M[r * ldm + j] = t0;
          }
        }
        for (int q = 0; q < w; ++q) Tp[q * ldm + j] = M[(p0 + q) * ldm + j];
      }
      __syncthreads();
      if (w1 > 0 && warp == 0) {
        // the next panel's columns take this panel's step (same arithmetic and order as below)
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int i = lane + 32 * t;
          const bool prow = i >= p0 && i < p0 + w;
          cplx<T> mi[FAC_W];
#pragma unroll
          for (int q = 0; q < FAC_W; ++q) mi[q] = (i < b && q < w) ? M[i * ldm + p0 + q] : mk<T>(0, 0);
#pragma unroll
          for (int q1 = 0; q1 < FAC_W; ++q1) {
            cplx<T> acc = mk<T>(0, 0);
            if (i < b && q1 < w1) {
              const int j = p1 + q1;
              acc = prow ? mk<T>(0, 0) : M[i * ldm + j];
#pragma unroll
              for (int q = 0; q < FAC_W; ++q)
                if (q < w) cfma(acc, mi[q], Tp[q * ldm + j]);
            }
            R[t][q1] = acc;
          }
        }
        eliminate(p1, w1);
      } else {
        // rank-w update of the other columns: warp per row set, lanes over columns (the pivot
        // rows' old values read from Tp, conflict-free along the lanes); the next panel's
        // columns are warp 0's
        const int busy = w1 > 0 ? 1 : 0;
        const int lo = w1 > 0 ? p1 : b, hi = w1 > 0 ? p1 + w1 : b;
        for (int i = warp - busy; i < b; i += nwarp - busy) {
          const bool prow = i >= p0 && i < p0 + w;
          cplx<T> mi[FAC_W];
#pragma unroll
          for (int q = 0; q < FAC_W; ++q) mi[q] = q < w ? M[i * ldm + p0 + q] : mk<T>(0, 0);
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int j = lane + 32 * jj;
            if (jj < njj && j < b && (j < p0 || j >= p0 + w) && (j < lo || j >= hi)) {
              cplx<T> acc = prow ? mk<T>(0, 0) : M[i * ldm + j];
#pragma unroll
              for (int q = 0; q < FAC_W; ++q)
                if (q < w) cfma(acc, mi[q], Tp[q * ldm + j]);
              M[i * ldm + j] = acc;
            }
          }
        }
      }
      __syncthreads();
    }
    // column map undoing the interchanges
    if (tid == 0) {
      for (int j = 0; j < b; ++j) cm[j] = j;
      for (int p = b - 1; p >= 0; --p) { int q = perm[p]; int t = cm[p]; cm[p] = cm[q]; cm[q] = t; }
    }
    __syncthreads();
    // write G_k transposed (column j of G_k contiguous: element (i, j) at (k b + j) ldb + i)
    for (int idx = tid; idx < b * ldb; idx += nth) {
      const int j = idx / ldb, i = idx - j * ldb;
      Gout[fofs + ((long long)k * b + j) * ldb + i] = i < b ? M[i * ldm + cm[j]] : mk<T>(0, 0);
    }
  }
  if (tid == 0 && s_bad) atomicOr(err, ERRBIT_SINGULAR);
}

// ---------------------------------------------------------------------------------------------
// complex64 factorisation with the Schur block held in registers.
//
// Same recurrence and output as k_factor2d.  Each D_k is inverted by Gauss-Jordan with partial
// (row) pivoting, the pivots applied implicitly: the pivot of step c is the unpivoted row r_c of
// largest |D[r][c]|, rows are never moved, and after the last step the stored matrix M satisfies
// D^{-1}[i][l] = M[r_i][c(l)] with c(l) the step whose pivot row is l.  Layout: warp w holds
// columns [8w, 8w + 8) of all rows in registers, lane l the rows l + 32 t, t < RL.  The columns are
// eliminated in panels of 8 (one warp's strip).  The owner of panel P eliminates it alone, in its
// registers: pivot search by warp shuffles on a key that packs |D|^2 (low mantissa bits dropped)
// with the row, the pivot row broadcast by shuffles.  It then publishes the panel's new columns X
// (the block Gauss-Jordan multipliers) and pivot rows.  Every other warp applies the step to its
// own columns as one rank-8 update,
//     M[i][j] = [i not a pivot row of P] M[i][j] + sum_q X[i][q] T[q][j],
// T[q][j] being the old value of pivot row r_q in column j.  T comes from the warp's own strip,
// mirrored in shared memory once per panel.  Look-ahead: the owner of panel P + 1 first applies
// panel P's update to its strip (alone, so that it is not slowed by the others), signals the
// other warps on a named barrier and eliminates panel P + 1 while they apply panel P; one CTA
// barrier per panel.  The elimination of a panel is one block of straight-line code per pivot
// (the pivot search is one warp max-reduction of the packed key), since this chain of 8 pivots
// per panel bounds the kernel.  At the end of a line the strips go to shared memory.  The
// permuted inverse is then written to global memory (column-major, as k_factor2d) and read back
// for the next line's Schur complement.
template <int RL, int NW = 4 * RL, int CW = 8>
struct FacRG {
  static constexpr int ROWS = 32 * RL;        // rows held
  static constexpr int LDC = ROWS + 2;        // row stride of the shared mirror (== 2 mod 16)
  static constexpr int NWARP = NW;            // column strips of CW: b <= CW NW
  static constexpr int THREADS = 32 * NWARP;
  static size_t smem() {
    return sizeof(c32) * ((size_t)ROWS * LDC + 2 * CW * ROWS + 6 * ROWS) + 2 * sizeof(int) * ROWS;
  }
};

// Eliminate the columns of panel pe held in R (rows lane + 32 t) with the rows flagged in pm
// excluded from the pivot search; writes the panel's new columns to X (column-major, ROWS per
// column) and its pivot rows to piv[8 pe + q].  W = 8 for a full panel (the loop is one block of
// straight-line code: no branch between the pivot steps); W = 0 takes the width from b.
template <int RL, int CW, int W>
__device__ __forceinline__ void rg_eliminate(c32 (&R)[RL][CW], unsigned pm, const int pe, const int b, const int lane,
                                             c32* X, int* piv, int* s_bad) {
  constexpr int ROWS = FacRG<RL>::ROWS;
  const int w = W ? W : min(CW, b - CW * pe);
  bool bad = false;
  int rsel = 0;
#pragma unroll
  for (int q = 0; q < CW; ++q) {
    if (!W && q >= w) break;
    // pivot: the unpivoted row of largest |M[r][c]|^2 (ties to the lowest row)
    unsigned key = 0u;
#pragma unroll
    for (int t = 0; t < RL; ++t) {
      const int i = lane + 32 * t;
      const unsigned kk = (__float_as_uint(cabs2(R[t][q])) & 0xFFFFFF00u) | (unsigned)(255 - i);
      key = (i < b && !((pm >> t) & 1u)) ? max(key, kk) : key;
    }
    key = __reduce_max_sync(0xffffffffu, key);
    const int r = key ? 255 - (int)(key & 0xFFu) : 0;
    const int tr = r >> 5, lr = r & 31;
    c32 sv[CW];
#pragma unroll
    for (int jo = 0; jo < CW; ++jo) {
      const int jj = (q + jo) & (CW - 1);
      c32 v = R[0][jj];
#pragma unroll
      for (int t = 1; t < RL; ++t) v = tr == t ? R[t][jj] : v;
      sv[jj].x = __shfl_sync(0xffffffffu, v.x, lr);
      sv[jj].y = __shfl_sync(0xffffffffu, v.y, lr);
    }
    const float pa = cabs2(sv[q]);
    const bool ok = key != 0u && pa > 0.f && isfinite(pa);
    bad = bad || !ok;
    const float rd = ok ? __frcp_rn(pa) : 0.f;
    const c32 inv = mk<float>(sv[q].x * rd, -sv[q].y * rd);
#pragma unroll
    for (int jj = 0; jj < CW; ++jj) sv[jj] = jj == q ? inv : sv[jj] * inv;
    c32 nf[RL];
#pragma unroll
    for (int t = 0; t < RL; ++t) nf[t] = lane + 32 * t == r ? mk<float>(1.f, 0.f) : -R[t][q];
#pragma unroll
    for (int jo = 1; jo <= CW; ++jo) {
      const int jj = (q + jo) & (CW - 1);
#pragma unroll
      for (int t = 0; t < RL; ++t) {
        const bool isr = lane + 32 * t == r;
        c32 base = (isr || jj == q) ? mk<float>(0.f, 0.f) : R[t][jj];
        cfma(base, nf[t], sv[jj]);
        R[t][jj] = base;
      }
    }
    pm |= lane == lr ? 1u << tr : 0u;
    rsel = lane == q ? r : rsel;
  }
  if (lane < w) piv[CW * pe + lane] = rsel;
  if (bad && lane == 0) *s_bad = 1;
#pragma unroll
  for (int t = 0; t < RL; ++t)
#pragma unroll
    for (int q = 0; q < CW; ++q) X[q * ROWS + lane + 32 * t] = R[t][q];
}

template <int RL, int CW>
__device__ __forceinline__ void rg_eliminate_any(c32 (&R)[RL][CW], unsigned pm, const int pe, const int b,
                                                 const int lane, c32* X, int* piv, int* s_bad) {
  if (CW * pe + CW <= b) rg_eliminate<RL, CW, CW>(R, pm, pe, b, lane, X, piv, s_bad);
  else rg_eliminate<RL, CW, 0>(R, pm, pe, b, lane, X, piv, s_bad);
}

template <int RL, int NW, int CW>
__global__ void __launch_bounds__(FacRG<RL, NW, CW>::THREADS, RL == 3 ? 2 : 1)
    k_factor2d_rg(Geom g, const int* fsel, int fsel_ofs, const int* reps, const long long* fofs_arr, const int* ldbs,
                  c32* Gout, int* err) {
  constexpr int ROWS = FacRG<RL, NW, CW>::ROWS, LDC = FacRG<RL, NW, CW>::LDC;
  extern __shared__ __align__(16) unsigned char smem[];
  c32* Mst = (c32*)smem;                 // ROWS x LDC mirror of the strips (row-major)
  c32* Xb = Mst + ROWS * LDC;            // 2 x (CW columns x ROWS): published panel columns
  c32* cC = Xb + 2 * CW * ROWS;          // centre of line k
  c32* cE = cC + ROWS;                   // x+ coupling
  c32* cW = cE + ROWS;                   // x- coupling
  c32* cS = cW + ROWS;                   // coupling of line k to line k-1
  c32* cNn = cS + ROWS;                  // coupling of line k to line k+1
  c32* cNp = cNn + ROWS;                 // coupling of line k-1 to line k
  int* piv = (int*)(cNp + ROWS);         // pivot row of each elimination step
  int* rinv = piv + ROWS;                // step whose pivot row is l
  __shared__ int s_bad;
  const int f = fsel[fsel_ofs + blockIdx.x];
  const SubDesc& sd = g.subs[reps[f]];
  const long long fofs = fofs_arr[f];
  const int ldb = ldbs[f];
  const int b = sd.ext[0], m = sd.ext[1];
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int npan = (b + CW - 1) / CW;
  const int col0 = CW * warp;
  const bool has_cols = col0 < b;
  if (tid == 0) s_bad = 0;
  c32 R[RL][CW];
  for (int k = 0; k <= m; ++k) {
    if (k < m) {
      const long long len = (long long)b * m;
      const c32* lc = (const c32*)g.lcoef + sd.vofs * 5 + (long long)k * b;
      for (int i = tid; i < ROWS; i += nth) {
        const bool v = i < b;
        const c32 z = mk<float>(0.f, 0.f);
        cC[i] = v ? lc[i] : z;
        cW[i] = v ? lc[len + i] : z;
        cE[i] = v ? lc[2 * len + i] : z;
        cS[i] = v ? lc[3 * len + i] : z;
        cNn[i] = v ? lc[4 * len + i] : z;
      }
    }
    __syncthreads();   // line k's couplings; line k-1's final strips, pivots and rinv
    if (k > 0) {       // G_(k-1)[i][j] = M[r_i][rinv[j]], column j contiguous
      c32* Gk = Gout + fofs + (long long)(k - 1) * b * ldb;
      for (int j = warp; j < b; j += nth >> 5) {
        const int cj = rinv[j];
        for (int i = lane; i < ldb; i += 32)
          Gk[(long long)j * ldb + i] = i < b ? Mst[piv[i] * LDC + cj] : mk<float>(0.f, 0.f);
      }
    }
    if (k == m) break;
    // D_k = T_k - L_k G_(k-1) U_(k-1) into the registers of this warp's strip
#pragma unroll
    for (int t = 0; t < RL; ++t) {
      const int i = lane + 32 * t;
#pragma unroll
      for (int jj = 0; jj < CW; ++jj) {
        const int j = col0 + jj;
        c32 d = mk<float>(0.f, 0.f);
        if (i < b && j < b) {
          if (k > 0) d = -(cS[i] * Mst[piv[i] * LDC + rinv[j]] * cNp[j]);
          if (j == i) d = d + cC[i];
          if (j == i + 1) d = d + cE[i];
          if (j == i - 1) d = d + cW[i];
        }
        R[t][jj] = d;
      }
    }
    unsigned pmask = 0u;
    __syncthreads();   // everyone has read line k-1's mirror, pivots and couplings
    for (int i = tid; i < ROWS; i += nth) cNp[i] = cNn[i];
    if (warp == 0) rg_eliminate_any<RL, CW>(R, 0u, 0, b, lane, Xb, piv, &s_bad);
    __syncthreads();
    for (int P = 0; P < npan; ++P) {
      const int w = min(CW, b - CW * P);
      const c32* X = Xb + (P & 1) * CW * ROWS;
      // the panel's pivot rows leave the search
      int rq[CW];
#pragma unroll
      for (int q = 0; q < CW; ++q) rq[q] = q < w ? piv[CW * P + q] : piv[CW * P];
      const unsigned before = pmask;
#pragma unroll
      for (int q = 0; q < CW; ++q) pmask |= (q < w && (rq[q] & 31) == lane) ? 1u << (rq[q] >> 5) : 0u;
      const unsigned fresh = pmask & ~before;
      // the owner of the next panel updates its strip first, then signals (named barrier 1) and
      // eliminates; the other warps update theirs after the signal, beside the elimination
      const bool ahead = P + 1 < npan;
      const bool owner_next = ahead && warp == P + 1;
      if (ahead && !owner_next) asm volatile("bar.sync 1, %0;" ::"r"(nth) : "memory");
      if (warp != P && has_cols) {
        // old values of this strip (the T rows) through the warp's part of the mirror
        c32* my = Mst + col0;
#pragma unroll
        for (int t = 0; t < RL; ++t) {
          float4* dst = (float4*)(my + (lane + 32 * t) * LDC);
#pragma unroll
          for (int h = 0; h < CW / 2; ++h) dst[h] = make_float4(R[t][2 * h].x, R[t][2 * h].y, R[t][2 * h + 1].x, R[t][2 * h + 1].y);
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < RL; ++t)
#pragma unroll
          for (int jj = 0; jj < CW; ++jj) R[t][jj] = ((fresh >> t) & 1u) ? mk<float>(0.f, 0.f) : R[t][jj];
#pragma unroll
        for (int q = 0; q < CW; ++q) {
          // q >= w (a partial last panel): X[q] is zero there, the product adds nothing
          const float4* src = (const float4*)(my + rq[q] * LDC);
          c32 T[CW];
#pragma unroll
          for (int h = 0; h < CW / 2; ++h) {
            const float4 v = src[h];
            T[2 * h] = mk<float>(v.x, v.y);
            T[2 * h + 1] = mk<float>(v.z, v.w);
          }
#pragma unroll
          for (int t = 0; t < RL; ++t) {
            const c32 xv = X[q * ROWS + lane + 32 * t];
#pragma unroll
            for (int jj = 0; jj < CW; ++jj) cfma(R[t][jj], xv, T[jj]);
          }
        }
        __syncwarp();
      }
      if (owner_next) {
        asm volatile("bar.arrive 1, %0;" ::"r"(nth) : "memory");
        rg_eliminate_any<RL, CW>(R, pmask, P + 1, b, lane, Xb + ((P + 1) & 1) * CW * ROWS, piv, &s_bad);
      }
      __syncthreads();
    }
    // final strips to the mirror, and the inverse pivot map
    if (has_cols) {
      c32* my = Mst + col0;
#pragma unroll
      for (int t = 0; t < RL; ++t) {
        float4* dst = (float4*)(my + (lane + 32 * t) * LDC);
#pragma unroll
        for (int h = 0; h < CW / 2; ++h) dst[h] = make_float4(R[t][2 * h].x, R[t][2 * h].y, R[t][2 * h + 1].x, R[t][2 * h + 1].y);
      }
    }
    for (int c = tid; c < b; c += nth) rinv[piv[c]] = c;
  }
  if (tid == 0 && s_bad) atomicOr(err, ERRBIT_SINGULAR);
}

size_t factor_smem_bytes(int b, int ldb, int prec) {
  size_t el = prec == DDM_MIXED ? sizeof(c32) : sizeof(z64);
  (void)ldb;
  return (size_t)(b + FAC_W) * (32 * ((b + 31) / 32) + 1) * el + 6 * (size_t)b * el + 2 * (size_t)b * sizeof(int) + 64;
}

// All distinct factors, one CTA each.  d_reps[f] is a subdomain using factor f, d_fofs[f] /
// d_ldb[f] its storage offset and leading dimension.  complex64: the register-resident kernel,
// one launch per block-width class (b <= 96: 12 warps, two CTAs per SM; b <= 128: 16 warps);
// complex128: k_factor2d.
template <int RL, int NW, int CW>
static cudaError_t launch_rg(ddm_ctx* c, int n, int ofs, const int* d_reps, const long long* d_fofs, const int* d_ldb) {
  if (n <= 0) return cudaSuccess;
  using F = FacRG<RL, NW, CW>;
  cudaError_t e = allow_dynamic_smem((const void*)k_factor2d_rg<RL, NW, CW>, F::smem());
  if (e != cudaSuccess) return e;
  ++c->nlaunch;
  k_factor2d_rg<RL, NW, CW><<<n, F::THREADS, F::smem(), c->st>>>(c->g, c->d_fsel, ofs, d_reps, d_fofs, d_ldb,
                                                                   (c32*)c->d_G, c->d_err);
  return cudaGetLastError();
}

cudaError_t launch_factor_all(ddm_ctx* c, const int* d_reps, const long long* d_fofs, const int* d_ldb) {
  cudaError_t e;
  if (c->prec == DDM_MIXED) {
    // width classes: b <= 96 (12 warps, two CTAs per SM), b <= 128 (16 warps, one CTA per SM)
    std::vector<int> sel;
    int cnt[2] = {0, 0};
    for (int k = 0; k < 2; ++k)
      for (int f = 0; f < c->nfac; ++f)
        if ((c->fac_b[f] > 96) == (k == 1)) { sel.push_back(f); ++cnt[k]; }
    if ((e = cudaMemcpyAsync(c->d_fsel, sel.data(), sizeof(int) * sel.size(), cudaMemcpyHostToDevice, c->st)) !=
        cudaSuccess)
      return e;
    if ((e = launch_rg<3, 12, 8>(c, cnt[0], 0, d_reps, d_fofs, d_ldb)) != cudaSuccess) return e;
    return launch_rg<4, 16, 8>(c, cnt[1], cnt[0], d_reps, d_fofs, d_ldb);
  }
  size_t sm = 0;
  for (int f = 0; f < c->nfac; ++f) sm = std::max(sm, factor_smem_bytes(c->fac_b[f], c->fac_ldb[f], c->prec));
  e = allow_dynamic_smem((const void*)k_factor2d<double>, sm);
  if (e != cudaSuccess) return e;
  ++c->nlaunch;
  k_factor2d<double><<<c->nfac, FAC_THREADS, sm, c->st>>>(c->g, d_reps, d_fofs, d_ldb, (z64*)c->d_G, c->d_err);
  return cudaGetLastError();
}

}  // namespace ddm

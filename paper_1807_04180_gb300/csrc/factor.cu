// Factorisation of the subdomain PML operators (the local problems of Algorithm 3.1).
//
// A subdomain operator in natural ordering (x fastest) is block tridiagonal over its
// x-lines: diagonal blocks T_k (tridiagonal, x-couplings of line k) and diagonal
// off-diagonal blocks L_k = diag(c_S(., k)), U_k = diag(c_N(., k)).  Block elimination
// gives D_0 = T_0, D_k = T_k - L_k D_{k-1}^{-1} U_{k-1}; the factor stores
// G_k = D_k^{-1} (dense b x b, column-major, leading dimension ldb), inverted in shared memory
// by Gauss-Jordan elimination with partial (row) pivoting inside the block.  One CTA per
// distinct factor walks the lines sequentially.
#include <algorithm>

#include "ddm_internal.cuh"

namespace ddm {

template <typename T>
__global__ void __launch_bounds__(512) k_factor2d(Geom g, const int* reps, const long long* fofs_arr,
                                                  const int* ldbs, cplx<T>* Gout, int* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  const SubDesc& s = g.subs[reps[blockIdx.x]];
  const long long fofs = fofs_arr[blockIdx.x];
  const int ldb = ldbs[blockIdx.x];
  const int b = s.ext[0], m = s.ext[1];
  const int njj = (b + 31) / 32;             // 32-column groups per row
  const int ldm = 32 * njj + 1;              // padded, odd: whole lane groups, conflict-free columns
  cplx<T>* M = (cplx<T>*)smem;               // b x ldm working block
  cplx<T>* colp = M + (long long)b * ldm;    // column p multipliers
  cplx<T>* cC = colp + b;                    // centre of line k
  cplx<T>* cE = cC + b;                      // x+ coupling
  cplx<T>* cW = cE + b;                      // x- coupling
  cplx<T>* cS = cW + b;                      // coupling of line k to line k-1
  cplx<T>* cNp = cS + b;                     // coupling of line k-1 to line k
  cplx<T>* cNn = cNp + b;
  int* perm = (int*)(cNn + b);
  int* cm = perm + b;
  __shared__ int s_piv, s_bad;
  __shared__ cplx<T> s_inv, s_app;
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

    // Gauss-Jordan inversion with partial pivoting, in place
    for (int p = 0; p < b; ++p) {
      if (warp == 0) {
        T best = (T)-1; int bi = p;
        for (int i = p + lane; i < b; i += 32) {
          T a = cabs2(M[i * ldm + p]);
          if (a > best) { best = a; bi = i; }
        }
        for (int o = 16; o; o >>= 1) {
          T ob = __shfl_xor_sync(0xffffffffu, best, o);
          int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) {
          s_piv = bi;
          s_app = M[p * ldm + p];
          cplx<T> pv = M[bi * ldm + p];
          if (!(best > (T)0) || !isfinite(best)) { s_bad = 1; s_inv = mk<T>(0, 0); }
          else s_inv = cinv(pv);
          perm[p] = bi;
        }
      }
      __syncthreads();
      const int r = s_piv;
      const cplx<T> inv = s_inv;
      // interchange rows p and r, scale the pivot row, keep the multipliers of column p and
      // clear column p in the other rows (their final entry there, -f_i / pivot, comes out of
      // the update below).  Thread j alone reads and writes M[p][j], M[r][j] and M[j][p]; the
      // old M[p][p], needed as row r's multiplier, was saved by the pivot search.
      if (tid < b) {
        const int j = tid;
        const cplx<T> ap = M[p * ldm + j];
        const cplx<T> ar = M[r * ldm + j];
        colp[j] = (j == p) ? mk<T>(0, 0) : (j == r ? s_app : M[j * ldm + p]);
        M[p * ldm + j] = (j == p) ? inv : ar * inv;
        if (r != p) M[r * ldm + j] = (j == p) ? mk<T>(0, 0) : ap;
        if (j != p && j != r) M[j * ldm + p] = mk<T>(0, 0);
      }
      __syncthreads();
      // eliminate column p from every other row (warp per row set, lanes over columns, the
      // pivot row in registers, zero in the padding columns so those stay inert)
      {
        cplx<T> mp[4];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          int j = lane + 32 * jj;
          mp[jj] = j < b ? M[p * ldm + j] : mk<T>(0, 0);
        }
        for (int i = warp; i < b; i += nwarp) {
          if (i == p) continue;
          const cplx<T> f = -colp[i];
          cplx<T>* Mi = M + i * ldm + lane;
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            if (jj < njj) {
              cplx<T> cur = Mi[32 * jj];
              cfma(cur, f, mp[jj]);
              Mi[32 * jj] = cur;
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

size_t factor_smem_bytes(int b, int ldb, int prec) {
  size_t el = prec == DDM_MIXED ? sizeof(c32) : sizeof(z64);
  (void)ldb;
  return (size_t)b * (32 * ((b + 31) / 32) + 1) * el + 7 * (size_t)b * el + 2 * (size_t)b * sizeof(int) + 64;
}

// All distinct factors in one launch, one CTA each.  d_reps[f] is a subdomain using factor
// f, d_fofs[f] / d_ldb[f] its storage offset and leading dimension.
cudaError_t launch_factor_all(ddm_ctx* c, const int* d_reps, const long long* d_fofs, const int* d_ldb) {
  size_t sm = 0;
  for (int f = 0; f < c->nfac; ++f) sm = std::max(sm, factor_smem_bytes(c->fac_b[f], c->fac_ldb[f], c->prec));
  cudaError_t e;
  if (c->prec == DDM_MIXED) {
    e = allow_dynamic_smem((const void*)k_factor2d<float>, sm);
    if (e != cudaSuccess) return e;
    ++c->nlaunch;
    k_factor2d<float><<<c->nfac, 512, sm, c->st>>>(c->g, d_reps, d_fofs, d_ldb, (c32*)c->d_G, c->d_err);
  } else {
    e = allow_dynamic_smem((const void*)k_factor2d<double>, sm);
    if (e != cudaSuccess) return e;
    ++c->nlaunch;
    k_factor2d<double><<<c->nfac, 512, sm, c->st>>>(c->g, d_reps, d_fofs, d_ldb, (z64*)c->d_G, c->d_err);
  }
  return cudaGetLastError();
}

}  // namespace ddm

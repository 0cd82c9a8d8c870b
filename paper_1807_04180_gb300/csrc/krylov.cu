// Global FP64 operator (the truncated problem of Section 3.1), reductions and the
// Arnoldi / Givens building blocks of flexible GMRES (Section 4.2.2).
#include "ddm_internal.cuh"

namespace ddm {

// y = A x, or y = bsub - A x when bsub != nullptr (global grid, FP64).
__global__ void k_global_apply(Geom g, const z64* x, z64* y, const z64* bsub, int nrhs) {
  long long n = g.nglob;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n * nrhs; i += (long long)gridDim.x * blockDim.x) {
    long long gi = i % n;
    long long base = i - gi;
    int xg[3] = {(int)(gi % g.N[0]), (int)((gi / g.N[0]) % g.N[1]), (int)(gi / ((long long)g.N[0] * g.N[1]))};
    z64 acc = mk<double>(0, 0);
    cfma(acc, g.gcoef[gi], x[i]);
    long long stride = 1;
    for (int a = 0; a < g.dim; ++a) {
      if (xg[a] + 1 < g.N[a]) cfma(acc, g.gcoef[(2 + 2 * a) * n + gi], x[base + gi + stride]);
      if (xg[a] > 0) cfma(acc, g.gcoef[(1 + 2 * a) * n + gi], x[base + gi - stride]);
      stride *= g.N[a];
    }
    y[i] = bsub ? bsub[i] - acc : acc;
  }
}

cudaError_t launch_global_apply(ddm_ctx* c, const z64* x, z64* y, const z64* bsub, int nrhs) {
  ++c->nlaunch;
  k_global_apply<<<1216, 256, 0, c->st>>>(c->g, x, y, bsub, nrhs);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// block-level reduction helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  return t;   // valid in thread 0
}

// part[blk * nvec + v] = sum |x_v|^2 over this block's share (nvec vectors of length n)
__global__ void k_norm2_partial(const z64* x, long long n, int nvec, double* part) {
  __shared__ double sh[32];
  for (int v = 0; v < nvec; ++v) {
    double s = 0;
    const z64* xv = x + (long long)v * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
      s += cabs2(xv[i]);
    double t = block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x * nvec + v] = t;
  }
}

constexpr int RED_BLOCKS = 304;   // 2 x 152 SMs

cudaError_t launch_norm2_partial(ddm_ctx* c, const z64* x, long long n, int nvec, double* part, int* nblocks) {
  ++c->nlaunch;
  k_norm2_partial<<<RED_BLOCKS, 256, 0, c->st>>>(x, n, nvec, part);
  *nblocks = RED_BLOCKS;
  return cudaGetLastError();
}

// out[v] = sum_b part[b * nvals + v]  (one block per value)
__global__ void k_sum_partials(const double* part, int nblocks, int nvals, double* out) {
  __shared__ double sh[32];
  int v = blockIdx.x;
  double s = 0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += part[(long long)b * nvals + v];
  double t = block_sum(s, sh);
  if (threadIdx.x == 0) out[v] = t;
}

cudaError_t launch_sum_partials(ddm_ctx* c, const double* part, int nblocks, int nvals, double* out) {
  ++c->nlaunch;
  k_sum_partials<<<nvals, 256, 0, c->st>>>(part, nblocks, nvals, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Classical Gram-Schmidt pieces.  dots: part[(blk * nv + v) * 2 + {0,1}] = partial of
// sum_i conj(V_v[i]) w[i] for v < nv (vectors of V are contiguous, stride n).
// ---------------------------------------------------------------------------
template <int NV>
__global__ void k_dots(const z64* V, int nv0, int nv, const z64* w, long long n, double* part, int nvtot) {
  __shared__ double sh[32];
  z64 acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = mk<double>(0, 0);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    z64 wi = w[i];
#pragma unroll
    for (int v = 0; v < NV; ++v)
      if (v < nv) cfma_conj(acc[v], V[(long long)(nv0 + v) * n + i], wi);
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    if (v >= nv) break;
    double re = block_sum(acc[v].x, sh);
    if (threadIdx.x == 0) part[((long long)blockIdx.x * nvtot + nv0 + v) * 2] = re;
    double im = block_sum(acc[v].y, sh);
    if (threadIdx.x == 0) part[((long long)blockIdx.x * nvtot + nv0 + v) * 2 + 1] = im;
  }
}

cudaError_t launch_dots(ddm_ctx* c, const z64* V, int nv, const z64* w, long long n, double* part, int* nblocks) {
  for (int v0 = 0; v0 < nv; v0 += 8) {
    int cnt = min(8, nv - v0);
    ++c->nlaunch;
    k_dots<8><<<RED_BLOCKS, 256, 0, c->st>>>(V, v0, cnt, w, n, part, nv);
  }
  *nblocks = RED_BLOCKS;
  return cudaGetLastError();
}

// coef[v] = sum over blocks; Hcol[v] += coef[v] (first pass: Hcol[v] = coef[v])
__global__ void k_arnoldi_coef(const double* part, int nblocks, int nv, z64* Hcol, z64* coef, int first) {
  __shared__ double sh[32];
  int v = blockIdx.x;
  double re = 0, im = 0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    re += part[((long long)b * nv + v) * 2];
    im += part[((long long)b * nv + v) * 2 + 1];
  }
  double tr = block_sum(re, sh);
  double ti = block_sum(im, sh);
  if (threadIdx.x == 0) {
    z64 cv = mk<double>(tr, ti);
    coef[v] = cv;
    Hcol[v] = first ? cv : Hcol[v] + cv;
  }
}

cudaError_t launch_arnoldi_coef(ddm_ctx* c, const double* part, int nblocks, int nv, z64* Hcol, z64* coef, int first) {
  ++c->nlaunch;
  k_arnoldi_coef<<<nv, 256, 0, c->st>>>(part, nblocks, nv, Hcol, coef, first);
  return cudaGetLastError();
}

// w -= sum_v coef[v] V_v
__global__ void k_sub_axpy(const z64* V, int nv, const z64* coef, z64* w, long long n) {
  __shared__ z64 cs[128];
  for (int v = threadIdx.x; v < nv; v += blockDim.x) cs[v] = coef[v];
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    z64 acc = w[i];
    for (int v = 0; v < nv; ++v) {
      z64 a = V[(long long)v * n + i];
      cfma(acc, -cs[v], a);
    }
    w[i] = acc;
  }
}

cudaError_t launch_sub_axpy(ddm_ctx* c, const z64* V, int nv, const z64* coef, z64* w, long long n) {
  ++c->nlaunch;
  k_sub_axpy<<<RED_BLOCKS * 2, 256, 0, c->st>>>(V, nv, coef, w, n);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Givens step (single thread).  H column-major (m+1) x m; gs = [cs(m) | sn(m) | g(m+1) | inv]
// nrm2 = ||w||^2 after orthogonalisation.  Applies earlier rotations to column j, builds
// rotation j, updates g, stores |g_{j+1}| in out_est and 1 / H[j+1,j] in gs[3m+1].
// ---------------------------------------------------------------------------
__global__ void k_givens(int j, int m, const double* nrm2, z64* H, z64* gs, double* out_est) {
  z64* cs = gs;
  z64* sn = gs + m;
  z64* gg = gs + 2 * m;
  z64* col = H + (long long)j * (m + 1);
  double hn = sqrt(nrm2[0]);
  col[j + 1] = mk<double>(hn, 0.0);
  gs[3 * m + 1] = mk<double>(hn > 0 ? 1.0 / hn : 0.0, 0.0);
  for (int i = 0; i < j; ++i) {
    z64 a = col[i], b = col[i + 1];
    z64 snc = mk<double>(sn[i].x, -sn[i].y);
    col[i] = cs[i] * a + sn[i] * b;
    col[i + 1] = cs[i] * b - snc * a;
  }
  z64 a = col[j], b = col[j + 1];
  double aa = sqrt(cabs2(a)), bb = sqrt(cabs2(b));
  double den = sqrt(aa * aa + bb * bb);
  z64 c, s;
  if (den == 0.0) { c = mk<double>(1, 0); s = mk<double>(0, 0); }
  else if (aa == 0.0) { c = mk<double>(0, 0); s = mk<double>(b.x / bb, -b.y / bb); }
  else {
    c = mk<double>(aa / den, 0.0);
    z64 ph = mk<double>(a.x / aa, a.y / aa);
    s = (1.0 / den) * (ph * mk<double>(b.x, -b.y));
  }
  cs[j] = c; sn[j] = s;
  col[j] = c * a + s * b;
  col[j + 1] = mk<double>(0, 0);
  z64 gj = gg[j];
  gg[j + 1] = -(mk<double>(s.x, -s.y) * gj);
  gg[j] = c * gj;
  out_est[0] = sqrt(cabs2(gg[j + 1]));
}

cudaError_t launch_givens(ddm_ctx* c, int j, int m, const double* nrm2, z64* H, z64* gs, double* out_est) {
  ++c->nlaunch;
  k_givens<<<1, 1, 0, c->st>>>(j, m, nrm2, H, gs, out_est);
  return cudaGetLastError();
}

// dst = x * s  where s = *sp (device scalar, complex)
__global__ void k_scale_dev(const z64* x, const z64* sp, z64* dst, long long n) {
  z64 s = *sp;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = s * x[i];
}

cudaError_t launch_scale(ddm_ctx* c, const z64* x, const z64* s, z64* dst, long long n) {
  ++c->nlaunch;
  k_scale_dev<<<1216, 256, 0, c->st>>>(x, s, dst, n);
  return cudaGetLastError();
}

__global__ void k_copy_scaled(const z64* src, double s, z64* dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = s * src[i];
}

cudaError_t launch_copy_scaled(ddm_ctx* c, const z64* src, double s, z64* dst, long long n) {
  ++c->nlaunch;
  k_copy_scaled<<<1216, 256, 0, c->st>>>(src, s, dst, n);
  return cudaGetLastError();
}

// x += s w
__global__ void k_axpy(double s, const z64* w, z64* x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = x[i] + s * w[i];
}

cudaError_t launch_axpy(ddm_ctx* c, double s, const z64* w, z64* x, long long n) {
  ++c->nlaunch;
  k_axpy<<<1216, 256, 0, c->st>>>(s, w, x, n);
  return cudaGetLastError();
}

// y = H(0:j,0:j)^{-1} g(0:j) (upper triangular, single thread), stored in gs[3m+2 ..]
__global__ void k_lsq(int j, int m, const z64* H, z64* gs) {
  const z64* gg = gs + 2 * m;
  z64* y = gs + 3 * m + 2;
  for (int i = j - 1; i >= 0; --i) {
    z64 acc = gg[i];
    for (int k = i + 1; k < j; ++k) acc = acc - H[(long long)k * (m + 1) + i] * y[k];
    y[i] = acc * cinv(H[(long long)i * (m + 1) + i]);
  }
}

// x += Z(:,0:j) y
__global__ void k_update_x(int j, int m, const z64* gs, const z64* Z, z64* x, long long n) {
  __shared__ z64 ys[128];
  for (int v = threadIdx.x; v < j; v += blockDim.x) ys[v] = gs[3 * m + 2 + v];
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    z64 acc = x[i];
    for (int v = 0; v < j; ++v) cfma(acc, ys[v], Z[(long long)v * n + i]);
    x[i] = acc;
  }
}

cudaError_t launch_lsq_update(ddm_ctx* c, int j, int m, z64* H, z64* gs, const z64* Z, z64* x, long long n) {
  ++c->nlaunch;
  k_lsq<<<1, 1, 0, c->st>>>(j, m, H, gs);
  ++c->nlaunch;
  k_update_x<<<RED_BLOCKS * 2, 256, 0, c->st>>>(j, m, gs, Z, x, n);
  return cudaGetLastError();
}

}  // namespace ddm

// ===========================================================================
// Batched variants: nb independent Krylov recurrences advanced together.  Basis vector v of
// right-hand side r is V + (v nb + r) n; right-hand side r's Hessenberg matrix is
// H + r (m+1) m (column-major), its Givens/LSQ scratch gs + r GSZ, GSZ = 5 m + 4.
// ===========================================================================
namespace ddm {

template <int NV>
__global__ void k_dots_b(const z64* V, int nb, int v0, int nv, const z64* w, long long n, double* part, int nvtot) {
  __shared__ double sh[32];
  const int r = blockIdx.z;
  const z64* wr = w + (long long)r * n;
  z64 acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = mk<double>(0, 0);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const z64 wi = wr[i];
#pragma unroll
    for (int v = 0; v < NV; ++v)
      if (v < nv) cfma_conj(acc[v], V[((long long)(v0 + v) * nb + r) * n + i], wi);
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    if (v >= nv) break;
    const double re = block_sum(acc[v].x, sh);
    const double im = block_sum(acc[v].y, sh);
    if (threadIdx.x == 0) {
      double* p = part + (((long long)r * gridDim.x + blockIdx.x) * nvtot + v0 + v) * 2;
      p[0] = re;
      p[1] = im;
    }
  }
}

cudaError_t launch_dots_b(ddm_ctx* c, const z64* V, int nb, int nv, const z64* w, long long n, double* part, int* nblocks) {
  for (int v0 = 0; v0 < nv; v0 += 8) {
    ++c->nlaunch;
    k_dots_b<8><<<dim3(RED_BLOCKS, 1, nb), 256, 0, c->st>>>(V, nb, v0, min(8, nv - v0), w, n, part, nv);
  }
  *nblocks = RED_BLOCKS;
  return cudaGetLastError();
}

__global__ void k_arnoldi_coef_b(const double* part, int nblocks, int nv, z64* H, int j, int m, z64* coef, int first) {
  __shared__ double sh[32];
  const int v = blockIdx.x, r = blockIdx.y;
  double re = 0, im = 0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    const double* p = part + (((long long)r * nblocks + b) * nv + v) * 2;
    re += p[0];
    im += p[1];
  }
  const double tr = block_sum(re, sh);
  const double ti = block_sum(im, sh);
  if (threadIdx.x == 0) {
    const z64 cv = mk<double>(tr, ti);
    coef[(long long)r * (m + 1) + v] = cv;
    z64* hc = H + (long long)r * (m + 1) * m + (long long)j * (m + 1);
    hc[v] = first ? cv : hc[v] + cv;
  }
}

cudaError_t launch_arnoldi_coef_b(ddm_ctx* c, const double* part, int nblocks, int nv, int nb, z64* H, int j, int m,
                                  z64* coef, int first) {
  ++c->nlaunch;
  k_arnoldi_coef_b<<<dim3(nv, nb), 256, 0, c->st>>>(part, nblocks, nv, H, j, m, coef, first);
  return cudaGetLastError();
}

__global__ void k_sub_axpy_b(const z64* V, int nb, int nv, const z64* coef, int m, z64* w, long long n) {
  __shared__ z64 cs[128];
  const int r = blockIdx.z;
  for (int v = threadIdx.x; v < nv; v += blockDim.x) cs[v] = coef[(long long)r * (m + 1) + v];
  __syncthreads();
  z64* wr = w + (long long)r * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    z64 acc = wr[i];
    for (int v = 0; v < nv; ++v) cfma(acc, -cs[v], V[((long long)v * nb + r) * n + i]);
    wr[i] = acc;
  }
}

cudaError_t launch_sub_axpy_b(ddm_ctx* c, const z64* V, int nb, int nv, const z64* coef, int m, z64* w, long long n) {
  ++c->nlaunch;
  k_sub_axpy_b<<<dim3(RED_BLOCKS * 2, 1, nb), 256, 0, c->st>>>(V, nb, nv, coef, m, w, n);
  return cudaGetLastError();
}

// one thread per right-hand side: the Givens step of k_givens on its own H and gs
__global__ void k_givens_b(int nb, int j, int m, const double* nrm2, z64* H, z64* gs, double* out_est) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nb) return;
  z64* Hr = H + (long long)r * (m + 1) * m;
  z64* g = gs + (long long)r * (5 * m + 4);
  z64* cs = g;
  z64* sn = g + m;
  z64* gg = g + 2 * m;
  z64* col = Hr + (long long)j * (m + 1);
  const double hn = sqrt(nrm2[r]);
  col[j + 1] = mk<double>(hn, 0.0);
  g[3 * m + 1] = mk<double>(hn > 0 ? 1.0 / hn : 0.0, 0.0);
  for (int i = 0; i < j; ++i) {
    const z64 a = col[i], b = col[i + 1];
    const z64 snc = mk<double>(sn[i].x, -sn[i].y);
    col[i] = cs[i] * a + sn[i] * b;
    col[i + 1] = cs[i] * b - snc * a;
  }
  const z64 a = col[j], b = col[j + 1];
  const double aa = sqrt(cabs2(a)), bb = sqrt(cabs2(b));
  const double den = sqrt(aa * aa + bb * bb);
  z64 cc, s;
  if (den == 0.0) { cc = mk<double>(1, 0); s = mk<double>(0, 0); }
  else if (aa == 0.0) { cc = mk<double>(0, 0); s = mk<double>(b.x / bb, -b.y / bb); }
  else {
    cc = mk<double>(aa / den, 0.0);
    const z64 ph = mk<double>(a.x / aa, a.y / aa);
    s = (1.0 / den) * (ph * mk<double>(b.x, -b.y));
  }
  cs[j] = cc;
  sn[j] = s;
  col[j] = cc * a + s * b;
  col[j + 1] = mk<double>(0, 0);
  const z64 gj = gg[j];
  gg[j + 1] = -(mk<double>(s.x, -s.y) * gj);
  gg[j] = cc * gj;
  out_est[r] = sqrt(cabs2(gg[j + 1]));
}

cudaError_t launch_givens_b(ddm_ctx* c, int nb, int j, int m, const double* nrm2, z64* H, z64* gs, double* out_est) {
  ++c->nlaunch;
  k_givens_b<<<(nb + 63) / 64, 64, 0, c->st>>>(nb, j, m, nrm2, H, gs, out_est);
  return cudaGetLastError();
}

// w_r *= gs_r[3m+1]
__global__ void k_scale_b(z64* w, const z64* gs, int m, long long n) {
  const int r = blockIdx.z;
  const z64 s = gs[(long long)r * (5 * m + 4) + 3 * m + 1];
  z64* wr = w + (long long)r * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    wr[i] = s * wr[i];
}

cudaError_t launch_scale_b(ddm_ctx* c, int nb, z64* w, const z64* gs, int m, long long n) {
  ++c->nlaunch;
  k_scale_b<<<dim3(1216, 1, nb), 256, 0, c->st>>>(w, gs, m, n);
  return cudaGetLastError();
}

// dst_r = src_r * s[r]  (host-computed per right-hand side factors, in device memory)
__global__ void k_scale_vec_b(const z64* src, const double* s, z64* dst, long long n) {
  const int r = blockIdx.z;
  const double sr = s[r];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[(long long)r * n + i] = sr * src[(long long)r * n + i];
}

cudaError_t launch_scale_vec_b(ddm_ctx* c, int nb, const z64* src, const double* s, z64* dst, long long n) {
  ++c->nlaunch;
  k_scale_vec_b<<<dim3(1216, 1, nb), 256, 0, c->st>>>(src, s, dst, n);
  return cudaGetLastError();
}

// y_r = H_r(0:j_r, 0:j_r)^{-1} g_r(0:j_r), one thread per right-hand side
__global__ void k_lsq_b(int nb, const int* jr, int m, const z64* H, z64* gs) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nb) return;
  const int j = jr[r];
  const z64* Hr = H + (long long)r * (m + 1) * m;
  z64* g = gs + (long long)r * (5 * m + 4);
  const z64* gg = g + 2 * m;
  z64* y = g + 3 * m + 2;
  for (int i = j - 1; i >= 0; --i) {
    z64 acc = gg[i];
    for (int k = i + 1; k < j; ++k) acc = acc - Hr[(long long)k * (m + 1) + i] * y[k];
    y[i] = acc * cinv(Hr[(long long)i * (m + 1) + i]);
  }
}

// x_r += Z_r(:, 0:j_r) y_r
__global__ void k_update_x_b(int nb, const int* jr, int m, const z64* gs, const z64* Z, z64* x, long long n) {
  __shared__ z64 ys[128];
  const int r = blockIdx.z;
  const int j = jr[r];
  for (int v = threadIdx.x; v < j; v += blockDim.x) ys[v] = gs[(long long)r * (5 * m + 4) + 3 * m + 2 + v];
  __syncthreads();
  if (j == 0) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    z64 acc = x[(long long)r * n + i];
    for (int v = 0; v < j; ++v) cfma(acc, ys[v], Z[((long long)v * nb + r) * n + i]);
    x[(long long)r * n + i] = acc;
  }
}

cudaError_t launch_lsq_update_b(ddm_ctx* c, int nb, const int* d_jr, int m, const z64* H, z64* gs, const z64* Z, z64* x,
                                long long n) {
  c->nlaunch += 2;
  k_lsq_b<<<(nb + 63) / 64, 64, 0, c->st>>>(nb, d_jr, m, H, gs);
  k_update_x_b<<<dim3(RED_BLOCKS * 2, 1, nb), 256, 0, c->st>>>(nb, d_jr, m, gs, Z, x, n);
  return cudaGetLastError();
}

}  // namespace ddm

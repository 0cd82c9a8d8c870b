// Set-up kernels: PML stretching tables, k^2, subdomain operator hashes for factor
// sharing, and the J-scaled right-hand side b = h^2 J f.
#include "ddm_internal.cuh"

namespace ddm {

// Shifted PML profile (Section 2.1, Eq. (11)): sigma = 0 for t <= ov cells beyond a
// box face, sigma0 ((t - ov) / npml)^power beyond.
__device__ __forceinline__ double sigma_of(double t, int ov, int npml, double sigma0, double power) {
  if (t <= (double)ov) return 0.0;
  return sigma0 * pow((t - (double)ov) / (double)npml, power);
}

// One block per table.  tdesc[3*t] = lo, [3*t+1] = hi (own node range of the box along the
// axis), [3*t+2] = offset into tab.  Writes alpha = 1 + i sigma at the ext nodes (positions
// lo-e+i+1/2) and 1/alpha at the half nodes (positions lo-e+j), j = 0..ext.
__global__ void k_build_tables(z64* tab, const int* tdesc, int e, int ov, int npml, double sigma0, double power) {
  int t = blockIdx.x;
  int lo = tdesc[3 * t], hi = tdesc[3 * t + 1], ofs = tdesc[3 * t + 2];
  int ext = hi - lo + 2 * e;
  for (int j = threadIdx.x; j <= ext; j += blockDim.x) {
    if (j < ext) {
      double pos = (double)(lo - e + j) + 0.5;
      double d = fmax(fmax((double)lo - pos, pos - (double)hi), 0.0);
      tab[ofs + j] = mk<double>(1.0, sigma_of(d, ov, npml, sigma0, power));
    }
    double pos = (double)(lo - e + j);
    double d = fmax(fmax((double)lo - pos, pos - (double)hi), 0.0);
    tab[ofs + ext + j] = cinv(mk<double>(1.0, sigma_of(d, ov, npml, sigma0, power)));
  }
}

cudaError_t launch_build_tables(ddm_ctx* c, const int* d_tdesc, int ntab, double sigma0, double power, int npml) {
  ++c->nlaunch;
  k_build_tables<<<ntab, 128, 0, c->st>>>(c->d_tab, d_tdesc, c->e, c->p.overlap, npml, sigma0, power);
  return cudaGetLastError();
}

// k(x) = omega / c(x) (Section 1)
__global__ void k_k2(double* k2, const double* cv, double omega, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double k = omega / cv[i];
    k2[i] = k * k;
  }
}

cudaError_t launch_k2(ddm_ctx* c, const double* c_dev) {
  ++c->nlaunch;
  k_k2<<<608, 256, 0, c->st>>>(c->d_k2, c_dev, c->omega, c->g.nglob);
  return cudaGetLastError();
}

// splitmix64 finaliser (Steele, Lea, Flood 2014) as a bit mixer
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ long long gindex(const Geom& g, const SubDesc& s, const int* x) {
  long long gi = 0;
  for (int a = g.dim - 1; a >= 0; --a) gi = gi * g.N[a] + (s.lo[a] + x[a]);   // global ext index of local x = lo + x
  return gi;
}

// Order-dependent hash of k^2 over each subdomain's extended window (one block per subdomain).
// The alpha tables depend only on the own widths, which the host compares separately.
__global__ void k_sub_hash(Geom g, unsigned long long* out) {
  const SubDesc& s = g.subs[blockIdx.x];
  long long len = (long long)s.ext[0] * s.ext[1] * s.ext[2];
  unsigned long long acc = 0;
  for (long long i = threadIdx.x; i < len; i += blockDim.x) {
    int x[3] = {(int)(i % s.ext[0]), (int)((i / s.ext[0]) % s.ext[1]), (int)(i / ((long long)s.ext[0] * s.ext[1]))};
    double v = g.k2[gindex(g, s, x)];
    acc += mix64((unsigned long long)__double_as_longlong(v) ^ mix64((unsigned long long)i));
  }
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ unsigned long long sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    out[blockIdx.x] = t;
  }
}

cudaError_t launch_sub_hash(ddm_ctx* c, unsigned long long* d_hash) {
  ++c->nlaunch;
  k_sub_hash<<<c->g.nsub, 256, 0, c->st>>>(c->g, d_hash);
  return cudaGetLastError();
}

// Exact comparison of k^2 windows of subdomain pairs (a, b) with equal own widths.
__global__ void k_sub_compare(Geom g, const int* pairs, int* mismatch) {
  const SubDesc& A = g.subs[pairs[2 * blockIdx.x]];
  const SubDesc& B = g.subs[pairs[2 * blockIdx.x + 1]];
  long long len = (long long)A.ext[0] * A.ext[1] * A.ext[2];
  int bad = 0;
  for (long long i = threadIdx.x; i < len; i += blockDim.x) {
    int x[3] = {(int)(i % A.ext[0]), (int)((i / A.ext[0]) % A.ext[1]), (int)(i / ((long long)A.ext[0] * A.ext[1]))};
    if (g.k2[gindex(g, A, x)] != g.k2[gindex(g, B, x)]) bad = 1;
  }
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) mismatch[blockIdx.x] = bad;
}

cudaError_t launch_sub_compare(ddm_ctx* c, const int* d_pairs, int npairs, int* d_mismatch) {
  if (npairs == 0) return cudaSuccess;
  ++c->nlaunch;
  k_sub_compare<<<npairs, 256, 0, c->st>>>(c->g, d_pairs, d_mismatch);
  return cudaGetLastError();
}

// Operator coefficients (assembly): per subdomain, planes of its local grid in the local
// precision T -- plane 0 the centre, plane 1+2a the coupling to x - e_a, 2+2a to x + e_a --
// evaluated in FP64 from the alpha tables and k^2 and rounded once; and the same planes of
// the global operator in FP64.  blockIdx.y = subdomain (or nsub for the global box).
template <typename T>
__global__ void k_coefs(Geom g, cplx<T>* lc, z64* gc) {
  const int nc = 2 * g.dim + 1;
  if ((int)blockIdx.y < g.nsub) {
    const SubDesc& s = g.subs[blockIdx.y];
    long long len = (long long)s.ext[0] * s.ext[1] * s.ext[2];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
      int x[3] = {(int)(i % s.ext[0]), (int)((i / s.ext[0]) % s.ext[1]), (int)(i / ((long long)s.ext[0] * s.ext[1]))};
      Coef cf = coef_at(g, s.tab, s.ext, x, g.k2[gindex(g, s, x)]);
      cplx<T>* base = lc + s.vofs * nc + i;
      base[0] = ccast<T>(cf.c);
      for (int a = 0; a < g.dim; ++a) { base[(1 + 2 * a) * len] = ccast<T>(cf.m[a]); base[(2 + 2 * a) * len] = ccast<T>(cf.p[a]); }
    }
  } else {
    long long n = g.nglob;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
      int x[3] = {(int)(i % g.N[0]), (int)((i / g.N[0]) % g.N[1]), (int)(i / ((long long)g.N[0] * g.N[1]))};
      Coef cf = coef_at(g, g.gtab, g.N, x, g.k2[i]);
      gc[i] = cf.c;
      for (int a = 0; a < g.dim; ++a) { gc[(1 + 2 * a) * n + i] = cf.m[a]; gc[(2 + 2 * a) * n + i] = cf.p[a]; }
    }
  }
}

cudaError_t launch_coefs(ddm_ctx* c) {
  dim3 grid(64, c->g.nsub + 1);
  ++c->nlaunch;
  if (c->prec == DDM_MIXED) k_coefs<float><<<grid, 256, 0, c->st>>>(c->g, (c32*)c->d_lcoef, c->d_gcoef);
  else k_coefs<double><<<grid, 256, 0, c->st>>>(c->g, (z64*)c->d_lcoef, c->d_gcoef);
  return cudaGetLastError();
}

// b = h^2 J f on the global grid (J = prod_a alpha_a of the global box).
__global__ void k_rhs(Geom g, const z64* f, z64* b, int nrhs) {
  long long n = g.nglob;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n * nrhs; i += (long long)gridDim.x * blockDim.x) {
    long long gi = i % n;
    int x[3] = {(int)(gi % g.N[0]), (int)((gi / g.N[0]) % g.N[1]), (int)(gi / ((long long)g.N[0] * g.N[1]))};
    z64 J = mk<double>(1.0, 0.0);
    for (int a = 0; a < g.dim; ++a) J = J * tab_node(g, g.gtab[a], x[a]);
    b[i] = g.h2 * (J * f[i]);
  }
}

cudaError_t launch_rhs(ddm_ctx* c, const z64* f, z64* b, int nrhs) {
  ++c->nlaunch;
  k_rhs<<<1216, 256, 0, c->st>>>(c->g, f, b, nrhs);
  return cudaGetLastError();
}

}  // namespace ddm

namespace ddm {
// beta[q] = beta_0(q / ov), q = 0..ov, with beta_0(t) = 1 - (10 t^3 - 15 t^4 + 6 t^5) on
// [0, 1]: C^2, monotone, 1 at t <= 0 and 0 at t >= 1 (Section 2.2).  A node q nodes beyond
// the first node outside a face takes beta[q] (so beta = 1 on the own box plus one layer).
__global__ void k_beta(double* beta, int ov) {
  int q = threadIdx.x;
  if (q > ov) return;
  double t = (double)q / (double)ov;
  t = fmin(fmax(t, 0.0), 1.0);
  beta[q] = 1.0 - t * t * t * (10.0 - 15.0 * t + 6.0 * t * t);
}

cudaError_t launch_beta(ddm_ctx* c) {
  ++c->nlaunch;
  k_beta<<<1, ((c->p.overlap + 32) / 32) * 32, 0, c->st>>>(c->d_beta, c->p.overlap);
  return cudaGetLastError();
}
}  // namespace ddm

// Source restriction, the fused directional-residual transfer (the Psi operators of
// Section 2.2 in Eq. (38)) with residual-norm partials, and the assembly of the DDM
// solution (Eq. (39)).
#include <algorithm>

#include "ddm_internal.cuh"

namespace ddm {

__device__ __forceinline__ void unflat(long long i, const int* ext, int* x) {
  x[0] = (int)(i % ext[0]);
  x[1] = (int)((i / ext[0]) % ext[1]);
  x[2] = (int)(i / ((long long)ext[0] * ext[1]));
}

__device__ __forceinline__ long long flat(const int* x, const int* ext) {
  return ((long long)x[2] * ext[1] + x[1]) * ext[0] + x[0];
}

__device__ __forceinline__ long long gflat(const Geom& g, const SubDesc& s, const int* x) {
  return ((long long)(s.lo[2] + x[2]) * g.N[1] + (s.lo[1] + x[1])) * g.N[0] + (s.lo[0] + x[0]);
}

// x in the own region of s: own box, continued through the global band on boundary sides
__device__ __forceinline__ bool in_own(const Geom& g, const SubDesc& s, const int* x) {
  for (int a = 0; a < g.dim; ++a) {
    int lo = g.e, hi = g.e + s.nown[a];
    if (x[a] < lo && !((s.at_lo >> a) & 1)) return false;
    if (x[a] >= hi && !((s.at_hi >> a) & 1)) return false;
  }
  return true;
}

// ---------------------------------------------------------------------------
// step-1 source f_ij = b chi_own (Section 2.2), cast to the local precision; zero U.
// grid: (ceil(maxlen/256), nsub, nrhs)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_restrict(Geom g, const z64* b, cplx<T>* src, cplx<T>* U) {
  const SubDesc& s = g.subs[blockIdx.y];
  long long len = (long long)s.ext[0] * s.ext[1] * s.ext[2];
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= len) return;
  int r = blockIdx.z;
  int x[3];
  unflat(i, s.ext, x);
  cplx<T> v = mk<T>(0, 0);
  if (in_own(g, s, x)) v = ccast<T>(b[(long long)r * g.nglob + gflat(g, s, x)]);
  long long o = lvofs(s, r, (int)gridDim.z) + i;
  src[o] = v;
  if (U) U[o] = mk<T>(0, 0);
}

template <typename T>
static cudaError_t restrict_t(ddm_ctx* c, const z64* b, void* src, void* U, int nrhs) {
  int maxlen = 0;
  for (auto& s : c->subs) maxlen = max(maxlen, s.ext[0] * s.ext[1] * s.ext[2]);
  dim3 grid((maxlen + 255) / 256, c->g.nsub, nrhs);
  ++c->nlaunch;
  k_restrict<T><<<grid, 256, 0, c->st>>>(c->g, b, (cplx<T>*)src, (cplx<T>*)U);
  return cudaGetLastError();
}

cudaError_t launch_restrict(ddm_ctx* c, const z64* b, void* src, void* U, int nrhs) {
  return c->prec == DDM_MIXED ? restrict_t<float>(c, b, src, U, nrhs) : restrict_t<double>(c, b, src, U, nrhs);
}

// ---------------------------------------------------------------------------
// Fused transfer.  For receiver R (blockIdx.y) and its extended node x:
//   src^{s+1}_R(x) = sum_d Psi_d(u_{R-d}^{s+1-lag(d)})(x)
//   res(x)         = sum_d Psi_d(u^s + .. + u^{s-lag(d)+1})(x)  on R's own region,
// with Psi_d(v) = -A_R(beta_d v) chi_d, beta_d the sender's cut-off(s) facing R and chi_d
// the receiver's side of the shared face(s) (Section 2.2).  Psi_d is non-zero only on
// receiver nodes at most ov nodes inside each shared face: the threads run over R's
// strip-node list (built at set-up: local index plus the mask of directions that reach the
// node), and beta_d is evaluated as a product of 1D cut-offs.  Sums of |res|^2 per block go
// to part[(r * nsub + R) * gridDim.x + blockIdx.x].
// ring[t % L] holds u^t (local layout), L = dim; res_slot[k] is the slot of u^{s-k}
// (-1 when s-k < 1, i.e. u = 0).
// ---------------------------------------------------------------------------
struct RingPtrs { const void* p[3]; int res_slot[3]; };

template <typename T>
struct CoefT { cplx<T> c, m[3], p[3]; };

// the fields of a sender that the transfer reads, staged in shared memory per receiver
struct NbrS { int lo[3], ext[3], nown[3], pad; long long vofs; };

// Each thread takes one strip node of R and TR_RG right-hand sides (blockIdx.z = group): the
// stencil terms of -A_R (beta_d .) at the node (sender index, coefficient x cut-off) are built
// once per direction and applied to every right-hand side of the group.  TR_RG = 1 for a single
// right-hand side (fewer registers, more resident warps), 8 otherwise.  The kernel is bound by the
// latency of its gathered loads, so the register caps favour resident warps over a small spill
// (2048^2, 64 right-hand sides: 2.09 ms per transfer at 96 registers against 2.60 ms at 141).
template <typename T, int TR_RG>
__global__ void __launch_bounds__(128, TR_RG == 1 ? 6 : 5) k_transfer(Geom g, RingPtrs ring, cplx<T>* src_next, double* part, int want_res,
                                                  int nrhs) {
  const int Rid = blockIdx.y;
  const SubDesc& R = g.subs[Rid];
  const int r0 = blockIdx.z * TR_RG, nr = min(TR_RG, nrhs - r0);
  const int e = g.e, ov = g.ov, dim = g.dim;
  __shared__ T beta_s[32];
  __shared__ double sh[TR_RG][4];
  __shared__ NbrS nb_s[NDIR];            // the receiver's neighbours, by direction code
  if (threadIdx.x <= ov && threadIdx.x < 32) beta_s[threadIdx.x] = (T)g.beta[threadIdx.x];
  if (threadIdx.x >= 32 && threadIdx.x < 32 + NDIR) {
    const int code = threadIdx.x - 32, id = R.nbr[code];
    if (id >= 0) {
      const SubDesc& S = g.subs[id];
      NbrS v;
      for (int a = 0; a < 3; ++a) { v.lo[a] = S.lo[a]; v.ext[a] = S.ext[a]; v.nown[a] = S.nown[a]; }
      v.pad = 0;
      v.vofs = S.vofs;
      nb_s[code] = v;
    }
  }
  __syncthreads();
  const int it = blockIdx.x * blockDim.x + threadIdx.x;
  double res2[TR_RG];
#pragma unroll
  for (int rr = 0; rr < TR_RG; ++rr) res2[rr] = 0.0;
  if (it < R.scnt) {
    const int li = g.sidx[R.sofs + it];
    const unsigned mask = g.smask[R.sofs + it];
    int x[3];
    unflat(li, R.ext, x);
    const long long len = (long long)R.ext[0] * R.ext[1] * R.ext[2];
    CoefT<T> cf;
    {
      const int nc = 2 * dim + 1;
      const cplx<T>* lc = (const cplx<T>*)g.lcoef + R.vofs * nc + li;
      cf.c = lc[0];
      for (int a = 0; a < dim; ++a) { cf.m[a] = lc[(1 + 2 * a) * len]; cf.p[a] = lc[(2 + 2 * a) * len]; }
    }
    cplx<T> acc_src[TR_RG], acc_res[TR_RG];
#pragma unroll
    for (int rr = 0; rr < TR_RG; ++rr) acc_src[rr] = acc_res[rr] = mk<T>(0, 0);
    unsigned dm = mask & 0x07ffffffu;
    while (dm) {
      const int code = __ffs(dm) - 1;
      dm &= dm - 1;
      const int d[3] = {code % 3 - 1, (code / 3) % 3 - 1, code / 9 - 1};
      const int lagd = (d[0] != 0) + (d[1] != 0) + (d[2] != 0);
      const NbrS& S = nb_s[code];
      // the stencil of x in S-local coordinates and the sender's cut-off there (1D factors)
      int y0[3];
      for (int a = 0; a < 3; ++a) y0[a] = x[a] + R.lo[a] - S.lo[a];
      // per axis: cut-off at offsets -1, 0, +1 along that axis (beta_d is a product of 1D cut-offs)
      T bw[3][3];
      bool inside[3][3];
      for (int a = 0; a < 3; ++a) {
        for (int o = -1; o <= 1; ++o) {
          const int ya = y0[a] + o;
          T bb = (T)1;
          bool in = a < dim ? (ya >= 0 && ya < S.ext[a]) : (o == 0);
          if (a < dim && d[a] != 0) {
            const int q = d[a] > 0 ? ya - (e + S.nown[a]) : (e - 1) - ya;
            bb = q < 0 ? (T)1 : (q >= ov ? (T)0 : beta_s[q]);
          }
          bw[a][o + 1] = bb;
          inside[a][o + 1] = in;
        }
      }
      // terms t = 0 (centre) and 1 + 2 a + (o > 0) (neighbour along axis a): S-local index and
      // coefficient x cut-off; `live` marks the terms that contribute
      int tix[7];
      cplx<T> tcf[7];
      unsigned live = 0;
      {
        const T w0 = bw[0][1] * bw[1][1] * bw[2][1];
        tix[0] = flat(y0, S.ext);
        tcf[0] = mk<T>(w0 * cf.c.x, w0 * cf.c.y);
        if (w0 != (T)0 && inside[0][1] && inside[1][1] && inside[2][1]) live |= 1u;
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int oi = 0; oi < 2; ++oi) {
          const int o = oi ? 1 : -1, t = 1 + 2 * a + oi;
          tix[t] = 0;
          tcf[t] = mk<T>(0, 0);
          if (a >= dim) continue;
          if ((o > 0 && x[a] + 1 >= R.ext[a]) || (o < 0 && x[a] == 0)) continue;   // R's Dirichlet ghost
          if (!inside[a][o + 1]) continue;
          bool okin = true;
          T w = (T)1;
          for (int bax = 0; bax < 3; ++bax) {
            const int oo = bax == a ? o + 1 : 1;
            okin = okin && inside[bax][oo];
            w *= bw[bax][oo];
          }
          if (!okin || w == (T)0) continue;
          int yy[3] = {y0[0], y0[1], y0[2]};
          yy[a] += o;
          tix[t] = flat(yy, S.ext);
          const cplx<T> cc = o > 0 ? cf.p[a] : cf.m[a];
          tcf[t] = mk<T>(w * cc.x, w * cc.y);
          live |= 1u << t;
        }
      }
      for (int k = 0; k < lagd; ++k) {
        if (!want_res && k != lagd - 1) continue;
        const int sl = ring.res_slot[k];
        if (sl < 0) continue;
        const cplx<T>* ub = (const cplx<T>*)ring.p[sl];
#pragma unroll
        for (int rr = 0; rr < TR_RG; ++rr) {
          if (rr >= nr) break;
          const cplx<T>* u = ub + S.vofs * nrhs + (long long)(r0 + rr) * ((long long)S.ext[0] * S.ext[1] * S.ext[2]);
          // -(A_R (beta_d u_S))(x)
          cplx<T> acc = mk<T>(0, 0);
#pragma unroll
          for (int t = 0; t < 7; ++t)
            if (live & (1u << t)) cfma(acc, tcf[t], u[tix[t]]);
          if (k == lagd - 1) acc_src[rr] = acc_src[rr] - acc;
          acc_res[rr] = acc_res[rr] - acc;
        }
      }
    }
#pragma unroll
    for (int rr = 0; rr < TR_RG; ++rr) {
      if (rr >= nr) break;
      src_next[lvofs(R, r0 + rr, nrhs) + li] = acc_src[rr];
      if (want_res && (mask & 0x80000000u))
        res2[rr] = (double)acc_res[rr].x * acc_res[rr].x + (double)acc_res[rr].y * acc_res[rr].y;
    }
  }
  if (want_res) {
    // sums of |res|^2 per block and right-hand side
#pragma unroll
    for (int rr = 0; rr < TR_RG; ++rr) {
      double v = res2[rr];
      for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) == 0) sh[rr][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if ((int)threadIdx.x < nr) {
      double t = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[threadIdx.x][w];
      part[((long long)(r0 + threadIdx.x) * g.nsub + Rid) * gridDim.x + blockIdx.x] = t;
    }
  }
}

int ring_slots(const ddm_ctx* c) { return c->dim; }

// s = index of the step just solved (u^s in ring[s % L]).
template <typename T>
static cudaError_t transfer_t(ddm_ctx* c, int s, void* src_next, double* part, int nrhs, int want_res, int* nblk) {
  int L = ring_slots(c);
  RingPtrs rp;
  for (int k = 0; k < 3; ++k) rp.p[k] = c->d_ring[k];
  // slots of u^s, u^{s-1}, u^{s-2} (-1 where the step index is < 1)
  for (int k = 0; k < 3; ++k) {
    int t = s - k;
    rp.res_slot[k] = (k < L && t >= 1) ? (t % L) : -1;
  }
  const int rg = nrhs == 1 ? 1 : 8;
  dim3 grid((std::max(c->max_scnt, 1) + 127) / 128, c->g.nsub, (nrhs + rg - 1) / rg);
  if (nblk) *nblk = grid.x;
  ++c->nlaunch;
  if (rg == 1) k_transfer<T, 1><<<grid, 128, 0, c->st>>>(c->g, rp, (cplx<T>*)src_next, part, want_res, nrhs);
  else k_transfer<T, 8><<<grid, 128, 0, c->st>>>(c->g, rp, (cplx<T>*)src_next, part, want_res, nrhs);
  return cudaGetLastError();
}

cudaError_t launch_transfer_n(ddm_ctx* c, int s, void* src_next, double* part, int nrhs, int want_res, int* nblk) {
  return c->prec == DDM_MIXED ? transfer_t<float>(c, s, src_next, part, nrhs, want_res, nblk)
                              : transfer_t<double>(c, s, src_next, part, nrhs, want_res, nblk);
}


// ---------------------------------------------------------------------------
// w = sum_R beta_{0;R} U_R (Eq. (39)) on the global grid.  A global node lies in the
// support of beta_{0;R} for at most two parts per axis: its owner and the neighbour whose
// face is within ov nodes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double cut_lo(const Geom& g, int part, int a, int p) {
  // beta_{<-} of part along axis a at global node p
  if (part == 0) return 1.0;
  int q = g.cuts[a][part] - 1 - p;
  return q < 0 ? 1.0 : (q >= g.ov ? 0.0 : g.beta[q]);
}
__device__ __forceinline__ double cut_hi(const Geom& g, int part, int a, int p) {
  if (part == g.parts[a] - 1) return 1.0;
  int q = p - g.cuts[a][part + 1];
  return q < 0 ? 1.0 : (q >= g.ov ? 0.0 : g.beta[q]);
}

// One thread per global node: its (at most 2 per axis) candidate parts and weights are found
// once, then applied to every right-hand side, accumulating in the local precision T (the
// local solutions are only T-accurate; FP64 is what the DDM_FP64 path needs).
template <typename T>
__global__ void k_assemble(Geom g, const cplx<T>* U, z64* w, int nrhs) {
  const long long n = g.nglob;
  for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < n; gi += (long long)gridDim.x * blockDim.x) {
    int xg[3] = {(int)(gi % g.N[0]), (int)((gi / g.N[0]) % g.N[1]), (int)(gi / ((long long)g.N[0] * g.N[1]))};
    int cand[3][2], ncand[3];
    double wt[3][2];
    for (int a = 0; a < 3; ++a) {
      ncand[a] = 0;
      if (a >= g.dim) { cand[a][0] = 0; wt[a][0] = 1.0; ncand[a] = 1; continue; }
      int p = xg[a] - g.e;                     // global node index
      int own = g.owner[a][xg[a]];
      for (int dp = -1; dp <= 1; ++dp) {
        int part = own + dp;
        if (part < 0 || part >= g.parts[a]) continue;
        double bwt = cut_lo(g, part, a, p) * cut_hi(g, part, a, p);
        // nodes outside the part's extended grid carry no value
        if (p < g.cuts[a][part] - g.e || p >= g.cuts[a][part + 1] + g.e) bwt = 0.0;
        if (bwt != 0.0 && ncand[a] < 2) { cand[a][ncand[a]] = part; wt[a][ncand[a]] = bwt; ncand[a]++; }
      }
    }
    // terms t = 4 i0 + 2 i1 + i2 (bit t of `live` when present): element offset of right-hand
    // side 0, stride between right-hand sides, weight
    long long tofs[8], tstr[8];
    T tw[8];
    unsigned live = 0;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int i0 = t >> 2, i1 = (t >> 1) & 1, i2 = t & 1;
      tofs[t] = 0;
      tstr[t] = 0;
      tw[t] = (T)0;
      if (i0 >= ncand[0] || i1 >= ncand[1] || i2 >= ncand[2]) continue;
      int part[3] = {cand[0][i0], cand[1][i1], cand[2][i2]};
      int sid = (part[2] * g.parts[1] + part[1]) * g.parts[0] + part[0];
      const SubDesc& s = g.subs[sid];
      int xl[3] = {xg[0] - s.lo[0], xg[1] - s.lo[1], g.dim == 3 ? xg[2] - s.lo[2] : 0};
      tofs[t] = lvofs(s, 0, nrhs) + flat(xl, s.ext);
      tstr[t] = (long long)s.ext[0] * s.ext[1] * s.ext[2];
      tw[t] = (T)(wt[0][i0] * wt[1][i1] * wt[2][i2]);
      live |= 1u << t;
    }
    for (int r = 0; r < nrhs; ++r) {
      cplx<T> acc = mk<T>(0, 0);
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (live & (1u << t)) acc = acc + tw[t] * U[tofs[t] + r * tstr[t]];
      w[(long long)r * n + gi] = mk<double>((double)acc.x, (double)acc.y);
    }
  }
}

cudaError_t launch_assemble(ddm_ctx* c, const void* U, z64* w, int nrhs) {
  ++c->nlaunch;
  if (c->prec == DDM_MIXED)
    k_assemble<float><<<1216, 256, 0, c->st>>>(c->g, (const c32*)U, w, nrhs);
  else
    k_assemble<double><<<1216, 256, 0, c->st>>>(c->g, (const z64*)U, w, nrhs);
  return cudaGetLastError();
}

}  // namespace ddm

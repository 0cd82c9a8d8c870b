// Batched block-tridiagonal solves u_R = A_R^{-1} src_R over all subdomains and right-hand
// sides (the local solves of Algorithm 3.1, Eqs. (talg_1)/(talg_2)).
//
// With G_k = D_k^{-1} from factor.cu:
//   forward   y_k = r_k - c_S(., k) * t_{k-1},   t_k = G_k y_k            (k = 0..m-1)
//   backward  x_{m-1} = t_{m-1},  x_k = t_k - G_k (c_N(., k) * x_{k+1})    (k = m-2..0)
// so every G_k is streamed from HBM twice per solve (once per sweep) and applied to NR
// right-hand sides at once.  G_k is stored column-major.  One CTA per (subdomain, group of
// NR right-hand sides): warp 8 is the producer, copying 16-column chunks of G_k into a ring
// of shared-memory stages with cp.async.bulk (1D TMA) on mbarriers; warps 0-7 consume them,
// thread (half, row) accumulating its row over half of each chunk's columns (conflict-free
// column reads, broadcast y).  The per-block vectors (source or t_k, U_k, couplings) are
// prefetched into registers one block ahead and outputs are staged in shared memory and
// written coalesced, so no global load sits on the sweep's critical path.  Waits are bounded:
// on time-out the kernel records ERRBIT_TIMEOUT and runs to completion without hanging.
#include <algorithm>

#include "ddm_internal.cuh"

namespace ddm {

constexpr int SOLVE_NCW = 8;     // consumer warps
constexpr int SOLVE_RCH = 16;    // columns of G_k per pipeline chunk
constexpr int SOLVE_THREADS = (SOLVE_NCW + 1) * 32;
constexpr long long WAIT_LIMIT = 1LL << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; false (and the error bit) on time-out
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, int* err) {
  for (long long it = 0; it < WAIT_LIMIT; ++it)
    if (mbar_try(a, parity)) return true;
  atomicOr(err, ERRBIT_TIMEOUT);
  return false;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, %0;" ::"r"(SOLVE_NCW * 32) : "memory"); }

// The block sequence: i = 0..m-1 forward over k = i, then i = m..2m-2 backward over k = 2m-2-i.
__device__ __forceinline__ void seq_block(int i, int m, int& pass, int& k) {
  pass = i < m ? 0 : 1;
  k = pass == 0 ? i : 2 * m - 2 - i;
}

template <typename T, int NR, int NST>
__global__ void __launch_bounds__(SOLVE_THREADS) k_solve2d(Geom g, const cplx<T>* __restrict__ G,
                                                          const cplx<T>* __restrict__ src, cplx<T>* out,
                                                          cplx<T>* U, int nrhs, int* err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const SubDesc& s = g.subs[blockIdx.x];
  const int b = s.ext[0], m = s.ext[1], ldb = s.pad;
  const int bpad = (b + 3) & ~3;
  const int r0 = blockIdx.y * NR;
  const int nr = min(NR, nrhs - r0);
  const int nch = (b + SOLVE_RCH - 1) / SOLVE_RCH;
  const int nblk = 2 * m - 1;

  cplx<T>* stage = (cplx<T>*)smem;                                   // NST x RCH x ldb
  cplx<T>* ys = stage + (size_t)NST * SOLVE_RCH * ldb;               // NR x bpad: right-hand side of the block GEMV
  cplx<T>* ts = ys + NR * bpad;                                      // NR x bpad: outputs of the previous block
  cplx<T>* tk = ts + NR * bpad;                                      // NR x bpad: t_k (backward)
  cplx<T>* uk = tk + NR * bpad;                                      // NR x bpad: U_k before accumulation
  cplx<T>* red = uk + NR * bpad;                                     // NR x bpad: second-half partial sums
  uint64_t* bars = (uint64_t*)(((uintptr_t)(red + NR * bpad) + 15) & ~(uintptr_t)15);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + NST);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < NST; ++i) { mbar_init(full0 + 8 * i, 1); mbar_init(empty0 + 8 * i, SOLVE_NCW); }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == SOLVE_NCW) {
    // ---------------- producer: column chunks of G_k in consumption order ----------------
    if (lane == 0) {
      long long c = 0;
      for (int i = 0; i < nblk; ++i) {
        int pass, k;
        seq_block(i, m, pass, k);
        for (int ch = 0; ch < nch; ++ch, ++c) {
          const int st = (int)(c % NST);
          if (c >= NST) mbar_wait(empty0 + 8 * st, (uint32_t)((c / NST - 1) & 1), err);
          const int cols = min(SOLVE_RCH, b - ch * SOLVE_RCH);
          const uint32_t bytes = (uint32_t)(cols * ldb * (int)sizeof(cplx<T>));
          mbar_expect_tx(full0 + 8 * st, bytes);
          bulk_g2s(smem_u32(stage + (size_t)st * SOLVE_RCH * ldb),
                   G + s.fofs + ((long long)k * b + ch * SOLVE_RCH) * ldb, bytes, full0 + 8 * st);
        }
      }
      const long long total = (long long)nblk * nch;
      for (long long cc = max(0LL, total - NST); cc < total; ++cc)   // bounded wait for copies in flight
        mbar_wait(full0 + 8 * (int)(cc % NST), (uint32_t)((cc / NST) & 1), err);
    }
    return;
  }

  // ---------------- consumers ----------------
  const long long lt = g.ltotal;
  const long long len = (long long)b * m;
  const cplx<T>* srcv = src + (long long)r0 * lt + s.vofs;
  cplx<T>* outv = out + (long long)r0 * lt + s.vofs;
  cplx<T>* Uv = U ? U + (long long)r0 * lt + s.vofs : nullptr;
  const cplx<T>* lc = (const cplx<T>*)g.lcoef + s.vofs * 5;      // planes: C, W, E, S, N
  const cplx<T>* cSp = lc + 3 * len;
  const cplx<T>* cNp = lc + 4 * len;
  constexpr int PI = (NR * 128 + SOLVE_NCW * 32 - 1) / (SOLVE_NCW * 32);   // items per thread (b <= 128)
  const int nitem = nr * b;
  // prefetched per-block values: forward (src_k, c_S(k)) or backward (t_k, U_k, c_N(k))
  cplx<T> pa[PI], pb[PI], pc[PI];
  auto load_block = [&](int i) {
    int pass, k;
    seq_block(i, m, pass, k);
#pragma unroll
    for (int q = 0; q < PI; ++q) {
      const int idx = tid + q * SOLVE_NCW * 32;
      if (idx < nitem) {
        const int rr = idx / b, j = idx - rr * b;
        const long long o = (long long)rr * lt + (long long)k * b + j;
        if (pass == 0) {
          pa[q] = srcv[o];
          pc[q] = k > 0 ? cSp[(long long)k * b + j] : mk<T>(0, 0);
          pb[q] = (Uv && k == m - 1) ? Uv[o] : mk<T>(0, 0);
        } else {
          pa[q] = outv[o];
          pc[q] = cNp[(long long)k * b + j];
          pb[q] = Uv ? Uv[o] : mk<T>(0, 0);
        }
      }
    }
  };
  load_block(0);
  long long c = 0;
  for (int i = 0; i < nblk; ++i) {
    int pass, k;
    seq_block(i, m, pass, k);
    // flush the previous block's outputs (coalesced), stage this block's vectors, form y
#pragma unroll
    for (int q = 0; q < PI; ++q) {
      const int idx = tid + q * SOLVE_NCW * 32;
      if (idx < nitem) {
        const int rr = idx / b, j = idx - rr * b;
        const int sidx = rr * bpad + j;
        if (i > 0) {
          int pp, pk;
          seq_block(i - 1, m, pp, pk);
          const long long o = (long long)rr * lt + (long long)pk * b + j;
          const cplx<T> v = ts[sidx];
          outv[o] = v;
          if (Uv && (pp == 1 || pk == m - 1)) Uv[o] = uk[sidx] + v;
        }
        cplx<T> y;
        if (pass == 0) {
          y = pa[q];
          if (k > 0) y = y - pc[q] * ts[sidx];      // y_k = r_k - c_S(., k) t_{k-1}
        } else {
          y = pc[q] * ts[sidx];                      // z = c_N(., k) x_{k+1}
          tk[sidx] = pa[q];
        }
        ys[sidx] = y;
        uk[sidx] = pb[q];
      }
    }
    if (i + 1 < nblk) load_block(i + 1);
    consumer_sync();
    // G_k y: thread (half h, row i) accumulates its row over the columns of each chunk that
    // fall in its half; the halves are combined at the end of the block
    cplx<T> acc[NR];
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) acc[rr] = mk<T>(0, 0);
    const int row = tid & 127, half = tid >> 7;
    for (int ch = 0; ch < nch; ++ch, ++c) {
      const int st = (int)(c % NST);
      mbar_wait(full0 + 8 * st, (uint32_t)((c / NST) & 1), err);
      const cplx<T>* sg = stage + (size_t)st * SOLVE_RCH * ldb;   // columns ch*16 .. ch*16+15
      if (row < b) {
        const int j0 = ch * SOLVE_RCH + half * (SOLVE_RCH / 2);
        const int jn = min(SOLVE_RCH / 2, b - j0);
#pragma unroll 8
        for (int jj = 0; jj < SOLVE_RCH / 2; ++jj) {
          if (jj >= jn) break;
          const cplx<T> gv = sg[(half * (SOLVE_RCH / 2) + jj) * ldb + row];
#pragma unroll
          for (int rr = 0; rr < NR; ++rr)
            if (rr < nr) cfma(acc[rr], gv, ys[rr * bpad + j0 + jj]);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(empty0 + 8 * st);
    }
    if (half == 1 && row < b) {
#pragma unroll
      for (int rr = 0; rr < NR; ++rr) if (rr < nr) red[rr * bpad + row] = acc[rr];
    }
    consumer_sync();
    if (half == 0 && row < b) {
#pragma unroll
      for (int rr = 0; rr < NR; ++rr) {
        if (rr < nr) {
          const int sidx = rr * bpad + row;
          const cplx<T> v = acc[rr] + red[sidx];
          ts[sidx] = pass == 0 ? v : tk[sidx] - v;     // t_k, or x_k = t_k - G_k z
        }
      }
    }
    consumer_sync();
  }
  // flush the last block (backward k = 0)
#pragma unroll
  for (int q = 0; q < PI; ++q) {
    const int idx = tid + q * SOLVE_NCW * 32;
    if (idx < nitem) {
      const int rr = idx / b, j = idx - rr * b;
      const int sidx = rr * bpad + j;
      int pp, pk;
      seq_block(nblk - 1, m, pp, pk);
      const long long o = (long long)rr * lt + (long long)pk * b + j;
      outv[o] = ts[sidx];
      if (Uv) Uv[o] = uk[sidx] + ts[sidx];
    }
  }
}

template <typename T, int NR>
static cudaError_t solve_nr(ddm_ctx* c, const void* src, void* out, void* U, int nrhs) {
  constexpr int NST = sizeof(T) == 4 ? 6 : 4;
  int maxb = 0, maxm = 0, maxld = 0;
  for (auto& s : c->subs) { maxb = std::max(maxb, s.ext[0]); maxm = std::max(maxm, s.ext[1]); maxld = std::max(maxld, s.pad); }
  const int bpad = (maxb + 3) & ~3;
  size_t el = sizeof(cplx<T>);
  size_t sm = (size_t)NST * SOLVE_RCH * maxld * el + (size_t)5 * NR * bpad * el + 16 + 2 * NST * 8 + 16;
  cudaError_t e = cudaFuncSetAttribute(k_solve2d<T, NR, NST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  dim3 grid(c->g.nsub, (nrhs + NR - 1) / NR);
  ++c->nlaunch;
  k_solve2d<T, NR, NST><<<grid, SOLVE_THREADS, sm, c->st>>>(c->g, (const cplx<T>*)c->d_G, (const cplx<T>*)src,
                                                           (cplx<T>*)out, (cplx<T>*)U, nrhs, c->d_err);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t solve_t(ddm_ctx* c, const void* src, void* out, void* U, int nrhs) {
  if (nrhs >= 8 && sizeof(T) == 4) return solve_nr<T, 8>(c, src, out, U, nrhs);
  if (nrhs >= 4) return solve_nr<T, 4>(c, src, out, U, nrhs);
  if (nrhs >= 2) return solve_nr<T, 2>(c, src, out, U, nrhs);
  return solve_nr<T, 1>(c, src, out, U, nrhs);
}

cudaError_t launch_local_solve(ddm_ctx* c, const void* src, void* out, void* accum, int nrhs) {
  return c->prec == DDM_MIXED ? solve_t<float>(c, src, out, accum, nrhs) : solve_t<double>(c, src, out, accum, nrhs);
}

}  // namespace ddm

// Batched block-tridiagonal solves u_R = A_R^{-1} src_R over all subdomains and right-hand
// sides (the local solves of Algorithm 3.1, Eqs. (talg_1)/(talg_2)).
//
// With G_k = D_k^{-1} from factor.cu:
//   forward   y_k = r_k - c_S(., k) * t_{k-1},   t_k = G_k y_k            (k = 0..m-1)
//   backward  x_{m-1} = t_{m-1},  x_k = t_k - G_k (c_N(., k) * x_{k+1})    (k = m-2..0)
// so every G_k is streamed from HBM twice per solve (once per sweep) and applied to NR
// right-hand sides at once.  One CTA per (subdomain, group of NR right-hand sides):
// warp 8 is the producer, copying row chunks of G_k into a ring of shared-memory stages with
// cp.async.bulk (1D TMA) on mbarriers; warps 0-7 consume the stages (each warp two rows of
// a 16-row chunk, lanes across columns, shuffle reduction).  Waits are bounded: on time-out
// the kernel records ERRBIT_TIMEOUT and runs to completion without hanging.
#include <algorithm>

#include "ddm_internal.cuh"

namespace ddm {

constexpr int SOLVE_NCW = 8;     // consumer warps
constexpr int SOLVE_RPW = 2;     // rows per warp per chunk
constexpr int SOLVE_RCH = SOLVE_NCW * SOLVE_RPW;
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

  cplx<T>* stage = (cplx<T>*)smem;                                   // NST x RCH x ldb
  cplx<T>* ys = stage + (size_t)NST * SOLVE_RCH * ldb;               // NR x bpad
  cplx<T>* ts = ys + NR * bpad;                                      // NR x bpad
  cplx<T>* ax = ts + NR * bpad;                                      // b: alpha_x at nodes
  cplx<T>* aiy = ax + bpad;                                          // m+1: 1/alpha_y at half nodes
  uint64_t* bars = (uint64_t*)(((uintptr_t)(aiy + m + 1) + 15) & ~(uintptr_t)15);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + NST);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < NST; ++i) { mbar_init(full0 + 8 * i, 1); mbar_init(empty0 + 8 * i, SOLVE_NCW); }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int j = tid; j < b; j += blockDim.x) ax[j] = ccast<T>(tab_node(g, s.tab[0], j));
  for (int k = tid; k <= m; k += blockDim.x) aiy[k] = ccast<T>(tab_ihalf(g, s.tab[1], m, k));
  __syncthreads();

  const long long total_chunks = (long long)(2 * m - 1) * nch;
  if (warp == SOLVE_NCW) {
    // ---------------- producer ----------------
    if (lane == 0) {
      long long c = 0;
      for (int pass = 0; pass < 2; ++pass) {
        const int nblk = pass == 0 ? m : m - 1;
        for (int bi = 0; bi < nblk; ++bi) {
          const int k = pass == 0 ? bi : (m - 2 - bi);
          for (int ch = 0; ch < nch; ++ch, ++c) {
            const int st = (int)(c % NST);
            if (c >= NST) mbar_wait(empty0 + 8 * st, (uint32_t)((c / NST - 1) & 1), err);
            const int rows = min(SOLVE_RCH, b - ch * SOLVE_RCH);
            const uint32_t bytes = (uint32_t)(rows * ldb * (int)sizeof(cplx<T>));
            mbar_expect_tx(full0 + 8 * st, bytes);
            bulk_g2s(smem_u32(stage + (size_t)st * SOLVE_RCH * ldb),
                     G + s.fofs + ((long long)k * b + ch * SOLVE_RCH) * ldb, bytes, full0 + 8 * st);
          }
        }
      }
      // wait (bounded) for the last copy of every stage before the CTA may exit
      for (long long cc = max(0LL, total_chunks - NST); cc < total_chunks; ++cc)
        mbar_wait(full0 + 8 * (int)(cc % NST), (uint32_t)((cc / NST) & 1), err);
    }
    return;
  }

  // ---------------- consumers ----------------
  const long long lt = g.ltotal;
  const cplx<T>* srcv = src + (long long)r0 * lt + s.vofs;
  cplx<T>* outv = out + (long long)r0 * lt + s.vofs;
  cplx<T>* Uv = U ? U + (long long)r0 * lt + s.vofs : nullptr;
  const int ctid = tid;   // 0 .. 255
  long long c = 0;
  for (int pass = 0; pass < 2; ++pass) {
    const int nblk = pass == 0 ? m : m - 1;
    for (int bi = 0; bi < nblk; ++bi) {
      const int k = pass == 0 ? bi : (m - 2 - bi);
      // right-hand side of this block: forward y_k = r_k - c_S(., k) t_{k-1};
      // backward z = c_N(., k) x_{k+1}, with c_S = alpha_x / alpha_y(k - 1/2), c_N = alpha_x / alpha_y(k + 1/2)
      for (int idx = ctid; idx < nr * b; idx += SOLVE_NCW * 32) {
        const int rr = idx / b, j = idx - rr * b;
        cplx<T> v;
        if (pass == 0) {
          v = srcv[(long long)rr * lt + (long long)k * b + j];
          if (k > 0) v = v - (ax[j] * aiy[k]) * ts[rr * bpad + j];
        } else {
          v = (ax[j] * aiy[k + 1]) * ts[rr * bpad + j];
        }
        ys[rr * bpad + j] = v;
      }
      consumer_sync();
      for (int ch = 0; ch < nch; ++ch, ++c) {
        const int st = (int)(c % NST);
        mbar_wait(full0 + 8 * st, (uint32_t)((c / NST) & 1), err);
        const cplx<T>* sg = stage + (size_t)st * SOLVE_RCH * ldb;
#pragma unroll
        for (int q = 0; q < SOLVE_RPW; ++q) {
          const int lrow = warp * SOLVE_RPW + q;
          const int row = ch * SOLVE_RCH + lrow;
          if (row >= b) break;
          cplx<T> acc[NR];
#pragma unroll
          for (int rr = 0; rr < NR; ++rr) acc[rr] = mk<T>(0, 0);
          for (int j = lane; j < b; j += 32) {
            const cplx<T> gv = sg[lrow * ldb + j];
#pragma unroll
            for (int rr = 0; rr < NR; ++rr)
              if (rr < nr) cfma(acc[rr], gv, ys[rr * bpad + j]);
          }
#pragma unroll
          for (int rr = 0; rr < NR; ++rr) {
            for (int o = 16; o; o >>= 1) {
              acc[rr].x += __shfl_xor_sync(0xffffffffu, acc[rr].x, o);
              acc[rr].y += __shfl_xor_sync(0xffffffffu, acc[rr].y, o);
            }
          }
          if (lane == 0) {
            for (int rr = 0; rr < nr; ++rr) {
              const long long o = (long long)rr * lt + (long long)k * b + row;
              cplx<T> v = acc[rr];
              if (pass == 1) v = outv[o] - v;      // x_k = t_k - G_k z
              outv[o] = v;
              ts[rr * bpad + row] = v;
              if (Uv && (pass == 1 || k == m - 1)) Uv[o] = Uv[o] + v;
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty0 + 8 * st);
      }
      consumer_sync();
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
  size_t sm = (size_t)NST * SOLVE_RCH * maxld * el + (2 * NR * bpad + bpad + maxm + 1) * el + 16 + 2 * NST * 8 + 16;
  cudaError_t e = cudaFuncSetAttribute(k_solve2d<T, NR, NST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  dim3 grid(c->g.nsub, (nrhs + NR - 1) / NR);
  k_solve2d<T, NR, NST><<<grid, SOLVE_THREADS, sm, c->st>>>(c->g, (const cplx<T>*)c->d_G, (const cplx<T>*)src,
                                                           (cplx<T>*)out, (cplx<T>*)U, nrhs, c->d_err);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t solve_t(ddm_ctx* c, const void* src, void* out, void* U, int nrhs) {
  if (nrhs >= 8) return solve_nr<T, 8>(c, src, out, U, nrhs);
  if (nrhs >= 4) return solve_nr<T, 4>(c, src, out, U, nrhs);
  if (nrhs >= 2) return solve_nr<T, 2>(c, src, out, U, nrhs);
  return solve_nr<T, 1>(c, src, out, U, nrhs);
}

cudaError_t launch_local_solve(ddm_ctx* c, const void* src, void* out, void* accum, int nrhs) {
  return c->prec == DDM_MIXED ? solve_t<float>(c, src, out, accum, nrhs) : solve_t<double>(c, src, out, accum, nrhs);
}

}  // namespace ddm

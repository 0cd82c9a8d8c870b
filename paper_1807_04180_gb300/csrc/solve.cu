// Batched block-tridiagonal solves u_R = A_R^{-1} src_R over all subdomains and right-hand
// sides (the local solves of Algorithm 3.1, Eqs. (37)/(38)).
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
#include <map>
#include <mutex>
#include <tuple>

#include "ddm_internal.cuh"

namespace ddm {

constexpr int SOLVE_NCW = 8;     // consumer warps
constexpr int SOLVE_RCH = 16;    // columns of G_k per pipeline chunk
constexpr int SOLVE_THREADS = (SOLVE_NCW + 1) * 32;
// bounded waits: each try_wait may suspend the thread up to WAIT_HINT_NS until the phase
// completes; WAIT_LIMIT tries (about 4 s at most) before giving up
constexpr long long WAIT_LIMIT = 1LL << 18;
constexpr uint32_t WAIT_HINT_NS = 16384;

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
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity), "r"(WAIT_HINT_NS)
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

template <typename T, int NR>
__global__ void __launch_bounds__(SOLVE_THREADS) k_solve2d(Geom g, const cplx<T>* __restrict__ G,
                                                          const cplx<T>* __restrict__ src, cplx<T>* out,
                                                          cplx<T>* U, int nrhs, int nst, int* err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const SubDesc& s = g.subs[blockIdx.x];
  const int b = s.ext[0], m = s.ext[1], ldb = s.pad;
  const int bpad = (b + 3) & ~3;
  const int r0 = blockIdx.y * NR;
  const int nr = min(NR, nrhs - r0);
  const int nch = (b + SOLVE_RCH - 1) / SOLVE_RCH;
  const int nblk = 2 * m - 1;

  cplx<T>* stage = (cplx<T>*)smem;                                   // nst x RCH x ldb
  cplx<T>* ys = stage + (size_t)nst * SOLVE_RCH * ldb;               // NR x bpad: right-hand side of the block GEMV
  cplx<T>* red = ys + NR * bpad;                                     // NR x bpad: second-half partial sums
  uint64_t* bars = (uint64_t*)(((uintptr_t)(red + NR * bpad) + 15) & ~(uintptr_t)15);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + nst);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < nst; ++i) { mbar_init(full0 + 8 * i, 1); mbar_init(empty0 + 8 * i, SOLVE_NCW); }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == SOLVE_NCW) {
    // ---------------- producer: column chunks of G_k in consumption order ----------------
    if (lane == 0) {
      int st = 0;
      uint32_t ph = 0;            // phase of the current pass over the ring
      long long c = 0;
      for (int i = 0; i < nblk; ++i) {
        int pass, k;
        seq_block(i, m, pass, k);
        for (int ch = 0; ch < nch; ++ch, ++c) {
          if (c >= nst) mbar_wait(empty0 + 8 * st, ph ^ 1u, err);
          const int cols = min(SOLVE_RCH, b - ch * SOLVE_RCH);
          const uint32_t bytes = (uint32_t)(cols * ldb * (int)sizeof(cplx<T>));
          mbar_expect_tx(full0 + 8 * st, bytes);
          bulk_g2s(smem_u32(stage + (size_t)st * SOLVE_RCH * ldb),
                   G + s.fofs + ((long long)k * b + ch * SOLVE_RCH) * ldb, bytes, full0 + 8 * st);
          if (++st == nst) { st = 0; ph ^= 1u; }
        }
      }
      // bounded wait for the copies still in flight before the CTA may exit
      const long long total = (long long)nblk * nch;
      for (long long cc = max(0LL, total - nst); cc < total; ++cc)
        mbar_wait(full0 + 8 * (int)(cc % nst), (uint32_t)((cc / nst) & 1), err);
    }
    return;
  }

  // ---------------- consumers ----------------
  // thread (half, row): half 0 owns row `row` of every block vector (epilogue, next right-hand
  // side, prefetch); both halves accumulate the GEMV over their half of each chunk.
  const int row = tid & 127, half = tid >> 7;
  const bool owner = half == 0 && row < b;
  const long long len = (long long)b * m;
  const long long lt = len;   // right-hand sides of one subdomain are adjacent (lvofs)
  const cplx<T>* srcv = src + lvofs(s, r0, nrhs);
  cplx<T>* outv = out + lvofs(s, r0, nrhs);
  cplx<T>* Uv = U ? U + lvofs(s, r0, nrhs) : nullptr;
  const cplx<T>* lc = (const cplx<T>*)g.lcoef + s.vofs * 5;      // planes: C, W, E, S, N
  const cplx<T>* cSp = lc + 3 * len;
  const cplx<T>* cNp = lc + 4 * len;
  // per-row registers: prefetched values of the next block (pa: src_k or t_k, pb: U_k,
  // pc: c_S(k) or c_N(k)), the current block's t_k (tk) and U_k (uk), and the last output t
  cplx<T> pa[NR], pb[NR], tk[NR], uk[NR], tv[NR];
  cplx<T> pc = mk<T>(0, 0);
  auto load_block = [&](int i) {
    int pass, k;
    seq_block(i, m, pass, k);
    const long long o = (long long)k * b + row;
    pc = pass == 0 ? (k > 0 ? cSp[o] : mk<T>(0, 0)) : cNp[o];
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) {
      if (rr < nr) {
        const long long oo = (long long)rr * lt + o;
        pa[rr] = pass == 0 ? srcv[oo] : outv[oo];
        pb[rr] = (Uv && (pass == 1 || k == m - 1)) ? Uv[oo] : mk<T>(0, 0);
      }
    }
  };
  // right-hand side of block i from the prefetched values and the previous output tv:
  // forward y_k = r_k - c_S(., k) t_{k-1}; backward z = c_N(., k) x_{k+1}
  auto form_rhs = [&](int i) {
    int pass, k;
    seq_block(i, m, pass, k);
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) {
      if (rr < nr) {
        cplx<T> y;
        if (pass == 0) {
          y = pa[rr];
          if (k > 0) y = y - pc * tv[rr];
        } else {
          y = pc * tv[rr];
          tk[rr] = pa[rr];
        }
        uk[rr] = pb[rr];
        ys[rr * bpad + row] = y;
      }
    }
  };
  if (owner) {
    load_block(0);
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) tv[rr] = mk<T>(0, 0);
    form_rhs(0);
    if (nblk > 1) load_block(1);
  }
  consumer_sync();
  int st = 0;
  uint32_t ph = 0;
  for (int i = 0; i < nblk; ++i) {
    int pass, k;
    seq_block(i, m, pass, k);
    cplx<T> acc[NR];
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) acc[rr] = mk<T>(0, 0);
    for (int ch = 0; ch < nch; ++ch) {
      mbar_wait(full0 + 8 * st, ph, err);
      const cplx<T>* sg = stage + (size_t)st * SOLVE_RCH * ldb;   // columns ch*16 .. ch*16+15
      if (row < b) {
        const int j0 = ch * SOLVE_RCH + half * (SOLVE_RCH / 2);
        const int jn = min(SOLVE_RCH / 2, b - j0);
        const cplx<T>* gcol = sg + (half * (SOLVE_RCH / 2)) * ldb + row;
        if (jn == SOLVE_RCH / 2) {     // full half-chunk: straight-line, loads hoisted
          cplx<T> gv[SOLVE_RCH / 2];
#pragma unroll
          for (int jj = 0; jj < SOLVE_RCH / 2; ++jj) gv[jj] = gcol[jj * ldb];
#pragma unroll
          for (int jj = 0; jj < SOLVE_RCH / 2; ++jj)
#pragma unroll
            for (int rr = 0; rr < NR; ++rr)
              if (rr < nr) cfma(acc[rr], gv[jj], ys[rr * bpad + j0 + jj]);
        } else {
          for (int jj = 0; jj < jn; ++jj) {
            const cplx<T> gv = gcol[jj * ldb];
#pragma unroll
            for (int rr = 0; rr < NR; ++rr)
              if (rr < nr) cfma(acc[rr], gv, ys[rr * bpad + j0 + jj]);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(empty0 + 8 * st);
      if (++st == nst) { st = 0; ph ^= 1u; }
    }
    if (half == 1 && row < b) {
#pragma unroll
      for (int rr = 0; rr < NR; ++rr) if (rr < nr) red[rr * bpad + row] = acc[rr];
    }
    consumer_sync();
    if (owner) {
#pragma unroll
      for (int rr = 0; rr < NR; ++rr) {
        if (rr < nr) {
          const cplx<T> v = acc[rr] + red[rr * bpad + row];
          tv[rr] = pass == 0 ? v : tk[rr] - v;                     // t_k, or x_k = t_k - G_k z
          const long long o = (long long)rr * lt + (long long)k * b + row;
          outv[o] = tv[rr];
          if (Uv && (pass == 1 || k == m - 1)) Uv[o] = uk[rr] + tv[rr];
        }
      }
      if (i + 1 < nblk) {
        form_rhs(i + 1);
        if (i + 2 < nblk) load_block(i + 2);
      }
    }
    consumer_sync();
  }
}

template <typename T, int NR>
static cudaError_t solve_nr(ddm_ctx* c, const void* src, void* out, void* U, int nrhs) {
  int maxb = 0, maxld = 0;
  for (auto& s : c->subs) { maxb = std::max(maxb, s.ext[0]); maxld = std::max(maxld, s.pad); }
  const int bpad = (maxb + 3) & ~3;
  const size_t el = sizeof(cplx<T>);
  const size_t fixed = (size_t)2 * NR * bpad * el + 16 + 2 * 32 * 8 + 16;
  const size_t stage = (size_t)SOLVE_RCH * maxld * el;
  int dev = 0, nsm = 152, smem_sm = 228 * 1024, smem_blk = 227 * 1024;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&smem_blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // CTAs per SM: what the grid needs, capped by what registers allow
  int reg_cap = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&reg_cap, k_solve2d<T, NR>, SOLVE_THREADS, 0);
  const long long ctas = (long long)c->g.nsub * ((nrhs + NR - 1) / NR);
  int per_sm = (int)std::min<long long>(4, std::max<long long>(1, (ctas + nsm - 1) / nsm));
  if (reg_cap > 0) per_sm = std::min(per_sm, reg_cap);
  // as many pipeline stages as fit with per_sm CTAs resident
  size_t budget = std::min<size_t>((size_t)smem_blk, (size_t)smem_sm / per_sm - 1024);
  int nst = (int)std::min<size_t>(32, budget > fixed ? (budget - fixed) / stage : 0);
  nst = std::max(nst, 2);
  const size_t sm = fixed + (size_t)nst * stage;
  cudaError_t e = allow_dynamic_smem((const void*)k_solve2d<T, NR>, sm);
  if (e != cudaSuccess) return e;
  dim3 grid(c->g.nsub, (nrhs + NR - 1) / NR);
  ++c->nlaunch;
  k_solve2d<T, NR><<<grid, SOLVE_THREADS, sm, c->st>>>(c->g, (const cplx<T>*)c->d_G, (const cplx<T>*)src,
                                                     (cplx<T>*)out, (cplx<T>*)U, nrhs, nst, c->d_err);
  return cudaGetLastError();
}

// nr <= 8: CUDA-core kernel with nr right-hand sides per CTA; nr = 64: tensor-core kernel
// (complex64 with a packed factor only), 64 right-hand sides per CTA
template <typename T>
static cudaError_t solve_with(ddm_ctx* c, int nr, const void* src, void* out, void* U, int nrhs) {
  if (nr > 8) return tc2d_solve(c, nr, src, out, U, nrhs);
  switch (nr) {
    case 8: return solve_nr<T, 8>(c, src, out, U, nrhs);
    case 4: return solve_nr<T, 4>(c, src, out, U, nrhs);
    case 2: return solve_nr<T, 2>(c, src, out, U, nrhs);
    default: return solve_nr<T, 1>(c, src, out, U, nrhs);
  }
}

// Kernel and right-hand sides per CTA for nrhs right-hand sides: measured once by timing every
// candidate on the call's own source into a scratch output, then cached.
// CUDA-core candidates: 1, 2, 4, 8 (8 only in complex64) right-hand sides per CTA -- more read
// each factor block fewer times but raise the registers per thread, which can cut the CTAs per
// SM.  Tensor-core candidate (complex64, packed factor, tensor cores enabled, nrhs >= 8): 64 per CTA.
// Choices are also shared across contexts of the process, keyed by the subdomain geometry, the
// precision, the tensor-core setting and nrhs: a later context with the same shapes (a served
// request, say) reuses the choice instead of timing again, possibly under other contexts' load,
// so the same shapes always run the same kernels (and give the same bits).
static std::mutex g_tune_mu;
static std::map<std::tuple<unsigned long long, int, int>, int> g_tune;

static unsigned long long geometry_key(const ddm_ctx* c) {
  unsigned long long h = 0x9E3779B97F4A7C15ull ^ (unsigned long long)c->dim ^ ((unsigned long long)c->prec << 8);
  auto mix = [&](unsigned long long v) {
    h ^= v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
  };
  mix((unsigned long long)c->g.nsub);
  for (const auto& s : c->subs) mix(((unsigned long long)s.ext[0] << 40) ^ ((unsigned long long)s.ext[1] << 20) ^ s.ext[2]);
  return h;
}

template <typename T>
static cudaError_t solve_t(ddm_ctx* c, const void* src, void* out, void* U, int nrhs) {
  if (nrhs == 1) return solve_nr<T, 1>(c, src, out, U, 1);
  const bool tc = sizeof(T) == 4 && c->use_tc && c->d_gtc2;
  if (c->forced_nr > 0 && (c->forced_nr <= 8 || tc)) return solve_with<T>(c, c->forced_nr, src, out, U, nrhs);
  const int key = tc ? nrhs : -nrhs;   // cached choices with and without the tensor cores
  auto it = c->tuned_nr.find(key);
  const auto gkey = std::make_tuple(geometry_key(c), key, (int)sizeof(T));
  if (it == c->tuned_nr.end()) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto g = g_tune.find(gkey);
    if (g != g_tune.end()) it = c->tuned_nr.emplace(key, g->second).first;
  }
  if (it == c->tuned_nr.end()) {
    // scratch output and accumulator: the candidates are timed with the accumulation the DDM
    // steps ask for
    void* scratch = nullptr;
    cudaError_t e = dev_alloc(c, &scratch, 2 * sizeof(cplx<T>) * c->g.ltotal * nrhs);
    if (e != cudaSuccess) return e;
    void* uscratch = (char*)scratch + sizeof(cplx<T>) * c->g.ltotal * nrhs;
    cudaMemsetAsync(uscratch, 0, sizeof(cplx<T>) * c->g.ltotal * nrhs, c->st);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = 1;
    float best_ms = 1e30f;
    for (int nr : {1, 2, 4, 8, 64}) {
      if (nr == 8 && sizeof(T) != 4) continue;
      if (nr <= 8 && nr > nrhs) continue;
      if (nr > 8 && (!tc || nrhs < 8 || !tc2d_supported(c, nr))) continue;
      if ((e = solve_with<T>(c, nr, src, scratch, uscratch, nrhs)) != cudaSuccess) break;   // warm
      cudaEventRecord(e0, c->st);
      if ((e = solve_with<T>(c, nr, src, scratch, uscratch, nrhs)) != cudaSuccess) break;
      cudaEventRecord(e1, c->st);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      c->tune_log.push_back({nrhs, nr, ms});
      if (ms < best_ms) { best_ms = ms; best = nr; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dev_free(c, scratch);
    if (e != cudaSuccess) return e;
    // a context that tuned the same shapes at the same time may have been first: use its choice
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const int chosen = g_tune.emplace(gkey, best).first->second;
    it = c->tuned_nr.emplace(key, chosen).first;
  }
  return solve_with<T>(c, it->second, src, out, U, nrhs);
}

cudaError_t launch_local_solve(ddm_ctx* c, const void* src, void* out, void* accum, int nrhs) {
  if (c->blockpath) return launch_local_solve3d(c, src, out, accum, nrhs);
  return c->prec == DDM_MIXED ? solve_t<float>(c, src, out, accum, nrhs) : solve_t<double>(c, src, out, accum, nrhs);
}

}  // namespace ddm

// Tensor-core (tcgen05) 2D local solves for many right-hand sides (mixed precision).
//
// The block solves of Algorithm 3.1 in 2D (x-lines as blocks, G_k = D_k^{-1} from factor.cu):
//   forward   y_k = r_k - c_S(., k) t_{k-1},  t_k = G_k y_k            (k = 0..m-1)
//   backward  x_{m-1} = t_{m-1},  x_k = t_k - G_k (c_N(., k) x_{k+1})   (k = m-2..0)
// With NRT right-hand sides per CTA every block step is a complex contraction of the b x b block
// G_k with a b x NRT operand, here on the 5th-generation tensor cores in split TF32 ("3xTF32",
// FP32 accumulation in tensor memory, FP32-level accuracy).  One CTA per (subdomain, group of NRT
// right-hand sides; the groups of a subdomain adjacent in launch order) runs the whole sweep:
//  - warp 8 (producer) streams the packed factor, chunk by chunk in consumption order, through a
//    ring of shared-memory stages with cp.async.bulk;
//  - warp 9 issues, per K step of 8 columns, six MMAs M = 128 (rows of G_k) x N = 2 NRT
//    ([Re y | Im y]) x K = 8:  P += Gr [Yr|Yi],  Q += Gi [Yr|Yi]  (hi*hi + hi*lo + lo*hi each),
//    so Re(G y) = P[Yr] - Q[Yi] and Im(G y) = P[Yi] + Q[Yr];
//  - warps 0-7 (two per TMEM lane quarter, each with half of the right-hand sides) read P and Q
//    back, apply the sweep's update to the local vectors, and write the next block's operand
//    (split into hi/lo planes) into shared memory; the values they need for the next block are
//    loaded while the tensor core works on the current one.
// Waits are bounded; a time-out sets ERRBIT_TIMEOUT and every role leaves its loop.
#include <algorithm>
#include <vector>

#include "ddm_internal.cuh"
#include "tcgen05.cuh"

namespace ddm {

constexpr int TC2_KC = 16;                        // K (columns j of G_k) per pipeline chunk
constexpr int TC2_NEPI = 8;                       // epilogue warps
constexpr int TC2_THREADS = (TC2_NEPI + 2) * 32;  // + producer warp + MMA warp
constexpr int TC2_MAXST = 8;
// K-direction stride of the operand's core matrices: 144 bytes (128 + 16 of padding) makes the
// epilogue's writes of one column of the operand (consecutive j) hit 32 distinct banks
constexpr uint32_t TC2_LBOY = 144;
// the M = 128 MMA reads 16 row groups of a factor plane; rows past b read whatever follows
// (their output rows are discarded), so the ring is followed by this much slack
constexpr uint32_t TC2_TAIL = 8192;

long long tc2d_packed_floats(int b, int m) {
  const long long ng = (b + 7) / 8, nKC = (b + TC2_KC - 1) / TC2_KC;
  return (long long)m * nKC * 4 * ng * 4 * 32;
}

struct TC2Fac { long long fofs, tofs; int b, m, ldb, pad; };

// packed factor: per block k and chunk kc (16 columns j) the planes {Re hi, Re lo, Im hi, Im lo},
// each ng row groups x 4 core matrices along K x (8 rows x 4 floats), contiguous
__global__ void k_g2_pack(const TC2Fac* __restrict__ facs, const c32* __restrict__ G, float* __restrict__ dst) {
  const TC2Fac f = facs[blockIdx.y];
  const int ng = (f.b + 7) / 8, nKC = (f.b + TC2_KC - 1) / TC2_KC;
  const long long nI = (long long)ng * 8, nJ = (long long)nKC * TC2_KC;
  const long long total = (long long)f.m * nJ * nI;
  float* out = dst + f.tofs;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % nI);
    const long long r = idx / nI;
    const int j = (int)(r % nJ);
    const int k = (int)(r / nJ);
    c32 v = mk<float>(0.f, 0.f);
    if (i < f.b && j < f.b) v = G[f.fofs + ((long long)k * f.b + j) * f.ldb + i];
    float rh, rl, ih, il;
    tc::split_tf32(v.x, rh, rl);
    tc::split_tf32(v.y, ih, il);
    const int kc = j / TC2_KC, jj = j % TC2_KC;
    float* chunk = out + ((long long)k * nKC + kc) * 512 * ng;
    const int e = ((i >> 3) * 4 + (jj >> 2)) * 32 + (i & 7) * 4 + (jj & 3);
    const long long ps = 128LL * ng;
    chunk[e] = rh;
    chunk[ps + e] = rl;
    chunk[2 * ps + e] = ih;
    chunk[3 * ps + e] = il;
  }
}

__device__ __forceinline__ void seq2(int bi, int m, int& pass, int& k) {
  pass = bi < m ? 0 : 1;
  k = pass == 0 ? bi : 2 * m - 2 - bi;
}

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"r"(TC2_NEPI * 32) : "memory"); }
__device__ __forceinline__ bool epi_any(bool p) {
  uint32_t r;
  asm volatile("{\n .reg .pred q, o;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred o, 1, %2, q;\n selp.u32 %0, 1, 0, o;\n}\n"
               : "=r"(r)
               : "r"((uint32_t)p), "r"(TC2_NEPI * 32)
               : "memory");
  return r != 0;
}

template <int NRT>
__global__ void __launch_bounds__(TC2_THREADS, 1)
    k_solve2d_tc(Geom g, const float* __restrict__ gtc, const long long* __restrict__ tcofs,
                 const c32* __restrict__ src, c32* out, c32* U, int nrhs, int nst, int* err) {
  constexpr int N = 2 * NRT;          // MMA N: [Re y | Im y]
  constexpr int NH = NRT / 2;         // right-hand sides per epilogue thread
  constexpr uint32_t TCOLS = 4 * NRT; // P: columns [0, N), Q: [N, 2N)
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t s_full[TC2_MAXST], s_empty[TC2_MAXST], s_yfull, s_dfull;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  volatile int* abort_flag = &s_abort;

  // the right-hand-side groups of one subdomain are adjacent in launch order, so that they run
  // at the same time and the second read of each factor block hits L2
  const SubDesc& s = g.subs[blockIdx.y];
  const int b = s.ext[0], m = s.ext[1];
  const int ng = (b + 7) / 8, nKC = (b + TC2_KC - 1) / TC2_KC, Kpad = nKC * TC2_KC;
  const int nblk = 2 * m - 1;
  const int r0 = blockIdx.x * NRT, nr = min(NRT, nrhs - r0);
  const uint32_t SBOY = (uint32_t)(Kpad / 4) * TC2_LBOY;   // 8-row group stride of the operand
  const uint32_t YPLANE = (uint32_t)(N / 8) * SBOY;        // one operand plane (hi or lo)
  const uint32_t STAGE = 2048u * (uint32_t)ng;              // one chunk: 4 planes x ng x 512 bytes
  const uint32_t raw = tc::smem_addr(smem_raw);
  const uint32_t ybase = (raw + 127u) & ~127u;
  const uint32_t ring = ybase + 2 * YPLANE;
  unsigned char* ygen = smem_raw + (ybase - raw);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(&s_tmem), TCOLS);
  if (tid == 0) {
    for (int i = 0; i < nst; ++i) {
      tc::bar_init(tc::smem_addr(&s_full[i]), 1);
      tc::bar_init(tc::smem_addr(&s_empty[i]), 1);
    }
    tc::bar_init(tc::smem_addr(&s_yfull), 1);
    tc::bar_init(tc::smem_addr(&s_dfull), 1);
    s_abort = 0;
    tc::bar_init_fence();
  }
  // the operand planes start at zero: their K padding (rows j >= b) must stay finite
  for (uint32_t o = (uint32_t)tid * 16; o < 2 * YPLANE; o += TC2_THREADS * 16)
    *reinterpret_cast<float4*>(ygen + o) = make_float4(0.f, 0.f, 0.f, 0.f);
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = s_tmem;

  if (warp == TC2_NEPI) {
    // ------------------------------------------------------------------ producer
    if (lane == 0) {
      const float* gsrc = gtc + tcofs[s.fid];
      long long c = 0;
      for (int bi = 0; bi < nblk && !*abort_flag; ++bi) {
        int pass, k;
        seq2(bi, m, pass, k);
        for (int kc = 0; kc < nKC; ++kc, ++c) {
          const int st = (int)(c % nst);
          if (c >= nst && !tc::bar_wait_or_abort(tc::smem_addr(&s_empty[st]), (uint32_t)((c / nst) - 1) & 1u,
                                                   abort_flag)) {
            atomicOr(err, ERRBIT_TIMEOUT);
            break;
          }
          const uint32_t fb = tc::smem_addr(&s_full[st]);
          tc::bar_expect_tx(fb, STAGE);
          tc::bulk_load(ring + (uint32_t)st * STAGE, gsrc + ((long long)k * nKC + kc) * 512 * ng, STAGE, fb);
        }
      }
      // the copies still in flight land before the CTA may exit (bounded)
      for (long long cc = c > nst ? c - nst : 0; cc < c; ++cc)
        tc::bar_wait(tc::smem_addr(&s_full[cc % nst]), (uint32_t)((cc / nst) & 1));
    }
  } else if (warp == TC2_NEPI + 1) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t ID = tc::idesc_tf32(128, N, false);
      const uint32_t accP = tmem, accQ = tmem + N;
      const uint32_t PL = 512u * (uint32_t)ng;   // factor plane stride in a stage
      long long c = 0;
      bool ok = true;
      for (int bi = 0; bi < nblk && ok; ++bi) {
        if (!tc::bar_wait_or_abort(tc::smem_addr(&s_yfull), (uint32_t)(bi & 1), abort_flag)) { ok = false; break; }
        tc::fence_after();
        for (int kc = 0; kc < nKC; ++kc, ++c) {
          const int st = (int)(c % nst);
          if (!tc::bar_wait_or_abort(tc::smem_addr(&s_full[st]), (uint32_t)((c / nst) & 1), abort_flag)) {
            ok = false;
            break;
          }
          tc::fence_after();
          const uint32_t g0 = ring + (uint32_t)st * STAGE;
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            const int ks = 2 * kc + t;
            if (8 * ks >= b) break;                   // K step entirely in the padding
            const uint32_t acc = ks > 0 ? 1u : 0u;
            const uint64_t Grh = tc::sdesc(g0 + t * 256, 128, 512), Grl = tc::sdesc(g0 + PL + t * 256, 128, 512);
            const uint64_t Gih = tc::sdesc(g0 + 2 * PL + t * 256, 128, 512);
            const uint64_t Gil = tc::sdesc(g0 + 3 * PL + t * 256, 128, 512);
            const uint32_t ya = ybase + (uint32_t)ks * 2 * TC2_LBOY;
            const uint64_t Yh = tc::sdesc(ya, TC2_LBOY, SBOY), Yl = tc::sdesc(ya + YPLANE, TC2_LBOY, SBOY);
            tc::mma_tf32(accP, Grh, Yh, ID, acc);
            tc::mma_tf32(accP, Grh, Yl, ID, 1u);
            tc::mma_tf32(accP, Grl, Yh, ID, 1u);
            tc::mma_tf32(accQ, Gih, Yh, ID, acc);
            tc::mma_tf32(accQ, Gih, Yl, ID, 1u);
            tc::mma_tf32(accQ, Gil, Yh, ID, 1u);
          }
          tc::mma_commit(tc::smem_addr(&s_empty[st]));
        }
        if (!ok) break;
        tc::mma_commit(tc::smem_addr(&s_dfull));
      }
      if (!ok) atomicOr(err, ERRBIT_TIMEOUT);
    }
  } else {
    // ------------------------------------------------------------------ epilogue warps 0-7
    const int i = (warp & 3) * 32 + lane;           // row of the block (TMEM lane)
    const int hh = warp >> 2;                        // right-hand-side half
    const bool rowok = i < b;
    const uint32_t lanebase = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    const long long lt = g.ltotal, len = (long long)b * m;
    const c32* lc = (const c32*)g.lcoef + s.vofs * 5;   // planes: C, W, E, S, N
    const c32* cSp = lc + 3 * len;
    const c32* cNp = lc + 4 * len;
    const c32* srcv = src + (long long)r0 * lt + s.vofs;
    c32* outv = out + (long long)r0 * lt + s.vofs;
    c32* Uv = U ? U + (long long)r0 * lt + s.vofs : nullptr;
    const int rh0 = hh * NH;                          // first right-hand side of this thread
    auto put = [&](int r, c32 y) {                    // operand element (row r, column j = i)
      float yrh, yrl, yih, yil;
      tc::split_tf32(y.x, yrh, yrl);
      tc::split_tf32(y.y, yih, yil);
      const uint32_t jo = (uint32_t)(i >> 2) * TC2_LBOY + (uint32_t)(i & 3) * 4;
      const uint32_t ore = (uint32_t)(r >> 3) * SBOY + (uint32_t)(r & 7) * 16 + jo;
      const uint32_t oim = (uint32_t)((NRT + r) >> 3) * SBOY + (uint32_t)((NRT + r) & 7) * 16 + jo;
      *reinterpret_cast<float*>(ygen + ore) = yrh;
      *reinterpret_cast<float*>(ygen + YPLANE + ore) = yrl;
      *reinterpret_cast<float*>(ygen + oim) = yih;
      *reinterpret_cast<float*>(ygen + YPLANE + oim) = yil;
    };
    // block 0: y_0 = r_0
    if (rowok)
      for (int rr = 0; rr < NH; ++rr)
        if (rh0 + rr < nr) put(rh0 + rr, srcv[(long long)(rh0 + rr) * lt + i]);
    tc::fence_async_smem();
    epi_sync();
    if (tid == 0) tc::bar_arrive(tc::smem_addr(&s_yfull));
    // values the epilogue of block bi needs, loaded one block ahead:
    //   pass 0: pa = r_{k+1} (next block's source), pb = U_k at k = m-1
    //   pass 1: pa = t_k, pb = U_k;  pc = coupling of the next block's operand
    c32 pa[NH], pb[NH];
    c32 pc = mk<float>(0.f, 0.f);
    auto prefetch = [&](int bi) {
      int pass, k;
      seq2(bi, m, pass, k);
      const bool upd = Uv && (pass == 1 || k == m - 1);
      const long long o = (long long)k * b + i;
      if (rowok) {
        if (bi + 1 < nblk) pc = pass == 0 ? (k + 1 < m ? cSp[o + b] : cNp[o - b]) : cNp[o - b];
#pragma unroll
        for (int rr = 0; rr < NH; ++rr) {
          const long long ro = (long long)(rh0 + rr) * lt;
          const bool ok = rh0 + rr < nr;
          pa[rr] = (ok && (pass == 1 || k + 1 < m)) ? (pass == 0 ? srcv[ro + o + b] : outv[ro + o]) : mk<float>(0.f, 0.f);
          pb[rr] = (ok && upd) ? Uv[ro + o] : mk<float>(0.f, 0.f);
        }
      }
    };
    // the values of block bi + 2 are pulled into L2 while block bi + 1's are loaded
    auto prefetch_l2 = [&](int bi) {
      if (bi >= nblk || !rowok) return;
      int pass, k;
      seq2(bi, m, pass, k);
      const long long o = (long long)k * b + i;
      const bool upd = Uv && (pass == 1 || k == m - 1);
#pragma unroll
      for (int rr = 0; rr < NH; ++rr) {
        if (rh0 + rr >= nr) break;
        const long long ro = (long long)(rh0 + rr) * lt;
        if (pass == 1) tc::prefetch_l2(outv + ro + o);
        else if (k + 1 < m) tc::prefetch_l2(srcv + ro + o + b);
        if (upd) tc::prefetch_l2(Uv + ro + o);
      }
    };
    prefetch(0);
    prefetch_l2(1);
    for (int bi = 0; bi < nblk; ++bi) {
      int pass, k;
      seq2(bi, m, pass, k);
      // one thread waits for the accumulators; the others sleep in the barrier
      bool got = true;
      if (tid == 0) got = tc::bar_wait_or_abort(tc::smem_addr(&s_dfull), (uint32_t)(bi & 1), abort_flag);
      if (epi_any(!got)) break;
      tc::fence_after();
      const bool upd = Uv && (pass == 1 || k == m - 1);
      const bool more = bi + 1 < nblk;
      int npass = 0, nk = 0;
      if (more) seq2(bi + 1, m, npass, nk);
#pragma unroll
      for (int c0 = 0; c0 < NH; c0 += 8) {
        const uint32_t col = (uint32_t)(rh0 + c0);
        uint32_t pr[8], pim[8], qr[8], qim[8];
        tc::tmem_ld8_async(lanebase + col, pr);             // Gr Yr
        tc::tmem_ld8_async(lanebase + NRT + col, pim);      // Gr Yi
        tc::tmem_ld8_async(lanebase + N + col, qr);         // Gi Yr
        tc::tmem_ld8_async(lanebase + N + NRT + col, qim);  // Gi Yi
        tc::tmem_wait_ld();
        if (rowok) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int rr = c0 + j, r = rh0 + rr;
            if (r >= nr) continue;
            const c32 C = mk<float>(__uint_as_float(pr[j]) - __uint_as_float(qim[j]),
                                    __uint_as_float(pim[j]) + __uint_as_float(qr[j]));
            const c32 v = pass == 0 ? C : pa[rr] - C;           // t_k, or x_k = t_k - G_k z
            const long long o = (long long)r * lt + (long long)k * b + i;
            outv[o] = v;
            if (upd) Uv[o] = pb[rr] + v;
            if (more) put(r, npass == 0 ? pa[rr] - pc * v : pc * v);
          }
        }
      }
      tc::fence_before();
      tc::fence_async_smem();
      epi_sync();
      if (more) {
        if (tid == 0) tc::bar_arrive(tc::smem_addr(&s_yfull));
        prefetch(bi + 1);
        prefetch_l2(bi + 2);
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, TCOLS);
}

// ------------------------------------------------------------------------------------ host
cudaError_t tc2d_pack_factors(ddm_ctx* c) {
  cudaError_t e = cudaSuccess;
  std::vector<TC2Fac> facs(c->nfac);
  long long total = 0;
  c->tc2_ofs.assign(c->nfac, 0);
  long long maxel = 0;
  for (int f = 0; f < c->nfac; ++f) {
    facs[f] = {c->fac_ofs[f], total, c->fac_b[f], c->fac_m[f], c->fac_ldb[f], 0};
    c->tc2_ofs[f] = total;
    const long long n = tc2d_packed_floats(c->fac_b[f], c->fac_m[f]);
    total += n;
    maxel = std::max(maxel, n);
  }
  if (c->d_gtc2) { cudaFree(c->d_gtc2); c->d_gtc2 = nullptr; }
  if (c->d_tc2ofs) { cudaFree(c->d_tc2ofs); c->d_tc2ofs = nullptr; }
  TC2Fac* d_facs = nullptr;
  if ((e = cudaMalloc((void**)&c->d_gtc2, sizeof(float) * (size_t)total)) != cudaSuccess) return e;
  if ((e = cudaMalloc((void**)&c->d_tc2ofs, sizeof(long long) * c->nfac)) != cudaSuccess) return e;
  if ((e = cudaMalloc((void**)&d_facs, sizeof(TC2Fac) * c->nfac)) != cudaSuccess) return e;
  cudaMemcpyAsync(d_facs, facs.data(), sizeof(TC2Fac) * c->nfac, cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(c->d_tc2ofs, c->tc2_ofs.data(), sizeof(long long) * c->nfac, cudaMemcpyHostToDevice, c->st);
  const int gx = (int)std::min<long long>(64, (maxel / 4 + 255) / 256 + 1);
  ++c->nlaunch;
  k_g2_pack<<<dim3(gx, c->nfac), 256, 0, c->st>>>(d_facs, (const c32*)c->d_G, c->d_gtc2);
  e = cudaGetLastError();
  cudaStreamSynchronize(c->st);
  cudaFree(d_facs);
  return e;
}

// shared memory of the solve for NRT right-hand sides per CTA; 0 if fewer than two stages fit
template <int NRT>
static size_t tc2d_smem(const ddm_ctx* c, int* nst_out) {
  int bmax = 0;
  for (auto& s : c->subs) bmax = std::max(bmax, s.ext[0]);
  const size_t ng = (bmax + 7) / 8, Kpad = (size_t)((bmax + TC2_KC - 1) / TC2_KC) * TC2_KC;
  const size_t yplane = (size_t)(2 * NRT / 8) * (Kpad / 4) * TC2_LBOY;
  const size_t stage = 2048 * ng;
  const size_t fixed = 128 + 2 * yplane + TC2_TAIL;
  const size_t limit = 227 * 1024;
  if (fixed + 2 * stage > limit) return 0;
  const int nst = (int)std::min<size_t>(TC2_MAXST, (limit - fixed) / stage);
  *nst_out = nst;
  return fixed + (size_t)nst * stage;
}

template <int NRT>
static cudaError_t tc2d_solve_n(ddm_ctx* c, const void* src, void* out, void* U, int nrhs) {
  int nst = 0;
  const size_t sm = tc2d_smem<NRT>(c, &nst);
  if (!sm) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(k_solve2d_tc<NRT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  dim3 grid((nrhs + NRT - 1) / NRT, c->g.nsub);
  ++c->nlaunch;
  k_solve2d_tc<NRT><<<grid, TC2_THREADS, sm, c->st>>>(c->g, c->d_gtc2, c->d_tc2ofs, (const c32*)src, (c32*)out,
                                                      (c32*)U, nrhs, nst, c->d_err);
  return cudaGetLastError();
}

bool tc2d_supported(const ddm_ctx* c, int nrt) {
  int nst = 0;
  if (!c->d_gtc2) return false;
  switch (nrt) {
    case 16: return tc2d_smem<16>(c, &nst) > 0;
    case 32: return tc2d_smem<32>(c, &nst) > 0;
    case 64: return tc2d_smem<64>(c, &nst) > 0;
    default: return false;
  }
}

cudaError_t tc2d_solve(ddm_ctx* c, int nrt, const void* src, void* out, void* U, int nrhs) {
  switch (nrt) {
    case 16: return tc2d_solve_n<16>(c, src, out, U, nrhs);
    case 32: return tc2d_solve_n<32>(c, src, out, U, nrhs);
    case 64: return tc2d_solve_n<64>(c, src, out, U, nrhs);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ddm

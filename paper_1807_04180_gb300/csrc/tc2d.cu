// Tensor-core (tcgen05) 2D local solves for many right-hand sides (mixed precision).
//
// The block solves of Algorithm 3.1 in 2D (x-lines as blocks, G_k = D_k^{-1} from factor.cu):
//   forward   y_k = r_k - c_S(., k) t_{k-1},  t_k = G_k y_k            (k = 0..m-1)
//   backward  x_{m-1} = t_{m-1},  x_k = t_k - G_k (c_N(., k) x_{k+1})   (k = m-2..0)
// With 64 right-hand sides per CTA every block step is a complex contraction of the b x b block
// G_k with a b x 64 operand, done here on the 5th-generation tensor cores in split TF32
// ("3xTF32": x = hi + lo with hi = tf32(x); hi*hi + hi*lo + lo*hi accumulated in FP32 in tensor
// memory, FP32-level accuracy) as ONE real product per split term:
//   A (M = 128 rows, in tensor memory): row 2r + a is the real (a = 0) or imaginary (a = 1)
//     part of right-hand side r's block vector, K = the b columns j;
//   B (N = 2 bp rows, bp = b rounded up to 8): rows [Re G_k ; Im G_k], K = j;
//   D = A B^T in tensor memory: D[2r+a][c bp + i] = sum_j Y_a(r, j) G_c(i, j),
// so that Re(G y) = D[2r][i] - D[2r+1][bp+i] and Im(G y) = D[2r][bp+i] + D[2r+1][i].  N = 2 bp
// (up to 256) keeps every MMA at the full tensor rate (measured: an M=128 x N x K=8 tf32 MMA takes
// N/2 cycles for N >= 128, but never fewer than ~44 cycles); three MMAs per K step of 8.
//
// One CTA per (subdomain, group of 64 right-hand sides; the groups of a subdomain adjacent in
// launch order) runs the whole sweep:
//  - warp 8 (producer) streams the factor, packed in FP32 chunk by chunk in consumption order,
//    through a ring of shared-memory stages with cp.async.bulk (half the bytes of pre-split
//    TF32 pairs);
//  - warps 10-11 (splitters) rewrite each landed chunk as its TF32 hi plane and write the lo
//    plane beside it;
//  - warp 9 issues the MMAs from precomputed descriptors;
//  - warps 0-7 read D back (warp w: TMEM lane quarter w % 4 = right-hand sides 16 (w % 4) ..,
//    column chunks of parity w / 4), combine real and imaginary parts with the partner lane by
//    shuffle, and write the next block's operand row (its own TMEM lane) with tcgen05.st.  The
//    block's t_k or x_k and the values the next block needs (loaded while the tensor core works)
//    go through a per-warp shared-memory transpose, so that each global access instruction
//    covers 8 consecutive rows of 4 right-hand sides instead of single rows of 16.
// Tensor memory: D in columns [0, 2 bp), operand hi in [256, 256 + bp), lo in [384, 384 + bp).
// The waits on the critical path (operand ready, stage ready, accumulators ready) spin without
// the suspend hint: a suspended thread resumed about a microsecond after the phase completed.
// The accumulation U += x of the DDM steps runs after the kernel as one coalesced pass.
// Waits are bounded; a time-out sets ERRBIT_TIMEOUT and every role leaves its loop.
//
// Measured alternatives that were slower on the 2048^2, 1024-subdomain, 64-right-hand-side
// workload: splitting each block's output rows into two halves so that the epilogue of one half
// overlaps the products of the other (the N = bp MMAs took about 150 cycles each in a per-block
// trace, waits for factor stages included, no fewer than the full-width ones), and 12 or 16
// epilogue warps instead of 8.
#include <algorithm>
#include <vector>

#include "ddm_internal.cuh"
#include "tcgen05.cuh"

namespace ddm {

constexpr int TC2_NRT = 64;                       // right-hand sides per CTA
constexpr int TC2_KC = 32;                        // K (columns j of G_k) per pipeline chunk
constexpr int TC2_KCC = TC2_KC / 4;               // core matrices along K per chunk
constexpr int TC2_KSTEPS = TC2_KC / 8;            // tf32 MMA K steps per chunk
constexpr int TC2_NEPI = 8;                       // epilogue warps
constexpr int TC2_NSPL = 2;                       // splitter warps
constexpr int TC2_THREADS = (TC2_NEPI + 2 + TC2_NSPL) * 32;   // + producer, MMA and splitter warps
constexpr int TC2_MAXST = 8;
constexpr int TC2_MAXCH = 8;                      // 8-column chunks per epilogue thread (b <= 128)
constexpr uint32_t TC2_AH = 256, TC2_AL = 384;    // TMEM columns of the operand's hi and lo parts
constexpr uint32_t TC2_TCOLS = 512;               // TMEM columns allocated (and freed) per CTA

long long tc2d_packed_floats(int b, int m) {
  const long long ng = (b + 7) / 8, nKC = (b + TC2_KC - 1) / TC2_KC;
  return (long long)m * nKC * (2 * ng) * TC2_KCC * 32;
}

struct TC2Fac { long long fofs, tofs; int b, m, ldb, pad; };

// packed factor: per block k and chunk kc (TC2_KC columns j) the 2 bp rows [Re G_k ; Im G_k] in
// FP32 as 2 ng row groups x TC2_KCC core matrices along K x (8 rows x 4 floats); the solve splits
// each chunk into TF32 hi and lo planes in shared memory
__global__ void k_g2_pack(const TC2Fac* __restrict__ facs, const c32* __restrict__ G, float* __restrict__ dst) {
  const TC2Fac f = facs[blockIdx.y];
  const int ng = (f.b + 7) / 8, nKC = (f.b + TC2_KC - 1) / TC2_KC, bp = 8 * ng;
  const long long nJ = (long long)nKC * TC2_KC;
  const long long total = (long long)f.m * nJ * bp;
  float* out = dst + f.tofs;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % bp);
    const long long r = idx / bp;
    const int j = (int)(r % nJ);
    const int k = (int)(r / nJ);
    c32 v = mk<float>(0.f, 0.f);
    if (i < f.b && j < f.b) v = G[f.fofs + ((long long)k * f.b + j) * f.ldb + i];
    const int kc = j / TC2_KC, jj = j % TC2_KC;
    const long long ps = 64LL * ng * TC2_KCC;          // plane: 2 ng groups x TC2_KCC x 32 floats
    float* chunk = out + ((long long)k * nKC + kc) * ps;
    const int er = ((i >> 3) * TC2_KCC + (jj >> 2)) * 32 + (i & 7) * 4 + (jj & 3);            // row i
    const int ei = (((bp + i) >> 3) * TC2_KCC + (jj >> 2)) * 32 + (i & 7) * 4 + (jj & 3);     // row bp + i
    chunk[er] = v.x;
    chunk[ei] = v.y;
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
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// One work item of the persistent solve: subdomain s and its right-hand-side group starting at r0.
struct TC2Item {
  const SubDesc* s;
  int b, m, ng, bp, nKC, nblk, r0, nr;
  uint32_t stage;   // bytes of one chunk of this subdomain's factor (2 planes x 2 ng row groups)
};
__device__ __forceinline__ TC2Item tc2_item(const Geom& g, int2 it, int nrhs) {
  TC2Item I;
  I.s = &g.subs[it.x];
  I.b = I.s->ext[0];
  I.m = I.s->ext[1];
  I.ng = (I.b + 7) / 8;
  I.bp = 8 * I.ng;
  I.nKC = (I.b + TC2_KC - 1) / TC2_KC;
  I.nblk = 2 * I.m - 1;
  I.r0 = it.y * TC2_NRT;
  I.nr = min(TC2_NRT, nrhs - I.r0);
  I.stage = 512u * TC2_KCC * (uint32_t)I.ng;
  return I;
}

// Persistent: CTA i runs the work items items[cta_ofs[i] .. cta_ofs[i + 1]) in order (the host
// deals the (subdomain, right-hand-side group) items out longest first to the least loaded CTA).
// Tensor memory and the barriers are set up once; the stage ring (slots of the widest subdomain's
// chunk) and the barrier phases run on across items, so the producer streams the next item's
// factor while the epilogue finishes the current one.
__global__ void __launch_bounds__(TC2_THREADS, 1)
    k_solve2d_tc(Geom g, const float* __restrict__ gtc, const long long* __restrict__ tcofs,
                 const c32* __restrict__ src, c32* out, int nrhs, int nst, int ngmax,
                 const int* __restrict__ cta_ofs, const int2* __restrict__ items, int* err) {
  extern __shared__ unsigned char smem_raw[];
  // s_raw: a stage's FP32 plane has landed (bulk copy); s_full: its hi / lo planes are written
  __shared__ __align__(8) uint64_t s_raw[TC2_MAXST], s_full[TC2_MAXST], s_empty[TC2_MAXST], s_yfull, s_dfull;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  __shared__ __align__(16) c32 s_coef[2][128];   // coupling of the next block's operand, per row
  // per epilogue warp: 8 rows x 16 right-hand sides (row stride 18) to transpose between the TMEM
  // lane order (one right-hand side per lane pair) and row-contiguous global accesses
  __shared__ __align__(16) c32 s_xpose[TC2_NEPI][8 * 18];
  volatile int* abort_flag = &s_abort;

  const int it0 = cta_ofs[blockIdx.x], it1 = cta_ofs[blockIdx.x + 1];
  const uint32_t SSTRIDE = 512u * TC2_KCC * (uint32_t)ngmax;   // ring slot: the widest chunk
  const uint32_t raw = tc::smem_addr(smem_raw);
  const uint32_t ring = (raw + 127u) & ~127u;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(&s_tmem), TC2_TCOLS);
  if (tid == 0) {
    for (int i = 0; i < nst; ++i) {
      tc::bar_init(tc::smem_addr(&s_raw[i]), 1);
      tc::bar_init(tc::smem_addr(&s_full[i]), 1);
      tc::bar_init(tc::smem_addr(&s_empty[i]), 1);
    }
    tc::bar_init(tc::smem_addr(&s_yfull), 1);
    tc::bar_init(tc::smem_addr(&s_dfull), 1);
    s_abort = 0;
    tc::bar_init_fence();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = s_tmem;
  // the operand columns start at zero (unused rows stay finite)
  if (warp < 4) {
    const float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (uint32_t c0 = TC2_AH; c0 < TC2_TCOLS; c0 += 8) tc::tmem_st8(tmem + ((uint32_t)(warp * 32) << 16) + c0, z);
    tc::tmem_wait_st();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();

  if (warp == TC2_NEPI) {
    // ------------------------------------------------------------------ producer
    if (lane == 0) {
      long long c = 0;
      bool ok = true;
      for (int ii = it0; ii < it1 && ok; ++ii) {
        const TC2Item I = tc2_item(g, items[ii], nrhs);
        const float* gsrc = gtc + tcofs[I.s->fid];
        for (int bi = 0; bi < I.nblk && ok && !*abort_flag; ++bi) {
          int pass, k;
          seq2(bi, I.m, pass, k);
          for (int kc = 0; kc < I.nKC; ++kc, ++c) {
            const int st = (int)(c % nst);
            if (c >= nst && !tc::bar_wait_or_abort(tc::smem_addr(&s_empty[st]), (uint32_t)((c / nst) - 1) & 1u,
                                                     abort_flag)) {
              atomicOr(err, ERRBIT_TIMEOUT);
              ok = false;
              break;
            }
            const uint32_t fb = tc::smem_addr(&s_raw[st]);
            tc::bar_expect_tx(fb, I.stage / 2);
            tc::bulk_load(ring + (uint32_t)st * SSTRIDE, gsrc + ((long long)k * I.nKC + kc) * (I.stage / 8),
                          I.stage / 2, fb);
          }
        }
      }
      // the copies still in flight land before the CTA may exit (bounded)
      for (long long cc = c > nst ? c - nst : 0; cc < c; ++cc)
        tc::bar_wait(tc::smem_addr(&s_raw[cc % nst]), (uint32_t)((cc / nst) & 1));
    }
  } else if (warp == TC2_NEPI + 1) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      // descriptor at the first stage and K step; others only move the start address (>> 4)
      const uint64_t dB = tc::sdesc(ring, 128, 128 * TC2_KCC);
      long long c = 0, gbi = 0;   // chunks and blocks over all items so far
      bool ok = true;
      for (int ii = it0; ii < it1 && ok; ++ii) {
      const TC2Item I = tc2_item(g, items[ii], nrhs);
      const uint32_t ID = tc::idesc_tf32(128, 2 * I.bp, false);
      const uint64_t BLO = (uint64_t)(I.stage / 2) >> 4;   // lo plane of a stage
      const int nks = (I.b + 7) / 8;                       // K steps that are not all padding
      for (int bi = 0; bi < I.nblk && ok; ++bi, ++gbi) {
        if (!tc::bar_spin_or_abort(tc::smem_addr(&s_yfull), (uint32_t)(gbi & 1), abort_flag)) { ok = false; break; }
        tc::fence_after();
        for (int kc = 0; kc < I.nKC; ++kc, ++c) {
          const int st = (int)(c % nst);
          if (!tc::bar_spin_or_abort(tc::smem_addr(&s_full[st]), (uint32_t)((c / nst) & 1), abort_flag)) {
            ok = false;
            break;
          }
          tc::fence_after();
          const uint64_t bst = dB + (((uint64_t)st * SSTRIDE) >> 4);
#pragma unroll
          for (int t = 0; t < TC2_KSTEPS; ++t) {
            const int ks = TC2_KSTEPS * kc + t;
            if (ks >= nks) break;
            const uint32_t ka = (uint32_t)(8 * ks);
            const uint64_t kb = (uint64_t)t * (256 / 16);
            const uint32_t acc = ks > 0 ? 1u : 0u;
            tc::mma_tf32_ts(tmem, tmem + TC2_AH + ka, bst + kb, ID, acc);
            tc::mma_tf32_ts(tmem, tmem + TC2_AH + ka, bst + BLO + kb, ID, 1u);
            tc::mma_tf32_ts(tmem, tmem + TC2_AL + ka, bst + kb, ID, 1u);
          }
          tc::mma_commit(tc::smem_addr(&s_empty[st]));
        }
        if (!ok) break;
        tc::mma_commit(tc::smem_addr(&s_dfull));
      }
      }
      if (!ok) atomicOr(err, ERRBIT_TIMEOUT);
    }
  } else if (warp >= TC2_NEPI + 2) {
    // ------------------------------------------------------------------ splitter warps
    // Each landed FP32 plane (plane 0 of its stage) is rewritten in place as its TF32 hi part and
    // its lo part goes to plane 1 (x = hi + lo exactly); the generic-proxy writes are fenced for
    // the tensor core before s_full is signalled.
    const int st_tid = tid - (TC2_NEPI + 2) * 32;
    long long c = 0;
    bool ok = true;
    for (int ii = it0; ii < it1 && ok; ++ii) {
    const TC2Item I = tc2_item(g, items[ii], nrhs);
    const int n4 = (int)(I.stage / 32);                    // float4 groups in one plane
    for (int bi = 0; bi < I.nblk && ok; ++bi) {
      for (int kc = 0; kc < I.nKC; ++kc, ++c) {
        const int st = (int)(c % nst);
        bool got = true;
        if (st_tid == 0) got = tc::bar_wait_or_abort(tc::smem_addr(&s_raw[st]), (uint32_t)((c / nst) & 1), abort_flag);
        uint32_t bad;   // bar.red.or over the splitter warps: all learn whether the wait succeeded
        asm volatile("{\n .reg .pred q, o;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred o, 2, %2, q;\n selp.u32 %0, 1, 0, o;\n}\n"
                     : "=r"(bad)
                     : "r"((uint32_t)!got), "r"(TC2_NSPL * 32)
                     : "memory");
        if (bad) { ok = false; break; }
        float4* hi = reinterpret_cast<float4*>(smem_raw + (ring - raw) + (uint32_t)st * SSTRIDE);
        float4* lo = hi + n4;
#pragma unroll 4
        for (int v = st_tid; v < n4; v += TC2_NSPL * 32) {
          const float4 x = hi[v];
          float4 h, l;
          tc::split_tf32(x.x, h.x, l.x);
          tc::split_tf32(x.y, h.y, l.y);
          tc::split_tf32(x.z, h.z, l.z);
          tc::split_tf32(x.w, h.w, l.w);
          hi[v] = h;
          lo[v] = l;
        }
        tc::fence_async_smem();
        asm volatile("bar.sync 2, %0;" ::"r"(TC2_NSPL * 32) : "memory");
        if (st_tid == 0) tc::bar_arrive(tc::smem_addr(&s_full[st]));
      }
    }
    }
    if (!ok) atomicOr(err, ERRBIT_TIMEOUT);
  } else {
    // ------------------------------------------------------------------ epilogue warps 0-7
    const int q4 = warp & 3, par = warp >> 2;
    const int n = q4 * 32 + lane;                   // TMEM lane = operand row 2r + a
    const int r = n >> 1, a = n & 1;                // right-hand side within the group, part
    const uint32_t lanebase = tmem + ((uint32_t)(q4 * 32) << 16);
    c32* xp = s_xpose[warp];
    // operand row write: this lane's row (part a of right-hand side r), columns j = 8 cc .. + 7
    auto put8 = [&](int cc, const float* v) {
      float hi[8], lo[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) tc::split_tf32(v[e], hi[e], lo[e]);
      tc::tmem_st8(lanebase + TC2_AH + (uint32_t)(8 * cc), hi);
      tc::tmem_st8(lanebase + TC2_AL + (uint32_t)(8 * cc), lo);
    };
    long long gbi = 0;   // blocks of the items before this one (phase of s_dfull)
    bool eok = true;
    for (int ii = it0; ii < it1 && eok; ++ii) {
    const TC2Item I = tc2_item(g, items[ii], nrhs);
    const SubDesc& s = *I.s;
    const int b = I.b, m = I.m, ng = I.ng, bp = I.bp, nblk = I.nblk, r0 = I.r0, nr = I.nr;
    const bool rok = r < nr;
    const long long len = (long long)b * m;
    const c32* lc = (const c32*)g.lcoef + s.vofs * 5;   // planes: C, W, E, S, N
    const c32* cSp = lc + 3 * len;
    const c32* cNp = lc + 4 * len;
    const long long vo = lvofs(s, r0 + (rok ? r : 0), nrhs);
    const c32* srcv = src + vo;
    // global accesses in row order: lane l serves right-hand side 16 q4 + 4 j + (l >> 3), row
    // l & 7 of a chunk, j = 0..3 (four rows of 64 contiguous bytes per instruction)
    const int rl = lane >> 1;                                  // my right-hand side in the warp
    const int crow = lane & 7, crhs = lane >> 3;
    long long gvo[4];
    bool gok[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int rr = 16 * q4 + 4 * j + crhs;
      gok[j] = rr < nr;
      gvo[j] = lvofs(s, r0 + (gok[j] ? rr : 0), nrhs);
    }
    // this thread's rows of every block: 4 consecutive rows i = 8 cc + 4 a + e (e = 0..3) of its
    // right-hand side r, for the 8-column chunks cc = par, par + 2, ... < ng
    const int nch = (ng - par + 1) / 2;
    // block 0: y_0 = r_0
    for (int ci = 0; ci < nch; ++ci) {
      const int cc = par + 2 * ci;
      float v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int i = 8 * cc + e;
        const c32 y = (rok && i < b) ? srcv[i] : mk<float>(0.f, 0.f);
        v[e] = a == 0 ? y.x : y.y;
      }
      put8(cc, v);
    }
    tc::tmem_wait_st();
    tc::fence_before();
    epi_sync();
    if (tid == 0) tc::bar_arrive(tc::smem_addr(&s_yfull));
    // values the epilogue of block bi needs, loaded one block ahead (4 rows per chunk):
    //   pass 0: pa = r_{k+1} (next block's source);  pass 1: pa = t_k
    // pa[ci][j]: right-hand side 16 q4 + 4 j + (lane >> 3), row 8 cc + (lane & 7) (row order)
    c32 pa[TC2_MAXCH][4];
    auto prefetch = [&](int bi) {
      int pass, k;
      seq2(bi, m, pass, k);
      const bool need = pass == 1 || k + 1 < m;
      const long long o = pass == 0 ? (long long)(k + 1) * b : (long long)k * b;
      const c32* p = pass == 0 ? src : out;
#pragma unroll
      for (int ci = 0; ci < TC2_MAXCH; ++ci) {
        const int i = 8 * (par + 2 * ci) + crow;
#pragma unroll
        for (int j = 0; j < 4; ++j)
          pa[ci][j] = (need && gok[j] && ci < nch && i < b) ? p[gvo[j] + o + i] : mk<float>(0.f, 0.f);
      }
    };
    // couplings of the operand of block bi + 1, used by the epilogue of block bi, copied
    // asynchronously into s_coef[bi & 1] one block ahead
    auto coef_copy = [&](int bi) {
      if (bi + 1 >= nblk) return;
      int npass, nk;
      seq2(bi + 1, m, npass, nk);
      const c32* cp = npass == 0 ? cSp + (long long)nk * b : cNp + (long long)nk * b;
      if (tid < b) cp_async8(tc::smem_addr(&s_coef[bi & 1][tid]), cp + tid);
      cp_async_commit();
    };
    prefetch(0);
    coef_copy(0);
    for (int bi = 0; bi < nblk; ++bi) {
      int pass, k;
      seq2(bi, m, pass, k);
      // one thread waits for the accumulators; the others sleep in the barrier, which also makes
      // every thread's coefficient copies visible
      cp_async_wait_all();
      bool got = true;
      if (tid == 0) got = tc::bar_spin_or_abort(tc::smem_addr(&s_dfull), (uint32_t)((gbi + bi) & 1), abort_flag);
      if (epi_any(!got)) { eok = false; break; }
      tc::fence_after();
      const bool more = bi + 1 < nblk;
      int npass = 0, nk = 0;
      if (more) seq2(bi + 1, m, npass, nk);
      const c32* cnext = s_coef[bi & 1];
      const long long ko = (long long)k * b;
#pragma unroll
      for (int ci = 0; ci < TC2_MAXCH; ++ci) {
        if (ci >= nch) break;                          // warp-uniform
        const int cc = par + 2 * ci;
        uint32_t u0[8], u1[8];
        tc::tmem_ld8_async(lanebase + (uint32_t)(8 * cc), u0);        // Y_a G_r, columns 8cc..
        tc::tmem_ld8_async(lanebase + (uint32_t)(bp + 8 * cc), u1);   // Y_a G_i
        tc::tmem_wait_ld();
        // the prefetched values in lane order: my right-hand side, rows 4 a + e of the chunk
        c32 pv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) xp[crow * 18 + 4 * j + crhs] = pa[ci][j];
        __syncwarp();
#pragma unroll
        for (int e = 0; e < 4; ++e) pv[e] = xp[(4 * a + e) * 18 + rl];
        __syncwarp();
        // this lane's 4 rows i = 8 cc + 4 a + e; the partner lane holds the other part of y
        c32 y[4], ov[4];
        const int i0 = 8 * cc + 4 * a;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          // lane a keeps rows 4a..4a+3 of the chunk and sends the partner its other four
          const float x0 = __uint_as_float(a == 0 ? u0[e] : u0[4 + e]);
          const float x1 = __uint_as_float(a == 0 ? u1[e] : u1[4 + e]);
          const float s0 = __uint_as_float(a == 0 ? u0[4 + e] : u0[e]);
          const float s1 = __uint_as_float(a == 0 ? u1[4 + e] : u1[e]);
          const float w0 = __shfl_xor_sync(0xffffffffu, s0, 1);   // partner's Y G_r at my row
          const float w1 = __shfl_xor_sync(0xffffffffu, s1, 1);   // partner's Y G_i at my row
          // even lane: x = (Yr Gr, Yr Gi), w = (Yi Gr, Yi Gi); odd lane: the reverse
          const float yrgr = a == 0 ? x0 : w0, yrgi = a == 0 ? x1 : w1;
          const float yigr = a == 0 ? w0 : x0, yigi = a == 0 ? w1 : x1;
          const c32 C = mk<float>(yrgr - yigi, yrgi + yigr);
          const int i = i0 + e;
          const c32 v = pass == 0 ? C : pv[e] - C;              // t_k, or x_k = t_k - G_k z
          ov[e] = v;
          c32 yv = mk<float>(0.f, 0.f);
          if (more && i < b) {
            const c32 cf = cnext[i];   // shared memory
            yv = npass == 0 ? pv[e] - cf * v : cf * v;
          }
          y[e] = yv;
        }
        // t_k / x_k to the local vectors in row order
#pragma unroll
        for (int e = 0; e < 4; ++e) xp[(4 * a + e) * 18 + rl] = ov[e];
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int i = 8 * cc + crow;
          const c32 v = xp[crow * 18 + 4 * j + crhs];
          if (gok[j] && i < b) out[gvo[j] + ko + i] = v;
        }
        __syncwarp();
        if (more) {
          // row values of the next operand: part a of y at the chunk's 8 rows; the partner lane
          // holds the other 4 rows
          float send[4], v8[8];
#pragma unroll
          for (int e = 0; e < 4; ++e) send[e] = a == 0 ? y[e].y : y[e].x;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float recv = __shfl_xor_sync(0xffffffffu, send[e], 1);
            v8[e] = a == 0 ? y[e].x : recv;
            v8[4 + e] = a == 0 ? recv : y[e].y;
          }
          put8(cc, v8);
        }
      }
      tc::tmem_wait_st();
      tc::fence_before();
      epi_sync();
      if (more) {
        if (tid == 0) tc::bar_arrive(tc::smem_addr(&s_yfull));
        prefetch(bi + 1);
        coef_copy(bi + 1);
      }
    }
    gbi += nblk;
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, TC2_TCOLS);
}

// U += x over the local vectors of nrhs right-hand sides (n complex values; 16-byte steps when
// both arrays are 16-byte aligned)
__global__ void k_accum_local(c32* __restrict__ U, const c32* __restrict__ x, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const bool vec = ((reinterpret_cast<uintptr_t>(U) | reinterpret_cast<uintptr_t>(x)) & 15) == 0;
  if (vec) {
    float4* U4 = reinterpret_cast<float4*>(U);
    const float4* x4 = reinterpret_cast<const float4*>(x);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n / 2; i += stride) {
      float4 u = U4[i];
      const float4 v = x4[i];
      u.x += v.x; u.y += v.y; u.z += v.z; u.w += v.w;
      U4[i] = u;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && (n & 1)) U[n - 1] = U[n - 1] + x[n - 1];
  } else {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) U[i] = U[i] + x[i];
  }
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
  // grow-only: a captured graph of M_K keeps addressing these buffers
  if ((size_t)total > c->gtc2_cap) {
    dev_free(c, c->d_gtc2);
    c->d_gtc2 = nullptr;
    c->gtc2_cap = 0;
    c->drop_graphs();
    if ((e = dev_alloc(c, (void**)&c->d_gtc2, sizeof(float) * (size_t)total)) != cudaSuccess) return e;
    c->gtc2_cap = (size_t)total;
  }
  if ((size_t)c->nfac > c->tc2ofs_cap) {
    dev_free(c, c->d_tc2ofs);
    c->d_tc2ofs = nullptr;
    c->tc2ofs_cap = 0;
    c->drop_graphs();
    if ((e = dev_alloc(c, (void**)&c->d_tc2ofs, sizeof(long long) * c->nfac)) != cudaSuccess) return e;
    c->tc2ofs_cap = (size_t)c->nfac;
  }
  TC2Fac* d_facs = nullptr;
  if ((e = dev_alloc(c, (void**)&d_facs, sizeof(TC2Fac) * c->nfac)) != cudaSuccess) return e;
  cudaMemcpyAsync(d_facs, facs.data(), sizeof(TC2Fac) * c->nfac, cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(c->d_tc2ofs, c->tc2_ofs.data(), sizeof(long long) * c->nfac, cudaMemcpyHostToDevice, c->st);
  const int gx = (int)std::min<long long>(64, (maxel / 4 + 255) / 256 + 1);
  ++c->nlaunch;
  k_g2_pack<<<dim3(gx, c->nfac), 256, 0, c->st>>>(d_facs, (const c32*)c->d_G, c->d_gtc2);
  e = cudaGetLastError();
  cudaStreamSynchronize(c->st);
  dev_free(c, d_facs);
  return e;
}

// shared memory of the solve; 0 if the blocks are too wide or fewer than two ring stages fit
static size_t tc2d_smem(const ddm_ctx* c, int* nst_out) {
  int bmax = 0;
  for (auto& s : c->subs) bmax = std::max(bmax, s.ext[0]);
  const size_t ng = (bmax + 7) / 8;
  const size_t stage = 512 * TC2_KCC * ng;
  const size_t fixed = 128;
  const size_t limit = 227 * 1024 - 12 * 1024;   // the kernel's static shared memory beside it
  if (bmax > 16 * TC2_MAXCH || fixed + 2 * stage > limit) return 0;
  const int nst = (int)std::min<size_t>(TC2_MAXST, (limit - fixed) / stage);
  *nst_out = nst;
  return fixed + (size_t)nst * stage;
}

bool tc2d_supported(const ddm_ctx* c, int nrt) {
  int nst = 0;
  return c->d_gtc2 && nrt == TC2_NRT && tc2d_smem(c, &nst) > 0;
}

// Work lists of the persistent solve for ngr right-hand-side groups: every (subdomain, group) item
// costs (2m - 1) b^2 (the factor entries it streams); items go out longest first, each to the
// CTA with the least work so far (LPT), one CTA per SM.
static cudaError_t tc2d_plan(ddm_ctx* c, int ngr, const ddm_ctx::TC2Plan** out) {
  auto it = c->tc2plans.find(ngr);
  if (it != c->tc2plans.end()) { *out = &it->second; return cudaSuccess; }
  int nsm = 0, dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  std::vector<std::pair<double, int2>> work;
  for (int sid = 0; sid < c->g.nsub; ++sid) {
    const double b = c->subs[sid].ext[0], m = c->subs[sid].ext[1];
    for (int gr = 0; gr < ngr; ++gr) work.push_back({(2 * m - 1) * b * b, make_int2(sid, gr)});
  }
  std::stable_sort(work.begin(), work.end(), [](const std::pair<double, int2>& x, const std::pair<double, int2>& y) {
    return x.first > y.first;
  });
  const int nctas = (int)std::min<size_t>(work.size(), (size_t)std::max(nsm, 1));
  std::vector<double> load(nctas, 0.0);
  std::vector<std::vector<int2>> lists(nctas);
  for (auto& w : work) {
    const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[k] += w.first;
    lists[k].push_back(w.second);
  }
  std::vector<int> ofs(nctas + 1, 0);
  std::vector<int2> items;
  for (int k = 0; k < nctas; ++k) {
    ofs[k + 1] = ofs[k] + (int)lists[k].size();
    items.insert(items.end(), lists[k].begin(), lists[k].end());
  }
  ddm_ctx::TC2Plan pl;
  pl.nctas = nctas;
  if ((e = dev_alloc(c, (void**)&pl.d_ofs, sizeof(int) * ofs.size())) != cudaSuccess) return e;
  if ((e = dev_alloc(c, (void**)&pl.d_items, sizeof(int2) * items.size())) != cudaSuccess) {
    dev_free(c, pl.d_ofs);
    return e;
  }
  if ((e = cudaMemcpyAsync(pl.d_ofs, ofs.data(), sizeof(int) * ofs.size(), cudaMemcpyHostToDevice, c->st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(pl.d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice, c->st)) !=
          cudaSuccess) {
    dev_free(c, pl.d_ofs);
    dev_free(c, pl.d_items);
    return e;
  }
  *out = &(c->tc2plans[ngr] = pl);
  return cudaSuccess;
}

cudaError_t tc2d_solve(ddm_ctx* c, int nrt, const void* src, void* out, void* U, int nrhs) {
  if (nrt != TC2_NRT) return cudaErrorInvalidValue;
  int nst = 0;
  const size_t sm = tc2d_smem(c, &nst);
  if (!sm) return cudaErrorInvalidConfiguration;
  cudaError_t e = allow_dynamic_smem((const void*)k_solve2d_tc, sm);
  if (e != cudaSuccess) return e;
  const ddm_ctx::TC2Plan* pl = nullptr;
  if ((e = tc2d_plan(c, (nrhs + TC2_NRT - 1) / TC2_NRT, &pl)) != cudaSuccess) return e;
  int bmax = 0;
  for (auto& s : c->subs) bmax = std::max(bmax, s.ext[0]);
  ++c->nlaunch;
  k_solve2d_tc<<<pl->nctas, TC2_THREADS, sm, c->st>>>(c->g, c->d_gtc2, c->d_tc2ofs, (const c32*)src, (c32*)out, nrhs,
                                                      nst, (bmax + 7) / 8, pl->d_ofs, pl->d_items, c->d_err);
  if (U) {
    // after the backward sweep `out` holds the solution of every block: U += out in one pass
    const long long n = c->g.ltotal * nrhs;
    ++c->nlaunch;
    k_accum_local<<<(int)std::min<long long>((n / 2 + 255) / 256, 152LL * 32), 256, 0, c->st>>>((c32*)U,
                                                                                               (const c32*)out, n);
  }
  return cudaGetLastError();
}

}  // namespace ddm

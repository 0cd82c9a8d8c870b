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
//   B (N rows): rows [Re G_k ; Im G_k] of the output rows i of one half (below), K = j;
//   D = A B^T in tensor memory: D[2r+a][c H + il] = sum_j Y_a(r, j) G_c(i, j),
// so that Re(G y) = D[2r][il] - D[2r+1][H+il] and Im(G y) = D[2r][H+il] + D[2r+1][il].
//
// Halves.  The rows i (and so the columns j of the next block) are split at H1 = 8 ceil(ng / 2)
// (ng = row groups of 8, bp = 8 ng): half 0 = [0, H1), half 1 = [H1, bp).  The factor is packed
// per block as four quarters (output half hN, column half hK) in the order the tensor core uses
// them: (0,0), (0,1), (1,0), (1,1).  Block k's products for output half 0 can start on column
// half 0 of its operand while the epilogue of block k-1 is still writing column half 1, and the
// epilogue of output half 0 runs while the tensor core computes output half 1:
//   MMA   (0,0) (0,1) | (1,0) (1,1) | next block (0,0) ...
//   epi               | half 0      | half 1 ...
// Tensor memory: D of half 0 in columns [0, 2 H1), of half 1 in [2 H1, 2 bp); the operand's hi
// part in [256, 256 + bp), lo in [384, 384 + bp).  Column half 0 of the operand is rewritten only
// after quarter (1,0), its last reader, has completed (mbarrier s_ofree).  An M = 128 x N tf32 MMA
// takes N/2 cycles for N >= 128 and never fewer than ~44 (measured), so halves of N = 2 H >= 64
// lose little.
//
// One CTA per (subdomain, group of 64 right-hand sides; the groups of a subdomain adjacent in
// launch order) runs the whole sweep:
//  - warp 12 (producer) streams the packed quarters through a ring of shared-memory stages with
//    cp.async.bulk;
//  - warp 13 issues the MMAs from precomputed descriptors;
//  - warps 0-11 read D back (warp w: TMEM lane quarter w % 4 = right-hand sides 16 (w % 4) ..,
//    8-row chunks c0 + w / 4 + 3 i of the half), combine real and imaginary parts with the
//    partner lane by shuffle, write the block's t_k or x_k to the local vectors (each thread 4
//    consecutive rows of one right-hand side) and the next block's operand row (its own TMEM
//    lane) with tcgen05.st; the values they need next are loaded while the tensor core works.
//    Fourteen warps keep 128 registers per thread (at most four warps share an SM sub-partition's
//    16K registers); sixteen epilogue warps would cap them at 96 and spill.
// The accumulation U += x of the DDM steps runs after the kernel as one coalesced pass.
// Waits are bounded; a time-out sets ERRBIT_TIMEOUT and every role leaves its loop.
#include <algorithm>
#include <vector>

#include "ddm_internal.cuh"
#include "tcgen05.cuh"

namespace ddm {

constexpr int TC2_NRT = 64;                       // right-hand sides per CTA
constexpr int TC2_NEPI = 12;                      // epilogue warps
constexpr int TC2_NPAR = TC2_NEPI / 4;            // epilogue warps per TMEM lane quarter
constexpr int TC2_THREADS = (TC2_NEPI + 2) * 32;  // + producer warp + MMA warp
constexpr int TC2_MAXST = 8;
constexpr int TC2_MAXCH = 3;                      // 8-row chunks per epilogue thread and half (b <= 128)
constexpr uint32_t TC2_AH = 256, TC2_AL = 384;    // TMEM columns of the operand's hi and lo parts
constexpr uint32_t TC2_TCOLS = 512;               // TMEM columns allocated (and freed) per CTA

// rows of half 0 (H1) for a block of bp = 8 ng rows; half 1 has bp - H1 rows
__host__ __device__ __forceinline__ int tc2_h1(int ng) { return 8 * ((ng + 1) / 2); }

long long tc2d_packed_floats(int b, int m) {
  const long long bp = 8LL * ((b + 7) / 8);
  return (long long)m * 4 * bp * bp;   // 2 planes x [Re; Im] x bp x bp per block
}

struct TC2Fac { long long fofs, tofs; int b, m, ldb, pad; };

// packed factor: per block k four quarters (hN, hK) in the order (0,0), (0,1), (1,0), (1,1); a
// quarter holds two planes {hi, lo} of the 2 H_hN rows [Re G_k(i, j) ; Im G_k(i, j)] (i in output
// half hN) x H_hK columns j (column half hK), as 8-row groups x core matrices along K x (8 rows x
// 4 floats)
__global__ void k_g2_pack(const TC2Fac* __restrict__ facs, const c32* __restrict__ G, float* __restrict__ dst) {
  const TC2Fac f = facs[blockIdx.y];
  const int ng = (f.b + 7) / 8, bp = 8 * ng, H1 = tc2_h1(ng);
  const int Hh[2] = {H1, bp - H1};
  const long long total = (long long)f.m * bp * bp;
  float* out = dst + f.tofs;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % bp);
    const long long rr = idx / bp;
    const int j = (int)(rr % bp);
    const int k = (int)(rr / bp);
    c32 v = mk<float>(0.f, 0.f);
    if (i < f.b && j < f.b) v = G[f.fofs + ((long long)k * f.b + j) * f.ldb + i];
    float rh, rl, ih, il;
    tc::split_tf32(v.x, rh, rl);
    tc::split_tf32(v.y, ih, il);
    const int hN = i >= H1, hK = j >= H1;
    const int R = 2 * Hh[hN], Kq = Hh[hK];
    const int li = i - (hN ? H1 : 0), lj = j - (hK ? H1 : 0);
    // quarter offsets in the block: (0,0) 0, (0,1) 4 H1 H1, (1,0) + 4 H1 H2, (1,1) + 4 H2 H1
    long long qo = 0;
    const int q = 2 * hN + hK;
    if (q >= 1) qo += 4LL * Hh[0] * Hh[0];
    if (q >= 2) qo += 4LL * Hh[0] * Hh[1];
    if (q >= 3) qo += 4LL * Hh[1] * Hh[0];
    const long long ps = (long long)R * Kq;   // floats per plane
    float* quarter = out + (long long)k * 4 * bp * bp + qo;
    const int kcc = Kq / 4;
    const int er = ((li >> 3) * kcc + (lj >> 2)) * 32 + (li & 7) * 4 + (lj & 3);                      // Re row
    const int ei = (((Hh[hN] + li) >> 3) * kcc + (lj >> 2)) * 32 + ((Hh[hN] + li) & 7) * 4 + (lj & 3);   // Im row
    quarter[er] = rh;
    quarter[ps + er] = rl;
    quarter[ei] = ih;
    quarter[ps + ei] = il;
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

__global__ void __launch_bounds__(TC2_THREADS, 1)
    k_solve2d_tc(Geom g, const float* __restrict__ gtc, const long long* __restrict__ tcofs,
                 const c32* __restrict__ src, c32* out, int nrhs, int nst, uint32_t stage_bytes, int* err) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t s_full[TC2_MAXST], s_empty[TC2_MAXST], s_yready[2], s_dfull[2], s_ofree;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  __shared__ __align__(16) c32 s_coef[2][128];   // coupling of the next block's operand, per row
  volatile int* abort_flag = &s_abort;

  // the right-hand-side groups of one subdomain are adjacent in launch order, so that they run
  // at the same time and the second read of each factor block hits L2
  const SubDesc& s = g.subs[blockIdx.y];
  const int b = s.ext[0], m = s.ext[1];
  const int ng = (b + 7) / 8, bp = 8 * ng, H1 = tc2_h1(ng), H2 = bp - H1;
  const int nblk = 2 * m - 1;
  const int r0 = blockIdx.x * TC2_NRT, nr = min(TC2_NRT, nrhs - r0);
  const uint32_t raw = tc::smem_addr(smem_raw);
  const uint32_t ring = (raw + 127u) & ~127u;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(&s_tmem), TC2_TCOLS);
  if (tid == 0) {
    for (int i = 0; i < nst; ++i) {
      tc::bar_init(tc::smem_addr(&s_full[i]), 1);
      tc::bar_init(tc::smem_addr(&s_empty[i]), 1);
    }
    for (int h = 0; h < 2; ++h) {
      tc::bar_init(tc::smem_addr(&s_yready[h]), 1);
      tc::bar_init(tc::smem_addr(&s_dfull[h]), 1);
    }
    tc::bar_init(tc::smem_addr(&s_ofree), 1);
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
      const float* gsrc = gtc + tcofs[s.fid];
      const long long blkf = 4LL * bp * bp;
      long long c = 0;
      for (int bi = 0; bi < nblk && !*abort_flag; ++bi) {
        int pass, k;
        seq2(bi, m, pass, k);
        long long qo = 0;
        for (int q = 0; q < 4; ++q, ++c) {
          // quarter q = (output half q / 2, column half q % 2): 4 H_hN H_hK floats
          const uint32_t qf = 4u * (uint32_t)((q >> 1) ? H2 : H1) * (uint32_t)((q & 1) ? H2 : H1);
          const int st = (int)(c % nst);
          if (c >= nst && !tc::bar_wait_or_abort(tc::smem_addr(&s_empty[st]), (uint32_t)((c / nst) - 1) & 1u,
                                                   abort_flag)) {
            atomicOr(err, ERRBIT_TIMEOUT);
            break;
          }
          const uint32_t fb = tc::smem_addr(&s_full[st]);
          tc::bar_expect_tx(fb, 4u * qf);
          tc::bulk_load(ring + (uint32_t)st * stage_bytes, gsrc + (long long)k * blkf + qo, 4u * qf, fb);
          qo += qf;
        }
      }
      // the copies still in flight land before the CTA may exit (bounded)
      for (long long cc = c > nst ? c - nst : 0; cc < c; ++cc)
        tc::bar_wait(tc::smem_addr(&s_full[cc % nst]), (uint32_t)((cc / nst) & 1));
    }
  } else if (warp == TC2_NEPI + 1) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t ID0 = tc::idesc_tf32(128, 2 * H1, false), ID1 = tc::idesc_tf32(128, 2 * H2, false);
      long long c = 0;
      bool ok = true;
      for (int bi = 0; bi < nblk && ok; ++bi) {
        for (int q = 0; q < 4 && ok; ++q, ++c) {
          const int hN = q >> 1, hK = q & 1;
          // output half 0 waits for the operand's column half hK of this block
          if (hN == 0) {
            if (!tc::bar_wait_or_abort(tc::smem_addr(&s_yready[hK]), (uint32_t)(bi & 1), abort_flag)) { ok = false; break; }
            tc::fence_after();
          }
          const int st = (int)(c % nst);
          if (!tc::bar_wait_or_abort(tc::smem_addr(&s_full[st]), (uint32_t)((c / nst) & 1), abort_flag)) {
            ok = false;
            break;
          }
          tc::fence_after();
          const int Kq = hK ? H2 : H1, Hn = hN ? H2 : H1;
          const uint32_t ID = hN ? ID1 : ID0;
          const uint32_t sbase = ring + (uint32_t)st * stage_bytes;
          const uint64_t dB = tc::sdesc(sbase, 128, 32u * (uint32_t)Kq);   // 8-row groups 8 x Kq floats apart
          const uint64_t lo = (uint64_t)((uint32_t)(8 * Hn * Kq) >> 4);    // lo plane: 2 H_hN x Kq floats on
          const uint32_t dcol = hN ? (uint32_t)(2 * H1) : 0u;
          const uint32_t j0 = hK ? (uint32_t)H1 : 0u;
          for (int t = 0; t < Kq / 8; ++t) {
            const uint32_t ka = j0 + (uint32_t)(8 * t);
            const uint64_t kb = (uint64_t)t * (256 / 16);
            const uint32_t acc = (hK > 0 || t > 0) ? 1u : 0u;
            tc::mma_tf32_ts(tmem + dcol, tmem + TC2_AH + ka, dB + kb, ID, acc);
            tc::mma_tf32_ts(tmem + dcol, tmem + TC2_AH + ka, dB + lo + kb, ID, 1u);
            tc::mma_tf32_ts(tmem + dcol, tmem + TC2_AL + ka, dB + kb, ID, 1u);
          }
          tc::mma_commit(tc::smem_addr(&s_empty[st]));
          if (q == 1) tc::mma_commit(tc::smem_addr(&s_dfull[0]));
          if (q == 2) tc::mma_commit(tc::smem_addr(&s_ofree));
          if (q == 3) tc::mma_commit(tc::smem_addr(&s_dfull[1]));
        }
      }
      if (!ok) atomicOr(err, ERRBIT_TIMEOUT);
    }
  } else {
    // ------------------------------------------------------------------ epilogue warps 0-11
    const int q4 = warp & 3, par = warp >> 2;
    const int n = q4 * 32 + lane;                   // TMEM lane = operand row 2r + a
    const int r = n >> 1, a = n & 1;                // right-hand side within the group, part
    const bool rok = r < nr;
    const uint32_t lanebase = tmem + ((uint32_t)(q4 * 32) << 16);
    const long long len = (long long)b * m;
    const c32* lc = (const c32*)g.lcoef + s.vofs * 5;   // planes: C, W, E, S, N
    const c32* cSp = lc + 3 * len;
    const c32* cNp = lc + 4 * len;
    const long long vo = lvofs(s, r0 + (rok ? r : 0), nrhs);
    const c32* srcv = src + vo;
    c32* outv = out + vo;
    const int nh1 = H1 / 8;
    // this thread's rows of half h: 4 consecutive rows i = 8 cc + 4 a + e (e = 0..3) of its
    // right-hand side r, for the 8-row chunks cc = c0h(h) + par + TC2_NPAR ci < c1h(h)
    auto c0h = [&](int h) { return h ? nh1 : 0; };
    auto c1h = [&](int h) { return h ? ng : nh1; };
    auto chunk = [&](int h, int ci) { return c0h(h) + par + TC2_NPAR * ci; };
    // operand row write: this lane's row (part a of right-hand side r), columns j = 8 cc .. + 7
    auto put8 = [&](int cc, const float* v) {
      float hi[8], lo[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) tc::split_tf32(v[e], hi[e], lo[e]);
      tc::tmem_st8(lanebase + TC2_AH + (uint32_t)(8 * cc), hi);
      tc::tmem_st8(lanebase + TC2_AL + (uint32_t)(8 * cc), lo);
    };
    // block 0: y_0 = r_0 (both halves)
    for (int h = 0; h < 2; ++h)
      for (int ci = 0; ci < TC2_MAXCH; ++ci) {
        const int cc = chunk(h, ci);
        if (cc >= c1h(h)) break;
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
    if (tid == 0) {
      tc::bar_arrive(tc::smem_addr(&s_yready[0]));
      tc::bar_arrive(tc::smem_addr(&s_yready[1]));
    }
    // values the epilogue of block bi needs, loaded one block ahead (4 rows per chunk):
    //   pass 0: pa = r_{k+1} (next block's source);  pass 1: pa = t_k
    c32 pa[2][TC2_MAXCH][4];
    auto prefetch = [&](int bi, int h) {
      int pass, k;
      seq2(bi, m, pass, k);
      const bool need = rok && (pass == 1 || k + 1 < m);
      const long long o = pass == 0 ? (long long)(k + 1) * b : (long long)k * b;
      const c32* p = pass == 0 ? srcv : outv;
#pragma unroll
      for (int ci = 0; ci < TC2_MAXCH; ++ci) {
        const int cc = chunk(h, ci);
        const int i0 = 8 * cc + 4 * a;
#pragma unroll
        for (int e = 0; e < 4; ++e)
          pa[h][ci][e] = (need && cc < c1h(h) && i0 + e < b) ? p[o + i0 + e] : mk<float>(0.f, 0.f);
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
    prefetch(0, 0);
    prefetch(0, 1);
    coef_copy(0);
    bool alive = true;
    for (int bi = 0; bi < nblk && alive; ++bi) {
      int pass, k;
      seq2(bi, m, pass, k);
      const bool more = bi + 1 < nblk;
      int npass = 0, nk = 0;
      if (more) seq2(bi + 1, m, npass, nk);
      const c32* cnext = s_coef[bi & 1];
      const long long ko = (long long)k * b;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        // one thread waits for the accumulators of this half; the others sleep in the barrier,
        // which also makes every thread's coefficient copies visible
        if (h == 0) cp_async_wait_all();
        bool got = true;
        if (tid == 0) got = tc::bar_wait_or_abort(tc::smem_addr(&s_dfull[h]), (uint32_t)(bi & 1), abort_flag);
        if (epi_any(!got)) { alive = false; break; }
        tc::fence_after();
        const uint32_t dre = (h ? (uint32_t)(2 * H1) : 0u), dim = dre + (uint32_t)(h ? H2 : H1);
        float v8[TC2_MAXCH][8];
#pragma unroll
        for (int ci = 0; ci < TC2_MAXCH; ++ci) {
          const int cc = chunk(h, ci);
          if (cc >= c1h(h)) break;                       // warp-uniform
          const uint32_t lcol = (uint32_t)(8 * (cc - c0h(h)));
          uint32_t u0[8], u1[8];
          tc::tmem_ld8_async(lanebase + dre + lcol, u0);   // Y_a G_r, rows 8cc..
          tc::tmem_ld8_async(lanebase + dim + lcol, u1);   // Y_a G_i
          tc::tmem_wait_ld();
          // this lane's 4 rows i = 8 cc + 4 a + e; the partner lane holds the other part of y
          c32 y[4];
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
            const c32 v = pass == 0 ? C : pa[h][ci][e] - C;          // t_k, or x_k = t_k - G_k z
            if (rok && i < b) outv[ko + i] = v;
            c32 yv = mk<float>(0.f, 0.f);
            if (more && i < b) {
              const c32 cf = cnext[i];   // shared memory
              yv = npass == 0 ? pa[h][ci][e] - cf * v : cf * v;
            }
            y[e] = yv;
          }
          // row values of the next operand: part a of y at the chunk's 8 rows; the partner lane
          // holds the other 4 rows
          float send[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) send[e] = a == 0 ? y[e].y : y[e].x;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float recv = __shfl_xor_sync(0xffffffffu, send[e], 1);
            v8[ci][e] = a == 0 ? y[e].x : recv;
            v8[ci][4 + e] = a == 0 ? recv : y[e].y;
          }
        }
        if (more) {
          // column half 0 of the operand is still read by quarter (1,0) of this block
          if (h == 0) {
            if (tid == 0) got = tc::bar_wait_or_abort(tc::smem_addr(&s_ofree), (uint32_t)(bi & 1), abort_flag);
            if (epi_any(!got)) { alive = false; break; }
            tc::fence_after();
          }
#pragma unroll
          for (int ci = 0; ci < TC2_MAXCH; ++ci) {
            const int cc = chunk(h, ci);
            if (cc >= c1h(h)) break;
            put8(cc, v8[ci]);
          }
          tc::tmem_wait_st();
          tc::fence_before();
          epi_sync();
          if (tid == 0) tc::bar_arrive(tc::smem_addr(&s_yready[h]));
          prefetch(bi + 1, h);
          if (h == 1) coef_copy(bi + 1);
        }
      }
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
    if (c->d_gtc2) cudaFree(c->d_gtc2);
    c->d_gtc2 = nullptr;
    c->gtc2_cap = 0;
    c->drop_graphs();
    if ((e = cudaMalloc((void**)&c->d_gtc2, sizeof(float) * (size_t)total)) != cudaSuccess) return e;
    c->gtc2_cap = (size_t)total;
  }
  if ((size_t)c->nfac > c->tc2ofs_cap) {
    if (c->d_tc2ofs) cudaFree(c->d_tc2ofs);
    c->d_tc2ofs = nullptr;
    c->tc2ofs_cap = 0;
    c->drop_graphs();
    if ((e = cudaMalloc((void**)&c->d_tc2ofs, sizeof(long long) * c->nfac)) != cudaSuccess) return e;
    c->tc2ofs_cap = (size_t)c->nfac;
  }
  TC2Fac* d_facs = nullptr;
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

// shared memory of the solve (ring of stages, each the largest quarter, 16 H1^2 bytes); 0 if the
// blocks are too wide (b > 128), too narrow for two halves (b <= 8) or fewer than two stages fit
static size_t tc2d_smem(const ddm_ctx* c, int* nst_out, uint32_t* stage_out) {
  int bmax = 0, bmin = 1 << 30;
  for (auto& s : c->subs) {
    bmax = std::max(bmax, s.ext[0]);
    bmin = std::min(bmin, s.ext[0]);
  }
  if (bmax > 128 || bmin <= 8) return 0;
  const size_t h1 = tc2_h1((bmax + 7) / 8);
  const size_t stage = 16 * h1 * h1;
  const size_t fixed = 128;
  const size_t limit = 227 * 1024 - 4096;   // the kernel's static shared memory beside it
  if (fixed + 2 * stage > limit) return 0;
  const int nst = (int)std::min<size_t>(TC2_MAXST, (limit - fixed) / stage);
  *nst_out = nst;
  *stage_out = (uint32_t)stage;
  return fixed + (size_t)nst * stage;
}

bool tc2d_supported(const ddm_ctx* c, int nrt) {
  int nst = 0;
  uint32_t stage = 0;
  return c->d_gtc2 && nrt == TC2_NRT && tc2d_smem(c, &nst, &stage) > 0;
}

cudaError_t tc2d_solve(ddm_ctx* c, int nrt, const void* src, void* out, void* U, int nrhs) {
  if (nrt != TC2_NRT) return cudaErrorInvalidValue;
  int nst = 0;
  uint32_t stage = 0;
  const size_t sm = tc2d_smem(c, &nst, &stage);
  if (!sm) return cudaErrorInvalidConfiguration;
  cudaError_t e = allow_dynamic_smem((const void*)k_solve2d_tc, sm);
  if (e != cudaSuccess) return e;
  dim3 grid((nrhs + TC2_NRT - 1) / TC2_NRT, c->g.nsub);
  ++c->nlaunch;
  k_solve2d_tc<<<grid, TC2_THREADS, sm, c->st>>>(c->g, c->d_gtc2, c->d_tc2ofs, (const c32*)src, (c32*)out, nrhs,
                                                 nst, stage, c->d_err);
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

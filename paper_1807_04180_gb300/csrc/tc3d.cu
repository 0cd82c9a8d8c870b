// Tensor-core (tcgen05) plane step of the 3D local solves in mixed precision.
//
// A 3D subdomain factor keeps, per z-plane k, the dense block G_k = D_k^{-1} (b x b complex,
// b = ext_x * ext_y); every subdomain and right-hand side that shares the factor is a column of
// one operand Y, so each plane step of the forward and backward sweeps is the complex
// contraction C = G_k Y (the block solves of Algorithm 3.1 in 3D).  Here it runs on the
// 5th-generation tensor cores as four real products per complex product (planar real and
// imaginary parts, the minus sign through the instruction's negate-B bit), each in "3xTF32":
// every FP32 operand x is split into hi = tf32(x) and lo = x - hi, and hi*hi + hi*lo + lo*hi is
// accumulated in FP32 in tensor memory, which keeps FP32-level accuracy.
//
// Data layout (all K-major, no swizzle, see tcgen05.cuh):
//  - factor, packed once after the factorisation: per plane k, i-tile (128 rows of G_k) and
//    K-chunk (8 columns j) one 16 KB block of four 4 KB planes {Re hi, Re lo, Im hi, Im lo};
//  - operand Y, packed before each plane step: per q-tile (128 columns) and K-chunk the same
//    four planes of Y^T (row q = column q of Y).
// One CTA computes the 128 x 128 output tile D[q][i] = sum_j Y[j][q] G_k[i][j] for one q-tile and
// one i-tile: a producer thread streams the (factor, operand) block pairs through a ring of
// shared-memory stages with cp.async.bulk, one thread issues the 12 MMAs per chunk and frees the
// stage with tcgen05.commit, and after the last chunk the four warps read the two accumulators
// (real: TMEM columns 0-127, imaginary: 128-255) back with tcgen05.ld and apply the sweep's
// update to the local vectors (the same update as the CUDA-core plane step).
#include <algorithm>
#include <vector>

#include "ddm_internal.cuh"
#include "tcgen05.cuh"


namespace ddm {

constexpr int TC3_TILE = 128;                  // rows of an i-tile, columns of a q-tile
constexpr int TC3_KC = 8;                      // K (j) per chunk = one tf32 MMA step
constexpr int TC3_PLANE = TC3_TILE * TC3_KC;   // floats per plane of a block (4 KB)
constexpr int TC3_BLOCK = 4 * TC3_PLANE;       // floats per block (16 KB)
constexpr int TC3_NST = 6;                     // ring stages, 32 KB each
constexpr int TC3_SMEM = TC3_NST * 2 * TC3_BLOCK * 4 + 1024;
constexpr uint32_t TC3_TCOLS = 256;            // TMEM columns allocated (and freed) per CTA

// packed factor of one plane: blocks (it, kc), it < nIT, kc < nKC
__global__ void k_g3_pack(const c32* __restrict__ G, long long fofs, int ldb, int b, int m, int nIT, int nKC,
                          float* __restrict__ gtc) {
  const long long nI = (long long)nIT * TC3_TILE, nJ = (long long)nKC * TC3_KC;
  const long long total = (long long)m * nJ * nI;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % nI);
    const long long r = idx / nI;
    const int j = (int)(r % nJ);
    const int k = (int)(r / nJ);
    c32 v = mk<float>(0.f, 0.f);
    if (i < b && j < b) v = G[fofs + ((long long)k * b + j) * ldb + i];
    float rh, rl, ih, il;
    tc::split_tf32(v.x, rh, rl);
    tc::split_tf32(v.y, ih, il);
    const int it = i / TC3_TILE, kc = j / TC3_KC;
    float* blk = gtc + (((long long)k * nIT + it) * nKC + kc) * TC3_BLOCK;
    const int e = tc::kmajor_index(i % TC3_TILE, j % TC3_KC, TC3_KC);
    blk[e] = rh;
    blk[TC3_PLANE + e] = rl;
    blk[2 * TC3_PLANE + e] = ih;
    blk[3 * TC3_PLANE + e] = il;
  }
}

// operand of plane step (pass, k) for the columns q < ncol (zero padding elsewhere):
//   pass 0: Y[j][q] = src_q[k b + j] - c_zm(j, k) out_q[(k-1) b + j]
//   pass 1: Y[j][q] = c_zp(j, k) out_q[(k+1) b + j]
__global__ void k_y3_pack(int pass, int k, int b, int nKC, int nQT, const long long* __restrict__ colofs, int ncol,
                          const c32* __restrict__ src, const c32* __restrict__ out, const c32* __restrict__ cS,
                          const c32* __restrict__ cN, float* __restrict__ ytc) {
  const long long nJ = (long long)nKC * TC3_KC;
  const long long total = (long long)nQT * TC3_TILE * nJ;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(idx % nJ);
    const int q = (int)(idx / nJ);
    c32 v = mk<float>(0.f, 0.f);
    if (q < ncol && j < b) {
      const long long base = colofs[q];
      if (pass == 0) {
        v = src[base + (long long)k * b + j];
        if (k > 0) v = v - cS[(long long)k * b + j] * out[base + (long long)(k - 1) * b + j];
      } else {
        v = cN[(long long)k * b + j] * out[base + (long long)(k + 1) * b + j];
      }
    }
    float rh, rl, ih, il;
    tc::split_tf32(v.x, rh, rl);
    tc::split_tf32(v.y, ih, il);
    const int qt = q / TC3_TILE, kc = j / TC3_KC;
    float* blk = ytc + ((long long)qt * nKC + kc) * TC3_BLOCK;
    const int e = tc::kmajor_index(q % TC3_TILE, j % TC3_KC, TC3_KC);
    blk[e] = rh;
    blk[TC3_PLANE + e] = rl;
    blk[2 * TC3_PLANE + e] = ih;
    blk[3 * TC3_PLANE + e] = il;
  }
}

// Contraction of one plane step (pass, k) on the tensor cores; grid (nIT, nQT, nsplit), 128
// threads.  Warp 0 lane 0 streams the (factor, operand) block pairs of this CTA's K range (the
// range is split nsplit ways across blockIdx.z so that the grid fills the SMs) through the stage
// ring, warp 1 lane 0 issues the MMAs, and the four warps then store the FP32 accumulators as
// the partial tile part[tile][split][q][0..127 real | 128..255 imaginary] (coalesced 16-byte
// stores).  k_epi3d adds the partials and applies the sweep's update.
__global__ void __launch_bounds__(128, 1)
    k_gemm3d_tc(const float* __restrict__ gplane, const float* __restrict__ ycur, int nKC, int nsplit,
                float* __restrict__ part, int* err) {
  extern __shared__ unsigned char dsm_raw[];
  __shared__ __align__(8) uint64_t s_full[TC3_NST], s_empty[TC3_NST], s_accf;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int it = blockIdx.x, qt = blockIdx.y, split = blockIdx.z;
  const int kc0 = (int)((long long)split * nKC / nsplit), kc1 = (int)((long long)(split + 1) * nKC / nsplit);
  // stages: 1 KB aligned (16 bytes is what the copies and descriptors need)
  const uint32_t dsm = (tc::smem_addr(dsm_raw) + 1023u) & ~1023u;
  const uint32_t STAGE_BYTES = 2 * TC3_BLOCK * 4;

  if (warp == 0) tc::tmem_alloc(tc::smem_addr(&s_tmem), TC3_TCOLS);
  if (tid == 0) {
    for (int s = 0; s < TC3_NST; ++s) {
      tc::bar_init(tc::smem_addr(&s_full[s]), 1);
      tc::bar_init(tc::smem_addr(&s_empty[s]), 1);
    }
    tc::bar_init(tc::smem_addr(&s_accf), 1);
    s_fail = 0;
    tc::bar_init_fence();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = s_tmem;

  const float* gbase = gplane + (long long)it * nKC * TC3_BLOCK;
  const float* ybase = ycur + (long long)qt * nKC * TC3_BLOCK;
  if (warp == 0 && lane == 0) {
    // producer
    for (int kc = kc0; kc < kc1; ++kc) {
      const int u = kc - kc0, s = u % TC3_NST;
      if (u >= TC3_NST && !tc::bar_wait(tc::smem_addr(&s_empty[s]), (uint32_t)((u / TC3_NST) - 1) & 1u)) {
        s_fail = 1;
        atomicOr(err, ERRBIT_TIMEOUT);
        break;
      }
      const uint32_t fb = tc::smem_addr(&s_full[s]);
      const uint32_t st = dsm + (uint32_t)s * STAGE_BYTES;
      tc::bar_expect_tx(fb, STAGE_BYTES);
      tc::bulk_load(st, gbase + (long long)kc * TC3_BLOCK, TC3_BLOCK * 4, fb);
      tc::bulk_load(st + TC3_BLOCK * 4, ybase + (long long)kc * TC3_BLOCK, TC3_BLOCK * 4, fb);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: A = Y^T tile (M = 128 columns q), B = G_k tile (N = 128 rows i), K = 8 per chunk
    constexpr uint32_t ID = tc::idesc_tf32(TC3_TILE, TC3_TILE, false);
    constexpr uint32_t IDN = tc::idesc_tf32(TC3_TILE, TC3_TILE, true);
    const uint32_t accR = tmem, accI = tmem + TC3_TILE;
    const uint32_t LBO = 128, SBO = (TC3_KC / 4) * 128;
    for (int kc = kc0; kc < kc1; ++kc) {
      const int u = kc - kc0, s = u % TC3_NST;
      if (!tc::bar_wait(tc::smem_addr(&s_full[s]), (uint32_t)(u / TC3_NST) & 1u)) {
        s_fail = 1;
        atomicOr(err, ERRBIT_TIMEOUT);
        break;
      }
      tc::fence_after();
      const uint32_t g0 = dsm + (uint32_t)s * STAGE_BYTES, y0 = g0 + TC3_BLOCK * 4;
      const uint64_t Grh = tc::sdesc(g0, LBO, SBO), Grl = tc::sdesc(g0 + TC3_PLANE * 4, LBO, SBO);
      const uint64_t Gih = tc::sdesc(g0 + 2 * TC3_PLANE * 4, LBO, SBO), Gil = tc::sdesc(g0 + 3 * TC3_PLANE * 4, LBO, SBO);
      const uint64_t Yrh = tc::sdesc(y0, LBO, SBO), Yrl = tc::sdesc(y0 + TC3_PLANE * 4, LBO, SBO);
      const uint64_t Yih = tc::sdesc(y0 + 2 * TC3_PLANE * 4, LBO, SBO), Yil = tc::sdesc(y0 + 3 * TC3_PLANE * 4, LBO, SBO);
      const uint32_t first = kc > kc0 ? 1u : 0u;
      // Re: Yr Gr - Yi Gi
      tc::mma_tf32(accR, Yrh, Grh, ID, first);
      tc::mma_tf32(accR, Yrh, Grl, ID, 1u);
      tc::mma_tf32(accR, Yrl, Grh, ID, 1u);
      tc::mma_tf32(accR, Yih, Gih, IDN, 1u);
      tc::mma_tf32(accR, Yih, Gil, IDN, 1u);
      tc::mma_tf32(accR, Yil, Gih, IDN, 1u);
      // Im: Yr Gi + Yi Gr
      tc::mma_tf32(accI, Yrh, Gih, ID, first);
      tc::mma_tf32(accI, Yrh, Gil, ID, 1u);
      tc::mma_tf32(accI, Yrl, Gih, ID, 1u);
      tc::mma_tf32(accI, Yih, Grh, ID, 1u);
      tc::mma_tf32(accI, Yih, Grl, ID, 1u);
      tc::mma_tf32(accI, Yil, Grh, ID, 1u);
      tc::mma_commit(tc::smem_addr(&s_empty[s]));
    }
    tc::mma_commit(tc::smem_addr(&s_accf));
  }
  __syncwarp();
  const bool got = tc::bar_wait(tc::smem_addr(&s_accf), 0u);
  const int bad = __syncthreads_or(!got || s_fail);
  tc::fence_after();
  if (!bad) {
    const int q = warp * 32 + lane;
    const long long tile = (long long)qt * gridDim.x + it;
    float4* dst = reinterpret_cast<float4*>(part + ((tile * nsplit + split) * TC3_TILE + q) * (2 * TC3_TILE));
    const uint32_t lanebase = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < 2 * TC3_TILE; c0 += 16) {
      float v[16];
      tc::tmem_ld16(lanebase + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 4; ++j) __stcg(dst + c0 / 4 + j, make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]));
    }
  } else if (tid == 0) {
    atomicOr(err, ERRBIT_TIMEOUT);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, TC3_TCOLS);
}

// Epilogue of plane step (pass, k): one thread per (tile, q, i), consecutive threads along i.
// C = sum of the nsplit partials (in split order), then the sweep's update
//   pass 0: out = C (at k = m-1 also U += C);  pass 1: x = out - C, out = x, U += x,
// and, when a next step (npass, nk) exists, its operand packed into ynext from the same values:
//   npass 0 (nk = k+1): Y[j][q] = src_q[nk b + j] - c_zm(j, nk) C[j][q]
//   npass 1 (nk = k-1, or m-2 at the turn): Y[j][q] = c_zp(j, nk) out_q[(nk+1) b + j]
// (coefn = the c_zm or c_zp plane nk; rows b <= j < 8 nKC of the operand are written as zeros).
__global__ void __launch_bounds__(256) k_epi3d(const float* __restrict__ part, int nIT, int nQT, int nsplit, int nKC,
                                               int b, int pass, int k, int m, int npass, int nk,
                                               const c32* __restrict__ coefn, const long long* __restrict__ colofs,
                                               int ncol, const c32* __restrict__ src, c32* out, c32* U,
                                               float* __restrict__ ynext) {
  const long long total = (long long)nIT * nQT * TC3_TILE * TC3_TILE;
  const int jpad = nKC * TC3_KC;
  const bool upd = U && (pass == 1 || k == m - 1);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int il = (int)(idx % TC3_TILE);
    const long long r = idx / TC3_TILE;
    const int ql = (int)(r % TC3_TILE);
    const long long tile = r / TC3_TILE;
    const int it = (int)(tile % nIT), qt = (int)(tile / nIT);
    const int q = qt * TC3_TILE + ql, i = it * TC3_TILE + il;
    if (q >= ncol || i >= jpad) continue;
    c32 v = mk<float>(0.f, 0.f);
    const long long base = colofs[q];
    if (i < b) {
      const float* p = part + (tile * nsplit * TC3_TILE + ql) * (2 * TC3_TILE) + il;
      float vr = 0.f, vi = 0.f;
      for (int sp = 0; sp < nsplit; ++sp) {
        vr += __ldcg(p + (long long)sp * TC3_TILE * (2 * TC3_TILE));
        vi += __ldcg(p + (long long)sp * TC3_TILE * (2 * TC3_TILE) + TC3_TILE);
      }
      v = mk<float>(vr, vi);
      const long long o = base + (long long)k * b + i;
      if (pass == 1) v = out[o] - v;
      out[o] = v;
      if (upd) U[o] = U[o] + v;
    }
    if (npass >= 0) {
      c32 y = mk<float>(0.f, 0.f);
      if (i < b) y = npass == 0 ? src[base + (long long)nk * b + i] - coefn[i] * v : coefn[i] * v;
      float rh, rl, ih, il2;
      tc::split_tf32(y.x, rh, rl);
      tc::split_tf32(y.y, ih, il2);
      float* blk = ynext + ((long long)qt * nKC + i / TC3_KC) * TC3_BLOCK;
      const int e = tc::kmajor_index(ql, i % TC3_KC, TC3_KC);
      blk[e] = rh;
      blk[TC3_PLANE + e] = rl;
      blk[2 * TC3_PLANE + e] = ih;
      blk[3 * TC3_PLANE + e] = il2;
    }
  }
}

// ------------------------------------------------------------------------------------ host
long long tc3d_packed_floats(int b, int m) {
  const long long nIT = (b + TC3_TILE - 1) / TC3_TILE, nKC = (b + TC3_KC - 1) / TC3_KC;
  return (long long)m * nIT * nKC * TC3_BLOCK;
}

// pack every factor after the factorisation (mixed precision only)
cudaError_t tc3d_pack_factors(ddm_ctx* c) {
  cudaError_t e = cudaSuccess;
  long long total = 0;
  c->tc_ofs.assign(c->nfac, 0);
  for (int f = 0; f < c->nfac; ++f) {
    c->tc_ofs[f] = total;
    total += tc3d_packed_floats(c->fac_b[f], c->fac_m[f]);
  }
  if ((size_t)total > c->gtc_cap) {
    dev_free(c, c->d_gtc);
    c->d_gtc = nullptr;
    c->gtc_cap = 0;
    if ((e = dev_alloc(c, (void**)&c->d_gtc, sizeof(float) * (size_t)total)) != cudaSuccess) return e;
    c->gtc_cap = (size_t)total;
  }
  for (int f = 0; f < c->nfac; ++f) {
    const int b = c->fac_b[f], m = c->fac_m[f];
    const int nIT = (b + TC3_TILE - 1) / TC3_TILE, nKC = (b + TC3_KC - 1) / TC3_KC;
    ++c->nlaunch;
    k_g3_pack<<<1216, 256, 0, c->st>>>((const c32*)c->d_G, c->fac_ofs[f], c->fac_ldb[f], b, m, nIT, nKC,
                                       c->d_gtc + c->tc_ofs[f]);
  }
  return cudaGetLastError();
}

// all plane steps of the forward and backward sweeps of one factor group
cudaError_t tc3d_sweeps(ddm_ctx* c, int f, const long long* d_colofs, int ncol, const c32* cS, const c32* cN,
                        const c32* src, c32* out, c32* U) {
  cudaError_t e = allow_dynamic_smem((const void*)k_gemm3d_tc, TC3_SMEM);
  if (e != cudaSuccess) return e;
  const int b = c->fac_b[f], m = c->fac_m[f];
  const int nIT = (b + TC3_TILE - 1) / TC3_TILE, nKC = (b + TC3_KC - 1) / TC3_KC;
  const int nQT = (ncol + TC3_TILE - 1) / TC3_TILE;
  const size_t need = (size_t)nQT * nKC * TC3_BLOCK;   // one operand buffer; two are kept
  if (need > c->ytc_cap) {
    dev_free(c, c->d_ytc);
    c->d_ytc = nullptr;
    c->ytc_cap = 0;
    if ((e = dev_alloc(c, (void**)&c->d_ytc, sizeof(float) * 2 * need)) != cudaSuccess) return e;
    // padding rows (columns q >= ncol) stay zero in both buffers
    if ((e = cudaMemsetAsync(c->d_ytc, 0, sizeof(float) * 2 * need, c->st)) != cudaSuccess) return e;
    c->ytc_cap = need;
  }
  // split K so that tiles x splits fill the SMs once (one CTA per SM: 197 KB of stages)
  int nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int tiles = nIT * nQT;
  const int nsplit = std::max(1, std::min({8, nKC, std::max(nsm, 1) / tiles}));
  const size_t pneed = (size_t)tiles * nsplit * TC3_TILE * 2 * TC3_TILE;
  if (pneed > c->tcpart_cap) {
    dev_free(c, c->d_tcpart);
    c->d_tcpart = nullptr;
    c->tcpart_cap = 0;
    if ((e = dev_alloc(c, (void**)&c->d_tcpart, sizeof(float) * pneed)) != cudaSuccess) return e;
    c->tcpart_cap = pneed;
  }
  const long long etotal = (long long)tiles * TC3_TILE * TC3_TILE;
  const int egrid = (int)std::min<long long>((etotal + 255) / 256, 152LL * 64);
  const long long plane = (long long)nIT * nKC * TC3_BLOCK;
  const float* gtc = c->d_gtc + c->tc_ofs[f];
  const long long packed = (long long)nQT * TC3_TILE * nKC * TC3_KC;
  const int pgrid = (int)std::min<long long>((packed + 255) / 256, 152LL * 16);
  float* ybuf[2] = {c->d_ytc, c->d_ytc + need};
  ++c->nlaunch;
  k_y3_pack<<<pgrid, 256, 0, c->st>>>(0, 0, b, nKC, nQT, d_colofs, ncol, src, out, cS, cN, ybuf[0]);
  for (int s = 0; s < 2 * m - 1; ++s) {
    const int pass = s < m ? 0 : 1;
    const int k = pass == 0 ? s : 2 * m - 2 - s;
    // the step after this one: forward k+1, the turn to backward m-2, backward k-1, or none
    const int sn = s + 1;
    const int npass = sn >= 2 * m - 1 ? -1 : (sn < m ? 0 : 1);
    const int nk = npass < 0 ? 0 : (npass == 0 ? sn : 2 * m - 2 - sn);
    const c32* coefn = npass == 0 ? cS + (long long)nk * b : cN + (long long)nk * b;
    c->nlaunch += 2;
    k_gemm3d_tc<<<dim3(nIT, nQT, nsplit), 128, TC3_SMEM, c->st>>>(gtc + k * plane, ybuf[s & 1], nKC, nsplit,
                                                                  c->d_tcpart, c->d_err);
    k_epi3d<<<egrid, 256, 0, c->st>>>(c->d_tcpart, nIT, nQT, nsplit, nKC, b, pass, k, m, npass, nk, coefn, d_colofs,
                                      ncol, src, out, U, ybuf[(s + 1) & 1]);
  }
  return cudaGetLastError();
}

}  // namespace ddm

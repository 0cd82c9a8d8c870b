// C ABI of libddm: set-up, factorisation with sharing of identical subdomains, the DDM
// step loop of Algorithm 3.1, the DDM(K) preconditioner, flexible GMRES and the stepping
// solver of Section 4.2.  Host code only orchestrates; all arithmetic runs in the kernels.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include <mutex>
#include <set>

#include "ddm_internal.cuh"

using namespace ddm;


static std::string g_setup_err;

namespace ddm {
// message of a failed call that has no context (read with ddm_last_error(NULL))
void set_global_error(const std::string& msg) { g_setup_err = msg; }
}  // namespace ddm

static ddm_status fail(ddm_ctx* c, ddm_status st, const std::string& msg) {
  if (c) c->err = msg; else g_setup_err = msg;
  return st;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t _e = (call);                                                                  \
    if (_e != cudaSuccess)                                                                    \
      return fail(c, _e == cudaErrorMemoryAllocation ? DDM_E_NOMEM : DDM_E_CUDA,              \
                  std::string(#call) + ": " + cudaGetErrorString(_e));                        \
  } while (0)

#define CKS(expr)                 \
  do {                            \
    ddm_status _s = (expr);       \
    if (_s != DDM_OK) return _s;  \
  } while (0)

static size_t local_elem(const ddm_ctx* c) { return c->prec == DDM_MIXED ? sizeof(c32) : sizeof(z64); }

// ------------------------------------------------------------------ timing helpers
static cudaEvent_t ev_get(ddm_ctx* c) {
  if (!c->ev_pool.empty()) { cudaEvent_t e = c->ev_pool.back(); c->ev_pool.pop_back(); return e; }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}
static void timing_drain(ddm_ctx* c) {
  for (auto& pe : c->ev_pending) {
    cudaEventSynchronize(pe.second.second);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, pe.second.first, pe.second.second);
    c->t_ms[pe.first] += ms;
    c->t_n[pe.first] += 1;
    c->ev_pool.push_back(pe.second.first);
    c->ev_pool.push_back(pe.second.second);
  }
  c->ev_pending.clear();
}
struct TScope {
  ddm_ctx* c; int slot; cudaEvent_t e0 = nullptr;
  TScope(ddm_ctx* cc, int s) : c(cc), slot(s) {
    if (c->timing) { e0 = ev_get(c); cudaEventRecord(e0, c->st); }
  }
  ~TScope() {
    if (c->timing) {
      cudaEvent_t e1 = ev_get(c);
      cudaEventRecord(e1, c->st);
      c->ev_pending.push_back({slot, {e0, e1}});
      if (c->ev_pending.size() > 4096) timing_drain(c);
    }
  }
};

static ddm_status check_err_word(ddm_ctx* c) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (h & ERRBIT_TIMEOUT) return fail(c, DDM_E_TIMEOUT, "a bounded device wait timed out");
  if (h & ERRBIT_SINGULAR) return fail(c, DDM_E_SINGULAR, "zero or non-finite pivot in a subdomain factor");
  return DDM_OK;
}

// =====================================================================================
// set-up
// =====================================================================================
extern "C" ddm_status ddm_setup(const ddm_params* p, double omega, const double* c_dev, void* stream, ddm_ctx** out) {
  ddm_ctx* c = nullptr;
  if (!p || !out || !c_dev) return fail(nullptr, DDM_E_INVAL, "null argument");
  *out = nullptr;
  if (p->dim != 2 && p->dim != 3) return fail(nullptr, DDM_E_INVAL, "dim must be 2 or 3");
  if (p->overlap < 1 || p->pml < 1) return fail(nullptr, DDM_E_INVAL, "overlap and pml must be >= 1");
  if (!(p->h > 0) || !(omega > 0) || p->sigma0 < 0) return fail(nullptr, DDM_E_INVAL, "h, omega must be > 0, sigma0 >= 0");
  if (p->precision != DDM_FP64 && p->precision != DDM_MIXED) return fail(nullptr, DDM_E_INVAL, "bad precision");
  if (p->max_rhs < 1 || p->max_rhs > 4096) return fail(nullptr, DDM_E_INVAL, "max_rhs must be in [1, 4096]");
  c = new ddm_ctx();
  c->p = *p;
  c->omega = omega;
  c->st = (cudaStream_t)stream;
  c->dim = p->dim;
  c->e = p->overlap + p->pml;
  c->prec = p->precision;
  const int d = c->dim, e = c->e, ov = p->overlap;
  Geom& g = c->g;
  memset(&g, 0, sizeof(g));
  g.dim = d; g.e = e; g.ov = ov; g.h2 = p->h * p->h;
  // cuts
  for (int a = 0; a < 3; ++a) {
    if (a >= d) { g.N[a] = 1; g.parts[a] = 1; continue; }
    if (p->n[a] < 1 || p->parts[a] < 1 || p->parts[a] > 4096) { delete c; return fail(nullptr, DDM_E_INVAL, "bad n / parts"); }
    g.N[a] = (int)(p->n[a] + 2 * e);
    g.parts[a] = p->parts[a];
    for (int i = 0; i <= p->parts[a]; ++i) {
      int64_t v = p->cuts[a] ? p->cuts[a][i] : (p->n[a] * i) / p->parts[a];
      c->cuts_h[a][i] = v;
    }
    if (c->cuts_h[a][0] != 0 || c->cuts_h[a][p->parts[a]] != p->n[a]) { delete c; return fail(nullptr, DDM_E_INVAL, "cuts must run from 0 to n"); }
    for (int i = 0; i < p->parts[a]; ++i) {
      int64_t w = c->cuts_h[a][i + 1] - c->cuts_h[a][i];
      if (w < 2 * ov || w < 2) { delete c; return fail(nullptr, DDM_E_INVAL, "every part must be at least 2*overlap nodes wide"); }
      if (d == 2 && a == 0 && w + 2 * e > 1024) { delete c; return fail(nullptr, DDM_E_INVAL, "x-extent of a 2D subdomain (own + 2(overlap+pml)) must be <= 1024"); }
      // the 2D kernels keep a block in shared memory / registers: up to 128 nodes in complex64,
      // 96 in complex128; wider x-lines take the dense-block path
      if (d == 2 && a == 0 && w + 2 * e > (p->precision == DDM_MIXED ? 128 : 96)) c->blockpath = true;
      if (d == 3 && a < 2 && w + 2 * e > 96) { delete c; return fail(nullptr, DDM_E_INVAL, "x- and y-extents of a 3D subdomain must be <= 96"); }
    }
  }
  if (d == 3) c->blockpath = true;
  g.nglob = (long long)g.N[0] * g.N[1] * g.N[2];
  // alpha tables: one per (axis, part), then the global box per axis
  std::vector<int> tdesc;
  int tab_total = 0;
  std::vector<std::vector<int>> part_tab(3);
  for (int a = 0; a < d; ++a) {
    for (int i = 0; i < g.parts[a]; ++i) {
      int lo = (int)c->cuts_h[a][i], hi = (int)c->cuts_h[a][i + 1];
      part_tab[a].push_back(tab_total);
      tdesc.push_back(lo); tdesc.push_back(hi); tdesc.push_back(tab_total);
      tab_total += 2 * (hi - lo + 2 * e) + 1;
    }
  }
  for (int a = 0; a < d; ++a) {
    g.gtab[a] = tab_total;
    tdesc.push_back(0); tdesc.push_back((int)p->n[a]); tdesc.push_back(tab_total);
    tab_total += 2 * (int)(p->n[a] + 2 * e) + 1;
  }
  // subdomains, C order (z slowest, x fastest)
  g.nsub = g.parts[0] * g.parts[1] * g.parts[2];
  c->subs.resize(g.nsub);
  long long vofs = 0;
  for (int sid = 0; sid < g.nsub; ++sid) {
    SubDesc& s = c->subs[sid];
    memset(&s, 0, sizeof(s));
    int idx[3] = {sid % g.parts[0], (sid / g.parts[0]) % g.parts[1], sid / (g.parts[0] * g.parts[1])};
    for (int a = 0; a < 3; ++a) {
      s.idx[a] = idx[a];
      if (a < d) {
        s.lo[a] = (int)c->cuts_h[a][idx[a]];
        s.nown[a] = (int)(c->cuts_h[a][idx[a] + 1] - c->cuts_h[a][idx[a]]);
        s.ext[a] = s.nown[a] + 2 * e;
        s.tab[a] = part_tab[a][idx[a]];
        if (idx[a] == 0) s.at_lo |= 1 << a;
        if (idx[a] == g.parts[a] - 1) s.at_hi |= 1 << a;
      } else {
        s.lo[a] = 0; s.nown[a] = 1; s.ext[a] = 1; s.tab[a] = 0;
      }
    }
    s.vofs = vofs;
    vofs += (long long)s.ext[0] * s.ext[1] * s.ext[2];
    for (int code = 0; code < NDIR; ++code) {
      int dd[3] = {code % 3 - 1, (code / 3) % 3 - 1, code / 9 - 1};
      int nb[3];
      bool ok = true;
      for (int a = 0; a < 3; ++a) {
        if (a >= d && dd[a] != 0) ok = false;
        nb[a] = idx[a] - dd[a];   // the sender sits at R - d (d = direction of propagation)
        if (nb[a] < 0 || nb[a] >= g.parts[a]) ok = false;
      }
      s.nbr[code] = ok ? (nb[2] * g.parts[1] + nb[1]) * g.parts[0] + nb[0] : -1;
    }
  }
  g.ltotal = vofs;
  // strip-node lists: every receiver node that some direction's chi_d covers, q in [0, ov]
  // nodes inside each shared face (Section 2.2), with the directions as a bit mask
  std::vector<int> sidx;
  std::vector<unsigned> smask;
  for (int sid = 0; sid < g.nsub; ++sid) {
    SubDesc& s = c->subs[sid];
    s.sofs = (int)sidx.size();
    const long long len = (long long)s.ext[0] * s.ext[1] * s.ext[2];
    for (long long li = 0; li < len; ++li) {
      int x[3] = {(int)(li % s.ext[0]), (int)((li / s.ext[0]) % s.ext[1]), (int)(li / ((long long)s.ext[0] * s.ext[1]))};
      // a receiver node lies within ov + 1 nodes inside some face; skip the others at once
      bool near_face = false;
      for (int a = 0; a < d; ++a) {
        const int ql = x[a] - e, qh = e + s.nown[a] - 1 - x[a];
        near_face = near_face || (ql >= 0 && ql <= ov) || (qh >= 0 && qh <= ov);
      }
      if (!near_face) continue;
      unsigned mask = 0;
      for (int code = 0; code < NDIR; ++code) {
        if (code == 13 || s.nbr[code] < 0) continue;
        int dd[3] = {code % 3 - 1, (code / 3) % 3 - 1, code / 9 - 1};
        bool ok = true;
        for (int a = 0; a < d; ++a) {
          if (dd[a] > 0) { int q = x[a] - e; ok = ok && q >= 0 && q <= ov; }
          else if (dd[a] < 0) { int q = e + s.nown[a] - 1 - x[a]; ok = ok && q >= 0 && q <= ov; }
        }
        if (ok) mask |= 1u << code;
      }
      if (!mask) continue;
      bool own = true;
      for (int a = 0; a < d; ++a) {
        if (x[a] < e && !((s.at_lo >> a) & 1)) own = false;
        if (x[a] >= e + s.nown[a] && !((s.at_hi >> a) & 1)) own = false;
      }
      sidx.push_back((int)li);
      smask.push_back(mask | (own ? 0x80000000u : 0u));
    }
    s.scnt = (int)sidx.size() - s.sofs;
    c->max_scnt = std::max(c->max_scnt, s.scnt);
  }
  if (sidx.empty()) { sidx.push_back(0); smask.push_back(0); }
  // owner tables (global extended index -> part along the axis)
  std::vector<int> owner;
  int own_ofs[3] = {0, 0, 0};
  for (int a = 0; a < 3; ++a) {
    own_ofs[a] = (int)owner.size();
    for (int gi = 0; gi < g.N[a]; ++gi) {
      if (a >= d) { owner.push_back(0); continue; }
      int pnode = gi - e, part = 0;
      while (part + 1 < g.parts[a] && pnode >= c->cuts_h[a][part + 1]) ++part;
      owner.push_back(part);
    }
  }
  std::vector<int> cutsv;
  int cut_ofs[3];
  for (int a = 0; a < 3; ++a) {
    cut_ofs[a] = (int)cutsv.size();
    for (int i = 0; i <= g.parts[a]; ++i) cutsv.push_back(a < d ? (int)c->cuts_h[a][i] : i);
  }
  // device allocations
  const int R = p->max_rhs;
  const size_t le = local_elem(c);
  int maxlen = 0;
  for (auto& s : c->subs) maxlen = std::max(maxlen, s.ext[0] * s.ext[1] * s.ext[2]);
  c->npart = std::max<long long>((long long)R * g.nsub * ((maxlen + 127) / 128 + 1),
                                  (long long)R * 304LL * 2 * 122);
  int* d_tdesc = nullptr;
#define ALLOC(ptr, bytes) CK(dev_alloc(c, (void**)&(ptr), (bytes)))
  ddm_status st = DDM_OK;
  auto body = [&]() -> ddm_status {
    ALLOC(c->d_k2, sizeof(double) * g.nglob);
    ALLOC(c->d_lcoef, le * g.ltotal * (2 * d + 1));
    ALLOC(c->d_gcoef, sizeof(z64) * g.nglob * (2 * d + 1));
    ALLOC(c->d_tab, sizeof(z64) * tab_total);
    ALLOC(c->d_beta, sizeof(double) * (ov + 1));
    ALLOC(c->d_owner, sizeof(int) * owner.size());
    ALLOC(c->d_sidx, sizeof(int) * sidx.size());
    ALLOC(c->d_smask, sizeof(unsigned) * smask.size());
    ALLOC(c->d_cuts, sizeof(int) * cutsv.size());
    ALLOC(c->d_subs, sizeof(SubDesc) * g.nsub);
    ALLOC(c->d_err, sizeof(int));
    ALLOC(c->d_part, sizeof(double) * c->npart);
    ALLOC(c->d_scal, sizeof(double) * 64);
    CK(host_pinned_alloc((void**)&c->h_scal, sizeof(double) * 64));
    ALLOC(d_tdesc, sizeof(int) * tdesc.size());
    ALLOC(c->d_src, le * g.ltotal * R);
    ALLOC(c->d_U, le * g.ltotal * R);
    for (int k = 0; k < ring_slots(c); ++k) ALLOC(c->d_ring[k], le * g.ltotal * R);
    ALLOC(c->d_gb, sizeof(z64) * g.nglob * R);
    ALLOC(c->d_gr, sizeof(z64) * g.nglob * R);
    ALLOC(c->d_gw, sizeof(z64) * g.nglob * R);
    ALLOC(c->d_hash, sizeof(unsigned long long) * g.nsub);
    ALLOC(c->d_pairs, sizeof(int) * 2 * g.nsub);
    ALLOC(c->d_mis, sizeof(int) * g.nsub);
    ALLOC(c->d_reps, sizeof(int) * g.nsub);
    ALLOC(c->d_ldb, sizeof(int) * g.nsub);
    ALLOC(c->d_fofs, sizeof(long long) * g.nsub);
    ALLOC(c->d_fsel, sizeof(int) * g.nsub);
    CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st));
    CK(cudaMemcpyAsync(d_tdesc, tdesc.data(), sizeof(int) * tdesc.size(), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->d_owner, owner.data(), sizeof(int) * owner.size(), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->d_sidx, sidx.data(), sizeof(int) * sidx.size(), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->d_smask, smask.data(), sizeof(unsigned) * smask.size(), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->d_cuts, cutsv.data(), sizeof(int) * cutsv.size(), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->d_subs, c->subs.data(), sizeof(SubDesc) * g.nsub, cudaMemcpyHostToDevice, c->st));
    g.k2 = c->d_k2; g.tab = c->d_tab; g.beta = c->d_beta; g.subs = c->d_subs;
    g.lcoef = c->d_lcoef; g.gcoef = c->d_gcoef;
    g.sidx = c->d_sidx; g.smask = c->d_smask;
    for (int a = 0; a < 3; ++a) { g.owner[a] = c->d_owner + own_ofs[a]; g.cuts[a] = c->d_cuts + cut_ofs[a]; }
    CK(launch_build_tables(c, d_tdesc, (int)(tdesc.size() / 3), p->sigma0, p->pml_power, p->pml));
    CK(launch_k2(c, c_dev));
    CK(launch_beta(c));
    CK(launch_coefs(c));
    CK(cudaStreamSynchronize(c->st));
    return DDM_OK;
  };
  st = body();
  dev_free(c, d_tdesc);
  if (st != DDM_OK) {
    std::string msg = c->err;
    ddm_destroy(c);
    return fail(nullptr, st, msg);
  }
  *out = c;
  return DDM_OK;
}

extern "C" ddm_status ddm_destroy(ddm_ctx* c) {
  if (!c) return DDM_OK;
  cudaStreamSynchronize(c->st);
  for (auto& gr : c->graphs) cudaGraphExecDestroy(gr.exec);
  nd_free(c);
  if (c->gstream) cudaStreamSynchronize(c->gstream), cudaStreamDestroy(c->gstream);
  for (auto ev : c->gev) if (ev) cudaEventDestroy(ev);
  dev_free(c, c->d_gin);
  dev_free(c, c->d_gout);
  host_pinned_free(c->h_bscal);
  dev_free(c, c->d_bscal);
  dev_free(c, c->d_jr);
  void* ptrs[] = {c->d_subs, c->d_k2, c->d_lcoef, c->d_gcoef, c->d_sidx, c->d_smask, c->d_tab, c->d_beta, c->d_owner, c->d_cuts, c->d_err, c->d_part,
                  c->d_scal, c->d_G, c->d_src, c->d_U, c->d_ring[0], c->d_ring[1], c->d_ring[2], c->d_gb,
                  c->d_gr, c->d_gw, c->d_hostbuf, c->d_chost, c->d_col3d, c->d_V, c->d_Z, c->d_H, c->d_gs,
                  c->d_gtc, c->d_ytc, c->d_tcpart, c->d_gtc2, c->d_tc2ofs, c->d_hash, c->d_pairs, c->d_mis,
                  c->d_reps, c->d_ldb, c->d_fofs, c->d_fsel, c->d_coef};
  for (void* q : ptrs) dev_free(c, q);
  for (auto& pl : c->tc2plans) { dev_free(c, pl.second.d_ofs); dev_free(c, pl.second.d_items); }
  cudaStreamSynchronize(c->st);   // the frees are stream-ordered: complete them before returning
  host_pinned_free(c->h_scal);
  for (auto& pe : c->ev_pending) { cudaEventDestroy(pe.second.first); cudaEventDestroy(pe.second.second); }
  for (auto ev : c->ev_pool) cudaEventDestroy(ev);
  delete c;
  return DDM_OK;
}

extern "C" const char* ddm_last_error(const ddm_ctx* c) { return c ? c->err.c_str() : g_setup_err.c_str(); }

extern "C" ddm_status ddm_set_medium(ddm_ctx* c, double omega, const double* c_dev) {
  if (!c) return fail(nullptr, DDM_E_INVAL, "null context");
  if (!(omega > 0) || !c_dev) return fail(c, DDM_E_INVAL, "omega must be > 0 and c_dev non-null");
  c->omega = omega;
  CK(launch_k2(c, c_dev));
  CK(launch_coefs(c));
  c->factored = false;
  return DDM_OK;
}

extern "C" ddm_status ddm_set_medium_host(ddm_ctx* c, double omega, const double* c_host) {
  if (!c) return fail(nullptr, DDM_E_INVAL, "null context");
  if (!c_host) return fail(c, DDM_E_INVAL, "c_host is null");
  if (!c->d_chost) CK(dev_alloc(c, (void**)&c->d_chost, sizeof(double) * c->g.nglob));
  CK(cudaMemcpyAsync(c->d_chost, c_host, sizeof(double) * c->g.nglob, cudaMemcpyHostToDevice, c->st));
  return ddm_set_medium(c, omega, c->d_chost);
}

extern "C" ddm_status ddm_kernel_launches(ddm_ctx* c, int64_t* count, int reset) {
  if (!c) return DDM_E_INVAL;
  if (count) *count = c->nlaunch;
  if (reset) c->nlaunch = 0;
  return DDM_OK;
}

// =====================================================================================
// factorisation
// =====================================================================================
extern "C" ddm_status ddm_factor(ddm_ctx* c) {
  if (!c) return fail(nullptr, DDM_E_INVAL, "null context");
  Geom& g = c->g;
  unsigned long long* d_hash = c->d_hash;
  CK(launch_sub_hash(c, d_hash));
  std::vector<unsigned long long> hash(g.nsub);
  CK(cudaMemcpyAsync(hash.data(), d_hash, sizeof(unsigned long long) * g.nsub, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  // group by (own widths, hash); confirm every member against its group's representative
  std::map<std::tuple<int, int, int, unsigned long long>, int> groups;
  std::vector<int> rep_of(g.nsub);
  for (int s = 0; s < g.nsub; ++s) {
    auto key = std::make_tuple(c->subs[s].nown[0], c->subs[s].nown[1], c->subs[s].nown[2], hash[s]);
    auto it = groups.find(key);
    if (it == groups.end()) { groups[key] = s; rep_of[s] = s; }
    else rep_of[s] = it->second;
  }
  std::vector<int> pairs;
  for (int s = 0; s < g.nsub; ++s) if (rep_of[s] != s) { pairs.push_back(s); pairs.push_back(rep_of[s]); }
  int npairs = (int)pairs.size() / 2;
  if (npairs) {
    int *d_pairs = c->d_pairs, *d_mis = c->d_mis;
    CK(cudaMemcpyAsync(d_pairs, pairs.data(), sizeof(int) * pairs.size(), cudaMemcpyHostToDevice, c->st));
    CK(launch_sub_compare(c, d_pairs, npairs, d_mis));
    std::vector<int> mis(npairs);
    CK(cudaMemcpyAsync(mis.data(), d_mis, sizeof(int) * npairs, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    for (int q = 0; q < npairs; ++q) if (mis[q]) rep_of[pairs[2 * q]] = pairs[2 * q];   // hash collision: own factor
  }
  // factor ids and storage
  std::vector<int> fid_of_rep(g.nsub, -1), reps;
  c->fac_b.clear(); c->fac_m.clear(); c->fac_ldb.clear(); c->fac_ofs.clear();
  long long ofs = 0;
  for (int s = 0; s < g.nsub; ++s) {
    int r = rep_of[s];
    if (fid_of_rep[r] < 0) {
      fid_of_rep[r] = (int)reps.size();
      reps.push_back(r);
      // blocks: x-lines in 2D, z-planes in 3D
      int b = c->dim == 2 ? c->subs[r].ext[0] : c->subs[r].ext[0] * c->subs[r].ext[1];
      int m = c->dim == 2 ? c->subs[r].ext[1] : c->subs[r].ext[2];
      int ldb = (b + 3) & ~3;
      c->fac_b.push_back(b); c->fac_m.push_back(m); c->fac_ldb.push_back(ldb); c->fac_ofs.push_back(ofs);
      ofs += (long long)m * b * ldb;
    }
    int f = fid_of_rep[r];
    c->subs[s].fid = f;
    c->subs[s].fofs = c->fac_ofs[f];
    c->subs[s].pad = c->fac_ldb[f];
  }
  c->nfac = (int)reps.size();
  const bool nd = c->local_solver == DDM_LOCAL_ND;
  if (nd) CK(nd_layout(c, reps, &ofs));   // the multifrontal blocks replace the block layout
  c->fac_elems = ofs;
  // the nested-dissection blocks are FP64 in both precisions
  const size_t gbytes = (size_t)ofs * (nd ? sizeof(z64) : local_elem(c));
  if (gbytes > c->G_cap) {
    dev_free(c, c->d_G);
    c->d_G = nullptr;
    c->G_cap = 0;
    c->drop_graphs();
    CK(dev_alloc(c, &c->d_G, gbytes));
    c->G_cap = gbytes;
  }
  CK(cudaMemcpyAsync(c->d_subs, c->subs.data(), sizeof(SubDesc) * g.nsub, cudaMemcpyHostToDevice, c->st));
  int *d_reps = c->d_reps, *d_ldb = c->d_ldb;
  long long* d_fofs = c->d_fofs;
  CK(cudaMemcpyAsync(d_reps, reps.data(), sizeof(int) * c->nfac, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(d_ldb, c->fac_ldb.data(), sizeof(int) * c->nfac, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(d_fofs, c->fac_ofs.data(), sizeof(long long) * c->nfac, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0); cudaEventCreate(&e1);
  cudaEventRecord(e0, c->st);
  {
    TScope ts(c, T_FACTOR);
    if (nd) {
      CK(nd_factor(c, reps));
    } else if (!c->blockpath) {
      CK(launch_factor_all(c, d_reps, d_fofs, d_ldb));
      if (c->prec == DDM_MIXED && c->p.max_rhs >= 16) CK(tc2d_pack_factors(c));
    }
    else {
      CK(launch_factor3d(c, reps));   // ends with a stream synchronisation
      if (c->piv_tau > 0) {
        // pivots were searched among each panel's diagonal rows: redo the factorisation with the
        // search over all rows if a threshold check failed (or a block had no usable pivot)
        int h = 0;
        CK(cudaMemcpyAsync(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        if (h & (ERRBIT_WEAKPIV | ERRBIT_SINGULAR)) {
          CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st));
          c->piv_full = true;
          const cudaError_t e = launch_factor3d(c, reps);
          c->piv_full = false;
          CK(e);
          ++c->piv_redone;
        }
      }
      if (c->prec == DDM_MIXED) CK(tc3d_pack_factors(c));
    }
  }
  cudaEventRecord(e1, c->st);
  CK(cudaStreamSynchronize(c->st));
  cudaEventElapsedTime(&c->factor_ms, e0, e1);
  cudaEventDestroy(e0); cudaEventDestroy(e1);
  CKS(check_err_word(c));
  c->factored = true;
  return DDM_OK;
}

// The batched local solves of Algorithm 3.1 with the context's local solver.
static cudaError_t local_solve(ddm_ctx* c, const void* src, void* out, void* accum, int nrhs) {
  if (c->local_solver == DDM_LOCAL_ND) return nd_solve(c, src, out, accum, nrhs);
  return launch_local_solve(c, src, out, accum, nrhs);
}

// =====================================================================================
// DDM steps (Algorithm 3.1) and the preconditioner
// =====================================================================================
// Runs K steps from the global J-scaled right-hand side b (nrhs vectors).  w_out (global,
// may be null) receives sum_R beta_0 U_R; res_host[s-1] (may be null, nrhs = 1) the norm of
// the own-region residual after step s; u_last (may be null) the last step's local solution.
static ddm_status run_steps(ddm_ctx* c, const z64* b, int nrhs, int K, z64* w_out, double* res_host, void* u_last,
                            double stop_abs = -1.0, int* steps_done = nullptr) {
  const int L = ring_slots(c);
  {
    TScope ts(c, T_ASSEMBLE);
    CK(launch_restrict(c, b, c->d_src, c->d_U, nrhs));
  }
  int s = 1;
  for (; s <= K; ++s) {
    {
      TScope ts(c, T_SOLVE);
      CK(local_solve(c, c->d_src, c->d_ring[s % L], c->d_U, nrhs));
    }
    const bool want_res = res_host != nullptr;
    if (s < K || want_res) {
      int nblk = 0;
      {
        TScope ts(c, T_TRANSFER);
        // after step 1 the next source lives on the strip nodes only: clear the step-1 source once
        if (s == 1) CK(cudaMemsetAsync(c->d_src, 0, local_elem(c) * c->g.ltotal * nrhs, c->st));
        CK(launch_transfer_n(c, s, c->d_src, c->d_part, nrhs, want_res ? 1 : 0, &nblk));
      }
      if (want_res) {
        // one value: total over all blocks of all receivers
        CK(launch_sum_partials(c, c->d_part, nblk * c->g.nsub, 1, c->d_scal));
        CK(cudaMemcpyAsync(c->h_scal, c->d_scal, sizeof(double), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        res_host[s - 1] = std::sqrt(c->h_scal[0]);
        if (stop_abs >= 0 && res_host[s - 1] <= stop_abs) { ++s; break; }
      }
    }
  }
  if (steps_done) *steps_done = s - 1;
  if (u_last) {
    const int last = s - 1;
    CK(cudaMemcpyAsync(u_last, c->d_ring[last % L], local_elem(c) * c->g.ltotal * nrhs, cudaMemcpyDeviceToDevice, c->st));
  }
  if (w_out) {
    TScope ts(c, T_ASSEMBLE);
    CK(launch_assemble(c, c->d_U, w_out, nrhs));
  }
  return DDM_OK;
}

// M_K through a CUDA graph: the kernels of one application (restriction, K local solves,
// K-1 transfers, assembly) are captured once per (nrhs, K) on a dedicated stream, reading and
// writing fixed staging vectors, and replayed; the staging copies and the replay are ordered
// after and before the context's stream with events.  The first call runs the application once
// outside capture so that the local solve's autotuner has settled (it allocates and times).
static ddm_status apply_graphed(ddm_ctx* c, const z64* src, z64* dst, int nrhs, int K) {
  const long long n = c->g.nglob;
  if (!c->gstream) {
    CK(cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->gev[0], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->gev[1], cudaEventDisableTiming));
    CK(dev_alloc(c, (void**)&c->d_gin, sizeof(z64) * n * c->p.max_rhs));
    CK(dev_alloc(c, (void**)&c->d_gout, sizeof(z64) * n * c->p.max_rhs));
  }
  ddm_ctx::GraphRec* rec = nullptr;
  for (auto& g : c->graphs) if (g.nrhs == nrhs && g.K == K) rec = &g;
  CK(cudaMemcpyAsync(c->d_gin, src, sizeof(z64) * n * nrhs, cudaMemcpyDeviceToDevice, c->st));
  if (!rec) {
    CKS(run_steps(c, c->d_gin, nrhs, K, c->d_gout, nullptr, nullptr));   // settle the autotuner
    CK(cudaStreamSynchronize(c->st));
    const bool timing = c->timing;
    c->timing = false;
    cudaStream_t keep = c->st;
    c->st = c->gstream;
    const long long n0 = c->nlaunch;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal);
    ddm_status st = DDM_OK;
    if (e == cudaSuccess) st = run_steps(c, c->d_gin, nrhs, K, c->d_gout, nullptr, nullptr);
    cudaError_t e2 = cudaStreamEndCapture(c->gstream, &graph);
    c->st = keep;
    c->timing = timing;
    if (e != cudaSuccess || e2 != cudaSuccess || st != DDM_OK)
      return fail(c, DDM_E_CUDA, std::string("graph capture failed: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    cudaGraphExec_t exec = nullptr;
    CK(cudaGraphInstantiate(&exec, graph, 0));
    cudaGraphDestroy(graph);
    c->graphs.push_back({nrhs, K, exec, c->nlaunch - n0});
    rec = &c->graphs.back();
  }
  CK(cudaEventRecord(c->gev[0], c->st));
  CK(cudaStreamWaitEvent(c->gstream, c->gev[0], 0));
  cudaError_t le;
  {
    cudaStream_t keep = c->st;
    c->st = c->gstream;   // the timing scope records on the stream the graph runs on
    {
      TScope ts(c, T_GRAPH);
      le = cudaGraphLaunch(rec->exec, c->gstream);
    }
    c->st = keep;
  }
  CK(le);
  c->nlaunch += rec->kernels;
  CK(cudaEventRecord(c->gev[1], c->gstream));
  CK(cudaStreamWaitEvent(c->st, c->gev[1], 0));
  CK(cudaMemcpyAsync(dst, c->d_gout, sizeof(z64) * n * nrhs, cudaMemcpyDeviceToDevice, c->st));
  return DDM_OK;
}

extern "C" ddm_status ddm_apply(ddm_ctx* c, int K, const void* src_dev, void* dst_dev, int nrhs) {
  if (!c) return fail(nullptr, DDM_E_INVAL, "null context");
  if (K < 1 || nrhs < 1 || nrhs > c->p.max_rhs || !src_dev || !dst_dev) return fail(c, DDM_E_INVAL, "bad K / nrhs / pointer");
  if (!c->factored) return fail(c, DDM_E_STATE, "ddm_factor must run before ddm_apply");
  if (c->use_graph) CKS(apply_graphed(c, (const z64*)src_dev, (z64*)dst_dev, nrhs, K));
  else CKS(run_steps(c, (const z64*)src_dev, nrhs, K, (z64*)dst_dev, nullptr, nullptr));
  CK(cudaGetLastError());
  return DDM_OK;
}

extern "C" ddm_status ddm_steps(ddm_ctx* c, const void* b_dev, int nsteps, void* w_dev, void* u_last_dev, double* res_host) {
  if (!c) return fail(nullptr, DDM_E_INVAL, "null context");
  if (nsteps < 1 || !b_dev) return fail(c, DDM_E_INVAL, "bad nsteps / pointer");
  if (!c->factored) return fail(c, DDM_E_STATE, "ddm_factor must run first");
  CKS(run_steps(c, (const z64*)b_dev, 1, nsteps, (z64*)w_dev, res_host, u_last_dev));
  CK(cudaStreamSynchronize(c->st));
  return check_err_word(c);
}

extern "C" ddm_status ddm_local_solve(ddm_ctx* c, const void* src_dev, void* u_dev, int nrhs) {
  if (!c) return fail(nullptr, DDM_E_INVAL, "null context");
  if (nrhs < 1 || nrhs > c->p.max_rhs) return fail(c, DDM_E_INVAL, "bad nrhs");
  if (!c->factored) return fail(c, DDM_E_STATE, "ddm_factor must run first");
  {
    TScope ts(c, T_SOLVE);
    CK(local_solve(c, src_dev, u_dev, nullptr, nrhs));
  }
  CK(cudaStreamSynchronize(c->st));
  return check_err_word(c);
}

// =====================================================================================
// global operator, residual, right-hand side
// =====================================================================================
extern "C" ddm_status ddm_rhs(ddm_ctx* c, const void* f_dev, void* b_dev, int nrhs) {
  if (!c) return fail(nullptr, DDM_E_INVAL, "null context");
  if (nrhs < 1) return fail(c, DDM_E_INVAL, "bad nrhs");
  CK(launch_rhs(c, (const z64*)f_dev, (z64*)b_dev, nrhs));
  return DDM_OK;
}

extern "C" ddm_status ddm_global_apply(ddm_ctx* c, const void* x_dev, void* y_dev, int nrhs) {
  if (!c) return fail(nullptr, DDM_E_INVAL, "null context");
  if (nrhs < 1) return fail(c, DDM_E_INVAL, "bad nrhs");
  TScope ts(c, T_GLOBAL);
  CK(launch_global_apply(c, (const z64*)x_dev, (z64*)y_dev, nullptr, nrhs));
  return DDM_OK;
}

// norms2_dev[i] = ||x_i||^2 for nvec vectors of length nglob (device doubles)
static ddm_status norms2(ddm_ctx* c, const z64* x, int nvec, double* norms2_dev) {
  int nblk = 0;
  CK(launch_norm2_partial(c, x, c->g.nglob, nvec, c->d_part, &nblk));
  CK(launch_sum_partials(c, c->d_part, nblk, nvec, norms2_dev));
  return DDM_OK;
}

extern "C" ddm_status ddm_residual(ddm_ctx* c, const void* b_dev, const void* x_dev, void* r_dev, int nrhs, double* norms_host) {
  if (!c) return fail(nullptr, DDM_E_INVAL, "null context");
  if (nrhs < 1 || nrhs > 16) return fail(c, DDM_E_INVAL, "nrhs must be in [1, 16]");
  {
    TScope ts(c, T_GLOBAL);
    CK(launch_global_apply(c, (const z64*)x_dev, (z64*)r_dev, (const z64*)b_dev, nrhs));
  }
  if (norms_host) {
    CKS(norms2(c, (const z64*)r_dev, nrhs, c->d_scal));
    CKS(norms2(c, (const z64*)b_dev, nrhs, c->d_scal + 16));
    CK(cudaMemcpyAsync(c->h_scal, c->d_scal, sizeof(double) * 32, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    for (int i = 0; i < nrhs; ++i) {
      norms_host[2 * i] = std::sqrt(c->h_scal[i]);
      norms_host[2 * i + 1] = std::sqrt(c->h_scal[16 + i]);
    }
  }
  return DDM_OK;
}

// =====================================================================================
// solvers
// =====================================================================================
static double host_norm(ddm_ctx* c, const z64* x, ddm_status* st) {
  *st = norms2(c, x, 1, c->d_scal + 32);
  if (*st != DDM_OK) return 0;
  cudaMemcpyAsync(c->h_scal + 32, c->d_scal + 32, sizeof(double), cudaMemcpyDeviceToHost, c->st);
  cudaError_t e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) { *st = fail(c, DDM_E_CUDA, cudaGetErrorString(e)); return 0; }
  return std::sqrt(c->h_scal[32]);
}

static ddm_status ensure_krylov(ddm_ctx* c, int m, int nb) {
  if (c->kry_m >= m && c->kry_nb >= nb) return DDM_OK;
  void* old[] = {c->d_V, c->d_Z, c->d_H, c->d_gs, c->d_bscal, c->d_jr, c->d_coef};
  for (void* q : old) dev_free(c, q);
  host_pinned_free(c->h_bscal);
  c->d_V = c->d_Z = c->d_H = c->d_gs = nullptr;
  c->d_bscal = nullptr; c->h_bscal = nullptr; c->d_jr = nullptr; c->d_coef = nullptr;
  c->kry_m = c->kry_nb = 0;
  const long long n = c->g.nglob;
  CK(dev_alloc(c, (void**)&c->d_V, sizeof(z64) * n * (m + 1) * nb));
  CK(dev_alloc(c, (void**)&c->d_Z, sizeof(z64) * n * m * nb));
  CK(dev_alloc(c, (void**)&c->d_H, sizeof(z64) * (m + 1) * m * nb));
  CK(dev_alloc(c, (void**)&c->d_gs, sizeof(z64) * (5 * m + 4) * nb));
  CK(dev_alloc(c, (void**)&c->d_bscal, sizeof(double) * 4 * nb));
  CK(host_pinned_alloc((void**)&c->h_bscal, sizeof(double) * 4 * nb));
  CK(dev_alloc(c, (void**)&c->d_jr, sizeof(int) * nb));
  CK(dev_alloc(c, (void**)&c->d_coef, sizeof(z64) * (m + 1) * nb));
  c->kry_m = m;
  c->kry_nb = nb;
  return DDM_OK;
}

// Flexible GMRES(m) for A x_r = b_r, r < nb, right-preconditioned by M_K (Section 4.2.2).
// The nb recurrences advance together: one nb-wide preconditioner application (the local
// solves stream each factor block once for up to 8 right-hand sides) and one nb-wide global
// operator per iteration; Arnoldi, Givens and the least-squares update are per right-hand side.
// A right-hand side that has converged keeps its iterate; later cycles run it on a zero basis.
static ddm_status fgmres_batch(ddm_ctx* c, const z64* b, z64* x, int nb, double tol, int max_it, int K, int m,
                               ddm_info* info) {
  const long long n = c->g.nglob;
  CKS(ensure_krylov(c, m, nb));
  double* d_nrm2 = c->d_bscal;         // nb: squared norms
  double* d_est = c->d_bscal + nb;     // nb: residual estimates
  double* d_sc = c->d_bscal + 2 * nb;  // nb: scale factors
  double* h = c->h_bscal;
  z64* V = c->d_V;
  z64* Z = c->d_Z;
  z64* H = c->d_H;
  z64* gs = c->d_gs;
  const int GSZ = 5 * m + 4;
  // coefficient scratch for the Gram-Schmidt passes: nb x (m+1), after the gs blocks' y part
  z64* coef = c->d_coef;
  auto cleanup = [&]() {};
  auto batch_norms = [&](const z64* v) -> ddm_status {
    int nblk = 0;
    CK(launch_norm2_partial(c, v, n, nb, c->d_part, &nblk));
    CK(launch_sum_partials(c, c->d_part, nblk, nb, d_nrm2));
    CK(cudaMemcpyAsync(h, d_nrm2, sizeof(double) * nb, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return DDM_OK;
  };
  std::vector<double> bnorm(nb), est(nb, 1.0);
  std::vector<char> conv(nb, 0);
  { ddm_status st = batch_norms(b); if (st != DDM_OK) { cleanup(); return st; } }
  for (int r = 0; r < nb; ++r) { bnorm[r] = std::sqrt(h[r]); if (bnorm[r] == 0.0) { conv[r] = 1; est[r] = 0; } }
  CK(cudaMemsetAsync(x, 0, sizeof(z64) * n * nb, c->st));
  int it = 0, steps = 0;
  auto all_done = [&]() { for (int r = 0; r < nb; ++r) if (!conv[r]) return false; return true; };
  while (it < max_it && !all_done()) {
    {
      TScope ts(c, T_GLOBAL);
      CK(launch_global_apply(c, x, c->d_gr, b, nb));
    }
    { ddm_status st = batch_norms(c->d_gr); if (st != DDM_OK) { cleanup(); return st; } }
    std::vector<double> beta(nb), scale(nb);
    for (int r = 0; r < nb; ++r) {
      beta[r] = std::sqrt(h[r]);
      if (!conv[r]) { est[r] = beta[r] / bnorm[r]; if (est[r] <= tol) conv[r] = 1; }
      scale[r] = (!conv[r] && beta[r] > 0) ? 1.0 / beta[r] : 0.0;
    }
    if (all_done()) break;
    CK(cudaMemcpyAsync(d_sc, scale.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, c->st));
    CK(launch_scale_vec_b(c, nb, c->d_gr, d_sc, V, n));
    CK(cudaMemsetAsync(gs, 0, sizeof(z64) * GSZ * nb, c->st));
    CK(cudaMemsetAsync(H, 0, sizeof(z64) * (m + 1) * m * nb, c->st));
    std::vector<z64> g0(nb);
    for (int r = 0; r < nb; ++r) g0[r] = mk<double>(conv[r] ? 0.0 : beta[r], 0.0);
    for (int r = 0; r < nb; ++r)
      CK(cudaMemcpyAsync(gs + (long long)r * GSZ + 2 * m, &g0[r], sizeof(z64), cudaMemcpyHostToDevice, c->st));
    std::vector<char> active(nb);
    std::vector<int> jr(nb, 0);
    for (int r = 0; r < nb; ++r) active[r] = !conv[r];
    int j = 0;
    for (; j < m && it < max_it; ++j) {
      z64* vj = V + (long long)j * nb * n;
      z64* zj = Z + (long long)j * nb * n;
      z64* w = V + (long long)(j + 1) * nb * n;
      {
        ddm_status st = c->use_graph ? apply_graphed(c, vj, zj, nb, K) : run_steps(c, vj, nb, K, zj, nullptr, nullptr);
        if (st != DDM_OK) { cleanup(); return st; }
      }
      steps += K;
      {
        TScope ts(c, T_GLOBAL);
        CK(launch_global_apply(c, zj, w, nullptr, nb));
      }
      {
        TScope ts(c, T_KRYLOV);
        for (int pass = 0; pass < 2; ++pass) {   // classical Gram-Schmidt, twice
          int nblk = 0;
          CK(launch_dots_b(c, V, nb, j + 1, w, n, c->d_part, &nblk));
          CK(launch_arnoldi_coef_b(c, c->d_part, nblk, j + 1, nb, H, j, m, coef, pass == 0));
          CK(launch_sub_axpy_b(c, V, nb, j + 1, coef, m, w, n));
        }
        int nblk = 0;
        CK(launch_norm2_partial(c, w, n, nb, c->d_part, &nblk));
        CK(launch_sum_partials(c, c->d_part, nblk, nb, d_nrm2));
        CK(launch_givens_b(c, nb, j, m, d_nrm2, H, gs, d_est));
        CK(launch_scale_b(c, nb, w, gs, m, n));
      }
      CK(cudaMemcpyAsync(h + nb, d_est, sizeof(double) * nb, cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      ++it;
      bool pending = false;
      for (int r = 0; r < nb; ++r) {
        if (!active[r] || jr[r] > 0) continue;
        est[r] = h[nb + r] / bnorm[r];
        if (!(est[r] == est[r])) { cleanup(); return fail(c, DDM_E_NOCONV, "non-finite residual estimate in FGMRES"); }
        if (est[r] <= tol) { conv[r] = 1; jr[r] = j + 1; }
        else pending = true;
      }
      if (!pending) { ++j; break; }
    }
    for (int r = 0; r < nb; ++r) if (active[r] && jr[r] == 0) jr[r] = j;
    CK(cudaMemcpyAsync(c->d_jr, jr.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, c->st));
    {
      TScope ts(c, T_KRYLOV);
      CK(launch_lsq_update_b(c, nb, c->d_jr, m, H, gs, Z, x, n));
    }
    CK(cudaStreamSynchronize(c->st));   // jr (host vector) must outlive the copy above
  }
  cleanup();
  double worst = 0;
  for (int r = 0; r < nb; ++r) worst = std::max(worst, est[r]);
  if (info) { info->iters += it; info->ddm_steps += steps; info->rel_residual_est = worst; }
  return DDM_OK;
}

// Algorithm 3.1 continued as an iteration (Section 4.2.1).  FP64: steps until the own-region
// residual (from the transfers) <= tol ||b||.  Mixed: iterative refinement x += M(r) with the
// inner complex64 iteration run to a relative 1e-4 (or stagnation), r = b - A x in FP64.
static ddm_status stepping_one(ddm_ctx* c, const z64* b, z64* x, double tol, int max_steps, ddm_info* info) {
  const long long n = c->g.nglob;
  ddm_status st;
  double bnorm = host_norm(c, b, &st);
  if (st != DDM_OK) return st;
  CK(cudaMemsetAsync(x, 0, sizeof(z64) * n, c->st));
  if (bnorm == 0.0) return DDM_OK;
  std::vector<double> hist(max_steps + 1);
  int total = 0;
  const bool mixed = c->prec == DDM_MIXED;
  const z64* rhs = b;
  double rnorm = bnorm;
  double est = 1.0;
  for (int outer = 0; outer < 64 && total < max_steps; ++outer) {
    double inner_tol = mixed ? std::max(tol * bnorm / rnorm * 0.5, 1e-4) : tol * bnorm / rnorm;
    int done = 0;
    CKS(run_steps(c, rhs, 1, max_steps - total, c->d_gw, hist.data(), nullptr, inner_tol * rnorm, &done));
    total += done;
    est = hist[std::max(done - 1, 0)] / bnorm;
    if (!mixed) {
      CK(cudaMemcpyAsync(x, c->d_gw, sizeof(z64) * n, cudaMemcpyDeviceToDevice, c->st));
      break;
    }
    // x += w; r = b - A x (FP64)
    {
      TScope ts(c, T_KRYLOV);
      CK(launch_axpy(c, 1.0, c->d_gw, x, n));
    }
    {
      TScope ts(c, T_GLOBAL);
      CK(launch_global_apply(c, x, c->d_gr, b, 1));
    }
    rnorm = host_norm(c, c->d_gr, &st);
    if (st != DDM_OK) return st;
    est = rnorm / bnorm;
    if (est <= tol) break;
    rhs = c->d_gr;
  }
  if (info) { info->iters += total; info->ddm_steps += total; info->rel_residual_est = est; }
  return DDM_OK;
}

static ddm_status solve_impl(ddm_ctx* c, const void* f_dev, void* u_dev, int nrhs, double tol, int max_it, int mode,
                             int K, int restart, ddm_info* info) {
  if (!c) return fail(nullptr, DDM_E_INVAL, "null context");
  if (nrhs < 1 || nrhs > c->p.max_rhs || !f_dev || !u_dev) return fail(c, DDM_E_INVAL, "bad nrhs / pointer");
  if (!(tol > 0) || max_it < 1) return fail(c, DDM_E_INVAL, "tol must be > 0 and max_it >= 1");
  if (mode != DDM_FGMRES && mode != DDM_STEPPING) return fail(c, DDM_E_INVAL, "bad mode");
  if (mode == DDM_FGMRES && (K < 1 || restart < 1 || restart > 120)) return fail(c, DDM_E_INVAL, "K >= 1 and restart in [1, 120]");
  if (!c->factored) return fail(c, DDM_E_STATE, "ddm_factor must run before ddm_solve");
  auto t0 = std::chrono::steady_clock::now();
  ddm_info loc;
  memset(&loc, 0, sizeof(loc));
  const long long n = c->g.nglob;
  CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st));
  CK(launch_rhs(c, (const z64*)f_dev, c->d_gb, nrhs));
  double worst = 0.0;
  bool all_conv = true;
  for (int r = 0; r < nrhs; ++r) {
    const z64* b = c->d_gb + (long long)r * n;
    z64* x = (z64*)u_dev + (long long)r * n;
    if (mode == DDM_FGMRES) {
      if (r == 0) CKS(fgmres_batch(c, c->d_gb, (z64*)u_dev, nrhs, tol, max_it, K, restart, &loc));
    } else {
      CKS(stepping_one(c, b, x, tol, max_it, &loc));
    }
    double nr[2];
    CKS(ddm_residual(c, b, x, c->d_gr, 1, nr));
    double rel = nr[1] > 0 ? nr[0] / nr[1] : 0.0;
    worst = std::max(worst, rel);
    if (!(rel <= tol * 1.0001)) all_conv = false;
  }
  CK(cudaStreamSynchronize(c->st));
  auto t1 = std::chrono::steady_clock::now();
  loc.rel_residual = worst;
  loc.converged = all_conv ? 1 : 0;
  loc.n_unique_factors = c->nfac;
  loc.factor_ms = c->factor_ms;
  loc.solve_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  if (info) *info = loc;
  CKS(check_err_word(c));
  if (!all_conv) return fail(c, DDM_E_NOCONV, "tolerance not reached (explicit residual " + std::to_string(worst) + ")");
  return DDM_OK;
}

extern "C" ddm_status ddm_solve(ddm_ctx* c, const void* f_dev, void* u_dev, int nrhs, double tol, int max_it, int mode,
                                int K, int restart, ddm_info* info) {
  return solve_impl(c, f_dev, u_dev, nrhs, tol, max_it, mode, K, restart, info);
}

extern "C" ddm_status ddm_solve_host(ddm_ctx* c, const void* f_host, void* u_host, int nrhs, double tol, int max_it,
                                     int mode, int K, int restart, ddm_info* info) {
  if (!c) return fail(nullptr, DDM_E_INVAL, "null context");
  if (nrhs < 1 || nrhs > c->p.max_rhs || !f_host || !u_host) return fail(c, DDM_E_INVAL, "bad nrhs / pointer");
  const long long n = c->g.nglob;
  if (!c->d_hostbuf) CK(dev_alloc(c, (void**)&c->d_hostbuf, sizeof(z64) * n * c->p.max_rhs * 2));
  z64* f = c->d_hostbuf;
  z64* u = c->d_hostbuf + n * c->p.max_rhs;
  CK(cudaMemcpyAsync(f, f_host, sizeof(z64) * n * nrhs, cudaMemcpyHostToDevice, c->st));
  ddm_status st = solve_impl(c, f, u, nrhs, tol, max_it, mode, K, restart, info);
  CK(cudaMemcpyAsync(u_host, u, sizeof(z64) * n * nrhs, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return st;
}

// =====================================================================================
// introspection
// =====================================================================================
extern "C" ddm_status ddm_local_layout(const ddm_ctx* c, int* n_sub, int64_t* total, int64_t* offsets, int* ext_x,
                                       int* ext_y, int* ext_z) {
  if (!c) return DDM_E_INVAL;
  if (n_sub) *n_sub = c->g.nsub;
  if (total) *total = c->g.ltotal;
  for (int s = 0; s < c->g.nsub; ++s) {
    if (offsets) offsets[s] = c->subs[s].vofs;
    if (ext_x) ext_x[s] = c->subs[s].ext[0];
    if (ext_y) ext_y[s] = c->subs[s].ext[1];
    if (ext_z) ext_z[s] = c->subs[s].ext[2];
  }
  return DDM_OK;
}

extern "C" ddm_status ddm_timing(ddm_ctx* c, int enable, int reset, double* out_ms, int64_t* out_launches) {
  if (!c) return DDM_E_INVAL;
  timing_drain(c);
  if (out_ms) for (int i = 0; i < T_NSLOT; ++i) out_ms[i] = c->t_ms[i];
  if (out_launches) for (int i = 0; i < T_NSLOT; ++i) out_launches[i] = c->t_n[i];
  if (reset) for (int i = 0; i < T_NSLOT; ++i) { c->t_ms[i] = 0; c->t_n[i] = 0; }
  c->timing = enable != 0;
  return DDM_OK;
}

extern "C" ddm_status ddm_set_graph(ddm_ctx* c, int enable) {
  if (!c) return fail(nullptr, DDM_E_INVAL, "null context");
  if (enable && c->blockpath && c->local_solver != DDM_LOCAL_ND)
    return fail(c, DDM_E_INVAL,
                "graph replay of M_K is implemented for 2D partitions: subdomains at most 128 nodes wide, or the "
                "nested-dissection local solver");
  c->use_graph = enable != 0;
  return DDM_OK;
}

extern "C" ddm_status ddm_set_pivoting(ddm_ctx* c, double tau) {
  if (!c) return fail(nullptr, DDM_E_INVAL, "null context");
  if (!(tau >= 0.0) || !(tau <= 1e6)) return fail(c, DDM_E_INVAL, "pivot threshold must be in [0, 1e6]");
  c->piv_tau = tau;
  return DDM_OK;
}

extern "C" ddm_status ddm_pivoting_info(const ddm_ctx* c, double* tau, int64_t* redone) {
  if (!c) return fail(nullptr, DDM_E_INVAL, "null context");
  if (tau) *tau = c->piv_tau;
  if (redone) *redone = c->piv_redone;
  return DDM_OK;
}

extern "C" ddm_status ddm_set_local_solver(ddm_ctx* c, int solver, int leaf) {
  if (!c) return fail(nullptr, DDM_E_INVAL, "null context");
  if (solver != DDM_LOCAL_BLOCK && solver != DDM_LOCAL_ND)
    return fail(c, DDM_E_INVAL, "local solver must be DDM_LOCAL_BLOCK or DDM_LOCAL_ND");
  if (leaf < 0 || leaf > 4096) return fail(c, DDM_E_INVAL, "leaf size must be 0 (default) .. 4096 nodes");
  if (solver == DDM_LOCAL_ND && c->dim != 2)
    return fail(c, DDM_E_INVAL, "the nested-dissection local solver is built for 2D partitions");
  if (solver == DDM_LOCAL_BLOCK && c->use_graph && c->blockpath)
    return fail(c, DDM_E_INVAL, "the block solver of these subdomains cannot replay graphs: turn the graph off first");
  const int lf = leaf == 0 ? DDM_ND_LEAF_DEFAULT : leaf;
  if (solver != c->local_solver || lf != c->nd_leaf) {
    c->factored = false;
    c->drop_graphs();
  }
  c->local_solver = solver;
  c->nd_leaf = lf;
  return DDM_OK;
}

extern "C" ddm_status ddm_set_tensor_cores(ddm_ctx* c, int enable) {
  if (!c) return fail(nullptr, DDM_E_INVAL, "null context");
  if (c->use_tc != (enable != 0)) c->drop_graphs();   // captured graphs hold the kernel choice
  c->use_tc = enable != 0;
  return DDM_OK;
}

extern "C" ddm_status ddm_set_rhs_per_cta(ddm_ctx* c, int nr) {
  if (!c) return fail(nullptr, DDM_E_INVAL, "null context");
  if (nr != 0 && nr != 1 && nr != 2 && nr != 4 && nr != 8 && nr != 64)
    return fail(c, DDM_E_INVAL, "right-hand sides per CTA must be 0 (autotuned), 1, 2, 4, 8 or 64");
  if (nr == 8 && c->prec != DDM_MIXED) return fail(c, DDM_E_INVAL, "8 right-hand sides per CTA need DDM_MIXED");
  if (nr == 64 && (c->dim != 2 || c->prec != DDM_MIXED || !c->d_gtc2 || !tc2d_supported(c, nr)))
    return fail(c, DDM_E_INVAL,
                "64 right-hand sides per CTA run on the tensor cores: 2D, DDM_MIXED, max_rhs >= 16, factored, "
                "blocks of at most 128 rows whose operand and two ring stages fit in shared memory");
  if (c->forced_nr != nr) c->drop_graphs();
  c->forced_nr = nr;
  return DDM_OK;
}

extern "C" ddm_status ddm_workspace_bytes(const ddm_params* p, int restart, int64_t* bytes) {
  if (!p || !bytes) return fail(nullptr, DDM_E_INVAL, "null argument");
  if ((p->dim != 2 && p->dim != 3) || p->overlap < 1 || p->pml < 1 || p->max_rhs < 1 || restart < 0)
    return fail(nullptr, DDM_E_INVAL, "bad parameters");
  const int d = p->dim, e = p->overlap + p->pml;
  const long long el = p->precision == DDM_MIXED ? 8 : 16;
  long long nglob = 1, ltotal = 1, nsub = 1, fac = 0, tab = 0;
  std::vector<std::vector<long long>> widths(3);
  for (int a = 0; a < d; ++a) {
    if (p->n[a] < 1 || p->parts[a] < 1) return fail(nullptr, DDM_E_INVAL, "bad n / parts");
    nglob *= p->n[a] + 2 * e;
    nsub *= p->parts[a];
    for (int i = 0; i < p->parts[a]; ++i) {
      long long lo = p->cuts[a] ? p->cuts[a][i] : (p->n[a] * i) / p->parts[a];
      long long hi = p->cuts[a] ? p->cuts[a][i + 1] : (p->n[a] * (i + 1)) / p->parts[a];
      widths[a].push_back(hi - lo + 2 * e);
      tab += 2 * (hi - lo + 2 * e) + 1;
    }
    tab += 2 * (p->n[a] + 2 * e) + 1;
  }
  // local length and factor storage (every subdomain distinct: the upper bound)
  long long lsum = 0, tcfac = 0, tcy = 0;
  bool anywide = false;   // a 2D partition with x-lines wider than 128 runs on the block path
  if (d == 2) for (long long wx : widths[0]) anywide = anywide || wx > (p->precision == DDM_MIXED ? 128 : 96);
  std::vector<long long> s1 = widths[0], s2 = d > 1 ? widths[1] : std::vector<long long>{1},
                         s3 = d > 2 ? widths[2] : std::vector<long long>{1};
  for (long long wz : s3)
    for (long long wy : s2)
      for (long long wx : s1) {
        lsum += wx * wy * wz;
        const long long b = d == 2 ? wx : wx * wy, m = d == 2 ? wy : wz, ldb = (b + 3) & ~3LL;
        fac += m * b * ldb;
        const bool block = d == 3 || anywide;
        if (!block && p->precision == DDM_MIXED && p->max_rhs >= 16) tcfac += 4 * tc2d_packed_floats((int)b, (int)m);
        if (block && p->precision == DDM_MIXED) {
          tcfac += 4 * tc3d_packed_floats((int)b, (int)m);
          tcy = std::max(tcy, 4 * tc3d_packed_floats((int)b, 1) / std::max(1LL, (b + 127) / 128));
        }
      }
  ltotal = lsum;
  const long long R = p->max_rhs;
  long long total = 0;
  total += 8 * nglob;                           // k^2
  total += el * ltotal * (2 * d + 1);           // local operator planes
  total += 16 * nglob * (2 * d + 1);            // global operator planes
  total += 16 * tab + 8 * ltotal;               // alpha tables, strip-node lists (upper bound)
  total += el * ltotal * R * (3 + d);           // source, U and the ring of d step solutions
  total += 16 * nglob * R * 3;                  // global work vectors
  total += 8 * std::max<long long>(R * nsub * ((lsum / std::max(nsub, 1LL) + 127) / 128 + 1), R * 304LL * 2 * 122);
  total += el * fac;                            // factors
  total += tcfac + tcy * ((nsub * R + 127) / 128);   // 3D tensor-core packs (factors, one operand)
  if (restart > 0) total += 16 * nglob * R * (2LL * restart + 1);   // FGMRES V and Z
  total += 64LL << 20;                          // descriptors, scalars, rounding
  *bytes = total;
  return DDM_OK;
}

extern "C" ddm_status ddm_autotune_log(const ddm_ctx* c, int cap, int* nrhs, int* nr, float* ms, int* count) {
  if (!c) return DDM_E_INVAL;
  const int n = (int)c->tune_log.size();
  if (count) *count = n;
  for (int i = 0; i < n && i < cap; ++i) {
    if (nrhs) nrhs[i] = c->tune_log[i].nrhs;
    if (nr) nr[i] = c->tune_log[i].nr;
    if (ms) ms[i] = c->tune_log[i].ms;
  }
  return DDM_OK;
}

extern "C" ddm_status ddm_factor_bytes(const ddm_ctx* c, int64_t* per_solve, int64_t* stored) {
  if (!c || !c->factored) return DDM_E_STATE;
  const long long el = (long long)local_elem(c);
  long long ps = 0;
  if (c->local_solver == DDM_LOCAL_ND) {
    ps = nd_read_elems(c) * (long long)sizeof(z64);
  } else if (!c->blockpath) {
    for (auto& s : c->subs) {
      long long b = s.ext[0], m = s.ext[1];
      ps += (2 * m - 1) * b * b * el;
    }
  } else {   // 3D: every factor is streamed once per sweep for all columns that share it
    for (int f = 0; f < c->nfac; ++f) ps += (2LL * c->fac_m[f] - 1) * c->fac_b[f] * (long long)c->fac_b[f] * el;
  }
  if (per_solve) *per_solve = ps;
  if (stored) *stored = c->fac_elems * (c->local_solver == DDM_LOCAL_ND ? (long long)sizeof(z64) : el);
  return DDM_OK;
}

// ------------------------------------------------------------------------------------------
namespace ddm {
cudaError_t allow_dynamic_smem(const void* func, size_t need) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, func)) != cudaSuccess) return e;
  const size_t maxdyn = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
  if (need > maxdyn) return cudaErrorInvalidValue;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({func, dev})) return cudaSuccess;
  if ((e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)maxdyn)) != cudaSuccess)
    return e;
  done.insert({func, dev});
  return cudaSuccess;
}
}  // namespace ddm

// ------------------------------------------------------------------------------------------
// device and pinned host memory of the contexts
namespace ddm {
namespace {
std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools;          // device ordinal -> the library's pool
std::mutex g_pin_mu;
std::multimap<size_t, void*> g_pin_free;       // released pinned blocks by size
std::map<void*, size_t> g_pin_size;            // every pinned block handed out, by address

cudaError_t pool_of_current_device(cudaMemPool_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  auto it = g_pools.find(dev);
  if (it != g_pools.end()) { *out = it->second; return cudaSuccess; }
  cudaMemPoolProps props;
  memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if ((e = cudaMemPoolCreate(&pool, &props)) != cudaSuccess) return e;
  g_pools[dev] = pool;
  *out = pool;
  return cudaSuccess;
}
}  // namespace

cudaError_t dev_alloc(ddm_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  cudaMemPool_t pool = nullptr;
  cudaError_t e = pool_of_current_device(&pool);
  if (e != cudaSuccess) return e;
  return cudaMallocFromPoolAsync(p, bytes ? bytes : 16, pool, c->st);
}

void dev_free(ddm_ctx* c, void* p) {
  if (p) cudaFreeAsync(p, c->st);
}

cudaError_t host_pinned_alloc(void** p, size_t bytes) {
  std::lock_guard<std::mutex> lk(g_pin_mu);
  auto it = g_pin_free.lower_bound(bytes);
  if (it != g_pin_free.end() && it->first <= 2 * bytes + 4096) {
    *p = it->second;
    g_pin_free.erase(it);
    return cudaSuccess;
  }
  cudaError_t e = cudaMallocHost(p, bytes);
  if (e == cudaSuccess) g_pin_size[*p] = bytes;
  return e;
}

void host_pinned_free(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pin_mu);
  auto it = g_pin_size.find(p);
  if (it != g_pin_size.end()) g_pin_free.insert({it->second, p});
}
}  // namespace ddm

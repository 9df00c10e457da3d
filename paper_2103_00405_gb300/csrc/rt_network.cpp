// rt_network.cpp -- validation and packing of reaction networks (host side).
//
// The paper stores the reactant, stoichiometric and species-update matrices as
// sparse COO (Sec. 5) and keeps reactions to at most two reactant molecules so
// the matrices fit in shared memory.  Here the COO input is turned into:
//   * one {s0, s1} reactant descriptor per reaction (h_k of Eq. 2),
//   * the net change v_k as a CSR of {species, delta} (Eq. 5),
//   * the species -> reactions-reading-it CSR: the Gibson-Bruck dependency
//     graph the paper mentions (Sec. 5), which tells which propensities a firing
//     can change,
//   * for networks with at most 64 reactions, a per-reaction dependency bitmask.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "rt_internal.h"

namespace rt {

static thread_local std::string g_err;

int set_error(int code, const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

void clear_error() { g_err.clear(); }

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

cudaError_t raise_smem_limit(const void *kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void *, int>, size_t> current;
  if (bytes <= 48 * 1024) return cudaSuccess;  // the default limit
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t &cur = current[{kernel, dev}];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

}  // namespace rt

using namespace rt;

extern "C" const char *rt_last_error(void) { return g_err.c_str(); }

extern "C" int64_t rt_grid_len(double t_end, double sample_dt) {
  if (!(sample_dt > 0.0) || !std::isfinite(t_end) || t_end < 0.0) return 0;
  return (int64_t)std::floor(t_end / sample_dt * (1.0 + 1e-12)) + 1;
}

extern "C" int rt_network_create(int32_t N, int32_t M, int64_t n_reac_nz, const int32_t *reac_rxn,
                                 const int32_t *reac_sp, const int32_t *reac_coef, int64_t n_stoi_nz,
                                 const int32_t *stoi_rxn, const int32_t *stoi_sp, const int32_t *stoi_delta,
                                 const double *c, rt_network **out) {
  clear_error();
  if (!out) return set_error(RT_ERR_INVALID_ARG, "rt_network_create: out is NULL");
  *out = nullptr;
  if (N < 1 || M < 1) return set_error(RT_ERR_INVALID_ARG, "need n_species >= 1 and n_reactions >= 1 (got %d, %d)", N, M);
  if (n_reac_nz < 0 || n_stoi_nz < 0) return set_error(RT_ERR_INVALID_ARG, "negative nonzero count");
  if ((n_reac_nz > 0 && (!reac_rxn || !reac_sp || !reac_coef)) ||
      (n_stoi_nz > 0 && (!stoi_rxn || !stoi_sp || !stoi_delta)) || !c)
    return set_error(RT_ERR_INVALID_ARG, "NULL network array");

  // reactants, merged per reaction
  std::vector<std::vector<std::pair<int32_t, int32_t>>> reac(M);
  for (int64_t i = 0; i < n_reac_nz; i++) {
    const int32_t k = reac_rxn[i], s = reac_sp[i], q = reac_coef[i];
    if (k < 0 || k >= M) return set_error(RT_ERR_INVALID_ARG, "reactant entry %lld: reaction %d out of range", (long long)i, k);
    if (s < 0 || s >= N) return set_error(RT_ERR_INVALID_ARG, "reactant entry %lld: species %d out of range", (long long)i, s);
    if (q <= 0) return set_error(RT_ERR_INVALID_ARG, "reactant entry %lld: coefficient %d must be positive", (long long)i, q);
    auto &L = reac[k];
    auto it = std::find_if(L.begin(), L.end(), [&](const std::pair<int32_t, int32_t> &p) { return p.first == s; });
    if (it == L.end()) L.push_back({s, q});
    else {
      if (it->second > 2 || q > 2) return set_error(RT_ERR_UNSUPPORTED, "reaction %d: more than two reactant molecules", k);
      it->second += q;
    }
  }
  std::vector<int2> rdesc(M);
  for (int32_t k = 0; k < M; k++) {
    int32_t order = 0;
    for (auto &p : reac[k]) order += p.second;
    if (order > 2) return set_error(RT_ERR_UNSUPPORTED, "reaction %d has %d reactant molecules; at most 2 are supported", k, order);
    auto &L = reac[k];
    if (order == 0) rdesc[k] = make_int2(-1, -1);
    else if (order == 1) rdesc[k] = make_int2(L[0].first, RD_UNI);
    else if (L.size() == 1) rdesc[k] = make_int2(L[0].first, RD_DIMER);
    else rdesc[k] = make_int2(std::min(L[0].first, L[1].first), std::max(L[0].first, L[1].first));
  }
  for (int32_t k = 0; k < M; k++)
    if (!std::isfinite(c[k]) || c[k] < 0.0)
      return set_error(RT_ERR_INVALID_ARG, "rate c[%d] = %g must be finite and >= 0", k, c[k]);

  // net change, merged per reaction, zeros dropped
  std::vector<std::map<int32_t, int64_t>> net(M);
  for (int64_t i = 0; i < n_stoi_nz; i++) {
    const int32_t k = stoi_rxn[i], s = stoi_sp[i];
    if (k < 0 || k >= M) return set_error(RT_ERR_INVALID_ARG, "stoichiometry entry %lld: reaction %d out of range", (long long)i, k);
    if (s < 0 || s >= N) return set_error(RT_ERR_INVALID_ARG, "stoichiometry entry %lld: species %d out of range", (long long)i, s);
    net[k][s] += stoi_delta[i];
  }
  std::vector<int32_t> vptr(M + 1, 0);
  std::vector<int2> vlist;
  int32_t max_vlen = 0;
  for (int32_t k = 0; k < M; k++) {
    int32_t len = 0;
    for (auto &kv : net[k]) {
      if (kv.second == 0) continue;
      if (kv.second < INT32_MIN || kv.second > INT32_MAX)
        return set_error(RT_ERR_INVALID_ARG, "reaction %d: net change of species %d out of int32 range", k, kv.first);
      if (kv.second < 0) {
        int32_t sig = 0;
        for (auto &p : reac[k])
          if (p.first == kv.first) sig = p.second;
        if (-kv.second > sig)
          return set_error(RT_ERR_INVALID_ARG,
                           "reaction %d consumes %lld of species %d but has only %d of it as reactant", k,
                           (long long)-kv.second, kv.first, sig);
      }
      vlist.push_back(make_int2(kv.first, (int32_t)kv.second));
      len++;
    }
    vptr[k + 1] = vptr[k] + len;
    max_vlen = std::max(max_vlen, len);
  }

  // species -> reactions that read it (each reaction once per distinct reactant species)
  std::vector<int32_t> sptr(N + 1, 0), slist;
  for (int32_t k = 0; k < M; k++)
    for (auto &p : reac[k]) sptr[p.first + 1]++;
  for (int32_t s = 0; s < N; s++) sptr[s + 1] += sptr[s];
  slist.resize(sptr[N]);
  {
    std::vector<int32_t> fill(sptr.begin(), sptr.end() - 1);
    for (int32_t k = 0; k < M; k++)
      for (auto &p : reac[k]) slist[fill[p.first]++] = k;
  }
  int32_t max_dep = 0;
  int64_t dep_nz = 0;
  for (int32_t k = 0; k < M; k++) {
    int64_t d = 0;
    for (int32_t i = vptr[k]; i < vptr[k + 1]; i++) d += sptr[vlist[i].x + 1] - sptr[vlist[i].x];
    dep_nz += d;
    max_dep = (int32_t)std::max<int64_t>(max_dep, d);
  }
  std::vector<uint64_t> depmask;
  if (M <= 64) {
    depmask.assign(M, 0);
    for (int32_t k = 0; k < M; k++)
      for (int32_t i = vptr[k]; i < vptr[k + 1]; i++)
        for (int32_t q = sptr[vlist[i].x]; q < sptr[vlist[i].x + 1]; q++) depmask[k] |= 1ull << slist[q];
  }
  // per reaction and lane of a G-lane segment: which of the lane's channels (l + G r, r < 8)
  // read a changed species
  auto dep_bytes = [&](int G) {
    std::vector<uint8_t> d((size_t)M * G, 0);
    for (int32_t k = 0; k < M; k++)
      for (int32_t i = vptr[k]; i < vptr[k + 1]; i++)
        for (int32_t q = sptr[vlist[i].x]; q < sptr[vlist[i].x + 1]; q++) {
          const int32_t ch = slist[q];
          d[(size_t)k * G + (ch % G)] |= (uint8_t)(1u << (ch / G));
        }
    return d;
  };
  std::vector<uint8_t> depw, depw16, depw8;
  if (M <= 256) depw = dep_bytes(32);
  if (M <= 128) depw16 = dep_bytes(16);
  if (M <= 64) depw8 = dep_bytes(8);
  // per reaction in 48 bytes, when every reaction changes at most 4 species by -128..127 and
  // N < 2^24: its packed net change and the reader lists of the species it changes (one load
  // per fired reaction in the tree mapping)
  std::vector<int4> vdep;
  {
    bool fits = max_vlen <= 4 && N < (1 << 24);
    for (size_t i = 0; i < vlist.size() && fits; i++) fits = vlist[i].y >= -128 && vlist[i].y <= 127;
    if (fits) {
      vdep.assign((size_t)3 * M, make_int4(0, 0, 0, 0));
      for (int32_t k = 0; k < M; k++) {
        int w[4] = {0, 0, 0, 0}, rb[4] = {0, 0, 0, 0}, rl[4] = {0, 0, 0, 0};
        for (int32_t i = vptr[k]; i < vptr[k + 1]; i++) {
          const int32_t sp = vlist[i].x, q = i - vptr[k];
          w[q] = (int)(((unsigned)sp << 8) | ((unsigned)vlist[i].y & 0xFFu));
          rb[q] = sptr[sp];
          rl[q] = sptr[sp + 1] - sptr[sp];
        }
        vdep[(size_t)3 * k] = make_int4(w[0], w[1], w[2], w[3]);
        vdep[(size_t)3 * k + 1] = make_int4(rb[0], rb[1], rb[2], rb[3]);
        vdep[(size_t)3 * k + 2] = make_int4(rl[0], rl[1], rl[2], rl[3]);
      }
    }
  }
  // per reaction the channels its firing touches: the reader lists of its changed species,
  // concatenated (small and mid-size networks; the block routine marks them from one list)
  std::vector<int32_t> dptr, dlist;
  if (M <= kDepListMaxM) {
    dptr.assign((size_t)M + 1, 0);
    for (int32_t k = 0; k < M; k++) {
      for (int32_t i = vptr[k]; i < vptr[k + 1]; i++)
        for (int32_t q = sptr[vlist[i].x]; q < sptr[vlist[i].x + 1]; q++) dlist.push_back(slist[q]);
      dptr[(size_t)k + 1] = (int32_t)dlist.size();
    }
  }
  std::vector<double> cc(c, c + M);
  for (auto &x : cc)
    if (x == 0.0) x = 0.0;  // -0.0 -> +0.0 so propensities are never negative zero

  // one arena: every array 256-byte aligned
  rt_network *g = new rt_network();
  size_t off = 0;
  g->off_rdesc = off; off = align_up(off + sizeof(int2) * M, 256);
  g->off_c = off; off = align_up(off + sizeof(double) * M, 256);
  g->off_c0 = off; off = align_up(off + sizeof(double) * M, 256);
  g->off_vptr = off; off = align_up(off + sizeof(int32_t) * (M + 1), 256);
  g->off_vlist = off; off = align_up(off + sizeof(int2) * std::max<size_t>(1, vlist.size()), 256);
  g->off_sptr = off; off = align_up(off + sizeof(int32_t) * (N + 1), 256);
  g->off_slist = off; off = align_up(off + sizeof(int32_t) * std::max<size_t>(1, slist.size()), 256);
  g->off_dep = off; off = align_up(off + sizeof(uint64_t) * std::max<size_t>(1, depmask.size()), 256);
  g->off_depw = off; off = align_up(off + std::max<size_t>(1, depw.size()), 256);
  g->off_depw16 = off; off = align_up(off + std::max<size_t>(1, depw16.size()), 256);
  g->off_depw8 = off; off = align_up(off + std::max<size_t>(1, depw8.size()), 256);
  g->off_vdep = off; off = align_up(off + sizeof(int4) * std::max<size_t>(1, vdep.size()), 256);
  g->off_dptr = off; off = align_up(off + sizeof(int32_t) * std::max<size_t>(1, dptr.size()), 256);
  g->off_dlist = off; off = align_up(off + sizeof(int32_t) * std::max<size_t>(1, dlist.size()), 256);
  g->arena_bytes = off;
  g->host_blob.assign(off, '\0');
  char *hb = &g->host_blob[0];
  memcpy(hb + g->off_rdesc, rdesc.data(), sizeof(int2) * M);
  memcpy(hb + g->off_c, cc.data(), sizeof(double) * M);
  memcpy(hb + g->off_c0, cc.data(), sizeof(double) * M);
  g->c_host = cc;
  memcpy(hb + g->off_vptr, vptr.data(), sizeof(int32_t) * (M + 1));
  if (!vlist.empty()) memcpy(hb + g->off_vlist, vlist.data(), sizeof(int2) * vlist.size());
  memcpy(hb + g->off_sptr, sptr.data(), sizeof(int32_t) * (N + 1));
  if (!slist.empty()) memcpy(hb + g->off_slist, slist.data(), sizeof(int32_t) * slist.size());
  if (!depmask.empty()) memcpy(hb + g->off_dep, depmask.data(), sizeof(uint64_t) * depmask.size());
  if (!depw.empty()) memcpy(hb + g->off_depw, depw.data(), depw.size());
  if (!depw16.empty()) memcpy(hb + g->off_depw16, depw16.data(), depw16.size());
  if (!depw8.empty()) memcpy(hb + g->off_depw8, depw8.data(), depw8.size());
  if (!vdep.empty()) memcpy(hb + g->off_vdep, vdep.data(), sizeof(int4) * vdep.size());
  if (!dptr.empty()) memcpy(hb + g->off_dptr, dptr.data(), sizeof(int32_t) * dptr.size());
  if (!dlist.empty()) memcpy(hb + g->off_dlist, dlist.data(), sizeof(int32_t) * dlist.size());

  cudaGetDevice(&g->device);
  cudaError_t e = cudaMalloc(&g->arena, g->arena_bytes);
  if (e != cudaSuccess) {
    delete g;
    return set_error(e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA, "cudaMalloc(%zu): %s", off,
                     cudaGetErrorString(e));
  }
  e = cudaMemcpy(g->arena, hb, g->arena_bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(g->arena);
    delete g;
    return set_error(RT_ERR_CUDA, "cudaMemcpy: %s", cudaGetErrorString(e));
  }
  char *db = (char *)g->arena;
  DevNet &d = g->dev;
  d.N = N;
  d.M = M;
  d.n_vnz = (int32_t)vlist.size();
  d.max_vlen = max_vlen;
  d.rdesc = (const int2 *)(db + g->off_rdesc);
  d.c = (const double *)(db + g->off_c);
  d.c0 = (const double *)(db + g->off_c0);
  d.vptr = (const int32_t *)(db + g->off_vptr);
  d.vlist = (const int2 *)(db + g->off_vlist);
  d.sptr = (const int32_t *)(db + g->off_sptr);
  d.slist = (const int32_t *)(db + g->off_slist);
  d.depmask = M <= 64 ? (const uint64_t *)(db + g->off_dep) : nullptr;
  d.depw = M <= 256 ? (const uint8_t *)(db + g->off_depw) : nullptr;
  d.depw16 = M <= 128 ? (const uint8_t *)(db + g->off_depw16) : nullptr;
  d.depw8 = M <= 64 ? (const uint8_t *)(db + g->off_depw8) : nullptr;
  d.vdep = vdep.empty() ? nullptr : (const int4 *)(db + g->off_vdep);
  d.dptr = dptr.empty() ? nullptr : (const int32_t *)(db + g->off_dptr);
  d.dlist = dptr.empty() ? nullptr : (const int32_t *)(db + g->off_dlist);
  g->max_dependents = max_dep;
  g->n_dep_nz = dep_nz;
  if (M <= kSmallM && N <= kSmallN) {
    SmallNet &sn = g->small;
    sn.ok = 1;
    for (int32_t k = 0; k < M; k++) {
      sn.s0[k] = rdesc[k].x;
      sn.s1[k] = rdesc[k].y;
      sn.c[k] = cc[k];
      sn.dep[k] = (uint32_t)depmask[k];
      for (int32_t i = vptr[k]; i < vptr[k + 1]; i++) sn.delta[k][vlist[i].x] = vlist[i].y;
    }
  }
  *out = g;
  return RT_OK;
}

extern "C" void rt_network_destroy(rt_network *g) {
  if (!g) return;
  if (g->beta_dev) cudaFree(g->beta_dev);
  if (g->arena) cudaFree(g->arena);
  delete g;
}

extern "C" int rt_network_info(const rt_network *g, int32_t *n_species, int32_t *n_reactions,
                               int32_t *max_dependents, int64_t *n_dependency_nz) {
  clear_error();
  if (!g) return set_error(RT_ERR_INVALID_ARG, "rt_network_info: NULL network");
  if (n_species) *n_species = g->dev.N;
  if (n_reactions) *n_reactions = g->dev.M;
  if (max_dependents) *max_dependents = g->max_dependents;
  if (n_dependency_nz) *n_dependency_nz = g->n_dep_nz;
  return RT_OK;
}

extern "C" int rt_network_set_enabled(rt_network *g, const uint8_t *enabled) {
  clear_error();
  if (!g) return set_error(RT_ERR_INVALID_ARG, "rt_network_set_enabled: NULL network");
  const int32_t M = g->dev.M;
  std::vector<double> eff(g->c_host);
  if (enabled)
    for (int32_t k = 0; k < M; k++)
      if (!enabled[k]) eff[k] = 0.0;
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != g->device) return set_error(RT_ERR_INVALID_ARG, "network lives on device %d, device %d is current", g->device, dev);
  const cudaError_t e = cudaMemcpy((char *)g->arena + g->off_c, eff.data(), sizeof(double) * M, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return set_error(RT_ERR_CUDA, "cudaMemcpy: %s", cudaGetErrorString(e));
  memcpy(&g->host_blob[0] + g->off_c, eff.data(), sizeof(double) * M);
  if (g->small.ok)
    for (int32_t k = 0; k < M; k++) g->small.c[k] = eff[k];
  return RT_OK;
}

extern "C" int rt_network_set_rate_slopes(rt_network *g, const double *beta) {
  clear_error();
  if (!g) return set_error(RT_ERR_INVALID_ARG, "rt_network_set_rate_slopes: NULL network");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != g->device) return set_error(RT_ERR_INVALID_ARG, "network lives on device %d, device %d is current", g->device, dev);
  const int32_t M = g->dev.M;
  if (!beta) {
    if (g->beta_dev) cudaFree(g->beta_dev);
    g->beta_dev = nullptr;
    g->dev.beta = nullptr;
    return RT_OK;
  }
  for (int32_t k = 0; k < M; k++)
    if (!std::isfinite(beta[k]) || !(beta[k] >= 0.0))
      return set_error(RT_ERR_INVALID_ARG, "rate slope beta[%d] = %g must be finite and >= 0", k, beta[k]);
  std::vector<double> b(beta, beta + M);
  for (auto &x : b)
    if (x == 0.0) x = 0.0;  // -0.0 -> +0.0
  if (!g->beta_dev) {
    const cudaError_t e = cudaMalloc(&g->beta_dev, sizeof(double) * M);
    if (e != cudaSuccess) {
      g->beta_dev = nullptr;
      return set_error(RT_ERR_OOM, "cudaMalloc: %s", cudaGetErrorString(e));
    }
  }
  const cudaError_t e = cudaMemcpy(g->beta_dev, b.data(), sizeof(double) * M, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return set_error(RT_ERR_CUDA, "cudaMemcpy: %s", cudaGetErrorString(e));
  g->dev.beta = g->beta_dev;
  return RT_OK;
}

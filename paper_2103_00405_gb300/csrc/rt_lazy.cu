// rt_lazy.cu -- large networks in the absolute-time form: a thread-block cluster per
// trajectory, the argmin kept in a min-tree, only the touched channels updated per event.
//
// The method in its absolute-time ("lazy") form, the Gibson-Bruck next reaction method
// with the dependency graph the paper describes (Sec. 5; Eq. 17, 24-27 in internal
// times): every channel keeps P_k, T_k (its internal time up to the real time s_k of
// its last update), a_k and its absolute firing time tau_k = s_k + (P_k - T_k) / a_k.
// An event at t = tau_mu touches only mu and the channels that read a species the
// event changed: T_k += a_k (t - s_k), s_k = t, P_mu += E (Eq. 27), a_k = c_k h_k(X)
// (Eq. 1-2), tau_k recomputed.  Every other tau_k stays as it is, so an event costs a
// few hundred channel updates instead of a pass over all M channels.
//
// The argmin over tau is the paper's "binary tree searching" of the next reaction
// (Sec. 6) in GPU form: the trajectory's channels are split into C contiguous slices,
// one per CTA of a thread-block cluster; a CTA keeps, in shared memory, the minimum
// (tau, k) of every group of 32 consecutive channels of its slice.  Per event a CTA
//   1. reduces its group minima (block reduction) to its slice minimum,
//   2. posts (tau, k, a) of it into every CTA's mailbox (distributed shared memory,
//      release stores) and polls its own mailbox (acquire loads, bounded: after
//      spin_limit polls the trajectory ends with RT_TRAJ_TIMEOUT) -- every CTA then
//      takes the same decision from the same C entries,
//   3. fires: updates its own copy of X, draws the new increment if it owns mu,
//   4. updates the touched channels of its slice (from the species -> readers lists),
//   5. updates the minima of the 32-channel groups that hold a touched channel (one thread per
//      group; a group whose minimum was touched re-reads its untouched channels, one warp each).
// Ties go to the smallest index at every level, so the minimum is the exact one.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdlib>

#include "rt_sim.cuh"

namespace cg = cooperative_groups;

namespace rt {

constexpr int kLazyThreads = 512;
constexpr int kLazyWarps = kLazyThreads / 32;
constexpr int kLazyMaxC = 16;
constexpr int kLazyMaxVlen = 16;  // net-change entries of one reaction kept in shared memory

// one channel's state; 32 bytes so a touched channel is one sector
struct __align__(32) ChanRec {
  double P;  // internal time of the next firing
  double T;  // internal time accounted up to s
  double s;  // real time of the last update
  double a;  // propensity since s
};

constexpr int kPostWarp = kLazyWarps - 1;         // the slice minimum, the posts and the L2 prefetch (no global stores)
constexpr int kDrawTid = (kLazyWarps - 2) * 32;    // lane 0 of warp 14 updates the fired channel

// a mailbox slot: the posting CTA's slice minimum for one event
struct __align__(16) Mail {
  unsigned long long w;     // bits of tau (+inf if none)
  unsigned long long a;     // bits of its propensity
  int4 v, rb, rl;           // its dependency record (DevNet::vdep; zeros if none)
  unsigned long long flag;  // (seq << 32) | (uint32)k, written last with release semantics
  unsigned long long pad;
};

struct LazyArgs {
  RunArgs r;
  int C;              // CTAs per trajectory (cluster size)
  int64_t Ms;         // row stride of CH / TAU / ENX / NK (multiple of 32 * C)
  int64_t chunk;      // channels per CTA slice (multiple of 32)
  ChanRec *CH;
  double *TAU;
  double *ENX;        // each channel's next Exp(1) increment, drawn ahead of its firing
  int32_t *NK;
  int cap;            // channels one event can touch in a slice, at most
  int sptr_smem;      // 1: the species -> readers offsets are copied to shared memory
  int tend_finite;
  int want_T;         // t_internal or loglik requested
  long long spin_limit;
};

// Absolute firing time of a channel updated at real time su (Eq. 25 in absolute form).
__device__ __forceinline__ double lazy_tau(double P, double T, double a, double su) {
  if (dbits(a) == 0) return bitsd(kInfBits);
  const double rem = __dsub_rn(P, T);
  const double w = dbits(rem) > 0 ? __ddiv_rn(rem, a) : 0.0;
  return __dadd_rn(su, w);
}

__global__ void k_lazy_init(const LazyArgs L) {
  const RunArgs &r = L.r;
  const int64_t total = r.n_traj * L.Ms;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = i / L.Ms;
    const int64_t k = i - j * L.Ms;
    ChanRec c;
    c.T = 0.0;
    c.s = 0.0;
    c.P = 0.0;
    c.a = 0.0;
    double tau = bitsd(kInfBits), enx = 0.0;
    if (k < r.net.M) {
      const int32_t *x0 = r.x0 + (r.per_traj_x0 ? j * r.net.N : 0);
      const uint64_t g = (uint64_t)(r.traj_offset + j);
      c.P = exp1_draw(r.seed, g, (uint32_t)k, 0u, r.stream_id);
      enx = exp1_draw(r.seed, g, (uint32_t)k, 1u, r.stream_id);
      c.a = propensity<false>(r.net.rdesc[k], r.net.c[k], [&](int s) { return x0[s]; });
      tau = lazy_tau(c.P, 0.0, c.a, 0.0);
    }
    L.CH[i] = c;
    L.TAU[i] = tau;
    L.ENX[i] = enx;
    L.NK[i] = 0;
  }
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t map_rank(uint32_t addr, uint32_t rank) {
  uint32_t out;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(addr), "r"(rank));
  return out;
}

__device__ __forceinline__ void st_cluster_v4(uint32_t addr, int4 v) {
  asm volatile("st.shared::cluster.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}

__device__ __forceinline__ void post_mail(uint32_t remote, unsigned long long w, unsigned long long a, int4 v, int4 rb,
                                          int4 rl, unsigned long long flag) {
  asm volatile("st.shared::cluster.v2.u64 [%0], {%1, %2};" ::"r"(remote), "l"(w), "l"(a) : "memory");
  st_cluster_v4(remote + 16, v);
  st_cluster_v4(remote + 32, rb);
  st_cluster_v4(remote + 48, rl);
  asm volatile("st.release.cluster.shared::cluster.u64 [%0], %1;" ::"r"(remote + 64), "l"(flag) : "memory");
}

// a hint: bring the line holding p into L2 (no register result, never faults on a valid address)
__device__ __forceinline__ void prefetch_l2(const void *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ unsigned long long acquire_flag(uint32_t cluster_addr) {
  unsigned long long v;
  asm volatile("ld.acquire.cluster.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(cluster_addr) : "memory");
  return v;
}

__device__ __forceinline__ bool lex_less(long long w1, int k1, long long w2, int k2) {
  return w1 < w2 || (w1 == w2 && k1 < k2);
}

// (w, k) lexicographic minimum over the 32 lanes of a warp
__device__ __forceinline__ void warp_lexmin(long long &w, int &k) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long w2 = __shfl_xor_sync(0xFFFFFFFFu, w, o);
    const int k2 = __shfl_xor_sync(0xFFFFFFFFu, k, o);
    if (lex_less(w2, k2, w, k)) {
      w = w2;
      k = k2;
    }
  }
}

struct LazyDecision {
  int mu;       // fired channel (-1: none can fire)
  int stop;     // 0 continue, else 1 + status
  int vlen;     // net-change entries of mu
  int grid;     // 1: grid points fall before this event
  double tmin;  // event time
  double a_mu;  // propensity of mu before the event
  int2 vl[kLazyMaxVlen];
};

// a warp's candidate for the slice minimum with its prefetched dependency record
struct PostStage {
  long long w;
  double a;
  int4 v, rb, rl;
  int k;
};

template <bool LL>
__global__ void __launch_bounds__(kLazyThreads, 1) k_lazy(const LazyArgs L) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Mail mbox[2][kLazyMaxC];
  __shared__ PostStage red[kLazyWarps];  // each warp's candidate for the slice minimum
  __shared__ LazyDecision dec;
  __shared__ int s_bad, s_ntouch, s_nrel, s_ngl;
  __shared__ int s_lofs[kLazyMaxVlen + 1];  // prefix offsets into the changed species' reader lists
  __shared__ int s_lbeg[kLazyMaxVlen];

  cg::cluster_group cluster = cg::this_cluster();
  const RunArgs &r = L.r;
  const int M = r.net.M, N = r.net.N;
  const int C = L.C;
  const int c = (int)cluster.block_rank();
  const int64_t j = blockIdx.x / C;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t k0 = (int64_t)c * L.chunk;
  const int64_t k1 = min((int64_t)M, k0 + L.chunk);
  const int ng = (int)(L.chunk / 32);  // 32-channel groups of this slice (the last CTA's may run past M)
  const int cap = L.cap;

  // shared memory: per group its minimum (tau bits, channel) and the head of this event's list
  // of its touched channels; the touched channels of an event with their new firing times and
  // list links; the touched groups; per reloaded group its touched-channel minimum and mask; X;
  // species offsets
  long long *gw = (long long *)smem;
  long long *tw = gw + ng;
  long long *rcw = tw + cap;
  int *gk = (int *)(rcw + cap);
  int *ghead = gk + ng;
  int *tk = ghead + ng;
  int *tnext = tk + cap;
  int *glist = tnext + cap;
  int *rq = glist + cap;
  int *rck = rq + cap;
  uint32_t *rmask = (uint32_t *)(rck + cap);
  int *Xs = (int *)(rmask + cap);
  int *sp = Xs + N;
  const int *sptr = L.sptr_smem ? sp : r.net.sptr;

  ChanRec *CH = L.CH + j * L.Ms;
  double *TAU = L.TAU + j * L.Ms;
  double *ENX = L.ENX + j * L.Ms;
  int32_t *NK = L.NK + j * L.Ms;
  const uint64_t g = (uint64_t)(r.traj_offset + j);
  const int32_t *x0 = r.x0 + (r.per_traj_x0 ? j * N : 0);

  for (int i = tid; i < 2 * kLazyMaxC; i += blockDim.x) {
    Mail &m = mbox[i / kLazyMaxC][i % kLazyMaxC];
    m.w = 0;
    m.a = 0;
    m.v = m.rb = m.rl = make_int4(0, 0, 0, 0);
    m.flag = 0;
    m.pad = 0;
  }
  if (tid == 0) {
    s_bad = 0;
    s_ntouch = 0;
    s_nrel = 0;
    s_ngl = 0;
  }
  __syncthreads();
  for (int s = tid; s < N; s += blockDim.x) {
    const int v = x0[s];
    Xs[s] = v;
    if (v < 0) s_bad = 1;
  }
  if (L.sptr_smem)
    for (int s = tid; s <= N; s += blockDim.x) sp[s] = r.net.sptr[s];
  for (int q = tid; q < ng; q += blockDim.x) ghead[q] = -1;
  // group minima of the slice from the initial firing times
  for (int q = warp; q < ng; q += kLazyWarps) {
    const int64_t k = k0 + (int64_t)q * 32 + lane;
    long long w = kInfBits;
    int kk = INT_MAX;
    if (k < k1) {
      w = dbits(TAU[k]);
      kk = (int)k;
    }
    warp_lexmin(w, kk);
    if (lane == 0) {
      gw[q] = w;
      gk[q] = kk;
    }
  }
  __syncthreads();
  cluster.sync();  // every mailbox is zeroed before any CTA posts into it
  const bool bad = s_bad != 0;

  const uint32_t mb_local = smem_addr(&mbox[0][0]);
  double t = 0.0, ll = 0.0;
  int32_t ev = 0;
  int status = bad ? RT_TRAJ_BAD_X0 : RT_TRAJ_TEND;
  unsigned int seq = 0;  // posts so far
  int64_t gi = 0;
  double next_g = 0.0;
  const int64_t tend_bits = dbits(r.t_end);
  int pend_k = -1;  // draw thread: channel whose next increment is due
  int32_t pend_n = 0;

  auto record = [&](int64_t gidx, bool known) {  // CTA 0, all threads
    if (r.out.grid_dev) {
      int32_t *gp = r.out.grid_dev + (j * r.G + gidx) * N;
      for (int s = tid; s < N; s += blockDim.x) gp[s] = known ? Xs[s] : -1;
    }
    if (r.out.grid_sum_dev && known) {
      for (int s = tid; s < N; s += blockDim.x) {
        const long long x = Xs[s];
        atomicAdd((unsigned long long *)(r.out.grid_sum_dev + gidx * N + s), (unsigned long long)x);
        if (r.out.grid_sumsq_dev)
          atomicAdd((unsigned long long *)(r.out.grid_sumsq_dev + gidx * N + s), (unsigned long long)(x * x));
      }
      if (tid == 0 && r.out.grid_count_dev) atomicAdd((unsigned long long *)(r.out.grid_count_dev + gidx), 1ull);
    }
  };
  // a touched channel of the slice and its new firing time join this event's list and the
  // list of its group; the first one of a group lists the group
  auto touch = [&](int64_t k, long long w) {
    const int i = atomicAdd(&s_ntouch, 1);
    tk[i] = (int)k;
    tw[i] = w;
    const int q = (int)((k - k0) >> 5);
    const int nx = atomicExch(&ghead[q], i);
    tnext[i] = nx;
    if (nx < 0) glist[atomicAdd(&s_ngl, 1)] = q;
  };

  if (!bad) {
    for (;;) {
      // ---- 1. the slice minimum over the group minima; each warp prefetches its candidate's
      // dependency record and propensity while the block reduction completes; a warp that never
      // stores to global memory takes the final minimum and posts it to every CTA of the cluster
      seq += 1;
      const int par = seq & 1;
      {
        long long w = kInfBits;
        int kk = INT_MAX;
        for (int q = tid; q < ng; q += blockDim.x)
          if (lex_less(gw[q], gk[q], w, kk)) {
            w = gw[q];
            kk = gk[q];
          }
        warp_lexmin(w, kk);
        if (lane == 0) {
          PostStage &st = red[warp];
          st.w = w;
          st.k = kk;
          st.v = st.rb = st.rl = make_int4(0, 0, 0, 0);
          st.a = 0.0;
          if (w != kInfBits) {
            if (r.net.vdep) {
              st.v = r.net.vdep[3 * (int64_t)kk];
              st.rb = r.net.vdep[3 * (int64_t)kk + 1];
              st.rl = r.net.vdep[3 * (int64_t)kk + 2];
            }
            st.a = CH[kk].a;
          }
        }
      }
      __syncthreads();
      if (warp == kPostWarp) {
        long long w = lane < kLazyWarps ? red[lane].w : kInfBits;
        int kk = lane < kLazyWarps ? red[lane].k : INT_MAX;
        int src = lane;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const long long w2 = __shfl_xor_sync(0xFFFFFFFFu, w, o);
          const int k2 = __shfl_xor_sync(0xFFFFFFFFu, kk, o);
          const int s2 = __shfl_xor_sync(0xFFFFFFFFu, src, o);
          if (lex_less(w2, k2, w, kk)) {
            w = w2;
            kk = k2;
            src = s2;
          }
        }
        if (lane < C) {
          const PostStage &st = red[src < kLazyWarps ? src : 0];
          const unsigned long long flag = ((unsigned long long)seq << 32) | (uint32_t)kk;
          const uint32_t slot = mb_local + (uint32_t)((par * kLazyMaxC + c) * sizeof(Mail));
          post_mail(map_rank(slot, lane), (unsigned long long)w, (unsigned long long)dbits(st.a), st.v, st.rb, st.rl,
                    flag);
        }
        // While the posts travel: if this slice's candidate is the one that fires, the touched-
        // channel phase of every CTA starts by reading its reader lists.  Prefetch their lines
        // into L2 now (one CTA's candidate fires, so one CTA's prefetch is the useful one; the
        // others cost L2 traffic only), with the fired channel's own record, increment and group.
        if (w != kInfBits && r.net.vdep) {
          const PostStage &st = red[src < kLazyWarps ? src : 0];
          const int vw[4] = {st.v.x, st.v.y, st.v.z, st.v.w};
          const int rb[4] = {st.rb.x, st.rb.y, st.rb.z, st.rb.w};
          const int rl[4] = {st.rl.x, st.rl.y, st.rl.z, st.rl.w};
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            if (vpack_delta(vw[i]) == 0 || rl[i] <= 0) continue;
            const uintptr_t b = (uintptr_t)(r.net.slist + rb[i]) & ~(uintptr_t)127;
            const uintptr_t e = (uintptr_t)(r.net.slist + rb[i] + rl[i] - 1);
            for (uintptr_t a = b + (uintptr_t)lane * 128; a <= e; a += 32 * 128) prefetch_l2((const void *)a);
          }
          if (lane == 0) {
            prefetch_l2(CH + kk);
            prefetch_l2(ENX + kk);
            prefetch_l2(TAU + (kk & ~31));
            prefetch_l2(TAU + (kk & ~31) + 16);
          }
        }
      }
      if (tid == kDrawTid && pend_k >= 0) {
        // the next increment of the channel this CTA fired last (Eq. 24, 27), drawn while the
        // cluster's posts arrive
        ENX[pend_k] = exp1_draw(r.seed, g, (uint32_t)pend_k, (uint32_t)(pend_n + 1), r.stream_id);
        pend_k = -1;
      }
      if (tid == 0) {
        // wait (bounded) for the C posts of this event, then decide
        bool ok = true;
        long long it = 0;
        long long w = kInfBits;
        int kk = INT_MAX;
        int qbest = 0;
        const uint32_t own = map_rank(mb_local, (uint32_t)c);
        for (int q = 0; q < C && ok; ++q) {
          const uint32_t fa = own + (uint32_t)((par * kLazyMaxC + q) * sizeof(Mail)) + 64;
          unsigned long long f = acquire_flag(fa);
          while ((unsigned int)(f >> 32) != seq) {
            if (++it > L.spin_limit) {
              ok = false;
              break;
            }
            if (it > 64) __nanosleep(32);
            f = acquire_flag(fa);
          }
          if (!ok) break;
          const long long wq = (long long)mbox[par][q].w;
          const int kq = (int)(uint32_t)f;
          if (lex_less(wq, kq, w, kk)) {
            w = wq;
            kk = kq;
            qbest = q;
          }
        }
        dec.stop = 0;
        dec.grid = 0;
        if (!ok) {
          dec.stop = 1 + RT_TRAJ_TIMEOUT;
        } else if (w == kInfBits) {
          dec.stop = 1 + RT_TRAJ_ABSORBED;
        } else if (w > tend_bits) {
          dec.stop = 1 + RT_TRAJ_TEND;
        } else if (ev == r.max_events) {
          dec.stop = 1 + RT_TRAJ_MAX_EVENTS;
        } else {
          int vlen = 0;
          int tot = 0;
          if (r.net.vdep) {
            const Mail &m = mbox[par][qbest];
            const int vw[4] = {m.v.x, m.v.y, m.v.z, m.v.w};
            const int rb[4] = {m.rb.x, m.rb.y, m.rb.z, m.rb.w};
            const int rl[4] = {m.rl.x, m.rl.y, m.rl.z, m.rl.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
              if (vpack_delta(vw[i]) != 0) {
                dec.vl[vlen] = make_int2(vpack_species(vw[i]), vpack_delta(vw[i]));
                s_lbeg[vlen] = rb[i];
                s_lofs[vlen] = tot;
                tot += rl[i];
                ++vlen;
              }
          } else {
            const int vb = r.net.vptr[kk], ve = r.net.vptr[kk + 1];
            for (int i = vb; i < ve; ++i) {
              const int2 e = r.net.vlist[i];
              dec.vl[vlen] = e;
              s_lbeg[vlen] = sptr[e.x];
              s_lofs[vlen] = tot;
              tot += sptr[e.x + 1] - sptr[e.x];
              ++vlen;
            }
          }
          s_lofs[vlen] = tot;
          bool over = false;
          for (int i = 0; i < vlen; ++i) {
            const long long nx = (long long)Xs[dec.vl[i].x] + dec.vl[i].y;
            over |= (nx > INT_MAX) | (nx < 0);
          }
          if (over) {
            dec.stop = 1 + RT_TRAJ_OVERFLOW;
          } else {
            dec.mu = kk;
            dec.vlen = vlen;
            dec.tmin = bitsd(w);
            dec.a_mu = __longlong_as_double((long long)mbox[par][qbest].a);
            dec.grid = (c == 0 && gi < r.G && dbits(next_g) < w) ? 1 : 0;
          }
        }
      }
      __syncthreads();
      if (dec.stop) {
        status = dec.stop - 1;
        break;
      }
      const int mu = dec.mu;
      const double tn = dec.tmin;
      if (dec.grid) {
        while (gi < r.G && dbits(next_g) < dbits(tn)) {
          record(gi, true);
          ++gi;
          next_g = __dmul_rn(__ll2double_rn(gi), r.sample_dt);
        }
        __syncthreads();  // X is read by the recording before it changes
      }
      // ---- 2. fire: X += v_mu (Eq. 5), bookkeeping
      t = tn;
      if (c == 0 && tid == 0) {
        trace_event(r.out, j, ev, mu, tn);
        if (LL) ll = __dadd_rn(ll, rt_ln(dec.a_mu));
      }
      ++ev;
      const int vlen = dec.vlen;
      if (tid < vlen) Xs[dec.vl[tid].x] += dec.vl[tid].y;  // species are distinct within one reaction
      __syncthreads();
      // ---- 3. the touched channels of this slice: new a_k and tau_k
      if (tid == kDrawTid && mu >= k0 && mu < k1) {
        // the fired channel: internal time up to the event, its next increment (drawn ahead,
        // Eq. 27), new propensity and firing time
        ChanRec q = CH[mu];
        const double E = ENX[mu];
        const int32_t n = NK[mu] + 1;
        NK[mu] = n;
        q.T = __dadd_rn(q.T, __dmul_rn(q.a, __dsub_rn(t, q.s)));
        q.s = t;
        q.P = __dadd_rn(q.P, E);
        q.a = propensity<false>(r.net.rdesc[mu], r.net.c[mu], [&](int s) { return Xs[s]; });
        CH[mu] = q;
        const double tau = lazy_tau(q.P, q.T, q.a, t);
        TAU[mu] = tau;
        touch(mu, dbits(tau));
        pend_k = mu;
        pend_n = n;
      } else if (tid < kDrawTid) {
        const int tot = s_lofs[vlen];
        for (int e = tid; e < tot; e += kDrawTid) {
          int li = 0;
          while (e >= s_lofs[li + 1]) ++li;
          const int64_t k = r.net.slist[s_lbeg[li] + (e - s_lofs[li])];
          if (k < k0 || k >= k1 || k == mu) continue;
          const int2 rd = r.net.rdesc[k];
          // a channel reading two changed species is updated once, from its first list
          bool dup = false;
          for (int i = 0; i < li; ++i) {
            const int s = dec.vl[i].x;
            dup |= rd.x == s || (rd.y >= 0 && rd.y == s);
          }
          if (dup) continue;
          ChanRec q = CH[k];
          q.T = __dadd_rn(q.T, __dmul_rn(q.a, __dsub_rn(t, q.s)));
          q.s = t;
          q.a = propensity<false>(rd, r.net.c[k], [&](int s) { return Xs[s]; });
          CH[k] = q;
          const double tau = lazy_tau(q.P, q.T, q.a, t);
          TAU[k] = tau;
          touch(k, dbits(tau));
        }
      }
      __syncthreads();
      // ---- 4. group minima, one thread per touched group.  A group takes the smaller of its
      // previous minimum and its touched channels' minimum, unless its previous minimum channel was
      // touched and its tau grew: then every untouched channel may now be smaller, and the group is
      // reloaded below (its untouched channels from memory).  (If that channel's tau did not grow,
      // every untouched channel still lies above it.)
      const int ngl = s_ngl;
      for (int gi2 = tid; gi2 < ngl; gi2 += blockDim.x) {
        const int q = glist[gi2];
        long long bw = kInfBits;
        int bk = INT_MAX;
        uint32_t bits = 0;
        bool hit = false;
        const int old_k = gk[q];
        const long long old_w = gw[q];
        for (int i = ghead[q]; i >= 0; i = tnext[i]) {
          const int k = tk[i];
          const long long w = tw[i];
          bits |= 1u << (k & 31);  // slices start at multiples of 32
          hit |= k == old_k && w > old_w;  // tau >= 0: bit patterns order like the values
          if (lex_less(w, k, bw, bk)) {
            bw = w;
            bk = k;
          }
        }
        ghead[q] = -1;
        if (hit) {
          const int ri = atomicAdd(&s_nrel, 1);
          rq[ri] = q;
          rcw[ri] = bw;
          rck[ri] = bk;
          rmask[ri] = bits;
        } else {
          if (lex_less(bw, bk, gw[q], gk[q])) {
            gw[q] = bw;
            gk[q] = bk;
          }
        }
      }
      __syncthreads();
      const int nrel = s_nrel;
      for (int ri = warp; ri < nrel; ri += kLazyWarps) {
        const int q = rq[ri];
        const int64_t k = k0 + (int64_t)q * 32 + lane;
        long long w = kInfBits;
        int kk = INT_MAX;
        if (k < k1 && !((rmask[ri] >> lane) & 1u)) {
          w = dbits(__ldcg(TAU + k));
          kk = (int)k;
        }
        warp_lexmin(w, kk);
        if (lane == 0) {
          if (lex_less(rcw[ri], rck[ri], w, kk)) {
            w = rcw[ri];
            kk = rck[ri];
          }
          gw[q] = w;
          gk[q] = kk;
        }
      }
      __syncthreads();
      if (tid == 0) {
        s_ntouch = 0;
        s_nrel = 0;
        s_ngl = 0;
      }
    }
  }

  // ---- finalise
  const bool known = status == RT_TRAJ_TEND || status == RT_TRAJ_ABSORBED;
  if (c == 0)
    for (; gi < r.G; ++gi) record(gi, known);
  if (L.want_T && !bad) {
    // every channel's internal time up to the end of the run
    const double tf = (known && L.tend_finite) ? r.t_end : t;
    for (int64_t k = k0 + tid; k < k1; k += blockDim.x) {
      ChanRec q = CH[k];
      q.T = __dadd_rn(q.T, __dmul_rn(q.a, __dsub_rn(tf, q.s)));
      q.s = tf;
      CH[k] = q;
    }
  }
  if (r.out.t_internal_dev)
    for (int64_t k = k0 + tid; k < k1; k += blockDim.x) r.out.t_internal_dev[j * M + k] = CH[k].T;
  if (r.out.counts_dev)
    for (int64_t k = k0 + tid; k < k1; k += blockDim.x) r.out.counts_dev[j * M + k] = NK[k];
  __threadfence();
  cluster.sync();  // every slice is final; no CTA posts into a mailbox after this point
  if (LL && c == 0 && tid == 0) {
    double sT = 0.0;
    if (!bad)
      for (int k = 0; k < M; ++k) sT = __dadd_rn(sT, __ldcg(&CH[k].T));
    r.out.loglik_dev[j] = bad ? __longlong_as_double(0x7FF8000000000000ll) : __dsub_rn(ll, sT);
  }
  if (c == 0) {
    trace_tail(r.out, j, ev, tid, blockDim.x);
    if (r.out.x_final_dev)
      for (int s = tid; s < N; s += blockDim.x) r.out.x_final_dev[j * N + s] = Xs[s];
    if (tid == 0) {
      if (r.out.n_events_dev) r.out.n_events_dev[j] = ev;
      if (r.out.status_dev) r.out.status_dev[j] = status;
      if (r.out.t_last_dev) r.out.t_last_dev[j] = t;
    }
  }
}

// ----------------------------------------------------------------------------------
// host side
// ----------------------------------------------------------------------------------

static int64_t round_up_l(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

struct LazyPlan {
  int C;
  int64_t chunk, Ms;
  size_t off_CH, off_TAU, off_ENX, off_NK, total;
  size_t smem;
  int sptr_smem;
  int cap;
};

static LazyPlan plan_lazy(const DevNet &net, int max_dependents, int64_t n_traj, int C, size_t smem_budget) {
  LazyPlan p;
  p.C = C;
  p.chunk = round_up_l((net.M + C - 1) / C, 32);
  p.Ms = p.chunk * C;
  const int64_t rows = n_traj > 0 ? n_traj : 1;
  size_t off = 0;
  p.off_CH = off; off += (size_t)rows * p.Ms * sizeof(ChanRec);
  p.off_TAU = off; off += (size_t)rows * p.Ms * 8;
  p.off_ENX = off; off += (size_t)rows * p.Ms * 8;
  p.off_NK = off; off += (size_t)round_up_l(rows * p.Ms * 4, 256);
  p.total = off;
  const int ng = (int)(p.chunk / 32);
  // touched channels of one event in one slice: at most the fired channel and the readers of
  // the species it changes (max_dependents counts them with multiplicity)
  p.cap = (int)std::min<int64_t>(p.chunk, (int64_t)max_dependents + 1);
  // gw, gk, ghead per group; tw, rcw, tk, tnext, glist, rq, rck, rmask per touched channel; X
  const size_t base = (size_t)ng * (8 + 4 + 4) + (size_t)p.cap * (8 + 8 + 4 + 4 + 4 + 4 + 4 + 4) + (size_t)net.N * 4;
  p.sptr_smem = base + (size_t)(net.N + 1) * 4 <= smem_budget ? 1 : 0;
  p.smem = base + (p.sptr_smem ? (size_t)(net.N + 1) * 4 : 0);
  return p;
}

constexpr size_t kLazySmemBudget = 200 * 1024;

// Clusters of C CTAs of the lazy kernel that can be resident at once (0: does not fit).
static int lazy_active_clusters(const LazyPlan &p, bool ll) {
  if (p.smem > kLazySmemBudget) return 0;
  auto kern = ll ? k_lazy<true> : k_lazy<false>;
  if (raise_smem_limit((const void *)kern, p.smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (p.C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)p.C);
  cfg.blockDim = dim3(kLazyThreads);
  cfg.dynamicSmemBytes = p.smem;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = (unsigned)p.C;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (void *)kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// CTAs per trajectory: the largest power of two (<= 8, and <= M / 32) with which every
// trajectory is resident at once, else the one that keeps the most trajectories resident.
static int choose_lazy_C(const DevNet &net, int maxdep, int64_t n_traj, int requested, bool ll) {
  if (requested > 0) return requested;
  int best = 1;
  int64_t best_res = -1;
  for (int C = 8; C >= 1; C /= 2) {
    if (C > 1 && (int64_t)net.M < 32 * (int64_t)C) continue;
    const int act = lazy_active_clusters(plan_lazy(net, maxdep, n_traj, C, kLazySmemBudget), ll);
    if (act <= 0) continue;
    if (act >= n_traj) return C;
    const int64_t res = (int64_t)act;
    if (res > best_res) {
      best_res = res;
      best = C;
    }
  }
  return best;
}

size_t lazy_workspace_bytes(const DevNet &net, int max_dependents, int64_t n_traj, int ctas_per_traj) {
  int C = 0;
  for (int ll = 0; ll < 2; ++ll) C = std::max(C, choose_lazy_C(net, max_dependents, n_traj, ctas_per_traj, ll));
  size_t b = 0;
  for (int c2 = 1; c2 <= C; c2 *= 2) b = std::max(b, plan_lazy(net, max_dependents, n_traj, c2, kLazySmemBudget).total);
  return std::max(b, plan_lazy(net, max_dependents, n_traj, C, kLazySmemBudget).total);
}

int launch_lazy_mapping(const RunArgs &a, int max_dependents, int ctas_per_traj, void *ws, size_t ws_bytes,
                        cudaStream_t s) {
  if (a.n_traj == 0) return RT_OK;
  if (a.net.max_vlen > kLazyMaxVlen)
    return set_error(RT_ERR_UNSUPPORTED, "absolute-time form: a reaction changes %d species (at most %d)",
                     a.net.max_vlen, kLazyMaxVlen);
  const bool ll = a.out.loglik_dev != nullptr;
  const int C = choose_lazy_C(a.net, max_dependents, a.n_traj, ctas_per_traj, ll);
  if (C < 1 || C > kLazyMaxC || (C & (C - 1)))
    return set_error(RT_ERR_INVALID_ARG, "absolute-time form: ctas_per_traj must be a power of two <= %d", kLazyMaxC);
  const LazyPlan p = plan_lazy(a.net, max_dependents, a.n_traj, C, kLazySmemBudget);
  if (p.smem > kLazySmemBudget)
    return set_error(RT_ERR_UNSUPPORTED, "absolute-time form: %d species and %lld channels per CTA do not fit in "
                     "shared memory (%zu bytes)", a.net.N, (long long)p.chunk, p.smem);
  if (!ws || ws_bytes < p.total)
    return set_error(RT_ERR_OOM, "absolute-time form needs %zu bytes of workspace (got %zu)", p.total, ws_bytes);
  if (((uintptr_t)ws & 255) != 0) return set_error(RT_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  // every check before the first enqueued operation
  if (a.n_traj * C > INT_MAX) return set_error(RT_ERR_UNSUPPORTED, "absolute-time form: too many trajectories for one launch");
  if (lazy_active_clusters(p, ll) < 1)
    return set_error(RT_ERR_UNSUPPORTED, "absolute-time form: a cluster of %d CTAs cannot be resident", C);
  char *w = (char *)ws;
  LazyArgs L;
  L.r = a;
  L.C = C;
  L.Ms = p.Ms;
  L.chunk = p.chunk;
  L.CH = (ChanRec *)(w + p.off_CH);
  L.TAU = (double *)(w + p.off_TAU);
  L.ENX = (double *)(w + p.off_ENX);
  L.NK = (int32_t *)(w + p.off_NK);
  L.cap = p.cap;
  L.sptr_smem = p.sptr_smem;
  L.tend_finite = std::isfinite(a.t_end) ? 1 : 0;
  L.want_T = (a.out.t_internal_dev || a.out.loglik_dev) ? 1 : 0;
  long long spin = 20000000;  // polls before a trajectory gives up (each a few tens of ns)
  if (const char *env = getenv("RT_DEBUG_SPIN_LIMIT")) spin = atoll(env);
  L.spin_limit = spin;
  k_lazy_init<<<152 * 8, 256, 0, s>>>(L);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(RT_ERR_CUDA, "init launch: %s", cudaGetErrorString(e));
  auto kern = ll ? k_lazy<true> : k_lazy<false>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.n_traj * C));
  cfg.blockDim = dim3(kLazyThreads);
  cfg.dynamicSmemBytes = p.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = (unsigned)C;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kern, L);
  if (e != cudaSuccess) return set_error(RT_ERR_CUDA, "absolute-time kernel launch: %s", cudaGetErrorString(e));
  return RT_OK;
}

}  // namespace rt

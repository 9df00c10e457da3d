// rt_traj_warp.cuh -- trajectories in warp segments: G lanes per trajectory, 32 / G
// trajectories per warp (channel k in sub-lane k % G, register slot k / G).
//
// The NRRTA loop of Table 2 (Liu & Wang, arXiv:2103.00405), each trajectory's channels
// spread over the G lanes of its segment (P_k, T_k, a_k, n_k; Eq. 17-27).  Per event every
// lane advances its internal times with the pre-event propensities and recomputes the
// ones the last firing changed (per reaction and sub-lane a dependency byte); a segment
// minimum of rigorous float upper bounds of the waiting times is the threshold, and only
// channels not certified to be above it are computed exactly; a shuffle reduction on
// (waiting time bits, channel) inside the segment gives the exact argmin with the
// smallest index on ties (Eq. 25-26).
//
// GB300 issues binary64 instructions at a small fraction of its integer rate, and a
// binary64 warp instruction costs the same with one active lane as with 32.  Everything a
// trajectory does once per event -- the exact division of its candidate, t + dt, P_mu + E
// -- is therefore done for all 32 / G trajectories of the warp in the same instructions:
// exact divisions are compacted (each lane takes its own next uncertified channel, one
// division pass for the whole warp), and so are propensity recomputations.  The Exp(1)
// increments of fired channels are drawn ahead and redrawn in lane-parallel batches when
// a used-up one is needed again, and with the likelihood ln a_mu is taken G events at a
// time, one event per lane.  Trajectories of one warp advance event by event together;
// a finished one leaves its lanes idle until the others finish.  The network arrays may
// live in shared or global memory (generic pointers); X is per trajectory in shared memory.
#pragma once
#include <climits>

#include "rt_sim.cuh"

namespace rt {

struct WarpNet {
  int M, N, nv;
  const int2 *rd;
  const double *c;
  const int *vp;
  const int2 *vl;
  const uint8_t *dep;  // [M][G]: bit r of dep[mu * G + l] -- channel l + G r reads a species mu changes
};

// The log-likelihood's sum_k T_k in k order for every segment of the warp (all lanes call it;
// segments past n_traj pass live = false).
template <int R, int G>
__device__ __forceinline__ double warp_sum_T_in_order(const double (&T)[R], int M, bool live) {
  const int lane = threadIdx.x & 31, base = (lane / G) * G;
  double sT = 0.0;
#pragma unroll
  for (int r = 0; r < R; ++r)
    for (int l = 0; l < G; ++l) {
      const double v = __shfl_sync(0xFFFFFFFFu, T[r], base + l);
      if (live && l + G * r < M) sT = __dadd_rn(sT, v);
    }
  return sT;
}

// Trajectories j0 .. j0 + 32/G - 1 (those < n_traj) in the segments of one warp.  X: the
// warp's 32/G state arrays of N counts; mom: block moment table (or null).
template <int R, int G, bool LL>
__device__ __forceinline__ void warp_trajectories(const RunArgs &A, const WarpNet &net, int *Xw,
                                                  unsigned long long *mom, const int64_t j0, const int tend_finite) {
  static_assert(G == 8 || G == 16 || G == 32, "segment width");
  constexpr unsigned FULL = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31, seg = lane / G, sl = lane % G, base = seg * G;
  const unsigned segmask = G == 32 ? FULL : (((1u << G) - 1u) << base);
  const int M = net.M, N = net.N;
  const int64_t j = j0 + seg;
  const bool live = j < A.n_traj;
  int *X = Xw + seg * N;
  const uint64_t g = (uint64_t)(A.traj_offset + j);
  const int32_t *x0 = A.x0 + (A.per_traj_x0 ? j * (int64_t)N : 0);
  bool badl = false;
  if (live)
    for (int s = sl; s < N; s += G) {
      const int v = x0[s];
      X[s] = v;
      badl |= v < 0;
    }
  const bool bad = (__ballot_sync(FULL, badl) & segmask) != 0;
  __syncwarp();
  auto xat = [&](int s) { return X[s]; };
  const int64_t GN = A.G * N;

  auto record = [&](int64_t gidx, bool known) {  // the segment's lanes
    if (A.out.grid_dev) {
      int32_t *gp = A.out.grid_dev + (j * A.G + gidx) * N;
      for (int s = sl; s < N; s += G) gp[s] = known ? X[s] : -1;
    }
    if (!known || !A.out.grid_sum_dev) return;
    for (int s = sl; s < N; s += G) {
      const long long x = X[s];
      if (mom) {
        atomicAdd(mom + gidx * N + s, (unsigned long long)x);
        atomicAdd(mom + GN + gidx * N + s, (unsigned long long)(x * x));
      } else {
        atomicAdd((unsigned long long *)(A.out.grid_sum_dev + gidx * N + s), (unsigned long long)x);
        if (A.out.grid_sumsq_dev)
          atomicAdd((unsigned long long *)(A.out.grid_sumsq_dev + gidx * N + s), (unsigned long long)(x * x));
      }
    }
    if (sl == 0) {
      if (mom) atomicAdd(mom + 2 * GN + gidx, 1ull);
      else if (A.out.grid_count_dev) atomicAdd((unsigned long long *)(A.out.grid_count_dev + gidx), 1ull);
    }
  };

  // Per channel: P_k, T_k, a_k, n_k and En_k, the Exp(1) increment its next firing adds to
  // P_k (Eq. 27), drawn ahead.
  double P[R], T[R], a[R], En[R];
  int32_t n[R];
  bool run = live && !bad;  // segment-uniform: this trajectory still fires events
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int k = sl + G * r;
    P[r] = 0.0;
    T[r] = 0.0;
    a[r] = 0.0;
    En[r] = 0.0;
    n[r] = 0;
    if (run && k < M) {
      P[r] = exp1_draw(A.seed, g, (uint32_t)k, 0u, A.stream_id);
      En[r] = exp1_draw(A.seed, g, (uint32_t)k, 1u, A.stream_id);
      a[r] = propensity<false>(net.rd[k], net.c[k], xat);
    }
  }
  uint32_t stale = 0;  // bit r: En[r] is used up (slot r's channel fired since its last draw)
  int status = bad ? RT_TRAJ_BAD_X0 : RT_TRAJ_TEND;
  double t = 0.0, ll = 0.0, dprev = 0.0;
  double ring = 0.0;  // with the likelihood: a_mu of event (ev & ~(G-1)) + sl of this trajectory
  int mu_prev = -1;
  int32_t ev = 0;
  int64_t gi = 0;
  double next_g = 0.0;
  const int64_t tend_bits = dbits(A.t_end);

  // ll += ln a_mu of the cnt buffered events of each segment, in event order (the segment's
  // lanes take the logarithms together); cnt is segment-uniform, 0..G
  auto flush_ring = [&](int cnt) {
    double L = 0.0;
    if (sl < cnt) L = rt_ln(ring);
    for (int i = 0; i < G; ++i) {
      const double v = __shfl_sync(FULL, L, base + i);
      if (sl == 0 && i < cnt) ll = __dadd_rn(ll, v);
    }
  };

  while (__any_sync(FULL, run)) {
    // ---- internal times advance with the pre-event propensities (Eq. 17)
    const bool adv = run && dbits(dprev) != 0;
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (adv && sl + G * r < M && dbits(a[r]) != 0) T[r] = __dadd_rn(T[r], __dmul_rn(a[r], dprev));
    // ---- propensities the last firing changed (Eq. 1-2), one compacted pass per slot a lane needs
    uint32_t todo = (run && mu_prev >= 0) ? net.dep[mu_prev * G + sl] : 0u;
    while (__any_sync(FULL, todo != 0)) {
      if (todo) {
        const int r = __ffs(todo) - 1;
        const int k = sl + G * r;
        const double v = propensity<false>(net.rd[k], net.c[k], xat);
#pragma unroll
        for (int q = 0; q < R; ++q)
          if (q == r) a[q] = v;
        todo &= todo - 1;
      }
    }
    // ---- the segment minimum of rigorous float upper bounds of the waiting times
    float ub = __int_as_float(0x7F800000);
    bool act = false;
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (run && sl + G * r < M && dbits(a[r]) != 0) {
        act = true;
        ub = fminf(ub, quot_upper(P[r], T[r], a[r]));
      }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) ub = fminf(ub, __shfl_xor_sync(FULL, ub, o));
    const unsigned actb = __ballot_sync(FULL, act);
    if (run && (actb & segmask) == 0) {
      status = RT_TRAJ_ABSORBED;
      run = false;
    }
    // ---- exact waiting times (Eq. 25) of the channels not certified above the bound: each
    // lane its next such channel per pass, so the divisions of all segments share passes
    const float thr = f32_next_up(ub);
    uint32_t need = 0;
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (run && sl + G * r < M && dbits(a[r]) != 0 && !exceeds(P[r], T[r], a[r], thr)) need |= 1u << r;
    long long bw = kInfBits;
    int bk = INT_MAX;
    while (__any_sync(FULL, need != 0)) {
      if (need) {
        const int r = __ffs(need) - 1;
        const long long wb = dbits(waiting_time(pick<R>(P, r), pick<R>(T, r), pick<R>(a, r)));
        const int k = sl + G * r;
        if (wb < bw || (wb == bw && k < bk)) {
          bw = wb;
          bk = k;
        }
        need &= need - 1;
      }
    }
    // the segment's exact argmin, smallest index on ties (Eq. 26)
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      const long long w2 = __shfl_xor_sync(FULL, bw, o);
      const int k2 = __shfl_xor_sync(FULL, bk, o);
      if (w2 < bw || (w2 == bw && k2 < bk)) {
        bw = w2;
        bk = k2;
      }
    }
    const int mu = bk;
    const double dmin = bitsd(bw);
    const double tn = __dadd_rn(t, dmin);
    if (run) {
      if (dbits(tn) > tend_bits) {
        status = RT_TRAJ_TEND;
        run = false;
      } else if (ev == A.max_events) {
        status = RT_TRAJ_MAX_EVENTS;
        run = false;
      }
    }
    // ---- the int32 range of the fired reaction's net change
    int vb = 0, ve = 0;
    if (run) {
      vb = net.vp[mu];
      ve = net.vp[mu + 1];
    }
    bool over = false;
    for (int i = vb + sl; i < ve; i += G) {
      const int2 e = net.vl[i];
      const long long nx = (long long)X[e.x] + e.y;
      over |= (nx > INT_MAX) | (nx < 0);
    }
    if ((__ballot_sync(FULL, over) & segmask) != 0) {
      status = RT_TRAJ_OVERFLOW;
      run = false;
      ve = vb;
    }
    // ---- fire (segments still running)
    if (run) {
      while (gi < A.G && dbits(next_g) < dbits(tn)) {
        record(gi, true);
        ++gi;
        next_g = __dmul_rn(__ll2double_rn(gi), A.sample_dt);
      }
      t = tn;
      if (sl == 0) trace_event(A.out, j, ev, mu, tn);
    }
    const int lmu = base + (mu & (G - 1)), rm = mu / G;  // owner lane and slot of mu
    if (LL) {
      const double amu = __shfl_sync(FULL, pick<R>(a, rm), lmu);
      if (run && sl == (ev & (G - 1))) ring = amu;
    }
    // the fired channel's increment: if it is used up, redraw every used-up one of the warp
    const uint32_t stale_mu = __shfl_sync(FULL, stale, lmu);
    const bool need_draw = run && rm < R && ((stale_mu >> rm) & 1u);
    if (__any_sync(FULL, need_draw)) {
      uint32_t pend = stale;
      while (__any_sync(FULL, pend != 0)) {
        if (pend) {
          const int r = __ffs(pend) - 1;
          const int k = sl + G * r;
          const double E = exp1_draw(A.seed, g, (uint32_t)k, (uint32_t)(pick<R>(n, r) + 1), A.stream_id);
#pragma unroll
          for (int q = 0; q < R; ++q)
            if (q == r) En[q] = E;
          pend &= pend - 1;
        }
      }
      stale = 0;
    }
    __syncwarp();
    if (run) {
      for (int i = vb + sl; i < ve; i += G) {
        const int2 e = net.vl[i];
        X[e.x] += e.y;
      }
      if (lane == lmu) {
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (r == rm) {
            n[r] += 1;
            P[r] = __dadd_rn(P[r], En[r]);  // Eq. 27
          }
        stale |= 1u << rm;
      }
      ++ev;
      dprev = dmin;
      mu_prev = mu;
    }
    __syncwarp();
    if (LL) {
      const int cnt = (run && (ev & (G - 1)) == 0) ? G : 0;
      if (__any_sync(FULL, cnt != 0)) flush_ring(cnt);
    }
  }
  if (LL) flush_ring(live ? (ev & (G - 1)) : 0);

  const bool known = status == RT_TRAJ_TEND || status == RT_TRAJ_ABSORBED;
  if (A.out.loglik_dev || A.out.t_internal_dev) {
    if (live && known && tend_finite && !bad) {
      const double rest = __dsub_rn(A.t_end, t);
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (sl + G * r < M) T[r] = __dadd_rn(T[r], __dmul_rn(a[r], rest));
    }
    if (A.out.loglik_dev) {
      const double sT = warp_sum_T_in_order<R, G>(T, M, live);  // every lane takes part
      if (live && sl == 0) A.out.loglik_dev[j] = bad ? __longlong_as_double(0x7FF8000000000000ll) : __dsub_rn(ll, sT);
    }
    if (live && A.out.t_internal_dev)
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (sl + G * r < M) A.out.t_internal_dev[j * M + sl + G * r] = T[r];
  }
  if (!live) return;
  for (; gi < A.G; ++gi) record(gi, known);
  trace_tail(A.out, j, ev, sl, G);
  if (A.out.counts_dev)
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (sl + G * r < M) A.out.counts_dev[j * M + sl + G * r] = n[r];
  if (A.out.x_final_dev)
    for (int s = sl; s < N; s += G) A.out.x_final_dev[j * N + s] = X[s];
  if (sl == 0) {
    if (A.out.n_events_dev) A.out.n_events_dev[j] = ev;
    if (A.out.status_dev) A.out.status_dev[j] = status;
    if (A.out.t_last_dev) A.out.t_last_dev[j] = t;
  }
}

}  // namespace rt

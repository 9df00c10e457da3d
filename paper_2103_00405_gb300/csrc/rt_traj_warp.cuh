// rt_traj_warp.cuh -- one warp per trajectory (channel k in lane k % 32, slot k / 32).
//
// The NRRTA loop of Table 2 (Liu & Wang, arXiv:2103.00405) with channel k held by
// lane k % 32 in register slot k / 32 (P_k, T_k, a_k, n_k; Eq. 17-27).  Per event
// every lane advances its internal times with the pre-event propensities and
// recomputes the ones the last firing changed (a per-lane dependency byte per
// reaction), then the warp picks the channel with the smallest certified float
// upper bound of its waiting time, computes that one exactly, broadcasts it, and
// every lane computes exactly only channels that are not certified to be larger.
// A shuffle reduction on (waiting time bits, channel) gives the exact argmin with
// the smallest index on ties (Eq. 25-26).  The network arrays may live in shared
// or global memory (generic pointers); X is per warp in shared memory.
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
  const uint8_t *dep;  // [M][32]
};

template <int R, bool LL>
__device__ __forceinline__ void warp_trajectory(const RunArgs &A, const WarpNet &net, int *X, unsigned long long *mom,
                                const int64_t j, const int tend_finite) {
  const int lane = threadIdx.x & 31;
  const int M = net.M, N = net.N;
  const uint64_t g = (uint64_t)(A.traj_offset + j);
  const int32_t *x0 = A.x0 + (A.per_traj_x0 ? j * (int64_t)N : 0);
  bool bad = false;
  for (int s = lane; s < N; s += 32) {
    const int v = x0[s];
    X[s] = v;
    bad |= v < 0;
  }
  bad = __any_sync(0xFFFFFFFFu, bad);
  __syncwarp();
  auto xat = [&](int s) { return X[s]; };
  const int64_t GN = A.G * N;

  auto record = [&](int64_t gidx, bool known) {
    if (A.out.grid_dev) {
      int32_t *gp = A.out.grid_dev + (j * A.G + gidx) * N;
      for (int s = lane; s < N; s += 32) gp[s] = known ? X[s] : -1;
    }
    if (!known || !A.out.grid_sum_dev) return;
    for (int s = lane; s < N; s += 32) {
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
    if (lane == 0) {
      if (mom) atomicAdd(mom + 2 * GN + gidx, 1ull);
      else if (A.out.grid_count_dev) atomicAdd((unsigned long long *)(A.out.grid_count_dev + gidx), 1ull);
    }
  };

  double P[R], T[R], a[R];
  int32_t n[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int k = lane + 32 * r;
    P[r] = 0.0;
    T[r] = 0.0;
    a[r] = 0.0;
    n[r] = 0;
    if (!bad && k < M) {
      P[r] = exp1_draw(A.seed, g, (uint32_t)k, 0u, A.stream_id);
      a[r] = propensity<false>(net.rd[k], net.c[k], xat);
    }
  }
  int status = bad ? RT_TRAJ_BAD_X0 : RT_TRAJ_TEND;
  double t = 0.0, ll = 0.0, dprev = 0.0;
  int mu_prev = -1;
  int32_t ev = 0;
  int64_t gi = 0;
  double next_g = 0.0;
  const int64_t tend_bits = dbits(A.t_end);

  if (!bad) {
    for (;;) {
      // internal times advance with the pre-event propensities (Eq. 17), then the
      // propensities the last firing changed are recomputed (Eq. 1-2)
      const uint32_t dep = mu_prev >= 0 ? net.dep[mu_prev * 32 + lane] : 0u;
      const bool adv = dbits(dprev) != 0;
      float ub = __int_as_float(0x7F800000);
      int kub = INT_MAX;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int k = lane + 32 * r;
        if (k < M) {
          if (adv && dbits(a[r]) != 0) T[r] = __dadd_rn(T[r], __dmul_rn(a[r], dprev));
          if ((dep >> r) & 1u) a[r] = propensity<false>(net.rd[k], net.c[k], xat);
          if (dbits(a[r]) != 0) {
            const float u = wait_estimate(P[r], T[r], a[r]);
            if (u < ub || kub == INT_MAX) {
              ub = u;
              kub = k;
            }
          }
        }
      }
      // candidate: smallest upper bound over the warp
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float u2 = __shfl_xor_sync(0xFFFFFFFFu, ub, o);
        const int k2 = __shfl_xor_sync(0xFFFFFFFFu, kub, o);
        if (u2 < ub || (u2 == ub && k2 < kub)) {
          ub = u2;
          kub = k2;
        }
      }
      if (kub == INT_MAX) {
        status = RT_TRAJ_ABSORBED;
        break;
      }
      // its exact waiting time, computed by the owning lane and broadcast
      long long wc = 0;
      if (lane == (kub & 31)) {
        const int rs = kub >> 5;
        wc = dbits(waiting_time(pick<R>(P, rs), pick<R>(T, rs), pick<R>(a, rs)));
      }
      wc = __shfl_sync(0xFFFFFFFFu, wc, kub & 31);
      const float thr = f32_upper(bitsd(wc));
      long long bw = wc;
      int bk = kub;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int k = lane + 32 * r;
        if (k < M && k != kub && dbits(a[r]) != 0 && !exceeds(P[r], T[r], a[r], thr)) {
          const long long wb = dbits(waiting_time(P[r], T[r], a[r]));
          if (wb < bw || (wb == bw && k < bk)) {
            bw = wb;
            bk = k;
          }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const long long w2 = __shfl_xor_sync(0xFFFFFFFFu, bw, o);
        const int k2 = __shfl_xor_sync(0xFFFFFFFFu, bk, o);
        if (w2 < bw || (w2 == bw && k2 < bk)) {
          bw = w2;
          bk = k2;
        }
      }
      const int mu = bk;
      const double dmin = bitsd(bw);
      const double tn = __dadd_rn(t, dmin);
      if (dbits(tn) > tend_bits) {
        status = RT_TRAJ_TEND;
        break;
      }
      if (ev == A.max_events) {
        status = RT_TRAJ_MAX_EVENTS;
        break;
      }
      const int vb = net.vp[mu], ve = net.vp[mu + 1];
      bool over = false;
      for (int i = vb + lane; i < ve; i += 32) {
        const int2 e = net.vl[i];
        const long long nx = (long long)X[e.x] + e.y;
        over |= (nx > INT_MAX) | (nx < 0);
      }
      if (__any_sync(0xFFFFFFFFu, over)) {
        status = RT_TRAJ_OVERFLOW;
        break;
      }
      while (gi < A.G && dbits(next_g) < dbits(tn)) {
        record(gi, true);
        ++gi;
        next_g = __dmul_rn(__ll2double_rn(gi), A.sample_dt);
      }
      t = tn;
      if (lane == 0) trace_event(A.out, j, ev, mu, tn);
      // The fired channel's new Exp(1) increment (Eq. 27) is -ln u and, with the
      // likelihood, ln a_mu is needed too: the owner lane and its neighbour prepare
      // their arguments, then run one fixed-point logarithm side by side.
      const int lmu = mu & 31, rm = mu >> 5, lll = lmu ^ 1;
      const double amu = LL ? __shfl_sync(0xFFFFFFFFu, pick<R>(a, rm), lmu) : 0.0;
      uint64_t lm = 1;
      int le = 0;
      int32_t nm = 0;
      if (lane == lmu) {
        nm = pick<R>(n, rm) + 1;
        lm = bits_to_x(draw_bits(A.seed, g, (uint32_t)mu, (uint32_t)nm, A.stream_id));
        le = -53;
      } else if (LL && lane == lll) {
        const uint64_t b = (uint64_t)__double_as_longlong(amu);
        const int ef = (int)((b >> 52) & 0x7FF);
        const uint64_t frac = b & 0x000FFFFFFFFFFFFFull;
        lm = ef == 0 ? frac : (frac | (1ull << 52));
        le = ef == 0 ? -1074 : ef - 1075;
      }
      double L = 0.0;
      if (lane == lmu || (LL && lane == lll)) L = fx_ln(lm, le);
      if (LL) {
        const double lv = __shfl_sync(0xFFFFFFFFu, L, lll);
        if (lane == 0) ll = __dadd_rn(ll, lv);
      }
      __syncwarp();
      for (int i = vb + lane; i < ve; i += 32) {
        const int2 e = net.vl[i];
        X[e.x] += e.y;
      }
      if (lane == lmu) {
        const double E = -L;
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (r == rm) {
            n[r] = nm;
            P[r] = __dadd_rn(P[r], E);
          }
      }
      __syncwarp();
      ++ev;
      dprev = dmin;
      mu_prev = mu;
    }
  }

  const bool known = status == RT_TRAJ_TEND || status == RT_TRAJ_ABSORBED;
  for (; gi < A.G; ++gi) record(gi, known);
  if (A.out.loglik_dev || A.out.t_internal_dev) {
    if (known && tend_finite && !bad) {
      const double rest = __dsub_rn(A.t_end, t);
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (lane + 32 * r < M) T[r] = __dadd_rn(T[r], __dmul_rn(a[r], rest));
    }
    if (A.out.t_internal_dev)
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (lane + 32 * r < M) A.out.t_internal_dev[j * M + lane + 32 * r] = T[r];
    if (A.out.loglik_dev) {
      double sT = 0.0;  // sum_k T_k in k order (lane 0 accumulates)
#pragma unroll
      for (int r = 0; r < R; ++r)
        for (int l = 0; l < 32; ++l) {
          const double v = __shfl_sync(0xFFFFFFFFu, T[r], l);
          if (l + 32 * r < M) sT = __dadd_rn(sT, v);
        }
      if (lane == 0) A.out.loglik_dev[j] = bad ? __longlong_as_double(0x7FF8000000000000ll) : __dsub_rn(ll, sT);
    }
  }
  if (A.out.counts_dev)
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (lane + 32 * r < M) A.out.counts_dev[j * M + lane + 32 * r] = n[r];
  if (A.out.x_final_dev)
    for (int s = lane; s < N; s += 32) A.out.x_final_dev[j * N + s] = X[s];
  trace_tail(A.out, j, ev, lane, 32);
  if (lane == 0) {
    if (A.out.n_events_dev) A.out.n_events_dev[j] = ev;
    if (A.out.status_dev) A.out.status_dev[j] = status;
    if (A.out.t_last_dev) A.out.t_last_dev[j] = t;
  }
}

// network tables in shared memory: c, rd, vl, vp, dep (rounded to 16 bytes)
}  // namespace rt

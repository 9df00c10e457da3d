// rt_traj_thread.cuh -- one thread per trajectory, state in registers.
//
// The NRRTA loop of Table 2 (Liu & Wang, arXiv:2103.00405) in internal-time form:
// a thread keeps its trajectory's P_k, T_k and a_k (Eq. 17-25) for all M <= 16
// channels in registers and its counts X in shared memory (a column per thread,
// X[s] at X[s * B], so accesses are bank-conflict free).  The network tables
// (reactant descriptors, rates, net changes, per-reaction dependency masks) are
// reached through generic pointers: shared memory in the single-network kernel,
// global memory in the batched kernel.
#pragma once
#include <climits>

#include "rt_moments.cuh"
#include "rt_sim.cuh"

namespace rt {

struct ThreadNet {
  double *c;
  uint64_t *dep;
  int2 *rd;
  int2 *vl;
  int *vp;
  int *X;
  unsigned long long *mom;  // start of the moment table share in shared memory
  MomTable mt;              // the share (smem_mom != 0)
};

// Lays the single-network kernel's shared memory out: c, dep, rd, vl, vp, X, moments.
__device__ __forceinline__ ThreadNet carve_thread_net(unsigned char *base, int M, int nv, int N, int B) {
  ThreadNet s;
  s.c = (double *)base;
  s.dep = (uint64_t *)(s.c + M);
  s.rd = (int2 *)(s.dep + M);
  s.vl = s.rd + M;
  s.vp = (int *)(s.vl + nv);
  s.X = s.vp + (M + 1);
  // per-block moment table (8-byte aligned): sum[G][N], sumsq[G][N], count[G]
  const size_t off = ((size_t)((unsigned char *)(s.X + (size_t)N * B) - base) + 7) & ~(size_t)7;
  s.mom = (unsigned long long *)(base + off);
  return s;
}


// MAXM: register slots; EXACT: the network has exactly MAXM reactions (loops fully resolved).
template <int MAXM, bool LL, bool EXACT = false>
__device__ __forceinline__ void simulate_one(const RunArgs &A, const ThreadNet &S, const int64_t j, const int B,
                                             const int tend_finite, const int smem_mom) {
  const int M = EXACT ? MAXM : A.net.M, N = A.net.N;
  int *X = S.X + threadIdx.x;  // X[s] lives at X[s * B]
  auto xat = [&](int s) { return X[s * B]; };
  const uint64_t g = (uint64_t)(A.traj_offset + j);
  const int32_t *x0 = A.x0 + (A.per_traj_x0 ? j * (int64_t)N : 0);
  bool bad = false;
  for (int s = 0; s < N; ++s) {
    const int v = x0[s];
    X[s * B] = v;
    bad |= v < 0;
  }

  double P[MAXM], T[MAXM], a[MAXM];
  int32_t n[MAXM];
  int status = RT_TRAJ_TEND;
  double t = 0.0, ll = 0.0;
  int32_t ev = 0;
  int64_t gi = 0;
  double next_g = 0.0;  // time of grid point gi

  // grid sampling: X at grid time gi (right-continuous: events at times <= g included)
  auto record = [&](int64_t gidx) {
    if (A.out.grid_dev) {
      int32_t *gp = A.out.grid_dev + (j * A.G + gidx) * N;
      for (int s = 0; s < N; ++s) gp[s] = X[s * B];
    }
    if (smem_mom) {
      mom_add(S.mt, gidx, N, xat);
    } else if (A.out.grid_sum_dev) {
      for (int s = 0; s < N; ++s) {
        const long long x = X[s * B];
        atomicAdd((unsigned long long *)(A.out.grid_sum_dev + gidx * N + s), (unsigned long long)x);
        if (A.out.grid_sumsq_dev)
          atomicAdd((unsigned long long *)(A.out.grid_sumsq_dev + gidx * N + s), (unsigned long long)(x * x));
      }
      if (A.out.grid_count_dev) atomicAdd((unsigned long long *)(A.out.grid_count_dev + gidx), 1ull);
    }
  };

#pragma unroll
  for (int k = 0; k < MAXM; ++k) {
    n[k] = 0;
    T[k] = 0.0;
    P[k] = 0.0;
    a[k] = 0.0;
  }
  if (bad) {
    status = RT_TRAJ_BAD_X0;
  } else {
    // initialise (Table 2): first Exp(1) increment per channel, propensities of X(0)
#pragma unroll
    for (int k = 0; k < MAXM; ++k)
      if (k < M) {
        P[k] = exp1_draw(A.seed, g, (uint32_t)k, 0u, A.stream_id);
        a[k] = propensity(S.rd[k], S.c[k], xat);
      }
    const int64_t tend_bits = dbits(A.t_end);
    for (;;) {
      // Eq. 25-26: waiting times and the first channel to fire (smallest k on ties).
      // One exact subtraction per channel; float bounds from its result pick a
      // candidate whose exact quotient is computed; every other channel is either
      // certified to be strictly larger or computed exactly as well.
      double rem[MAXM];
      float ub_min = __int_as_float(0x7F800000);
      int ks = -1;
#pragma unroll
      for (int k = 0; k < MAXM; ++k) {
        rem[k] = 0.0;
        if (k < M && dbits(a[k]) != 0) {
          rem[k] = __dsub_rn(P[k], T[k]);
          const float ub = dbits(rem[k]) > 0 ? quot_estimate(rem[k], a[k]) : 0.0f;
          if (ks < 0 || ub < ub_min) {
            ub_min = ub;
            ks = k;
          }
        }
      }
      int64_t best = kInfBits;
      int mu = -1;
      if (ks >= 0) {
        double rks = 0.0, aks = 1.0;
#pragma unroll
        for (int k = 0; k < MAXM; ++k)
          if (k == ks) {
            rks = rem[k];
            aks = a[k];
          }
        best = dbits(waiting_time_rem(rks, aks));
        mu = ks;
        const float thr = f32_upper(bitsd(best));
#pragma unroll
        for (int k = 0; k < MAXM; ++k)
          if (k < M && k != ks && dbits(a[k]) != 0) {
            if (dbits(rem[k]) > 0 && quot_exceeds(rem[k], a[k], thr)) continue;
            const int64_t wb = dbits(waiting_time_rem(rem[k], a[k]));
            if (wb < best || (wb == best && k < mu)) {
              best = wb;
              mu = k;
            }
          }
      }
      if (mu < 0) {
        status = RT_TRAJ_ABSORBED;
        break;
      }
      const double dmin = bitsd(best);
      const double tn = __dadd_rn(t, dmin);
      if (dbits(tn) > tend_bits) {
        status = RT_TRAJ_TEND;
        break;
      }
      if (ev == A.max_events) {
        status = RT_TRAJ_MAX_EVENTS;
        break;
      }
      const int vb = S.vp[mu], ve = S.vp[mu + 1];
      bool over = false;
      for (int i = vb; i < ve; ++i) {
        const int2 e = S.vl[i];
        const long long nx = (long long)X[e.x * B] + e.y;
        over |= (nx > INT_MAX) | (nx < 0);
      }
      if (over) {
        status = RT_TRAJ_OVERFLOW;
        break;
      }
      while (gi < A.G && dbits(next_g) < dbits(tn)) {
        record(gi);
        ++gi;
        next_g = __dmul_rn(__ll2double_rn(gi), A.sample_dt);
      }
      t = tn;
      trace_event(A.out, j, ev, mu, tn);
      // every internal time advances by a_k dt (Eq. 17)
      double a_mu = 0.0;
#pragma unroll
      for (int k = 0; k < MAXM; ++k)
        if (k < M) {
          if (k == mu) a_mu = a[k];
          T[k] = __dadd_rn(T[k], __dmul_rn(a[k], dmin));
        }
      if (LL) ll = __dadd_rn(ll, rt_ln(a_mu));
      for (int i = vb; i < ve; ++i) {
        const int2 e = S.vl[i];
        X[e.x * B] += e.y;
      }
      int32_t nmu = 0;
#pragma unroll
      for (int k = 0; k < MAXM; ++k)
        if (k == mu) {
          n[k] += 1;
          nmu = n[k];
        }
      ++ev;
      // Eq. 27: only the fired channel draws a new increment
      const double E = exp1_draw(A.seed, g, (uint32_t)mu, (uint32_t)nmu, A.stream_id);
      const uint64_t dm = S.dep[mu];
#pragma unroll
      for (int k = 0; k < MAXM; ++k)
        if (k < M) {
          if (k == mu) P[k] = __dadd_rn(P[k], E);
          if ((dm >> k) & 1ull) a[k] = propensity(S.rd[k], S.c[k], xat);
        }
    }
  }

  const bool known = status == RT_TRAJ_TEND || status == RT_TRAJ_ABSORBED;
  for (; gi < A.G; ++gi) {
    if (known) {
      record(gi);
    } else if (A.out.grid_dev) {
      int32_t *gp = A.out.grid_dev + (j * A.G + gi) * N;
      for (int s = 0; s < N; ++s) gp[s] = -1;
    }
  }
  if (A.out.loglik_dev || A.out.t_internal_dev) {
    if (known && tend_finite) {
      const double rest = __dsub_rn(A.t_end, t);
#pragma unroll
      for (int k = 0; k < MAXM; ++k)
        if (k < M) T[k] = __dadd_rn(T[k], __dmul_rn(a[k], rest));
    }
    if (A.out.t_internal_dev)
#pragma unroll
      for (int k = 0; k < MAXM; ++k)
        if (k < M) A.out.t_internal_dev[j * M + k] = T[k];
    if (A.out.loglik_dev) {
      double sT = 0.0;
#pragma unroll
      for (int k = 0; k < MAXM; ++k)
        if (k < M) sT = __dadd_rn(sT, T[k]);
      A.out.loglik_dev[j] = status == RT_TRAJ_BAD_X0 ? __longlong_as_double(0x7FF8000000000000ll) : __dsub_rn(ll, sT);
    }
  }
  if (A.out.counts_dev)
#pragma unroll
    for (int k = 0; k < MAXM; ++k)
      if (k < M) A.out.counts_dev[j * M + k] = n[k];
  if (A.out.x_final_dev)
    for (int s = 0; s < N; ++s) A.out.x_final_dev[j * N + s] = X[s * B];
  trace_tail(A.out, j, ev, 0, 1);
  if (A.out.n_events_dev) A.out.n_events_dev[j] = ev;
  if (A.out.status_dev) A.out.status_dev[j] = status;
  if (A.out.t_last_dev) A.out.t_last_dev[j] = t;
}

// Table 3's form of the method ("parallel NRRTA", Sec. 5): each channel keeps its relative
// waiting time w_k; after an event that took dt every propensity is recomputed (no
// dependency graph) and every other channel's waiting time is rescaled,
// w_k = (p_k / a_k) (w_k - dt) with p_k the propensity w_k was computed with (the previous
// a_k); the fired channel draws w_mu = E / a_mu.  A channel whose propensity is 0 keeps its
// remaining internal time p_k (w_k - dt) frozen in its w_k slot until it can fire again
// (w_k = q_k / a_k).  Internal times for the likelihood accumulate T_k += a_k dt.  The same
// process and the same random numbers as Table 2's internal-time form; the roundings differ.
template <int MAXM, bool LL, bool EXACT = false>
__device__ __forceinline__ void simulate_rescaled(const RunArgs &A, const ThreadNet &S, const int64_t j, const int B,
                                                  const int tend_finite, const int smem_mom, const int want_T) {
  const int M = EXACT ? MAXM : A.net.M, N = A.net.N;
  int *X = S.X + threadIdx.x;  // X[s] lives at X[s * B]
  auto xat = [&](int s) { return X[s * B]; };
  const uint64_t g = (uint64_t)(A.traj_offset + j);
  const int32_t *x0 = A.x0 + (A.per_traj_x0 ? j * (int64_t)N : 0);
  bool bad = false;
  for (int s = 0; s < N; ++s) {
    const int v = x0[s];
    X[s * B] = v;
    bad |= v < 0;
  }
  double w[MAXM], T[MAXM], a[MAXM];
  int32_t n[MAXM];
  int status = RT_TRAJ_TEND;
  double t = 0.0, ll = 0.0;
  int32_t ev = 0;
  int64_t gi = 0;
  double next_g = 0.0;
  auto record = [&](int64_t gidx) {
    if (A.out.grid_dev) {
      int32_t *gp = A.out.grid_dev + (j * A.G + gidx) * N;
      for (int s = 0; s < N; ++s) gp[s] = X[s * B];
    }
    if (smem_mom) {
      mom_add(S.mt, gidx, N, xat);
    } else if (A.out.grid_sum_dev) {
      for (int s = 0; s < N; ++s) {
        const long long x = X[s * B];
        atomicAdd((unsigned long long *)(A.out.grid_sum_dev + gidx * N + s), (unsigned long long)x);
        if (A.out.grid_sumsq_dev)
          atomicAdd((unsigned long long *)(A.out.grid_sumsq_dev + gidx * N + s), (unsigned long long)(x * x));
      }
      if (A.out.grid_count_dev) atomicAdd((unsigned long long *)(A.out.grid_count_dev + gidx), 1ull);
    }
  };
#pragma unroll
  for (int k = 0; k < MAXM; ++k) {
    n[k] = 0;
    T[k] = 0.0;
    w[k] = 0.0;
    a[k] = 0.0;
  }
  if (bad) {
    status = RT_TRAJ_BAD_X0;
  } else {
    // initialise: a_k, w_k = ln(1/r_k) / a_k (p_k = a_k)
#pragma unroll
    for (int k = 0; k < MAXM; ++k)
      if (k < M) {
        const double E = exp1_draw(A.seed, g, (uint32_t)k, 0u, A.stream_id);
        a[k] = propensity(S.rd[k], S.c[k], xat);
        w[k] = dbits(a[k]) != 0 ? __ddiv_rn(E, a[k]) : E;  // frozen: the remaining internal time
      }
    const int64_t tend_bits = dbits(A.t_end);
    for (;;) {
      // scan for the smallest waiting time (ties: smallest index); frozen channels cannot fire
      int64_t best = kInfBits;
      int mu = -1;
#pragma unroll
      for (int k = 0; k < MAXM; ++k)
        if (k < M && dbits(a[k]) != 0 && dbits(w[k]) < best) {
          best = dbits(w[k]);
          mu = k;
        }
      if (mu < 0) {
        status = RT_TRAJ_ABSORBED;
        break;
      }
      const double dmin = bitsd(best);
      const double tn = __dadd_rn(t, dmin);
      if (dbits(tn) > tend_bits) {
        status = RT_TRAJ_TEND;
        break;
      }
      if (ev == A.max_events) {
        status = RT_TRAJ_MAX_EVENTS;
        break;
      }
      const int vb = S.vp[mu], ve = S.vp[mu + 1];
      bool over = false;
      for (int i = vb; i < ve; ++i) {
        const int2 e = S.vl[i];
        const long long nx = (long long)X[e.x * B] + e.y;
        over |= (nx > INT_MAX) | (nx < 0);
      }
      if (over) {
        status = RT_TRAJ_OVERFLOW;
        break;
      }
      while (gi < A.G && dbits(next_g) < dbits(tn)) {
        record(gi);
        ++gi;
        next_g = __dmul_rn(__ll2double_rn(gi), A.sample_dt);
      }
      t = tn;
      trace_event(A.out, j, ev, mu, tn);
      double a_mu = 0.0;
#pragma unroll
      for (int k = 0; k < MAXM; ++k)
        if (k < M) {
          if (k == mu) a_mu = a[k];
          if (want_T) T[k] = __dadd_rn(T[k], __dmul_rn(a[k], dmin));
        }
      if (LL) ll = __dadd_rn(ll, rt_ln(a_mu));
      for (int i = vb; i < ve; ++i) {
        const int2 e = S.vl[i];
        X[e.x * B] += e.y;
      }
      int32_t nmu = 0;
#pragma unroll
      for (int k = 0; k < MAXM; ++k)
        if (k == mu) {
          n[k] += 1;
          nmu = n[k];
        }
      ++ev;
      const double E = exp1_draw(A.seed, g, (uint32_t)mu, (uint32_t)nmu, A.stream_id);
      // recalculate every propensity; rescale every other waiting time; the fired one redraws
#pragma unroll
      for (int k = 0; k < MAXM; ++k)
        if (k < M) {
          const double an = propensity(S.rd[k], S.c[k], xat);
          if (k == mu) {
            w[k] = dbits(an) != 0 ? __ddiv_rn(E, an) : E;
          } else if (dbits(a[k]) != 0) {
            const double rem = __dsub_rn(w[k], dmin);
            w[k] = dbits(an) != 0 ? __dmul_rn(__ddiv_rn(a[k], an), rem) : __dmul_rn(a[k], rem);
          } else if (dbits(an) != 0) {
            w[k] = __ddiv_rn(w[k], an);  // a frozen channel resumes
          }
          a[k] = an;
        }
    }
  }
  const bool known = status == RT_TRAJ_TEND || status == RT_TRAJ_ABSORBED;
  for (; gi < A.G; ++gi) {
    if (known) {
      record(gi);
    } else if (A.out.grid_dev) {
      int32_t *gp = A.out.grid_dev + (j * A.G + gi) * N;
      for (int s = 0; s < N; ++s) gp[s] = -1;
    }
  }
  if (want_T) {
    if (known && tend_finite && status != RT_TRAJ_BAD_X0) {
      const double rest = __dsub_rn(A.t_end, t);
#pragma unroll
      for (int k = 0; k < MAXM; ++k)
        if (k < M) T[k] = __dadd_rn(T[k], __dmul_rn(a[k], rest));
    }
    if (A.out.t_internal_dev)
#pragma unroll
      for (int k = 0; k < MAXM; ++k)
        if (k < M) A.out.t_internal_dev[j * M + k] = T[k];
    if (A.out.loglik_dev) {
      double sT = 0.0;
#pragma unroll
      for (int k = 0; k < MAXM; ++k)
        if (k < M) sT = __dadd_rn(sT, T[k]);
      A.out.loglik_dev[j] = status == RT_TRAJ_BAD_X0 ? __longlong_as_double(0x7FF8000000000000ll) : __dsub_rn(ll, sT);
    }
  }
  if (A.out.counts_dev)
#pragma unroll
    for (int k = 0; k < MAXM; ++k)
      if (k < M) A.out.counts_dev[j * M + k] = n[k];
  if (A.out.x_final_dev)
    for (int s = 0; s < N; ++s) A.out.x_final_dev[j * N + s] = X[s * B];
  trace_tail(A.out, j, ev, 0, 1);
  if (A.out.n_events_dev) A.out.n_events_dev[j] = ev;
  if (A.out.status_dev) A.out.status_dev[j] = status;
  if (A.out.t_last_dev) A.out.t_last_dev[j] = t;
}

// ---------------------------------------------------------------------------------
// Time-dependent rates c_k(t) = c_k (1 + beta_k t) (Sec. 6, Eq. 29): with A_k = c_k h_k(X)
// constant between events, channel k's internal time over [t, t + d] grows by
// A_k I_k(t, d), I_k = d (1 + beta_k t) + beta_k d^2 / 2, and its waiting time solves
// A_k I_k(t, d) = P_k - T_k, written without cancellation.  beta_k = 0 runs exactly the
// constant-rate operations.
// ---------------------------------------------------------------------------------
template <int MAXM, bool LL>
__device__ __forceinline__ void simulate_tdep(const RunArgs &A, const ThreadNet &S, const double *beta, const int64_t j,
                                              const int B, const int tend_finite, const int smem_mom) {
  const int M = A.net.M, N = A.net.N;
  int *X = S.X + threadIdx.x;  // X[s] lives at X[s * B]
  auto xat = [&](int s) { return X[s * B]; };
  const uint64_t g = (uint64_t)(A.traj_offset + j);
  const int32_t *x0 = A.x0 + (A.per_traj_x0 ? j * (int64_t)N : 0);
  bool bad = false;
  for (int s = 0; s < N; ++s) {
    const int v = x0[s];
    X[s * B] = v;
    bad |= v < 0;
  }
  double P[MAXM], T[MAXM], a[MAXM], bt[MAXM];
  int32_t n[MAXM];
  int status = RT_TRAJ_TEND;
  double t = 0.0, ll = 0.0;
  int32_t ev = 0;
  int64_t gi = 0;
  double next_g = 0.0;
  auto record = [&](int64_t gidx) {
    if (A.out.grid_dev) {
      int32_t *gp = A.out.grid_dev + (j * A.G + gidx) * N;
      for (int s = 0; s < N; ++s) gp[s] = X[s * B];
    }
    if (smem_mom) {
      mom_add(S.mt, gidx, N, xat);
    } else if (A.out.grid_sum_dev) {
      for (int s = 0; s < N; ++s) {
        const long long x = X[s * B];
        atomicAdd((unsigned long long *)(A.out.grid_sum_dev + gidx * N + s), (unsigned long long)x);
        if (A.out.grid_sumsq_dev)
          atomicAdd((unsigned long long *)(A.out.grid_sumsq_dev + gidx * N + s), (unsigned long long)(x * x));
      }
      if (A.out.grid_count_dev) atomicAdd((unsigned long long *)(A.out.grid_count_dev + gidx), 1ull);
    }
  };
#pragma unroll
  for (int k = 0; k < MAXM; ++k) {
    n[k] = 0;
    T[k] = 0.0;
    P[k] = 0.0;
    a[k] = 0.0;
    bt[k] = k < M ? beta[k] : 0.0;
  }
  if (bad) {
    status = RT_TRAJ_BAD_X0;
  } else {
#pragma unroll
    for (int k = 0; k < MAXM; ++k)
      if (k < M) {
        P[k] = exp1_draw(A.seed, g, (uint32_t)k, 0u, A.stream_id);
        a[k] = propensity(S.rd[k], S.c[k], xat);
      }
    const int64_t tend_bits = dbits(A.t_end);
    for (;;) {
      // every channel's waiting time from its own integral (Eq. 29); smallest index on ties
      int64_t best = kInfBits;
      int mu = -1;
#pragma unroll
      for (int k = 0; k < MAXM; ++k)
        if (k < M && dbits(a[k]) != 0) {
          const int64_t wb = dbits(tdep_wait(a[k], bt[k], __dsub_rn(P[k], T[k]), t));
          if (wb < best) {
            best = wb;
            mu = k;
          }
        }
      if (mu < 0) {
        status = RT_TRAJ_ABSORBED;
        break;
      }
      const double dmin = bitsd(best);
      const double tn = __dadd_rn(t, dmin);
      if (dbits(tn) > tend_bits) {
        status = RT_TRAJ_TEND;
        break;
      }
      if (ev == A.max_events) {
        status = RT_TRAJ_MAX_EVENTS;
        break;
      }
      const int vb = S.vp[mu], ve = S.vp[mu + 1];
      bool over = false;
      for (int i = vb; i < ve; ++i) {
        const int2 e = S.vl[i];
        const long long nx = (long long)X[e.x * B] + e.y;
        over |= (nx > INT_MAX) | (nx < 0);
      }
      if (over) {
        status = RT_TRAJ_OVERFLOW;
        break;
      }
      while (gi < A.G && dbits(next_g) < dbits(tn)) {
        record(gi);
        ++gi;
        next_g = __dmul_rn(__ll2double_rn(gi), A.sample_dt);
      }
      const double tprev = t;
      t = tn;
      trace_event(A.out, j, ev, mu, tn);
      double a_mu = 0.0, b_mu = 0.0;
#pragma unroll
      for (int k = 0; k < MAXM; ++k)
        if (k < M) {
          if (k == mu) {
            a_mu = a[k];
            b_mu = bt[k];
          }
          T[k] = __dadd_rn(T[k], __dmul_rn(a[k], tdep_integral(bt[k], tprev, dmin)));
        }
      if (LL) ll = __dadd_rn(ll, rt_ln(__dmul_rn(a_mu, __dadd_rn(1.0, __dmul_rn(b_mu, t)))));
      for (int i = vb; i < ve; ++i) {
        const int2 e = S.vl[i];
        X[e.x * B] += e.y;
      }
      int32_t nmu = 0;
#pragma unroll
      for (int k = 0; k < MAXM; ++k)
        if (k == mu) {
          n[k] += 1;
          nmu = n[k];
        }
      ++ev;
      const double E = exp1_draw(A.seed, g, (uint32_t)mu, (uint32_t)nmu, A.stream_id);
      const uint64_t dm = S.dep[mu];
#pragma unroll
      for (int k = 0; k < MAXM; ++k)
        if (k < M) {
          if (k == mu) P[k] = __dadd_rn(P[k], E);
          if ((dm >> k) & 1ull) a[k] = propensity(S.rd[k], S.c[k], xat);
        }
    }
  }
  const bool known = status == RT_TRAJ_TEND || status == RT_TRAJ_ABSORBED;
  for (; gi < A.G; ++gi) {
    if (known) {
      record(gi);
    } else if (A.out.grid_dev) {
      int32_t *gp = A.out.grid_dev + (j * A.G + gi) * N;
      for (int s = 0; s < N; ++s) gp[s] = -1;
    }
  }
  if (A.out.loglik_dev || A.out.t_internal_dev) {
    if (known && tend_finite && status != RT_TRAJ_BAD_X0) {
      const double rest = __dsub_rn(A.t_end, t);
#pragma unroll
      for (int k = 0; k < MAXM; ++k)
        if (k < M) T[k] = __dadd_rn(T[k], __dmul_rn(a[k], tdep_integral(bt[k], t, rest)));
    }
    if (A.out.t_internal_dev)
#pragma unroll
      for (int k = 0; k < MAXM; ++k)
        if (k < M) A.out.t_internal_dev[j * M + k] = T[k];
    if (A.out.loglik_dev) {
      double sT = 0.0;
#pragma unroll
      for (int k = 0; k < MAXM; ++k)
        if (k < M) sT = __dadd_rn(sT, T[k]);
      A.out.loglik_dev[j] = status == RT_TRAJ_BAD_X0 ? __longlong_as_double(0x7FF8000000000000ll) : __dsub_rn(ll, sT);
    }
  }
  if (A.out.counts_dev)
#pragma unroll
    for (int k = 0; k < MAXM; ++k)
      if (k < M) A.out.counts_dev[j * M + k] = n[k];
  if (A.out.x_final_dev)
    for (int s = 0; s < N; ++s) A.out.x_final_dev[j * N + s] = X[s * B];
  trace_tail(A.out, j, ev, 0, 1);
  if (A.out.n_events_dev) A.out.n_events_dev[j] = ev;
  if (A.out.status_dev) A.out.status_dev[j] = status;
  if (A.out.t_last_dev) A.out.t_last_dev[j] = t;
}

}  // namespace rt

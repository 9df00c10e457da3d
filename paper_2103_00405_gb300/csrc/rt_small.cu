// rt_small.cu -- ensemble mode for small networks (M <= 4 reactions, N <= 4 species),
// one thread per trajectory with nothing per event in memory.
//
// The NRRTA loop of Table 2 in internal-time form, as in rt_traj_thread.cuh, but the
// counts X live in registers next to P, T, a and n, and the network (reactant
// descriptors, rates, dependency masks, dense net changes) is a kernel parameter:
// loops over channels and species are unrolled, so every table read is a
// constant-bank operand and a per-event value indexed by the fired reaction is a
// chain of selects.  The thread kernel's shared-memory X and tables cost a
// shared-memory round trip (tens of cycles of latency) on the event's critical path
// for every propensity, net change and dependency lookup.
//
// Results are bit-identical to the other mappings: the same operations in the same
// order (tested against the oracle).
#include <cuda_runtime.h>

#include <climits>

#include "rt_moments.cuh"
#include "rt_sim.cuh"

namespace rt {

template <int MAXM, int NMAX, bool LL>
__device__ __forceinline__ void simulate_small(const RunArgs &A, const SmallNet &SN, const MomTable &mt,
                                               const int64_t j, const int tend_finite, const int smem_mom) {
  const int N = A.net.N;
  const uint64_t g = (uint64_t)(A.traj_offset + j);
  const int32_t *x0 = A.x0 + (A.per_traj_x0 ? j * (int64_t)N : 0);
  int X[NMAX];
  bool bad = false;
#pragma unroll
  for (int s = 0; s < NMAX; ++s) {
    X[s] = s < N ? x0[s] : 0;
    bad |= X[s] < 0;
  }
  auto xat = [&](int s) { return pick<NMAX>(X, s); };

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
#pragma unroll
      for (int s = 0; s < NMAX; ++s)
        if (s < N) gp[s] = X[s];
    }
    if (smem_mom) {
      mom_add(mt, gidx, N, xat);
    } else if (A.out.grid_sum_dev) {
#pragma unroll
      for (int s = 0; s < NMAX; ++s)
        if (s < N) {
          const long long x = X[s];
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
    for (int k = 0; k < MAXM; ++k) {
      P[k] = exp1_draw(A.seed, g, (uint32_t)k, 0u, A.stream_id);
      a[k] = propensity(make_int2(SN.s0[k], SN.s1[k]), SN.c[k], xat);
    }
    const int64_t tend_bits = dbits(A.t_end);
    for (;;) {
      // Eq. 25-26: waiting times and the first channel to fire (smallest k on ties);
      // float bounds pick a candidate whose exact quotient is computed first, every
      // other channel is certified strictly larger or computed exactly as well.
      double rem[MAXM];
      float ub_min = __int_as_float(0x7F800000);
      int ks = -1;
#pragma unroll
      for (int k = 0; k < MAXM; ++k) {
        rem[k] = 0.0;
        if (dbits(a[k]) != 0) {
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
        best = dbits(waiting_time_rem(pick<MAXM>(rem, ks), pick<MAXM>(a, ks)));
        mu = ks;
        const float thr = f32_upper(bitsd(best));
#pragma unroll
        for (int k = 0; k < MAXM; ++k)
          if (k != ks && dbits(a[k]) != 0) {
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
      // net change of the fired reaction, from the parameter tables
      int d[NMAX];
      bool over = false;
#pragma unroll
      for (int s = 0; s < NMAX; ++s) {
        d[s] = SN.delta[0][s];
#pragma unroll
        for (int k = 1; k < MAXM; ++k) d[s] = (k == mu) ? SN.delta[k][s] : d[s];
        const long long nx = (long long)X[s] + d[s];
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
      for (int k = 0; k < MAXM; ++k) {
        if (k == mu) a_mu = a[k];
        T[k] = __dadd_rn(T[k], __dmul_rn(a[k], dmin));
      }
      if (LL) ll = __dadd_rn(ll, rt_ln(a_mu));
#pragma unroll
      for (int s = 0; s < NMAX; ++s) X[s] += d[s];
      int32_t nmu = 0;
      uint32_t dm = SN.dep[0];
#pragma unroll
      for (int k = 0; k < MAXM; ++k)
        if (k == mu) {
          n[k] += 1;
          nmu = n[k];
          dm = SN.dep[k];
        }
      ++ev;
      // Eq. 27: only the fired channel draws a new increment
      const double E = exp1_draw(A.seed, g, (uint32_t)mu, (uint32_t)nmu, A.stream_id);
      const double Pmu = __dadd_rn(pick<MAXM>(P, mu), E);  // one FP64 add, placed by selects
#pragma unroll
      for (int k = 0; k < MAXM; ++k) {
        if (k == mu) P[k] = Pmu;
        if ((dm >> k) & 1u) a[k] = propensity(make_int2(SN.s0[k], SN.s1[k]), SN.c[k], xat);
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
      for (int k = 0; k < MAXM; ++k) T[k] = __dadd_rn(T[k], __dmul_rn(a[k], rest));
    }
    if (A.out.t_internal_dev)
#pragma unroll
      for (int k = 0; k < MAXM; ++k) A.out.t_internal_dev[j * MAXM + k] = T[k];
    if (A.out.loglik_dev) {
      double sT = 0.0;
#pragma unroll
      for (int k = 0; k < MAXM; ++k) sT = __dadd_rn(sT, T[k]);
      A.out.loglik_dev[j] = status == RT_TRAJ_BAD_X0 ? __longlong_as_double(0x7FF8000000000000ll) : __dsub_rn(ll, sT);
    }
  }
  if (A.out.counts_dev)
#pragma unroll
    for (int k = 0; k < MAXM; ++k) A.out.counts_dev[j * MAXM + k] = n[k];
  if (A.out.x_final_dev)
#pragma unroll
    for (int s = 0; s < NMAX; ++s)
      if (s < N) A.out.x_final_dev[j * N + s] = X[s];
  trace_tail(A.out, j, ev, 0, 1);
  if (A.out.n_events_dev) A.out.n_events_dev[j] = ev;
  if (A.out.status_dev) A.out.status_dev[j] = status;
  if (A.out.t_last_dev) A.out.t_last_dev[j] = t;
}

// MAXM = M exactly; NMAX >= N.  64 registers: 8 resident blocks of 128 threads.
template <int MAXM, int NMAX, bool LL>
__global__ void __launch_bounds__(128, 8)
    k_ens_small(const RunArgs A, const SmallNet SN, const int tend_finite, const int mom_cl) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int smem_mom = mom_cl > 0 ? 1 : 0;
  const MomTable mt = mom_table((unsigned long long *)smem, A.G, mom_cl);
  if (smem_mom) mom_zero_and_sync(mt, A.net.N);  // every share is zeroed before any block adds to it
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < A.n_traj) simulate_small<MAXM, NMAX, LL>(A, SN, mt, j, tend_finite, smem_mom);
  if (smem_mom) mom_sync_and_flush(mt, A);
}

template <int MAXM, int NMAX>
static cudaError_t launch_small_m(const RunArgs &a, const SmallNet &sn, int B, cudaStream_t s, int tend_finite) {
  const int cl = moment_cluster(a);
  const size_t smem = cl ? moment_share_bytes(a, cl) : 0;
  unsigned grid = (unsigned)((a.n_traj + B - 1) / B);
  if (cl > 1) grid = (grid + cl - 1) / cl * cl;  // whole clusters; blocks past n_traj only hold table shares
  auto kern = a.out.loglik_dev ? k_ens_small<MAXM, NMAX, true> : k_ens_small<MAXM, NMAX, false>;
  return launch_clustered(kern, grid, B, smem, s, cl, a, sn, tend_finite, cl);
}

template <int NMAX>
static cudaError_t launch_small_n(const RunArgs &a, const SmallNet &sn, int B, cudaStream_t s, int tf) {
  switch (a.net.M) {
    case 1: return launch_small_m<1, NMAX>(a, sn, B, s, tf);
    case 2: return launch_small_m<2, NMAX>(a, sn, B, s, tf);
    case 3: return launch_small_m<3, NMAX>(a, sn, B, s, tf);
    default: return launch_small_m<4, NMAX>(a, sn, B, s, tf);
  }
}

int launch_small_mapping(const RunArgs &a, const SmallNet &sn, int B, cudaStream_t s) {
  if (a.n_traj == 0) return RT_OK;
  if (!sn.ok || a.net.M > kSmallM || a.net.N > kSmallN || a.net.M < 1 || a.net.N < 1)
    return set_error(RT_ERR_UNSUPPORTED, "small-network kernel: needs 1 <= M <= %d and 1 <= N <= %d", kSmallM,
                     kSmallN);
  if (B <= 0) B = 128;
  if (B > 128 || B % 32) return set_error(RT_ERR_INVALID_ARG, "thread mapping: block_threads must be a multiple of 32 <= 128");
  const int tf = isfinite(a.t_end) ? 1 : 0;
  const cudaError_t e = a.net.N <= 2 ? launch_small_n<2>(a, sn, B, s, tf) : launch_small_n<4>(a, sn, B, s, tf);
  if (e != cudaSuccess) return set_error(RT_ERR_CUDA, "small-network kernel launch: %s", cudaGetErrorString(e));
  return RT_OK;
}

}  // namespace rt

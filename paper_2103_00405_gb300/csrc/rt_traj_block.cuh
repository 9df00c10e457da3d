// rt_traj_block.cuh -- one thread block per trajectory, state in registers.
//
// The NRRTA loop of Table 2 (Liu & Wang, arXiv:2103.00405) for networks of up to
// 8 * blockDim.x reactions: channel k lives in thread k % B, register slot k / B
// (P_k, T_k, a_k, n_k; Eq. 17-27), X in shared memory.  Per event:
//   1. the channels that read a species the last firing changed are marked in a
//      shared bitmap from the species -> reactions lists (dependency graph, Sec. 5);
//   2. each thread fires its own bookkeeping (new Exp(1) draw, Eq. 27), advances
//      its internal times with the pre-event propensities (Eq. 17), recomputes the
//      marked propensities (Eq. 1-2) and proposes its smallest certified upper
//      bound of the waiting time;
//   3. each warp's best candidate publishes a float upper bound of its waiting time; every
//      thread takes the block's best candidate's bound as threshold, computes exactly only
//      channels not certified to be larger, and a block reduction on (waiting time bits,
//      channel) gives the exact argmin (Eq. 25-26).
#pragma once
#include <climits>

#include "rt_sim.cuh"

namespace rt {

struct BlockNet {
  int M, N;
  const int2 *rd;
  const double *c;
  const int *vp;
  const int2 *vl;
  const int *sptr;
  const int *slist;
  const int *dptr;   // per reaction the channels its firing touches (or null: from sptr/slist)
  const int *dlist;
};

// shared-memory scratch of one block trajectory
struct BlockScratch {
  int *X;           // [N]
  int *NK;          // [M] firing counts n_k
  uint32_t *bm;     // [ceil(M/32)] channels whose propensity must be recomputed
  float *red_u;     // [warps]
  int *red_k;       // [warps]
  long long *red_w; // [warps]
  float *red_q;     // [warps] float upper bound of each warp's candidate's waiting time
  int *red_k2;      // [warps]
  double *buf;      // [B] (and the broadcast slots below)
  double *s_amu;    // propensity of the fired channel
  double *s_E;      // the fired channel's new Exp(1) increment
  int *s_over;      // set if the fired reaction would leave the int32 range
};

__host__ __device__ inline size_t block_scratch_bytes(int M, int N, int B) {
  const int W = B / 32;
  return (size_t)N * 4 + (size_t)M * 4 + (size_t)((M + 31) / 32) * 4 + (size_t)W * (4 + 4 + 4 + 8 + 4) +
         (size_t)B * 8 + 32 + 64;
}

__device__ inline BlockScratch carve_block_scratch(unsigned char *base, int M, int N, int B) {
  const int W = B / 32;
  BlockScratch s;
  s.buf = (double *)base;
  s.red_w = (long long *)(s.buf + B);
  s.s_amu = (double *)(s.red_w + W);
  s.s_E = s.s_amu + 1;
  s.red_u = (float *)(s.s_E + 1);
  s.red_q = s.red_u + W;
  s.red_k = (int *)(s.red_q + W);
  s.red_k2 = s.red_k + W;
  s.s_over = s.red_k2 + W;
  s.bm = (uint32_t *)(s.s_over + 1);
  s.X = (int *)(s.bm + (M + 31) / 32);
  s.NK = s.X + N;
  return s;
}

// Per event (after the first): phase X, right after the argmin is known, runs three
// independent pieces at once -- the fired reaction's net change applied to X by one
// thread per changed species (with the int32 range check), its dependents marked in
// the bitmap, and its new Exp(1) increment drawn by the last thread of the block --
// then one barrier; phase Y advances every T_k with the pre-event a_k (Eq. 17),
// recomputes and unmarks the marked propensities and proposes waiting-time bounds.
// Grid samples, when an event crosses a grid time, are written from the pre-event X
// before phase X behind their own barrier.
template <int R, bool LL>
__device__ __forceinline__ void block_trajectory(const RunArgs &A, const BlockNet &net, const BlockScratch &S, const int64_t j,
                                 const int tend_finite) {
  const int tid = threadIdx.x, B = blockDim.x, lane = tid & 31, warp = tid >> 5, W = B >> 5;
  const int M = net.M, N = net.N;
  const int nbm = (M + 31) / 32;
  const uint64_t g = (uint64_t)(A.traj_offset + j);
  const int32_t *x0 = A.x0 + (A.per_traj_x0 ? j * (int64_t)N : 0);
  int *X = S.X;
  for (int s = tid; s < N; s += B) X[s] = x0[s];
  for (int w = tid; w < nbm; w += B) S.bm[w] = 0u;
  for (int k = tid; k < M; k += B) S.NK[k] = 0;
  if (tid == 0) *S.s_over = 0;
  __syncthreads();
  int badl = 0;
  for (int s = tid; s < N; s += B) badl |= X[s] < 0;
  const bool bad = __syncthreads_or(badl) != 0;
  auto xat = [&](int s) { return X[s]; };

  auto record = [&](int64_t gidx, bool known) {
    if (A.out.grid_dev) {
      int32_t *gp = A.out.grid_dev + (j * A.G + gidx) * N;
      for (int s = tid; s < N; s += B) gp[s] = known ? X[s] : -1;
    }
    if (!known || !A.out.grid_sum_dev) return;
    for (int s = tid; s < N; s += B) {
      const long long x = X[s];
      atomicAdd((unsigned long long *)(A.out.grid_sum_dev + gidx * N + s), (unsigned long long)x);
      if (A.out.grid_sumsq_dev)
        atomicAdd((unsigned long long *)(A.out.grid_sumsq_dev + gidx * N + s), (unsigned long long)(x * x));
    }
    if (tid == 0 && A.out.grid_count_dev) atomicAdd((unsigned long long *)(A.out.grid_count_dev + gidx), 1ull);
  };

  double P[R], T[R], a[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int k = tid + B * r;
    P[r] = 0.0;
    T[r] = 0.0;
    a[r] = 0.0;
    if (!bad && k < M) {
      P[r] = exp1_draw(A.seed, g, (uint32_t)k, 0u, A.stream_id);
      a[r] = propensity<false>(net.rd[k], net.c[k], xat);
    }
  }
  int status = bad ? RT_TRAJ_BAD_X0 : RT_TRAJ_TEND;
  double t = 0.0, ll = 0.0, dmin = 0.0;
  int mu = -1;  // the last fired channel (uniform)
  int32_t ev = 0;
  int64_t gi = 0;
  double next_g = 0.0;
  const int64_t tend_bits = dbits(A.t_end);

  if (!bad) {
    for (;;) {
      // ---- phase Y: the last firing's bookkeeping, T advance, recompute, bounds
      const bool fired = mu >= 0;
      if (fired && tid == mu % B) {  // Eq. 27: the fired channel's new increment
        const int rm = mu / B;
        const double E = *S.s_E;
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (r == rm) P[r] = __dadd_rn(P[r], E);
      }
      if (LL && fired && tid == 0) ll = __dadd_rn(ll, rt_ln(*S.s_amu));
      if (tid == 0) *S.s_over = 0;
      const bool adv = fired && dbits(dmin) != 0;
      float ub = __int_as_float(0x7F800000);
      int kub = INT_MAX;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int k = tid + B * r;
        if (k < M) {
          if (adv && dbits(a[r]) != 0) T[r] = __dadd_rn(T[r], __dmul_rn(a[r], dmin));
          const uint32_t bit = 1u << (k & 31);
          if (S.bm[k >> 5] & bit) {
            a[r] = propensity<false>(net.rd[k], net.c[k], xat);
            atomicAnd(&S.bm[k >> 5], ~bit);
          }
          if (dbits(a[r]) != 0) {
            const float u = wait_estimate(P[r], T[r], a[r]);
            if (kub == INT_MAX || u < ub) {
              ub = u;
              kub = k;
            }
          }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float u2 = __shfl_xor_sync(0xFFFFFFFFu, ub, o);
        const int k2 = __shfl_xor_sync(0xFFFFFFFFu, kub, o);
        if (u2 < ub || (u2 == ub && k2 < kub)) {
          ub = u2;
          kub = k2;
        }
      }
      // the warp candidate's owner publishes a float upper bound of its waiting time with it, so
      // the block's threshold is known right after the reduction (one barrier, no division)
      if (kub != INT_MAX && tid == kub % B) {
        const int rs = kub / B;
        S.red_q[warp] = quot_upper(pick<R>(P, rs), pick<R>(T, rs), pick<R>(a, rs));
        S.red_u[warp] = ub;
        S.red_k[warp] = kub;
      } else if (kub == INT_MAX && lane == 0) {
        S.red_u[warp] = ub;
        S.red_k[warp] = kub;
      }
      __syncthreads();
      // every warp reduces the W warp minima itself (lane w reads warp w's): the block minimum
      // in every thread without another barrier (lexicographic minimum: order-independent)
      ub = lane < W ? S.red_u[lane] : __int_as_float(0x7F800000);
      kub = lane < W ? S.red_k[lane] : INT_MAX;
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
      // ---- every channel not certified to lie above the block candidate's upper bound, exactly
      // (the candidate itself is never certified above its own bound) (Eq. 25-26)
      const float thr = S.red_q[(kub % B) >> 5];
      long long bw = LLONG_MAX;
      int bk = INT_MAX;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int k = tid + B * r;
        if (k < M && dbits(a[r]) != 0 && !exceeds(P[r], T[r], a[r], thr)) {
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
      if (lane == 0) {
        S.red_w[warp] = bw;
        S.red_k2[warp] = bk;
      }
      __syncthreads();
      bw = lane < W ? S.red_w[lane] : LLONG_MAX;
      bk = lane < W ? S.red_k2[lane] : INT_MAX;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const long long w2 = __shfl_xor_sync(0xFFFFFFFFu, bw, o);
        const int k2 = __shfl_xor_sync(0xFFFFFFFFu, bk, o);
        if (w2 < bw || (w2 == bw && k2 < bk)) {
          bw = w2;
          bk = k2;
        }
      }
      const double dnext = bitsd(bw);
      const double tn = __dadd_rn(t, dnext);
      if (dbits(tn) > tend_bits) {
        status = RT_TRAJ_TEND;
        break;
      }
      if (ev == A.max_events) {
        status = RT_TRAJ_MAX_EVENTS;
        break;
      }
      const int vb = net.vp[bk], ve = net.vp[bk + 1];
      if (gi < A.G && dbits(next_g) < dbits(tn)) {
        // grid samples from the pre-event X, after the range check (an overflowing event
        // records nothing); X is only read until the barrier below
        bool over = false;
        for (int i = vb; i < ve; ++i) {
          const int2 e = net.vl[i];
          const long long nx = (long long)X[e.x] + e.y;
          over |= (nx > INT_MAX) | (nx < 0);
        }
        if (over) {
          status = RT_TRAJ_OVERFLOW;
          break;
        }
        while (gi < A.G && dbits(next_g) < dbits(tn)) {
          record(gi, true);
          ++gi;
          next_g = __dmul_rn(__ll2double_rn(gi), A.sample_dt);
        }
        __syncthreads();
      }
      // ---- phase X: net change with range check, dependents, new draw (all at once)
      for (int i = vb + tid; i < ve; i += B) {
        const int2 e = net.vl[i];
        const long long nx = (long long)X[e.x] + e.y;
        if ((nx > INT_MAX) | (nx < 0)) *S.s_over = 1;
        X[e.x] = (int)(uint32_t)((uint32_t)X[e.x] + (uint32_t)e.y);
      }
      if (net.dptr) {  // one list per reaction: two dependent loads instead of four
        for (int q = net.dptr[bk] + tid; q < net.dptr[bk + 1]; q += B) {
          const int ch = net.dlist[q];
          atomicOr(&S.bm[ch >> 5], 1u << (ch & 31));
        }
      } else {
        for (int i = vb; i < ve; ++i) {
          const int s = net.vl[i].x;
          for (int q = net.sptr[s] + tid; q < net.sptr[s + 1]; q += B) {
            const int ch = net.slist[q];
            atomicOr(&S.bm[ch >> 5], 1u << (ch & 31));
          }
        }
      }
      if (tid == B - 1) {
        const int32_t n = S.NK[bk] + 1;
        S.NK[bk] = n;
        *S.s_E = exp1_draw(A.seed, g, (uint32_t)bk, (uint32_t)n, A.stream_id);
      }
      if (LL && tid == (bk % B)) *S.s_amu = pick<R>(a, bk / B);
      __syncthreads();
      if (*S.s_over) {  // undo: the event does not fire
        for (int i = vb + tid; i < ve; i += B) {
          const int2 e = net.vl[i];
          X[e.x] = (int)(uint32_t)((uint32_t)X[e.x] - (uint32_t)e.y);
        }
        if (tid == B - 1) S.NK[bk] -= 1;
        status = RT_TRAJ_OVERFLOW;
        break;
      }
      t = tn;
      if (tid == 0) trace_event(A.out, j, ev, bk, tn);
      ++ev;
      dmin = dnext;
      mu = bk;
    }
  }

  __syncthreads();
  const bool known = status == RT_TRAJ_TEND || status == RT_TRAJ_ABSORBED;
  for (; gi < A.G; ++gi) record(gi, known);
  if (A.out.loglik_dev || A.out.t_internal_dev) {
    if (known && tend_finite && !bad) {
      const double rest = __dsub_rn(A.t_end, t);
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (tid + B * r < M) T[r] = __dadd_rn(T[r], __dmul_rn(a[r], rest));
    }
    if (A.out.t_internal_dev)
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (tid + B * r < M) A.out.t_internal_dev[j * M + tid + B * r] = T[r];
    if (A.out.loglik_dev) {
      double sT = 0.0;  // sum_k T_k in k order, B values at a time through shared memory
#pragma unroll
      for (int r = 0; r < R; ++r) {
        S.buf[tid] = T[r];
        __syncthreads();
        if (tid == 0)
          for (int l = 0; l < B && l + B * r < M; ++l) sT = __dadd_rn(sT, S.buf[l]);
        __syncthreads();
      }
      if (tid == 0) A.out.loglik_dev[j] = bad ? __longlong_as_double(0x7FF8000000000000ll) : __dsub_rn(ll, sT);
    }
  }
  if (A.out.counts_dev)
    for (int k = tid; k < M; k += B) A.out.counts_dev[j * M + k] = S.NK[k];
  if (A.out.x_final_dev)
    for (int s = tid; s < N; s += B) A.out.x_final_dev[j * N + s] = X[s];
  trace_tail(A.out, j, ev, tid, B);
  if (tid == 0) {
    if (A.out.n_events_dev) A.out.n_events_dev[j] = ev;
    if (A.out.status_dev) A.out.status_dev[j] = status;
    if (A.out.t_last_dev) A.out.t_last_dev[j] = t;
  }
  __syncthreads();
}

}  // namespace rt

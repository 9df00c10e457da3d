// rt_bundle.cu -- large-network mode: a "bundle" of thread blocks per trajectory.
//
// The paper's GPU layout (Sec. 5) gives each trajectory a bundle of blocks with one
// thread per reaction and a two-level (block, then bundle) argmin reduction.  Here a
// trajectory's M channels are split into C contiguous slices, one per co-resident
// block (cooperative launch); per event every block streams its slice of P, T, a
// through HBM in one fused pass (16-byte asynchronous copies into a per-thread ring
// of shared-memory stages, several pairs of channels per thread in flight):
//   T_k += a_k * dt_prev                       (Eq. 17, with the pre-event a_k)
//   a_k = c_k h_k(X) if k depends on a species the last event changed (Eq. 1-2)
//   w_k = (P_k - T_k) / a_k and a running argmin (Eq. 25-26)
// then the C block minima meet in global memory behind a bounded-spin barrier, and
// every block takes the same decision (fire mu, or stop) from the same data.  Each
// block mirrors X in shared memory, so firing needs no second barrier.
//
// The exact binary64 division is skipped for channels whose certified float lower
// bound exceeds a threshold: the block's running best, and a per-event threshold
// K / sum(a) that catches all but ~e^-K of minima (sum(a) retaken every 64 events).
// If no channel beat the threshold, the event is re-scanned without it (read-only),
// so the minimum is always the exact one, with the smallest index on ties.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdlib>

#include "rt_filter.cuh"
#include "rt_sim.cuh"

namespace rt {

constexpr int kBundleThreads = 512;
constexpr float kThresholdK = 12.0f;  // per-event threshold K / sum(a): P(re-scan) ~ e^-12
constexpr int kSumEvery = 64;         // events between two sums of a (the threshold's sum(a))
constexpr int kMaxDepth = 6;          // stages of the per-thread copy ring, at most

struct __align__(16) Partial {
  long long wbits;  // bits of the block's minimum waiting time (+inf if none)
  int k;            // its channel (-1 if none)
  int pad;
  double a;         // its propensity
  float asum;       // block sum of float lower bounds of a_k
  int pad2;
};

struct BundleArgs {
  RunArgs r;
  int C;             // blocks per trajectory
  int64_t traj0;     // first trajectory of this launch
  int64_t Ms;        // row stride of P/T/A/NK (multiple of 32)
  int64_t chunk;     // channels per block slice (multiple of 32)
  double *P, *T, *A;
  int32_t *NK;
  Partial *part;     // [n_traj][2][C]
  unsigned long long *bar;  // [n_traj] monotonic arrival counters
  int tend_finite;
  long long spin_limit;
  int want_T;        // finalise T at t_end (t_internal or loglik requested)
  int depth;         // stages of the per-thread copy ring, 1..kMaxDepth
};

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Arrive at the trajectory's barrier and wait (thread 0 only).  Returns false if the
// wait gave up after spin_limit polls.
__device__ bool bundle_barrier(unsigned long long *ctr, unsigned long long target, long long limit) {
  __threadfence();
  atomicAdd(ctr, 1ull);
  long long it = 0;
  while (ld_acquire(ctr) < target) {
    if (++it > limit) return false;
    __nanosleep(100);
  }
  __threadfence();
  return true;
}

__global__ void k_bundle_init(const BundleArgs B) {
  const RunArgs &r = B.r;
  const int64_t total = r.n_traj * (int64_t)r.net.M;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = i / r.net.M;
    const int k = (int)(i - j * r.net.M);
    const int32_t *x0 = r.x0 + (r.per_traj_x0 ? j * r.net.N : 0);
    const int64_t o = j * B.Ms + k;
    B.T[o] = 0.0;
    B.NK[o] = 0;
    B.P[o] = exp1_draw(r.seed, (uint64_t)(r.traj_offset + j), (uint32_t)k, 0u, r.stream_id);
    B.A[o] = propensity<false>(r.net.rdesc[k], r.net.c[k], [&](int s) { return x0[s]; });
  }
}

// ---- per-thread asynchronous global -> shared copies (16 B) in commit groups ----
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most n of this thread's most recent groups are pending (n < kMaxDepth)
__device__ __forceinline__ void cp_async_wait(int n) {
  switch (n) {
    case 0: asm volatile("cp.async.wait_group 0;" ::: "memory"); break;
    case 1: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
    case 3: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
    case 4: asm volatile("cp.async.wait_group 4;" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 5;" ::: "memory"); break;
  }
}

struct Decision {
  int mu;
  int stop;      // 0 continue, else 1 + status
  int rescan;
  int pad;
  double dt;
  double a_mu;
  float tau;
};

template <bool LL>
__global__ void __launch_bounds__(kBundleThreads) k_bundle(const BundleArgs B) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long red_w[kBundleThreads / 32];
  __shared__ int red_k[kBundleThreads / 32];
  __shared__ double red_a[kBundleThreads / 32];
  __shared__ float red_s[kBundleThreads / 32];
  __shared__ Decision dec;

  const RunArgs &r = B.r;
  const int M = r.net.M, N = r.net.N;
  const int C = B.C;
  const int c = blockIdx.x % C;
  const int64_t j = B.traj0 + blockIdx.x / C;
  if (j >= r.n_traj) return;
  const int64_t k0 = (int64_t)c * B.chunk;
  const int64_t k1 = min((int64_t)M, k0 + B.chunk);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int D = B.depth;
  double *ring = (double *)smem;  // [D][3][kBundleThreads][2]: P, T, a pairs of each thread
  int *Xs = (int *)(ring + (size_t)D * 3 * 2 * kBundleThreads);
  uint32_t *bm = (uint32_t *)(Xs + N);
  const int nbm = (int)((B.chunk + 31) / 32);
  double *P = B.P + j * B.Ms, *T = B.T + j * B.Ms, *A = B.A + j * B.Ms;
  int32_t *NK = B.NK + j * B.Ms;
  Partial *part = B.part + j * 2 * C;
  unsigned long long *bar = B.bar + j;
  const uint64_t g = (uint64_t)(r.traj_offset + j);
  const int32_t *x0 = r.x0 + (r.per_traj_x0 ? j * N : 0);

  __shared__ int s_bad;
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int s = tid; s < N; s += blockDim.x) {
    const int v = x0[s];
    Xs[s] = v;
    if (v < 0) s_bad = 1;
  }
  for (int w = tid; w < nbm; w += blockDim.x) bm[w] = 0u;
  __syncthreads();
  const bool bad = s_bad != 0;
  auto xat = [&](int s) { return Xs[s]; };

  double t = 0.0, dprev = 0.0, ll = 0.0;
  int mu_prev = -1;
  int32_t ev = 0;
  int status = bad ? RT_TRAJ_BAD_X0 : RT_TRAJ_TEND;
  unsigned long long rounds = 0;
  float tau = __int_as_float(0x7F800000);
  float tau_last = __int_as_float(0x7F800000);  // block thread 0: K / sum(a) at the last summed event
  int64_t gi = 0;
  double next_g = 0.0;
  const int64_t tend_bits = dbits(r.t_end);

  auto record = [&](int64_t gidx, bool known) {  // block 0, all threads
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

  // mark (set) or clear the slice bits of the channels that read a species changed by `mu`
  auto touch_dependents = [&](int mu, bool set) {
    const int vb = r.net.vptr[mu], ve = r.net.vptr[mu + 1];
    for (int i = vb; i < ve; ++i) {
      const int s = r.net.vlist[i].x;
      const int qb = r.net.sptr[s], qe = r.net.sptr[s + 1];
      for (int q = qb + tid; q < qe; q += blockDim.x) {
        const int64_t rr = r.net.slist[q];
        if (rr >= k0 && rr < k1) {
          const int off = (int)(rr - k0);
          if (set) atomicOr(&bm[off >> 5], 1u << (off & 31));
          else bm[off >> 5] = 0u;
        }
      }
    }
  };

  bool timed_out = false;
  if (!bad) {
    for (;;) {
      // ---- fire the previous event's bookkeeping: new Exp(1) for P_mu (Eq. 27), dependents
      if (mu_prev >= 0) {
        if (tid == 0 && mu_prev >= k0 && mu_prev < k1) {
          const int32_t n = NK[mu_prev] + 1;
          NK[mu_prev] = n;
          P[mu_prev] = __dadd_rn(P[mu_prev], exp1_draw(r.seed, g, (uint32_t)mu_prev, (uint32_t)n, r.stream_id));
        }
        touch_dependents(mu_prev, true);
      }
      __syncthreads();

      // ---- fused pass over the slice
      long long bestb = kInfBits;
      int bestk = -1;
      double besta = 0.0;
      float asum = 0.0f;
      float thr = tau;  // min(tau, float upper bound of the running best)
      // sum(a) drifts slowly (an event changes few propensities): it is taken on every
      // kSumEvery-th event only, and the threshold K / sum(a) is kept in between
      const bool summed = (ev % kSumEvery) == 0;
      const bool advance = dbits(dprev) != 0;
      // pairs of channels k, k+1 per thread.  Each thread streams its own pairs through
      // a ring of D shared-memory stages filled by asynchronous copies, so D - 1 pairs
      // per thread are in flight while one is processed, without holding registers.
      // A pair is copied as 16 bytes even when only k is in the slice: then k + 1 = M
      // is the row's padding (rows are padded to a multiple of 32) and is not used.
      const int64_t stride = 2 * (int64_t)blockDim.x;
      const int64_t kb = k0 + 2 * tid;
      const int nmine = kb < k1 ? (int)((k1 - kb + stride - 1) / stride) : 0;
      auto slot = [&](int st, int arr) { return ring + ((size_t)(st * 3 + arr) * kBundleThreads + tid) * 2; };
      int st_issue = 0, st_use = 0;
      auto issue = [&](int i) {  // pair i of this thread, one commit group (empty past the end)
        if (i < nmine) {
          const int64_t kk = kb + (int64_t)i * stride;
          cp_async16(slot(st_issue, 0), P + kk);
          cp_async16(slot(st_issue, 1), T + kk);
          cp_async16(slot(st_issue, 2), A + kk);
        }
        cp_async_commit();
        st_issue = st_issue + 1 == D ? 0 : st_issue + 1;
      };
      for (int i = 0; i < D - 1; ++i) issue(i);
      for (int i = 0; i < nmine; ++i) {
        issue(i + D - 1);  // into the stage processed in the previous iteration
        cp_async_wait(D - 1);
        const int64_t k = kb + (int64_t)i * stride;
        const double2 a2 = *(const double2 *)slot(st_use, 2);
        const double2 t2 = *(const double2 *)slot(st_use, 1);
        const double2 p2 = *(const double2 *)slot(st_use, 0);
        st_use = st_use + 1 == D ? 0 : st_use + 1;
        const bool two = k + 1 < k1;
        double av[2] = {a2.x, a2.y}, tv[2] = {t2.x, t2.y};
        const double pv[2] = {p2.x, p2.y};
        const uint32_t bits = bm[(k - k0) >> 5] >> ((k - k0) & 31);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (h == 1 && !two) break;
          if (advance && dbits(av[h]) != 0) tv[h] = __dadd_rn(tv[h], __dmul_rn(av[h], dprev));
          if ((bits >> h) & 1u) {
            av[h] = propensity<false>(r.net.rdesc[k + h], r.net.c[k + h], xat);
            A[k + h] = av[h];
          }
          if (dbits(av[h]) != 0) {
            if (summed) asum = __fadd_rn(asum, f32_lower(av[h]));
            if (!exceeds(pv[h], tv[h], av[h], thr)) {
              const long long wb = dbits(waiting_time(pv[h], tv[h], av[h]));
              if (wb < bestb) {
                bestb = wb;
                bestk = (int)(k + h);
                besta = av[h];
                thr = fminf(tau, f32_upper(bitsd(wb)));
              }
            }
          }
        }
        if (advance) {
          if (two) *(double2 *)(T + k) = make_double2(tv[0], tv[1]);
          else T[k] = tv[0];
        }
      }
      cp_async_wait(0);  // only empty groups can remain; none is left behind

      // ---- block argmin (lexicographic on (w, k)) and sum of a
      auto reduce_and_publish = [&](long long wb, int kk, double aa, float ss) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const long long w2 = __shfl_xor_sync(0xFFFFFFFFu, wb, o);
          const int k2 = __shfl_xor_sync(0xFFFFFFFFu, kk, o);
          const double a2v = __shfl_xor_sync(0xFFFFFFFFu, aa, o);
          ss = __fadd_rn(ss, __shfl_xor_sync(0xFFFFFFFFu, ss, o));
          if (w2 < wb || (w2 == wb && (unsigned)k2 < (unsigned)kk)) {
            wb = w2;
            kk = k2;
            aa = a2v;
          }
        }
        if (lane == 0) {
          red_w[warp] = wb;
          red_k[warp] = kk;
          red_a[warp] = aa;
          red_s[warp] = ss;
        }
        __syncthreads();
        if (tid == 0) {
          long long w = red_w[0];
          int k = red_k[0];
          double a = red_a[0];
          float s = red_s[0];
          for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
            if (red_w[i] < w || (red_w[i] == w && (unsigned)red_k[i] < (unsigned)k)) {
              w = red_w[i];
              k = red_k[i];
              a = red_a[i];
            }
            s = __fadd_rn(s, red_s[i]);
          }
          Partial p;
          p.wbits = w;
          p.k = k;
          p.pad = 0;
          p.a = a;
          p.asum = s;
          p.pad2 = 0;
          part[(rounds & 1) * C + c] = p;
        }
      };
      reduce_and_publish(bestb, bestk, besta, asum);

      // ---- meet the other blocks of this trajectory; every block takes the same decision
      bool rescan_needed, rescanning = false;
      for (;;) {
        if (tid == 0) {
          bool ok = true;
          if (C > 1) ok = bundle_barrier(bar, (rounds + 1) * (unsigned long long)C, B.spin_limit);
          dec.stop = 0;
          dec.rescan = 0;
          if (!ok) {
            dec.stop = 1 + RT_TRAJ_TIMEOUT;
          } else {
            long long w = kInfBits;
            int k = -1;
            double a = 0.0;
            float s = 0.0f;
            const Partial *pp = part + (rounds & 1) * C;
            for (int i = 0; i < C; ++i) {
              const long long wi = __ldcg(&pp[i].wbits);
              const int ki = __ldcg(&pp[i].k);
              const double ai = __ldcg(&pp[i].a);
              s = __fadd_rn(s, __ldcg(&pp[i].asum));
              if (wi < w || (wi == w && (unsigned)ki < (unsigned)k)) {
                w = wi;
                k = ki;
                a = ai;
              }
            }
            if (summed && !rescanning) tau_last = s > 0.0f ? __fdiv_ru(kThresholdK, s) : __int_as_float(0x7F800000);
            // a threshold-filtered scan is exact only if its minimum is below the threshold
            const bool filtered = tau != __int_as_float(0x7F800000);
            if (filtered && !(w < dbits((double)tau))) {
              dec.rescan = 1;
            } else {
              dec.mu = k;
              dec.dt = bitsd(w);
              dec.a_mu = a;
              dec.tau = tau_last;
            }
          }
        }
        __syncthreads();
        rounds += 1;
        rescan_needed = dec.rescan != 0;
        if (!rescan_needed || dec.stop) break;
        // read-only exact re-scan of the (already advanced) slice
        rescanning = true;
        tau = __int_as_float(0x7F800000);
        bestb = kInfBits;
        bestk = -1;
        besta = 0.0;
        for (int64_t k = k0 + tid; k < k1; k += blockDim.x) {
          const double a = A[k];
          if (dbits(a) == 0) continue;
          const double p = P[k], tt = T[k];
          if (bestb != kInfBits && exceeds(p, tt, a, f32_upper(bitsd(bestb)))) continue;
          const long long wb = dbits(waiting_time(p, tt, a));
          if (wb < bestb) {
            bestb = wb;
            bestk = (int)k;
            besta = a;
          }
        }
        __syncthreads();
        reduce_and_publish(bestb, bestk, besta, 0.0f);
      }
      if (dec.stop) {
        timed_out = true;
        status = RT_TRAJ_TIMEOUT;
        break;
      }
      // clear this event's dependents bits before they change meaning
      if (mu_prev >= 0) touch_dependents(mu_prev, false);

      const int mu = dec.mu;
      if (mu < 0) {
        status = RT_TRAJ_ABSORBED;
        break;
      }
      const double dmin = dec.dt;
      const double tn = __dadd_rn(t, dmin);
      if (dbits(tn) > tend_bits) {
        status = RT_TRAJ_TEND;
        break;
      }
      if (ev == r.max_events) {
        status = RT_TRAJ_MAX_EVENTS;
        break;
      }
      {
        bool over = false;
        for (int i = r.net.vptr[mu]; i < r.net.vptr[mu + 1]; ++i) {
          const int2 e = r.net.vlist[i];
          const long long nx = (long long)Xs[e.x] + e.y;
          over |= (nx > INT_MAX) | (nx < 0);
        }
        if (over) {
          status = RT_TRAJ_OVERFLOW;
          break;
        }
      }
      if (c == 0) {
        while (gi < r.G && dbits(next_g) < dbits(tn)) {
          record(gi, true);
          ++gi;
          next_g = __dmul_rn(__ll2double_rn(gi), r.sample_dt);
        }
      }
      t = tn;
      if (c == 0 && tid == 0) trace_event(r.out, j, ev, mu, tn);
      if (LL && c == 0 && tid == 0) ll = __dadd_rn(ll, rt_ln(dec.a_mu));
      __syncthreads();  // everyone has read Xs for this event
      if (tid == 0)
        for (int i = r.net.vptr[mu]; i < r.net.vptr[mu + 1]; ++i) {
          const int2 e = r.net.vlist[i];
          Xs[e.x] += e.y;
        }
      ++ev;
      dprev = dmin;
      mu_prev = mu;
      tau = dec.tau;
      __syncthreads();
    }
  }
  (void)timed_out;

  // ---- finalise
  const bool known = status == RT_TRAJ_TEND || status == RT_TRAJ_ABSORBED;
  if (c == 0)
    for (; gi < r.G; ++gi) record(gi, known);
  if (B.want_T && known && B.tend_finite && !bad) {
    const double rest = __dsub_rn(r.t_end, t);
    for (int64_t k = k0 + tid; k < k1; k += blockDim.x) T[k] = __dadd_rn(T[k], __dmul_rn(A[k], rest));
  }
  if (r.out.t_internal_dev)
    for (int64_t k = k0 + tid; k < k1; k += blockDim.x) r.out.t_internal_dev[j * M + k] = T[k];
  if (r.out.counts_dev)
    for (int64_t k = k0 + tid; k < k1; k += blockDim.x) r.out.counts_dev[j * M + k] = NK[k];
  if (LL) {
    __syncthreads();
    bool ok = true;
    if (tid == 0 && C > 1 && status != RT_TRAJ_TIMEOUT) ok = bundle_barrier(bar, (rounds + 1) * (unsigned long long)C, B.spin_limit);
    rounds += 1;
    if (c == 0 && tid == 0) {
      if (!ok) status = RT_TRAJ_TIMEOUT;
      double sT = 0.0;
      for (int k = 0; k < M; ++k) sT = __dadd_rn(sT, __ldcg(T + k));
      r.out.loglik_dev[j] = bad ? __longlong_as_double(0x7FF8000000000000ll) : __dsub_rn(ll, sT);
    }
  }
  if (c == 0) {
    __syncthreads();
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

static int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

struct BundlePlan {
  int C;
  int64_t Ms, chunk;
  size_t off_P, off_T, off_A, off_NK, off_part, off_bar, total;
  size_t smem;
  int depth;  // stages of the per-thread copy ring
};

constexpr int kRingDepth = 4;               // preferred ring depth (3 pairs per thread in flight)
constexpr size_t kSmemBudget = 220 * 1024;  // dynamic shared memory per block
static_assert(kRingDepth <= kMaxDepth, "ring deeper than cp_async_wait supports");

static BundlePlan plan_bundle(const DevNet &net, int64_t n_traj, int C) {
  BundlePlan p;
  p.C = C;
  p.Ms = round_up(net.M, 32);
  p.chunk = round_up((net.M + C - 1) / C, 32);
  const int64_t rows = n_traj > 0 ? n_traj : 1;
  size_t off = 0;
  p.off_P = off; off += (size_t)rows * p.Ms * 8;
  p.off_T = off; off += (size_t)rows * p.Ms * 8;
  p.off_A = off; off += (size_t)rows * p.Ms * 8;
  p.off_NK = off; off += (size_t)round_up(rows * p.Ms * 4, 256);
  p.off_part = off; off += (size_t)round_up(rows * 2 * C * sizeof(Partial), 256);
  p.off_bar = off; off += (size_t)round_up(rows * sizeof(unsigned long long), 256);
  p.total = off;
  const size_t rest = (size_t)net.N * 4 + (size_t)((p.chunk + 31) / 32) * 4;
  const size_t stage = (size_t)3 * 2 * kBundleThreads * 8;  // 24 KB per ring stage
  int want = kRingDepth;  // RT_BUNDLE_RING_DEPTH (1..kMaxDepth) overrides, for tuning
  if (const char *env = getenv("RT_BUNDLE_RING_DEPTH")) want = std::min(kMaxDepth, std::max(1, atoi(env)));
  p.depth = 1;
  for (int d = want; d > 1; --d)
    if (d * stage + rest <= kSmemBudget) {
      p.depth = d;
      break;
    }
  p.smem = p.depth * stage + rest;
  return p;
}

// Blocks of the bundle kernel resident on the whole GPU at a given shared-memory size;
// 0 when the size is above the opt-in limit (checked first, so that no attribute call
// fails and leaves an error behind for the caller's next CUDA call).
static int bundle_capacity(size_t smem, bool ll) {
  int dev = 0, sms = 0, optin = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem > (size_t)optin - 1024) return 0;  // static shared memory (barriers) included
  auto kern = ll ? k_bundle<true> : k_bundle<false>;
  if (raise_smem_limit((const void *)kern, smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBundleThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * sms;
}

// Blocks per trajectory.  The per-block channel bitmap shrinks as C grows, so the
// smallest C whose shared memory fits is found first; from there C is raised until
// the trajectories of one wave fill the GPU (n_traj * C <= capacity), keeping at
// least 32 channels per block.
static int choose_C(const DevNet &net, int64_t n_traj, int requested, bool ll) {
  if (requested > 0) return requested;
  int c_min = 1, cap = 0;
  for (; c_min <= 4096; c_min *= 2)
    if ((cap = bundle_capacity(plan_bundle(net, 1, c_min).smem, ll)) >= c_min) break;
  if (cap < c_min) return 1;  // nothing fits: the launch reports it
  int64_t C = n_traj > 0 ? cap / std::max<int64_t>(1, std::min<int64_t>(n_traj, cap)) : 1;
  C = std::min<int64_t>(C, std::max<int64_t>(1, net.M / 32));
  return (int)std::max<int64_t>(c_min, C);
}

size_t bundle_workspace_bytes(const DevNet &net, int64_t n_traj, int ctas_per_traj) {
  const int C = std::max(choose_C(net, n_traj, ctas_per_traj, false), choose_C(net, n_traj, ctas_per_traj, true));
  return plan_bundle(net, n_traj, C).total;
}

int launch_bundle_mapping(const RunArgs &a, int ctas_per_traj, void *ws, size_t ws_bytes, cudaStream_t s) {
  if (a.n_traj == 0) return RT_OK;
  const bool ll = a.out.loglik_dev != nullptr;
  const int C = choose_C(a.net, a.n_traj, ctas_per_traj, ll);
  const BundlePlan p = plan_bundle(a.net, a.n_traj, C);
  if (!ws || ws_bytes < p.total)
    return set_error(RT_ERR_OOM, "bundle mapping needs %zu bytes of workspace (got %zu)", p.total, ws_bytes);
  if (((uintptr_t)ws & 255) != 0) return set_error(RT_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  if (p.smem > kSmemBudget)
    return set_error(RT_ERR_UNSUPPORTED,
                     "bundle mapping: %d species and %lld channels per block do not fit in shared memory",
                     a.net.N, (long long)p.chunk);
  char *w = (char *)ws;
  BundleArgs B;
  B.r = a;
  B.C = C;
  B.Ms = p.Ms;
  B.chunk = p.chunk;
  B.P = (double *)(w + p.off_P);
  B.T = (double *)(w + p.off_T);
  B.A = (double *)(w + p.off_A);
  B.NK = (int32_t *)(w + p.off_NK);
  B.part = (Partial *)(w + p.off_part);
  B.bar = (unsigned long long *)(w + p.off_bar);
  B.tend_finite = std::isfinite(a.t_end) ? 1 : 0;
  B.want_T = (a.out.t_internal_dev || a.out.loglik_dev) ? 1 : 0;
  B.depth = p.depth;
  long long spin = 20000000;  // ~2 s of 100 ns polls
  if (const char *env = getenv("RT_DEBUG_SPIN_LIMIT")) spin = atoll(env);
  B.spin_limit = spin;
  B.traj0 = 0;
  // every check comes before the first enqueued operation: a refused launch leaves
  // the stream, the workspace and the outputs untouched
  auto kern = ll ? k_bundle<true> : k_bundle<false>;
  const int64_t cap = bundle_capacity(p.smem, ll);
  if (cap < C) return set_error(RT_ERR_UNSUPPORTED, "bundle of %d blocks cannot be co-resident (capacity %lld)", C, (long long)cap);
  const int64_t per_wave = cap / C;
  cudaError_t e = cudaMemsetAsync(B.bar, 0, sizeof(unsigned long long) * a.n_traj, s);
  if (e != cudaSuccess) return set_error(RT_ERR_CUDA, "memset: %s", cudaGetErrorString(e));
  k_bundle_init<<<152 * 8, 256, 0, s>>>(B);
  if ((e = cudaGetLastError()) != cudaSuccess) return set_error(RT_ERR_CUDA, "init launch: %s", cudaGetErrorString(e));

  for (int64_t t0 = 0; t0 < a.n_traj; t0 += per_wave) {
    B.traj0 = t0;
    const int64_t nw = std::min<int64_t>(per_wave, a.n_traj - t0);
    void *args[] = {&B};
    if (C > 1) {
      e = cudaLaunchCooperativeKernel((const void *)kern, dim3((unsigned)(nw * C)), dim3(kBundleThreads), args, p.smem, s);
    } else {
      kern<<<(unsigned)nw, kBundleThreads, p.smem, s>>>(B);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return set_error(RT_ERR_CUDA, "bundle launch: %s", cudaGetErrorString(e));
  }
  return RT_OK;
}

// ----------------------------------------------------------------------------------
// Allocation-free entry point
//
// Some callers cannot call cudaMalloc where they run a simulation: a host
// application whose device memory is owned by its own pool allocator (a direct
// cudaMalloc would go around its budget), or a latency-critical loop that must not
// enter the driver's allocator, which can synchronise the device.  rt_run's large-
// network mapping needs a caller-allocated workspace; rt_run_bundle_noalloc runs
// the same kernels with their scratch (P, T, a, counts, block minima, barrier
// counters) in the fixed array below instead.
//
// The array is a file-scope __device__ variable: every GPU that loads this library
// holds kNoAllocScratchBytes of it until the process exits.  In host code the
// array's name is only a host-side stand-in, so its device address is obtained with
// cudaGetSymbolAddress, by every call (with the calling device current; the lookup
// allocates nothing and is cheap, and it stays right if the device's context is
// torn down and re-created between calls, where the module and its array may be
// loaded at a new address).  The first call on a device loads the library's module
// there, so it should come before any stream capture.  Every call on a device uses
// the same array and leaves its contents behind; the launch zeroes what must start
// at zero (the barrier counters) and initialises the rest.  Calls whose work
// overlaps on the GPU (different streams, or threads without ordering) race on the
// array: order them on one stream or synchronise between them.
// ----------------------------------------------------------------------------------

constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch array on the current device.
static int noalloc_scratch(void **out) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    return set_error(RT_ERR_CUDA, "cudaGetSymbolAddress of the scratch array: %s", cudaGetErrorString(e));
  *out = p;
  return RT_OK;
}

}  // namespace rt

extern "C" int rt_run_bundle_noalloc(const rt_network *net, const rt_run_params *p, const rt_outputs *o,
                                     int32_t ctas_per_traj, void *stream) {
  using namespace rt;
  clear_error();
  int rc = validate_run(net, p, o);
  if (rc) return rc;
  if ((rc = check_device(net))) return rc;
  if (p->form != RT_FORM_INTERNAL || net->dev.beta)
    return set_error(RT_ERR_UNSUPPORTED, "rt_run_bundle_noalloc runs the internal-time form with constant rates only");
  RunArgs a;
  a.net = net->dev;
  a.x0 = p->x0_dev;
  a.per_traj_x0 = p->per_traj_x0 ? 1 : 0;
  a.stream_id = p->stream_id;
  a.t_end = p->t_end;
  a.max_events = (int32_t)p->max_events;
  a.seed = p->seed;
  a.n_traj = p->n_traj;
  a.traj_offset = p->traj_offset;
  a.sample_dt = p->sample_dt;
  const bool want_grid = o->grid_dev || o->grid_sum_dev;
  a.G = want_grid ? rt_grid_len(p->t_end, p->sample_dt) : 0;
  a.out = *o;
  const size_t need = bundle_workspace_bytes(net->dev, p->n_traj, ctas_per_traj);
  if (need > kNoAllocScratchBytes)
    return set_error(RT_ERR_OOM,
                     "rt_run_bundle_noalloc: %lld trajectories of %d reactions need %zu bytes of scratch, more than "
                     "the fixed %zu-byte array; use fewer trajectories per call or rt_run with a workspace",
                     (long long)p->n_traj, net->dev.M, need, kNoAllocScratchBytes);
  void *scratch = nullptr;
  if ((rc = noalloc_scratch(&scratch))) return rc;
  return launch_bundle_mapping(a, ctas_per_traj, scratch, kNoAllocScratchBytes, (cudaStream_t)stream);
}

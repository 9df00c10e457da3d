// rt_warp.cu -- warp segments per trajectory (8, 16 or 32 lanes each) for networks of up
// to 256 reactions: the single-network kernel around warp_trajectories (rt_traj_warp.cuh);
// the network is copied to shared memory once per block of four warps.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>

#include "rt_traj_warp.cuh"

namespace rt {

constexpr int kWarpBlock = 128;  // 4 warps per block

static size_t warp_moment_bytes(const RunArgs &a) {
  if (!a.out.grid_sum_dev) return 0;
  const size_t b = (size_t)a.G * a.net.N * 16 + (size_t)a.G * 8;
  return b <= 64 * 1024 ? b : 0;
}

// Eight channels per lane need about 150 registers; bounding them to 128 keeps four blocks
// (16 warps) per SM.
template <int R, int G, bool LL>
__global__ void __launch_bounds__(kWarpBlock, R >= 8 ? 4 : 1)
    k_ens_warp(const RunArgs A, const int tend_finite, const int use_mom) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int S = 32 / G;  // trajectories per warp
  const DevNet &d = A.net;
  const int M = d.M, N = d.N, nv = d.n_vnz;
  const uint8_t *depg = G == 8 ? d.depw8 : G == 16 ? d.depw16 : d.depw;
  // carve: c[M], rd[M], vl[nv], moments, vp[M+1], dep[M*G], X[warps * S][N]
  double *s_c = (double *)smem;
  int2 *s_rd = (int2 *)(s_c + M);
  int2 *s_vl = s_rd + M;
  unsigned long long *s_mom = (unsigned long long *)(s_vl + nv);
  const int64_t GN = A.G * N;
  const int64_t nmom = use_mom ? 2 * GN + A.G : 0;
  int *s_vp = (int *)(s_mom + nmom);
  uint8_t *s_dep = (uint8_t *)(s_vp + M + 1);
  int *s_X = (int *)(s_dep + (((size_t)M * G + 15) & ~(size_t)15));
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    s_c[i] = d.c[i];
    s_rd[i] = d.rdesc[i];
  }
  for (int i = threadIdx.x; i < nv; i += blockDim.x) s_vl[i] = d.vlist[i];
  for (int i = threadIdx.x; i <= M; i += blockDim.x) s_vp[i] = d.vptr[i];
  for (int i = threadIdx.x; i < M * G; i += blockDim.x) s_dep[i] = depg[i];
  for (int64_t i = threadIdx.x; i < nmom; i += blockDim.x) s_mom[i] = 0ull;
  __syncthreads();
  const WarpNet net{M, N, nv, s_rd, s_c, s_vp, s_vl, s_dep};
  const int warp = threadIdx.x >> 5;
  const int64_t j0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * S;
  if (j0 < A.n_traj)
    warp_trajectories<R, G, LL>(A, net, s_X + warp * S * N, use_mom ? s_mom : nullptr, j0, tend_finite);
  if (use_mom) {
    __syncthreads();
    for (int64_t i = threadIdx.x; i < GN; i += blockDim.x) {
      if (s_mom[i]) atomicAdd((unsigned long long *)A.out.grid_sum_dev + i, s_mom[i]);
      if (s_mom[GN + i] && A.out.grid_sumsq_dev) atomicAdd((unsigned long long *)A.out.grid_sumsq_dev + i, s_mom[GN + i]);
    }
    if (A.out.grid_count_dev)
      for (int64_t i = threadIdx.x; i < A.G; i += blockDim.x)
        if (s_mom[2 * GN + i]) atomicAdd((unsigned long long *)A.out.grid_count_dev + i, s_mom[2 * GN + i]);
  }
}

// ---------------------------------------------------------------------------------
// Shared steps of the warp-per-trajectory kernels below (channel k in lane k % 32, slot
// k / 32; X of the trajectory in shared memory, read and written by the warp's lanes).
// ---------------------------------------------------------------------------------

// X = X0 (the warp's lanes); true if a count is negative (every lane gets the answer)
__device__ __forceinline__ bool warp_load_x0(const RunArgs &A, int64_t j, int *X, int lane) {
  const int N = A.net.N;
  const int32_t *x0 = A.x0 + (A.per_traj_x0 ? j * (int64_t)N : 0);
  bool badl = false;
  for (int sp = lane; sp < N; sp += 32) {
    const int v = x0[sp];
    X[sp] = v;
    badl |= v < 0;
  }
  const bool bad = __any_sync(0xFFFFFFFFu, badl);
  __syncwarp();
  return bad;
}

// grid point gidx from the current X (-1 where unknown), into the per-trajectory grid and/or the
// moment sums
__device__ __forceinline__ void warp_record(const RunArgs &A, int64_t j, const int *X, int lane, int64_t gidx,
                                            bool known) {
  const int N = A.net.N;
  if (A.out.grid_dev) {
    int32_t *gp = A.out.grid_dev + (j * A.G + gidx) * N;
    for (int sp = lane; sp < N; sp += 32) gp[sp] = known ? X[sp] : -1;
  }
  if (!known || !A.out.grid_sum_dev) return;
  for (int sp = lane; sp < N; sp += 32) {
    const long long x = X[sp];
    atomicAdd((unsigned long long *)(A.out.grid_sum_dev + gidx * N + sp), (unsigned long long)x);
    if (A.out.grid_sumsq_dev)
      atomicAdd((unsigned long long *)(A.out.grid_sumsq_dev + gidx * N + sp), (unsigned long long)(x * x));
  }
  if (lane == 0 && A.out.grid_count_dev) atomicAdd((unsigned long long *)(A.out.grid_count_dev + gidx), 1ull);
}

// would firing reaction kb push a count out of [0, INT32_MAX]? (every lane gets the answer)
__device__ __forceinline__ bool warp_overflow(const DevNet &d, int kb, const int *X, int lane) {
  bool over = false;
  for (int i = d.vptr[kb] + lane; i < d.vptr[kb + 1]; i += 32) {
    const int2 e = d.vlist[i];
    const long long nx = (long long)X[e.x] + e.y;
    over |= (nx > INT_MAX) | (nx < 0);
  }
  return __any_sync(0xFFFFFFFFu, over);
}

// X += v_kb (after every read of the pre-event X; the species of one reaction are distinct)
__device__ __forceinline__ void warp_fire(const DevNet &d, int kb, int *X, int lane) {
  __syncwarp();
  for (int i = d.vptr[kb] + lane; i < d.vptr[kb + 1]; i += 32) {
    const int2 e = d.vlist[i];
    X[e.x] += e.y;
  }
  __syncwarp();
}

// the per-trajectory outputs after the run (internal times already final)
template <int R>
__device__ __forceinline__ void warp_write_outputs(const RunArgs &A, int64_t j, const int *X, int lane, bool bad,
                                                   const double (&T)[R], const int32_t (&n)[R], double ll, int32_t ev,
                                                   int status, double t) {
  const int M = A.net.M, N = A.net.N;
  if (A.out.t_internal_dev)
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (lane + 32 * r < M) A.out.t_internal_dev[j * M + lane + 32 * r] = T[r];
  if (A.out.loglik_dev) {
    const double sT = warp_sum_T_in_order<R, 32>(T, M, true);  // sum_k T_k in k order
    if (lane == 0) A.out.loglik_dev[j] = bad ? __longlong_as_double(0x7FF8000000000000ll) : __dsub_rn(ll, sT);
  }
  if (A.out.counts_dev)
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (lane + 32 * r < M) A.out.counts_dev[j * M + lane + 32 * r] = n[r];
  if (A.out.x_final_dev)
    for (int sp = lane; sp < N; sp += 32) A.out.x_final_dev[j * N + sp] = X[sp];
  trace_tail(A.out, j, ev, lane, 32);
  if (lane == 0) {
    if (A.out.n_events_dev) A.out.n_events_dev[j] = ev;
    if (A.out.status_dev) A.out.status_dev[j] = status;
    if (A.out.t_last_dev) A.out.t_last_dev[j] = t;
  }
}

// ---------------------------------------------------------------------------------
// Time-dependent rates c_k(t) = c_k (1 + beta_k t) (Sec. 6, Eq. 29) for networks of up to
// 256 reactions: a warp per trajectory, channel k in lane k % 32, register slot k / 32.
// Every waiting time is the root of its channel's own integral, computed exactly (the
// float-bound filter of the constant-rate routines is for plain quotients only); a warp
// shuffle on (waiting time bits, channel) gives the smallest, smallest index on ties.  The
// same operations, in the same order per channel, as the one-thread routine, so the results
// are bit-identical to it and to the oracle.
// ---------------------------------------------------------------------------------
template <int R, bool LL>
__global__ void __launch_bounds__(kWarpBlock) k_ens_tdep_warp(const RunArgs A, const int tend_finite) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr unsigned FULL = 0xFFFFFFFFu;
  const DevNet &d = A.net;
  const int M = d.M, N = d.N;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t j = (int64_t)blockIdx.x * (kWarpBlock / 32) + warp;
  if (j >= A.n_traj) return;  // whole warps only; the kernel has no block-wide barrier
  int *X = (int *)smem + (size_t)warp * N;
  auto xat = [&](int sp) { return X[sp]; };
  const uint64_t g = (uint64_t)(A.traj_offset + j);
  const bool bad = warp_load_x0(A, j, X, lane);
  double P[R], T[R], a[R], bt[R];
  int32_t n[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int k = lane + 32 * r;
    n[r] = 0;
    T[r] = 0.0;
    P[r] = 0.0;
    a[r] = 0.0;
    bt[r] = k < M ? d.beta[k] : 0.0;
    if (!bad && k < M) {
      P[r] = exp1_draw(A.seed, g, (uint32_t)k, 0u, A.stream_id);
      a[r] = propensity(d.rdesc[k], d.c[k], xat);
    }
  }
  int status = bad ? RT_TRAJ_BAD_X0 : RT_TRAJ_TEND;
  double t = 0.0, ll = 0.0;
  int32_t ev = 0;
  int64_t gi = 0;
  double next_g = 0.0;
  auto record = [&](int64_t gidx, bool known) { warp_record(A, j, X, lane, gidx, known); };
  if (!bad) {
    const int64_t tend_bits = dbits(A.t_end);
    for (;;) {
      int64_t best = kInfBits;
      int kb = INT_MAX;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int k = lane + 32 * r;
        if (k < M && dbits(a[r]) != 0) {
          const int64_t wb = dbits(tdep_wait(a[r], bt[r], __dsub_rn(P[r], T[r]), t));
          if (wb < best) {
            best = wb;
            kb = k;
          }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const int64_t w2 = __shfl_xor_sync(FULL, best, o);
        const int k2 = __shfl_xor_sync(FULL, kb, o);
        if (w2 < best || (w2 == best && k2 < kb)) {
          best = w2;
          kb = k2;
        }
      }
      if (kb == INT_MAX) {
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
      if (warp_overflow(d, kb, X, lane)) {
        status = RT_TRAJ_OVERFLOW;
        break;
      }
      while (gi < A.G && dbits(next_g) < dbits(tn)) {
        record(gi, true);
        ++gi;
        next_g = __dmul_rn(__ll2double_rn(gi), A.sample_dt);
      }
      const double tprev = t;
      t = tn;
      if (lane == 0) trace_event(A.out, j, ev, kb, tn);
      const int ol = kb & 31, os = kb >> 5;
      const double a_mu = __shfl_sync(FULL, pick<R>(a, os), ol);
      const double b_mu = __shfl_sync(FULL, pick<R>(bt, os), ol);
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (lane + 32 * r < M) T[r] = __dadd_rn(T[r], __dmul_rn(a[r], tdep_integral(bt[r], tprev, dmin)));
      if (LL && lane == 0) ll = __dadd_rn(ll, rt_ln(__dmul_rn(a_mu, __dadd_rn(1.0, __dmul_rn(b_mu, t)))));
      warp_fire(d, kb, X, lane);
      if (lane == ol) {
        int32_t nmu = 0;
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (r == os) {
            n[r] += 1;
            nmu = n[r];
          }
        const double E = exp1_draw(A.seed, g, (uint32_t)kb, (uint32_t)nmu, A.stream_id);
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (r == os) P[r] = __dadd_rn(P[r], E);
      }
      ++ev;
      const uint32_t dm = d.depw[(size_t)kb * 32 + lane];
#pragma unroll
      for (int r = 0; r < R; ++r)
        if ((dm >> r) & 1u) a[r] = propensity(d.rdesc[lane + 32 * r], d.c[lane + 32 * r], xat);
    }
  }
  const bool known = status == RT_TRAJ_TEND || status == RT_TRAJ_ABSORBED;
  for (; gi < A.G; ++gi) record(gi, known);
  if (A.out.loglik_dev || A.out.t_internal_dev) {
    if (known && tend_finite && !bad) {
      const double rest = __dsub_rn(A.t_end, t);
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (lane + 32 * r < M) T[r] = __dadd_rn(T[r], __dmul_rn(a[r], tdep_integral(bt[r], t, rest)));
    }
  }
  warp_write_outputs<R>(A, j, X, lane, bad, T, n, ll, ev, status, t);
}

template <int R>
static cudaError_t launch_tdep_r(const RunArgs &a, cudaStream_t s, int tend_finite) {
  const size_t smem = (size_t)a.net.N * 4 * (kWarpBlock / 32);
  const unsigned grid = (unsigned)((a.n_traj + kWarpBlock / 32 - 1) / (kWarpBlock / 32));
  auto kern = a.out.loglik_dev ? k_ens_tdep_warp<R, true> : k_ens_tdep_warp<R, false>;
  raise_smem_limit((const void *)kern, smem);
  kern<<<grid, kWarpBlock, smem, s>>>(a, tend_finite);
  return cudaGetLastError();
}

int launch_tdep_warp_mapping(const RunArgs &a, int lanes_per_traj, cudaStream_t s) {
  if (a.n_traj == 0) return RT_OK;
  const int M = a.net.M;
  if (lanes_per_traj != 0 && lanes_per_traj != 32)
    return set_error(RT_ERR_UNSUPPORTED, "time-dependent rates on the warp mapping use 32 lanes per trajectory");
  if (M > 256 || !a.net.depw || !a.net.beta)
    return set_error(RT_ERR_UNSUPPORTED, "time-dependent rates run on the warp mapping with M <= 256 (got %d)", M);
  if ((size_t)a.net.N * 4 * (kWarpBlock / 32) > 200 * 1024)
    return set_error(RT_ERR_UNSUPPORTED, "warp mapping: too many species for shared memory");
  if ((a.n_traj + kWarpBlock / 32 - 1) / (kWarpBlock / 32) > INT_MAX)
    return set_error(RT_ERR_UNSUPPORTED, "warp mapping: too many trajectories for one launch");
  const int tf = std::isfinite(a.t_end) ? 1 : 0;
  const int need = (M + 31) / 32;
  cudaError_t e;
  if (need <= 1) e = launch_tdep_r<1>(a, s, tf);
  else if (need <= 2) e = launch_tdep_r<2>(a, s, tf);
  else if (need <= 4) e = launch_tdep_r<4>(a, s, tf);
  else e = launch_tdep_r<8>(a, s, tf);
  if (e != cudaSuccess) return set_error(RT_ERR_CUDA, "time-dependent warp kernel launch: %s", cudaGetErrorString(e));
  return RT_OK;
}

// ---------------------------------------------------------------------------------
// Table 3's form ("parallel NRRTA", Sec. 5) for networks of up to 256 reactions: a warp per
// trajectory, channel k in lane k % 32, register slot k / 32 -- the paper's own GPU layout of a
// thread per reaction channel with a parallel reduction for the next reaction.  Per event every
// propensity is recomputed (no dependency graph) and every other relative waiting time is
// rescaled, w_k = (p_k / a_k)(w_k - dt); the fired channel draws w_mu = E / a_mu; a channel whose
// propensity drops to 0 keeps its remaining internal time p_k (w_k - dt) until it can fire again.
// The per-channel operations and their order are those of the one-thread routine.
// ---------------------------------------------------------------------------------
template <int R, bool LL>
__global__ void __launch_bounds__(kWarpBlock) k_ens_rescaled_warp(const RunArgs A, const int tend_finite) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr unsigned FULL = 0xFFFFFFFFu;
  const DevNet &d = A.net;
  const int M = d.M, N = d.N;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t j = (int64_t)blockIdx.x * (kWarpBlock / 32) + warp;
  if (j >= A.n_traj) return;  // whole warps only; the kernel has no block-wide barrier
  const bool want_T = A.out.loglik_dev || A.out.t_internal_dev;
  int *X = (int *)smem + (size_t)warp * N;
  auto xat = [&](int sp) { return X[sp]; };
  const uint64_t g = (uint64_t)(A.traj_offset + j);
  const bool bad = warp_load_x0(A, j, X, lane);
  double w[R], T[R], a[R];
  int32_t n[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int k = lane + 32 * r;
    n[r] = 0;
    T[r] = 0.0;
    w[r] = 0.0;
    a[r] = 0.0;
    if (!bad && k < M) {
      const double E = exp1_draw(A.seed, g, (uint32_t)k, 0u, A.stream_id);
      a[r] = propensity(d.rdesc[k], d.c[k], xat);
      w[r] = dbits(a[r]) != 0 ? __ddiv_rn(E, a[r]) : E;  // frozen: the remaining internal time
    }
  }
  int status = bad ? RT_TRAJ_BAD_X0 : RT_TRAJ_TEND;
  double t = 0.0, ll = 0.0;
  int32_t ev = 0;
  int64_t gi = 0;
  double next_g = 0.0;
  auto record = [&](int64_t gidx, bool known) { warp_record(A, j, X, lane, gidx, known); };
  if (!bad) {
    const int64_t tend_bits = dbits(A.t_end);
    for (;;) {
      // the smallest waiting time (ties: smallest index); frozen channels cannot fire
      int64_t best = kInfBits;
      int kb = INT_MAX;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int k = lane + 32 * r;
        if (k < M && dbits(a[r]) != 0 && dbits(w[r]) < best) {
          best = dbits(w[r]);
          kb = k;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const int64_t w2 = __shfl_xor_sync(FULL, best, o);
        const int k2 = __shfl_xor_sync(FULL, kb, o);
        if (w2 < best || (w2 == best && k2 < kb)) {
          best = w2;
          kb = k2;
        }
      }
      if (kb == INT_MAX) {
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
      if (warp_overflow(d, kb, X, lane)) {
        status = RT_TRAJ_OVERFLOW;
        break;
      }
      while (gi < A.G && dbits(next_g) < dbits(tn)) {
        record(gi, true);
        ++gi;
        next_g = __dmul_rn(__ll2double_rn(gi), A.sample_dt);
      }
      t = tn;
      if (lane == 0) trace_event(A.out, j, ev, kb, tn);
      const int ol = kb & 31, os = kb >> 5;
      const double a_mu = __shfl_sync(FULL, pick<R>(a, os), ol);
      if (want_T)
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (lane + 32 * r < M) T[r] = __dadd_rn(T[r], __dmul_rn(a[r], dmin));
      if (LL && lane == 0) ll = __dadd_rn(ll, rt_ln(a_mu));
      warp_fire(d, kb, X, lane);
      double E = 0.0;
      if (lane == ol) {
        int32_t nmu = 0;
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (r == os) {
            n[r] += 1;
            nmu = n[r];
          }
        E = exp1_draw(A.seed, g, (uint32_t)kb, (uint32_t)nmu, A.stream_id);
      }
      ++ev;
      // recalculate every propensity; rescale every other waiting time; the fired one redraws
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int k = lane + 32 * r;
        if (k < M) {
          const double an = propensity(d.rdesc[k], d.c[k], xat);
          if (k == kb) {
            w[r] = dbits(an) != 0 ? __ddiv_rn(E, an) : E;
          } else if (dbits(a[r]) != 0) {
            const double rem = __dsub_rn(w[r], dmin);
            w[r] = dbits(an) != 0 ? __dmul_rn(__ddiv_rn(a[r], an), rem) : __dmul_rn(a[r], rem);
          } else if (dbits(an) != 0) {
            w[r] = __ddiv_rn(w[r], an);  // a frozen channel resumes
          }
          a[r] = an;
        }
      }
    }
  }
  const bool known = status == RT_TRAJ_TEND || status == RT_TRAJ_ABSORBED;
  for (; gi < A.G; ++gi) record(gi, known);
  if (want_T) {
    if (known && tend_finite && !bad) {
      const double rest = __dsub_rn(A.t_end, t);
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (lane + 32 * r < M) T[r] = __dadd_rn(T[r], __dmul_rn(a[r], rest));
    }
  }
  warp_write_outputs<R>(A, j, X, lane, bad, T, n, ll, ev, status, t);
}

template <int R>
static cudaError_t launch_rescaled_r(const RunArgs &a, cudaStream_t s, int tend_finite) {
  const size_t smem = (size_t)a.net.N * 4 * (kWarpBlock / 32);
  const unsigned grid = (unsigned)((a.n_traj + kWarpBlock / 32 - 1) / (kWarpBlock / 32));
  auto kern = a.out.loglik_dev ? k_ens_rescaled_warp<R, true> : k_ens_rescaled_warp<R, false>;
  raise_smem_limit((const void *)kern, smem);
  kern<<<grid, kWarpBlock, smem, s>>>(a, tend_finite);
  return cudaGetLastError();
}

int launch_rescaled_warp_mapping(const RunArgs &a, int lanes_per_traj, cudaStream_t s) {
  if (a.n_traj == 0) return RT_OK;
  const int M = a.net.M;
  if (lanes_per_traj != 0 && lanes_per_traj != 32)
    return set_error(RT_ERR_UNSUPPORTED, "Table 3's form on the warp mapping uses 32 lanes per trajectory");
  if (M > 256) return set_error(RT_ERR_UNSUPPORTED, "Table 3's form runs on the warp mapping with M <= 256 (got %d)", M);
  if ((size_t)a.net.N * 4 * (kWarpBlock / 32) > 200 * 1024)
    return set_error(RT_ERR_UNSUPPORTED, "warp mapping: too many species for shared memory");
  if ((a.n_traj + kWarpBlock / 32 - 1) / (kWarpBlock / 32) > INT_MAX)
    return set_error(RT_ERR_UNSUPPORTED, "warp mapping: too many trajectories for one launch");
  const int tf = std::isfinite(a.t_end) ? 1 : 0;
  const int need = (M + 31) / 32;
  cudaError_t e;
  if (need <= 1) e = launch_rescaled_r<1>(a, s, tf);
  else if (need <= 2) e = launch_rescaled_r<2>(a, s, tf);
  else if (need <= 4) e = launch_rescaled_r<4>(a, s, tf);
  else e = launch_rescaled_r<8>(a, s, tf);
  if (e != cudaSuccess) return set_error(RT_ERR_CUDA, "Table 3 warp kernel launch: %s", cudaGetErrorString(e));
  return RT_OK;
}

int warp_mapping_max_m() { return 256; }

static size_t warp_net_bytes(const DevNet &d, int G) {
  return (size_t)d.M * (8 + 8) + (size_t)d.n_vnz * 8 + (size_t)(d.M + 1) * 4 + (((size_t)d.M * G + 15) & ~(size_t)15);
}

template <int R, int G>
static cudaError_t launch_rg(const RunArgs &a, cudaStream_t s, int tend_finite) {
  constexpr int wpb = kWarpBlock / 32, S = 32 / G;
  const size_t mom = warp_moment_bytes(a);
  const size_t smem = warp_net_bytes(a.net, G) + mom + (size_t)a.net.N * 4 * wpb * S;
  const int64_t per_block = (int64_t)wpb * S;
  const unsigned grid = (unsigned)((a.n_traj + per_block - 1) / per_block);
  auto kern = a.out.loglik_dev ? k_ens_warp<R, G, true> : k_ens_warp<R, G, false>;
  raise_smem_limit((const void *)kern, smem);
  kern<<<grid, kWarpBlock, smem, s>>>(a, tend_finite, mom ? 1 : 0);
  return cudaGetLastError();
}

// Lanes per trajectory: 8 up to 64 reactions, 16 up to 128, else 32 (at most 8 channels per lane).
static int choose_lanes(int M, int requested) {
  if (requested > 0) return requested;
  return M <= 64 ? 8 : M <= 128 ? 16 : 32;
}

int launch_warp_mapping(const RunArgs &a, int block_threads, int lanes_per_traj, cudaStream_t s) {
  (void)block_threads;
  if (a.n_traj == 0) return RT_OK;
  const int M = a.net.M;
  const int G = choose_lanes(M, lanes_per_traj);
  if (G != 8 && G != 16 && G != 32)
    return set_error(RT_ERR_INVALID_ARG, "warp mapping: lanes_per_traj must be 8, 16 or 32 (got %d)", G);
  if (M > 8 * G) return set_error(RT_ERR_UNSUPPORTED, "warp mapping with %d lanes per trajectory supports M <= %d (got %d)",
                                  G, 8 * G, M);
  const uint8_t *dep = G == 8 ? a.net.depw8 : G == 16 ? a.net.depw16 : a.net.depw;
  if (!dep) return set_error(RT_ERR_UNSUPPORTED, "warp mapping: no dependency table for %d lanes", G);
  const size_t smem = warp_net_bytes(a.net, G) + (size_t)a.net.N * 4 * (kWarpBlock / 32) * (32 / G);
  if (smem > 200 * 1024) return set_error(RT_ERR_UNSUPPORTED, "warp mapping: network too large for shared memory");
  const int64_t per_block = (int64_t)(kWarpBlock / 32) * (32 / G);
  if ((a.n_traj + per_block - 1) / per_block > INT_MAX)
    return set_error(RT_ERR_UNSUPPORTED, "warp mapping: too many trajectories for one launch");
  const int tf = std::isfinite(a.t_end) ? 1 : 0;
  const int need = (M + G - 1) / G;
  cudaError_t e;
  if (G == 32) {
    if (need <= 1) e = launch_rg<1, 32>(a, s, tf);
    else if (need <= 2) e = launch_rg<2, 32>(a, s, tf);
    else if (need <= 4) e = launch_rg<4, 32>(a, s, tf);
    else e = launch_rg<8, 32>(a, s, tf);
  } else if (G == 16) {
    if (need <= 4) e = launch_rg<4, 16>(a, s, tf);
    else e = launch_rg<8, 16>(a, s, tf);
  } else {
    if (need <= 2) e = launch_rg<2, 8>(a, s, tf);
    else if (need <= 4) e = launch_rg<4, 8>(a, s, tf);
    else e = launch_rg<8, 8>(a, s, tf);
  }
  if (e != cudaSuccess) return set_error(RT_ERR_CUDA, "warp kernel launch: %s", cudaGetErrorString(e));
  return RT_OK;
}

}  // namespace rt

// rt_warp.cu -- one warp per trajectory for networks of up to 256 reactions: the
// single-network kernel around warp_trajectory (rt_traj_warp.cuh); the network is
// copied to shared memory once per block of four warps.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>

#include "rt_traj_warp.cuh"

namespace rt {

constexpr int kWarpBlock = 128;  // 4 trajectories per block

static size_t warp_net_bytes(const DevNet &d) {
  return (size_t)d.M * (8 + 8) + (size_t)d.n_vnz * 8 + (size_t)(d.M + 1) * 4 + (((size_t)d.M * 32 + 15) & ~(size_t)15);
}

static size_t warp_moment_bytes(const RunArgs &a) {
  if (!a.out.grid_sum_dev) return 0;
  const size_t b = (size_t)a.G * a.net.N * 16 + (size_t)a.G * 8;
  return b <= 64 * 1024 ? b : 0;
}

template <int R, bool LL>
__global__ void __launch_bounds__(kWarpBlock) k_ens_warp(const RunArgs A, const int tend_finite, const int use_mom) {
  extern __shared__ __align__(16) unsigned char smem[];
  const DevNet &d = A.net;
  const int M = d.M, N = d.N, nv = d.n_vnz;
  // carve: c[M], rd[M], vl[nv], moments, vp[M+1], dep[M*32], X[warps][N]
  double *s_c = (double *)smem;
  int2 *s_rd = (int2 *)(s_c + M);
  int2 *s_vl = s_rd + M;
  unsigned long long *s_mom = (unsigned long long *)(s_vl + nv);
  const int64_t GN = A.G * N;
  const int64_t nmom = use_mom ? 2 * GN + A.G : 0;
  int *s_vp = (int *)(s_mom + nmom);
  uint8_t *s_dep = (uint8_t *)(s_vp + M + 1);
  int *s_X = (int *)(s_dep + (((size_t)M * 32 + 15) & ~(size_t)15));
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    s_c[i] = d.c[i];
    s_rd[i] = d.rdesc[i];
  }
  for (int i = threadIdx.x; i < nv; i += blockDim.x) s_vl[i] = d.vlist[i];
  for (int i = threadIdx.x; i <= M; i += blockDim.x) s_vp[i] = d.vptr[i];
  for (int i = threadIdx.x; i < M * 32; i += blockDim.x) s_dep[i] = d.depw[i];
  for (int64_t i = threadIdx.x; i < nmom; i += blockDim.x) s_mom[i] = 0ull;
  __syncthreads();
  const WarpNet net{M, N, nv, s_rd, s_c, s_vp, s_vl, s_dep};
  const int warp = threadIdx.x >> 5;
  const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (j < A.n_traj) warp_trajectory<R, LL>(A, net, s_X + warp * N, use_mom ? s_mom : nullptr, j, tend_finite);
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

int warp_mapping_max_m() { return 256; }

template <int R>
static cudaError_t launch_r(const RunArgs &a, cudaStream_t s, int tend_finite) {
  const int wpb = kWarpBlock / 32;
  const size_t mom = warp_moment_bytes(a);
  const size_t smem = warp_net_bytes(a.net) + mom + (size_t)a.net.N * 4 * wpb;
  const unsigned grid = (unsigned)((a.n_traj + wpb - 1) / wpb);
  auto kern = a.out.loglik_dev ? k_ens_warp<R, true> : k_ens_warp<R, false>;
  raise_smem_limit((const void *)kern, smem);
  kern<<<grid, kWarpBlock, smem, s>>>(a, tend_finite, mom ? 1 : 0);
  return cudaGetLastError();
}

int launch_warp_mapping(const RunArgs &a, int block_threads, cudaStream_t s) {
  (void)block_threads;
  if (a.n_traj == 0) return RT_OK;
  if (a.net.M > 256 || !a.net.depw) return set_error(RT_ERR_UNSUPPORTED, "warp mapping supports M <= 256 (got %d)", a.net.M);
  const size_t smem = warp_net_bytes(a.net) + (size_t)a.net.N * 4 * (kWarpBlock / 32);
  if (smem > 200 * 1024) return set_error(RT_ERR_UNSUPPORTED, "warp mapping: network too large for shared memory");
  const int tf = std::isfinite(a.t_end) ? 1 : 0;
  cudaError_t e;
  if (a.net.M <= 32) e = launch_r<1>(a, s, tf);
  else if (a.net.M <= 64) e = launch_r<2>(a, s, tf);
  else if (a.net.M <= 128) e = launch_r<4>(a, s, tf);
  else e = launch_r<8>(a, s, tf);
  if (e != cudaSuccess) return set_error(RT_ERR_CUDA, "warp kernel launch: %s", cudaGetErrorString(e));
  return RT_OK;
}

}  // namespace rt

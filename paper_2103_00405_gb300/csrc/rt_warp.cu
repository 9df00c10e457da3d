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

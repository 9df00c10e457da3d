// rt_block.cu -- one thread block per trajectory (RT_MAP_BLOCK): the single-network
// kernel around block_trajectory (rt_traj_block.cuh), for networks of up to
// 8 * block_threads reactions with all per-channel state in registers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "rt_traj_block.cuh"

namespace rt {

// Two resident blocks per SM (64 registers): one trajectory's block waits at barriers and on
// dependent loads for much of each event, and a second one fills that time (measured
// 1.09-1.14x on 600- to 4000-reaction networks).
template <int R, bool LL>
__global__ void __launch_bounds__(512, 2) k_ens_block(const RunArgs A, const int tend_finite) {
  extern __shared__ __align__(16) unsigned char smem[];
  const BlockScratch S = carve_block_scratch(smem, A.net.M, A.net.N, blockDim.x);
  const BlockNet net{A.net.M, A.net.N, A.net.rdesc, A.net.c, A.net.vptr, A.net.vlist, A.net.sptr, A.net.slist,
                     A.net.dptr, A.net.dlist};
  for (int64_t j = blockIdx.x; j < A.n_traj; j += gridDim.x) block_trajectory<R, LL>(A, net, S, j, tend_finite);
}

int block_mapping_max_m() { return 4096; }

template <int R>
static cudaError_t launch_r(const RunArgs &a, int B, cudaStream_t s, int tf) {
  const size_t smem = block_scratch_bytes(a.net.M, a.net.N, B);
  auto kern = a.out.loglik_dev ? k_ens_block<R, true> : k_ens_block<R, false>;
  raise_smem_limit((const void *)kern, smem);
  int per_sm = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, B, smem);
  const int64_t grid = std::min<int64_t>(a.n_traj, (int64_t)std::max(1, per_sm) * sms);
  kern<<<(unsigned)grid, B, smem, s>>>(a, tf);
  return cudaGetLastError();
}

int launch_block_mapping(const RunArgs &a, int block_threads, cudaStream_t s) {
  if (a.n_traj == 0) return RT_OK;
  const int M = a.net.M;
  int B = block_threads;
  if (B <= 0) B = std::min(512, std::max(64, ((M + 7) / 8 + 31) / 32 * 32));
  if (B % 32 || B > 512) return set_error(RT_ERR_INVALID_ARG, "block mapping: block_threads must be a multiple of 32 <= 512");
  const int R = (M + B - 1) / B;
  if (R > 8) return set_error(RT_ERR_UNSUPPORTED, "block mapping supports M <= 8 * block_threads (M = %d)", M);
  if (block_scratch_bytes(M, a.net.N, B) > 200 * 1024)
    return set_error(RT_ERR_UNSUPPORTED, "block mapping: %d species do not fit in shared memory", a.net.N);
  const int tf = std::isfinite(a.t_end) ? 1 : 0;
  cudaError_t e;
  if (R <= 1) e = launch_r<1>(a, B, s, tf);
  else if (R <= 2) e = launch_r<2>(a, B, s, tf);
  else if (R <= 4) e = launch_r<4>(a, B, s, tf);
  else e = launch_r<8>(a, B, s, tf);
  if (e != cudaSuccess) return set_error(RT_ERR_CUDA, "block kernel launch: %s", cudaGetErrorString(e));
  return RT_OK;
}

}  // namespace rt

// rt_moments.cuh -- per-block ensemble moment tables for the one-thread-per-trajectory
// kernels.
//
// With grid="moments" a launch returns, per grid point g and species s, the exact
// integer sums over trajectories of X_s(t_g) and X_s(t_g)^2, and the number of
// trajectories whose state at t_g is known.  2^20 trajectories adding into the same
// few thousand global counters would serialise on atomics, so each block adds into a
// table in shared memory -- sum[rows][N], sumsq[rows][N], count[rows] -- flushed to
// global memory once per block.  A large table would cap the blocks per SM, so it is
// split across a thread-block cluster of `cl` blocks: grid point g lives in block
// g % cl at row g / cl, reached through distributed shared memory.
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "rt_internal.h"

namespace rt {

struct MomTable {
  unsigned long long *mom;  // this block's share: sum[rows][N], sumsq[rows][N], count[rows]
  int cl;                   // blocks sharing one table (1: no cluster)
  int64_t rows;             // grid points per block share
};

__device__ __forceinline__ MomTable mom_table(unsigned long long *base, int64_t G, int mom_cl) {
  MomTable t;
  t.mom = base;
  t.cl = mom_cl > 0 ? mom_cl : 1;
  t.rows = (G + t.cl - 1) / t.cl;
  return t;
}

// Adds the state x(0..N-1) of one trajectory at grid point gidx.
template <typename XAt>
__device__ __forceinline__ void mom_add(const MomTable &t, int64_t gidx, int N, XAt x) {
  unsigned long long *m = t.mom;
  int64_t row = gidx;
  if (t.cl > 1) {
    m = cooperative_groups::this_cluster().map_shared_rank(t.mom, (unsigned)(gidx % t.cl));
    row = gidx / t.cl;
  }
  const int64_t GNl = t.rows * N;
  for (int s = 0; s < N; ++s) {
    const long long v = x(s);
    atomicAdd(m + row * N + s, (unsigned long long)v);
    atomicAdd(m + GNl + row * N + s, (unsigned long long)(v * v));
  }
  atomicAdd(m + 2 * GNl + row, 1ull);
}

// Zeroes this block's share (all threads), then waits until every share of the
// cluster is zeroed.
__device__ __forceinline__ void mom_zero_and_sync(const MomTable &t, int N) {
  const int64_t n = 2 * t.rows * N + t.rows;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) t.mom[i] = 0ull;
  if (t.cl > 1) cooperative_groups::this_cluster().sync();
  else __syncthreads();
}

// Waits until every block of the cluster has finished adding, then adds this
// block's share into the global sums (all threads).
__device__ __forceinline__ void mom_sync_and_flush(const MomTable &t, const RunArgs &A) {
  const int N = A.net.N;
  unsigned rank = 0;
  if (t.cl > 1) {
    cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
    cl.sync();
    rank = cl.block_rank();
  } else {
    __syncthreads();
  }
  const int64_t GNl = t.rows * N;
  for (int64_t i = threadIdx.x; i < GNl; i += blockDim.x) {
    const int64_t g = (i / N) * t.cl + rank;
    if (g >= A.G) continue;
    const int64_t o = g * N + i % N;
    const unsigned long long v = t.mom[i], q = t.mom[GNl + i];
    if (v) atomicAdd((unsigned long long *)A.out.grid_sum_dev + o, v);
    if (q && A.out.grid_sumsq_dev) atomicAdd((unsigned long long *)A.out.grid_sumsq_dev + o, q);
  }
  if (A.out.grid_count_dev)
    for (int64_t i = threadIdx.x; i < t.rows; i += blockDim.x) {
      const int64_t g = i * t.cl + rank;
      const unsigned long long v = t.mom[2 * GNl + i];
      if (g < A.G && v) atomicAdd((unsigned long long *)A.out.grid_count_dev + g, v);
    }
}

// Host side: the share of one block for a cluster of cl blocks, and the cluster size
// (smallest power of two <= 8 bringing the share to kMomentShare bytes; 0 if moments
// are not requested or a share would exceed kMomentMax).
constexpr size_t kMomentShare = 12 * 1024;
constexpr size_t kMomentMax = 96 * 1024;

inline size_t moment_share_bytes(const RunArgs &a, int cl) {
  const int64_t rows = (a.G + cl - 1) / cl;
  return (size_t)rows * a.net.N * 16 + (size_t)rows * 8 + 8;
}

inline int moment_cluster(const RunArgs &a) {
  if (!a.out.grid_sum_dev) return 0;
  for (int cl = 1; cl <= 8; cl *= 2)
    if (moment_share_bytes(a, cl) <= kMomentShare) return cl;
  return moment_share_bytes(a, 8) <= kMomentMax ? 8 : 0;
}

// Launch of a one-thread-per-trajectory kernel whose blocks share moment tables in
// clusters of cl blocks (cl <= 1: a plain launch); grid is a multiple of cl.
template <typename... Params, typename... Args>
cudaError_t launch_clustered(void (*kern)(Params...), unsigned grid, int block, size_t smem, cudaStream_t s, int cl,
                             Args... args) {
  raise_smem_limit((const void *)kern, smem);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl > 1 ? cl : 1;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = cl > 1 ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

}  // namespace rt

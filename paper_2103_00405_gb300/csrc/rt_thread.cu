// rt_thread.cu -- ensemble mode, one thread per trajectory: the single-network
// kernel around simulate_one (rt_traj_thread.cuh), with the network copied to
// shared memory once per block and ensemble moments accumulated in shared memory
// (split across a thread-block cluster when the table is large) before one flush
// to global memory.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <climits>

#include "rt_traj_thread.cuh"

namespace rt {

size_t thread_smem_bytes(int M, int N, int nv, int B) {
  return (size_t)(8 + 8 + 8) * M + 8 * (size_t)nv + 4 * (size_t)(M + 1) + 4 * (size_t)N * B;
}

// Per-block ensemble moments: a table sum[G][N], sumsq[G][N], count[G] in shared
// memory, flushed to global memory once per block.  A large table would cap the
// blocks per SM, so it is split across a thread-block cluster of `cl` blocks
// (grid point g in block g % cl, row g / cl) and reached through distributed shared
// memory; cl is the smallest power of two <= 8 that brings a block's share down to
// kMomentShare bytes.
constexpr size_t kMomentShare = 12 * 1024;
constexpr size_t kMomentMax = 96 * 1024;

static size_t moment_share_bytes(const RunArgs &a, int cl) {
  const int64_t rows = (a.G + cl - 1) / cl;
  return (size_t)rows * a.net.N * 16 + (size_t)rows * 8 + 8;
}

// cluster size for the moment table, 0 if moments are not requested or do not fit
static int moment_cluster(const RunArgs &a) {
  if (!a.out.grid_sum_dev) return 0;
  for (int cl = 1; cl <= 8; cl *= 2)
    if (moment_share_bytes(a, cl) <= kMomentShare) return cl;
  return moment_share_bytes(a, 8) <= kMomentMax ? 8 : 0;
}

// Minimum resident blocks: 8 (64 registers) for the exact-M kernels of M <= 4, whose
// few spills cost less than the extra warps gain; 4 for M <= 8; none above.
template <int MAXM, bool LL, bool EXACT>
__global__ void __launch_bounds__(128, EXACT ? 8 : (MAXM <= 8 ? 4 : 1))
    k_ens_thread(const RunArgs A, const int tend_finite, const int mom_cl) {
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) unsigned char smem[];
  const int M = A.net.M, N = A.net.N, nv = A.net.n_vnz;
  ThreadNet S = carve_thread_net(smem, M, nv, N, blockDim.x);
  const int smem_mom = mom_cl > 0 ? 1 : 0;
  S.mom_cl = mom_cl > 0 ? mom_cl : 1;
  S.mom_rows = (A.G + S.mom_cl - 1) / S.mom_cl;
  const int64_t GNl = S.mom_rows * N;
  if (smem_mom)
    for (int64_t i = threadIdx.x; i < 2 * GNl + S.mom_rows; i += blockDim.x) S.mom[i] = 0ull;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    S.c[i] = A.net.c[i];
    S.dep[i] = A.net.depmask[i];
    S.rd[i] = A.net.rdesc[i];
  }
  for (int i = threadIdx.x; i < nv; i += blockDim.x) S.vl[i] = A.net.vlist[i];
  for (int i = threadIdx.x; i <= M; i += blockDim.x) S.vp[i] = A.net.vptr[i];
  if (S.mom_cl > 1) cg::this_cluster().sync();  // every share is zeroed before any block adds to it
  else __syncthreads();

  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = j < A.n_traj;
  const int B = blockDim.x;
  if (active) simulate_one<MAXM, LL, EXACT>(A, S, j, B, tend_finite, smem_mom);
  if (smem_mom) {
    unsigned rank = 0;
    if (S.mom_cl > 1) {
      cg::cluster_group cl = cg::this_cluster();
      cl.sync();  // every block of the cluster has finished adding
      rank = cl.block_rank();
    } else {
      __syncthreads();
    }
    for (int64_t i = threadIdx.x; i < GNl; i += blockDim.x) {
      const int64_t g = (i / N) * S.mom_cl + rank;
      if (g >= A.G) continue;
      const int64_t o = g * N + i % N;
      const unsigned long long v = S.mom[i], q = S.mom[GNl + i];
      if (v) atomicAdd((unsigned long long *)A.out.grid_sum_dev + o, v);
      if (q && A.out.grid_sumsq_dev) atomicAdd((unsigned long long *)A.out.grid_sumsq_dev + o, q);
    }
    if (A.out.grid_count_dev)
      for (int64_t i = threadIdx.x; i < S.mom_rows; i += blockDim.x) {
        const int64_t g = i * S.mom_cl + rank;
        const unsigned long long v = S.mom[2 * GNl + i];
        if (g < A.G && v) atomicAdd((unsigned long long *)A.out.grid_count_dev + g, v);
      }
  }
}

int thread_mapping_max_m() { return 16; }

template <int MAXM, bool EXACT = false>
static cudaError_t launch_m(const RunArgs &a, int B, cudaStream_t s, int tend_finite) {
  const int cl = moment_cluster(a);
  const size_t mom = cl ? moment_share_bytes(a, cl) : 0;
  const size_t smem = ((thread_smem_bytes(a.net.M, a.net.N, a.net.n_vnz, B) + 7) & ~(size_t)7) + mom;
  unsigned grid = (unsigned)((a.n_traj + B - 1) / B);
  if (cl > 1) grid = (grid + cl - 1) / cl * cl;  // whole clusters; blocks past n_traj only hold table shares
  auto kern = a.out.loglik_dev ? k_ens_thread<MAXM, true, EXACT> : k_ens_thread<MAXM, false, EXACT>;
  if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(B);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl > 1 ? cl : 1;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = cl > 1 ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, a, tend_finite, cl);
}

int launch_thread_mapping(const RunArgs &a, int B, cudaStream_t s) {
  if (a.n_traj == 0) return RT_OK;
  if (B <= 0) B = 128;
  if (B > 128 || B % 32) return set_error(RT_ERR_INVALID_ARG, "thread mapping: block_threads must be a multiple of 32 <= 128");
  if (thread_smem_bytes(a.net.M, a.net.N, a.net.n_vnz, B) > 200 * 1024)
    return set_error(RT_ERR_UNSUPPORTED, "thread mapping: network too large for shared memory");
  const int tend_finite = isfinite(a.t_end) ? 1 : 0;
  cudaError_t e;
  if (a.net.M == 1) e = launch_m<1, true>(a, B, s, tend_finite);
  else if (a.net.M == 2) e = launch_m<2, true>(a, B, s, tend_finite);
  else if (a.net.M == 3) e = launch_m<3, true>(a, B, s, tend_finite);
  else if (a.net.M == 4) e = launch_m<4, true>(a, B, s, tend_finite);
  else if (a.net.M <= 8) e = launch_m<8>(a, B, s, tend_finite);
  else if (a.net.M <= 16) e = launch_m<16>(a, B, s, tend_finite);
  else return set_error(RT_ERR_UNSUPPORTED, "thread mapping supports M <= 16 (got %d)", a.net.M);
  if (e != cudaSuccess) return set_error(RT_ERR_CUDA, "thread kernel launch: %s", cudaGetErrorString(e));
  return RT_OK;
}

}  // namespace rt

// rt_thread.cu -- ensemble mode, one thread per trajectory: the single-network
// kernel around simulate_one (rt_traj_thread.cuh), with the network copied to
// shared memory once per block and ensemble moments accumulated per block in
// shared memory before one flush to global memory.
#include <cuda_runtime.h>

#include <climits>

#include "rt_traj_thread.cuh"

namespace rt {

size_t thread_smem_bytes(int M, int N, int nv, int B) {
  return (size_t)(8 + 8 + 8) * M + 8 * (size_t)nv + 4 * (size_t)(M + 1) + 4 * (size_t)N * B;
}

// bytes of the per-block moment table, 0 if it is not used or does not fit
static size_t moment_smem_bytes(const RunArgs &a) {
  if (!a.out.grid_sum_dev) return 0;
  const size_t b = (size_t)a.G * a.net.N * 16 + (size_t)a.G * 8 + 8;
  return b <= 96 * 1024 ? b : 0;
}

template <int MAXM, bool LL, bool EXACT>
__global__ void __launch_bounds__(128) k_ens_thread(const RunArgs A, const int tend_finite, const int smem_mom) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int M = A.net.M, N = A.net.N, nv = A.net.n_vnz;
  const ThreadNet S = carve_thread_net(smem, M, nv, N, blockDim.x);
  const int64_t GN = A.G * N;
  if (smem_mom)
    for (int64_t i = threadIdx.x; i < 2 * GN + A.G; i += blockDim.x) S.mom[i] = 0ull;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    S.c[i] = A.net.c[i];
    S.dep[i] = A.net.depmask[i];
    S.rd[i] = A.net.rdesc[i];
  }
  for (int i = threadIdx.x; i < nv; i += blockDim.x) S.vl[i] = A.net.vlist[i];
  for (int i = threadIdx.x; i <= M; i += blockDim.x) S.vp[i] = A.net.vptr[i];
  __syncthreads();

  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = j < A.n_traj;
  const int B = blockDim.x;
  if (active) simulate_one<MAXM, LL, EXACT>(A, S, j, B, tend_finite, smem_mom);
  if (smem_mom) {
    __syncthreads();
    for (int64_t i = threadIdx.x; i < GN; i += blockDim.x) {
      const unsigned long long v = S.mom[i], q = S.mom[GN + i];
      if (v) atomicAdd((unsigned long long *)A.out.grid_sum_dev + i, v);
      if (q && A.out.grid_sumsq_dev) atomicAdd((unsigned long long *)A.out.grid_sumsq_dev + i, q);
    }
    if (A.out.grid_count_dev)
      for (int64_t i = threadIdx.x; i < A.G; i += blockDim.x) {
        const unsigned long long v = S.mom[2 * GN + i];
        if (v) atomicAdd((unsigned long long *)A.out.grid_count_dev + i, v);
      }
  }
}

int thread_mapping_max_m() { return 16; }

template <int MAXM, bool EXACT = false>
static cudaError_t launch_m(const RunArgs &a, int B, cudaStream_t s, int tend_finite) {
  const size_t mom = moment_smem_bytes(a);
  const size_t smem = ((thread_smem_bytes(a.net.M, a.net.N, a.net.n_vnz, B) + 7) & ~(size_t)7) + mom;
  const unsigned grid = (unsigned)((a.n_traj + B - 1) / B);
  const int smem_mom = mom ? 1 : 0;
  if (a.out.loglik_dev) {
    auto kern = k_ens_thread<MAXM, true, EXACT>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<grid, B, smem, s>>>(a, tend_finite, smem_mom);
  } else {
    auto kern = k_ens_thread<MAXM, false, EXACT>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<grid, B, smem, s>>>(a, tend_finite, smem_mom);
  }
  return cudaGetLastError();
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

// rt_thread.cu -- ensemble mode, one thread per trajectory: the single-network
// kernel around simulate_one (rt_traj_thread.cuh), with the network copied to
// shared memory once per block and ensemble moments accumulated in shared memory
// (split across a thread-block cluster when the table is large) before one flush
// to global memory.
#include <cuda_runtime.h>

#include <climits>

#include "rt_traj_thread.cuh"

namespace rt {

size_t thread_smem_bytes(int M, int N, int nv, int B) {
  return (size_t)(8 + 8 + 8) * M + 8 * (size_t)nv + 4 * (size_t)(M + 1) + 4 * (size_t)N * B;
}

// Minimum resident blocks: 8 (64 registers) for the exact-M kernels of M <= 4, whose
// few spills cost less than the extra warps gain; 4 for M <= 8; none above.
template <int MAXM, bool LL, bool EXACT>
__global__ void __launch_bounds__(128, EXACT ? 8 : (MAXM <= 8 ? 4 : 1))
    k_ens_thread(const RunArgs A, const int tend_finite, const int mom_cl) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int M = A.net.M, N = A.net.N, nv = A.net.n_vnz;
  ThreadNet S = carve_thread_net(smem, M, nv, N, blockDim.x);
  const int smem_mom = mom_cl > 0 ? 1 : 0;
  S.mt = mom_table(S.mom, A.G, mom_cl);
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    S.c[i] = A.net.c[i];
    S.dep[i] = A.net.depmask[i];
    S.rd[i] = A.net.rdesc[i];
  }
  for (int i = threadIdx.x; i < nv; i += blockDim.x) S.vl[i] = A.net.vlist[i];
  for (int i = threadIdx.x; i <= M; i += blockDim.x) S.vp[i] = A.net.vptr[i];
  if (smem_mom) mom_zero_and_sync(S.mt, N);  // every share is zeroed before any block adds to it
  else __syncthreads();

  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = j < A.n_traj;
  const int B = blockDim.x;
  if (active) simulate_one<MAXM, LL, EXACT>(A, S, j, B, tend_finite, smem_mom);
  if (smem_mom) mom_sync_and_flush(S.mt, A);
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
  return launch_clustered(kern, grid, B, smem, s, cl, a, tend_finite, cl);
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

// ---------------------------------------------------------------------------------
// Table 3's rescaled form (RT_FORM_RESCALED), one thread per trajectory, M <= 8.
// ---------------------------------------------------------------------------------
template <int MAXM, bool LL, bool EXACT>
__global__ void __launch_bounds__(128, EXACT ? 8 : 4)
    k_ens_rescaled(const RunArgs A, const int tend_finite, const int mom_cl, const int want_T) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int M = A.net.M, N = A.net.N, nv = A.net.n_vnz;
  ThreadNet S = carve_thread_net(smem, M, nv, N, blockDim.x);
  const int smem_mom = mom_cl > 0 ? 1 : 0;
  S.mt = mom_table(S.mom, A.G, mom_cl);
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    S.c[i] = A.net.c[i];
    S.dep[i] = A.net.depmask[i];
    S.rd[i] = A.net.rdesc[i];
  }
  for (int i = threadIdx.x; i < nv; i += blockDim.x) S.vl[i] = A.net.vlist[i];
  for (int i = threadIdx.x; i <= M; i += blockDim.x) S.vp[i] = A.net.vptr[i];
  if (smem_mom) mom_zero_and_sync(S.mt, N);
  else __syncthreads();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < A.n_traj) simulate_rescaled<MAXM, LL, EXACT>(A, S, j, blockDim.x, tend_finite, smem_mom, want_T);
  if (smem_mom) mom_sync_and_flush(S.mt, A);
}

template <int MAXM, bool EXACT = false>
static cudaError_t launch_rescaled_m(const RunArgs &a, int B, cudaStream_t s, int tend_finite) {
  const int cl = moment_cluster(a);
  const size_t mom = cl ? moment_share_bytes(a, cl) : 0;
  const size_t smem = ((thread_smem_bytes(a.net.M, a.net.N, a.net.n_vnz, B) + 7) & ~(size_t)7) + mom;
  unsigned grid = (unsigned)((a.n_traj + B - 1) / B);
  if (cl > 1) grid = (grid + cl - 1) / cl * cl;
  const int want_T = (a.out.loglik_dev || a.out.t_internal_dev) ? 1 : 0;
  auto kern = a.out.loglik_dev ? k_ens_rescaled<MAXM, true, EXACT> : k_ens_rescaled<MAXM, false, EXACT>;
  return launch_clustered(kern, grid, B, smem, s, cl, a, tend_finite, cl, want_T);
}

int launch_rescaled_mapping(const RunArgs &a, int B, cudaStream_t s) {
  if (a.n_traj == 0) return RT_OK;
  if (B <= 0) B = 128;
  if (B > 128 || B % 32) return set_error(RT_ERR_INVALID_ARG, "thread mapping: block_threads must be a multiple of 32 <= 128");
  if (a.net.M > 8 || !a.net.depmask)
    return set_error(RT_ERR_UNSUPPORTED, "Table 3's rescaled form runs on the thread mapping with M <= 8 (got %d)", a.net.M);
  if (thread_smem_bytes(a.net.M, a.net.N, a.net.n_vnz, B) > 200 * 1024)
    return set_error(RT_ERR_UNSUPPORTED, "thread mapping: network too large for shared memory");
  const int tf = isfinite(a.t_end) ? 1 : 0;
  cudaError_t e;
  switch (a.net.M) {
    case 1: e = launch_rescaled_m<1, true>(a, B, s, tf); break;
    case 2: e = launch_rescaled_m<2, true>(a, B, s, tf); break;
    case 3: e = launch_rescaled_m<3, true>(a, B, s, tf); break;
    case 4: e = launch_rescaled_m<4, true>(a, B, s, tf); break;
    default: e = launch_rescaled_m<8>(a, B, s, tf); break;
  }
  if (e != cudaSuccess) return set_error(RT_ERR_CUDA, "rescaled-form kernel launch: %s", cudaGetErrorString(e));
  return RT_OK;
}

// ---------------------------------------------------------------------------------
// Time-dependent rates (networks with rate slopes), one thread per trajectory, M <= 16.
// ---------------------------------------------------------------------------------
template <int MAXM, bool LL>
__global__ void __launch_bounds__(128, MAXM <= 8 ? 4 : 1)
    k_ens_tdep(const RunArgs A, const int tend_finite, const int mom_cl) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int M = A.net.M, N = A.net.N, nv = A.net.n_vnz;
  ThreadNet S = carve_thread_net(smem, M, nv, N, blockDim.x);
  const int smem_mom = mom_cl > 0 ? 1 : 0;
  S.mt = mom_table(S.mom, A.G, mom_cl);
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    S.c[i] = A.net.c[i];
    S.dep[i] = A.net.depmask[i];
    S.rd[i] = A.net.rdesc[i];
  }
  for (int i = threadIdx.x; i < nv; i += blockDim.x) S.vl[i] = A.net.vlist[i];
  for (int i = threadIdx.x; i <= M; i += blockDim.x) S.vp[i] = A.net.vptr[i];
  if (smem_mom) mom_zero_and_sync(S.mt, N);
  else __syncthreads();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < A.n_traj) simulate_tdep<MAXM, LL>(A, S, A.net.beta, j, blockDim.x, tend_finite, smem_mom);
  if (smem_mom) mom_sync_and_flush(S.mt, A);
}

template <int MAXM>
static cudaError_t launch_tdep_m(const RunArgs &a, int B, cudaStream_t s, int tend_finite) {
  const int cl = moment_cluster(a);
  const size_t mom = cl ? moment_share_bytes(a, cl) : 0;
  const size_t smem = ((thread_smem_bytes(a.net.M, a.net.N, a.net.n_vnz, B) + 7) & ~(size_t)7) + mom;
  unsigned grid = (unsigned)((a.n_traj + B - 1) / B);
  if (cl > 1) grid = (grid + cl - 1) / cl * cl;
  auto kern = a.out.loglik_dev ? k_ens_tdep<MAXM, true> : k_ens_tdep<MAXM, false>;
  return launch_clustered(kern, grid, B, smem, s, cl, a, tend_finite, cl);
}

int launch_tdep_mapping(const RunArgs &a, int B, cudaStream_t s) {
  if (a.n_traj == 0) return RT_OK;
  if (B <= 0) B = 128;
  if (B > 128 || B % 32) return set_error(RT_ERR_INVALID_ARG, "thread mapping: block_threads must be a multiple of 32 <= 128");
  if (a.net.M > 16 || !a.net.depmask || !a.net.beta)
    return set_error(RT_ERR_UNSUPPORTED, "time-dependent rates run on the thread mapping with M <= 16 (got %d)", a.net.M);
  if (thread_smem_bytes(a.net.M, a.net.N, a.net.n_vnz, B) > 200 * 1024)
    return set_error(RT_ERR_UNSUPPORTED, "thread mapping: network too large for shared memory");
  const int tf = isfinite(a.t_end) ? 1 : 0;
  cudaError_t e;
  if (a.net.M <= 4) e = launch_tdep_m<4>(a, B, s, tf);
  else if (a.net.M <= 8) e = launch_tdep_m<8>(a, B, s, tf);
  else e = launch_tdep_m<16>(a, B, s, tf);
  if (e != cudaSuccess) return set_error(RT_ERR_CUDA, "time-dependent kernel launch: %s", cudaGetErrorString(e));
  return RT_OK;
}

}  // namespace rt

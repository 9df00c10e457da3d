// rt_batch.cu -- batched mode: thousands of networks of uneven size in one
// persistent launch.
//
// Every network of the batch is copied into one device arena and given a mapping
// class by size (thread, warp or block per trajectory).  The flattened work list
// is (network rank in its class, trajectory), networks sorted by decreasing size
// so the longest items start first; it is cut into block-sized tasks: one
// block-class trajectory, block_threads/32 warp-class trajectories or
// block_threads thread-class trajectories.  Persistent blocks take tasks from an
// atomic counter and run the same per-trajectory routines as the single-network
// kernels (rt_traj_*.cuh), reading the network tables through generic pointers
// into the arena.  Network i uses its own Philox stream (the fourth counter word;
// by default i).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "rt_traj_block.cuh"
#include "rt_traj_thread.cuh"
#include "rt_traj_warp.cuh"

namespace rt {

enum { CLS_THREAD = 0, CLS_WARP = 1, CLS_BLOCK = 2 };

struct BNet {
  DevNet d;
  int64_t xoff;  // first species of this network in the packed x0 / x_final rows
  int64_t moff;  // first reaction of this network in the packed counts / t_internal rows
  int32_t cls;
  int32_t R;     // register slots (warp and block: 1, 2, 4 or 8)
  uint32_t stream_id;
  int32_t pad;
};

struct BatchArgs {
  const BNet *nets;
  const int32_t *order[3];  // network indices of each class, largest first
  int32_t n_cls[3];
  int64_t n_traj;
  int64_t tasks[3];          // tasks per class
  int64_t n_tasks;
  unsigned long long *counter;
  const int32_t *x0;
  const double *t_end;
  int32_t max_events;
  uint64_t seed;
  rt_batch_outputs out;
  int maxN_thread, maxN_warp, maxM_block, maxN_block;
};

__device__ __forceinline__ RunArgs item_args(const BatchArgs &B, int net_index, const BNet &bn) {
  RunArgs A;
  A.net = bn.d;
  A.x0 = B.x0 + bn.xoff;
  A.per_traj_x0 = 0;
  A.stream_id = bn.stream_id;
  A.t_end = B.t_end[net_index];
  A.max_events = B.max_events;
  A.seed = B.seed;
  A.n_traj = B.n_traj;
  A.traj_offset = 0;
  A.sample_dt = 0.0;
  A.G = 0;
  memset(&A.out, 0, sizeof(A.out));
  const rt_batch_outputs &o = B.out;
  const int64_t row = (int64_t)net_index * B.n_traj;  // first [net][traj] row of this network
  A.out.x_final_dev = o.x_final_dev ? o.x_final_dev + B.n_traj * bn.xoff : nullptr;
  A.out.n_events_dev = o.n_events_dev ? o.n_events_dev + row : nullptr;
  A.out.status_dev = o.status_dev ? o.status_dev + row : nullptr;
  A.out.t_last_dev = o.t_last_dev ? o.t_last_dev + row : nullptr;
  A.out.loglik_dev = o.loglik_dev ? o.loglik_dev + row : nullptr;
  A.out.counts_dev = o.counts_dev ? o.counts_dev + B.n_traj * bn.moff : nullptr;
  A.out.t_internal_dev = o.t_internal_dev ? o.t_internal_dev + B.n_traj * bn.moff : nullptr;
  A.out.trace_len = o.trace_len;
  A.out.trace_mu_dev = o.trace_mu_dev ? o.trace_mu_dev + row * o.trace_len : nullptr;
  A.out.trace_t_dev = o.trace_t_dev ? o.trace_t_dev + row * o.trace_len : nullptr;
  return A;
}

// Two resident blocks per SM (64 registers; the block routine's channel state partly
// spills to L1-backed local memory): a block-class trajectory is latency-bound (barriers,
// dependent loads, one thread's Exp(1) draw per event), and a second block on the SM
// runs while the first waits -- measured 1.28x the single-block kernel on the 4096-network
// batch.
template <bool LL>
__global__ void __launch_bounds__(512, 2) k_batch(const BatchArgs B) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long s_task;
  const int tid = threadIdx.x, BT = blockDim.x, W = BT >> 5, warp = tid >> 5;
  for (;;) {
    __syncthreads();
    if (tid == 0) s_task = (long long)atomicAdd(B.counter, 1ull);
    __syncthreads();
    long long t = s_task;
    if (t >= B.n_tasks) break;
    if (t < B.tasks[CLS_BLOCK]) {
      // one block-class trajectory
      const int64_t f = t;
      const int ni = B.order[CLS_BLOCK][f / B.n_traj];
      const int64_t j = f % B.n_traj;
      const BNet bn = B.nets[ni];
      const RunArgs A = item_args(B, ni, bn);
      const BlockScratch S = carve_block_scratch(smem, B.maxM_block, B.maxN_block, BT);
      const BlockNet net{bn.d.M, bn.d.N, bn.d.rdesc, bn.d.c, bn.d.vptr, bn.d.vlist, bn.d.sptr, bn.d.slist,
                         bn.d.dptr, bn.d.dlist};
      const int tf = isfinite(A.t_end) ? 1 : 0;
      switch (bn.R) {
        case 1: block_trajectory<1, LL>(A, net, S, j, tf); break;
        case 2: block_trajectory<2, LL>(A, net, S, j, tf); break;
        case 4: block_trajectory<4, LL>(A, net, S, j, tf); break;
        case 8: block_trajectory<8, LL>(A, net, S, j, tf); break;
        default: block_trajectory<16, LL>(A, net, S, j, tf); break;
      }
      continue;
    }
    t -= B.tasks[CLS_BLOCK];
    if (t < B.tasks[CLS_WARP]) {
      // W warp-class trajectories
      const int64_t f = t * W + warp;
      if (f < (int64_t)B.n_cls[CLS_WARP] * B.n_traj) {
        const int ni = B.order[CLS_WARP][f / B.n_traj];
        const int64_t j = f % B.n_traj;
        const BNet bn = B.nets[ni];
        const RunArgs A = item_args(B, ni, bn);
        const WarpNet net{bn.d.M, bn.d.N, bn.d.n_vnz, bn.d.rdesc, bn.d.c, bn.d.vptr, bn.d.vlist, bn.d.depw};
        int *X = (int *)smem + warp * B.maxN_warp;
        const int tf = isfinite(A.t_end) ? 1 : 0;
        switch (bn.R) {
          case 1: warp_trajectories<1, 32, LL>(A, net, X, nullptr, j, tf); break;
          case 2: warp_trajectories<2, 32, LL>(A, net, X, nullptr, j, tf); break;
          case 4: warp_trajectories<4, 32, LL>(A, net, X, nullptr, j, tf); break;
          default: warp_trajectories<8, 32, LL>(A, net, X, nullptr, j, tf); break;
        }
      }
      continue;
    }
    t -= B.tasks[CLS_WARP];
    {
      // BT thread-class trajectories
      const int64_t f = t * BT + tid;
      if (f < (int64_t)B.n_cls[CLS_THREAD] * B.n_traj) {
        const int ni = B.order[CLS_THREAD][f / B.n_traj];
        const int64_t j = f % B.n_traj;
        const BNet bn = B.nets[ni];
        const RunArgs A = item_args(B, ni, bn);
        ThreadNet S;
        S.c = const_cast<double *>(bn.d.c);
        S.dep = const_cast<uint64_t *>(bn.d.depmask);
        S.rd = const_cast<int2 *>(bn.d.rdesc);
        S.vl = const_cast<int2 *>(bn.d.vlist);
        S.vp = const_cast<int *>(bn.d.vptr);
        S.X = (int *)smem;
        S.mom = nullptr;
        S.mt = mom_table(nullptr, 0, 1);
        simulate_one<8, LL>(A, S, j, BT, isfinite(A.t_end) ? 1 : 0, 0);
      }
    }
  }
}

}  // namespace rt

using namespace rt;

struct rt_batch {
  int device = 0;
  int32_t n_nets = 0;
  void *arena = nullptr;
  BNet *d_nets = nullptr;
  int32_t *d_order[3] = {nullptr, nullptr, nullptr};
  unsigned long long *d_counter = nullptr;
  int32_t n_cls[3] = {0, 0, 0};
  int64_t total_species = 0, total_reactions = 0;
  rt_batch_policy policy;
  int maxN_thread = 1, maxN_warp = 1, maxM_block = 1, maxN_block = 1;
  size_t smem = 0;
  int grid = 0;
};

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

extern "C" int rt_batch_create(int32_t n_nets, const rt_network *const *nets, const uint32_t *stream_ids,
                               const rt_batch_policy *policy, rt_batch **out) {
  clear_error();
  if (!out) return set_error(RT_ERR_INVALID_ARG, "rt_batch_create: out is NULL");
  *out = nullptr;
  if (n_nets < 1 || !nets) return set_error(RT_ERR_INVALID_ARG, "need at least one network");
  rt_batch_policy pol{8, 256, 512, 0};
  if (policy) pol = *policy;
  if (pol.thread_max_m < 0 || pol.thread_max_m > 8)
    return set_error(RT_ERR_INVALID_ARG, "thread_max_m must be in [0, 8]");
  if (pol.warp_max_m < pol.thread_max_m || pol.warp_max_m > 256)
    return set_error(RT_ERR_INVALID_ARG, "warp_max_m must be in [thread_max_m, 256]");
  if (pol.block_threads != 128 && pol.block_threads != 256 && pol.block_threads != 512)
    return set_error(RT_ERR_INVALID_ARG, "block_threads must be 128, 256 or 512");
  int dev = 0;
  cudaGetDevice(&dev);
  rt_batch *b = new rt_batch();
  b->device = dev;
  b->n_nets = n_nets;
  b->policy = pol;
  std::vector<BNet> hn(n_nets);
  std::vector<size_t> off(n_nets);
  size_t total = 0;
  for (int i = 0; i < n_nets; i++) {
    const rt_network *g = nets[i];
    if (!g || g->device != dev) {
      delete b;
      return set_error(RT_ERR_INVALID_ARG, "network %d is NULL or on another device", i);
    }
    if (g->dev.beta) {
      delete b;
      return set_error(RT_ERR_UNSUPPORTED, "network %d has time-dependent rates; batches take constant rates", i);
    }
    off[i] = total;
    total += align256(g->arena_bytes);
    const int M = g->dev.M, N = g->dev.N;
    int cls;
    if (M <= pol.thread_max_m && N <= 8) cls = CLS_THREAD;
    else if (M <= pol.warp_max_m) cls = CLS_WARP;
    else if (M <= 16 * pol.block_threads) cls = CLS_BLOCK;
    else {
      delete b;
      return set_error(RT_ERR_UNSUPPORTED, "network %d has %d reactions; this policy supports up to %d (16 per thread)",
                       i, M, 16 * pol.block_threads);
    }
    int R = 1;
    if (cls == CLS_WARP) R = M <= 32 ? 1 : M <= 64 ? 2 : M <= 128 ? 4 : 8;
    if (cls == CLS_BLOCK) {
      const int need = (M + pol.block_threads - 1) / pol.block_threads;
      R = need <= 1 ? 1 : need <= 2 ? 2 : need <= 4 ? 4 : need <= 8 ? 8 : 16;
      b->maxM_block = std::max(b->maxM_block, M);
      b->maxN_block = std::max(b->maxN_block, N);
    }
    if (cls == CLS_WARP) b->maxN_warp = std::max(b->maxN_warp, N);
    if (cls == CLS_THREAD) b->maxN_thread = std::max(b->maxN_thread, N);
    hn[i].xoff = b->total_species;
    hn[i].moff = b->total_reactions;
    hn[i].cls = cls;
    hn[i].R = R;
    hn[i].stream_id = stream_ids ? stream_ids[i] : (uint32_t)i;
    hn[i].pad = 0;
    b->total_species += N;
    b->total_reactions += M;
    b->n_cls[cls]++;
  }
  // class lists, largest networks first
  std::vector<int32_t> order[3];
  for (int i = 0; i < n_nets; i++) order[hn[i].cls].push_back(i);
  for (int c = 0; c < 3; c++)
    std::stable_sort(order[c].begin(), order[c].end(),
                     [&](int32_t x, int32_t y) { return nets[x]->dev.M > nets[y]->dev.M; });
  const size_t off_nets = total;
  total += align256(sizeof(BNet) * n_nets);
  size_t off_order[3];
  for (int c = 0; c < 3; c++) {
    off_order[c] = total;
    total += align256(sizeof(int32_t) * std::max<size_t>(1, order[c].size()));
  }
  const size_t off_ctr = total;
  total += 256;
  cudaError_t e = cudaMalloc(&b->arena, total);
  if (e != cudaSuccess) {
    delete b;
    return set_error(RT_ERR_OOM, "cudaMalloc(%zu): %s", total, cudaGetErrorString(e));
  }
  std::vector<char> host(total, 0);
  char *base = (char *)b->arena;
  for (int i = 0; i < n_nets; i++) {
    const rt_network *g = nets[i];
    memcpy(host.data() + off[i], g->host_blob.data(), g->arena_bytes);
    char *db = base + off[i];
    DevNet d = g->dev;  // same layout, rebased into the batch arena
    d.beta = nullptr;
    d.rdesc = (const int2 *)(db + g->off_rdesc);
    d.c = (const double *)(db + g->off_c);
    d.c0 = (const double *)(db + g->off_c0);
    d.vptr = (const int32_t *)(db + g->off_vptr);
    d.vlist = (const int2 *)(db + g->off_vlist);
    d.sptr = (const int32_t *)(db + g->off_sptr);
    d.slist = (const int32_t *)(db + g->off_slist);
    d.depmask = g->dev.depmask ? (const uint64_t *)(db + g->off_dep) : nullptr;
    d.depw = g->dev.depw ? (const uint8_t *)(db + g->off_depw) : nullptr;
    d.depw16 = g->dev.depw16 ? (const uint8_t *)(db + g->off_depw16) : nullptr;
    d.depw8 = g->dev.depw8 ? (const uint8_t *)(db + g->off_depw8) : nullptr;
    d.vdep = g->dev.vdep ? (const int4 *)(db + g->off_vdep) : nullptr;
    d.dptr = g->dev.dptr ? (const int32_t *)(db + g->off_dptr) : nullptr;
    d.dlist = g->dev.dptr ? (const int32_t *)(db + g->off_dlist) : nullptr;
    hn[i].d = d;
  }
  memcpy(host.data() + off_nets, hn.data(), sizeof(BNet) * n_nets);
  for (int c = 0; c < 3; c++)
    if (!order[c].empty()) memcpy(host.data() + off_order[c], order[c].data(), sizeof(int32_t) * order[c].size());
  e = cudaMemcpy(b->arena, host.data(), total, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(b->arena);
    delete b;
    return set_error(RT_ERR_CUDA, "cudaMemcpy: %s", cudaGetErrorString(e));
  }
  b->d_nets = (BNet *)(base + off_nets);
  for (int c = 0; c < 3; c++) b->d_order[c] = (int32_t *)(base + off_order[c]);
  b->d_counter = (unsigned long long *)(base + off_ctr);

  // shared memory: the largest of the three uses (a block runs one task at a time)
  const int BT = pol.block_threads;
  const size_t s_block = b->n_cls[CLS_BLOCK] ? block_scratch_bytes(b->maxM_block, b->maxN_block, BT) : 0;
  const size_t s_warp = (size_t)(BT / 32) * b->maxN_warp * 4;
  const size_t s_thread = (size_t)BT * b->maxN_thread * 4;
  b->smem = std::max({s_block, s_warp, s_thread, (size_t)16});
  if (b->smem > 200 * 1024) {
    const size_t need = b->smem;
    cudaFree(b->arena);
    delete b;
    return set_error(RT_ERR_UNSUPPORTED, "batch networks need %zu bytes of shared memory", need);
  }
  raise_smem_limit((const void *)k_batch<false>, b->smem);
  raise_smem_limit((const void *)k_batch<true>, b->smem);
  int per_sm = 0, per_sm_ll = 0, sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<false>, BT, b->smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_ll, k_batch<true>, BT, b->smem);
  per_sm = std::min(per_sm, per_sm_ll);
  if (per_sm < 1) per_sm = 1;
  if (pol.blocks_per_sm > 0) per_sm = std::min(per_sm, pol.blocks_per_sm);
  b->grid = per_sm * sms;
  *out = b;
  return RT_OK;
}

extern "C" void rt_batch_destroy(rt_batch *b) {
  if (!b) return;
  if (b->arena) cudaFree(b->arena);
  delete b;
}

extern "C" int rt_batch_info(const rt_batch *b, int64_t *total_species, int64_t *total_reactions,
                             int32_t *n_thread_class, int32_t *n_warp_class, int32_t *n_block_class) {
  clear_error();
  if (!b) return set_error(RT_ERR_INVALID_ARG, "rt_batch_info: NULL batch");
  if (total_species) *total_species = b->total_species;
  if (total_reactions) *total_reactions = b->total_reactions;
  if (n_thread_class) *n_thread_class = b->n_cls[CLS_THREAD];
  if (n_warp_class) *n_warp_class = b->n_cls[CLS_WARP];
  if (n_block_class) *n_block_class = b->n_cls[CLS_BLOCK];
  return RT_OK;
}

extern "C" int rt_batch_run(rt_batch *b, const int32_t *x0_dev, const double *t_end_dev, int64_t max_events,
                            uint64_t seed, int64_t n_traj_per_net, const rt_batch_outputs *outputs, void *stream) {
  clear_error();
  if (!b) return set_error(RT_ERR_INVALID_ARG, "rt_batch_run: NULL batch");
  if (n_traj_per_net < 0) return set_error(RT_ERR_INVALID_ARG, "n_traj_per_net must be >= 0");
  if (max_events < 0 || max_events > INT32_MAX) return set_error(RT_ERR_INVALID_ARG, "max_events must be in [0, INT32_MAX]");
  if (!x0_dev || !t_end_dev) return set_error(RT_ERR_INVALID_ARG, "x0 and t_end are required");
  if (outputs && outputs->trace_len < 0) return set_error(RT_ERR_INVALID_ARG, "trace_len must be >= 0");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != b->device) return set_error(RT_ERR_INVALID_ARG, "batch lives on device %d, device %d is current", b->device, dev);
  if (n_traj_per_net == 0) return RT_OK;
  BatchArgs A;
  A.nets = b->d_nets;
  for (int c = 0; c < 3; c++) {
    A.order[c] = b->d_order[c];
    A.n_cls[c] = b->n_cls[c];
  }
  A.n_traj = n_traj_per_net;
  const int BT = b->policy.block_threads;
  A.tasks[CLS_BLOCK] = (int64_t)b->n_cls[CLS_BLOCK] * n_traj_per_net;
  A.tasks[CLS_WARP] = ((int64_t)b->n_cls[CLS_WARP] * n_traj_per_net + BT / 32 - 1) / (BT / 32);
  A.tasks[CLS_THREAD] = ((int64_t)b->n_cls[CLS_THREAD] * n_traj_per_net + BT - 1) / BT;
  A.n_tasks = A.tasks[0] + A.tasks[1] + A.tasks[2];
  A.counter = b->d_counter;
  A.x0 = x0_dev;
  A.t_end = t_end_dev;
  A.max_events = (int32_t)max_events;
  A.seed = seed;
  memset(&A.out, 0, sizeof(A.out));
  if (outputs) A.out = *outputs;
  A.maxN_thread = b->maxN_thread;
  A.maxN_warp = b->maxN_warp;
  A.maxM_block = b->maxM_block;
  A.maxN_block = b->maxN_block;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return set_error(RT_ERR_CUDA, "memset: %s", cudaGetErrorString(e));
  const int grid = (int)std::min<int64_t>(b->grid, std::max<int64_t>(1, A.n_tasks));
  if (A.out.loglik_dev) k_batch<true><<<grid, BT, b->smem, s>>>(A);
  else k_batch<false><<<grid, BT, b->smem, s>>>(A);
  e = cudaGetLastError();
  return e == cudaSuccess ? RT_OK : set_error(RT_ERR_CUDA, "batch launch: %s", cudaGetErrorString(e));
}

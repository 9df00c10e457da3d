// rt_api.cu -- C ABI entry points: argument checks, mapping choice, launches.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>

#include "rt_sim.cuh"

namespace rt {

int check_device(const rt_network *net) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return set_error(RT_ERR_CUDA, "cudaGetDevice failed");
  if (dev != net->device)
    return set_error(RT_ERR_INVALID_ARG, "network lives on device %d but device %d is current", net->device, dev);
  return RT_OK;
}

static int choose_mapping(const rt_network *net, const rt_launch_cfg *cfg, int form = RT_FORM_INTERNAL) {
  if (cfg && cfg->mapping != RT_MAP_AUTO) return cfg->mapping;
  if (form == RT_FORM_ABSOLUTE) return RT_MAP_TREE;
  if (form == RT_FORM_RESCALED) return net->dev.M <= 8 ? RT_MAP_THREAD : RT_MAP_WARP;
  if (net->dev.M <= thread_mapping_max_m()) return RT_MAP_THREAD;
  if (net->dev.M <= warp_mapping_max_m()) return RT_MAP_WARP;
  if (net->dev.M <= block_mapping_max_m()) return RT_MAP_BLOCK;
  return RT_MAP_BUNDLE;
}

int validate_run(const rt_network *net, const rt_run_params *p, const rt_outputs *o) {
  if (!net) return set_error(RT_ERR_INVALID_ARG, "rt_run: NULL network");
  if (!p || !o) return set_error(RT_ERR_INVALID_ARG, "rt_run: NULL params or outputs");
  if (p->n_traj < 0) return set_error(RT_ERR_INVALID_ARG, "n_traj must be >= 0");
  if (p->n_traj > (int64_t)INT32_MAX * 64) return set_error(RT_ERR_INVALID_ARG, "n_traj too large");
  if (p->traj_offset < 0) return set_error(RT_ERR_INVALID_ARG, "traj_offset must be >= 0");
  if (p->max_events < 0 || p->max_events > INT32_MAX)
    return set_error(RT_ERR_INVALID_ARG, "max_events must be in [0, INT32_MAX]");
  if (std::isnan(p->t_end) || p->t_end < 0.0) return set_error(RT_ERR_INVALID_ARG, "t_end must be >= 0");
  if (!p->x0_dev && p->n_traj > 0) return set_error(RT_ERR_INVALID_ARG, "x0 is NULL");
  const bool want_grid = o->grid_dev || o->grid_sum_dev || o->grid_sumsq_dev || o->grid_count_dev;
  if (want_grid && !(p->sample_dt > 0.0)) return set_error(RT_ERR_INVALID_ARG, "grid outputs need sample_dt > 0");
  if (want_grid && !std::isfinite(p->t_end)) return set_error(RT_ERR_INVALID_ARG, "grid outputs need a finite t_end");
  if ((o->grid_sumsq_dev || o->grid_count_dev) && !o->grid_sum_dev)
    return set_error(RT_ERR_INVALID_ARG, "grid_sumsq/grid_count need grid_sum");
  if (o->trace_len < 0) return set_error(RT_ERR_INVALID_ARG, "trace_len must be >= 0");
  if (p->form != RT_FORM_INTERNAL && p->form != RT_FORM_ABSOLUTE && p->form != RT_FORM_RESCALED)
    return set_error(RT_ERR_INVALID_ARG, "form must be RT_FORM_INTERNAL, RT_FORM_ABSOLUTE or RT_FORM_RESCALED");
  return RT_OK;
}

}  // namespace rt

using namespace rt;

extern "C" int rt_workspace_bytes(const rt_network *net, const rt_run_params *params, const rt_launch_cfg *cfg,
                                  size_t *bytes) {
  clear_error();
  if (!net || !params || !bytes) return set_error(RT_ERR_INVALID_ARG, "rt_workspace_bytes: NULL argument");
  *bytes = 0;
  const int mapping = choose_mapping(net, cfg, params->form);
  if (mapping == RT_MAP_THREAD || mapping == RT_MAP_WARP || mapping == RT_MAP_BLOCK) return RT_OK;
  if (mapping == RT_MAP_BUNDLE) {
    *bytes = bundle_workspace_bytes(net->dev, params->n_traj, cfg ? cfg->ctas_per_traj : 0);
    return RT_OK;
  }
  if (mapping == RT_MAP_TREE) {
    *bytes = lazy_workspace_bytes(net->dev, net->max_dependents, params->n_traj, cfg ? cfg->ctas_per_traj : 0);
    return RT_OK;
  }
  return set_error(RT_ERR_UNSUPPORTED, "mapping %d not available", mapping);
}

extern "C" int rt_run(const rt_network *net, const rt_run_params *p, const rt_outputs *o, const rt_launch_cfg *cfg,
                      void *workspace, size_t workspace_bytes, void *stream) {
  clear_error();
  int rc = validate_run(net, p, o);
  if (rc) return rc;
  if ((rc = check_device(net))) return rc;
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
  const int mapping = choose_mapping(net, cfg, p->form);
  const int B = cfg ? cfg->block_threads : 0;
  cudaStream_t s = (cudaStream_t)stream;
  if ((p->form == RT_FORM_ABSOLUTE) != (mapping == RT_MAP_TREE))
    return set_error(RT_ERR_UNSUPPORTED, "the absolute-time form runs on the tree mapping (RT_MAP_TREE) and the "
                     "tree mapping runs the absolute-time form only");
  if (net->dev.beta) {  // time-dependent rates: the internal-time form on the thread or warp mapping
    if (p->form != RT_FORM_INTERNAL || (mapping != RT_MAP_THREAD && mapping != RT_MAP_WARP))
      return set_error(RT_ERR_UNSUPPORTED,
                       "time-dependent rates run the internal-time form on the thread (M <= 16) or warp (M <= 256) "
                       "mapping");
    return mapping == RT_MAP_THREAD ? launch_tdep_mapping(a, B, s)
                                    : launch_tdep_warp_mapping(a, cfg ? cfg->lanes_per_traj : 0, s);
  }
  if (p->form == RT_FORM_RESCALED) {
    if (mapping == RT_MAP_THREAD) return launch_rescaled_mapping(a, B, s);
    if (mapping == RT_MAP_WARP) return launch_rescaled_warp_mapping(a, cfg ? cfg->lanes_per_traj : 0, s);
    return set_error(RT_ERR_UNSUPPORTED, "Table 3's rescaled form runs on the thread (M <= 8) or warp (M <= 256) mapping");
  }
  switch (mapping) {
    case RT_MAP_THREAD:
      // networks of <= 4 reactions and <= 4 species: network in the parameter space, X in registers
      return net->small.ok ? launch_small_mapping(a, net->small, B, s) : launch_thread_mapping(a, B, s);
    case RT_MAP_WARP:
      return launch_warp_mapping(a, B, cfg ? cfg->lanes_per_traj : 0, s);
    case RT_MAP_BLOCK:
      return launch_block_mapping(a, B, s);
    case RT_MAP_BUNDLE:
      return launch_bundle_mapping(a, cfg ? cfg->ctas_per_traj : 0, workspace, workspace_bytes, s);
    case RT_MAP_TREE:
      return launch_lazy_mapping(a, net->max_dependents, cfg ? cfg->ctas_per_traj : 0, workspace, workspace_bytes, s);
    default:
      return set_error(RT_ERR_UNSUPPORTED, "mapping %d not available", mapping);
  }
}

// ---------------------------------------------------------------------------
// Utility kernels: the draws and the logarithm exposed for testing and reuse.
// ---------------------------------------------------------------------------

__global__ void k_draw_exp1(uint64_t seed, uint32_t stream_id, int64_t count, const uint64_t *traj,
                            const uint32_t *channel, const uint64_t *index, double *u, double *e) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t bits = draw_bits(seed, traj[i], channel[i], (uint32_t)index[i], stream_id);
    if (u) u[i] = __dmul_rn(__ull2double_rn(bits_to_x(bits)), 0x1p-53);
    if (e) e[i] = exp1_from_bits(bits);
  }
}

__global__ void k_log_eval(int64_t count, const double *x, double *y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = rt_ln(x[i]);
}

__global__ void k_philox(int64_t count, const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    const uint4 o = philox4x32_10(c, k0, k1);
    out[4 * i] = o.x;
    out[4 * i + 1] = o.y;
    out[4 * i + 2] = o.z;
    out[4 * i + 3] = o.w;
  }
}

static unsigned util_grid(int64_t count) {
  const int64_t b = (count + 255) / 256;
  return (unsigned)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

extern "C" int rt_draw_exp1(uint64_t seed, uint32_t stream_id, int64_t count, const uint64_t *traj,
                            const uint32_t *channel, const uint64_t *index, double *u, double *e, void *stream) {
  clear_error();
  if (count < 0) return set_error(RT_ERR_INVALID_ARG, "count must be >= 0");
  if (count == 0) return RT_OK;
  if (!traj || !channel || !index) return set_error(RT_ERR_INVALID_ARG, "NULL input array");
  k_draw_exp1<<<util_grid(count), 256, 0, (cudaStream_t)stream>>>(seed, stream_id, count, traj, channel, index, u, e);
  const cudaError_t err = cudaGetLastError();
  return err == cudaSuccess ? RT_OK : set_error(RT_ERR_CUDA, "%s", cudaGetErrorString(err));
}

extern "C" int rt_log_eval(int64_t count, const double *x, double *y, void *stream) {
  clear_error();
  if (count < 0) return set_error(RT_ERR_INVALID_ARG, "count must be >= 0");
  if (count == 0) return RT_OK;
  if (!x || !y) return set_error(RT_ERR_INVALID_ARG, "NULL array");
  k_log_eval<<<util_grid(count), 256, 0, (cudaStream_t)stream>>>(count, x, y);
  const cudaError_t err = cudaGetLastError();
  return err == cudaSuccess ? RT_OK : set_error(RT_ERR_CUDA, "%s", cudaGetErrorString(err));
}

extern "C" int rt_philox(int64_t count, const uint32_t *ctr, uint32_t key0, uint32_t key1, uint32_t *out,
                         void *stream) {
  clear_error();
  if (count < 0) return set_error(RT_ERR_INVALID_ARG, "count must be >= 0");
  if (count == 0) return RT_OK;
  if (!ctr || !out) return set_error(RT_ERR_INVALID_ARG, "NULL array");
  k_philox<<<util_grid(count), 256, 0, (cudaStream_t)stream>>>(count, ctr, key0, key1, out);
  const cudaError_t err = cudaGetLastError();
  return err == cudaSuccess ? RT_OK : set_error(RT_ERR_CUDA, "%s", cudaGetErrorString(err));
}

// ---------------------------------------------------------------------------
// Backward: grad_c[k] = sum_j g_j (n_jk - T_jk) / c_k.  One block per 32
// channels; each of 32 row lanes sums every 32nd trajectory in index order,
// then the 32 lane sums are added in lane order: a fixed summation order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_loglik_backward(int32_t M, int64_t n_traj, const double *g,
                                                          const int32_t *counts, const double *Tend,
                                                          const double *c, double *grad) {
  __shared__ double part[32][33];
  const int col = blockIdx.x * 32 + threadIdx.x;
  double s = 0.0;
  if (col < M) {
    const double ck = c[col];
    for (int64_t j = threadIdx.y; j < n_traj; j += 32) {
      const double d = __dsub_rn(__int2double_rn(counts[j * M + col]), Tend[j * M + col]);
      s = __dadd_rn(s, __dmul_rn(g[j], __ddiv_rn(d, ck)));
    }
  }
  part[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && col < M) {
    double r = 0.0;
    for (int y = 0; y < 32; ++y) r = __dadd_rn(r, part[y][threadIdx.x]);
    grad[col] = r;
  }
}

extern "C" int rt_loglik_backward(const rt_network *net, int64_t n_traj, const double *grad_ll,
                                  const int32_t *counts, const double *Tend, double *grad_c, void *stream) {
  clear_error();
  if (!net) return set_error(RT_ERR_INVALID_ARG, "NULL network");
  if (n_traj < 0) return set_error(RT_ERR_INVALID_ARG, "n_traj must be >= 0");
  if (!grad_c || (n_traj > 0 && (!grad_ll || !counts || !Tend))) return set_error(RT_ERR_INVALID_ARG, "NULL array");
  int rc = check_device(net);
  if (rc) return rc;
  const int M = net->dev.M;
  dim3 block(32, 32);
  k_loglik_backward<<<(M + 31) / 32, block, 0, (cudaStream_t)stream>>>(M, n_traj, grad_ll, counts, Tend, net->dev.c0,
                                                                     grad_c);
  const cudaError_t err = cudaGetLastError();
  return err == cudaSuccess ? RT_OK : set_error(RT_ERR_CUDA, "%s", cudaGetErrorString(err));
}

// ---------------------------------------------------------------------------
// Measurement aid: the binary64 add/multiply issue rate of this GPU.  Each thread
// runs kProbeChains independent chains x <- x * m + c (one DMUL and one DADD, never
// fused: the library is built with --fmad=false and the intrinsics round each op),
// so the FP64 pipe, not latency, bounds the loop.  The result is written only if
// it equals an impossible value, which keeps the loop alive without memory traffic.
// ---------------------------------------------------------------------------
constexpr int kProbeChains = 8;
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) k_fp64_probe(int64_t iters, double *sink) {
  double x[kProbeChains];
#pragma unroll
  for (int i = 0; i < kProbeChains; ++i) x[i] = 1.0 + 1e-3 * (threadIdx.x + i);
  const double m = 0.9999999, c = 1e-9;
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) x[i] = __dadd_rn(__dmul_rn(x[i], m), c);
  }
  double acc = 0.0;
#pragma unroll
  for (int i = 0; i < kProbeChains; ++i) acc = __dadd_rn(acc, x[i]);
  if (acc == -1.0) sink[0] = acc;
}

extern "C" int rt_fp64_probe(int64_t iters, int32_t blocks_per_sm, double *sink_dev, double *ops, void *stream) {
  clear_error();
  if (iters < 1 || blocks_per_sm < 1 || blocks_per_sm > 64) return set_error(RT_ERR_INVALID_ARG, "iters >= 1, 1 <= blocks_per_sm <= 64");
  if (!sink_dev) return set_error(RT_ERR_INVALID_ARG, "sink_dev is NULL");
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t grid = (int64_t)sms * blocks_per_sm;
  k_fp64_probe<<<(unsigned)grid, kProbeThreads, 0, (cudaStream_t)stream>>>(iters, sink_dev);
  const cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return set_error(RT_ERR_CUDA, "%s", cudaGetErrorString(err));
  if (ops) *ops = 2.0 * kProbeChains * (double)kProbeThreads * (double)grid * (double)iters;
  return RT_OK;
}

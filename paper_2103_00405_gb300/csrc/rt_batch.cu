// rt_batch.cu -- batched mode: many networks of uneven size in one persistent launch.
#include <cuda_runtime.h>

#include "rt_internal.h"

using namespace rt;

extern "C" int rt_batch_create(int32_t n_nets, const rt_network *const *nets, rt_batch **out) {
  (void)n_nets;
  (void)nets;
  if (out) *out = nullptr;
  return set_error(RT_ERR_UNSUPPORTED, "batched mode not built yet");
}

extern "C" void rt_batch_destroy(rt_batch *batch) { (void)batch; }

extern "C" int rt_batch_info(const rt_batch *batch, int64_t *total_species, int64_t *total_reactions) {
  (void)batch;
  (void)total_species;
  (void)total_reactions;
  return set_error(RT_ERR_UNSUPPORTED, "batched mode not built yet");
}

extern "C" int rt_batch_run(rt_batch *batch, const int32_t *x0_dev, const double *t_end_dev, int64_t max_events,
                            uint64_t seed, int64_t n_traj_per_net, int32_t *x_final_dev, int64_t *n_events_dev,
                            int32_t *status_dev, double *t_last_dev, const rt_launch_cfg *cfg, void *stream) {
  (void)batch; (void)x0_dev; (void)t_end_dev; (void)max_events; (void)seed; (void)n_traj_per_net;
  (void)x_final_dev; (void)n_events_dev; (void)status_dev; (void)t_last_dev; (void)cfg; (void)stream;
  return set_error(RT_ERR_UNSUPPORTED, "batched mode not built yet");
}

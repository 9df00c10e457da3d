// rt_internal.h -- shared declarations of librandtime's translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "randtime.h"

namespace rt {

// Reactant descriptor of one reaction (at most two reactant molecules, as in the
// paper's Sec. 5): h = 1 (s0 < 0), x[s0] (s1 == -1), x[s0](x[s0]-1)/2 (s1 == -2),
// or x[s0] * x[s1] (s1 >= 0).
enum : int32_t { RD_NONE = -1, RD_UNI = -1, RD_DIMER = -2 };

// Device view of a packed network.
struct DevNet {
  int32_t N, M;
  int32_t n_vnz;           // entries in vlist
  int32_t max_vlen;        // largest number of species one reaction changes
  const int2 *rdesc;       // [M] {s0, s1}
  const double *c;         // [M] rates in effect (0 for forbidden channels)
  const double *c0;        // [M] the network's rates (the gradient divides by these)
  const int32_t *vptr;     // [M+1] net change of reaction k: vlist[vptr[k]..vptr[k+1])
  const int2 *vlist;       // {species, delta}
  const int32_t *sptr;     // [N+1] reactions with species s as a reactant: slist[sptr[s]..sptr[s+1])
  const int32_t *slist;
  const uint64_t *depmask; // [M] (M <= 64 only) bit k: firing changes a species channel k reads
  const uint8_t *depw;     // [M][32] (M <= 256 only) bit r of depw[mu*32 + l]: channel l + 32 r depends on mu
  const uint8_t *depw16;   // [M][16] (M <= 128 only) the same for 16-lane segments: channel l + 16 r
  const uint8_t *depw8;    // [M][8]  (M <= 64 only)  the same for 8-lane segments: channel l + 8 r
  const double *beta;      // [M] rate slopes, c_k(t) = c_k (1 + beta_k t); null for constant rates
  const int4 *vdep;        // [M][3] per reaction, when it fits (else null): its net change packed in
                           // 4 words (species << 8) | (delta & 0xFF), unused words 0; then for each
                           // changed species the begin and the length of its reader list in slist
  const int32_t *dptr;     // [M+1] (M <= kDepListMaxM, else null) the channels whose propensity
  const int32_t *dlist;    // reaction k's firing changes: dlist[dptr[k]..dptr[k+1]) (the reader
                           // lists of its changed species, concatenated; repeats possible)
};

// Networks up to this many reactions get the per-reaction dependent lists (dptr/dlist).
constexpr int kDepListMaxM = 8192;

// Packed net-change word: species in the high 24 bits, delta (-128..127, never 0) in the low 8.
__host__ __device__ inline int vpack_species(int w) { return (int)((unsigned)w >> 8); }
__host__ __device__ inline int vpack_delta(int w) { return (int)(signed char)(w & 0xFF); }

// Networks of at most kSmallM reactions and kSmallN species: the whole network by
// value, for kernels that take it in their parameter space (rt_small.cu).
constexpr int kSmallM = 4, kSmallN = 4;
struct SmallNet {
  int32_t ok;                        // 1 if the network fits
  int32_t s0[kSmallM], s1[kSmallM];  // reactant descriptor of each channel (as DevNet::rdesc)
  double c[kSmallM];                 // rate constants
  uint32_t dep[kSmallM];             // bit k: firing this reaction changes a species channel k reads
  int32_t delta[kSmallM][kSmallN];   // net change of each species when the reaction fires
};

}  // namespace rt

struct rt_network {
  rt::DevNet dev;
  void *arena = nullptr;   // device allocation holding every array of dev
  size_t arena_bytes = 0;
  int device = 0;
  int32_t max_dependents = 0;  // upper bound, counted with multiplicity
  int64_t n_dep_nz = 0;
  // host copies used by the batched mode's packer
  std::string host_blob;  // the arena's bytes
  size_t off_rdesc = 0, off_c = 0, off_c0 = 0, off_vptr = 0, off_vlist = 0, off_sptr = 0, off_slist = 0, off_dep = 0;
  std::vector<double> c_host;  // the network's rates (host copy)
  double *beta_dev = nullptr;  // rate slopes on the device (rt_network_set_rate_slopes), or null
  size_t off_depw = 0, off_depw16 = 0, off_depw8 = 0;
  size_t off_vdep = 0, off_dptr = 0, off_dlist = 0;
  rt::SmallNet small = {};  // filled when M <= kSmallM and N <= kSmallN
};

namespace rt {

// Thread-local error message; returns `code`.
int set_error(int code, const char *fmt, ...);
void clear_error();

// Raise a kernel's dynamic shared-memory limit on the current device to at least
// `bytes` (never lowers it).  The limit is a property of the kernel, shared by
// every caller and thread of the process, so lowering it for one launch could
// break another that is already configured (or captured in a graph); a
// process-wide running maximum per (kernel, device) is kept under a mutex.
cudaError_t raise_smem_limit(const void *kernel, size_t bytes);

// Arguments of a simulation launch (plain data, passed by value to kernels).
struct RunArgs {
  DevNet net;
  const int32_t *x0;
  int32_t per_traj_x0;
  uint32_t stream_id;
  double t_end;
  int32_t max_events;
  uint64_t seed;
  int64_t n_traj;
  int64_t traj_offset;
  double sample_dt;
  int64_t G;
  rt_outputs out;
};

// Argument checks shared by the entry points (rt_api.cu).
int check_device(const rt_network *net);
int validate_run(const rt_network *net, const rt_run_params *p, const rt_outputs *o);

// Launchers implemented in the .cu files (return RT_OK or an error code).
int launch_thread_mapping(const RunArgs &a, int block_threads, cudaStream_t s);
int launch_rescaled_mapping(const RunArgs &a, int block_threads, cudaStream_t s);
int launch_tdep_mapping(const RunArgs &a, int block_threads, cudaStream_t s);
int launch_tdep_warp_mapping(const RunArgs &a, int lanes_per_traj, cudaStream_t s);
int launch_rescaled_warp_mapping(const RunArgs &a, int lanes_per_traj, cudaStream_t s);
int launch_small_mapping(const RunArgs &a, const SmallNet &net, int block_threads, cudaStream_t s);
int thread_mapping_max_m();
size_t bundle_workspace_bytes(const DevNet &net, int64_t n_traj, int ctas_per_traj);
int launch_warp_mapping(const RunArgs &a, int block_threads, int lanes_per_traj, cudaStream_t s);
int warp_mapping_max_m();
int launch_block_mapping(const RunArgs &a, int block_threads, cudaStream_t s);
int block_mapping_max_m();
int launch_bundle_mapping(const RunArgs &a, int ctas_per_traj, void *ws, size_t ws_bytes, cudaStream_t s);
size_t lazy_workspace_bytes(const DevNet &net, int max_dependents, int64_t n_traj, int ctas_per_traj);
int launch_lazy_mapping(const RunArgs &a, int max_dependents, int ctas_per_traj, void *ws, size_t ws_bytes,
                        cudaStream_t s);

}  // namespace rt

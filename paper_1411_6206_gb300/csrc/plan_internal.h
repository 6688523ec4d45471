// Internal to the library: the plan object and the host helpers shared by the translation
// units of the C ABI (plans, batches, the serving loop, the autotuner).
#pragma once

#include "lps_api.h"
#include "lps_internal.cuh"

#include <cuda_runtime.h>

#include <vector>

namespace lps {

void set_err(const char* fmt, ...);

}  // namespace lps

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      lps::set_err("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return (e_ == cudaErrorMemoryAllocation) ? LPS_ERR_OOM : LPS_ERR_CUDA;              \
    }                                                                                   \
  } while (0)

#define ARG(cond, ...)              \
  do {                              \
    if (!(cond)) {                  \
      lps::set_err(__VA_ARGS__);    \
      return LPS_ERR_INVALID_ARG;   \
    }                               \
  } while (0)

using lps::Geom;
using lps::DevPersist;
using lps::DevCtrl;
using lps::IterRec;
using lps::DcArgs;

struct lps_plan {
  lps_params p;
  Geom g;
  cudaStream_t st = nullptr;
  cudaStream_t cap = nullptr;    // capture stream of the frame graph
  cudaStream_t side = nullptr;   // second stream: the sparse step beside the eigen kernel
  cudaStream_t cap_side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // device state
  float2 *X = nullptr, *L = nullptr, *S = nullptr, *R = nullptr, *coils = nullptr;
  __half2* coils_h = nullptr;   // LPS_COILS_FP16: half-precision copy of the (rounded) coil maps
  __half2* dhyb_h = nullptr;    // LPS_DATA_FP16: half-precision copy of the (rounded) hybrid samples
  int stall_polls = 0;          // lps_test_stall_wait: one-shot hook for the next operator call
  float2* S2 = nullptr;   // second sparse-part buffer: iteration k writes S_k while S_{k-1} is read
  float2 *dhyb = nullptr, *kstage = nullptr, *hscratch = nullptr, *istage = nullptr;
  float2 *W = nullptr, *V = nullptr, *gram_part = nullptr;
  // float64 eigen mode: Gram, refined eigenvectors, A = V^H G V, eigenvalues
  float2 *G64in = nullptr, *Vref = nullptr;
  double2* A64 = nullptr;
  double* lam64 = nullptr;
  float2* Lnew = nullptr;   // reprojection output of the precision modes
  float2 *tw_x = nullptr, *tw_y = nullptr, *tw_z = nullptr;
  int* lines = nullptr;
  float *dc_part = nullptr, *lrs_part = nullptr;
  float* lrs_part2 = nullptr;     // second buffer of the sparse step's partials
  double *sigma_out = nullptr, *sigma_prev = nullptr;
  uint32_t *sup_out = nullptr, *sup_prior = nullptr;
  uint32_t* sup_out2 = nullptr;   // second buffer of the sparse step's support words
  DevPersist* persist = nullptr;
  DevCtrl* ctrl = nullptr;
  IterRec* hist = nullptr;
  // The small per-plan buffers (control block, statistics, Gram partials, W, V, sigma,
  // bitmaps, line table, twiddles) live in one contiguous allocation so that a kernel
  // starting on any SM touches few address-translation pages.
  unsigned char* arena = nullptr;
  size_t arena_bytes = 0, arena_used = 0;
  // Host-owned persistent fields; the device copy is refreshed by stream-ordered uploads.
  DevPersist hp{};
  // Pinned upload sources, a ring of kSlots: an upload takes the next slot, waiting only for
  // the upload made kSlots uploads earlier from it, so the host can queue several frames
  // ahead of the device.
  static constexpr int kSlots = 8;
  DevCtrl* h_ctrl = nullptr;
  DevPersist* h_persist_slots = nullptr;   // [kSlots]
  int* h_lines_slots = nullptr;            // [kSlots][plane]
  cudaEvent_t slot_done[kSlots] = {};
  bool slot_pending[kSlots] = {};
  int slot_next = 0;
  // host state
  int nlines = 0, m_cap = 0;
  bool have_mask = false, have_coils = false, have_data = false, state_ready = false;
  int iters_done = 0;
  size_t dev_bytes = 0;
  cudaGraph_t graph = nullptr;         // the captured per-frame graph (kept for batches)
  cudaGraphExec_t gexec = nullptr;
  bool graph_valid = false;
  unsigned graph_gen = 0;              // incremented at every capture
  // x-slab sharding: the reduced record the eigen kernel reads (device, caller-owned) while
  // lps_slab_iterate / lps_slab_end enqueue work; nullptr otherwise
  const float* slab_rec = nullptr;
  bool slab_open = false;
  // profiling: event pairs around every kernel of the frame graph, by kernel class
  bool profiling = false;
  std::vector<cudaEvent_t> ev;      // 2 per recorded launch
  std::vector<int> ev_class;        // class of each pair
  int ev_used = 0;
};

namespace lps {

// Reduction record of x-slab sharding (floats): [0..3] data-consistency statistic sums,
// [4..5] sparse-step sums, [6..7] zero, [8 .. 8 + 2 nc^2) the Gram (complex, row-major) -- the
// part the slabs add up -- then one float, max |T(X_0)|, that they take the maximum of.
constexpr int kSlabRecHead = 8;
inline size_t slab_sum_floats(int nc) { return (size_t)kSlabRecHead + 2 * (size_t)nc * nc; }
cudaError_t launch_slab_pack(const float2* gram_part, int nparts, int nc, const float* dc_part, int ndc,
                             const float* lrs_part, int nlrs, const DevCtrl* ctrl, float* rec, cudaStream_t st);

// Helpers of lps_api.cu used by the other host translation units.
int plan_build_graph(lps_plan* P);        // capture + instantiate the per-frame graph if stale
int plan_need_ready(lps_plan* P);         // coils, mask and data set
int plan_upload_persist(lps_plan* P, bool with_v);
int plan_frame_done(lps_plan* P);         // host bookkeeping after one frame of the graph ran
DcArgs plan_dc_args(lps_plan* P);
bool plan_is_device_ptr(const void* p);

}  // namespace lps

// internal.h -- shared host-side declarations of libds (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "ds.h"

namespace ds {

constexpr int kMaxP = 16;
constexpr int kMaxQ = 64;
constexpr int kMaxK = 16;

// Fast-path classes: (dtype, p/q, K) combinations with a hand-tuned TMA
// kernel instantiation.  Everything else runs on the general kernels.
enum FastClass : int {
  kFcNone = -1,
  kFcF32_38 = 0,  // float, 3/8, K=8
  kFcF32_12,      // float, 1/2, K=6
  kFcF32_23,      // float, 2/3, K=6
  kFcF16_38,
  kFcF16_12,
  kFcF16_23,
  kFcU8C3_38,     // uint8 RGB, 3/8, K=8
  kFcU8C3_12,     // uint8 RGB, 1/2, K=6
  kFcU8C3_23,     // uint8 RGB, 2/3, K=6
  kFcU8C3_CIF,    // uint8 RGB, horizontal 3/8 K=8, vertical 4/9 K=8 (the paper's CIF case)
  kFcU8C1_CIF,    // uint8 one plane (4:2:0 Y, U, V), the same axes
  kFcU8C1_38,     // uint8 one channel, 3/8, K=8
  kFcU8C1_12,     // uint8 one channel, 1/2, K=6
  kFcU8C1_23,     // uint8 one channel, 2/3, K=6
  kFcCount
};

// The last few tensor maps a plan's launches used, keyed by input pointer,
// frame count and tile shape (a plan is immutable but its launches may come
// from several host threads at once: the cache has its own lock).
struct TmapCache {
  struct Entry {
    CUtensorMap map;  // 64-byte aligned by its type
    const void* in = nullptr;
    int n_frames = 0, shape = 0;
    bool narrow = false;  // the (x, frame, row) map of a narrow tail strip
    bool used = false;
    unsigned long long stamp = 0;
  };
  std::mutex mu;
  Entry e[8];
  unsigned long long clock = 0;
};

}  // namespace ds

struct ds_plan {
  int in_h = 0, in_w = 0, channels = 1, elem_size = 4;
  // horizontal axis (along a row)
  int p = 1, q = 2, K = 2;
  ds_dtype dtype = DS_F32;
  int out_h = 0, out_w = 0;
  int b[ds::kMaxP] = {};                     // window start of each phase
  double w64[ds::kMaxP * ds::kMaxK] = {};    // FP64 taps [p][K]
  float w32[ds::kMaxP * ds::kMaxK] = {};     // (float) of w64
  short q14[ds::kMaxP * ds::kMaxK] = {};     // Q14 taps
  // vertical axis (along a column), the same tables
  int pv = 1, qv = 2, Kv = 2;
  int bv[ds::kMaxP] = {};
  double w64v[ds::kMaxP * ds::kMaxK] = {};
  float w32v[ds::kMaxP * ds::kMaxK] = {};
  short q14v[ds::kMaxP * ds::kMaxK] = {};
  ds_boundary boundary = DS_CLAMP;
  bool given_taps = false;                   // a tap table came from the caller
  int fast_class = ds::kFcNone;              // -1: general kernels only
  int row_blocks = 0;                        // fused tile: output row blocks per tile
  int ctas_per_sm = 0;                       // persistent grid: 0 = occupancy
  bool schedule_set = false;                 // row_blocks fixed by the caller or the autotuner;
                                             // else a launch too small to fill the GPU uses
                                             // shorter bands (more tiles).  Either way the
                                             // launch's last tiles run at a quarter band
  int shape = 0;                             // compiled tile shape of the fast class
  bool force_general = false;                // DS_NO_TMA or unsupported alignment
  std::unique_ptr<ds::TmapCache> tmaps;      // fast plans: recent tensor maps

  size_t in_frame_elems() const { return (size_t)in_h * in_w * channels; }
  size_t out_frame_elems() const { return (size_t)out_h * out_w * channels; }
};

namespace ds {

// Error reporting (thread-local message).  Errors are also logged at level 1.
void set_error(const char* fmt, ...);
// Logging to stderr, prefixed "[ds] ", when the DS_LOG environment variable
// (read once) is at least `level`: 1 = plans and errors, 2 = every launch too.
int log_level();
void log_msg(int level, const char* fmt, ...);
void clear_error();
ds_status cuda_fail(cudaError_t e, const char* what);

// Launch accounting (per host thread).
void count_launches(long long n);

// Plan helpers (plan.cpp).
int fast_class_of(int p, int q, int K, int pv, int qv, int Kv, ds_dtype dtype);
bool frame_tma_ok(const ds_plan* plan, const void* in, size_t frame_stride_bytes);

// Kernel launchers.
// fused_fast.cu: all jobs must have fast_class >= 0 and TMA-compatible input.
struct FastJob {
  const ds_plan* plan;
  const void* in;
  void* out;
  int n_frames;
};
ds_status launch_fast(const FastJob* jobs, int n, cudaStream_t stream);
// While non-null (on this thread), fused launches are being captured into a
// CUDA graph: each takes a scheduling slot of its own and records it here, to
// be given back with release_graph_slots when the graph is destroyed.
extern thread_local std::vector<int>* g_capture_slots;
void release_graph_slots(const std::vector<int>& slots);
int fast_max_jobs_per_launch();
// Tile shapes compiled for fast class `cls` (0 for none), what shape `shape`
// is, and the resident CTAs per SM of a plan's kernel at its current shape.
struct FastShapeInfo {
  int packets_per_lane, stage_rows, stages, warps_per_cta, ctas_per_sm_budget;
  int strip_pixels, frames_per_warp, smem_per_cta;
};
int fast_tile_shapes(int cls);
bool fast_shape_info(int cls, int shape, FastShapeInfo* out);
int fast_ctas_per_sm(const ds_plan* plan);
// Whether the fast kernel of class `cls` runs modular tilers on rows of
// in_w pixels (they have tile shape 0 only).
bool fast_wrap_fits(int cls, int in_w);
// reads and clears the status word (1: a wait gave up, 3: a bounds check
// failed, with kind and offset in info)
ds_status read_device_status(int* status, long long* info);
ds_status launch_timeout_probe(long long limit_cycles, cudaStream_t stream);
bool bounds_checked();  // built with -DDS_CHECK_BOUNDS
ds_status launch_bounds_probe(cudaStream_t stream);
ds_status debug_check_plan(const ds_plan* plan, std::string& msg);

// general.cu: any plan, any alignment.
ds_status launch_general_fused(const ds_plan* plan, const void* in, void* out, int n_frames,
                               cudaStream_t stream);
ds_status launch_unfused(const ds_plan* plan, const void* in, void* out, int n_frames,
                         void* workspace, cudaStream_t stream);

// Dispatch of one job to the best kernel (abi.cpp).
ds_status run_jobs(const ds_job* jobs, int n, cudaStream_t stream);

}  // namespace ds

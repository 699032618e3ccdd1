// tune.cpp -- autotuner of the fused kernel's tile schedule.
//
// The paper derives the launch topology of each repetitive task from its
// multiplicity with fixed threshold levels (Sec. 3.B.1, "Launch Topology").
// Here the topology is measured instead: every candidate band height (output
// row blocks per tile) is timed on the caller's buffers with CUDA events and
// the fastest is kept in the plan.  Every candidate computes the same bits
// (the per-output accumulation order does not depend on the tiling), so the
// choice only moves time.
#include <algorithm>
#include <vector>

#include "internal.h"

using namespace ds;

extern "C" {

ds_status ds_plan_autotune(ds_plan* plan, const void* in, void* out, int n_frames, void* stream, int iters,
                           int* best_row_blocks, float* best_us) {
  clear_error();
  if (!plan || !in || !out || n_frames < 1 || iters < 1) {
    set_error("ds_plan_autotune: bad arguments");
    return DS_ERR_ARG;
  }
  const int nby = (plan->out_h + plan->p - 1) / plan->p;
  std::vector<int> cand;
  for (int c : {3, 4, 6, 8, 10, 12, 16, 20, 24, 34, 48, 64})
    if (c <= nby) cand.push_back(c);
  if (cand.empty() || cand.back() < nby) cand.push_back(std::min(nby, 96));
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_fail(cudaGetLastError(), "ds_plan_autotune: events");
  }
  const int keep_rb = plan->row_blocks, keep_ctas = plan->ctas_per_sm;
  const bool keep_set = plan->schedule_set;
  plan->schedule_set = true;  // time each candidate as given
  int best = keep_rb;
  float best_t = 1e30f;
  ds_status s = DS_OK;
  for (int c : cand) {
    plan->row_blocks = c;
    s = ds_run_frames(plan, in, out, n_frames, stream);  // warm-up
    if (s != DS_OK) break;
    cudaEventRecord(e0, st);
    for (int i = 0; i < iters && s == DS_OK; ++i) s = ds_run_frames(plan, in, out, n_frames, stream);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    if (s != DS_OK) break;
    if (e != cudaSuccess) {
      s = cuda_fail(e, "ds_plan_autotune: timing");
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_t) {
      best_t = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  plan->ctas_per_sm = keep_ctas;
  if (s != DS_OK) {
    plan->row_blocks = keep_rb;
    plan->schedule_set = keep_set;
    return s;
  }
  plan->row_blocks = best;
  plan->schedule_set = true;
  if (best_row_blocks) *best_row_blocks = best;
  if (best_us) *best_us = best_t * 1000.0f / iters;
  return DS_OK;
}

}  // extern "C"

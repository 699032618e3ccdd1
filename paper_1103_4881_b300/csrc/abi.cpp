// abi.cpp -- extern "C" entry points of libds that launch work: single runs,
// batches, the unfused form, stream status, CUDA graphs and the host-buffer
// pipeline.  Each job goes to the fused TMA kernel when its plan has a fast
// class and its input satisfies the TMA alignment rules, else to the general
// fused kernel.
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

namespace ds {

namespace {

// NVTX range over one entry point (visible in timeline profilers; a no-op
// when no tool is attached).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

bool uses_fast(const ds_plan* pl, const void* in, int n_frames) {
  if (pl->fast_class < 0 || pl->force_general) return false;
  return frame_tma_ok(pl, in, pl->in_frame_elems() * pl->elem_size) && n_frames >= 1;
}

ds_status check_job(const ds_job& j, const char* who) {
  if (!j.plan || !j.in || !j.out || j.n_frames < 0) {
    set_error("%s: a job has a NULL plan or pointer, or a negative frame count", who);
    return DS_ERR_ARG;
  }
  return DS_OK;
}

}  // namespace

ds_status run_jobs(const ds_job* jobs, int n, cudaStream_t st) {
  std::vector<FastJob> fast;
  fast.reserve(n);
  for (int i = 0; i < n; ++i) {
    ds_status s = check_job(jobs[i], "ds_batch_run");
    if (s != DS_OK) return s;
  }
  for (int i = 0; i < n; ++i) {
    const ds_job& j = jobs[i];
    const int nf = j.n_frames == 0 ? 1 : j.n_frames;
    if (uses_fast(j.plan, j.in, nf)) {
      fast.push_back(FastJob{j.plan, j.in, j.out, nf});
    } else {
      ds_status s = launch_general_fused(j.plan, j.in, j.out, nf, st);
      if (s != DS_OK) return s;
    }
  }
  if (!fast.empty()) return launch_fast(fast.data(), (int)fast.size(), st);
  return DS_OK;
}

}  // namespace ds

using namespace ds;

struct ds_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long launches = 0;
  std::vector<int> slots;  // tile-scheduling slots of the captured fused launches
};

struct ds_pipeline {
  const ds_plan* plan = nullptr;
  int chunk = 1, depth = 2;
  size_t in_chunk_bytes = 0, out_chunk_bytes = 0;
  std::vector<void*> dev_in, dev_out;
  std::vector<cudaStream_t> streams;
};

extern "C" {

ds_status ds_run(const ds_plan* plan, const void* in, void* out, void* stream) {
  return ds_run_frames(plan, in, out, 1, stream);
}

ds_status ds_run_frames(const ds_plan* plan, const void* in, void* out, int n_frames, void* stream) {
  clear_error();
  if (!plan || !in || !out || n_frames < 0) {
    set_error("ds_run: NULL plan or pointer, or negative frame count");
    return DS_ERR_ARG;
  }
  if (n_frames == 0) return DS_OK;
  Range r("ds_run_frames");
  ds_job j{plan, in, out, n_frames};
  return run_jobs(&j, 1, (cudaStream_t)stream);
}

ds_status ds_batch_run(const ds_job* jobs, int n, void* stream) {
  clear_error();
  if (n < 0 || (n > 0 && !jobs)) {
    set_error("ds_batch_run: bad job array");
    return DS_ERR_ARG;
  }
  if (n == 0) return DS_OK;
  Range r("ds_batch_run");
  return run_jobs(jobs, n, (cudaStream_t)stream);
}

size_t ds_plan_workspace_bytes(const ds_plan* plan) {
  if (!plan) return 0;
  const size_t inter = (plan->dtype == DS_U8 || plan->dtype == DS_U8_RGB) ? 1 : 4;
  return (size_t)plan->in_h * plan->out_w * plan->channels * inter;
}

ds_status ds_run_unfused(const ds_plan* plan, const void* in, void* out, int n_frames, void* workspace,
                         size_t workspace_bytes, void* stream) {
  clear_error();
  if (!plan || !in || !out || !workspace || n_frames < 0) {
    set_error("ds_run_unfused: NULL plan or pointer, or negative frame count");
    return DS_ERR_ARG;
  }
  if (workspace_bytes < ds_plan_workspace_bytes(plan) * (size_t)n_frames) {
    set_error("ds_run_unfused: workspace of %zu bytes, need %zu", workspace_bytes,
              ds_plan_workspace_bytes(plan) * (size_t)n_frames);
    return DS_ERR_ARG;
  }
  if (n_frames == 0) return DS_OK;
  Range r("ds_run_unfused");
  return launch_unfused(plan, in, out, n_frames, workspace, (cudaStream_t)stream);
}

ds_status ds_debug_check_plan(const ds_plan* plan) {
  clear_error();
  if (!plan) {
    set_error("ds_debug_check_plan: NULL plan");
    return DS_ERR_ARG;
  }
  std::string msg;
  ds_status s = debug_check_plan(plan, msg);
  if (s != DS_OK) set_error("ds_debug_check_plan: %s", msg.c_str());
  return s;
}

ds_status ds_stream_check(void* stream) {
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "ds_stream_check");
  int status = 0;
  long long info[2];
  ds_status s = read_device_status(&status, info);
  if (s != DS_OK) return s;
  if (status == 3) {
    static const char* kinds[] = {"", "shared-memory row read", "border write", "output row", "tensor copy"};
    set_error("a bounds check failed: %s at offset %lld", info[0] >= 1 && info[0] <= 4 ? kinds[info[0]] : "probe",
              info[1]);
    return DS_ERR_BOUNDS;
  }
  if (status != 0) {
    set_error("a kernel gave up a bounded wait (device status %d)", status);
    return DS_ERR_TIMEOUT;
  }
  return DS_OK;
}

int ds_bounds_checked(void) { return bounds_checked() ? 1 : 0; }

ds_status ds_debug_bounds_probe(void* stream) {
  clear_error();
  if (!bounds_checked()) {
    set_error("ds_debug_bounds_probe: this library was built without DS_CHECK_BOUNDS");
    return DS_ERR_UNSUPPORTED;
  }
  return launch_bounds_probe((cudaStream_t)stream);
}

ds_status ds_debug_timeout_probe(long long limit_cycles, void* stream) {
  clear_error();
  if (limit_cycles < 0 || limit_cycles > 4000000000ll) {
    set_error("ds_debug_timeout_probe: limit of %lld cycles outside [0, 4e9]", limit_cycles);
    return DS_ERR_ARG;
  }
  return launch_timeout_probe(limit_cycles, (cudaStream_t)stream);
}

// ------------------------------------------------------------------ graphs

ds_graph* ds_graph_create(const ds_job* jobs, int n) {
  clear_error();
  if (n < 1 || !jobs) {
    set_error("ds_graph_create: empty batch");
    return nullptr;
  }
  ds_graph* g = new (std::nothrow) ds_graph();
  if (!g) {
    set_error("ds_graph_create: out of host memory");
    return nullptr;
  }
  cudaStream_t st = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cuda_fail(e, "ds_graph_create: stream");
    delete g;
    return nullptr;
  }
  ds_launch_count();  // the nodes captured below are counted for the graph
  e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  g_capture_slots = &g->slots;
  ds_status s = (e == cudaSuccess) ? run_jobs(jobs, n, st) : cuda_fail(e, "begin capture");
  g_capture_slots = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(st, &g->graph);
  g->launches = ds_launch_count();
  cudaStreamDestroy(st);
  if (s == DS_OK && e2 != cudaSuccess) s = cuda_fail(e2, "end capture");
  if (s == DS_OK) {
    e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) s = cuda_fail(e, "graph instantiate");
  }
  if (s != DS_OK) {
    ds_graph_destroy(g);
    return nullptr;
  }
  return g;
}

ds_status ds_graph_launch(ds_graph* g, void* stream) {
  if (!g || !g->exec) {
    set_error("ds_graph_launch: NULL graph");
    return DS_ERR_ARG;
  }
  cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "ds_graph_launch");
  count_launches(g->launches);
  return DS_OK;
}

void ds_graph_destroy(ds_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  release_graph_slots(g->slots);
  delete g;
}

// ---------------------------------------------------------------- pipeline

void ds_pipeline_destroy(ds_pipeline* pp) {
  if (!pp) return;
  for (cudaStream_t s : pp->streams)
    if (s) cudaStreamSynchronize(s);
  for (void* p : pp->dev_in) cudaFree(p);
  for (void* p : pp->dev_out) cudaFree(p);
  for (cudaStream_t s : pp->streams)
    if (s) cudaStreamDestroy(s);
  delete pp;
}

ds_pipeline* ds_pipeline_create(const ds_plan* plan, int chunk_frames, int depth) {
  clear_error();
  if (!plan || chunk_frames < 1 || depth < 1 || depth > 16) {
    set_error("ds_pipeline_create: bad arguments");
    return nullptr;
  }
  ds_pipeline* pp = new (std::nothrow) ds_pipeline();
  if (!pp) {
    set_error("ds_pipeline_create: out of host memory");
    return nullptr;
  }
  pp->plan = plan;
  pp->chunk = chunk_frames;
  pp->depth = depth;
  pp->in_chunk_bytes = plan->in_frame_elems() * plan->elem_size * (size_t)chunk_frames;
  pp->out_chunk_bytes = plan->out_frame_elems() * plan->elem_size * (size_t)chunk_frames;
  for (int i = 0; i < depth; ++i) {
    void *a = nullptr, *b = nullptr;
    cudaStream_t s = nullptr;
    if (cudaMalloc(&a, pp->in_chunk_bytes) != cudaSuccess || cudaMalloc(&b, pp->out_chunk_bytes) != cudaSuccess) {
      if (a) cudaFree(a);
      set_error("ds_pipeline_create: device allocation of %zu bytes failed", pp->in_chunk_bytes + pp->out_chunk_bytes);
      ds_pipeline_destroy(pp);
      return nullptr;
    }
    pp->dev_in.push_back(a);
    pp->dev_out.push_back(b);
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      set_error("ds_pipeline_create: stream creation failed");
      ds_pipeline_destroy(pp);
      return nullptr;
    }
    pp->streams.push_back(s);
  }
  return pp;
}

ds_status ds_pipeline_run(ds_pipeline* pp, const void* in, void* out, int n_frames) {
  clear_error();
  if (!pp || !in || !out || n_frames < 0) {
    set_error("ds_pipeline_run: bad arguments");
    return DS_ERR_ARG;
  }
  Range r("ds_pipeline_run");
  const size_t fin = pp->in_chunk_bytes / pp->chunk, fout = pp->out_chunk_bytes / pp->chunk;
  int slot = 0;
  for (int f0 = 0; f0 < n_frames; f0 += pp->chunk, slot = (slot + 1) % pp->depth) {
    const int nf = std::min(pp->chunk, n_frames - f0);
    cudaStream_t s = pp->streams[slot];
    // chunk i reuses the buffers of chunk i - depth: same stream, so ordered
    cudaError_t e = cudaMemcpyAsync(pp->dev_in[slot], (const char*)in + fin * f0, fin * nf, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "ds_pipeline_run: host to device copy");
    ds_job j{pp->plan, pp->dev_in[slot], pp->dev_out[slot], nf};
    ds_status st = run_jobs(&j, 1, s);
    if (st != DS_OK) return st;
    e = cudaMemcpyAsync((char*)out + fout * f0, pp->dev_out[slot], fout * nf, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "ds_pipeline_run: device to host copy");
  }
  for (cudaStream_t s : pp->streams) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "ds_pipeline_run: synchronise");
  }
  return DS_OK;
}

}  // extern "C"

// serve.cpp -- the continuous-batching request loop, native: admission by
// device memory, batching, streams, completions and latency, with no
// allocation and no interpreter on the request path.
//
// Requests are single frames of any plan (size, ratio, dtype).  A queued
// request is admitted when a stream slot is free and its bytes fit the
// memory budget; the admitted group of a slot is one ds_batch_run (one
// persistent launch per kernel class present) on that slot's stream,
// wrapped, in the copy mode, in the host-to-device copies of its inputs into
// the slot's resident device arena and the device-to-host copies of its
// outputs.  Requests that arrive while earlier groups run are admitted as
// slots and memory free up, so their work overlaps on the device.  Latency
// is arrival -> observed completion of the request's group (the loop polls
// the slots' events).
//
// The paper's measurements are of its whole downscaler on a video stream,
// host-device transfers included (Sec. 4); the copy mode is that end-to-end
// form, the kernel-only mode takes inputs already resident on the device.
#include <algorithm>
#include <chrono>
#include <deque>
#include <new>
#include <thread>
#include <vector>

#include "internal.h"

using namespace ds;

struct ds_server {
  size_t budget = 0;
  int n_streams = 0, max_batch = 0;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  std::vector<void*> arenas;  // copy mode: one device arena of budget / n_streams bytes per slot
  size_t arena_bytes = 0;
};

namespace {

constexpr size_t kAlign = 256;  // arena offsets: TMA and vector loads want 16 bytes, keep whole 256 B sectors
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Slot {
  bool busy = false;
  std::vector<int> reqs;
  size_t bytes = 0;
};

void destroy_server(ds_server* sv) {
  for (cudaStream_t s : sv->streams)
    if (s) cudaStreamSynchronize(s);
  for (void* p : sv->arenas)
    if (p) cudaFree(p);
  for (cudaEvent_t e : sv->events)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t s : sv->streams)
    if (s) cudaStreamDestroy(s);
  delete sv;
}

ds_status ensure_arenas(ds_server* sv) {
  if (!sv->arenas.empty()) return DS_OK;
  sv->arena_bytes = sv->budget / (size_t)sv->n_streams / kAlign * kAlign;
  for (int i = 0; i < sv->n_streams; ++i) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, sv->arena_bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();  // a failed allocation is not a sticky error: clear it
      for (void* q : sv->arenas) cudaFree(q);
      sv->arenas.clear();
      set_error("ds_server_run: device arena of %zu bytes: %s", sv->arena_bytes, cudaGetErrorString(e));
      return DS_ERR_NOMEM;
    }
    sv->arenas.push_back(p);
  }
  return DS_OK;
}

}  // namespace

extern "C" {

ds_server* ds_server_create(size_t mem_budget_bytes, int n_streams, int max_batch) {
  clear_error();
  if (mem_budget_bytes < kAlign || n_streams < 1 || n_streams > 64 || max_batch < 1 || max_batch > 4096) {
    set_error("ds_server_create: budget of at least %zu bytes, 1..64 streams and 1..4096 requests per batch",
              kAlign);
    return nullptr;
  }
  ds_server* sv = new (std::nothrow) ds_server();
  if (!sv) {
    set_error("ds_server_create: out of host memory");
    return nullptr;
  }
  sv->budget = mem_budget_bytes;
  sv->n_streams = n_streams;
  sv->max_batch = max_batch;
  for (int i = 0; i < n_streams; ++i) {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (s) sv->streams.push_back(s);
    if (ev) sv->events.push_back(ev);
    if (e != cudaSuccess) {
      cuda_fail(e, "ds_server_create: streams and events");
      destroy_server(sv);
      return nullptr;
    }
  }
  return sv;
}

void ds_server_destroy(ds_server* sv) {
  if (sv) destroy_server(sv);
}

ds_status ds_server_run(ds_server* sv, const ds_request* reqs, int n, int flags, double* latency_ms,
                        ds_serve_stats* stats) {
  clear_error();
  if (!sv || n < 0 || (n > 0 && !reqs)) {
    set_error("ds_server_run: NULL server or requests");
    return DS_ERR_ARG;
  }
  const bool realtime = (flags & DS_SERVE_REALTIME) != 0;
  const bool copies = (flags & DS_SERVE_COPIES) != 0;
  const bool plain = (flags & DS_SERVE_PLAIN) != 0;
  if (flags & ~(DS_SERVE_REALTIME | DS_SERVE_COPIES | DS_SERVE_PLAIN)) {
    set_error("ds_server_run: unknown flags 0x%x", flags);
    return DS_ERR_ARG;
  }
  if (plain && copies) {
    set_error("ds_server_run: DS_SERVE_PLAIN takes device buffers (no DS_SERVE_COPIES)");
    return DS_ERR_ARG;
  }
  // bytes of each request: input and output, each padded to the arena alignment
  std::vector<size_t> need(n), fin(n), fout(n);
  for (int i = 0; i < n; ++i) {
    const ds_request& r = reqs[i];
    if (!r.plan || !r.in || !r.out) {
      set_error("ds_server_run: request %d has a NULL plan or buffer", i);
      return DS_ERR_ARG;
    }
    ds_plan_frame_bytes(r.plan, &fin[i], &fout[i]);
    need[i] = align_up(fin[i]) + align_up(fout[i]);
  }
  if (copies) {
    ds_status s = ensure_arenas(sv);
    if (s != DS_OK) return s;
  }
  const size_t cap = copies ? sv->arena_bytes : sv->budget;  // what one group may hold
  for (int i = 0; i < n; ++i)
    if (need[i] > cap) {
      set_error("ds_server_run: request %d needs %zu bytes, more than a %s of %zu", i, need[i],
                copies ? "slot's arena" : "budget", cap);
      return DS_ERR_ARG;
    }
  // arrival order (stable)
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  if (realtime)
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return reqs[a].arrival_s < reqs[b].arrival_s; });
  ds_serve_stats st{};
  ds_launch_count();
  std::vector<ds_job> jobs((size_t)(plain ? 1 : sv->max_batch));
  const auto t0 = std::chrono::steady_clock::now();
  auto elapsed = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); };
  ds_status status = DS_OK;

  // Waiting for an arrival or a completion: the loop keeps its core, with the
  // CPU's spin hint, rather than yielding it -- a yield on a busy host can
  // hand the core to another process for a scheduler time slice, which then
  // shows as request latency.
  auto relax = []() {
#if defined(__x86_64__) || defined(__i386__)
    __builtin_ia32_pause();
#elif defined(__aarch64__)
    asm volatile("yield" ::: "memory");
#else
    std::this_thread::yield();
#endif
  };

  if (plain) {
    // the baseline: one plain fused launch per request, in arrival order, on one stream
    for (int k = 0; k < n && status == DS_OK; ++k) {
      const int i = order[k];
      if (realtime)
        while (elapsed() < reqs[i].arrival_s) relax();
      jobs[0] = ds_job{reqs[i].plan, reqs[i].in, reqs[i].out, 1};
      status = run_jobs(jobs.data(), 1, sv->streams[0]);
    }
    cudaError_t e = cudaStreamSynchronize(sv->streams[0]);
    if (status == DS_OK && e != cudaSuccess) status = cuda_fail(e, "ds_server_run: synchronise");
    st.completed = status == DS_OK ? n : 0;
    st.batches = n;
    st.max_batch = n > 0 ? 1 : 0;
    st.wall_s = elapsed();
    if (latency_ms)  // one completion for all: the stream is waited on once at the end
      for (int i = 0; i < n; ++i) latency_ms[i] = 1e3 * (st.wall_s - (realtime ? reqs[i].arrival_s : 0.0));
    st.launches = ds_launch_count();
    if (stats) *stats = st;
    return status;
  }

  std::vector<Slot> slots((size_t)sv->n_streams);
  std::deque<int> queue;
  size_t admitted = 0;
  int next = 0, done = 0;
  while (done < n && status == DS_OK) {
    bool progress = false;
    const double now = elapsed();
    while (next < n && (!realtime || reqs[order[next]].arrival_s <= now)) queue.push_back(order[next++]);
    st.max_queue = std::max(st.max_queue, (int)queue.size());
    // completions
    for (int s = 0; s < sv->n_streams; ++s) {
      Slot& sl = slots[(size_t)s];
      if (!sl.busy) continue;
      cudaError_t q = cudaEventQuery(sv->events[(size_t)s]);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) {
        status = cuda_fail(q, "ds_server_run: a batch failed");
        break;
      }
      const double t_done = elapsed();
      for (int i : sl.reqs)
        if (latency_ms) latency_ms[i] = 1e3 * (t_done - (realtime ? reqs[i].arrival_s : 0.0));
      done += (int)sl.reqs.size();
      admitted -= sl.bytes;
      sl.busy = false;
      sl.reqs.clear();
      progress = true;
    }
    if (status != DS_OK) break;
    // admission and launch on a free slot
    if (!queue.empty()) {
      int free_slot = -1;
      for (int s = 0; s < sv->n_streams && free_slot < 0; ++s)
        if (!slots[(size_t)s].busy) free_slot = s;
      if (free_slot >= 0) {
        Slot& sl = slots[(size_t)free_slot];
        const size_t room = copies ? sv->arena_bytes : sv->budget - admitted;
        size_t bytes = 0;
        while (!queue.empty() && (int)sl.reqs.size() < sv->max_batch && bytes + need[(size_t)queue.front()] <= room &&
               (copies ? admitted + bytes + need[(size_t)queue.front()] <= sv->budget : true)) {
          bytes += need[(size_t)queue.front()];
          sl.reqs.push_back(queue.front());
          queue.pop_front();
        }
        if (!sl.reqs.empty()) {
          cudaStream_t cs = sv->streams[(size_t)free_slot];
          char* arena = copies ? static_cast<char*>(sv->arenas[(size_t)free_slot]) : nullptr;
          size_t off = 0;
          int k = 0;
          for (int i : sl.reqs) {
            if (copies) {
              char* din = arena + off;
              char* dout = arena + off + align_up(fin[(size_t)i]);
              off += need[(size_t)i];
              cudaError_t e = cudaMemcpyAsync(din, reqs[i].in, fin[(size_t)i], cudaMemcpyHostToDevice, cs);
              if (e != cudaSuccess) {
                status = cuda_fail(e, "ds_server_run: host to device copy");
                break;
              }
              jobs[(size_t)k++] = ds_job{reqs[i].plan, din, dout, 1};
            } else {
              jobs[(size_t)k++] = ds_job{reqs[i].plan, reqs[i].in, reqs[i].out, 1};
            }
          }
          if (status == DS_OK) status = run_jobs(jobs.data(), k, cs);
          if (status == DS_OK && copies) {
            for (int m = 0; m < k; ++m) {
              const int i = sl.reqs[(size_t)m];
              cudaError_t e = cudaMemcpyAsync(reqs[i].out, jobs[(size_t)m].out, fout[(size_t)i],
                                              cudaMemcpyDeviceToHost, cs);
              if (e != cudaSuccess) {
                status = cuda_fail(e, "ds_server_run: device to host copy");
                break;
              }
            }
          }
          if (status == DS_OK) {
            cudaError_t e = cudaEventRecord(sv->events[(size_t)free_slot], cs);
            if (e != cudaSuccess) status = cuda_fail(e, "ds_server_run: event");
          }
          if (status != DS_OK) break;
          sl.busy = true;
          sl.bytes = bytes;
          admitted += bytes;
          st.peak_admitted_bytes = std::max(st.peak_admitted_bytes, admitted);
          st.batches += 1;
          st.max_batch = std::max(st.max_batch, (int)sl.reqs.size());
          progress = true;
        }
      }
    }
    if (!progress) relax();
  }
  // leave nothing in flight (also after an error)
  for (cudaStream_t s : sv->streams) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (status == DS_OK && e != cudaSuccess) status = cuda_fail(e, "ds_server_run: synchronise");
  }
  st.completed = done;
  st.wall_s = elapsed();
  st.launches = ds_launch_count();
  if (stats) *stats = st;
  return status;
}

}  // extern "C"

// fused_fast.cu -- host side of the fused horizontal + vertical kernel
// (rows.cuh): the table of compiled classes and tile shapes, tensor maps,
// tile schedules (band heights, launch tails), scheduling slots, launches,
// and the device status word.
//
// A batch is cut into one persistent launch per kernel class (dtype, ratio
// and taps of each axis; the paper's downscaler filter, Sec. 3).  The jobs of
// a launch travel in its __grid_constant__ parameters, with their tiles
// numbered in job order; warps take tiles from a per-launch counter.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "rows.cuh"

namespace ds {
namespace rows {

// The status word and scheduling counters of every launch on this GPU.
__device__ DevState g_dev_state;

namespace {

// Exercise of the timeout path: one warp waits, with the kernels' bounded
// wait, on an mbarrier that nothing will ever complete (no copy is issued
// and no thread arrives), gives up after `limit` cycles and records the
// timeout in the status word exactly as k_rows does.
__global__ void k_timeout_probe(long long limit) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  const bool ok = __all_sync(0xffffffffu, mbar_wait(&bar, 0u, limit));
  if (!ok && threadIdx.x == 0) atomicCAS(&g_dev_state.status, 0, kStatusTimeout);
}

// Exercise of the bounds-check report (bounds-checking builds): one thread
// runs the kernels' check on an offset one past a 64-byte buffer, which
// fails; the access itself is never made.
__global__ void k_bounds_probe() {
  if (threadIdx.x == 0) {
    const long long off = 64, size = 64;
    if (off + 1 > size) bounds_fail(&g_dev_state, 9, off);
  }
}

// ---------------------------------------------------------------------------
// compiled classes and shapes
// ---------------------------------------------------------------------------
const RowsTable& table() {
  static RowsTable t = {};
  static std::once_flag once;
  std::call_once(once, [] {
    register_f32(t);
    register_f16(t);
    register_u8rgb(t);
    register_u8c1(t);
    register_cif(t);
  });
  return t;
}

const RowsEntry& entry(int cls, int shape) {
  const RowsEntry& e = table()[cls][shape >= 0 && shape < kShapes ? shape : 0];
  return e.present ? e : table()[cls][0];
}

const RowsEntry& entry_of(const ds_plan* pl) { return entry(pl->fast_class, pl->shape); }

// Device address of g_dev_state on the current device (the array's name is
// only a host-side stand-in in host code), looked up once per device.
DevState* dev_state() {
  static DevState* addr[64] = {};
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_dev_state) != cudaSuccess) return nullptr;
    addr[dev] = static_cast<DevState*>(p);
  }
  return addr[dev];
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// Resident CTAs per SM of a kernel, computed once per kernel (one device).
int ctas_per_sm(const KernelInfo& ki) {
  static std::mutex mu;
  static std::vector<std::pair<const void*, int>> cache;
  std::lock_guard<std::mutex> lock(mu);
  for (auto& e : cache)
    if (e.first == ki.fn) return e.second;
  int occ = 0;
  if (cudaFuncSetAttribute(ki.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, ki.smem) != cudaSuccess) return 0;
  // all of the SM's configurable memory as shared memory: the rings set the
  // resident CTAs of most classes, and the kernels read their inputs through
  // TMA into shared memory, not through L1
  if (cudaFuncSetAttribute(ki.fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
      cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ki.fn, ki.threads, ki.smem) != cudaSuccess) return 0;
  cache.emplace_back(ki.fn, occ);
  return occ;
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// int16 tap pairs of one axis for dp2a (see ClassTaps::tap2h).
void pair_taps(const short* q14, int p, int K, uint32_t (*out)[kMaxPhases][kMaxPairs]) {
  for (int par = 0; par < 2; ++par)
    for (int j = 0; j < p; ++j)
      for (int i = 0; i < kMaxPairs; ++i) {
        const int ta = 2 * i - par, tb = 2 * i + 1 - par;
        const int qa = (ta >= 0 && ta < K) ? q14[j * K + ta] : 0;
        const int qb = (tb >= 0 && tb < K) ? q14[j * K + tb] : 0;
        out[par][j][i] = (uint32_t)(uint16_t)(int16_t)qa | ((uint32_t)(uint16_t)(int16_t)qb << 16);
      }
}

// The launch tap tables of a plan with a fast class: FP32 taps (or Q14 taps
// as floats) per axis, and the int16 pairs of the Q14 taps for dp2a.
void plan_taps(const ds_plan* pl, ClassTaps& t) {
  std::memset(&t, 0, sizeof(t));
  const bool u8 = pl->dtype == DS_U8 || pl->dtype == DS_U8_RGB;
  for (int i = 0; i < pl->p * pl->K; ++i) t.taps[i] = u8 ? (float)pl->q14[i] : pl->w32[i];
  for (int i = 0; i < pl->pv * pl->Kv; ++i) t.tapsv[i] = u8 ? (float)pl->q14v[i] : pl->w32v[i];
  if (u8) {
    pair_taps(pl->q14, pl->p, pl->K, t.tap2h);
    pair_taps(pl->q14v, pl->pv, pl->Kv, t.tap2v);
  }
}

// The taps of fast class `cls` with the library's own taps.  They depend only
// on its axes: built once for every class with a throwaway plan.
const ClassTaps& class_taps(int cls) {
  static ClassTaps all[kFcCount];
  static std::once_flag once;
  std::call_once(once, [] {
    std::memset(all, 0, sizeof(all));
    struct Axes {
      int p, q, K, pv, qv, Kv;
      ds_dtype dt;
    };
    std::vector<Axes> specs;
    const int pq[3][3] = {{3, 8, 8}, {1, 2, 6}, {2, 3, 6}};
    const ds_dtype dts[4] = {DS_F32, DS_F16, DS_U8_RGB, DS_U8};
    for (int d = 0; d < 4; ++d)
      for (int r = 0; r < 3; ++r)
        specs.push_back({pq[r][0], pq[r][1], pq[r][2], pq[r][0], pq[r][1], pq[r][2], dts[d]});
    specs.push_back({3, 8, 8, 4, 9, 8, DS_U8_RGB});
    specs.push_back({3, 8, 8, 4, 9, 8, DS_U8});
    for (const Axes& a : specs) {
      ds_plan_desc d{};
      d.in_h = d.in_w = 72;
      d.ratio_h = ds_ratio{a.p, a.q};
      d.taps_h = a.K;
      d.ratio_v = ds_ratio{a.pv, a.qv};
      d.taps_v = a.Kv;
      d.dtype = a.dt;
      d.boundary = DS_CLAMP;
      ds_plan* pl = ds_plan_create_ex(&d);
      if (!pl || pl->fast_class < 0) {
        ds_destroy(pl);
        continue;
      }
      plan_taps(pl, all[pl->fast_class]);
      ds_destroy(pl);
    }
  });
  return all[cls];
}

// Tile geometry of a job (everything but the tensor map).  `band`: output
// row blocks per tile, 0 = the plan's.
void fill_job_geometry(JobDesc& jd, const ds_plan* pl, void* out, int n_frames, int band = 0) {
  const HostGeom& hg = entry_of(pl).geom;
  jd.nar = 0;
  jd.strip0 = 0;
  jd.out = out;
  jd.out_frame = (long long)pl->out_frame_elems();
  jd.H = pl->in_h;
  jd.W = pl->in_w;
  jd.OH = pl->out_h;
  jd.OW = pl->out_w;
  jd.nframes = n_frames;
  jd.cls = pl->fast_class;
  const int nbx = (pl->out_w + hg.p - 1) / hg.p;
  const int nby = (pl->out_h + hg.pv - 1) / hg.pv;
  jd.strips = (nbx + hg.sblk - 1) / hg.sblk;
  jd.rbc = std::max(1, std::min(band > 0 ? band : pl->row_blocks, nby));
  jd.chunks = (nby + jd.rbc - 1) / jd.rbc;
  jd.tiles = jd.strips * jd.chunks * ((n_frames + hg.fpw - 1) / hg.fpw);  // per group of fpw frames
  jd.out_vec = (((uintptr_t)out & 3u) == 0 && ((size_t)pl->out_w * pl->channels) % 4 == 0) ? 1 : 0;
  jd.wrap = pl->boundary == DS_WRAP ? 1 : 0;
}

// The tensor map of a job's input: 3-D (row bytes / 8 eight-byte elements, H
// rows, n frames), boxes of the shape's strip window by its stage rows.  A
// narrow tail strip's map orders the axes (x, frame, row) instead, with boxes
// of its window by 2 frames by the stage rows, so that a box lands two
// frames' windows side by side in each row.  Plans keep the maps of their
// last few (input, frame count, shape, kind) in a small cache, so repeated
// launches on the same buffers skip the encode.
ds_status job_tensor_map(const FastJob& job, CUtensorMap* out, bool narrow = false) {
  const ds_plan* pl = job.plan;
  TmapCache* tc = pl->tmaps.get();
  if (tc) {
    std::lock_guard<std::mutex> lock(tc->mu);
    for (TmapCache::Entry& e : tc->e)
      if (e.used && e.in == job.in && e.n_frames == job.n_frames && e.shape == pl->shape && e.narrow == narrow) {
        e.stamp = ++tc->clock;
        std::memcpy(out, &e.map, sizeof(CUtensorMap));
        return DS_OK;
      }
  }
  const HostGeom& hg = entry_of(pl).geom;
  auto enc = encode_fn();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return DS_ERR_CUDA;
  }
  const cuuint64_t row_bytes = (cuuint64_t)pl->in_w * pl->channels * hg.sz;  // a multiple of 16
  cuuint64_t dims[3] = {row_bytes / kTmaElem, (cuuint64_t)pl->in_h, (cuuint64_t)job.n_frames};
  cuuint64_t strides[2] = {row_bytes, row_bytes * (cuuint64_t)pl->in_h};
  cuuint32_t box[3] = {(cuuint32_t)hg.boxe, (cuuint32_t)hg.sr, 1};
  if (narrow) {
    dims[1] = (cuuint64_t)job.n_frames;
    dims[2] = (cuuint64_t)pl->in_h;
    strides[0] = row_bytes * (cuuint64_t)pl->in_h;
    strides[1] = row_bytes;
    box[0] = (cuuint32_t)(hg.wn / kTmaElem);
    box[1] = 2;
    box[2] = (cuuint32_t)hg.sr;
  }
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(out, hg.dt, 3, const_cast<void*>(job.in), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d) for a %dx%d frame", (int)r, pl->in_h, pl->in_w);
    return DS_ERR_CUDA;
  }
  if (tc) {
    std::lock_guard<std::mutex> lock(tc->mu);
    TmapCache::Entry* victim = &tc->e[0];
    for (TmapCache::Entry& e : tc->e) {
      if (!e.used) {
        victim = &e;
        break;
      }
      if (e.stamp < victim->stamp) victim = &e;
    }
    victim->used = true;
    victim->in = job.in;
    victim->n_frames = job.n_frames;
    victim->shape = pl->shape;
    victim->narrow = narrow;
    victim->stamp = ++tc->clock;
    std::memcpy(&victim->map, out, sizeof(CUtensorMap));
  }
  return DS_OK;
}

// Whether a plan's frames take a narrow tail-strip job: one-channel classes
// with frame pairs, clamp-to-edge tilers, a last strip of at most npn packets
// whose border fix is at most one element per lane of the four frames.
bool narrow_split(const ds_plan* pl) {
  const RowsEntry& e = entry_of(pl);
  if (!e.geom.narrow || pl->boundary == DS_WRAP) return false;
  const int npk = (pl->out_w + e.geom.p - 1) / e.geom.p;  // packets with outputs
  const int strips = (npk + e.geom.sblk - 1) / e.geom.sblk;
  return npk - (strips - 1) * e.geom.sblk <= e.geom.npn && e.narrow_fix(strips - 1, pl->in_w, pl->out_w) <= 32;
}

// Split a job descriptor (geometry filled) into the job without its last
// strip (none if that was its only strip) and the last strip's narrow job,
// four frames per tile.  Returns the number of descriptors written to out.
int split_narrow_geometry(const JobDesc& full, JobDesc* out) {
  int n = 0;
  if (full.strips > 1) {
    out[n] = full;
    out[n].strips = full.strips - 1;
    out[n].tiles = out[n].strips * full.chunks * ((full.nframes + 1) / 2);
    ++n;
  }
  out[n] = full;
  out[n].nar = 1;
  out[n].strip0 = full.strips - 1;
  out[n].strips = 1;
  out[n].tiles = full.chunks * ((full.nframes + 3) / 4);
  return n + 1;
}

ds_status encode_job(JobDesc& jd, const FastJob& job, int band) {
  // (modular tilers too: their stages that lie inside the frame take the
  // tensor copy, the others row copies)
  ds_status s = job_tensor_map(job, &jd.tmap);
  if (s != DS_OK) return s;
  fill_job_geometry(jd, job.plan, job.out, job.n_frames, band);
  jd.in = static_cast<const uint8_t*>(job.in);
  return DS_OK;
}

// The descriptors of one job: encode_job's, or with `narrow` its split into
// the job without the last strip and the narrow tail-strip job (which gets
// its own tensor map).  Returns the number written to out (1 or 2).
ds_status encode_job_split(JobDesc* out, int room, const FastJob& job, int band, bool narrow, int* n) {
  JobDesc full;
  ds_status s = encode_job(full, job, band);
  if (s != DS_OK) return s;
  if (!narrow || room < 2) {
    out[0] = full;
    *n = 1;
    return DS_OK;
  }
  *n = split_narrow_geometry(full, out);
  return job_tensor_map(job, &out[*n - 1].tmap, true);
}

// Band heights (output row blocks per tile) of the jobs of one launch.  A
// tile is processed serially by one warp, and tiles are handed out in job
// order, so:
//  - a launch with fewer block rows of work than the GPU has pipelines
//    finishes sooner with shorter bands: the band is cut to
//    ceil(block rows / pipelines), never above the plans' own value (plans
//    whose band the caller or the autotuner fixed keep theirs);
//  - the launch ends when the last warp finishes its last tile, so the work
//    at the end (about two tiles per pipeline) runs at a quarter of the band,
//    the last job being split by frames where the boundary falls inside it.
struct BandedJob {
  FastJob job;
  int band;  // 0 = the plan's
};

// The launch's last tiles, from the end: tiles per pipeline at band / div.
struct TailLevel {
  int div, tiles_per_pipeline;
};
constexpr TailLevel kTail[] = {{4, 2}};

int plan_bands(const FastJob* jobs, int n, int pipelines, BandedJob* out) {
  // units: block rows of one strip of a group of fpw frames (one warp's work per block step)
  auto geometry = [](const FastJob& j, long long& per_group, long long& groups, int& fpw) {
    const ds_plan* pl = j.plan;
    const HostGeom& hg = entry_of(pl).geom;
    const long long nbx = (pl->out_w + hg.p - 1) / hg.p, nby = (pl->out_h + hg.pv - 1) / hg.pv;
    fpw = hg.fpw;
    per_group = (nbx + hg.sblk - 1) / hg.sblk * nby;
    groups = (j.n_frames + hg.fpw - 1) / hg.fpw;
  };
  long long units = 0;
  int cap = 0;
  for (int i = 0; i < n; ++i) {
    long long pg = 0, ng = 0;
    int f = 1;
    geometry(jobs[i], pg, ng, f);
    units += pg * ng;
    if (!jobs[i].plan->schedule_set) cap = std::max(cap, jobs[i].plan->row_blocks);
  }
  pipelines = std::max(1, pipelines);
  const int adaptive = (int)std::max<long long>(1, std::min<long long>(cap, (units + pipelines - 1) / pipelines));
  for (int i = 0; i < n; ++i)
    out[i] = BandedJob{jobs[i], jobs[i].plan->schedule_set ? std::max(1, jobs[i].plan->row_blocks) : adaptive};
  const int band = out[n - 1].band;
  if (band < 4) return n;
  // walk back from the last job, giving each tail level its units (whole
  // jobs, or the last groups of a job split in two)
  int count = n, i = n - 1;
  for (const TailLevel& lv : kTail) {
    const int lband = std::max(1, band / lv.div);
    const long long target = (long long)lv.tiles_per_pipeline * pipelines * lband;
    long long acc = 0;
    while (i >= 0 && acc < target) {
      long long pg = 0, ng = 0;
      int f = 1;
      geometry(out[i].job, pg, ng, f);
      const long long whole = pg * ng;
      if (acc + whole <= target || ng < 2) {
        out[i].band = std::min(out[i].band, lband);
        acc += whole;
        --i;
        continue;
      }
      if (count + 1 > kMaxJobs) return count;
      // the level takes the job's last kg whole groups (a partial last group
      // stays at the end); the head stays at index i for the next level
      const long long kg = std::min<long long>(ng - 1, (target - acc + pg - 1) / pg);
      const FastJob j = out[i].job;
      const int head_band = out[i].band;
      size_t fin = 0, fout = 0;
      ds_plan_frame_bytes(j.plan, &fin, &fout);
      const int head = (int)(ng - kg) * f;
      for (int m = count; m > i + 1; --m) out[m] = out[m - 1];
      out[i] = BandedJob{FastJob{j.plan, j.in, j.out, head}, head_band};
      out[i + 1] = BandedJob{FastJob{j.plan, static_cast<const uint8_t*>(j.in) + (size_t)head * fin,
                                     static_cast<uint8_t*>(j.out) + (size_t)head * fout, j.n_frames - head},
                             std::min(head_band, lband)};
      ++count;
      acc = target;
    }
  }
  return count;
}

std::string check_plan(const ds_plan* pl) {
  if (pl->fast_class < 0 || pl->fast_class >= kFcCount) return std::string();
  // rows that are not whole 16-byte units never reach the fast kernel (every
  // launch of the plan takes the general one)
  if (((size_t)pl->in_w * pl->channels * pl->elem_size) % 16 != 0) return std::string();
  JobDesc jd, jds[2];
  std::memset(&jd, 0, sizeof(jd));
  fill_job_geometry(jd, pl, nullptr, 1);
  if (!narrow_split(pl)) return entry_of(pl).check(&jd, 1);
  const int n = split_narrow_geometry(jd, jds);
  return entry_of(pl).check(jds, n);
}

// ---------------------------------------------------------------------------
// scheduling slots
// ---------------------------------------------------------------------------
// Slots owned by live graphs.
std::mutex g_slot_mu;
bool g_slot_used[kSchedSlots - kGraphSlot0] = {};

int take_graph_slot() {
  std::lock_guard<std::mutex> lock(g_slot_mu);
  for (int i = 0; i < kSchedSlots - kGraphSlot0; ++i)
    if (!g_slot_used[i]) {
      g_slot_used[i] = true;
      return kGraphSlot0 + i;
    }
  return -1;
}

// Slots of direct launches, per device: each slot's counters serve one launch
// at a time.  A launch takes a slot whose last launch has completed (its
// event, recorded on the launch's stream right after it, has fired) and that
// no other host thread is launching on right now; when every slot is busy
// the host waits for the oldest one.
struct DirectSlots {
  std::mutex mu;
  cudaEvent_t ev[kGraphSlot0] = {};
  bool pending[kGraphSlot0] = {};
  int next = 0;
};

DirectSlots* direct_slots() {
  static DirectSlots* per_dev[64] = {};
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!per_dev[dev]) per_dev[dev] = new (std::nothrow) DirectSlots();  // held until the process exits
  return per_dev[dev];
}

ds_status take_direct_slot(DirectSlots* ds_, int* slot) {
  for (;;) {
    cudaEvent_t wait_on = nullptr;
    {
      std::lock_guard<std::mutex> lock(ds_->mu);
      for (int k = 0; k < kGraphSlot0; ++k) {
        const int s = (ds_->next + k) % kGraphSlot0;
        if (ds_->pending[s]) continue;
        if (!ds_->ev[s]) {
          cudaError_t e = cudaEventCreateWithFlags(&ds_->ev[s], cudaEventDisableTiming);
          if (e != cudaSuccess) return cuda_fail(e, "k_rows: slot event");
        } else {
          cudaError_t q = cudaEventQuery(ds_->ev[s]);
          if (q == cudaErrorNotReady) continue;
          if (q != cudaSuccess) return cuda_fail(q, "k_rows: slot event query");
        }
        ds_->pending[s] = true;
        ds_->next = (s + 1) % kGraphSlot0;
        *slot = s;
        return DS_OK;
      }
      // every slot is busy: wait for the one that comes next in turn
      const int s = ds_->next;
      if (!ds_->pending[s]) wait_on = ds_->ev[s];
    }
    if (wait_on) {
      cudaError_t e = cudaEventSynchronize(wait_on);
      if (e != cudaSuccess) return cuda_fail(e, "k_rows: waiting for a scheduling slot");
    } else {
      std::this_thread::yield();
    }
  }
}

void give_direct_slot(DirectSlots* ds_, int slot, cudaStream_t st, bool launched) {
  std::lock_guard<std::mutex> lock(ds_->mu);
  if (launched) cudaEventRecord(ds_->ev[slot], st);
  ds_->pending[slot] = false;
}

// Fill the launch parameters and launch.
// `narrow`: jobs whose plan takes narrow tail strips get their split (the
// caller has checked that the descriptors fit).
template <int MAXJ>
ds_status launch_with(FastParams<MAXJ>& prm, const KernelInfo& ki, int cls, const ClassTaps& taps,
                      const BandedJob* banded, int nb, int occ, cudaStream_t st, bool narrow) {
  const int per_cta = ki.threads / 32;  // one tile per warp
  prm.t = taps;
  int tiles = 0, nj = 0;
  for (int i = 0; i < nb; ++i) {
    int k = 0;
    ds_status s = encode_job_split(prm.jobs + nj, MAXJ - nj, banded[i].job, banded[i].band,
                                   narrow && narrow_split(banded[i].job.plan), &k);
    if (s != DS_OK) return s;
    for (int m = nj; m < nj + k; ++m) {
      prm.jobs[m].tile_begin = tiles;
      tiles += prm.jobs[m].tiles;
    }
    nj += k;
  }
  prm.n_jobs = nj;
  prm.total_tiles = tiles;
  if (tiles == 0) return DS_OK;
  prm.dev = dev_state();
  if (!prm.dev) return cuda_fail(cudaGetLastError(), "k_rows: device state address");
  DirectSlots* direct = nullptr;
  if (g_capture_slots) {
    const int slot = take_graph_slot();
    if (slot < 0) {
      set_error("more than %d fused launches held by live CUDA graphs", kSchedSlots - kGraphSlot0);
      return DS_ERR_UNSUPPORTED;
    }
    g_capture_slots->push_back(slot);
    prm.sched_slot = slot;
  } else {
    direct = direct_slots();
    if (!direct) {
      set_error("k_rows: no scheduling slots for this device");
      return DS_ERR_UNSUPPORTED;
    }
    ds_status s = take_direct_slot(direct, &prm.sched_slot);
    if (s != DS_OK) return s;
  }
  const int grid = std::min((tiles + per_cta - 1) / per_cta, sm_count() * occ);
  log_msg(2, "k_rows class %d: %d jobs, %d tiles, grid %d x %d threads, %d B shared, slot %d", cls, nb, tiles, grid,
          ki.threads, ki.smem, prm.sched_slot);
  void* args[] = {&prm};
  cudaError_t e = cudaLaunchKernel(ki.fn, dim3(grid), dim3(ki.threads), args, (size_t)ki.smem, st);
  if (direct) give_direct_slot(direct, prm.sched_slot, st, e == cudaSuccess);
  if (e != cudaSuccess) return cuda_fail(e, "k_rows launch");
  count_launches(1);
  return DS_OK;
}

ds_status launch_chunk(const FastJob* jobs, int n, cudaStream_t st) {
  // launch_fast groups jobs by class, tile shape and tap table: a plan with
  // given taps launches with its own tables, every other plan with its class's
  const ds_plan* pl0 = jobs[0].plan;
  const int cls = pl0->fast_class;
  static thread_local ClassTaps given;
  if (pl0->given_taps) plan_taps(pl0, given);
  const ClassTaps& taps = pl0->given_taps ? given : class_taps(cls);
  int want_ctas = pl0->ctas_per_sm;
  for (int i = 0; i < n; ++i) want_ctas = std::max(want_ctas, jobs[i].plan->ctas_per_sm);
  // the jobs of a launch share the boundary: the kernel is compiled for one
  const RowsEntry& re = entry_of(pl0);
  const bool wrap = pl0->boundary == DS_WRAP;
  if (wrap && !re.has_wrap) {
    set_error("fused kernel class %d shape %d is not compiled for modular tilers", cls, pl0->shape);
    return DS_ERR_UNSUPPORTED;
  }
  const KernelInfo& kfew = wrap ? re.few_wrap : re.few;
  const KernelInfo& kmany = wrap ? re.many_wrap : re.many;
  // both instantiations of a class and shape have the same footprint and occupancy
  int occ = ctas_per_sm(kmany);
  if (occ <= 0) {
    set_error("fused kernel does not fit on this device (%d bytes of shared memory)", kmany.smem);
    return DS_ERR_UNSUPPORTED;
  }
  if (want_ctas > 0) occ = std::min(occ, want_ctas);
  BandedJob banded[kMaxJobs];
  const int nb = plan_bands(jobs, n, sm_count() * occ * (kmany.threads / 32), banded);
  // descriptors with the narrow tail-strip jobs; without them if they would
  // not fit one launch
  int nd = nb;
  for (int i = 0; i < nb; ++i) {
    const ds_plan* pl = banded[i].job.plan;
    const int npk = (pl->out_w + re.geom.p - 1) / re.geom.p;
    if (narrow_split(pl) && npk > re.geom.sblk) ++nd;  // a second descriptor when the frame has other strips
  }
  const bool narrow = nd <= kMaxJobs;
  if (!narrow) nd = nb;
  if (nd <= kFewJobs) {
    static thread_local FastParams<kFewJobs> few;
    if (ctas_per_sm(kfew) <= 0) return cuda_fail(cudaGetLastError(), "k_rows attributes");
    return launch_with(few, kfew, cls, taps, banded, nb, occ, st, narrow);
  }
  static thread_local FastParams<kMaxJobs> many;  // ~17 KB: not on the caller's stack
  return launch_with(many, kmany, cls, taps, banded, nb, occ, st, narrow);
}

}  // namespace
}  // namespace rows

using namespace rows;

int fast_max_jobs_per_launch() { return kMaxJobs; }

int fast_tile_shapes(int cls) {
  if (cls < 0 || cls >= kFcCount) return 0;
  int n = 0;
  for (int s = 0; s < kShapes; ++s)
    if (table()[cls][s].present) n = s + 1;
  return n;
}

bool fast_shape_info(int cls, int shape, FastShapeInfo* out) {
  if (cls < 0 || cls >= kFcCount || shape < 0 || shape >= fast_tile_shapes(cls)) return false;
  const RowsEntry& e = table()[cls][shape];
  out->packets_per_lane = e.nb;
  out->stage_rows = e.sr;
  out->stages = e.nst;
  out->warps_per_cta = e.wpc;
  out->ctas_per_sm_budget = e.minb;
  out->strip_pixels = e.geom.spx;
  out->frames_per_warp = e.geom.fpw;
  out->smem_per_cta = e.many.smem;
  return true;
}

bool fast_wrap_fits(int cls, int in_w) {
  if (cls < 0 || cls >= kFcCount) return false;
  const RowsEntry& e = table()[cls][0];  // modular tilers: tile shape 0
  if (!e.present || !e.has_wrap) return false;
  // the row copies of a strip's window reach at most one period past either
  // end of the row: the row is at least a strip and its halo
  const long long row = (long long)in_w * e.geom.c * e.geom.sz;
  return row >= (long long)e.geom.spx * e.geom.c * e.geom.sz + e.geom.rhb && row >= e.geom.hlb;
}

int fast_ctas_per_sm(const ds_plan* pl) {
  if (pl->fast_class < 0) return 0;
  return ctas_per_sm(entry_of(pl).many);
}

thread_local std::vector<int>* g_capture_slots = nullptr;

void release_graph_slots(const std::vector<int>& slots) {
  std::lock_guard<std::mutex> lock(g_slot_mu);
  for (int s : slots)
    if (s >= kGraphSlot0 && s < kSchedSlots) g_slot_used[s - kGraphSlot0] = false;
}

// One launch per class and tile shape present (each kernel is specialised
// for its class), at most kMaxJobs descriptors per launch, one after the
// other on the caller's stream.  (Running them concurrently on side streams
// made the serving mix about 5 % slower: the serving loop already overlaps
// batches on several streams.)
ds_status launch_fast(const FastJob* jobs, int n, cudaStream_t st) {
  if (!g_capture_slots) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
      set_error("fused launch inside a stream capture the library did not start: capture with ds_graph_create, "
                "which gives each captured launch a scheduling slot of its own");
      return DS_ERR_UNSUPPORTED;
    }
  }
  if (n == 1) return launch_chunk(jobs, 1, st);  // the common single-job case
  // the groups: one per (class, shape, boundary) for the plans with the
  // library's taps, one per plan with given taps (its own tap tables), at
  // most kMaxJobs jobs each
  std::vector<FastJob> order;
  std::vector<int> bounds{0};
  order.reserve(n);
  auto close_group = [&]() {
    if ((int)order.size() > bounds.back()) bounds.push_back((int)order.size());
  };
  auto add = [&](const FastJob& j) {
    order.push_back(j);
    if ((int)order.size() - bounds.back() == kMaxJobs) close_group();
  };
  for (int cls = 0; cls < kFcCount; ++cls)
    for (int shape = 0; shape < kShapes; ++shape)
      for (int bnd : {DS_CLAMP, DS_WRAP}) {
        for (int i = 0; i < n; ++i) {
          const ds_plan* pl = jobs[i].plan;
          if (pl->fast_class == cls && pl->shape == shape && pl->boundary == bnd && !pl->given_taps) add(jobs[i]);
        }
        close_group();
      }
  for (int i = 0; i < n; ++i) {
    const ds_plan* pl = jobs[i].plan;
    if (!pl->given_taps) continue;
    bool seen = false;
    for (int k = 0; k < i && !seen; ++k) seen = jobs[k].plan == pl;
    if (seen) continue;
    for (int k = i; k < n; ++k)
      if (jobs[k].plan == pl) add(jobs[k]);
    close_group();
  }
  ds_status s = DS_OK;
  for (size_t g = 0; g + 1 < bounds.size() && s == DS_OK; ++g)
    s = launch_chunk(order.data() + bounds[g], bounds[g + 1] - bounds[g], st);
  return s;
}

ds_status launch_timeout_probe(long long limit_cycles, cudaStream_t st) {
  k_timeout_probe<<<1, 32, 0, st>>>(limit_cycles);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "timeout probe launch");
  count_launches(1);
  return DS_OK;
}

bool bounds_checked() { return kCheckBounds; }

ds_status launch_bounds_probe(cudaStream_t st) {
  k_bounds_probe<<<1, 32, 0, st>>>();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "bounds probe launch");
  count_launches(1);
  return DS_OK;
}

ds_status debug_check_plan(const ds_plan* pl, std::string& msg) {
  msg = check_plan(pl);
  return msg.empty() ? DS_OK : DS_ERR_ARG;
}

// The status word and, after a failed bounds check, its record; the word is
// cleared by the read.  The scheduling counters need no reset here: every
// warp of a launch, one that gave up a wait included, reaches the end of the
// kernel, where the last one out resets its slot.
ds_status read_device_status(int* status, long long* info) {
  DevState* dev = dev_state();
  if (!dev) return cuda_fail(cudaGetLastError(), "device state address");
  int v = 0, zero = 0;
  cudaError_t e = cudaMemcpy(&v, &dev->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "reading the device status word");
  info[0] = info[1] = 0;
  if (v == kStatusBounds) {
    e = cudaMemcpy(info, dev->bounds_info, 2 * sizeof(long long), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading the bounds-check record");
  }
  if (v != 0) {
    e = cudaMemcpy(&dev->status, &zero, sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the device status word");
  }
  *status = v;
  return DS_OK;
}

}  // namespace ds

// plan.cpp -- host plan layer of libds: argument checks, phase windows, tap
// tables (FP64 -> FP32 / Q14), kernel choice.  No device work happens here.
//
// The filter (paper Sec. 3): each axis maps packets of q input pixels to p
// outputs; output o = r*p + j reads K pixels starting at r*q + b_j.  The tap
// weights are not given by the paper; this library uses a Lanczos-3 window
// stretched over the K taps (see ds.h for the full list of readings).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <new>

#include "internal.h"

namespace ds {

namespace {
thread_local std::string g_last_error;
thread_local long long g_launches = 0;

int gcd(int a, int b) {
  while (b != 0) {
    const int t = a % b;
    a = b;
    b = t;
  }
  return a;
}

// floor(a / b) for b > 0.
long long floor_div(long long a, long long b) {
  long long d = a / b;
  if (a % b != 0 && a < 0) --d;
  return d;
}

// Lanczos window of order 3 written as 3 sin(pi x) sin(pi x / 3) / (pi x)^2,
// equal to sinc(x) sinc(x/3) on |x| < 3 and 0 outside.
double lanczos_a3(double x) {
  if (x == 0.0) return 1.0;
  if (std::fabs(x) >= 3.0) return 0.0;
  const double px = M_PI * x;
  return 3.0 * std::sin(px) * std::sin(px / 3.0) / (px * px);
}

// Phase windows and taps of one axis: p/q with K taps.  `given`: NULL for
// the Lanczos-3 taps, else the caller's FP64 table [p][K].  The Q14 table
// rounds half up and puts the residual floor(16384 * row sum + 1/2) - sum(q)
// on the row's largest tap (16384 - sum(q) for rows summing to 1).
// Returns false, with the reason in `why`, if a given tap is not finite or
// (for uint8, `u8`) the Q14 table cannot be used exactly.
bool build_axis(int p, int q, int K, const double* given, bool u8, int* b, double* w64, float* w32, short* q14,
                char* why, size_t why_len) {
  const double stretch = 6.0 / K;  // Lanczos-3 support spread over K taps
  for (int j = 0; j < p; ++j) {
    // centre of phase j relative to the block start, as num / den
    const long long num = (long long)(2 * j + 1) * q - p;
    const long long den = 2LL * p;
    const double centre = (double)num / (double)den;
    b[j] = (int)(floor_div(num, den) - K / 2 + 1);
    double* row = w64 + j * K;
    if (given) {
      for (int t = 0; t < K; ++t) {
        row[t] = given[j * K + t];
        if (!std::isfinite(row[t])) {
          std::snprintf(why, why_len, "tap [%d][%d] is not finite", j, t);
          return false;
        }
      }
    } else {
      double total = 0.0;
      for (int t = 0; t < K; ++t) {
        row[t] = lanczos_a3(stretch * ((double)(b[j] + t) - centre));
        total += row[t];
      }
      for (int t = 0; t < K; ++t) row[t] /= total;
    }
    int largest = 0;
    long long qsum = 0;
    double wsum = 0.0;
    long long qv[kMaxK];
    for (int t = 0; t < K; ++t) {
      w32[j * K + t] = (float)row[t];
      qv[t] = (long long)std::floor(row[t] * 16384.0 + 0.5);
      qsum += qv[t];
      wsum += row[t];
      if (row[t] > row[largest]) largest = t;
    }
    // the rounding residual goes to the largest tap (so rows summing to 1
    // give Q14 rows summing to 2^14 exactly)
    qv[largest] += (long long)std::floor(wsum * 16384.0 + 0.5) - qsum;
    long long mag = 0;
    for (int t = 0; t < K; ++t) {
      if (u8 && (qv[t] < -32768 || qv[t] > 32767)) {
        std::snprintf(why, why_len, "Q14 tap [%d][%d] = %lld outside int16", j, t, qv[t]);
        return false;
      }
      mag += qv[t] < 0 ? -qv[t] : qv[t];
      q14[j * K + t] = (short)(qv[t] < -32768 ? -32768 : (qv[t] > 32767 ? 32767 : qv[t]));
    }
    if (u8 && mag > 65535) {
      std::snprintf(why, why_len, "Q14 row %d magnitudes sum to %lld > 65535", j, mag);
      return false;
    }
  }
  return true;
}

bool axis_ok(const char* who, const char* axis, int p, int q, int K) {
  if (p < 1 || q <= p || gcd(p, q) != 1 || p > kMaxP || q > kMaxQ) {
    set_error("%s: %sratio %d/%d must be in lowest terms, 0 < p < q, p <= %d, q <= %d", who, axis, p, q, kMaxP,
              kMaxQ);
    return false;
  }
  if (K < 2 || K > kMaxK || (K % 2) != 0) {
    set_error("%s: %staps %d must be even and in [2,%d]", who, axis, K, kMaxK);
    return false;
  }
  return true;
}

// Default band of output row blocks per tile (measured on a B300 over the
// 1080p / 4K workloads; the autotuner refines it per plan).
int default_row_blocks(int fast_class) {
  switch (fast_class) {
    case kFcF32_38: return 12;
    case kFcF16_38: return 16;
    case kFcU8C3_38: return 16;
    case kFcF32_12: case kFcF16_12: return 24;
    case kFcU8C3_12: return 40;
    case kFcF32_23: case kFcF16_23: case kFcU8C3_23: return 20;
    case kFcU8C3_CIF: case kFcU8C1_CIF: return 16;
    case kFcU8C1_38: return 16;
    case kFcU8C1_12: return 24;
    case kFcU8C1_23: return 20;
    default: return 0;
  }
}

int default_band(int fast_class) {
  const int b = default_row_blocks(fast_class);
  return b > 0 ? b : 8;
}
}  // namespace

int log_level() {
  static const int level = [] {
    const char* s = std::getenv("DS_LOG");
    return s ? std::atoi(s) : 0;
  }();
  return level;
}

void log_msg(int level, const char* fmt, ...) {
  if (log_level() < level) return;
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  std::fprintf(stderr, "[ds] %s\n", buf);
}

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  log_msg(1, "error: %s", buf);
}

void clear_error() { g_last_error.clear(); }

ds_status cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return DS_ERR_CUDA;
}

void count_launches(long long n) { g_launches += n; }

int fast_class_of(int p, int q, int K, int pv, int qv, int Kv, ds_dtype dtype) {
  if (p == 3 && q == 8 && K == 8 && pv == 4 && qv == 9 && Kv == 8) {
    if (dtype == DS_U8_RGB) return kFcU8C3_CIF;
    if (dtype == DS_U8) return kFcU8C1_CIF;
    return kFcNone;
  }
  if (p != pv || q != qv || K != Kv) return kFcNone;
  int r = -1;
  if (p == 3 && q == 8 && K == 8) r = 0;
  if (p == 1 && q == 2 && K == 6) r = 1;
  if (p == 2 && q == 3 && K == 6) r = 2;
  if (r < 0) return kFcNone;
  switch (dtype) {
    case DS_F32: return kFcF32_38 + r;
    case DS_F16: return kFcF16_38 + r;
    case DS_U8_RGB: return kFcU8C3_38 + r;
    case DS_U8: return kFcU8C1_38 + r;
    default: return kFcNone;
  }
}

// TMA tensor maps need a 16-byte aligned base and 16-byte multiple strides.
bool frame_tma_ok(const ds_plan* pl, const void* in, size_t frame_stride_bytes) {
  const size_t row_bytes = (size_t)pl->in_w * pl->channels * pl->elem_size;
  if (((uintptr_t)in & 15u) != 0) return false;
  if (row_bytes % 16 != 0) return false;
  if (frame_stride_bytes % 16 != 0) return false;
  if ((size_t)pl->in_w * pl->channels >= (1ull << 32)) return false;
  return true;
}

}  // namespace ds

using namespace ds;

extern "C" {

const char* ds_last_error(void) { return g_last_error.c_str(); }

const char* ds_version(void) { return "libds 0.1 (sm_103a)"; }

long long ds_launch_count(void) {
  const long long n = g_launches;
  g_launches = 0;
  return n;
}

namespace {

ds_plan* create_plan(const ds_plan_desc& d, const char* who) {
  if (d.in_h < 1 || d.in_w < 1) {
    set_error("%s: frame %dx%d must be at least 1x1", who, d.in_h, d.in_w);
    return nullptr;
  }
  const bool same = d.ratio_h.p == d.ratio_v.p && d.ratio_h.q == d.ratio_v.q && d.taps_h == d.taps_v;
  if (!axis_ok(who, same ? "" : "horizontal ", d.ratio_h.p, d.ratio_h.q, d.taps_h)) return nullptr;
  if (!axis_ok(who, same ? "" : "vertical ", d.ratio_v.p, d.ratio_v.q, d.taps_v)) return nullptr;
  int channels = 1, elem = 4;
  switch (d.dtype) {
    case DS_F32: channels = 1; elem = 4; break;
    case DS_F16: channels = 1; elem = 2; break;
    case DS_U8: channels = 1; elem = 1; break;
    case DS_U8_RGB: channels = 3; elem = 1; break;
    default:
      set_error("%s: unknown dtype %d", who, (int)d.dtype);
      return nullptr;
  }
  if (d.boundary != DS_CLAMP && d.boundary != DS_WRAP) {
    set_error("%s: unknown boundary %d", who, (int)d.boundary);
    return nullptr;
  }
  const long long oh = (long long)d.in_h * d.ratio_v.p / d.ratio_v.q;
  const long long ow = (long long)d.in_w * d.ratio_h.p / d.ratio_h.q;
  if (oh < 1 || ow < 1) {
    set_error("%s: %dx%d at %d/%d x %d/%d gives an empty output", who, d.in_h, d.in_w, d.ratio_v.p, d.ratio_v.q,
              d.ratio_h.p, d.ratio_h.q);
    return nullptr;
  }
  if ((long long)d.in_h * d.in_w * channels >= (1LL << 40)) {
    set_error("%s: frame too large", who);
    return nullptr;
  }
  ds_plan* pl = new (std::nothrow) ds_plan();
  if (!pl) {
    set_error("%s: out of host memory", who);
    return nullptr;
  }
  pl->in_h = d.in_h;
  pl->in_w = d.in_w;
  pl->channels = channels;
  pl->elem_size = elem;
  pl->p = d.ratio_h.p;
  pl->q = d.ratio_h.q;
  pl->K = d.taps_h;
  pl->pv = d.ratio_v.p;
  pl->qv = d.ratio_v.q;
  pl->Kv = d.taps_v;
  pl->dtype = d.dtype;
  pl->boundary = d.boundary;
  pl->given_taps = d.weights_h || d.weights_v;
  pl->out_h = (int)oh;
  pl->out_w = (int)ow;
  const bool u8 = d.dtype == DS_U8 || d.dtype == DS_U8_RGB;
  char why[160];
  if (!build_axis(pl->p, pl->q, pl->K, d.weights_h, u8, pl->b, pl->w64, pl->w32, pl->q14, why, sizeof(why)) ||
      !build_axis(pl->pv, pl->qv, pl->Kv, d.weights_v, u8, pl->bv, pl->w64v, pl->w32v, pl->q14v, why,
                  sizeof(why))) {
    set_error("%s: %s", who, why);
    delete pl;
    return nullptr;
  }
  // the fast kernels take clamp-to-edge, and modular tilers on frames at
  // least a strip and its halo wide (a plan's given taps travel with its
  // launch)
  pl->fast_class = fast_class_of(pl->p, pl->q, pl->K, pl->pv, pl->qv, pl->Kv, d.dtype);
  if (d.boundary == DS_WRAP && !fast_wrap_fits(pl->fast_class, pl->in_w)) pl->fast_class = kFcNone;
  pl->row_blocks = default_band(pl->fast_class);
  if (pl->fast_class >= 0) {
    pl->tmaps.reset(new (std::nothrow) TmapCache());  // without it every launch encodes its maps
  }
  const char* no_tma = std::getenv("DS_NO_TMA");
  pl->force_general = (no_tma && no_tma[0] && no_tma[0] != '0');
  log_msg(1, "plan %dx%dx%d dtype %d: h %d/%d K%d, v %d/%d K%d, %s%s -> %s (class %d, band %d)", pl->in_h,
          pl->in_w, pl->channels, (int)pl->dtype, pl->p, pl->q, pl->K, pl->pv, pl->qv, pl->Kv,
          pl->boundary == DS_WRAP ? "wrap" : "clamp", pl->given_taps ? ", given taps" : "",
          pl->fast_class >= 0 && !pl->force_general ? "fused_tma" : "fused_general", pl->fast_class, pl->row_blocks);
  return pl;
}

}  // namespace

ds_plan* ds_plan_create(int in_h, int in_w, ds_ratio ratio, int taps, ds_dtype dtype) {
  clear_error();
  ds_plan_desc d{};
  d.in_h = in_h;
  d.in_w = in_w;
  d.ratio_h = d.ratio_v = ratio;
  d.taps_h = d.taps_v = taps;
  d.dtype = dtype;
  d.boundary = DS_CLAMP;
  return create_plan(d, "ds_plan_create");
}

ds_plan* ds_plan_create_ex(const ds_plan_desc* desc) {
  clear_error();
  if (!desc) {
    set_error("ds_plan_create_ex: NULL descriptor");
    return nullptr;
  }
  return create_plan(*desc, "ds_plan_create_ex");
}

void ds_destroy(ds_plan* plan) { delete plan; }

ds_status ds_plan_get_params(const ds_plan* pl, int* in_h, int* in_w, int* p, int* q, int* taps, int* dtype) {
  if (!pl) {
    set_error("ds_plan_get_params: NULL plan");
    return DS_ERR_ARG;
  }
  if (in_h) *in_h = pl->in_h;
  if (in_w) *in_w = pl->in_w;
  if (p) *p = pl->p;
  if (q) *q = pl->q;
  if (taps) *taps = pl->K;
  if (dtype) *dtype = (int)pl->dtype;
  return DS_OK;
}

ds_status ds_plan_out_shape(const ds_plan* pl, int* out_h, int* out_w, int* channels) {
  if (!pl) {
    set_error("ds_plan_out_shape: NULL plan");
    return DS_ERR_ARG;
  }
  if (out_h) *out_h = pl->out_h;
  if (out_w) *out_w = pl->out_w;
  if (channels) *channels = pl->channels;
  return DS_OK;
}

ds_status ds_plan_frame_bytes(const ds_plan* pl, size_t* in_bytes, size_t* out_bytes) {
  if (!pl) {
    set_error("ds_plan_frame_bytes: NULL plan");
    return DS_ERR_ARG;
  }
  if (in_bytes) *in_bytes = pl->in_frame_elems() * pl->elem_size;
  if (out_bytes) *out_bytes = pl->out_frame_elems() * pl->elem_size;
  return DS_OK;
}

ds_status ds_plan_get_taps(const ds_plan* pl, double* fp64, float* fp32, short* q14,
                           int* window_start) {
  return ds_plan_get_axis_taps(pl, 0, fp64, fp32, q14, window_start);
}

ds_status ds_plan_get_axis_taps(const ds_plan* pl, int axis, double* fp64, float* fp32, short* q14,
                                int* window_start) {
  if (!pl || (axis != 0 && axis != 1)) {
    set_error("ds_plan_get_axis_taps: NULL plan or axis not 0 / 1");
    return DS_ERR_ARG;
  }
  const bool v = axis == 1;
  const int p = v ? pl->pv : pl->p, n = p * (v ? pl->Kv : pl->K);
  if (fp64) std::memcpy(fp64, v ? pl->w64v : pl->w64, sizeof(double) * n);
  if (fp32) std::memcpy(fp32, v ? pl->w32v : pl->w32, sizeof(float) * n);
  if (q14) std::memcpy(q14, v ? pl->q14v : pl->q14, sizeof(short) * n);
  if (window_start) std::memcpy(window_start, v ? pl->bv : pl->b, sizeof(int) * p);
  return DS_OK;
}

ds_status ds_plan_get_axes(const ds_plan* pl, int* p_h, int* q_h, int* taps_h, int* p_v, int* q_v, int* taps_v,
                           int* boundary) {
  if (!pl) {
    set_error("ds_plan_get_axes: NULL plan");
    return DS_ERR_ARG;
  }
  if (p_h) *p_h = pl->p;
  if (q_h) *q_h = pl->q;
  if (taps_h) *taps_h = pl->K;
  if (p_v) *p_v = pl->pv;
  if (q_v) *q_v = pl->qv;
  if (taps_v) *taps_v = pl->Kv;
  if (boundary) *boundary = (int)pl->boundary;
  return DS_OK;
}

ds_status ds_plan_set_schedule(ds_plan* pl, int row_blocks, int ctas_per_sm) {
  if (!pl || row_blocks < 1 || ctas_per_sm < 0) {
    set_error("ds_plan_set_schedule: bad arguments");
    return DS_ERR_ARG;
  }
  pl->row_blocks = row_blocks;
  pl->ctas_per_sm = ctas_per_sm;
  pl->schedule_set = true;
  return DS_OK;
}

ds_status ds_plan_get_schedule(const ds_plan* pl, int* row_blocks, int* ctas_per_sm) {
  if (!pl) {
    set_error("ds_plan_get_schedule: NULL plan");
    return DS_ERR_ARG;
  }
  if (row_blocks) *row_blocks = pl->row_blocks;
  if (ctas_per_sm) *ctas_per_sm = pl->ctas_per_sm;
  return DS_OK;
}

int ds_plan_tile_shapes(const ds_plan* pl) {
  if (!pl || pl->fast_class < 0) return 0;
  if (pl->boundary == DS_WRAP) return 1;  // modular tilers: tile shape 0 only
  return fast_tile_shapes(pl->fast_class);
}

ds_status ds_plan_set_schedule_ex(ds_plan* pl, const ds_schedule* sc) {
  if (!pl || !sc || sc->row_blocks < 0 || sc->ctas_per_sm < 0 || sc->shape < 0 ||
      sc->shape >= std::max(1, ds_plan_tile_shapes(pl))) {
    set_error("ds_plan_set_schedule_ex: bad arguments (shape must be below ds_plan_tile_shapes)");
    return DS_ERR_ARG;
  }
  pl->schedule_set = sc->row_blocks > 0;
  pl->row_blocks = sc->row_blocks > 0 ? sc->row_blocks : default_band(pl->fast_class);
  pl->ctas_per_sm = sc->ctas_per_sm;
  pl->shape = sc->shape;
  return DS_OK;
}

ds_status ds_plan_get_schedule_ex(const ds_plan* pl, ds_schedule* sc) {
  if (!pl || !sc) {
    set_error("ds_plan_get_schedule_ex: NULL argument");
    return DS_ERR_ARG;
  }
  sc->row_blocks = pl->schedule_set ? pl->row_blocks : 0;
  sc->ctas_per_sm = pl->ctas_per_sm;
  sc->shape = pl->shape;
  return DS_OK;
}

ds_status ds_plan_describe(const ds_plan* pl, char* buf, size_t len) {
  if (!pl || !buf || len == 0) {
    set_error("ds_plan_describe: bad arguments");
    return DS_ERR_ARG;
  }
  static const char* names[] = {"f32_3_8_k8", "f32_1_2_k6", "f32_2_3_k6", "f16_3_8_k8", "f16_1_2_k6",
                                "f16_2_3_k6", "u8rgb_3_8_k8", "u8rgb_1_2_k6", "u8rgb_2_3_k6",
                                "u8rgb_h3_8_v4_9_k8", "u8_h3_8_v4_9_k8", "u8_3_8_k8", "u8_1_2_k6", "u8_2_3_k6"};
  static_assert(sizeof(names) / sizeof(names[0]) == kFcCount, "a name per fast class");
  const bool fast = pl->fast_class >= 0 && !pl->force_general;
  FastShapeInfo si{};
  char shape[256] = "null";
  if (pl->fast_class >= 0 && fast_shape_info(pl->fast_class, pl->shape, &si))
    std::snprintf(shape, sizeof(shape),
                  "{\"index\": %d, \"of\": %d, \"packets_per_lane\": %d, \"strip_pixels\": %d, "
                  "\"frames_per_warp\": %d, \"stage_rows\": %d, \"stages\": %d, \"warps_per_cta\": %d, "
                  "\"ctas_per_sm_budget\": %d, \"smem_per_cta\": %d}",
                  pl->shape, ds_plan_tile_shapes(pl), si.packets_per_lane, si.strip_pixels,
                  si.frames_per_warp, si.stage_rows, si.stages, si.warps_per_cta, si.ctas_per_sm_budget,
                  si.smem_per_cta);
  std::snprintf(buf, len,
                "{\"kernel\": \"%s\", \"class\": \"%s\", \"in\": [%d, %d, %d], \"out\": [%d, %d, %d], "
                "\"ratio\": [%d, %d], \"taps\": %d, \"ratio_v\": [%d, %d], \"taps_v\": %d, "
                "\"boundary\": \"%s\", \"given_taps\": %s, \"row_blocks\": %d, \"band\": \"%s\", "
                "\"ctas_per_sm\": %d, \"tile_shape\": %s}",
                fast ? "fused_tma" : "fused_general", pl->fast_class >= 0 ? names[pl->fast_class] : "general",
                pl->in_h, pl->in_w, pl->channels, pl->out_h, pl->out_w, pl->channels, pl->p, pl->q, pl->K, pl->pv,
                pl->qv, pl->Kv, pl->boundary == DS_WRAP ? "wrap" : "clamp", pl->given_taps ? "true" : "false",
                pl->row_blocks, pl->schedule_set ? "fixed" : "adaptive", pl->ctas_per_sm, shape);
  return DS_OK;
}

}  // extern "C"

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

// Phase windows and taps of a p/q, K-tap plan.
void build_taps(ds_plan* pl) {
  const int p = pl->p, q = pl->q, K = pl->K;
  const double stretch = 6.0 / K;  // Lanczos-3 support spread over K taps
  for (int j = 0; j < p; ++j) {
    // centre of phase j relative to the block start, as num / den
    const long long num = (long long)(2 * j + 1) * q - p;
    const long long den = 2LL * p;
    const double centre = (double)num / (double)den;
    pl->b[j] = (int)(floor_div(num, den) - K / 2 + 1);
    double* row = pl->w64 + j * K;
    double total = 0.0;
    for (int t = 0; t < K; ++t) {
      row[t] = lanczos_a3(stretch * ((double)(pl->b[j] + t) - centre));
      total += row[t];
    }
    int largest = 0;
    long long qsum = 0;
    for (int t = 0; t < K; ++t) {
      row[t] /= total;
      pl->w32[j * K + t] = (float)row[t];
      const long long qv = (long long)std::floor(row[t] * 16384.0 + 0.5);
      pl->q14[j * K + t] = (short)qv;
      qsum += qv;
      if (row[t] > row[largest]) largest = t;
    }
    // the rounding residual goes to the largest tap so each row sums to 2^14
    pl->q14[j * K + largest] = (short)(pl->q14[j * K + largest] + (16384 - qsum));
  }
}

// Default band of output row blocks per tile (measured on a B300 over the
// 1080p / 4K workloads; the autotuner refines it per plan).
int default_row_blocks(int fast_class) {
  switch (fast_class) {
    case kFcF32_38: return 8;
    case kFcF16_38: return 10;
    case kFcU8C3_38: return 16;
    case kFcF32_12: case kFcF16_12: case kFcU8C3_12: return 24;
    case kFcF32_23: case kFcF16_23: case kFcU8C3_23: return 20;
    default: return 0;
  }
}
}  // namespace

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

void clear_error() { g_last_error.clear(); }

ds_status cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return DS_ERR_CUDA;
}

void count_launches(long long n) { g_launches += n; }

int fast_class_of(int p, int q, int K, ds_dtype dtype) {
  int r = -1;
  if (p == 3 && q == 8 && K == 8) r = 0;
  if (p == 1 && q == 2 && K == 6) r = 1;
  if (p == 2 && q == 3 && K == 6) r = 2;
  if (r < 0) return kFcNone;
  switch (dtype) {
    case DS_F32: return kFcF32_38 + r;
    case DS_F16: return kFcF16_38 + r;
    case DS_U8_RGB: return kFcU8C3_38 + r;
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

ds_plan* ds_plan_create(int in_h, int in_w, ds_ratio ratio, int taps, ds_dtype dtype) {
  clear_error();
  if (in_h < 1 || in_w < 1) {
    set_error("ds_plan_create: frame %dx%d must be at least 1x1", in_h, in_w);
    return nullptr;
  }
  const int p = ratio.p, q = ratio.q;
  if (p < 1 || q <= p || gcd(p, q) != 1 || p > kMaxP || q > kMaxQ) {
    set_error("ds_plan_create: ratio %d/%d must be in lowest terms, 0 < p < q, p <= %d, q <= %d",
              p, q, kMaxP, kMaxQ);
    return nullptr;
  }
  if (taps < 2 || taps > kMaxK || (taps % 2) != 0) {
    set_error("ds_plan_create: taps %d must be even and in [2,%d]", taps, kMaxK);
    return nullptr;
  }
  int channels = 1, elem = 4;
  switch (dtype) {
    case DS_F32: channels = 1; elem = 4; break;
    case DS_F16: channels = 1; elem = 2; break;
    case DS_U8: channels = 1; elem = 1; break;
    case DS_U8_RGB: channels = 3; elem = 1; break;
    default:
      set_error("ds_plan_create: unknown dtype %d", (int)dtype);
      return nullptr;
  }
  const long long oh = (long long)in_h * p / q, ow = (long long)in_w * p / q;
  if (oh < 1 || ow < 1) {
    set_error("ds_plan_create: %dx%d at %d/%d gives an empty output", in_h, in_w, p, q);
    return nullptr;
  }
  if ((long long)in_h * in_w * channels >= (1LL << 40)) {
    set_error("ds_plan_create: frame too large");
    return nullptr;
  }
  ds_plan* pl = new (std::nothrow) ds_plan();
  if (!pl) {
    set_error("ds_plan_create: out of host memory");
    return nullptr;
  }
  pl->in_h = in_h;
  pl->in_w = in_w;
  pl->channels = channels;
  pl->elem_size = elem;
  pl->p = p;
  pl->q = q;
  pl->K = taps;
  pl->dtype = dtype;
  pl->out_h = (int)oh;
  pl->out_w = (int)ow;
  build_taps(pl);
  pl->fast_class = fast_class_of(p, q, taps, dtype);
  pl->row_blocks = default_row_blocks(pl->fast_class);
  if (pl->row_blocks == 0) pl->row_blocks = 8;
  const char* no_tma = std::getenv("DS_NO_TMA");
  pl->force_general = (no_tma && no_tma[0] && no_tma[0] != '0');
  return pl;
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
  if (!pl) {
    set_error("ds_plan_get_taps: NULL plan");
    return DS_ERR_ARG;
  }
  const int n = pl->p * pl->K;
  if (fp64) std::memcpy(fp64, pl->w64, sizeof(double) * n);
  if (fp32) std::memcpy(fp32, pl->w32, sizeof(float) * n);
  if (q14) std::memcpy(q14, pl->q14, sizeof(short) * n);
  if (window_start) std::memcpy(window_start, pl->b, sizeof(int) * pl->p);
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

ds_status ds_plan_describe(const ds_plan* pl, char* buf, size_t len) {
  if (!pl || !buf || len == 0) {
    set_error("ds_plan_describe: bad arguments");
    return DS_ERR_ARG;
  }
  static const char* names[] = {"f32_3_8_k8", "f32_1_2_k6", "f32_2_3_k6", "f16_3_8_k8", "f16_1_2_k6",
                                "f16_2_3_k6", "u8rgb_3_8_k8", "u8rgb_1_2_k6", "u8rgb_2_3_k6"};
  const bool fast = pl->fast_class >= 0 && !pl->force_general;
  std::snprintf(buf, len,
                "{\"kernel\": \"%s\", \"class\": \"%s\", \"in\": [%d, %d, %d], \"out\": [%d, %d, %d], "
                "\"ratio\": [%d, %d], \"taps\": %d, \"row_blocks\": %d, \"ctas_per_sm\": %d}",
                fast ? "fused_tma" : "fused_general", pl->fast_class >= 0 ? names[pl->fast_class] : "general",
                pl->in_h, pl->in_w, pl->channels, pl->out_h, pl->out_w, pl->channels, pl->p, pl->q, pl->K,
                pl->row_blocks, pl->ctas_per_sm);
  return DS_OK;
}

}  // extern "C"

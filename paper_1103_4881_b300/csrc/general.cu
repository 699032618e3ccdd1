// general.cu -- general kernels of libds: any ratio p/q (p <= 16, q <= 64),
// any even K <= 16, any dtype, any alignment.
//
//  * k_fused_general: one CTA per output tile; the horizontal pass of the
//    tile's input rows (plus the vertical halo) goes to shared memory, the
//    vertical pass reads it there (paper Sec. 3: horizontal filter, then
//    vertical filter; Sec. 3.B.3: no round trip for the intermediate).
//  * k_hpass / k_vpass: the unfused two-kernel form with the intermediate in
//    device memory (FP32 for float dtypes, uint8 for uint8).
//
// Every output accumulates its K products in tap order t = 0..K-1 with
// fmaf from 0, the same sequence as the fast fused kernel, so all kernels of
// the library agree bit for bit.
#include <algorithm>

#include "internal.h"
#include "pixel.cuh"

namespace ds {

namespace {

// One axis of the filter: phase windows and taps (FP32, or Q14 as floats
// for uint8).
struct GenAxis {
  float w[kMaxP * kMaxK];
  int b[kMaxP];   // window start of each phase
  int p, q, K;
  int bmin, L;    // first window offset and pattern length
};

struct GenParams {
  GenAxis h, v;   // horizontal (along a row) and vertical (along a column)
  int C;
  int H, W, OH, OW;
  int wrap;       // 0: clamp-to-edge, 1: modular indexing
  int nby;        // output row blocks: ceil(OH / v.p)
  int tob, tox;   // fused tile: row blocks x output pixels
};

GenAxis make_axis(int p, int q, int K, const int* b, const float* w32, const short* q14, bool u8) {
  GenAxis a{};
  for (int i = 0; i < p * K; ++i) a.w[i] = u8 ? (float)q14[i] : w32[i];
  for (int j = 0; j < p; ++j) a.b[j] = b[j];
  a.p = p;
  a.q = q;
  a.K = K;
  a.bmin = b[0];
  a.L = b[p - 1] + K - b[0];
  return a;
}

GenParams make_params(const ds_plan* pl) {
  GenParams g{};
  const bool u8 = pl->dtype == DS_U8 || pl->dtype == DS_U8_RGB;
  g.h = make_axis(pl->p, pl->q, pl->K, pl->b, pl->w32, pl->q14, u8);
  g.v = make_axis(pl->pv, pl->qv, pl->Kv, pl->bv, pl->w32v, pl->q14v, u8);
  g.C = pl->channels;
  g.H = pl->in_h;
  g.W = pl->in_w;
  g.OH = pl->out_h;
  g.OW = pl->out_w;
  g.wrap = pl->boundary == DS_WRAP ? 1 : 0;
  g.nby = (pl->out_h + pl->pv - 1) / pl->pv;
  g.tob = std::max(1, 64 / pl->qv);  // about 64 input rows of progress per tile
  g.tox = 32;
  return g;
}

// Index i of an axis of n elements under the plan's boundary: modulo n
// (WRAP), else clamped to the edge.  A window reaches at most one period past
// the frame but for the tiniest frames, so the modulo takes a division only
// then.
template <bool WRAP>
__device__ __forceinline__ int fix_index(int i, int n) {
  if constexpr (WRAP) {
    if (i < 0) i += n;
    else if (i >= n) i -= n;
    if ((unsigned)i < (unsigned)n) return i;
    const int m = i % n;
    return m < 0 ? m + n : m;
  } else {
    return clampi(i, 0, n - 1);
  }
}

// Horizontal dot product of output pixel o (channel c) on input row `row`.
template <typename T, bool WRAP>
__device__ __forceinline__ float hdot(const GenParams& g, const T* __restrict__ row, int o, int c) {
  const int j = o % g.h.p;
  const int s = (o / g.h.p) * g.h.q + g.h.b[j];
  const float* w = g.h.w + j * g.h.K;
  float acc = 0.0f;
  for (int t = 0; t < g.h.K; ++t) {
    const int x = fix_index<WRAP>(s + t, g.W);
    acc = fmaf(w[t], px_to_f(row[(size_t)x * g.C + c]), acc);
  }
  return pass_round<T>(acc);
}

template <typename T, bool WRAP>
__global__ void __launch_bounds__(256) k_fused_general(const T* __restrict__ in, T* __restrict__ out,
                                                        const __grid_constant__ GenParams g, int frame0) {
  extern __shared__ float sh[];
  const int f = frame0 + blockIdx.z;
  const int rb0 = blockIdx.y * g.tob;
  const int nb = min(g.tob, g.nby - rb0);
  const int ox0 = blockIdx.x * g.tox;
  const int npx = min(g.tox, g.OW - ox0);
  const int ne = npx * g.C;         // elements per tile row
  const int te = g.tox * g.C;       // shared row stride
  const int ys = rb0 * g.v.q + g.v.bmin;
  const int nr = (nb - 1) * g.v.q + g.v.L;
  const T* src = in + (size_t)f * g.H * g.W * g.C;
  T* dst = out + (size_t)f * g.OH * g.OW * g.C;

  // horizontal pass: shared row i holds the filtered input row ys + i
  // (clamped or wrapped)
  for (int idx = threadIdx.x; idx < nr * ne; idx += blockDim.x) {
    const int i = idx / ne, e = idx - i * ne;
    const int y = fix_index<WRAP>(ys + i, g.H);
    const int o = ox0 + e / g.C, c = e % g.C;
    sh[i * te + e] = hdot<T, WRAP>(g, src + (size_t)y * g.W * g.C, o, c);
  }
  __syncthreads();
  // vertical pass over the shared rows
  for (int idx = threadIdx.x; idx < nb * g.v.p * ne; idx += blockDim.x) {
    const int orow = idx / ne, e = idx - orow * ne;
    const int r = rb0 + orow / g.v.p, j = orow % g.v.p;
    const int oy = r * g.v.p + j;
    if (oy >= g.OH) continue;
    const int base = r * g.v.q + g.v.b[j] - ys;
    const float* w = g.v.w + j * g.v.K;
    float acc = 0.0f;
    for (int t = 0; t < g.v.K; ++t) acc = fmaf(w[t], sh[(base + t) * te + e], acc);
    dst[(size_t)oy * g.OW * g.C + (size_t)ox0 * g.C + e] = f_to_px<T>(pass_round<T>(acc));
  }
}

// Unfused horizontal pass: inter[f][y][e] for e < OW*C.  I is the
// intermediate type (float for float dtypes, uint8 for uint8).
template <typename T, typename I, bool WRAP>
__global__ void __launch_bounds__(256) k_hpass(const T* __restrict__ in, I* __restrict__ inter,
                                                const __grid_constant__ GenParams g, int frame0) {
  const int f = frame0 + blockIdx.z;
  const int y = blockIdx.y;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int ne = g.OW * g.C;
  if (e >= ne) return;
  const T* row = in + ((size_t)f * g.H + y) * g.W * g.C;
  const float v = hdot<T, WRAP>(g, row, e / g.C, e % g.C);
  inter[((size_t)f * g.H + y) * ne + e] = (I)v;
}

// Unfused vertical pass over the intermediate.
template <typename T, typename I, bool WRAP>
__global__ void __launch_bounds__(256) k_vpass(const I* __restrict__ inter, T* __restrict__ out,
                                                const __grid_constant__ GenParams g, int frame0) {
  const int f = frame0 + blockIdx.z;
  const int oy = blockIdx.y;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int ne = g.OW * g.C;
  if (e >= ne) return;
  const int j = oy % g.v.p;
  const int s = (oy / g.v.p) * g.v.q + g.v.b[j];
  const float* w = g.v.w + j * g.v.K;
  const I* col = inter + (size_t)f * g.H * ne + e;
  float acc = 0.0f;
  for (int t = 0; t < g.v.K; ++t) {
    const int y = fix_index<WRAP>(s + t, g.H);
    acc = fmaf(w[t], (float)col[(size_t)y * ne], acc);
  }
  out[((size_t)f * g.OH + oy) * ne + e] = f_to_px<T>(pass_round<T>(acc));
}

constexpr int kMaxGridZ = 65535;

template <typename T, bool WRAP>
ds_status fused_general_t(const GenParams& g, const void* in, void* out, int n_frames, cudaStream_t st) {
  const int nr_max = (g.tob - 1) * g.v.q + g.v.L;
  const size_t smem = (size_t)nr_max * g.tox * g.C * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_fused_general<T, WRAP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "k_fused_general smem attribute");
  }
  for (int f0 = 0; f0 < n_frames; f0 += kMaxGridZ) {
    const int nf = std::min(kMaxGridZ, n_frames - f0);
    dim3 grid((g.OW + g.tox - 1) / g.tox, (g.nby + g.tob - 1) / g.tob, nf);
    log_msg(2, "k_fused_general: %d frames, grid %d x %d x %d, %zu B shared", nf, grid.x, grid.y, grid.z, smem);
    k_fused_general<T, WRAP><<<grid, 256, smem, st>>>((const T*)in, (T*)out, g, f0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_fused_general launch");
    count_launches(1);
  }
  return DS_OK;
}

template <typename T, typename I, bool WRAP>
ds_status unfused_t(const GenParams& g, const void* in, void* out, int n_frames, void* ws, cudaStream_t st) {
  const int ne = g.OW * g.C;
  if (g.H > 65535) {
    set_error("ds_run_unfused: frames taller than 65535 rows are not supported");
    return DS_ERR_UNSUPPORTED;
  }
  for (int f0 = 0; f0 < n_frames; f0 += kMaxGridZ) {
    const int nf = std::min(kMaxGridZ, n_frames - f0);
    dim3 gh((ne + 255) / 256, g.H, nf);
    log_msg(2, "k_hpass + k_vpass: %d frames", nf);
    k_hpass<T, I, WRAP><<<gh, 256, 0, st>>>((const T*)in, (I*)ws, g, f0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_hpass launch");
    dim3 gv((ne + 255) / 256, g.OH, nf);
    k_vpass<T, I, WRAP><<<gv, 256, 0, st>>>((const I*)ws, (T*)out, g, f0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_vpass launch");
    count_launches(2);
  }
  return DS_OK;
}

template <typename T>
ds_status fused_general_any(const ds_plan* pl, const void* in, void* out, int n_frames, cudaStream_t st) {
  const GenParams g = make_params(pl);
  return g.wrap ? fused_general_t<T, true>(g, in, out, n_frames, st) : fused_general_t<T, false>(g, in, out, n_frames, st);
}

template <typename T, typename I>
ds_status unfused_any(const ds_plan* pl, const void* in, void* out, int n_frames, void* ws, cudaStream_t st) {
  const GenParams g = make_params(pl);
  return g.wrap ? unfused_t<T, I, true>(g, in, out, n_frames, ws, st) : unfused_t<T, I, false>(g, in, out, n_frames, ws, st);
}

}  // namespace

ds_status launch_general_fused(const ds_plan* pl, const void* in, void* out, int n_frames, cudaStream_t st) {
  switch (pl->dtype) {
    case DS_F32: return fused_general_any<float>(pl, in, out, n_frames, st);
    case DS_F16: return fused_general_any<__half>(pl, in, out, n_frames, st);
    case DS_U8:
    case DS_U8_RGB: return fused_general_any<uint8_t>(pl, in, out, n_frames, st);
  }
  set_error("launch_general_fused: unknown dtype");
  return DS_ERR_ARG;
}

ds_status launch_unfused(const ds_plan* pl, const void* in, void* out, int n_frames, void* ws, cudaStream_t st) {
  switch (pl->dtype) {
    case DS_F32: return unfused_any<float, float>(pl, in, out, n_frames, ws, st);
    case DS_F16: return unfused_any<__half, float>(pl, in, out, n_frames, ws, st);
    case DS_U8:
    case DS_U8_RGB: return unfused_any<uint8_t, uint8_t>(pl, in, out, n_frames, ws, st);
  }
  set_error("launch_unfused: unknown dtype");
  return DS_ERR_ARG;
}

}  // namespace ds

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

struct GenParams {
  float w[kMaxP * kMaxK];  // FP32 taps, or Q14 taps as floats for uint8
  int b[kMaxP];            // window start of each phase
  int p, q, K, C;
  int H, W, OH, OW;
  int bmin, L;             // first window offset and pattern length
  int nby;                 // output row blocks: ceil(OH / p)
  int tob, tox;            // fused tile: row blocks x output pixels
};

GenParams make_params(const ds_plan* pl) {
  GenParams g{};
  const int n = pl->p * pl->K;
  const bool u8 = pl->dtype == DS_U8 || pl->dtype == DS_U8_RGB;
  for (int i = 0; i < n; ++i) g.w[i] = u8 ? (float)pl->q14[i] : pl->w32[i];
  for (int j = 0; j < pl->p; ++j) g.b[j] = pl->b[j];
  g.p = pl->p;
  g.q = pl->q;
  g.K = pl->K;
  g.C = pl->channels;
  g.H = pl->in_h;
  g.W = pl->in_w;
  g.OH = pl->out_h;
  g.OW = pl->out_w;
  g.bmin = pl->b[0];
  g.L = pl->b[pl->p - 1] + pl->K - pl->b[0];
  g.nby = (pl->out_h + pl->p - 1) / pl->p;
  g.tob = std::max(1, 32 / pl->q);
  g.tox = 32;
  return g;
}

// Horizontal dot product of output pixel o (channel c) on input row `row`.
template <typename T>
__device__ __forceinline__ float hdot(const GenParams& g, const T* __restrict__ row, int o, int c) {
  const int j = o % g.p;
  const int s = (o / g.p) * g.q + g.b[j];
  const float* w = g.w + j * g.K;
  float acc = 0.0f;
  for (int t = 0; t < g.K; ++t) {
    const int x = clampi(s + t, 0, g.W - 1);
    acc = fmaf(w[t], px_to_f(row[(size_t)x * g.C + c]), acc);
  }
  return pass_round<T>(acc);
}

template <typename T>
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
  const int ys = rb0 * g.q + g.bmin;
  const int nr = (nb - 1) * g.q + g.L;
  const T* src = in + (size_t)f * g.H * g.W * g.C;
  T* dst = out + (size_t)f * g.OH * g.OW * g.C;

  // horizontal pass: shared row i holds the filtered input row clamp(ys + i)
  for (int idx = threadIdx.x; idx < nr * ne; idx += blockDim.x) {
    const int i = idx / ne, e = idx - i * ne;
    const int y = clampi(ys + i, 0, g.H - 1);
    const int o = ox0 + e / g.C, c = e % g.C;
    sh[i * te + e] = hdot<T>(g, src + (size_t)y * g.W * g.C, o, c);
  }
  __syncthreads();
  // vertical pass over the shared rows
  for (int idx = threadIdx.x; idx < nb * g.p * ne; idx += blockDim.x) {
    const int orow = idx / ne, e = idx - orow * ne;
    const int r = rb0 + orow / g.p, j = orow % g.p;
    const int oy = r * g.p + j;
    if (oy >= g.OH) continue;
    const int base = r * g.q + g.b[j] - ys;
    const float* w = g.w + j * g.K;
    float acc = 0.0f;
    for (int t = 0; t < g.K; ++t) acc = fmaf(w[t], sh[(base + t) * te + e], acc);
    dst[(size_t)oy * g.OW * g.C + (size_t)ox0 * g.C + e] = f_to_px<T>(pass_round<T>(acc));
  }
}

// Unfused horizontal pass: inter[f][y][e] for e < OW*C.  I is the
// intermediate type (float for float dtypes, uint8 for uint8).
template <typename T, typename I>
__global__ void __launch_bounds__(256) k_hpass(const T* __restrict__ in, I* __restrict__ inter,
                                                const __grid_constant__ GenParams g, int frame0) {
  const int f = frame0 + blockIdx.z;
  const int y = blockIdx.y;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int ne = g.OW * g.C;
  if (e >= ne) return;
  const T* row = in + ((size_t)f * g.H + y) * g.W * g.C;
  const float v = hdot<T>(g, row, e / g.C, e % g.C);
  inter[((size_t)f * g.H + y) * ne + e] = (I)v;
}

// Unfused vertical pass over the intermediate.
template <typename T, typename I>
__global__ void __launch_bounds__(256) k_vpass(const I* __restrict__ inter, T* __restrict__ out,
                                                const __grid_constant__ GenParams g, int frame0) {
  const int f = frame0 + blockIdx.z;
  const int oy = blockIdx.y;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int ne = g.OW * g.C;
  if (e >= ne) return;
  const int j = oy % g.p;
  const int s = (oy / g.p) * g.q + g.b[j];
  const float* w = g.w + j * g.K;
  const I* col = inter + (size_t)f * g.H * ne + e;
  float acc = 0.0f;
  for (int t = 0; t < g.K; ++t) {
    const int y = clampi(s + t, 0, g.H - 1);
    acc = fmaf(w[t], (float)col[(size_t)y * ne], acc);
  }
  out[((size_t)f * g.OH + oy) * ne + e] = f_to_px<T>(pass_round<T>(acc));
}

constexpr int kMaxGridZ = 65535;

template <typename T>
ds_status fused_general_t(const ds_plan* pl, const void* in, void* out, int n_frames, cudaStream_t st) {
  const GenParams g = make_params(pl);
  const int nr_max = (g.tob - 1) * g.q + g.L;
  const size_t smem = (size_t)nr_max * g.tox * g.C * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_fused_general<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "k_fused_general smem attribute");
  }
  for (int f0 = 0; f0 < n_frames; f0 += kMaxGridZ) {
    const int nf = std::min(kMaxGridZ, n_frames - f0);
    dim3 grid((g.OW + g.tox - 1) / g.tox, (g.nby + g.tob - 1) / g.tob, nf);
    k_fused_general<T><<<grid, 256, smem, st>>>((const T*)in, (T*)out, g, f0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_fused_general launch");
    count_launches(1);
  }
  return DS_OK;
}

template <typename T, typename I>
ds_status unfused_t(const ds_plan* pl, const void* in, void* out, int n_frames, void* ws, cudaStream_t st) {
  const GenParams g = make_params(pl);
  const int ne = g.OW * g.C;
  if (g.H > 65535) {
    set_error("ds_run_unfused: frames taller than 65535 rows are not supported");
    return DS_ERR_UNSUPPORTED;
  }
  for (int f0 = 0; f0 < n_frames; f0 += kMaxGridZ) {
    const int nf = std::min(kMaxGridZ, n_frames - f0);
    dim3 gh((ne + 255) / 256, g.H, nf);
    k_hpass<T, I><<<gh, 256, 0, st>>>((const T*)in, (I*)ws, g, f0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_hpass launch");
    dim3 gv((ne + 255) / 256, g.OH, nf);
    k_vpass<T, I><<<gv, 256, 0, st>>>((const I*)ws, (T*)out, g, f0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_vpass launch");
    count_launches(2);
  }
  return DS_OK;
}

}  // namespace

ds_status launch_general_fused(const ds_plan* pl, const void* in, void* out, int n_frames, cudaStream_t st) {
  switch (pl->dtype) {
    case DS_F32: return fused_general_t<float>(pl, in, out, n_frames, st);
    case DS_F16: return fused_general_t<__half>(pl, in, out, n_frames, st);
    case DS_U8:
    case DS_U8_RGB: return fused_general_t<uint8_t>(pl, in, out, n_frames, st);
  }
  set_error("launch_general_fused: unknown dtype");
  return DS_ERR_ARG;
}

ds_status launch_unfused(const ds_plan* pl, const void* in, void* out, int n_frames, void* ws, cudaStream_t st) {
  switch (pl->dtype) {
    case DS_F32: return unfused_t<float, float>(pl, in, out, n_frames, ws, st);
    case DS_F16: return unfused_t<__half, float>(pl, in, out, n_frames, ws, st);
    case DS_U8:
    case DS_U8_RGB: return unfused_t<uint8_t, uint8_t>(pl, in, out, n_frames, ws, st);
  }
  set_error("launch_unfused: unknown dtype");
  return DS_ERR_ARG;
}

}  // namespace ds

// fused_fast.cu -- the fused horizontal + vertical decimating FIR for B300.
//
// One persistent kernel runs the whole filter stage of the paper's
// downscaler (Sec. 3: horizontal filter, then vertical filter, packets of q
// pixels -> p outputs).  Work is cut into tiles: a strip of output columns
// x a band of output row blocks of one frame.  Per CTA:
//
//   producer warp (one elected lane): TMA tensor loads
//     (cp.async.bulk.tensor.3d) of SR input rows of the strip plus its left
//     and right halo into an NSTAGE-deep shared-memory ring, completion
//     tracked by mbarrier transaction counts;
//   4 consumer warps:
//     H pass -- every thread loads one contiguous chunk of a row (NB packets
//       of q pixels) with conflict-free vector ld.shared, takes the halo
//       pixels from its neighbour lanes with warp shuffles, and computes
//       NB*p outputs per channel with the phase taps (kernel parameters, so
//       FFMA operands come from the constant bank);
//     the horizontal results go to an on-chip ring of intermediate rows
//       (the intermediate never reaches HBM -- the paper's Sec. 3.B.4 removes
//       host round trips between the two filters; this removes the device
//       memory round trip as well);
//     V pass -- as soon as the rows of an output block are in the ring,
//       threads read them column-wise and write the p output rows.
//
// The H and V dot products accumulate in tap order t = 0..K-1 with fmaf from
// 0, the same sequence as the general kernels, so results are identical bit
// for bit whatever kernel, tile or batch computes them.
//
// Every wait on an mbarrier is bounded (2e9 SM clock cycles, about 1 s).  On expiry the
// kernel records DS_ERR_TIMEOUT in a device status word, the consumers agree
// on leaving through a barrier with OR-reduction, and the producer waits
// (bounded) for the copies it issued before it returns.
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "pixel.cuh"

namespace ds {

__device__ int g_fast_status = 0;  // 0 = fine; 1 = wait timed out; 2 = bad class

// Dynamic tile scheduling of the row-streaming kernel: launch slot s hands out
// tiles from g_tile_next[s]; the last warp to finish puts both counters of
// its slot back to zero.  Launches take slots in turn, so launches that can
// overlap (different streams) use different counters.
constexpr int kSchedSlots = 1024;
__device__ unsigned int g_tile_next[kSchedSlots];
__device__ unsigned int g_warps_done[kSchedSlots];

namespace {

constexpr int kNH = 8;                        // horizontal-pass warps
constexpr int kNV = 4;                        // vertical-pass warps
constexpr int kNWC = kNH + kNV;               // consumer warps
constexpr int kThreads = (kNWC + 1) * 32;     // + one producer warp
constexpr int kNRS = 4;                       // intermediate ring capacity, in stages
constexpr int kMaxJobs = 64;                  // job descriptors per launch
constexpr int kMaxTaps = 24;                  // p*K of the fast classes
constexpr long long kWaitLimitCycles = 2000000000ll;  // ~1 s at the B300's 2.03 GHz
constexpr uint32_t kSuspendHintNs = 20000;             // a waiting thread sleeps up to 20 us per poll
constexpr int kStatusTimeout = 1;
constexpr int kStatusBadClass = 2;

// ---------------------------------------------------------------------------
// compile-time geometry
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int cfloordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
__host__ __device__ constexpr int cdiv(int a, int b) { return (a + b - 1) / b; }
__host__ __device__ constexpr int rup(int a, int m) { return cdiv(a, m) * m; }
// window start of phase j: floor(((2j+1) q - p) / (2p)) - K/2 + 1
__host__ __device__ constexpr int phase_b(int P, int Q, int K, int j) {
  return cfloordiv((2 * j + 1) * Q - P, 2 * P) - K / 2 + 1;
}
__host__ __device__ constexpr int pow2_at_least(int a) { return a <= 1 ? 1 : 2 * pow2_at_least((a + 1) / 2); }
constexpr int cmax(int a) { return a; }
template <typename... R>
constexpr int cmax(int a, int b, R... r) { return cmax(a > b ? a : b, r...); }

template <typename T>
struct TmaType;
template <>
struct TmaType<float> { static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; };
template <>
struct TmaType<__half> { static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_FLOAT16; };
template <>
struct TmaType<uint8_t> { static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_UINT8; };

// Intermediate type in the on-chip ring: FP32 for float data; FP16 for uint8
// data, whose intermediate values are integers 0..255 (exact in FP16).
template <typename T>
struct RingOf { using type = float; };
template <>
struct RingOf<uint8_t> { using type = __half; };

// A fast-path class: data type, channels, ratio P/Q, taps K, and the tile
// shape -- NB packets per thread and row, WX warps across a strip, SR input
// rows per pipeline stage, VE columns per thread in the V pass.
template <int ID, typename T_, int C_, int P_, int Q_, int K_, int NB_, int WX_, int SR_, int VE_>
struct Cls {
  using T = T_;
  using R = typename RingOf<T_>::type;
  static constexpr int id = ID, C = C_, P = P_, Q = Q_, K = K_, NB = NB_, WX = WX_, SR = SR_, VE = VE_;
  static constexpr int WY = kNH / WX;
  static constexpr int SZ = (int)sizeof(T);
  static constexpr int BMIN = phase_b(P, Q, K, 0);
  static constexpr int BMAX = phase_b(P, Q, K, P - 1);
  static constexpr int L = BMAX - BMIN + K;   // pattern length (rows or pixels per block window)
  static constexpr int LH = -BMIN;            // halo pixels left of a block
  static constexpr int RH = BMAX + K - Q;     // halo pixels right of a block
  static constexpr int E = NB * Q * C;        // elements per thread and row
  static constexpr int EB = E * SZ;
  static constexpr int EW = EB / 4;
  static constexpr int HLB = rup(LH * C * SZ, 16);  // left halo bytes in the window (TMA x alignment)
  static constexpr int RHB = rup(RH * C * SZ, 16);
  static constexpr int SBLK = 32 * NB * WX;         // packets (blocks) per strip
  static constexpr int SPX = SBLK * Q;              // input pixels per strip
  static constexpr int WINB = HLB + SPX * C * SZ + RHB;
  static constexpr int NBOX = cdiv(WINB / SZ, 256);
  static constexpr int BOXB = rup(cdiv(WINB, NBOX), 16);
  static constexpr int BOXE = BOXB / SZ;
  static constexpr int BOXSTR = rup(SR * BOXB, 128);  // each box lands 128-B aligned
  static constexpr int STAGE_BYTES = NBOX * BOXSTR;
  static constexpr int TX_BYTES = NBOX * SR * BOXB;
  static constexpr int SOE = SBLK * P * C;            // intermediate elements per ring row
  static constexpr int RING = kNRS * SR;              // ring rows: kNRS stages of SR rows
  static constexpr int RING_MASK = RING - 1;
  static constexpr int D = cdiv(L - 1, SR);           // V of stage k reads rows of stages k-D..k
  static constexpr int RING_BYTES = rup(RING * SOE * (int)sizeof(R), 16);
  static constexpr int NX = (LH + NB * Q + RH) * C;   // elements one thread reads per row
  static constexpr int VB = (EB % 16 == 0) ? 16 : ((EB % 8 == 0) ? 8 : 4);
  static constexpr int NV = EB / VB;
  static constexpr int HB = cdiv(LH * C * SZ, VB);   // halo vectors a thread loads before its chunk
  static constexpr int HA = cdiv(RH * C * SZ, VB);   // ... and after it
  static constexpr int NVT = HB + NV + HA;           // vectors per thread and row
  static constexpr int NWT = NVT * VB / 4;           // words per thread and row
  // With 16-byte vectors and a 32-byte lane stride, the lanes of one
  // 8-lane shared-memory phase cover only half the 16-byte bank groups for a
  // fixed vector index (2-way conflicts).  Lanes 4-7 of each phase then load
  // their 4 vectors in the order 1,2,3,0, which makes every phase hit 8
  // distinct bank groups; the vectors are put back in order with selects.
  static constexpr bool ROT = (VB == 16 && EB == 32 && NVT == 4);
  static constexpr int NOUT = NB * P * C;             // H outputs per thread and row
  __host__ __device__ static constexpr int b(int j) { return phase_b(P, Q, K, j); }
  static_assert(EB % 4 == 0, "a thread's chunk must be whole words");
  static_assert(HB * VB <= HLB && HA * VB <= RHB, "halo vectors must lie in the loaded window");
  static_assert(BOXE <= 256 && BOXB % 16 == 0, "TMA box limits");
  static_assert(NBOX * BOXB >= WINB, "boxes must cover the window");
  static_assert(SR % WY == 0 && kNH % WX == 0, "stage rows must split over warp rows");
  static_assert((SR & (SR - 1)) == 0 && kNRS >= D + 1, "ring of kNRS power-of-two stages");
  static_assert(SOE % 4 == 0 && VE == 4, "V pass works on groups of 4 columns");
  static_assert((RING & RING_MASK) == 0, "ring size");
  static_assert(P * K <= kMaxTaps, "tap table size");
  static_assert(BOXB % VB == 0 && HLB % VB == 0, "vector loads must not straddle boxes");
};

//                 id        T     C  P  Q  K  NB WX  SR VE
using CF32_38 = Cls<kFcF32_38, float, 1, 3, 8, 8, 1, 1, 16, 4>;
using CF32_12 = Cls<kFcF32_12, float, 1, 1, 2, 6, 4, 1, 16, 4>;
using CF32_23 = Cls<kFcF32_23, float, 1, 2, 3, 6, 2, 1, 16, 4>;
using CF16_38 = Cls<kFcF16_38, __half, 1, 3, 8, 8, 1, 1, 16, 4>;
using CF16_12 = Cls<kFcF16_12, __half, 1, 1, 2, 6, 4, 1, 16, 4>;
using CF16_23 = Cls<kFcF16_23, __half, 1, 2, 3, 6, 2, 1, 16, 4>;
using CU8_38 = Cls<kFcU8C3_38, uint8_t, 3, 3, 8, 8, 1, 1, 8, 4>;
using CU8_12 = Cls<kFcU8C3_12, uint8_t, 3, 1, 2, 6, 2, 2, 8, 4>;
using CU8_23 = Cls<kFcU8C3_23, uint8_t, 3, 2, 3, 6, 4, 1, 8, 4>;

// ---------------------------------------------------------------------------
// launch parameters
// ---------------------------------------------------------------------------
struct JobDesc {
  CUtensorMap tmap;        // 3-D map: (W*C elements, H rows, n_frames)
  void* out;
  long long out_frame;     // elements per output frame
  int H, W, OH, OW;
  int nframes, cls, strips, chunks;
  int rbc, tile_begin, tiles, out_vec;
};
static_assert(sizeof(JobDesc) == 256 && alignof(JobDesc) == 128, "job descriptor layout");

// Q14 taps of the uint8 classes as pairs of int16 for dp2a, [class - first
// uint8 class][window-start parity][phase][pair]: for parity a, pair i holds
// taps 2i - a (low half) and 2i + 1 - a (high half), zero outside 0..K-1, so
// a window that starts on an odd slot is read from the even slot before it.
constexpr int kU8Classes = 3;
constexpr int kMaxPairs = 5;  // (K + 1) / 2 + 1 for K <= 8

struct FastParams {
  JobDesc jobs[kMaxJobs];
  float taps[kFcCount][kMaxTaps];  // FP32 taps, or Q14 taps as floats for uint8
  uint32_t tap2[kU8Classes][2][3][kMaxPairs];
  int n_jobs;
  int total_tiles;
  int sched_slot;                  // row kernel: dynamic scheduling slot
};

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t saddr32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(saddr32(bar)), "r"(parity), "r"(kSuspendHintNs)
      : "memory");
  return ok != 0;
}
// Wait for the phase of `parity` to complete; false after about a second
// (kWaitLimitCycles SM clock cycles, counted from the 4th failed poll), or at
// once when *abort_flag becomes non-zero (if given).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, const volatile int* abort_flag) {
#pragma unroll 1
  for (int it = 0; it < 4; ++it)
    if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 3u) == 0) {
      if (abort_flag && *abort_flag) return false;
      if (clock64() - t0 > kWaitLimitCycles) return false;
    }
  }
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(saddr32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(saddr32(bar))
      : "memory");
}
// ---------------------------------------------------------------------------
// tiles
// ---------------------------------------------------------------------------
struct Tile {
  int job, frame, strip, chunk;
};

__host__ __device__ __forceinline__ Tile decode_tile(const FastParams& prm, int t) {
  int lo = 0, hi = prm.n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prm.jobs[mid].tile_begin <= t) lo = mid;
    else hi = mid - 1;
  }
  const JobDesc& jd = prm.jobs[lo];
  const int tl = t - jd.tile_begin;
  const int per_frame = jd.strips * jd.chunks;
  Tile r;
  r.job = lo;
  r.frame = tl / per_frame;
  const int rem = tl - r.frame * per_frame;
  r.chunk = rem / jd.strips;  // strips vary fastest: neighbouring CTAs share halos in L2
  r.strip = rem - r.chunk * jd.strips;
  return r;
}

struct Geo {
  int rb0;   // first output row block of the tile
  int nblk;  // row blocks in the tile
  int ys;    // first input row of the tile's pattern (may be < 0)
  int rows;  // input rows the tile needs
  int nst;   // pipeline stages of the tile
  int xw;    // first element (x coordinate) of the loaded window
  int ox0;   // first output pixel of the strip
};

template <class Cl>
__host__ __device__ __forceinline__ Geo tile_geo(const JobDesc& jd, const Tile& tl) {
  Geo g;
  g.rb0 = tl.chunk * jd.rbc;
  const int nby = (jd.OH + Cl::P - 1) / Cl::P;
  g.nblk = jd.rbc < nby - g.rb0 ? jd.rbc : nby - g.rb0;
  g.ys = g.rb0 * Cl::Q + Cl::BMIN;
  g.rows = (g.nblk - 1) * Cl::Q + Cl::L;
  g.nst = (g.rows + Cl::SR - 1) / Cl::SR;
  g.xw = tl.strip * Cl::SPX * Cl::C - Cl::HLB / Cl::SZ;
  g.ox0 = tl.strip * Cl::SBLK * Cl::P;
  return g;
}

// Offset of byte `byte` of window row 0 inside a stage: boxes are stored one
// after the other, each as SR rows of BOXB bytes (BOXSTR bytes apart), so row
// r of the window starts r * BOXB bytes further in every box.
template <class Cl>
__host__ __device__ __forceinline__ int win_off(int byte) {
  const int box = byte / Cl::BOXB;
  return byte + box * (Cl::BOXSTR - Cl::BOXB);
}

// ---------------------------------------------------------------------------
// producer
// ---------------------------------------------------------------------------
template <class Cl, int NSTAGE, int STAGE_MAX>
__device__ bool produce_tile(const JobDesc& jd, const Tile& tl, uint8_t* stages, uint64_t* full, uint64_t* empty,
                             uint32_t& g, const volatile int* abort_flag) {
  const Geo G = tile_geo<Cl>(jd, tl);
  for (int k = 0; k < G.nst; ++k, ++g) {
    const uint32_t slot = g % NSTAGE, round = g / NSTAGE;
    if (round > 0 && !mbar_wait(&empty[slot], (round - 1) & 1u, abort_flag)) return false;
    uint8_t* dst = stages + slot * STAGE_MAX;
    mbar_expect_tx(&full[slot], Cl::TX_BYTES);
#pragma unroll
    for (int bx = 0; bx < Cl::NBOX; ++bx)
      tma_load_3d(dst + bx * Cl::BOXSTR, &jd.tmap, &full[slot], G.xw + bx * Cl::BOXE, G.ys + k * Cl::SR, tl.frame);
  }
  return true;
}

// ---------------------------------------------------------------------------
// consumer: horizontal pass of one row
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ float word_elem(const uint32_t* w, int byte);
template <>
__device__ __forceinline__ float word_elem<float>(const uint32_t* w, int byte) { return __uint_as_float(w[byte >> 2]); }
template <>
__device__ __forceinline__ float word_elem<__half>(const uint32_t* w, int byte) {
  const uint32_t v = w[byte >> 2];
  const unsigned short h = (byte & 2) ? (unsigned short)(v >> 16) : (unsigned short)(v & 0xffffu);
  return __half2float(__ushort_as_half(h));
}
template <>
__device__ __forceinline__ float word_elem<uint8_t>(const uint32_t* w, int byte) {
  // byte -> float through the bit pattern of 2^23 + byte
  return __uint_as_float(__byte_perm(w[byte >> 2], 0x4B000000u, 0x7540u | (unsigned)(byte & 3))) - 8388608.0f;
}

template <typename T>
__device__ __forceinline__ float smem_elem(const uint8_t* p) { return px_to_f(*reinterpret_cast<const T*>(p)); }

// Per-thread shared-memory offsets (row 0 of a stage) of the vectors the H
// pass loads: HB halo vectors, the thread's own NV vectors, HA halo vectors,
// consecutive in the window, in the (possibly rotated) order they are loaded.
// They depend only on the lane: computed once.
template <class Cl>
struct Offs {
  int v[Cl::NVT];
  bool rot;
};

template <class Cl>
__device__ __forceinline__ Offs<Cl> thread_offs(int lg) {
  Offs<Cl> o;
  const int first = Cl::HLB + lg * Cl::EB - Cl::HB * Cl::VB;
  o.rot = Cl::ROT && ((lg >> 2) & 1);
#pragma unroll
  for (int v = 0; v < Cl::NVT; ++v) {
    const int pv = o.rot ? (v + 1) % Cl::NVT : v;
    o.v[v] = win_off<Cl>(first + pv * Cl::VB);
  }
  return o;
}

// Load the thread's vectors of one window row into words w[0..NWT).
template <class Cl>
__device__ __forceinline__ void load_row(const uint8_t* rowbase, const Offs<Cl>& o, uint32_t* w) {
  constexpr int WPV = Cl::VB / 4;
  if constexpr (Cl::ROT) {
    uint4 r[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) r[v] = *reinterpret_cast<const uint4*>(rowbase + o.v[v]);
    // r[v] holds vector (v + rot) mod 4
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const uint4 x = o.rot ? r[(v + 3) & 3] : r[v];
      w[v * 4] = x.x; w[v * 4 + 1] = x.y; w[v * 4 + 2] = x.z; w[v * 4 + 3] = x.w;
    }
  } else {
#pragma unroll
    for (int v = 0; v < Cl::NVT; ++v) {
      const uint8_t* p = rowbase + o.v[v];
      if constexpr (Cl::VB == 16) {
        const uint4 x = *reinterpret_cast<const uint4*>(p);
        w[v * WPV] = x.x; w[v * WPV + 1] = x.y; w[v * WPV + 2] = x.z; w[v * WPV + 3] = x.w;
      } else if constexpr (Cl::VB == 8) {
        const uint2 x = *reinterpret_cast<const uint2*>(p);
        w[v * WPV] = x.x; w[v * WPV + 1] = x.y;
      } else {
        w[v] = *reinterpret_cast<const uint32_t*>(p);
      }
    }
  }
}

// Clamp-to-edge in the loaded window: the columns of a warp's read range that
// lie outside the frame (TMA filled them with zeros) get the value of the
// first / last column of their row.  Pixel ranges [l_lo, 0) and [r_lo, r_hi).
struct EdgeFix {
  int l_lo, nl, r_lo, nr;  // first pixel and element counts, left and right
};

template <class Cl>
__host__ __device__ __forceinline__ EdgeFix edge_fix(int strip, int wx, int W) {
  const int seg0 = strip * Cl::SPX + wx * 32 * Cl::NB * Cl::Q - Cl::LH;       // first pixel the warp reads
  const int seg1 = strip * Cl::SPX + (wx + 1) * 32 * Cl::NB * Cl::Q + Cl::RH;  // one past the last
  EdgeFix f;
  f.l_lo = seg0;
  f.nl = seg0 < 0 ? ((seg1 < 0 ? seg1 : 0) - seg0) * Cl::C : 0;
  f.r_lo = W > seg0 ? W : seg0;
  const int lim = W + Cl::NB * Cl::Q + Cl::RH;  // active lanes read no further
  const int r_hi = seg1 < lim ? seg1 : lim;
  f.nr = r_hi > f.r_lo ? (r_hi - f.r_lo) * Cl::C : 0;
  return f;
}

template <class Cl>
__device__ __forceinline__ void apply_edge_fix(uint8_t* rowbase, const EdgeFix& f, int lane, int W, int xw) {
  using T = typename Cl::T;
  for (int e = lane; e < f.nl + f.nr; e += 32) {
    const bool left = e < f.nl;
    const int k = left ? e : e - f.nl;
    const int px = (left ? f.l_lo : f.r_lo) + k / Cl::C, c = k % Cl::C;
    const int src = (left ? 0 : W - 1) * Cl::C + c - xw;
    const int dst = px * Cl::C + c - xw;
    *reinterpret_cast<T*>(rowbase + win_off<Cl>(dst * Cl::SZ)) =
        *reinterpret_cast<const T*>(rowbase + win_off<Cl>(src * Cl::SZ));
  }
  // these generic-proxy writes must land before the TMA refills the stage
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();
}

// Store a thread's NOUT horizontal results into its slice of a ring row with
// the widest aligned vector stores (the slice starts at lg * NOUT elements).
template <class Cl>
__device__ __forceinline__ void ring_store(typename Cl::R* dst, const float* o) {
  constexpr int N = Cl::NOUT;
  if constexpr (sizeof(typename Cl::R) == 4) {
    if constexpr (N % 4 == 0) {
#pragma unroll
      for (int i = 0; i < N / 4; ++i)
        reinterpret_cast<float4*>(dst)[i] = make_float4(o[4 * i], o[4 * i + 1], o[4 * i + 2], o[4 * i + 3]);
    } else if constexpr (N % 2 == 0) {
#pragma unroll
      for (int i = 0; i < N / 2; ++i) reinterpret_cast<float2*>(dst)[i] = make_float2(o[2 * i], o[2 * i + 1]);
    } else {
#pragma unroll
      for (int i = 0; i < N; ++i) dst[i] = o[i];
    }
  } else {
    if constexpr (N % 2 == 0) {
      uint32_t hw[N / 2];
#pragma unroll
      for (int i = 0; i < N / 2; ++i) {
        const __half2 h2 = __floats2half2_rn(o[2 * i], o[2 * i + 1]);
        hw[i] = *reinterpret_cast<const uint32_t*>(&h2);
      }
      if constexpr (N % 8 == 0) {
#pragma unroll
        for (int i = 0; i < N / 8; ++i)
          reinterpret_cast<uint4*>(dst)[i] = make_uint4(hw[4 * i], hw[4 * i + 1], hw[4 * i + 2], hw[4 * i + 3]);
      } else if constexpr (N % 4 == 0) {
#pragma unroll
        for (int i = 0; i < N / 4; ++i) reinterpret_cast<uint2*>(dst)[i] = make_uint2(hw[2 * i], hw[2 * i + 1]);
      } else {
#pragma unroll
        for (int i = 0; i < N / 2; ++i) reinterpret_cast<uint32_t*>(dst)[i] = hw[i];
      }
    } else {
#pragma unroll
      for (int i = 0; i < N; ++i) dst[i] = __float2half_rn(o[i]);
    }
  }
}

// Horizontal pass of one window row whose words the thread has loaded (see
// load_row): NB packets of Q pixels per thread, each giving P outputs per
// channel, pass-rounded, in o[(n*P + j)*C + c].
template <class Cl>
__device__ __forceinline__ void hcompute(const uint32_t* w, const float* __restrict__ taps, float* o) {
  using T = typename Cl::T;
  float x[Cl::NX];
  constexpr int first = Cl::HB * Cl::VB - Cl::LH * Cl::C * Cl::SZ;  // byte of the first halo element in w
#pragma unroll
  for (int e = 0; e < Cl::NX; ++e) x[e] = word_elem<T>(w, first + e * Cl::SZ);
#pragma unroll
  for (int n = 0; n < Cl::NB; ++n) {
#pragma unroll
    for (int j = 0; j < Cl::P; ++j) {
#pragma unroll
      for (int c = 0; c < Cl::C; ++c) {
        float acc = 0.0f;
#pragma unroll
        for (int t = 0; t < Cl::K; ++t)
          acc = fmaf(taps[j * Cl::K + t], x[(n * Cl::Q + Cl::b(j) - Cl::BMIN + t) * Cl::C + c], acc);
        o[(n * Cl::P + j) * Cl::C + c] = pass_round<T>(acc);
      }
    }
  }
}

// ... and stored to the thread's slice of a ring row.
template <class Cl>
__device__ __forceinline__ void hrow(const uint32_t* w, const float* __restrict__ taps,
                                     typename Cl::R* __restrict__ dst) {
  float o[Cl::NOUT];
  hcompute<Cl>(w, taps, o);
  ring_store<Cl>(dst, o);
}

// ---------------------------------------------------------------------------
// consumer: vertical pass of the blocks that became ready at stage k
// ---------------------------------------------------------------------------
// Row blocks (tile-relative) whose V pass runs at stage k: block m is ready
// once its last pattern row m*Q + L - 1 has been loaded.
template <class Cl>
__host__ __device__ __forceinline__ void ready_blocks(const Geo& G, int k, int& m_lo, int& m_hi) {
  m_lo = k * Cl::SR - Cl::L + 1;
  m_lo = m_lo <= 0 ? 0 : (m_lo + Cl::Q - 1) / Cl::Q;
  m_hi = (k + 1) * Cl::SR - Cl::L;
  m_hi = m_hi < 0 ? -1 : m_hi / Cl::Q;
  if (m_hi > G.nblk - 1 || k == G.nst - 1) m_hi = G.nblk - 1;
}

// Four consecutive intermediate values of one ring row.
template <class Cl>
__device__ __forceinline__ void ring_load4(const typename Cl::R* p, float* h) {
  if constexpr (sizeof(typename Cl::R) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    h[0] = v.x; h[1] = v.y; h[2] = v.z; h[3] = v.w;
  } else {
    const uint2 v = *reinterpret_cast<const uint2*>(p);
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
    h[0] = a.x; h[1] = a.y; h[2] = b.x; h[3] = b.y;
  }
}

// Store four output values (vector store when aligned and complete).
template <typename T>
__device__ __forceinline__ void store4(T* o, const float* v, bool vec, int n_valid) {
  if (vec && n_valid >= 4) {
    if constexpr (sizeof(T) == 4) {
      *reinterpret_cast<float4*>(o) = make_float4(v[0], v[1], v[2], v[3]);
    } else if constexpr (sizeof(T) == 2) {
      const __half2 a = __floats2half2_rn(v[0], v[1]), b = __floats2half2_rn(v[2], v[3]);
      *reinterpret_cast<uint2*>(o) = make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
    } else {
      uint32_t pk = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i) pk |= (uint32_t)f_to_px<T>(v[i]) << (8 * i);
      *reinterpret_cast<uint32_t*>(o) = pk;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (i < n_valid) o[i] = f_to_px<T>(v[i]);
  }
}

// Output row r*P + J, columns e0..e0+3 of the strip: the K taps of phase J
// over the ring rows of its window, in tap order.  `rbase` is the ring row of
// the tile's relative row 0.
template <class Cl, int J>
__device__ __forceinline__ void vtask(const JobDesc& jd, const Geo& G, const float* __restrict__ taps,
                                      const typename Cl::R* __restrict__ ring, int rbase, int r, int e0,
                                      typename Cl::T* o, int n_valid) {
  using T = typename Cl::T;
  const int row0 = r * Cl::Q + Cl::b(J);  // first input row of the window
  float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  float h[4];
  if (row0 >= 0 && row0 + Cl::K - 1 < jd.H) {
    const int q0 = rbase + row0 - G.ys;
    const int s0 = q0 & Cl::RING_MASK;
    if (s0 + Cl::K <= Cl::RING) {
      const typename Cl::R* p = ring + s0 * Cl::SOE + e0;  // K consecutive ring rows
#pragma unroll
      for (int t = 0; t < Cl::K; ++t) {
        ring_load4<Cl>(p + t * Cl::SOE, h);
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[v] = fmaf(taps[J * Cl::K + t], h[v], acc[v]);
      }
    } else {
#pragma unroll
      for (int t = 0; t < Cl::K; ++t) {
        ring_load4<Cl>(ring + ((q0 + t) & Cl::RING_MASK) * Cl::SOE + e0, h);
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[v] = fmaf(taps[J * Cl::K + t], h[v], acc[v]);
      }
    }
  } else {
    // frame top / bottom: clamp-to-edge rows
#pragma unroll
    for (int t = 0; t < Cl::K; ++t) {
      const int yc = clampi(row0 + t, 0, jd.H - 1);
      ring_load4<Cl>(ring + ((rbase + yc - G.ys) & Cl::RING_MASK) * Cl::SOE + e0, h);
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[v] = fmaf(taps[J * Cl::K + t], h[v], acc[v]);
    }
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) acc[v] = pass_round<T>(acc[v]);
  store4<T>(o, acc, jd.out_vec != 0, n_valid);
}

template <class Cl, int J>
__device__ __forceinline__ void vtask_phase(int j, const JobDesc& jd, const Geo& G, const float* taps,
                                            const typename Cl::R* ring, int rbase, int r, int e0,
                                            typename Cl::T* o, int n_valid) {
  if constexpr (J < Cl::P) {
    if (j == J) vtask<Cl, J>(jd, G, taps, ring, rbase, r, e0, o, n_valid);
    else vtask_phase<Cl, J + 1>(j, jd, G, taps, ring, rbase, r, e0, o, n_valid);
  }
}

// ---------------------------------------------------------------------------
// consumers: one tile
// ---------------------------------------------------------------------------
// Three pipelines meet here.  TMA -> H warps through full/empty (one stage
// of input rows each).  H warps -> V warps through hdone/vdone over the ring
// of intermediate rows, which holds kNRS stages: the rows of stage g live in
// ring rows (g*SR .. g*SR+SR-1) mod RING.  The V pass of stage g reads rows of
// stages g-D..g only (its blocks' windows are L <= D*SR+1 rows tall), so the
// H pass of stage g may overwrite stage g-kNRS once the V pass of stage
// g-kNRS+D is done.  When the class changes between tiles (the all-class
// kernel), the ring layout changes with it and the H pass waits for every
// earlier V pass instead.
template <class Cl, int NSTAGE, int STAGE_MAX>
__device__ bool h_tile(const FastParams& prm, const JobDesc& jd, const Tile& tl, uint8_t* stages,
                       uint8_t* ring_raw, uint64_t* full, uint64_t* empty, uint64_t* hdone, uint64_t* vdone,
                       uint32_t& g, bool class_changed, const volatile int* abort_flag) {
  using R = typename Cl::R;
  R* ring = reinterpret_cast<R*>(ring_raw);
  const float* taps = prm.taps[Cl::id];
  const Geo G = tile_geo<Cl>(jd, tl);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wx = warp % Cl::WX, wy = warp / Cl::WX;
  const int lg = wx * 32 + lane;                         // chunk index across the strip
  const int blk0 = tl.strip * Cl::SBLK + lg * Cl::NB;   // first packet of the chunk (frame coords)
  const int px0 = blk0 * Cl::Q;
  const bool active = blk0 * Cl::P < jd.OW;
  (void)px0;
  const Offs<Cl> of = thread_offs<Cl>(lg);
  const EdgeFix fix = edge_fix<Cl>(tl.strip, wx, jd.W);
  R* const ring_mine = ring + lg * Cl::NOUT;
  for (int k = 0; k < G.nst; ++k, ++g) {
    const uint32_t slot = g % NSTAGE;
    // wait results are made warp-uniform, so a timeout takes the whole warp out
    bool ok = __all_sync(0xffffffffu, mbar_wait(&full[slot], (g / NSTAGE) & 1u, abort_flag));
    const int dep = (class_changed && k == 0) ? (int)g - 1 : (int)g - kNRS + Cl::D;
    if (ok && dep >= 0)
      ok = __all_sync(0xffffffffu, mbar_wait(&vdone[dep % kNRS], (uint32_t)(dep / kNRS) & 1u, abort_flag));
    if (!ok) return false;
    uint8_t* stage = stages + slot * STAGE_MAX;
    // the warp's rows of this stage: border fix-ups, then all loads, then the
    // arithmetic (so the loads of every row are in flight together)
    constexpr int NR = Cl::SR / Cl::WY;
    bool valid[NR];
    uint32_t w[NR][Cl::NWT];
#pragma unroll
    for (int s = 0; s < NR; ++s) {
      const int i = wy + s * Cl::WY;
      const int rel = k * Cl::SR + i;
      const int y = G.ys + rel;
      valid[s] = y >= 0 && y < jd.H && rel < G.rows;  // other rows are never read by the V pass
      if (valid[s] && fix.nl + fix.nr > 0) apply_edge_fix<Cl>(stage + i * Cl::BOXB, fix, lane, jd.W, G.xw);
    }
#pragma unroll
    for (int s = 0; s < NR; ++s)
      if (valid[s]) load_row<Cl>(stage + (wy + s * Cl::WY) * Cl::BOXB, of, w[s]);
    if (active) {
#pragma unroll
      for (int s = 0; s < NR; ++s)
        if (valid[s])
          hrow<Cl>(w[s], taps, ring_mine + ((g * Cl::SR + wy + s * Cl::WY) & Cl::RING_MASK) * Cl::SOE);
    }
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(&empty[slot]);
      mbar_arrive(&hdone[g % kNRS]);
    }
  }
  return true;
}

template <class Cl>
__device__ bool v_tile(const FastParams& prm, const JobDesc& jd, const Tile& tl, const uint8_t* ring_raw,
                       uint64_t* hdone, uint64_t* vdone, uint32_t& g, const volatile int* abort_flag) {
  using T = typename Cl::T;
  using R = typename Cl::R;
  const R* ring = reinterpret_cast<const R*>(ring_raw);
  const float* taps = prm.taps[Cl::id];
  const Geo G = tile_geo<Cl>(jd, tl);
  const int vw = (threadIdx.x >> 5) - kNH, lane = threadIdx.x & 31;
  const int ncols = min(Cl::SOE, (jd.OW - G.ox0) * Cl::C);
  const int rowe = jd.OW * Cl::C;
  T* const obase = reinterpret_cast<T*>(jd.out) + (long long)tl.frame * jd.out_frame + (long long)G.ox0 * Cl::C;
  const int rbase = (int)((g * Cl::SR) & Cl::RING_MASK);  // ring row of the tile's first row
  for (int k = 0; k < G.nst; ++k, ++g) {
    if (!__all_sync(0xffffffffu, mbar_wait(&hdone[g % kNRS], (g / kNRS) & 1u, abort_flag))) return false;
    int m_lo, m_hi;
    ready_blocks<Cl>(G, k, m_lo, m_hi);
    // one (block, phase) pair per warp at a time, so the phase -- and with it
    // the compiled tap sequence -- is uniform across the warp; lanes take
    // groups of 4 columns (groups past the frame's right edge are skipped)
    constexpr int TPR = Cl::SOE / 4;
    const int npairs = (m_hi - m_lo + 1) * Cl::P;
    for (int pair = vw; pair < npairs; pair += kNV) {
      const int mb = pair / Cl::P, j = pair - mb * Cl::P;
      const int r = G.rb0 + m_lo + mb;
      const int oy = r * Cl::P + j;
      if (oy >= jd.OH) continue;
      T* const orow = obase + (long long)oy * rowe;
      for (int grp = lane; grp < TPR; grp += 32) {
        const int e0 = grp * 4;
        if (e0 >= ncols) break;
        vtask_phase<Cl, 0>(j, jd, G, taps, ring, rbase, r, e0, orow + e0, ncols - e0);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&vdone[g % kNRS]);
  }
  return true;
}

// ---------------------------------------------------------------------------
// class dispatch and the kernel
// ---------------------------------------------------------------------------
template <class... Cs>
struct Dispatch;
template <>
struct Dispatch<> {
  template <class F>
  __device__ static bool run(int, F&&) { return false; }
};
template <class C0, class... Rest>
struct Dispatch<C0, Rest...> {
  template <class F>
  __device__ static bool run(int cls, F&& f) {
    if (cls == C0::id) return f(C0{});
    return Dispatch<Rest...>::run(cls, f);
  }
};

template <int NSTAGE, class... Cs>
struct KernelShape {
  static constexpr int STAGE_MAX = cmax(Cs::STAGE_BYTES...);
  static constexpr int RING_MAX = cmax(Cs::RING_BYTES...);
  static constexpr int BAR_OFF = NSTAGE * STAGE_MAX + RING_MAX;
  static constexpr int SMEM = 128 + BAR_OFF + (2 * NSTAGE + 2 * kNRS) * 8 + 16;
};

// MINB: resident CTAs per SM the registers are budgeted for (2 for the
// single-class kernels; 1 for the all-class kernel, whose union of code paths
// needs more registers).
template <int NSTAGE, int MINB, class... Cs>
__global__ void __launch_bounds__(kThreads, MINB) k_fused_tma(const __grid_constant__ FastParams prm) {
  using KS = KernelShape<NSTAGE, Cs...>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  uint8_t* stages = smem;
  uint8_t* ring = smem + NSTAGE * KS::STAGE_MAX;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + KS::BAR_OFF);
  uint64_t* empty = full + NSTAGE;
  uint64_t* hdone = empty + NSTAGE;
  uint64_t* vdone = hdone + kNRS;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(vdone + kNRS);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kNH);
    }
    for (int s = 0; s < kNRS; ++s) {
      mbar_init(&hdone[s], kNH);
      mbar_init(&vdone[s], kNV);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  if (warp == kNWC) {
    // ------------------------------- producer
    if (lane != 0) return;
    uint32_t g = 0;
    bool ok = true;
    for (int t = blockIdx.x; ok && t < prm.total_tiles; t += gridDim.x) {
      const Tile tl = decode_tile(prm, t);
      const JobDesc& jd = prm.jobs[tl.job];
      ok = Dispatch<Cs...>::run(jd.cls, [&](auto cl) {
        return produce_tile<decltype(cl), NSTAGE, KS::STAGE_MAX>(jd, tl, stages, full, empty, g, abort_flag);
      });
    }
    if (!ok) {
      // leave no copy in flight: wait (bounded) for the last round of each slot
      *abort_flag = 1;
      atomicCAS(&g_fast_status, 0, kStatusTimeout);
      for (uint32_t s = 0; s < NSTAGE && s < g; ++s) {
        const uint32_t last = g - 1 - s;
        mbar_wait(&full[last % NSTAGE], (last / NSTAGE) & 1u, nullptr);
      }
    }
    return;
  }

  // --------------------------------- consumers: H warps and V warps
  uint32_t g = 0;
  int prev_cls = -1;
  for (int t = blockIdx.x; t < prm.total_tiles; t += gridDim.x) {
    const Tile tl = decode_tile(prm, t);
    const JobDesc& jd = prm.jobs[tl.job];
    int code = kStatusBadClass;
    const bool changed = prev_cls >= 0 && prev_cls != jd.cls;
    prev_cls = jd.cls;
    const bool ok = Dispatch<Cs...>::run(jd.cls, [&](auto cl) {
      code = kStatusTimeout;
      if (warp < kNH)
        return h_tile<decltype(cl), NSTAGE, KS::STAGE_MAX>(prm, jd, tl, stages, ring, full, empty, hdone, vdone, g,
                                                         changed, abort_flag);
      return v_tile<decltype(cl)>(prm, jd, tl, ring, hdone, vdone, g, abort_flag);
    });
    if (!ok) {
      if (lane == 0) {
        *abort_flag = 1;
        atomicCAS(&g_fast_status, 0, code);
      }
      return;
    }
  }
}

// ---------------------------------------------------------------------------
// row-streaming kernel: one self-contained pipeline per warp
// ---------------------------------------------------------------------------
// Each warp owns a tile (a strip of 32*NB packets x a band of output row
// blocks of one frame) and runs the whole filter on it by itself:
//   lane 0 issues TMA loads of SR input rows (plus the strip's halo) into the
//   warp's private ring of NST stages, each stage with its own mbarrier;
//   every input row goes through the horizontal pass in registers and lands
//   in a sliding window of the last L filtered rows, also in registers
//   (L rows x NOUT values per lane: the intermediate never leaves the SM);
//   each time Q new rows have entered the window, the warp computes the P
//   output rows of one block from the window and stores them.
// Rows above / below the frame are never loaded: their window slots take a
// copy of the first / last filtered row (clamp-to-edge); columns outside the
// frame are fixed up in shared memory as in the other kernel.  Warps
// synchronise with nothing but their own TMA completions.
__host__ __device__ constexpr int cgcd(int a, int b) { return b == 0 ? a : cgcd(b, a % b); }

template <class B, int SR_, int NST_>
struct RCls : B {
  static constexpr int SRR = SR_;                          // input rows per stage
  static constexpr int NST = NST_;                         // stages per warp
  static constexpr int BOXSTR = rup(SR_ * B::BOXB, 128);   // (hides the base's stage layout)
  static constexpr int RSTAGE = B::NBOX * BOXSTR;
  static constexpr int RTX = B::NBOX * SR_ * B::BOXB;      // TMA bytes per stage
  static constexpr int WARP_BYTES = NST_ * RSTAGE;
  static constexpr bool ROT = false;                       // bank rotation off: the selects cost more here
  // The stream of a tile is cut so that the window prologue (the first L-Q
  // pattern rows) fills whole stages, EXTRA rows being loaded before the first
  // pattern row; after it, every group of U = lcm(SR, Q) rows is USTG stages
  // and UBLK block steps, so each row's stage offset and window slot are
  // compile-time constants.
  static constexpr int PRE = B::L - B::Q;
  static constexpr int NPS = cdiv(PRE, SR_);
  static constexpr int EXTRA = NPS * SR_ - PRE;
  static constexpr int U = SR_ / cgcd(SR_, B::Q) * B::Q;
  static constexpr int USTG = U / SR_;
  static constexpr int UBLK = U / B::Q;
  static_assert(B::WX == 1, "one warp per strip");
  static_assert(PRE > B::LH, "the window prologue must reach frame row 0");
  static_assert(B::L * (sizeof(typename B::T) == 1 ? (B::NOUT + 3) / 4 : B::NOUT) <= 48,
                "register window too large");
  static_assert(U <= 16, "iteration unit too long to unroll");
};

//                 base class   SR NST
using RF32_38 = RCls<CF32_38, 4, 3>;
using RF32_12 = RCls<CF32_12, 4, 3>;
using RF32_23 = RCls<CF32_23, 6, 3>;
using RF16_38 = RCls<CF16_38, 4, 3>;
using RF16_12 = RCls<CF16_12, 4, 3>;
using RF16_23 = RCls<CF16_23, 6, 3>;
// uint8 RGB (integer row math): one warp per strip, chunks of whole words
using CU8_38r = Cls<kFcU8C3_38, uint8_t, 3, 3, 8, 8, 1, 1, 8, 4>;
using CU8_12r = Cls<kFcU8C3_12, uint8_t, 3, 1, 2, 6, 4, 1, 8, 4>;
using CU8_23r = Cls<kFcU8C3_23, uint8_t, 3, 2, 3, 6, 4, 1, 8, 4>;
using RU8_38 = RCls<CU8_38r, 4, 3>;
using RU8_12 = RCls<CU8_12r, 4, 3>;
using RU8_23 = RCls<CU8_23r, 3, 3>;

// Store n_valid (<= N) consecutive output values with the widest aligned stores.
template <typename T, int N>
__device__ __forceinline__ void store_run(T* o, const float* v, int n_valid) {
  constexpr int BYTES = N * (int)sizeof(T);
  const uintptr_t a = reinterpret_cast<uintptr_t>(o);
  if (n_valid >= N) {
    if constexpr (sizeof(T) == 4) {
      if constexpr (BYTES % 16 == 0) {
        if ((a & 15) == 0) {
#pragma unroll
          for (int i = 0; i < N / 4; ++i)
            reinterpret_cast<float4*>(o)[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
          return;
        }
      }
      if constexpr (BYTES % 8 == 0) {
        if ((a & 7) == 0) {
#pragma unroll
          for (int i = 0; i < N / 2; ++i) reinterpret_cast<float2*>(o)[i] = make_float2(v[2 * i], v[2 * i + 1]);
          return;
        }
      }
    } else if constexpr (sizeof(T) == 2) {
      if constexpr (N % 2 == 0) {
        if ((a & 3) == 0) {
#pragma unroll
          for (int i = 0; i < N / 2; ++i) reinterpret_cast<__half2*>(o)[i] = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
          return;
        }
      }
    } else {
      if constexpr (N % 2 == 0) {
        if ((a & 1) == 0) {
#pragma unroll
          for (int i = 0; i < N / 2; ++i)
            reinterpret_cast<unsigned short*>(o)[i] =
                (unsigned short)((uint32_t)f_to_px<T>(v[2 * i]) | ((uint32_t)f_to_px<T>(v[2 * i + 1]) << 8));
          return;
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < N; ++i)
    if (i < n_valid) o[i] = f_to_px<T>(v[i]);
}

// ---------------------------------------------------------------------------
// row math of the row-streaming kernel
// ---------------------------------------------------------------------------
// What one row of the register window holds, how the H pass fills it from a
// loaded input row and how the V pass turns the window into P output rows.

template <class Cl, bool INT = (sizeof(typename Cl::T) == 1)>
struct RowMath;

// Float data: FP32 values, FMA chains in tap order.
template <class Cl>
struct RowMath<Cl, false> {
  using T = typename Cl::T;
  static constexpr int N = Cl::NOUT;
  struct Row {
    float v[N];
  };
  __device__ static __forceinline__ void h(const uint32_t* w, const FastParams& prm, Row& r) {
    hcompute<Cl>(w, prm.taps[Cl::id], r.v);
  }
  __device__ static __forceinline__ void copy(Row& d, const Row& s) {
#pragma unroll
    for (int k = 0; k < N; ++k) d.v[k] = s.v[k];
  }
  // the P output rows of block rr from the window
  __device__ static __forceinline__ void v(const Row (&win)[Cl::L], const FastParams& prm, T* obase,
                                           long long rowe, int rr, int OH, int n_valid) {
    const float* taps = prm.taps[Cl::id];
#pragma unroll
    for (int jv = 0; jv < Cl::P; ++jv) {
      const int oy = rr * Cl::P + jv;
      if (oy < OH) {
        float acc[N];
#pragma unroll
        for (int k = 0; k < N; ++k) acc[k] = 0.0f;
#pragma unroll
        for (int tt = 0; tt < Cl::K; ++tt) {
          const float wt = taps[jv * Cl::K + tt];
#pragma unroll
          for (int k = 0; k < N; ++k) acc[k] = fmaf(wt, win[Cl::b(jv) - Cl::BMIN + tt].v[k], acc[k]);
        }
#pragma unroll
        for (int k = 0; k < N; ++k) acc[k] = pass_round<T>(acc[k]);
        store_run<T, N>(obase + (long long)oy * rowe, acc, n_valid);
      }
    }
  }
};

// dp2a: c + a.lo16 * b.byte(2h) + a.hi16 * b.byte(2h+1), taps signed,
// pixels unsigned; h = 0 (.lo) or 1 (.hi).
template <int HALF>
__device__ __forceinline__ int dp2a(uint32_t taps, uint32_t px, int c) {
  int d;
  if constexpr (HALF == 0) asm("dp2a.lo.s32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(taps), "r"(px), "r"(c));
  else asm("dp2a.hi.s32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(taps), "r"(px), "r"(c));
  return d;
}

// Bytes p0 <= p1 <= p2 <= p3 of the word array w (spanning at most four
// words, every one of them inside the array) as one word, byte k = byte pk.
// The positions are compile-time constants after unrolling, so the selectors
// fold and only the words that hold one of the bytes are read.
__device__ __forceinline__ uint32_t gather4(const uint32_t* w, int p0, int p1, int p2, int p3) {
  const int pos[4] = {p0, p1, p2, p3};
  const int a = p0 >> 2, top = (p3 >> 2) - a;
  unsigned s1 = 0, s2 = 0, s3 = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int wi = (pos[k] >> 2) - a, by = pos[k] & 3;
    if (wi <= 1) {
      s1 |= (unsigned)(wi * 4 + by) << (4 * k);
      s3 |= (unsigned)k << (4 * k);
    } else {
      s2 |= (unsigned)((wi - 2) * 4 + by) << (4 * k);
      s3 |= (unsigned)(4 + (top == 2 ? by : k)) << (4 * k);
    }
  }
  if (top == 0) return __byte_perm(w[a], w[a], s1);
  const uint32_t r1 = __byte_perm(w[a], w[a + 1], s1);
  if (top == 1) return r1;
  if (top == 2) return __byte_perm(r1, w[a + 2], s3);
  return __byte_perm(r1, __byte_perm(w[a + 2], w[a + 3], s2), s3);
}

// (acc + 2^13) >> 14 has been taken by starting acc at 2^13: floor shift, clamp.
__device__ __forceinline__ int u8_round(int acc) { return __vimin_s32_relu(acc >> 14, 255); }

// Four values 0..255 as the bytes of one word (v0 lowest).
__device__ __forceinline__ uint32_t pack4(int v0, int v1, int v2, int v3) {
  return __byte_perm(__byte_perm((uint32_t)v0, (uint32_t)v1, 0x0040u), __byte_perm((uint32_t)v2, (uint32_t)v3, 0x0040u),
                     0x5410u);
}

// Store n_valid (<= 4*NW) bytes of words w to o with the widest aligned stores.
template <int NB>
__device__ __forceinline__ void store_bytes(uint8_t* o, const uint32_t* w, int n_valid) {
  constexpr int NW = (NB + 3) / 4;
  const uintptr_t a = reinterpret_cast<uintptr_t>(o);
  if (n_valid >= NB && (a & 3) == 0) {
#pragma unroll
    for (int i = 0; i < NB / 4; ++i) reinterpret_cast<uint32_t*>(o)[i] = w[i];
#pragma unroll
    for (int i = NB / 4 * 4; i < NB; ++i) o[i] = (uint8_t)(w[i >> 2] >> (8 * (i & 3)));
    return;
  }
  if (n_valid >= NB && (a & 1) == 0) {
#pragma unroll
    for (int i = 0; i < NB / 2; ++i)
      reinterpret_cast<unsigned short*>(o)[i] = (unsigned short)(w[(2 * i) >> 2] >> (8 * ((2 * i) & 3)));
    if constexpr (NB % 2) o[NB - 1] = (uint8_t)(w[(NB - 1) >> 2] >> (8 * ((NB - 1) & 3)));
    return;
  }
  (void)NW;
#pragma unroll
  for (int i = 0; i < NB; ++i)
    if (i < n_valid) o[i] = (uint8_t)(w[i >> 2] >> (8 * (i & 3)));
}

// uint8 data: exact integer arithmetic with packed bytes.  A window row holds
// the lane's NOUT horizontal results as bytes (4 per word, in output order).
// The H pass first gathers each channel's pixels into words of 4 consecutive
// pixels, then every output is K/2 (+1 for a window starting on an odd
// pixel) dp2a steps over pixel pairs against the int16 tap pairs; the V pass
// interleaves the bytes of window rows 2m and 2m+1 column by column and does
// the same over row pairs.  Sums start at 2^13, so (acc + 2^13) >> 14 is a
// plain shift; the results are the bits of the float kernels and the oracle.
template <class Cl>
struct RowMath<Cl, true> {
  using T = uint8_t;
  static constexpr int C = Cl::C, Q = Cl::Q, P = Cl::P, K = Cl::K, L = Cl::L, BMIN = Cl::BMIN;
  static constexpr int N = Cl::NOUT;
  static constexpr int NW = (N + 3) / 4;
  static constexpr int NXP = Cl::LH + Cl::NB * Q + Cl::RH;  // window pixels of a lane
  static constexpr int NCW = (NXP + 1 + 3) / 4;             // channel words (+1: odd-start pad)
  static constexpr int NPR = (L + 2) / 2;                   // window row pairs (+1 slot of pad)
  static constexpr int U8I = Cl::id - kFcU8C3_38;
  static_assert(Cl::HB * Cl::VB >= Cl::LH * C, "pixel slot 0 must be a loaded byte");
  static_assert(Cl::HB * Cl::VB - Cl::LH * C + NXP * C <= Cl::NVT * Cl::VB, "gathered bytes must be loaded");
  static_assert(U8I >= 0 && U8I < kU8Classes && P <= 3 && (K + 2) / 2 <= kMaxPairs, "tap pair table");
  struct Row {
    uint32_t w[NW];
  };
  __device__ static __forceinline__ void copy(Row& d, const Row& s) {
#pragma unroll
    for (int k = 0; k < NW; ++k) d.w[k] = s.w[k];
  }
  __device__ static __forceinline__ uint32_t tp(const FastParams& prm, int par, int j, int i) {
    return prm.tap2[U8I][par][j][i];
  }
  __device__ static __forceinline__ void h(const uint32_t* w, const FastParams& prm, Row& r) {
    constexpr int first = Cl::HB * Cl::VB - Cl::LH * C;  // byte of pixel slot 0, channel 0
    uint32_t cw[C][NCW];
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int k = 0; k < NCW; ++k) {
        int pos[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int slot = (4 * k + i < NXP) ? 4 * k + i : NXP - 1;  // pad slots: any byte
          pos[i] = first + slot * C + c;
        }
        cw[c][k] = gather4(w, pos[0], pos[1], pos[2], pos[3]);
      }
    int v[N];
#pragma unroll
    for (int n = 0; n < Cl::NB; ++n)
#pragma unroll
      for (int j = 0; j < P; ++j) {
        const int s0 = n * Q + Cl::b(j) - BMIN;  // first window slot of the output
        const int par = s0 & 1, pr0 = (s0 - par) / 2, npair = (K + par + 1) / 2;
#pragma unroll
        for (int c = 0; c < C; ++c) {
          int acc = 8192;
#pragma unroll
          for (int i = 0; i < npair; ++i) {
            const int pi = pr0 + i;
            acc = (pi & 1) ? dp2a<1>(tp(prm, par, j, i), cw[c][pi >> 1], acc)
                           : dp2a<0>(tp(prm, par, j, i), cw[c][pi >> 1], acc);
          }
          v[(n * P + j) * C + c] = u8_round(acc);
        }
      }
#pragma unroll
    for (int k = 0; k < NW; ++k) {
      const int e = 4 * k;
      r.w[k] = pack4(v[e], e + 1 < N ? v[e + 1] : 0, e + 2 < N ? v[e + 2] : 0, e + 3 < N ? v[e + 3] : 0);
    }
  }
  __device__ static __forceinline__ void v(const Row (&win)[L], const FastParams& prm, T* obase, long long rowe,
                                           int rr, int OH, int n_valid) {
    // one word column g (4 output columns) at a time: row-pair words
    // pl = bytes 0,1 of rows 2m and 2m+1 interleaved, ph = bytes 2,3
    uint32_t o[P][NW];
#pragma unroll
    for (int g = 0; g < NW; ++g) {
      uint32_t pl[NPR], ph[NPR];
#pragma unroll
      for (int m = 0; m < NPR; ++m) {
        const int r0 = 2 * m < L ? 2 * m : L - 1, r1 = 2 * m + 1 < L ? 2 * m + 1 : L - 1;
        pl[m] = __byte_perm(win[r0].w[g], win[r1].w[g], 0x5140u);
        ph[m] = __byte_perm(win[r0].w[g], win[r1].w[g], 0x7362u);
      }
#pragma unroll
      for (int jv = 0; jv < P; ++jv) {
        const int s0 = Cl::b(jv) - BMIN;
        const int par = s0 & 1, pr0 = (s0 - par) / 2, npair = (K + par + 1) / 2;
        int v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          int acc = 8192;
#pragma unroll
          for (int i = 0; i < npair; ++i) {
            const uint32_t word = (e & 2) ? ph[pr0 + i] : pl[pr0 + i];
            acc = (e & 1) ? dp2a<1>(tp(prm, par, jv, i), word, acc) : dp2a<0>(tp(prm, par, jv, i), word, acc);
          }
          v[e] = u8_round(acc);
        }
        o[jv][g] = pack4(v[0], v[1], v[2], v[3]);
      }
    }
#pragma unroll
    for (int jv = 0; jv < P; ++jv) {
      const int oy = rr * P + jv;
      if (oy < OH) store_bytes<N>(obase + (long long)oy * rowe, o[jv], n_valid);
    }
  }
};

template <class Cl, int WPC, int MINB>
__global__ void __launch_bounds__(WPC * 32, MINB) k_rows(const __grid_constant__ FastParams prm) {
  using T = typename Cl::T;
  using RM = RowMath<Cl>;
  using Row = typename RM::Row;
  constexpr int L = Cl::L, Q = Cl::Q, P = Cl::P, SR = Cl::SRR, NST = Cl::NST;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* const ring = smem + warp * Cl::WARP_BYTES;
  uint64_t* const full = reinterpret_cast<uint64_t*>(smem + WPC * Cl::WARP_BYTES) + warp * NST;
  if (lane == 0) {
    for (int s = 0; s < NST; ++s) mbar_init(&full[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncwarp();
  const Offs<Cl> of = thread_offs<Cl>(lane);
  const unsigned nwarps = gridDim.x * WPC;
  unsigned* const next = &g_tile_next[prm.sched_slot];
  auto next_tile = [&]() -> int {
    unsigned t = 0;
    if (lane == 0) t = atomicAdd(next, 1u);
    return (int)__shfl_sync(0xffffffffu, t, 0);
  };
  uint32_t g = 0;       // this warp's stage counter over all its tiles (mbarrier phases)
  uint32_t issued = 0;  // one past the last stage issued
  bool ok = true;
  for (int t = next_tile(); ok && t < prm.total_tiles; t = next_tile()) {
    const Tile tl = decode_tile(prm, t);
    const JobDesc& jd = prm.jobs[tl.job];
    if (jd.cls != Cl::id) {
      ok = false;
      break;
    }
    const int H = jd.H;
    const int nby = (jd.OH + P - 1) / P;
    const int rb0 = tl.chunk * jd.rbc;
    const int nblk = min(jd.rbc, nby - rb0);
    const int ys = rb0 * Q + Cl::BMIN;  // first pattern row; < 0 only for the top band (then == BMIN)
    const int nst = Cl::NPS + (nblk * Q + SR - 1) / SR;
    const int ystream = ys - Cl::EXTRA;  // frame row of stage 0's first row
    const int xw = tl.strip * Cl::SPX * Cl::C - Cl::HLB / Cl::SZ;
    const EdgeFix fix = edge_fix<Cl>(tl.strip, 0, jd.W);
    const bool fixing = fix.nl + fix.nr > 0;
    const int blk0 = tl.strip * Cl::SBLK + lane * Cl::NB;
    const bool active = blk0 * P < jd.OW;
    const int n_valid = jd.OW * Cl::C - blk0 * P * Cl::C;
    T* const obase = reinterpret_cast<T*>(jd.out) + (long long)tl.frame * jd.out_frame + (long long)blk0 * P * Cl::C;
    const long long rowe = (long long)jd.OW * Cl::C;

    auto issue = [&](int s) {  // stage s of the tile into slot (g + s) mod NST
      const uint32_t G = g + (uint32_t)s, slot = G % NST;
      mbar_expect_tx(&full[slot], Cl::RTX);
#pragma unroll
      for (int bx = 0; bx < Cl::NBOX; ++bx)
        tma_load_3d(ring + slot * Cl::RSTAGE + bx * Cl::BOXSTR, &jd.tmap, &full[slot], xw + bx * Cl::BOXE,
                    ystream + s * SR, tl.frame);
    };
    if (lane == 0)
      for (int s = 0; s < NST && s < nst; ++s) issue(s);
    issued = g + (uint32_t)min(NST, nst);
    // wait for stage s; returns the stage's row-0 base, or nullptr on timeout
    auto stage_wait = [&](int s) -> uint8_t* {
      const uint32_t G = g + (uint32_t)s, slot = G % NST;
      if (!__all_sync(0xffffffffu, mbar_wait(&full[slot], (G / NST) & 1u, nullptr))) return nullptr;
      return ring + slot * Cl::RSTAGE;
    };
    // stage s fully read: refill its slot with stage s + NST
    auto stage_release = [&](int s) {
      __syncwarp();
      if (s + NST < nst) {
        if (lane == 0) issue(s + NST);
        issued = g + (uint32_t)(s + NST + 1);
      }
    };
    // H pass of one loaded row into a window row
    auto hrow_regs = [&](uint8_t* rowbase, Row& o) {
      if (fixing) apply_edge_fix<Cl>(rowbase, fix, lane, jd.W, xw);
      uint32_t w[Cl::NWT];
      load_row<Cl>(rowbase, of, w);
      if (active) RM::h(w, prm, o);
    };

    Row win[L];
    // ---- prologue: pattern rows 0 .. L-Q-1
#pragma unroll
    for (int ps = 0; ps < Cl::NPS; ++ps) {
      uint8_t* sb = stage_wait(ps);
      if (!sb) {
        ok = false;
        break;
      }
#pragma unroll
      for (int r = 0; r < SR; ++r) {
        const int i = ps * SR + r - Cl::EXTRA;  // pattern row index
        if (i < 0) continue;                    // loaded only to align the stages
        const int y = ys + i;
        if (y < 0) continue;                    // top band: filled from frame row 0 below
        if (i > 0 && y >= H) {
          RM::copy(win[i], win[i - 1]);
        } else {
          hrow_regs(sb + r * Cl::BOXB, win[i]);
        }
      }
      stage_release(ps);
    }
    if (!ok) break;
    if (ys < 0) {  // ys == BMIN: slots 0..LH-1 are frame row 0, held in slot LH
#pragma unroll
      for (int i = 0; i < Cl::LH; ++i) RM::copy(win[i], win[Cl::LH]);
    }
    // ---- block steps, U rows (USTG stages, UBLK blocks) at a time
    const int nunits = (nblk + Cl::UBLK - 1) / Cl::UBLK;
    for (int u = 0; ok && u < nunits; ++u) {
#pragma unroll
      for (int st = 0; st < Cl::USTG; ++st) {
        const int s = Cl::NPS + u * Cl::USTG + st;
        if (s >= nst) break;
        uint8_t* sb = stage_wait(s);
        if (!sb) {
          ok = false;
          break;
        }
#pragma unroll
        for (int r = 0; r < SR; ++r) {
          constexpr int dummy = 0;
          (void)dummy;
          const int ru = st * SR + r;       // row within the unit
          const int bq = ru / Q, q = ru - bq * Q;
          const int m = u * Cl::UBLK + bq;  // block step
          if (m < nblk) {
            const int i = L - Q + q;
            const int y = ys + m * Q + i;
            if (y >= H) {
              RM::copy(win[i], win[i - 1]);
            } else {
              hrow_regs(sb + r * Cl::BOXB, win[i]);
            }
            if (q == Q - 1) {
              // the window holds block m's pattern: its P output rows
              if (active) RM::v(win, prm, obase, rowe, rb0 + m, jd.OH, n_valid);
#pragma unroll
              for (int i2 = 0; i2 < L - Q; ++i2) RM::copy(win[i2], win[i2 + Q]);
            }
          }
        }
        stage_release(s);
      }
    }
    g += (uint32_t)nst;
  }
  if (!ok) {
    // a wait gave up (or a job of the wrong class): record it and leave no
    // copy in flight
    if (lane == 0) {
      atomicCAS(&g_fast_status, 0, kStatusTimeout);
      for (uint32_t G = (issued > (uint32_t)NST ? issued - NST : 0); G < issued; ++G)
        mbar_wait(&full[G % NST], (G / NST) & 1u, nullptr);
    }
  }
  // the last warp out resets the slot for its next launch
  if (lane == 0) {
    __threadfence();
    if (atomicAdd(&g_warps_done[prm.sched_slot], 1u) == nwarps - 1) {
      g_tile_next[prm.sched_slot] = 0;
      g_warps_done[prm.sched_slot] = 0;
      __threadfence();
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct HostGeom {
  int sblk, spx, p, q, boxe, sr, sz, c, ve;
  CUtensorMapDataType dt;
};

template <class Cl>
HostGeom host_geom() {
  return HostGeom{Cl::SBLK, Cl::SPX, Cl::P, Cl::Q, Cl::BOXE, Cl::SR, Cl::SZ, Cl::C, Cl::VE, TmaType<typename Cl::T>::v};
}
template <class Cl>
HostGeom host_geom_rows() {
  HostGeom g = host_geom<Cl>();
  g.sr = Cl::SRR;
  return g;
}

// Classes with a row-streaming kernel (their register window fits).
bool has_rows_kernel(int cls) {
  switch (cls) {
    case kFcF32_38: case kFcF32_12: case kFcF32_23:
    case kFcF16_38: case kFcF16_12: case kFcF16_23:
    case kFcU8C3_38: case kFcU8C3_12: case kFcU8C3_23: return true;
    default: return false;
  }
}

// Geometry of the kernel that runs class `cls`.
HostGeom geom_of(int cls) {
  switch (cls) {
    case kFcF32_38: return host_geom_rows<RF32_38>();
    case kFcF32_12: return host_geom_rows<RF32_12>();
    case kFcF32_23: return host_geom_rows<RF32_23>();
    case kFcF16_38: return host_geom_rows<RF16_38>();
    case kFcF16_12: return host_geom_rows<RF16_12>();
    case kFcF16_23: return host_geom_rows<RF16_23>();
    case kFcU8C3_38: return host_geom_rows<RU8_38>();
    case kFcU8C3_12: return host_geom_rows<RU8_12>();
    default: return host_geom_rows<RU8_23>();
  }
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

struct KernelInfo {
  const void* fn;
  int smem;
  int threads;
};

template <int NSTAGE, class... Cs>
KernelInfo kernel_info() {
  constexpr int minb = sizeof...(Cs) == 1 ? 2 : 1;
  return KernelInfo{reinterpret_cast<const void*>(&k_fused_tma<NSTAGE, minb, Cs...>), KernelShape<NSTAGE, Cs...>::SMEM,
                    kThreads};
}

constexpr int kRowsWPC = 4;  // warps (independent pipelines) per CTA of the row-streaming kernel

// Registers are budgeted for 4 resident CTAs (16 warps) per SM, which the
// shared-memory footprint of the stage rings also allows.
template <class Cl>
KernelInfo rows_info() {
  constexpr int smem = 128 + kRowsWPC * (Cl::WARP_BYTES + Cl::NST * 8);
  return KernelInfo{reinterpret_cast<const void*>(&k_rows<Cl, kRowsWPC, 4>), smem, kRowsWPC * 32};
}

// The kernel that runs class `cls` (all jobs of a launch share the class).
KernelInfo kernel_for(int cls) {
  switch (cls) {
    case kFcF32_38: return rows_info<RF32_38>();
    case kFcF32_12: return rows_info<RF32_12>();
    case kFcF32_23: return rows_info<RF32_23>();
    case kFcF16_38: return rows_info<RF16_38>();
    case kFcF16_12: return rows_info<RF16_12>();
    case kFcF16_23: return rows_info<RF16_23>();
    case kFcU8C3_38: return rows_info<RU8_38>();
    case kFcU8C3_12: return rows_info<RU8_12>();
    default: return rows_info<RU8_23>();
  }
}

// Occupancy per kernel, computed once per process (one device).
int ctas_per_sm(const KernelInfo& ki) {
  static std::mutex mu;
  static std::vector<std::pair<const void*, int>> cache;
  std::lock_guard<std::mutex> lock(mu);
  for (auto& e : cache)
    if (e.first == ki.fn) return e.second;
  int occ = 0;
  if (cudaFuncSetAttribute(ki.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, ki.smem) != cudaSuccess) return 0;
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

void fill_taps(FastParams& prm) {
  // the fast classes' taps depend only on (p, q, K): build them once with a
  // throwaway plan of each class
  static FastParams taps_only;
  static std::once_flag once;
  std::call_once(once, [] {
    std::memset(&taps_only, 0, sizeof(taps_only));
    const int pq[3][3] = {{3, 8, 8}, {1, 2, 6}, {2, 3, 6}};
    const ds_dtype dts[3] = {DS_F32, DS_F16, DS_U8_RGB};
    for (int d = 0; d < 3; ++d)
      for (int r = 0; r < 3; ++r) {
        ds_plan* pl = ds_plan_create(64, 64, ds_ratio{pq[r][0], pq[r][1]}, pq[r][2], dts[d]);
        if (!pl) continue;
        const int cls = pl->fast_class;
        for (int i = 0; i < pl->p * pl->K; ++i)
          taps_only.taps[cls][i] = (dts[d] == DS_U8_RGB) ? (float)pl->q14[i] : pl->w32[i];
        if (dts[d] == DS_U8_RGB) {
          const int u = cls - kFcU8C3_38;
          for (int par = 0; par < 2; ++par)
            for (int j = 0; j < pl->p; ++j)
              for (int i = 0; i < kMaxPairs; ++i) {
                const int ta = 2 * i - par, tb = 2 * i + 1 - par;
                const int qa = (ta >= 0 && ta < pl->K) ? pl->q14[j * pl->K + ta] : 0;
                const int qb = (tb >= 0 && tb < pl->K) ? pl->q14[j * pl->K + tb] : 0;
                taps_only.tap2[u][par][j][i] = (uint32_t)(uint16_t)(int16_t)qa | ((uint32_t)(uint16_t)(int16_t)qb << 16);
              }
        }
        ds_destroy(pl);
      }
  });
  std::memcpy(prm.taps, taps_only.taps, sizeof(prm.taps));
  std::memcpy(prm.tap2, taps_only.tap2, sizeof(prm.tap2));
}

// Tile geometry of a job (everything but the tensor map).  `band`: output
// row blocks per tile, 0 = the plan's.
void fill_job_geometry(JobDesc& jd, const ds_plan* pl, void* out, int n_frames, int band = 0) {
  const HostGeom hg = geom_of(pl->fast_class);
  jd.out = out;
  jd.out_frame = (long long)pl->out_frame_elems();
  jd.H = pl->in_h;
  jd.W = pl->in_w;
  jd.OH = pl->out_h;
  jd.OW = pl->out_w;
  jd.nframes = n_frames;
  jd.cls = pl->fast_class;
  const int nbx = (pl->out_w + hg.p - 1) / hg.p;
  const int nby = (pl->out_h + hg.p - 1) / hg.p;
  jd.strips = (nbx + hg.sblk - 1) / hg.sblk;
  jd.rbc = std::max(1, std::min(band > 0 ? band : pl->row_blocks, nby));
  jd.chunks = (nby + jd.rbc - 1) / jd.rbc;
  jd.tiles = jd.strips * jd.chunks * n_frames;
  jd.out_vec = (((uintptr_t)out & 3u) == 0 && ((size_t)pl->out_w * pl->channels) % 4 == 0) ? 1 : 0;
}

ds_status encode_job(JobDesc& jd, const FastJob& job, int band) {
  const ds_plan* pl = job.plan;
  const HostGeom hg = geom_of(pl->fast_class);
  auto enc = encode_fn();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return DS_ERR_CUDA;
  }
  const cuuint64_t row_elems = (cuuint64_t)pl->in_w * pl->channels;
  cuuint64_t dims[3] = {row_elems, (cuuint64_t)pl->in_h, (cuuint64_t)job.n_frames};
  cuuint64_t strides[2] = {row_elems * hg.sz, row_elems * hg.sz * (cuuint64_t)pl->in_h};
  cuuint32_t box[3] = {(cuuint32_t)hg.boxe, (cuuint32_t)hg.sr, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(&jd.tmap, hg.dt, 3, const_cast<void*>(job.in), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d) for a %dx%d frame", (int)r, pl->in_h, pl->in_w);
    return DS_ERR_CUDA;
  }
  fill_job_geometry(jd, pl, job.out, job.n_frames, band);
  return DS_OK;
}

// Band height for the jobs of one launch.  A tile is processed serially by
// one warp (row kernel) or CTA, so a launch with fewer band-rows of work than
// the GPU has pipelines finishes sooner with shorter bands: the band is cut
// to ceil(block rows of work / pipelines), never above the plans' own value.
// Plans with a caller-set (or autotuned) schedule keep theirs.
int launch_band(const FastJob* jobs, int n, int pipelines) {
  long long units = 0;
  int cap = 0;
  for (int i = 0; i < n; ++i) {
    const ds_plan* pl = jobs[i].plan;
    if (pl->schedule_set) return 0;
    const HostGeom hg = geom_of(pl->fast_class);
    const long long nbx = (pl->out_w + hg.p - 1) / hg.p, nby = (pl->out_h + hg.p - 1) / hg.p;
    units += (nbx + hg.sblk - 1) / hg.sblk * nby * (long long)jobs[i].n_frames;
    cap = std::max(cap, pl->row_blocks);
  }
  const long long fill = (units + pipelines - 1) / std::max(1, pipelines);
  return (int)std::max<long long>(1, std::min<long long>(cap, fill));
}

// ---------------------------------------------------------------------------
// host-side check of the kernel's index arithmetic
// ---------------------------------------------------------------------------
// Walks every tile of one frame the way the kernel does and checks: TMA x
// coordinates are 16-byte aligned; every shared-memory read of the H pass
// (vector chunks, halo words, clamped border reads) stays inside the loaded
// window and never straddles a box; ring writes stay inside a ring row;
// every ring row the V pass reads was written by the H pass of an earlier or
// the same stage and is not overwritten by the next stage's H pass; every
// output element is written exactly once; the shared-memory footprint fits.
template <class Cl, int STAGE_MAX, int SMEM>
std::string check_class(const JobDesc& jd) {
  char buf[256];
  auto fail = [&](const char* what, int a, int b) {
    std::snprintf(buf, sizeof(buf), "class %d: %s (%d, %d)", Cl::id, what, a, b);
    return std::string(buf);
  };
  if (SMEM > 227 * 1024) return fail("shared memory above 227 KB", SMEM, 0);
  if (Cl::STAGE_BYTES > STAGE_MAX || Cl::BOXSTR < Cl::SR * Cl::BOXB) return fail("stage layout", Cl::STAGE_BYTES, STAGE_MAX);
  const int win = Cl::NBOX * Cl::BOXB;
  std::vector<int> written((size_t)jd.OH * jd.OW * Cl::C, 0);
  for (int chunk = 0; chunk < jd.chunks; ++chunk) {
    for (int strip = 0; strip < jd.strips; ++strip) {
      const Tile tl{0, 0, strip, chunk};
      const Geo G = tile_geo<Cl>(jd, tl);
      if (G.nblk < 1 || G.ox0 >= jd.OW) return fail("empty tile", chunk, strip);
      for (int bx = 0; bx < Cl::NBOX; ++bx) {
        const long long xb = (long long)(G.xw + bx * Cl::BOXE) * Cl::SZ;
        if (((xb % 16) + 16) % 16 != 0) return fail("TMA x not 16-byte aligned", G.xw, bx);
      }
      for (int wx = 0; wx < Cl::WX; ++wx) {
        const EdgeFix fx = edge_fix<Cl>(strip, wx, jd.W);
        // fix-up sources and destinations stay in the window
        for (int e = 0; e < fx.nl + fx.nr; ++e) {
          const bool left = e < fx.nl;
          const int k2 = left ? e : e - fx.nl;
          const int px = (left ? fx.l_lo : fx.r_lo) + k2 / Cl::C, c = k2 % Cl::C;
          const int src = (left ? 0 : jd.W - 1) * Cl::C + c - G.xw, dst = px * Cl::C + c - G.xw;
          if (src < 0 || (src + 1) * Cl::SZ > win || dst < 0 || (dst + 1) * Cl::SZ > win)
            return fail("edge fix outside the window", src, dst);
          if (px >= 0 && px < jd.W) return fail("edge fix inside the frame", px, jd.W);
        }
        for (int lane = 0; lane < 32; ++lane) {
          const int lg = wx * 32 + lane;
          const int first = Cl::HLB + lg * Cl::EB - Cl::HB * Cl::VB;
          for (int v = 0; v < Cl::NVT; ++v) {
            const int b0 = first + v * Cl::VB;
            if (b0 < 0 || b0 + Cl::VB > win || b0 / Cl::BOXB != (b0 + Cl::VB - 1) / Cl::BOXB)
              return fail("vector read", lg, b0);
          }
          const int blk0 = strip * Cl::SBLK + lg * Cl::NB;
          const int px0 = blk0 * Cl::Q;
          if (blk0 * Cl::P >= jd.OW) continue;  // inactive lane: loads only
          // element e of the thread (pixel px0 - LH + e/C) sits at window element px*C + c - xw
          const int el0 = (px0 - Cl::LH) * Cl::C - G.xw;
          if (el0 * Cl::SZ != first + Cl::HB * Cl::VB - Cl::LH * Cl::C * Cl::SZ) return fail("chunk not at its pixels", lg, el0);
          for (int px = px0 - Cl::LH; px < px0 + Cl::NB * Cl::Q + Cl::RH; ++px) {
            if (px < 0 && !(px >= fx.l_lo && fx.nl > 0)) return fail("left border pixel not fixed", lg, px);
            if (px >= jd.W && !(px >= fx.r_lo && px < fx.r_lo + fx.nr / Cl::C)) return fail("right border pixel not fixed", lg, px);
          }
          if (lg * Cl::NOUT + Cl::NOUT > Cl::SOE) return fail("ring write", lg, Cl::SOE);
        }
      }
      // ring rule: the V pass of stage k may read only rows the H pass wrote in
      // stages k-D..k (the H pass of stage k+kNRS-D overwrites stage k-D)
      std::vector<int> done(G.nblk, 0);
      for (int k = 0; k < G.nst; ++k) {
        int m_lo, m_hi;
        ready_blocks<Cl>(G, k, m_lo, m_hi);
        for (int m = m_lo; m <= m_hi; ++m) {
          if (m < 0 || m >= G.nblk || done[m]) return fail("block scheduled twice or out of range", m, k);
          done[m] = 1;
          const int r = G.rb0 + m;
          for (int i = 0; i < Cl::L; ++i) {
            int yc = r * Cl::Q + Cl::BMIN + i;
            yc = yc < 0 ? 0 : (yc > jd.H - 1 ? jd.H - 1 : yc);
            const int rel = yc - G.ys;
            if (rel < 0 || rel >= G.rows) return fail("V row outside the tile", rel, G.rows);
            const int st = rel / Cl::SR;
            if (st > k) return fail("V row not yet written", rel, k);
            if (k - st > Cl::D) return fail("V row older than the ring keeps", rel, k);
          }
          const int ncols = std::min(Cl::SOE, (jd.OW - G.ox0) * Cl::C);
          for (int j = 0; j < Cl::P; ++j) {
            const int oy = r * Cl::P + j;
            if (oy >= jd.OH) break;
            for (int e = 0; e < ncols; ++e) written[((size_t)oy * jd.OW + G.ox0) * Cl::C + e]++;
          }
        }
      }
      for (int m = 0; m < G.nblk; ++m)
        if (!done[m]) return fail("block never scheduled", m, chunk);
    }
  }
  for (size_t i = 0; i < written.size(); ++i)
    if (written[i] != 1) return fail("output element written != 1 times", (int)i, written[i]);
  return std::string();
}

// Host-side walk of the row-streaming kernel: the same TMA / window / edge
// checks as above, plus a replay of its stream and register-window logic on
// frame-row indices -- every V block must see exactly the clamped rows of
// its window, every stream row must be the next frame row in order, every
// output element is written once.
template <class Cl, int WPC>
std::string check_rows(const JobDesc& jd) {
  char buf[256];
  auto fail = [&](const char* what, int a, int b) {
    std::snprintf(buf, sizeof(buf), "rows class %d: %s (%d, %d)", Cl::id, what, a, b);
    return std::string(buf);
  };
  constexpr int smem = 128 + WPC * (Cl::WARP_BYTES + Cl::NST * 8);
  if (smem > 227 * 1024) return fail("shared memory above 227 KB", smem, 0);
  if (Cl::BOXSTR < Cl::SRR * Cl::BOXB) return fail("stage layout", Cl::BOXSTR, 0);
  const int win = Cl::NBOX * Cl::BOXB;
  constexpr int L = Cl::L, Q = Cl::Q, P = Cl::P;
  std::vector<int> written((size_t)jd.OH * jd.OW * Cl::C, 0);
  const int nby = (jd.OH + P - 1) / P;
  for (int chunk = 0; chunk < jd.chunks; ++chunk) {
    for (int strip = 0; strip < jd.strips; ++strip) {
      const int rb0 = chunk * jd.rbc;
      const int nblk = std::min(jd.rbc, nby - rb0);
      if (nblk < 1) return fail("empty tile", chunk, strip);
      const int ys = rb0 * Q + Cl::BMIN;
      const int ye = (rb0 + nblk - 1) * Q + Cl::BMIN + L;
      const int y0 = std::max(ys, 0), nrow = std::min(ye, jd.H) - y0;
      if (nrow < 1) return fail("empty stream", ys, ye);
      if (ys < 0 && ys != Cl::BMIN) return fail("top band offset", ys, 0);
      const int xw = strip * Cl::SPX * Cl::C - Cl::HLB / Cl::SZ;
      for (int bx = 0; bx < Cl::NBOX; ++bx) {
        const long long xb = (long long)(xw + bx * Cl::BOXE) * Cl::SZ;
        if (((xb % 16) + 16) % 16 != 0) return fail("TMA x not 16-byte aligned", xw, bx);
      }
      const EdgeFix fx = edge_fix<Cl>(strip, 0, jd.W);
      for (int e = 0; e < fx.nl + fx.nr; ++e) {
        const bool left = e < fx.nl;
        const int k2 = left ? e : e - fx.nl;
        const int px = (left ? fx.l_lo : fx.r_lo) + k2 / Cl::C, c = k2 % Cl::C;
        const int src = (left ? 0 : jd.W - 1) * Cl::C + c - xw, dst = px * Cl::C + c - xw;
        if (src < 0 || (src + 1) * Cl::SZ > win || dst < 0 || (dst + 1) * Cl::SZ > win)
          return fail("edge fix outside the window", src, dst);
      }
      for (int lane = 0; lane < 32; ++lane) {
        const int first = Cl::HLB + lane * Cl::EB - Cl::HB * Cl::VB;
        for (int v = 0; v < Cl::NVT; ++v) {
          const int b0 = first + v * Cl::VB;
          if (b0 < 0 || b0 + Cl::VB > win || b0 / Cl::BOXB != (b0 + Cl::VB - 1) / Cl::BOXB)
            return fail("vector read", lane, b0);
        }
        const int blk0 = strip * Cl::SBLK + lane * Cl::NB, px0 = blk0 * Cl::Q;
        if (blk0 * P >= jd.OW) continue;
        for (int px = px0 - Cl::LH; px < px0 + Cl::NB * Cl::Q + Cl::RH; ++px) {
          if (px < 0 && !(px >= fx.l_lo && fx.nl > 0)) return fail("left border pixel not fixed", lane, px);
          if (px >= jd.W && !(px >= fx.r_lo && px < fx.r_lo + fx.nr / Cl::C)) return fail("right border pixel not fixed", lane, px);
        }
      }
      // replay of the stream and window on frame-row indices: stage s holds
      // frame rows ystream + s*SR .. + SR - 1
      const int nst = Cl::NPS + (nblk * Q + Cl::SRR - 1) / Cl::SRR;
      const int ystream = ys - Cl::EXTRA;
      int wrow[64];
      int sr = 0;  // rows consumed from the stream, checked against their position
      auto take = [&](int s, int r, int i) -> std::string {
        if (s >= nst) return fail("stage beyond the tile", s, nst);
        wrow[i] = ystream + s * Cl::SRR + r;
        ++sr;
        return std::string();
      };
      for (int ps = 0; ps < Cl::NPS; ++ps)
        for (int r = 0; r < Cl::SRR; ++r) {
          const int i = ps * Cl::SRR + r - Cl::EXTRA;
          if (i < 0) continue;
          const int y = ys + i;
          if (y < 0) continue;
          if (i > 0 && y >= jd.H) { wrow[i] = wrow[i - 1]; continue; }
          std::string e = take(ps, r, i);
          if (!e.empty()) return e;
          if (wrow[i] != y) return fail("prologue row mismatch", i, wrow[i]);
        }
      if (ys < 0)
        for (int i = 0; i < Cl::LH; ++i) wrow[i] = wrow[Cl::LH];
      const int nunits = (nblk + Cl::UBLK - 1) / Cl::UBLK;
      for (int u = 0; u < nunits; ++u)
        for (int st = 0; st < Cl::USTG; ++st) {
          const int s = Cl::NPS + u * Cl::USTG + st;
          if (s >= nst) break;
          for (int r = 0; r < Cl::SRR; ++r) {
            const int ru = st * Cl::SRR + r, bq = ru / Q, q = ru - bq * Q, m = u * Cl::UBLK + bq;
            if (m >= nblk) continue;
            const int i = L - Q + q, y = ys + m * Q + i;
            if (y >= jd.H) wrow[i] = wrow[i - 1];
            else {
              std::string e = take(s, r, i);
              if (!e.empty()) return e;
              if (wrow[i] != y) return fail("stream row mismatch", i, wrow[i]);
            }
            if (q != Q - 1) continue;
            const int rr = rb0 + m;
            for (int i2 = 0; i2 < L; ++i2) {
              int want = rr * Q + Cl::BMIN + i2;
              want = want < 0 ? 0 : (want > jd.H - 1 ? jd.H - 1 : want);
              if (wrow[i2] != want) return fail("window row mismatch", i2, wrow[i2]);
            }
            for (int lane = 0; lane < 32; ++lane) {
              const int blk0 = strip * Cl::SBLK + lane * Cl::NB;
              if (blk0 * P >= jd.OW) continue;
              const int nv = std::min(Cl::NOUT, jd.OW * Cl::C - blk0 * P * Cl::C);
              for (int jv = 0; jv < P; ++jv) {
                const int oy = rr * P + jv;
                if (oy >= jd.OH) continue;
                for (int k = 0; k < nv; ++k) written[((size_t)oy * jd.OW) * Cl::C + (size_t)blk0 * P * Cl::C + k]++;
              }
            }
            for (int i2 = 0; i2 < L - Q; ++i2) wrow[i2] = wrow[i2 + Q];
          }
        }
      if (sr != nrow) return fail("stream rows left over", sr, nrow);
    }
  }
  for (size_t i = 0; i < written.size(); ++i)
    if (written[i] != 1) return fail("output element written != 1 times", (int)i, written[i]);
  return std::string();
}

template <int NSTAGE, class Cl>
std::string check_single(const JobDesc& jd) {
  using KS = KernelShape<NSTAGE, Cl>;
  return check_class<Cl, KS::STAGE_MAX, KS::SMEM>(jd);
}

template <class Cl>
std::string check_mixed(const JobDesc& jd) {
  using KS = KernelShape<3, CF32_38, CF32_12, CF32_23, CF16_38, CF16_12, CF16_23, CU8_38, CU8_12, CU8_23>;
  return check_class<Cl, KS::STAGE_MAX, KS::SMEM>(jd);
}

std::string check_plan(const ds_plan* pl) {
  JobDesc jd;
  std::memset(&jd, 0, sizeof(jd));
  fill_job_geometry(jd, pl, nullptr, 1);
  std::string a, b;
  if (has_rows_kernel(pl->fast_class)) {
    switch (pl->fast_class) {
      case kFcF32_38: return check_rows<RF32_38, kRowsWPC>(jd);
      case kFcF32_12: return check_rows<RF32_12, kRowsWPC>(jd);
      case kFcF32_23: return check_rows<RF32_23, kRowsWPC>(jd);
      case kFcF16_38: return check_rows<RF16_38, kRowsWPC>(jd);
      case kFcF16_12: return check_rows<RF16_12, kRowsWPC>(jd);
      case kFcF16_23: return check_rows<RF16_23, kRowsWPC>(jd);
      case kFcU8C3_38: return check_rows<RU8_38, kRowsWPC>(jd);
      case kFcU8C3_12: return check_rows<RU8_12, kRowsWPC>(jd);
      default: return check_rows<RU8_23, kRowsWPC>(jd);
    }
  }
  switch (pl->fast_class) {
    case kFcF32_38: a = check_single<4, CF32_38>(jd); b = check_mixed<CF32_38>(jd); break;
    case kFcF32_12: a = check_single<4, CF32_12>(jd); b = check_mixed<CF32_12>(jd); break;
    case kFcF32_23: a = check_single<4, CF32_23>(jd); b = check_mixed<CF32_23>(jd); break;
    case kFcF16_38: a = check_single<6, CF16_38>(jd); b = check_mixed<CF16_38>(jd); break;
    case kFcF16_12: a = check_single<6, CF16_12>(jd); b = check_mixed<CF16_12>(jd); break;
    case kFcF16_23: a = check_single<6, CF16_23>(jd); b = check_mixed<CF16_23>(jd); break;
    case kFcU8C3_38: a = check_single<8, CU8_38>(jd); b = check_mixed<CU8_38>(jd); break;
    case kFcU8C3_12: a = check_single<8, CU8_12>(jd); b = check_mixed<CU8_12>(jd); break;
    case kFcU8C3_23: a = check_single<4, CU8_23>(jd); b = check_mixed<CU8_23>(jd); break;
    default: return std::string();
  }
  return a.empty() ? b : a;
}

ds_status launch_chunk(const FastJob* jobs, int n, cudaStream_t st) {
  static thread_local FastParams prm;  // ~13 KB, too large for the stack of some callers
  std::memset(&prm, 0, sizeof(prm));
  fill_taps(prm);
  const int cls = jobs[0].plan->fast_class;  // launch_fast groups jobs by class
  int want_ctas = jobs[0].plan->ctas_per_sm;
  for (int i = 0; i < n; ++i) want_ctas = std::max(want_ctas, jobs[i].plan->ctas_per_sm);
  const KernelInfo ki = kernel_for(cls);
  int occ = ctas_per_sm(ki);
  if (occ <= 0) {
    set_error("fused kernel does not fit on this device (%d bytes of shared memory)", ki.smem);
    return DS_ERR_UNSUPPORTED;
  }
  if (want_ctas > 0) occ = std::min(occ, want_ctas);
  // the row-streaming kernel runs one tile per warp, the other one per CTA
  const int per_cta = has_rows_kernel(cls) ? ki.threads / 32 : 1;
  const int band = launch_band(jobs, n, sm_count() * occ * per_cta);
  int tiles = 0;
  for (int i = 0; i < n; ++i) {
    ds_status s = encode_job(prm.jobs[i], jobs[i], band);
    if (s != DS_OK) return s;
    prm.jobs[i].tile_begin = tiles;
    tiles += prm.jobs[i].tiles;
  }
  prm.n_jobs = n;
  prm.total_tiles = tiles;
  static std::atomic<unsigned> slot_counter{0};
  prm.sched_slot = (int)(slot_counter.fetch_add(1) % kSchedSlots);
  if (tiles == 0) return DS_OK;
  const int grid = std::min((tiles + per_cta - 1) / per_cta, sm_count() * occ);
  void* args[] = {&prm};
  cudaError_t e = cudaLaunchKernel(ki.fn, dim3(grid), dim3(ki.threads), args, (size_t)ki.smem, st);
  if (e != cudaSuccess) return cuda_fail(e, "k_fused_tma launch");
  count_launches(1);
  return DS_OK;
}

}  // namespace

int fast_max_jobs_per_launch() { return kMaxJobs; }

// One launch per class present (each kernel is specialised for its class),
// at most kMaxJobs descriptors per launch.
ds_status launch_fast(const FastJob* jobs, int n, cudaStream_t st) {
  std::vector<FastJob> group;
  for (int cls = 0; cls < kFcCount; ++cls) {
    group.clear();
    for (int i = 0; i < n; ++i)
      if (jobs[i].plan->fast_class == cls) group.push_back(jobs[i]);
    for (size_t i = 0; i < group.size(); i += kMaxJobs) {
      ds_status s = launch_chunk(group.data() + i, (int)std::min<size_t>(kMaxJobs, group.size() - i), st);
      if (s != DS_OK) return s;
    }
  }
  return DS_OK;
}

ds_status debug_check_plan(const ds_plan* pl, std::string& msg) {
  msg = check_plan(pl);
  return msg.empty() ? DS_OK : DS_ERR_ARG;
}

ds_status read_device_status(int* status) {
  int v = 0, zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_fast_status, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "reading the device status word");
  if (v != 0) {
    e = cudaMemcpyToSymbol(g_fast_status, &zero, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "clearing the device status word");
    // a kernel that gave up may have left its scheduling slot unreset
    static const unsigned zeros[kSchedSlots] = {};
    cudaMemcpyToSymbol(g_tile_next, zeros, sizeof(zeros));
    cudaMemcpyToSymbol(g_warps_done, zeros, sizeof(zeros));
  }
  *status = v;
  return DS_OK;
}

}  // namespace ds

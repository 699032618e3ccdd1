// rows.cuh -- the fused horizontal + vertical decimating FIR kernel of libds
// (the filter stage of the paper's downscaler, Sec. 3: a horizontal filter,
// then a vertical filter, packets of q pixels -> p outputs on each axis) and
// the host-side templates that go with each of its compiled classes.
//
// One persistent kernel per class runs the whole stage.  Work is cut into
// tiles: a strip of output columns x a band of output row blocks of one
// frame; tiles are handed to warps from a per-launch counter.  Each warp runs
// its tile by itself:
//
//   lane 0 issues TMA tensor loads (cp.async.bulk.tensor.3d) of SR input rows
//     of the strip plus its left and right halo into the warp's private ring
//     of NST shared-memory stages, completion tracked by one mbarrier each;
//   every input row goes through the horizontal pass in registers: each lane
//     reads one contiguous chunk of the row (NB packets of q pixels plus the
//     halo) with vector ld.shared and computes NB*p outputs per channel with
//     the phase taps (kernel parameters, i.e. constant-bank operands);
//   the results enter a sliding window of the last L filtered rows, also in
//     registers, so the intermediate never leaves the SM (the paper's
//     Sec. 3.B.3 removes host round trips between the two filters; this
//     removes the device-memory round trip as well);
//   each time q new rows have entered the window, the warp computes the p
//     output rows of one block from it and stores them.
//
// Per class: a warp may split into groups of 32/FPW lanes that filter the
// same strip and band of FPW frames (narrow frames), and the window may be
// filled by lead blocks run through the loop body instead of a separate
// unrolled prologue.  The row loop has no per-lane branch: lanes past the
// frame's edge compute on in-window data with their stores masked.
//
// Float data accumulate in FP32 with fmaf in tap order t = 0..K-1 from 0, the
// same sequence as the general kernels; uint8 data use exact integer dot
// products (dp2a) whose rounding is the same integer formula; so results are
// identical bit for bit whatever kernel, tile, tile shape or batch computes
// them.
//
// Every wait on an mbarrier is bounded (2e9 SM clock cycles, about 1 s).  On
// expiry the warp records DS_ERR_TIMEOUT in the device status word, waits
// (bounded) for the copies it issued and leaves.
//
// Each class is compiled in more than one tile shape (pipeline depth and
// the resident warps it is budgeted for); the rows_*.cu files instantiate
// the kernel for their classes and shapes and register them in a table that
// the host side (fused_fast.cu) looks up by class and shape.
#pragma once

#include <cudaTypedefs.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "pixel.cuh"

namespace ds {
namespace rows {

// Bounds-checking builds (-DDS_CHECK_BOUNDS): the kernel checks its own shared
// memory row reads, border writes, TMA copies and output rows against their
// buffers, and a failed check records what failed (kind, offset) and skips
// the access instead of making it.
#ifdef DS_CHECK_BOUNDS
constexpr bool kCheckBounds = true;
#else
constexpr bool kCheckBounds = false;
#endif

// Dynamic tile scheduling: launch slot s hands out tiles from tile_next[s];
// the last warp to finish puts both counters of its slot back to zero.  The
// host gives direct launches the slots below kGraphSlot0 and reuses a slot
// only once the launch that last used it has completed; launches captured
// into a CUDA graph own a slot at or above it until the graph is destroyed
// (replays of one graph are serialised by CUDA).
constexpr int kSchedSlots = 1024;
constexpr int kGraphSlot0 = 512;
constexpr int kStatusTimeout = 1;  // a bounded wait gave up, or a job of the wrong class
constexpr int kStatusBounds = 3;   // a bounds check failed (DS_CHECK_BOUNDS builds)

// Device-side state shared by every launch of the fused kernel on one GPU:
// the status word that ds_stream_check reads, the bounds-check record, and
// the tile-scheduling counters.  One static instance per device
// (fused_fast.cu); kernels get its address in their launch parameters.
struct DevState {
  int status;                  // 0 fine, kStatusTimeout, kStatusBounds
  int pad_;
  long long bounds_info[2];    // kind (1 row read, 2 border write, 3 output row, 4 copy), offset
  unsigned tile_next[kSchedSlots];
  unsigned warps_done[kSchedSlots];
};

__device__ __forceinline__ void bounds_fail(DevState* dev, int kind, long long offset) {
  if (atomicCAS(&dev->status, 0, kStatusBounds) == 0) {
    dev->bounds_info[0] = kind;
    dev->bounds_info[1] = offset;
  }
}

constexpr int kMaxJobs = 64;                  // job descriptors per launch
constexpr int kMaxTaps = 32;                  // p*K of the fast classes (per axis)
constexpr long long kWaitLimitCycles = 2000000000ll;  // ~1 s at the B300's 2.03 GHz
constexpr uint32_t kSuspendHintNs = 20000;             // a waiting thread sleeps up to 20 us per poll

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
__host__ __device__ constexpr int cgcd(int a, int b) { return b == 0 ? a : cgcd(b, a % b); }

// The tensor maps view every row as 8-byte elements, whatever the pixel type:
// a box row can then hold 256 x 8 bytes, so one box covers a strip's window
// (one TMA copy per stage and frame).  Rows are a multiple of 16 bytes on
// the fast path, and every strip's window starts on a 16-byte boundary.
constexpr int kTmaElem = 8;
constexpr CUtensorMapDataType kTmaType = CU_TENSOR_MAP_DATA_TYPE_UINT64;

// A fast-path class: data type, channels, horizontal ratio P/Q and taps K,
// vertical ratio PV/QV and taps KV (by default those of the horizontal axis),
// and the tile shape -- NB packets (of Q input pixels) per lane and row, so a
// strip is 32*NB packets wide (32/FPW*NB with frame groups); SR input rows per
// pipeline stage, NST stages per warp;
// FP: whether interior units run a second, check-free copy of the loop body
// (faster for some classes, slower where the larger code costs more than the
// checks, measured per class);
// FPW: frames per warp -- the warp's lanes split into FPW groups of 32/FPW,
// each filtering the same strip and band of its own frame (for narrow frames,
// whose width is a poor multiple of 32 lanes' packets);
// PRO: the window prologue runs through the loop body as lead blocks whose
// outputs are dropped (less code, a few more rows filtered per tile) instead
// of a separate unrolled copy of the row code;
// WPC warps per CTA, with registers budgeted for MINB resident CTAs per SM.
template <int ID, typename T_, int C_, int P_, int Q_, int K_, int NB_, int SR_, int NST_, bool FP_, int PV_, int QV_,
          int KV_, int FPW_, bool PRO_, int WPC_, int MINB_>
struct Cls {
  using T = T_;
  static constexpr int id = ID, C = C_, P = P_, Q = Q_, K = K_, NB = NB_;
  static constexpr int PV = PV_, QV = QV_, KV = KV_;
  static constexpr bool FASTPATH = FP_;             // check-free copy of the body for interior units
  // warps (independent tile pipelines) per CTA, and the resident CTAs per SM
  // the registers are budgeted for (__launch_bounds__)
  static constexpr int WPC = WPC_, MINB = MINB_;
  static constexpr int SRR = SR_;                   // input rows per stage
  static constexpr int NST = NST_;                  // stages per warp
  static constexpr int SZ = (int)sizeof(T);
  static constexpr int FPW = FPW_;                  // frames per warp
  static constexpr int LPS = 32 / FPW_;             // lanes per frame (a strip's lanes)
  // horizontal axis: the strip, its halo columns and the lane chunks
  static constexpr int BMIN = phase_b(P, Q, K, 0);
  static constexpr int BMAX = phase_b(P, Q, K, P - 1);
  static constexpr int LH = -BMIN;                  // halo pixels left of a block
  static constexpr int RH = BMAX + K - Q;           // halo pixels right of a block
  static constexpr int E = NB * Q * C;              // elements per lane and row
  static constexpr int EB = E * SZ;
  static constexpr int HLB = rup(LH * C * SZ, 16);  // left halo bytes in the window (TMA x alignment)
  static constexpr int RHB = rup(RH * C * SZ, 16);
  static constexpr int SBLK = LPS * NB;             // packets (blocks) per strip
  static constexpr int SPX = SBLK * Q;              // input pixels per strip
  static constexpr int WINB = HLB + SPX * C * SZ + RHB;
  static constexpr int NBOX = cdiv(WINB / kTmaElem, 256);
  static constexpr int BOXB = rup(cdiv(WINB, NBOX), 16);
  static constexpr int BOXE = BOXB / kTmaElem;         // box width in TMA elements
  static constexpr int BOXSTR = rup(SR_ * BOXB, 128);  // each box lands 128-B aligned
  static constexpr int FSTR = NBOX * BOXSTR;          // one frame's window in a stage
  static constexpr int RSTAGE = FPW_ * FSTR;
  static constexpr int RTX = NBOX * SR_ * BOXB;        // TMA bytes per stage and frame
  static constexpr int WARP_BYTES = NST_ * RSTAGE;
  static constexpr int NX = (LH + NB * Q + RH) * C;    // elements one lane reads per row
  static constexpr int VB = (EB % 16 == 0) ? 16 : ((EB % 8 == 0) ? 8 : 4);
  static constexpr int NV = EB / VB;
  static constexpr int HB = cdiv(LH * C * SZ, VB);     // halo vectors a lane loads before its chunk
  static constexpr int HA = cdiv(RH * C * SZ, VB);     // ... and after it
  static constexpr int NVT = HB + NV + HA;             // vectors per lane and row
  static constexpr int NWT = NVT * VB / 4;             // words per lane and row
  static constexpr int NOUT = NB * P * C;              // H outputs per lane and row
  // Narrow tail strips (one-channel classes with frame pairs): a frame's last
  // strip, when it has at most NPN packets, is filtered four frames per warp
  // in groups of 8 lanes.  Its window (WN bytes: NPN packets and the halo) is
  // half a box row, so one TMA box of (WN bytes, 2 frames, SR rows) puts two
  // frames' windows side by side at the usual row pitch: four frames fill
  // exactly the stage of a frame pair, with the same bytes per stage.
  static constexpr int NPN = (BOXB / 2 - HLB - RHB) / (Q * C * SZ);
  static constexpr int WN = HLB + NPN * Q * C * SZ + RHB;
  static constexpr bool NARROW =
      FPW_ == 2 && C_ == 1 && NB_ == 1 && NBOX == 1 && NPN >= 1 && NPN <= 8 && 2 * WN == BOXB && WN % 16 == 0;
  // vertical axis: the row stream and the register window
  static constexpr int BMINV = phase_b(PV, QV, KV, 0);
  static constexpr int BMAXV = phase_b(PV, QV, KV, PV - 1);
  static constexpr int LV = BMAXV - BMINV + KV;     // pattern length (rows per block window)
  static constexpr int LHV = -BMINV;                // halo rows above a block
  // The stream of a tile is cut so that the window prologue (the first LV-QV
  // pattern rows) fills whole stages, EXTRA rows being loaded before the first
  // pattern row; after it, every group of U = lcm(SR, QV) rows is USTG stages
  // and UBLK block steps, so each row's stage offset and window slot are
  // compile-time constants.
  static constexpr int PRE = LV - QV;
  static constexpr int NPS = cdiv(PRE, SR_);
  static constexpr int EXTRA = NPS * SR_ - PRE;
  static constexpr int U = SR_ / cgcd(SR_, QV) * QV;
  static constexpr int USTG = U / SR_;
  static constexpr int UBLK = U / QV;
  // With PRO, the stream instead starts VBLK blocks early (whole units): the
  // lead blocks fill the window, their outputs are not computed.
  static constexpr bool PRO = PRO_;
  static constexpr int VBLK = PRO_ ? rup(cdiv(PRE, QV), UBLK) : 0;  // lead blocks
  static constexpr int STG0 = PRO_ ? 0 : NPS;                         // first stage of unit 0
  static constexpr int YOFF = PRO_ ? PRE - VBLK * QV : -EXTRA;        // stream start - first pattern row
  // Stage 0 of a tile is loaded S0SHIFT rows later than the stream grid puts
  // it: it starts at the first pattern row, so the EXTRA alignment rows are
  // not read from memory (its last EXTRA rows repeat the first rows of
  // stage 1, fetched at the same time and served from L2).
  static constexpr int S0SHIFT = PRO_ ? 0 : EXTRA;
  __host__ __device__ static constexpr int b(int j) { return phase_b(P, Q, K, j); }
  __host__ __device__ static constexpr int bv(int j) { return phase_b(PV, QV, KV, j); }
  static_assert(EB % 4 == 0, "a lane's chunk must be whole words");
  static_assert(HB * VB <= HLB && HA * VB <= RHB, "halo vectors must lie in the loaded window");
  static_assert(BOXE <= 256 && BOXB % 16 == 0, "TMA box limits");
  static_assert((SPX * C * SZ) % 16 == 0 && HLB % 16 == 0, "strip windows start on 16-byte boundaries");
  static_assert(NBOX * BOXB >= WINB, "boxes must cover the window");
  static_assert(NBOX == 1 && BOXB == WINB, "one box per window row: the row copies of modular tilers rely on it");
  static_assert(P * K <= kMaxTaps && PV * KV <= kMaxTaps, "tap table size");
  static_assert(BOXB % VB == 0 && HLB % VB == 0, "vector loads must not straddle boxes");
  static_assert(PRE > LHV, "the window prologue must reach frame row 0");
  static_assert(LV * (SZ == 1 ? (NOUT + 3) / 4 : NOUT) <= 48, "register window too large");
  static_assert(U <= 16, "iteration unit too long to unroll");
  static_assert(FPW_ == 1 || FPW_ == 2 || FPW_ == 4, "frames per warp");
  static_assert(NX == (LH + NB * Q + RH) * C, "lane window (float row math)");
};

// ---------------------------------------------------------------------------
// launch parameters
// ---------------------------------------------------------------------------
struct JobDesc {
  CUtensorMap tmap;        // 3-D map: (W*C elements, H rows, n_frames); clamped tilers
  void* out;
  long long out_frame;     // elements per output frame
  int H, W, OH, OW;
  int nframes, cls, strips, chunks;
  int rbc, tile_begin, tiles, out_vec;
  const uint8_t* in;       // the frames, for the row copies of modular tilers
  int wrap;                // 1: modular tilers (launched on the WRAP kernels)
  int nar;                 // 1: a narrow tail strip (four frames per warp; tmap is (x, frame, row))
  int strip0;              // the job's first strip of the frame
};
static_assert(sizeof(JobDesc) == 256 && alignof(JobDesc) == 128, "job descriptor layout");

// The taps of one class.  tap2h / tap2v: the Q14 taps of a uint8 class as
// pairs of int16 for dp2a, [window-start parity][phase][pair]: for parity a,
// pair i holds taps 2i - a (low half) and 2i + 1 - a (high half), zero
// outside 0..K-1, so a window that starts on an odd slot is read from the
// even slot before it.
constexpr int kMaxPairs = 5;  // (K + 1) / 2 + 1 for K <= 8
constexpr int kMaxPhases = 4;

struct ClassTaps {
  float taps[kMaxTaps];   // horizontal FP32 taps, or Q14 taps as floats for uint8
  float tapsv[kMaxTaps];  // the same for the vertical axis
  uint32_t tap2h[2][kMaxPhases][kMaxPairs];
  uint32_t tap2v[2][kMaxPhases][kMaxPairs];
};

// Launch parameters (a __grid_constant__ kernel argument) with room for MAXJ
// job descriptors: a small size for single jobs keeps the argument -- copied
// by the driver at every launch -- short.
template <int MAXJ>
struct FastParams {
  JobDesc jobs[MAXJ];
  ClassTaps t;
  int n_jobs;
  int total_tiles;
  int sched_slot;                  // dynamic scheduling slot
  DevState* dev;                   // status word and scheduling counters of this GPU
};
constexpr int kFewJobs = 2;        // one job, or one job split for the launch tail

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
// Count `bytes` of the current phase's expected transactions as done (no copy).
__device__ __forceinline__ void mbar_complete_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.complete_tx.shared::cta.b64 [%0], %1;" ::"r"(saddr32(bar)), "r"(bytes) : "memory");
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
// Wait for the phase of `parity` to complete; false after `limit` SM clock
// cycles (about a second by default), counted from the 4th failed poll.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit = kWaitLimitCycles) {
#pragma unroll 1
  for (int it = 0; it < 4; ++it)
    if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 3u) == 0 && clock64() - t0 > limit) return false;
  }
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(saddr32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(saddr32(bar))
      : "memory");
}
// One contiguous global -> shared copy (16-byte aligned addresses, a size that
// is a multiple of 16), completing `bytes` on the mbarrier.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          saddr32(dst)),
      "l"(src), "r"(bytes), "r"(saddr32(bar))
      : "memory");
}

// ---------------------------------------------------------------------------
// tiles
// ---------------------------------------------------------------------------
struct Tile {
  int job, frame, strip, chunk;  // frame: the group of the job's frames FPW * frame .. + FPW - 1
};

template <class PR>
__host__ __device__ __forceinline__ Tile decode_tile(const PR& prm, int t) {
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

// Offset of byte `byte` of window row 0 inside a stage: boxes are stored one
// after the other, each as SR rows of BOXB bytes (BOXSTR bytes apart), so row
// r of the window starts r * BOXB bytes further in every box.
template <class Cl>
__host__ __device__ __forceinline__ int win_off(int byte) {
  const int box = byte / Cl::BOXB;
  return byte + box * (Cl::BOXSTR - Cl::BOXB);
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


// Per-lane shared-memory offsets (row 0 of a stage) of the vectors the H
// pass loads: HB halo vectors, the lane's own NV vectors, HA halo vectors,
// consecutive in the window.  They depend only on the lane: computed once.
template <class Cl>
struct Offs {
  int v[Cl::NVT];
};

template <class Cl>
__device__ __forceinline__ Offs<Cl> thread_offs(int lane) {
  Offs<Cl> o;
  const int sub = lane / Cl::LPS, li = lane % Cl::LPS;  // the lane's frame in the group, its lane in the strip
  const int first = Cl::HLB + li * Cl::EB - Cl::HB * Cl::VB;
#pragma unroll
  for (int v = 0; v < Cl::NVT; ++v) o.v[v] = sub * Cl::FSTR + win_off<Cl>(first + v * Cl::VB);
  return o;
}

// Narrow tail strips: lane group g = lane / 8 holds frame g of the tile; box
// g / 2 of the stage holds frames 2(g/2) and 2(g/2) + 1 side by side, WN
// bytes each, in rows of BOXB bytes.  Offset of byte `byte` of the window
// row 0 of group g.
template <class Cl>
__host__ __device__ __forceinline__ int narrow_base(int g) {
  return (g >> 1) * Cl::FSTR + (g & 1) * Cl::WN;
}

// The lane's vector offsets in a narrow tail strip.  Lanes past the window's
// NPN packets (never active: their packets lie past the frame's last one)
// read the last packet's vectors.
template <class Cl>
__device__ __forceinline__ Offs<Cl> thread_offs_narrow(int lane) {
  Offs<Cl> o;
  const int g = lane >> 3, li = min(lane & 7, Cl::NPN - 1);
  const int first = narrow_base<Cl>(g) + Cl::HLB + li * Cl::EB - Cl::HB * Cl::VB;
#pragma unroll
  for (int v = 0; v < Cl::NVT; ++v) o.v[v] = first + v * Cl::VB;
  return o;
}

// Load the lane's vectors of one window row into words w[0..NWT).
template <class Cl>
__device__ __forceinline__ void load_row(const uint8_t* rowbase, const Offs<Cl>& o, uint32_t* w) {
  constexpr int WPV = Cl::VB / 4;
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

// Clamp-to-edge in the loaded window: the columns of a warp's read range that
// lie outside the frame (TMA filled them with zeros) get the value of the
// first / last column of their row.  Pixel ranges [l_lo, 0) and [r_lo, r_hi).
struct EdgeFix {
  int l_lo, nl, r_lo, nr;  // first pixel and element counts, left and right
};

template <class Cl>
__host__ __device__ __forceinline__ EdgeFix edge_fix(int strip, int W, int OW) {
  const int seg0 = strip * Cl::SPX - Cl::LH;             // first pixel the warp reads
  const int seg1 = (strip + 1) * Cl::SPX + Cl::RH;       // one past the last
  EdgeFix f;
  f.l_lo = seg0;
  f.nl = seg0 < 0 ? ((seg1 < 0 ? seg1 : 0) - seg0) * Cl::C : 0;
  f.r_lo = W > seg0 ? W : seg0;
  // active lanes (those with outputs) read no further than the chunk of the
  // last of them and its right halo
  const int npk = (OW + Cl::P - 1) / Cl::P;  // packets with outputs
  const int lim = ((npk - 1) / Cl::NB + 1) * Cl::NB * Cl::Q + Cl::RH;
  const int r_hi = seg1 < lim ? seg1 : lim;
  f.nr = r_hi > f.r_lo ? (r_hi - f.r_lo) * Cl::C : 0;
  return f;
}

// Element e2 of the fix (frames of the group one after the other): its source
// and destination offsets in row 0 of a stage.
template <class Cl>
__device__ __forceinline__ void edge_elem(const EdgeFix& f, int e2, int W, int xw, int& src, int& dst) {
  const int n = f.nl + f.nr;  // elements to fix per row of a frame window
  int sub = 0;                // e2 / n, for at most 4 frames
  if constexpr (Cl::FPW > 1) sub = (e2 >= n) + (Cl::FPW > 2 ? (e2 >= 2 * n) + (e2 >= 3 * n) : 0);
  const int e = e2 - sub * n;
  const bool left = e < f.nl;
  const int k = left ? e : e - f.nl;
  const int px = (left ? f.l_lo : f.r_lo) + k / Cl::C, c = k % Cl::C;
  src = sub * Cl::FSTR + win_off<Cl>(((left ? 0 : W - 1) * Cl::C + c - xw) * Cl::SZ);
  dst = sub * Cl::FSTR + win_off<Cl>((px * Cl::C + c - xw) * Cl::SZ);
}

// The same for a narrow tail strip (four frames, at most one element per lane).
template <class Cl>
__device__ __forceinline__ void edge_elem_narrow(const EdgeFix& f, int e2, int W, int xw, int& src, int& dst) {
  const int n = f.nl + f.nr;
  const int g = e2 / n, e = e2 - g * n;
  const bool left = e < f.nl;
  const int k = left ? e : e - f.nl;
  const int px = (left ? f.l_lo : f.r_lo) + k / Cl::C, c = k % Cl::C;
  src = narrow_base<Cl>(g) + ((left ? 0 : W - 1) * Cl::C + c - xw) * Cl::SZ;
  dst = narrow_base<Cl>(g) + (px * Cl::C + c - xw) * Cl::SZ;
}

// One element's copy in all SR rows of a stage.
template <class Cl>
__device__ __forceinline__ void edge_copy(uint8_t* stagebase, int src, int dst, DevState* dev) {
  using T = typename Cl::T;
#pragma unroll
  for (int r = 0; r < Cl::SRR; ++r) {
    if constexpr (kCheckBounds) {  // both elements inside this stage
      const int lo = r * Cl::BOXB + (src < dst ? src : dst), hi = r * Cl::BOXB + (src > dst ? src : dst);
      if (lo < 0 || hi + Cl::SZ > Cl::RSTAGE) {
        bounds_fail(dev, 2, lo < 0 ? lo : hi);
        continue;
      }
    }
    *reinterpret_cast<T*>(stagebase + r * Cl::BOXB + dst) = *reinterpret_cast<const T*>(stagebase + r * Cl::BOXB + src);
  }
}

// Applied to all SR rows of a stage at once.  When the fix has at most one
// element per lane, each lane's offsets come from the tile (`one`: src, dst;
// dst < 0 for a lane without an element); otherwise they are worked out
// here, once for the stage (one copy of this code per stage wait, not per row).
template <class Cl>
__device__ __forceinline__ void apply_edge_fix(uint8_t* stagebase, const EdgeFix& f, int lane, int W, int xw,
                                               bool one, int src1, int dst1, DevState* dev) {
  if (one) {
    if (dst1 >= 0) edge_copy<Cl>(stagebase, src1, dst1, dev);
  } else {
    for (int e2 = lane; e2 < Cl::FPW * (f.nl + f.nr); e2 += 32) {
      int src, dst;
      edge_elem<Cl>(f, e2, W, xw, src, dst);
      edge_copy<Cl>(stagebase, src, dst, dev);
    }
  }
  // these generic-proxy writes must land before the TMA refills the stage
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();
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

// ---------------------------------------------------------------------------
// row-streaming kernel: one self-contained pipeline per warp
// ---------------------------------------------------------------------------
// Rows above / below the frame are never loaded: their window slots take a
// copy of the first / last filtered row (clamp-to-edge); columns outside the
// frame are fixed up in shared memory.  Warps synchronise with nothing but
// their own TMA completions.

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
  template <class PR>
  __device__ static __forceinline__ void h(const uint32_t* w, const PR& prm, Row& r) {
    hcompute<Cl>(w, prm.t.taps, r.v);
  }
  __device__ static __forceinline__ void copy(Row& d, const Row& s) {
#pragma unroll
    for (int k = 0; k < N; ++k) d.v[k] = s.v[k];
  }
  // the PV output rows of block rr from the window (CHECK: rows past OH are
  // skipped; without it the caller knows they are all inside); `words`: see
  // the uint8 form
  template <bool CHECK, class PR>
  __device__ static __forceinline__ void v(const Row (&win)[Cl::LV], const PR& prm, T* obase, long long rowe,
                                           int rr, int OH, int n_valid, bool /*words*/) {
    const float* taps = prm.t.tapsv;
#pragma unroll
    for (int jv = 0; jv < Cl::PV; ++jv) {
      const int oy = rr * Cl::PV + jv;
      if (!CHECK || oy < OH) {
        float acc[N];
#pragma unroll
        for (int k = 0; k < N; ++k) acc[k] = 0.0f;
#pragma unroll
        for (int tt = 0; tt < Cl::KV; ++tt) {
          const float wt = taps[jv * Cl::KV + tt];
#pragma unroll
          for (int k = 0; k < N; ++k) acc[k] = fmaf(wt, win[Cl::bv(jv) - Cl::BMINV + tt].v[k], acc[k]);
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

// Bytes p0..p3 of the word array w as one word, byte k = byte pk; p0 is the
// lowest position and p3 the highest, and the words they span (at most four)
// are all inside the array.
// The positions are compile-time constants after unrolling, so the selectors
// fold and only the words that hold one of the bytes are read.
__device__ __forceinline__ uint32_t gather4(const uint32_t* w, int p0, int p1, int p2, int p3) {
  if ((p0 & 3) == 0 && p1 == p0 + 1 && p2 == p0 + 2 && p3 == p0 + 3) return w[p0 >> 2];  // a whole word
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

// (acc + 2^13) >> 14 has been taken by starting acc at 2^13: a floor shift.
// The clamp to [0, 255] happens when the values are packed.
__device__ __forceinline__ int u8_round(int acc) { return acc >> 14; }

// Four shifted sums as the bytes of one word (v0 lowest), each saturated to
// [0, 255]: two saturating pack conversions (each converts two s32 values to
// u8 and places them below the low half of its third operand).
__device__ __forceinline__ uint32_t pack4(int v0, int v1, int v2, int v3) {
  uint32_t hi, d;
  asm("cvt.pack.sat.u8.s32.b32 %0, %1, %2, %3;" : "=r"(hi) : "r"(v3), "r"(v2), "r"(0u));
  asm("cvt.pack.sat.u8.s32.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(v1), "r"(v0), "r"(hi));
  return d;
}

// Store the first n_valid (<= N) of a lane's N output bytes (packed 4 to a
// word in w).  Every lane of a warp takes the same path: wide stores when N
// is a multiple of 4 (so all lanes share the row's alignment), byte stores
// otherwise or at a frame's right edge.
template <int N>
__device__ __forceinline__ void store_bytes(uint8_t* o, const uint32_t* w, int n_valid) {
  if constexpr (N % 4 == 0) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(o);
    if (n_valid >= N) {
      if constexpr (N % 16 == 0) {
        if ((a & 15) == 0) {
#pragma unroll
          for (int i = 0; i < N / 16; ++i)
            reinterpret_cast<uint4*>(o)[i] = make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
          return;
        }
      }
      if constexpr (N % 8 == 0) {
        if ((a & 7) == 0) {
#pragma unroll
          for (int i = 0; i < N / 8; ++i) reinterpret_cast<uint2*>(o)[i] = make_uint2(w[2 * i], w[2 * i + 1]);
          return;
        }
      }
      if ((a & 3) == 0) {
#pragma unroll
        for (int i = 0; i < N / 4; ++i) reinterpret_cast<uint32_t*>(o)[i] = w[i];
        return;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < N; ++i)
    if (i < n_valid) o[i] = (uint8_t)(w[i >> 2] >> (8 * (i & 3)));
}

// Word stores of runs whose length N is not a multiple of 4, for a warp whose
// lanes' runs follow one another in a row that starts on a word boundary, with
// each strip starting and ending on one: lane runs then start a = 0..3 bytes
// into a word.  A lane shifts its bytes (zero above byte N-1) to their place
// in the words they span and stores every word that starts inside its run,
// the word across its end completed with the first bytes of the next lane's
// run (a shuffle; that lane is active whenever the run ends inside a word,
// since a row's end is on a word boundary).  A lane past the frame's edge
// stores nothing.  Every lane of the warp must call this (the shuffle).
template <int N>
__device__ __forceinline__ void store_words(uint8_t* o, const uint32_t* w, int n_valid) {
  static_assert(N % 4 != 0 && N >= 3, "runs of 3 or more bytes that are not whole words");
  constexpr int NW = (N + 3) / 4;      // words of the run in w
  constexpr int NX = (N + 3 + 3) / 4;  // words a run spans at offsets 0..3
  const int a = (int)(reinterpret_cast<uintptr_t>(o) & 3u), sh = 8 * a;
  uint32_t x[NX];
  x[0] = w[0] << sh;
#pragma unroll
  for (int k = 1; k < NX; ++k) x[k] = __funnelshift_l(w[k - 1], k < NW ? w[k] : 0u, sh);
  const uint32_t next = __shfl_down_sync(0xffffffffu, x[0], 1);
  const uint32_t carry = ((a + N) & 3) ? next : 0u;
  const int end = a + (n_valid < N ? n_valid : N);  // n_valid < N: the row's end, a word boundary
  uint32_t* const base = reinterpret_cast<uint32_t*>(o - a);
#pragma unroll
  for (int k = 0; k < NX; ++k)
    if ((k > 0 || a == 0) && 4 * k < end) base[k] = (4 * k + 4 > a + N) ? (x[k] | carry) : x[k];
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
  static constexpr int C = Cl::C, Q = Cl::Q, P = Cl::P, K = Cl::K, BMIN = Cl::BMIN;  // horizontal
  static constexpr int PV = Cl::PV, KV = Cl::KV, LV = Cl::LV, BMINV = Cl::BMINV;      // vertical
  static constexpr int N = Cl::NOUT;
  static constexpr int NW = (N + 3) / 4;
  static constexpr int NXP = Cl::LH + Cl::NB * Q + Cl::RH;  // window pixels of a lane
  static constexpr int NPR = (LV + 2) / 2;                  // window row pairs (+1 slot of pad)
  static_assert(Cl::HB * Cl::VB >= Cl::LH * C, "pixel slot 0 must be a loaded byte");
  static_assert(Cl::HB * Cl::VB - Cl::LH * C + NXP * C <= Cl::NVT * Cl::VB, "gathered bytes must be loaded");
  static_assert(P <= kMaxPhases && PV <= kMaxPhases &&
                    (K + 2) / 2 <= kMaxPairs && (KV + 2) / 2 <= kMaxPairs, "tap pair table");
  struct Row {
    uint32_t w[NW];
  };
  __device__ static __forceinline__ void copy(Row& d, const Row& s) {
#pragma unroll
    for (int k = 0; k < NW; ++k) d.w[k] = s.w[k];
  }
  template <class PR>
  __device__ static __forceinline__ uint32_t tp(const PR& prm, int par, int j, int i) {
    return prm.t.tap2h[par][j][i];
  }
  template <class PR>
  __device__ static __forceinline__ uint32_t tpv(const PR& prm, int par, int j, int i) {
    return prm.t.tap2v[par][j][i];
  }
  template <class PR>
  __device__ static __forceinline__ void h(const uint32_t* w, const PR& prm, Row& r) {
    constexpr int first = Cl::HB * Cl::VB - Cl::LH * C;  // byte of pixel slot 0, channel 0
    auto pos = [&](int slot, int c) { return first + (slot < NXP ? slot : NXP - 1) * C + c; };  // pads: any byte
    int v[N];
    if constexpr (C == 3) {
      // Pixel pair m (slots 2m, 2m+1): one word holds its R pair (low half)
      // and G pair (high half) -- five consecutive bytes, so one byte_perm --
      // and another its B pair (low half).
      constexpr int NPW = (NXP + 2) / 2;
      uint32_t rg[NPW], bb[NPW];
#pragma unroll
      for (int m = 0; m < NPW; ++m) {
        rg[m] = gather4(w, pos(2 * m, 0), pos(2 * m + 1, 0), pos(2 * m, 1), pos(2 * m + 1, 1));
        bb[m] = gather4(w, pos(2 * m, 2), pos(2 * m + 1, 2), pos(2 * m + 1, 2), pos(2 * m + 1, 2));
      }
#pragma unroll
      for (int n = 0; n < Cl::NB; ++n)
#pragma unroll
        for (int j = 0; j < P; ++j) {
          const int s0 = n * Q + Cl::b(j) - BMIN;  // first window slot of the output
          const int par = s0 & 1, pr0 = (s0 - par) / 2, npair = (K + par + 1) / 2;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            int acc = 8192;
#pragma unroll
            for (int i = 0; i < npair; ++i) {
              const int m = pr0 + i;
              acc = (c == 1) ? dp2a<1>(tp(prm, par, j, i), rg[m], acc)
                             : dp2a<0>(tp(prm, par, j, i), c == 0 ? rg[m] : bb[m], acc);
            }
            v[(n * P + j) * C + c] = u8_round(acc);
          }
        }
    } else {
      // one channel word per 4 consecutive pixel slots (pairs 2k, 2k+1).  For
      // one channel the slots start D pixels left of the lane's window, so
      // that slot 0 is the first byte of a loaded word and every channel
      // word is a loaded word as it is (no byte_perm); the D extra slots
      // only ever meet zero taps.
      constexpr int D = (C == 1) ? (first & 3) : 0;
      constexpr int first1 = first - D, loaded = Cl::NVT * Cl::VB;
      auto pos1 = [&](int slot, int c) {
        const int p = C == 1 ? first1 + slot : first + (slot < NXP ? slot : NXP - 1) * C + c;
        return p < loaded ? p : loaded - 1;  // past the loaded bytes: pads, any byte
      };
      constexpr int NCW = (NXP + D + 1 + 3) / 4;  // channel words (+1: odd-start pad)
      uint32_t cw[C][NCW];
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int k = 0; k < NCW; ++k)
          cw[c][k] = gather4(w, pos1(4 * k, c), pos1(4 * k + 1, c), pos1(4 * k + 2, c), pos1(4 * k + 3, c));
#pragma unroll
      for (int n = 0; n < Cl::NB; ++n)
#pragma unroll
        for (int j = 0; j < P; ++j) {
          const int s0 = n * Q + Cl::b(j) - BMIN + D;  // first window slot of the output
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
    }
#pragma unroll
    for (int k = 0; k < NW; ++k) {
      const int e = 4 * k;
      r.w[k] = pack4(v[e], e + 1 < N ? v[e + 1] : 0, e + 2 < N ? v[e + 2] : 0, e + 3 < N ? v[e + 3] : 0);
    }
  }
  // Runs whose length is not a whole number of words are stored as words
  // (store_words) when `words` is set (the same for every lane of the warp),
  // else as bytes.  Not for runs of 3 bytes: there the shifts and the
  // shuffle cost as much as the byte stores they replace (measured slower).
  static constexpr bool kWordRuns = N % 4 != 0 && N >= 6 && (Cl::SBLK * P * C) % 4 == 0;
  // V windows that start on an odd row read odd-aligned row pairs (rows 2m+1
  // and 2m+2) with the even-parity tap pairs: KV/2 dp2a per output instead of
  // KV/2 + 1, for two more byte permutes per pair.  Three-channel classes,
  // where dp2a is the busier pipe, except the 3/8 vertical axis, where it
  // measured slower (CIF RGB -0.7 %, RGB 2/3 -2.2 %, RGB 3/8 +0.5 %).
  static constexpr bool VODD = C == 3 && KV % 2 == 0 && !(PV == 3 && Cl::QV == 8);
  template <bool CHECK, class PR>
  __device__ static __forceinline__ void v(const Row (&win)[LV], const PR& prm, T* obase, long long rowe,
                                           int rr, int OH, int n_valid, bool words) {
    // one word column g (4 output columns) at a time: row-pair words
    // pl = bytes 0,1 of rows 2m and 2m+1 interleaved, ph = bytes 2,3
    uint32_t o[PV][NW];
#pragma unroll
    for (int g = 0; g < NW; ++g) {
      uint32_t pl[NPR], ph[NPR], ql[NPR], qh[NPR];
#pragma unroll
      for (int m = 0; m < NPR; ++m) {
        const int r0 = 2 * m < LV ? 2 * m : LV - 1, r1 = 2 * m + 1 < LV ? 2 * m + 1 : LV - 1;
        pl[m] = __byte_perm(win[r0].w[g], win[r1].w[g], 0x5140u);
        ph[m] = __byte_perm(win[r0].w[g], win[r1].w[g], 0x7362u);
        if constexpr (VODD) {  // odd-aligned pairs, the same interleave
          const int q0 = 2 * m + 1 < LV ? 2 * m + 1 : LV - 1, q1 = 2 * m + 2 < LV ? 2 * m + 2 : LV - 1;
          ql[m] = __byte_perm(win[q0].w[g], win[q1].w[g], 0x5140u);
          qh[m] = __byte_perm(win[q0].w[g], win[q1].w[g], 0x7362u);
        }
      }
#pragma unroll
      for (int jv = 0; jv < PV; ++jv) {
        const int s0 = Cl::bv(jv) - BMINV;
        const int par = s0 & 1;
        const bool odd = VODD && par;  // an odd start read from odd-aligned pairs
        const int pr0 = odd ? (s0 - 1) / 2 : (s0 - par) / 2, npair = odd ? KV / 2 : (KV + par + 1) / 2;
        const int tpar = odd ? 0 : par;
        int v[4] = {0, 0, 0, 0};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (4 * g + e >= N) continue;  // past the lane's outputs: never stored, not computed
          int acc = 8192;
#pragma unroll
          for (int i = 0; i < npair; ++i) {
            const uint32_t word = odd ? ((e & 2) ? qh[pr0 + i] : ql[pr0 + i]) : ((e & 2) ? ph[pr0 + i] : pl[pr0 + i]);
            acc = (e & 1) ? dp2a<1>(tpv(prm, tpar, jv, i), word, acc) : dp2a<0>(tpv(prm, tpar, jv, i), word, acc);
          }
          v[e] = u8_round(acc);
        }
        o[jv][g] = pack4(v[0], v[1], v[2], v[3]);
      }
    }
#pragma unroll
    for (int jv = 0; jv < PV; ++jv) {
      const int oy = rr * PV + jv;
      if (!CHECK || oy < OH) {
        if constexpr (kWordRuns) {
          if (words) {
            store_words<N>(obase + (long long)oy * rowe, o[jv], n_valid);
            continue;
          }
        }
        store_bytes<N>(obase + (long long)oy * rowe, o[jv], n_valid);
      }
    }
  }
};

// WRAP: modular tilers (every job of the launch has them), else clamp-to-edge.
template <class Cl, int MAXJ, bool WRAP>
__global__ void __launch_bounds__(Cl::WPC * 32, Cl::MINB) k_rows(const __grid_constant__ FastParams<MAXJ> prm) {
  using T = typename Cl::T;
  using RM = RowMath<Cl>;
  using Row = typename RM::Row;
  // L, Q, P: the vertical axis (row stream, window, output rows); the
  // horizontal one is Cl::P / Cl::Q / Cl::K
  constexpr int L = Cl::LV, Q = Cl::QV, P = Cl::PV, SR = Cl::SRR, NST = Cl::NST, WPC = Cl::WPC;
  extern __shared__ uint8_t smem_raw[];
  // 128-byte aligned start, derived from the __shared__ array by an offset
  // (not through an integer cast) so that every access stays a shared-memory
  // access (ld.shared / st.shared), not a generic one
  uint8_t* smem = smem_raw + ((128u - (saddr32(smem_raw) & 127u)) & 127u);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* const ring = smem + warp * Cl::WARP_BYTES;
  uint64_t* const full = reinterpret_cast<uint64_t*>(smem + WPC * Cl::WARP_BYTES) + warp * NST;
  if constexpr (kCheckBounds) {
    // poison the ring (all-ones bytes: NaN for float data) so that a read of
    // staging memory before its copy lands shows up in the results
    for (int i = lane; i < Cl::WARP_BYTES / 4; i += 32) reinterpret_cast<uint32_t*>(ring)[i] = 0xffffffffu;
    __syncwarp();
  }
  if (lane == 0) {
    for (int s = 0; s < NST; ++s) mbar_init(&full[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncwarp();
  const unsigned nwarps = gridDim.x * WPC;
  unsigned* const next = &prm.dev->tile_next[prm.sched_slot];
  // the first tile of every warp is its warp index (so the launch does not
  // start with every warp hitting one counter); later ones come from the
  // counter, offset by the number of warps
  auto next_tile = [&]() -> int {
    unsigned t = 0;
    if (lane == 0) t = nwarps + atomicAdd(next, 1u);
    return (int)__shfl_sync(0xffffffffu, t, 0);
  };
  uint32_t g = 0;       // this warp's stage counter over all its tiles (mbarrier phases)
  uint32_t issued = 0;  // one past the last stage issued
  bool ok = true;
  for (int t = (int)(blockIdx.x * WPC + warp); ok && t < prm.total_tiles; t = next_tile()) {
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
    const int ys = rb0 * Q + Cl::BMINV;  // first pattern row; < 0 only for the top band (then == BMINV)
    const int nst = Cl::STG0 + ((nblk + Cl::VBLK) * Q + SR - 1) / SR;
    const int ystream = ys + Cl::YOFF;  // frame row of stage 0's first row
    // a narrow tail strip (its own job): four frames per warp in 8-lane
    // groups, the windows of frames 2k and 2k + 1 side by side in box k
    const bool nar = !WRAP && Cl::NARROW && jd.nar != 0;
    const int fpw = nar ? 4 : Cl::FPW, lps = nar ? 8 : Cl::LPS;
    const int strip = Cl::NARROW ? jd.strip0 + tl.strip : tl.strip;  // the strip of the frame
    const Offs<Cl> of = nar ? thread_offs_narrow<Cl>(lane) : thread_offs<Cl>(lane);
    const int xw = strip * Cl::SPX * Cl::C - Cl::HLB / Cl::SZ;  // window start, in elements
    const int xt = xw * Cl::SZ / kTmaElem;                          // ... in TMA elements (exact)
    const EdgeFix fix = edge_fix<Cl>(strip, jd.W, jd.OW);
    constexpr bool wrap = WRAP;
    const bool fixing = !wrap && fix.nl + fix.nr > 0;
    // a fix of at most one element per lane: the lane's offsets, once per
    // tile.  For one-channel classes (fp32, fp16 and uint8 planes: 4K fp16
    // -1.9 %, 4:2:0 CIF -3.8 %); three-channel classes keep the per-stage
    // offsets, which measured faster there (RGB CIF +2.3 % per tile, 1080p
    // RGB 1/2 unchanged)
    const bool fix_one = nar || (Cl::C == 1 && Cl::FPW * (fix.nl + fix.nr) <= 32);  // narrow: at most 32 (host)
    int fix_src = 0, fix_dst = -1;
    if (fixing && fix_one && lane < fpw * (fix.nl + fix.nr)) {
      if (nar) edge_elem_narrow<Cl>(fix, lane, jd.W, xw, fix_src, fix_dst);
      else edge_elem<Cl>(fix, lane, jd.W, xw, fix_src, fix_dst);
    }
    const int frame0 = tl.frame * fpw;                  // the group's first frame
    const int nf = Cl::FPW == 1 ? 1 : min(fpw, jd.nframes - frame0);  // frames in the group
    const int sub = lane / lps;                         // this lane's frame in the group
    const int blk0 = strip * Cl::SBLK + (lane % lps) * Cl::NB;
    const bool active = sub < nf && blk0 * Cl::P < jd.OW;
    // elements this lane stores per output row (none for an inactive lane,
    // which runs the same code on in-window data with its stores masked)
    const int n_valid = active ? jd.OW * Cl::C - blk0 * Cl::P * Cl::C : 0;
    T* const obase = reinterpret_cast<T*>(jd.out) + (long long)(frame0 + sub) * jd.out_frame +
                     (long long)blk0 * Cl::P * Cl::C;
    const long long rowe = (long long)jd.OW * Cl::C;
    // uint8 runs of a length that is not whole words: stored as words when the
    // output and its rows start on word boundaries (the same choice for the
    // whole warp), else as bytes
    const bool words = sizeof(T) == 1 && (reinterpret_cast<uintptr_t>(jd.out) & 3u) == 0 && (rowe & 3) == 0;

    auto issue = [&](int s) {  // stage s of the tile into slot (g + s) mod NST
      const uint32_t G = g + (uint32_t)s, slot = G % NST;
      if constexpr (kCheckBounds) {  // frames of the job, window start on 16 bytes
        if (frame0 < 0 || frame0 + nf > jd.nframes || (xt * kTmaElem) % 16 != 0) {
          bounds_fail(prm.dev, 4, (long long)xt * kTmaElem);
          mbar_expect_tx(&full[slot], 0u);  // completes the phase with no copy
          return;
        }
      }
      if (nar) {  // box k: frames frame0 + 2k and + 2k + 1 (x, frame, row map)
        const int nbx = (nf + 1) >> 1;
        mbar_expect_tx(&full[slot], (uint32_t)(nbx * Cl::RTX));
        for (int k = 0; k < nbx; ++k)
          tma_load_3d(ring + slot * Cl::RSTAGE + k * Cl::FSTR, &jd.tmap, &full[slot], xt, frame0 + 2 * k,
                      ystream + s * SR + (s == 0 ? Cl::S0SHIFT : 0));
        return;
      }
      mbar_expect_tx(&full[slot], (uint32_t)(nf * Cl::RTX));
      for (int f = 0; f < nf; ++f)
#pragma unroll
        for (int bx = 0; bx < Cl::NBOX; ++bx)
          tma_load_3d(ring + slot * Cl::RSTAGE + f * Cl::FSTR + bx * Cl::BOXSTR, &jd.tmap, &full[slot],
                      xt + bx * Cl::BOXE, ystream + s * SR + (s == 0 ? Cl::S0SHIFT : 0), frame0 + f);
    };
    // Modular tilers: a stage whose rows and window columns all lie inside
    // the frame is the tensor copy of the clamped form (classes of one frame
    // per warp: 4K fp16 440 -> 416 us, 1080p RGB 1/2 474 -> 458 us; the CIF
    // classes, whose strips are mostly frame edges, measured slower with it:
    // RGB CIF 187 -> 195 us).  In any other stage every row is copied by
    // itself from frame row (y mod H), the window's bytes left of the row
    // from the row's last bytes and those past its end from its first bytes
    // (one 1-D bulk copy each, lane k taking row k); so the stage holds the
    // window modulo the frame and no border needs fixing.  The plan only
    // takes this path when a window spans less than one period of the row.
    const long long rowb = (long long)jd.W * Cl::C * Cl::SZ;
    const bool cols_inside = (long long)xw * Cl::SZ >= 0 && (long long)xw * Cl::SZ + Cl::WINB <= rowb;
    auto issue_wrap = [&](int s) {  // all lanes
      const uint32_t G = g + (uint32_t)s, slot = G % NST;
      if (lane == 0) mbar_expect_tx(&full[slot], (uint32_t)(nf * SR * Cl::WINB));
      __syncwarp();
      const long long lo = (long long)xw * Cl::SZ, hi = lo + Cl::WINB;  // window bytes within the row
      for (int k = lane; k < nf * SR; k += 32) {
        const int f = k / SR, r = k - f * SR;
        int y = ystream + s * SR + (s == 0 ? Cl::S0SHIFT : 0) + r;
        if (y < 0) y += H;  // within one period of the frame: no division
        else if (y >= H) y -= H;
        if ((unsigned)y >= (unsigned)H) y = ((y % H) + H) % H;  // frames of fewer rows than a window
        const uint8_t* row = jd.in + ((long long)(frame0 + f) * H + y) * rowb;
        uint8_t* dst = ring + slot * Cl::RSTAGE + f * Cl::FSTR + r * Cl::BOXB;
        const long long m0 = lo > 0 ? lo : 0, m1 = hi < rowb ? hi : rowb;
        if constexpr (kCheckBounds) {
          const long long off = (long long)(dst - ring);
          const bool bad = off < 0 || off + Cl::WINB > Cl::WARP_BYTES || frame0 + f >= jd.nframes ||
                           -lo > rowb || hi - rowb > rowb || m1 <= m0;
          if (bad) {  // skip the row's copies and take their bytes off the barrier's count
            bounds_fail(prm.dev, 4, off);
            mbar_complete_tx(&full[slot], (uint32_t)Cl::WINB);
            continue;
          }
        }
        if (lo < 0) bulk_load(dst, row + rowb + lo, (uint32_t)(-lo), &full[slot]);
        bulk_load(dst + (m0 - lo), row + m0, (uint32_t)(m1 - m0), &full[slot]);
        if (hi > rowb) bulk_load(dst + (rowb - lo), row, (uint32_t)(hi - rowb), &full[slot]);
      }
    };
    // fill stage s of modular tilers (all lanes call it)
    auto fill_wrap = [&](int s) {
      const int y0 = ystream + s * SR + (s == 0 ? Cl::S0SHIFT : 0);
      if (Cl::FPW > 1 || !(cols_inside && y0 >= 0 && y0 + SR <= H)) issue_wrap(s);
      else if (lane == 0) issue(s);
    };
    if constexpr (WRAP) {
      for (int s = 0; s < NST && s < nst; ++s) fill_wrap(s);
    } else {
      if (lane == 0)
        for (int s = 0; s < NST && s < nst; ++s) issue(s);
    }
    issued = g + (uint32_t)min(NST, nst);
    // wait for stage s; returns the stage's row-0 base, or nullptr on timeout.
    // The stage's columns outside the frame get their border values (only
    // tiles whose strip needs it)
    auto stage_wait = [&](int s) -> uint8_t* {
      const uint32_t G = g + (uint32_t)s, slot = G % NST;
      if (!__all_sync(0xffffffffu, mbar_wait(&full[slot], (G / NST) & 1u))) return nullptr;
      uint8_t* const sb = ring + slot * Cl::RSTAGE;
      if (fixing) apply_edge_fix<Cl>(sb, fix, lane, jd.W, xw, fix_one, fix_src, fix_dst, prm.dev);
      return sb;
    };
    // stage s fully read: refill its slot with stage s + NST
    auto stage_release = [&](int s) {
      __syncwarp();
      if (s + NST < nst) {
        if constexpr (WRAP) fill_wrap(s + NST);
        else if (lane == 0) issue(s + NST);
        issued = g + (uint32_t)(s + NST + 1);
      }
    };
    // H pass of one loaded row into a window row
    // every vector a lane reads of a row lies in the warp's ring
    auto row_ok = [&](const uint8_t* rowbase) -> bool {
      if constexpr (kCheckBounds) {
#pragma unroll
        for (int v = 0; v < Cl::NVT; ++v) {
          const long long off = (long long)(rowbase - ring) + of.v[v];
          if (off < 0 || off + Cl::VB > Cl::WARP_BYTES) {
            bounds_fail(prm.dev, 1, off);
            return false;
          }
        }
      }
      return true;
    };
    // the output rows of block rr this lane stores lie in its frame
    auto store_ok = [&](int rr) -> bool {
      if constexpr (kCheckBounds) {
        if (n_valid > 0) {
          const long long first = (long long)blk0 * Cl::P * Cl::C + (long long)rr * P * rowe;
          const int last_row = min(rr * P + P, jd.OH) - 1 - rr * P;
          const long long last = first + (long long)last_row * rowe + min(n_valid, Cl::NOUT) - 1;
          if (first < 0 || last >= jd.out_frame || frame0 + sub >= jd.nframes) {
            bounds_fail(prm.dev, 3, first < 0 ? first : last);
            return false;
          }
        }
      }
      return true;
    };
    auto hrow_regs = [&](uint8_t* rowbase, Row& o) {
      if (!row_ok(rowbase)) return;
      uint32_t w[Cl::NWT];
      load_row<Cl>(rowbase, of, w);
      RM::h(w, prm, o);
    };

    Row win[L];
    // ---- prologue: pattern rows 0 .. L-Q-1 (with PRO: the lead blocks below)
#pragma unroll
    for (int ps = 0; ps < (Cl::PRO ? 0 : Cl::NPS); ++ps) {
      uint8_t* sb = stage_wait(ps);
      if (!sb) {
        ok = false;
        break;
      }
#pragma unroll
      for (int r = 0; r < SR; ++r) {
        // pattern row index: stage 0 holds pattern rows 0.. (S0SHIFT), and
        // its last EXTRA rows repeat rows of stage 1
        const int i = ps == 0 ? r - Cl::EXTRA + Cl::S0SHIFT : ps * SR + r - Cl::EXTRA;
        if (i < 0 || (ps == 0 && r >= SR - Cl::S0SHIFT)) continue;
        const int y = ys + i;
        if (y < 0 && !wrap) continue;           // top band: filled from frame row 0 below
        if (i > 0 && y >= H && !wrap) {
          RM::copy(win[i], win[i - 1]);
        } else {
          hrow_regs(sb + r * Cl::BOXB, win[i]);
        }
      }
      stage_release(ps);
    }
    if (!ok) break;
    // top band (ys == BMINV): slots 0..LHV-1 are frame row 0, held in slot LHV
    // (modular tilers: they hold the frame's last rows, as loaded)
    auto top_fix = [&]() {
      if (ys < 0 && !wrap) {
#pragma unroll
        for (int i = 0; i < Cl::LHV; ++i) RM::copy(win[i], win[Cl::LHV]);
      }
    };
    if constexpr (!Cl::PRO) top_fix();
    // ---- block steps, U rows (USTG stages, UBLK blocks) at a time.  A unit
    // whose blocks are all inside the tile, whose rows are all above the
    // frame's last row and whose output rows are all inside the frame, in a
    // group with every frame present, runs a copy of the body without any of
    // those checks.  Both copies fix up the border columns of each stage and
    // mask the stores of lanes past the frame's right edge, so the left and
    // right strips of a frame run the check-free copy too.  With PRO, blocks
    // m < 0 are the lead blocks: their rows (those above frame row 0
    // included, filtered from the zero fill and then overwritten) only fill
    // the window.
    auto unit = [&](auto fast, int u) {
      constexpr bool FAST = decltype(fast)::value;
#pragma unroll
      for (int st = 0; st < Cl::USTG; ++st) {
        const int s = Cl::STG0 + u * Cl::USTG + st;
        if (!FAST && s >= nst) break;
        uint8_t* sb = stage_wait(s);
        if (!sb) {
          ok = false;
          return;
        }
#pragma unroll
        for (int r = 0; r < SR; ++r) {
          const int ru = st * SR + r;       // row within the unit
          const int bq = ru / Q, q = ru - bq * Q;
          const int m = u * Cl::UBLK + bq - Cl::VBLK;  // block step
          if (FAST || m < nblk) {
            const int i = L - Q + q;
            if constexpr (FAST) {
              uint32_t w[Cl::NWT];
              if (row_ok(sb + r * Cl::BOXB)) load_row<Cl>(sb + r * Cl::BOXB, of, w);
              RM::h(w, prm, win[i]);
            } else {
              hrow_regs(sb + r * Cl::BOXB, win[i]);
            }
            if (q == Q - 1) {
              // rows below the frame's last repeat it: filtered from the zero
              // fill, then replaced, once per block and only in blocks that
              // reach below the frame (modular tilers loaded the frame's
              // first rows there)
              if constexpr (!FAST && !WRAP) {
                if (ys + m * Q + L - 1 >= H) {
#pragma unroll
                  for (int i2 = L - Q; i2 < L; ++i2)
                    if (ys + m * Q + i2 >= H) RM::copy(win[i2], win[i2 - 1]);
                }
              }
              // the window holds block m's pattern: its P output rows
              // (a lane whose rows fail the bounds check stores nothing but
              // still runs the V pass: its stores may shuffle across lanes)
              if constexpr (FAST) {
                RM::template v<false>(win, prm, obase, rowe, rb0 + m, jd.OH, store_ok(rb0 + m) ? n_valid : 0, words);
              } else if (!Cl::PRO || m >= 0) {
                RM::template v<true>(win, prm, obase, rowe, rb0 + m, jd.OH, store_ok(rb0 + m) ? n_valid : 0, words);
              }
#pragma unroll
              for (int i2 = 0; i2 < L - Q; ++i2) RM::copy(win[i2], win[i2 + Q]);
              if constexpr (!FAST && Cl::PRO)
                if (m == -1) top_fix();
            }
          }
        }
        stage_release(s);
      }
    };
    // every frame of the group present
    const bool group_full = nf == fpw;
    const int nunits = (nblk + Cl::VBLK + Cl::UBLK - 1) / Cl::UBLK;
    for (int u = 0; ok && u < nunits; ++u) {
      if constexpr (Cl::FASTPATH) {
        const int mend = (u + 1) * Cl::UBLK - Cl::VBLK;  // one past the unit's last block
        if (group_full && mend - Cl::UBLK >= 0 && mend <= nblk && ys + (mend - 1) * Q + L - 1 < H &&
            (rb0 + mend) * P <= jd.OH) {
          unit(std::true_type{}, u);
          continue;
        }
      }
      unit(std::false_type{}, u);
    }
    g += (uint32_t)nst;
  }
  if (!ok) {
    // a wait gave up (or a job of the wrong class): record it and leave no
    // copy in flight
    if (lane == 0) {
      atomicCAS(&prm.dev->status, 0, kStatusTimeout);
      for (uint32_t G = (issued > (uint32_t)NST ? issued - NST : 0); G < issued; ++G)
        mbar_wait(&full[G % NST], (G / NST) & 1u);
    }
  }
  // the last warp out resets the slot for its next launch
  if (lane == 0) {
    __threadfence();
    if (atomicAdd(&prm.dev->warps_done[prm.sched_slot], 1u) == nwarps - 1) {
      prm.dev->tile_next[prm.sched_slot] = 0;
      prm.dev->warps_done[prm.sched_slot] = 0;
      __threadfence();
    }
  }
}

// ---------------------------------------------------------------------------
// host side of one class and shape
// ---------------------------------------------------------------------------
struct HostGeom {
  int sblk, spx, p, q, pv, boxe, sr, sz, c, fpw;
  CUtensorMapDataType dt;
  int hlb, rhb;  // halo bytes of a strip's window, left and right
  bool narrow;   // narrow tail strips: last strips of at most npn packets, windows of wn bytes
  int npn, wn;
};

struct KernelInfo {
  const void* fn;
  int smem;
  int threads;
};

// What the host needs of one compiled (class, tile shape): its geometry, its
// kernel with room for kFewJobs or kMaxJobs job descriptors, the host replay
// of its index arithmetic, and its shape for descriptions.
struct RowsEntry {
  bool present, has_wrap;     // has_wrap: compiled for modular tilers too
  HostGeom geom;
  KernelInfo few, many;       // clamp-to-edge
  KernelInfo few_wrap, many_wrap;
  std::string (*check)(const JobDesc* jds, int njobs);
  int nb, sr, nst, wpc, minb;
  int (*narrow_fix)(int strip, int W, int OW);  // border-fix elements of a narrow strip's four frames
};

template <class Cl>
HostGeom host_geom() {
  return HostGeom{Cl::SBLK, Cl::SPX, Cl::P, Cl::Q, Cl::PV, Cl::BOXE, Cl::SRR, Cl::SZ, Cl::C, Cl::FPW, kTmaType,
                  Cl::HLB, Cl::RHB, Cl::NARROW, Cl::NPN, Cl::WN};
}

// Registers are budgeted for Cl::MINB resident CTAs (of Cl::WPC warps) per SM.
template <class Cl, bool WRAP>
KernelInfo rows_info(bool few) {
  constexpr int smem = 128 + Cl::WPC * (Cl::WARP_BYTES + Cl::NST * 8);
  const void* fn = few ? reinterpret_cast<const void*>(&k_rows<Cl, kFewJobs, WRAP>)
                       : reinterpret_cast<const void*>(&k_rows<Cl, kMaxJobs, WRAP>);
  return KernelInfo{fn, smem, Cl::WPC * 32};
}

// ---------------------------------------------------------------------------
// host-side check of the kernel's index arithmetic
// ---------------------------------------------------------------------------
// Host-side walk of the row-streaming kernel over every tile of one frame:
// TMA x coordinates are 16-byte aligned; every shared-memory read of the H
// pass (vector chunks, halo words, clamped border pixels) stays inside the
// loaded window and never straddles a box; the shared-memory footprint fits;
// a replay of the stream and register-window logic on frame-row indices --
// every V block must see exactly the clamped rows of its window, every
// stream row must be the next frame row in order, every output element is
// written once.
// The jobs of one frame: a plan's one job, or its job without the last strip
// and the narrow tail-strip job (four frames per warp).
template <class Cl>
std::string check_rows(const JobDesc* jds, int njobs) {
  constexpr int WPC = Cl::WPC;
  char buf[256];
  auto fail = [&](const char* what, int a, int b) {
    std::snprintf(buf, sizeof(buf), "rows class %d: %s (%d, %d)", Cl::id, what, a, b);
    return std::string(buf);
  };
  constexpr int smem = 128 + WPC * (Cl::WARP_BYTES + Cl::NST * 8);
  if (smem > 227 * 1024) return fail("shared memory above 227 KB", smem, 0);
  if (Cl::BOXSTR < Cl::SRR * Cl::BOXB || Cl::BOXSTR % 128 != 0) return fail("stage layout", Cl::BOXSTR, 0);
  if (Cl::LPS * Cl::FPW != 32) return fail("lanes per frame", Cl::LPS, Cl::FPW);
  if (njobs < 1) return fail("no jobs", njobs, 0);
  // L, Q, P: the vertical axis; PH: the horizontal phases per packet
  constexpr int L = Cl::LV, Q = Cl::QV, P = Cl::PV, PH = Cl::P;
  std::vector<int> written((size_t)jds[0].OH * jds[0].OW * Cl::C, 0);
  for (int jx = 0; jx < njobs; ++jx) {
  const JobDesc& jd = jds[jx];
  const bool nar = jd.nar != 0;
  if (nar && !Cl::NARROW) return fail("narrow job on a class without narrow strips", jx, 0);
  if (nar && (jd.strips != 1 || jd.wrap)) return fail("narrow job shape", jd.strips, jd.wrap);
  // a lane's window: the box row (frame pairs), or its half (narrow strips)
  const int win = nar ? Cl::WN : Cl::NBOX * Cl::BOXB;
  const int lps = nar ? 8 : Cl::LPS;
  if (nar && (2 * Cl::WN != Cl::BOXB || 2 * Cl::SRR * Cl::WN != Cl::RTX))
    return fail("narrow box layout", Cl::WN, Cl::BOXB);
  const int nby = (jd.OH + P - 1) / P;
  for (int chunk = 0; chunk < jd.chunks; ++chunk) {
    for (int strip_i = 0; strip_i < jd.strips; ++strip_i) {
      const int strip = jd.strip0 + strip_i;
      const int rb0 = chunk * jd.rbc;
      const int nblk = std::min(jd.rbc, nby - rb0);
      if (nblk < 1) return fail("empty tile", chunk, strip);
      const int ys = rb0 * Q + Cl::BMINV;
      const int ye = (rb0 + nblk - 1) * Q + Cl::BMINV + L;
      const int y0 = std::max(ys, 0), nrow = std::min(ye, jd.H) - y0;
      if (nrow < 1) return fail("empty stream", ys, ye);
      if (ys < 0 && ys != Cl::BMINV) return fail("top band offset", ys, 0);
      const int xw = strip * Cl::SPX * Cl::C - Cl::HLB / Cl::SZ;
      if ((xw * Cl::SZ) % kTmaElem != 0) return fail("window start not a whole TMA element", xw, 0);
      for (int bx = 0; bx < Cl::NBOX; ++bx) {
        const long long xb = (long long)(xw * Cl::SZ / kTmaElem + bx * Cl::BOXE) * kTmaElem;
        if (((xb % 16) + 16) % 16 != 0) return fail("TMA x not 16-byte aligned", xw, bx);
      }
      const bool wrap = jd.wrap != 0;
      auto wrapped = [&](int y) { return ((y % jd.H) + jd.H) % jd.H; };
      if (wrap) {
        // the row copies of modular tilers: 16-byte aligned pieces that fill
        // the window exactly, each at most one period of the row away
        const long long rowb = (long long)jd.W * Cl::C * Cl::SZ, lo = (long long)xw * Cl::SZ, hi = lo + Cl::WINB;
        const long long m0 = std::max(lo, 0LL), m1 = std::min(hi, rowb);
        if (rowb % 16 || lo % 16 || hi % 16) return fail("row copy not 16-byte aligned", (int)lo, (int)hi);
        if (-lo > rowb || hi - rowb > rowb || m1 <= m0) return fail("row copy beyond one period", (int)lo, (int)hi);
      }
      const EdgeFix fx = edge_fix<Cl>(strip, jd.W, jd.OW);
      if (nar && 4 * (fx.nl + fx.nr) > 32) return fail("narrow border fix above one element per lane", fx.nl, fx.nr);
      for (int e = 0; e < (wrap ? 0 : fx.nl + fx.nr); ++e) {
        const bool left = e < fx.nl;
        const int k2 = left ? e : e - fx.nl;
        const int px = (left ? fx.l_lo : fx.r_lo) + k2 / Cl::C, c = k2 % Cl::C;
        const int src = (left ? 0 : jd.W - 1) * Cl::C + c - xw, dst = px * Cl::C + c - xw;
        if (src < 0 || (src + 1) * Cl::SZ > win || dst < 0 || (dst + 1) * Cl::SZ > win)
          return fail("edge fix outside the window", src, dst);
      }
      // every frame of a warp's group has the same window layout: lanes li of the strip
      for (int lane = 0; lane < lps; ++lane) {
        const int li = nar ? std::min(lane, Cl::NPN - 1) : lane;  // narrow: lanes past the window read its last packet
        const int first = Cl::HLB + li * Cl::EB - Cl::HB * Cl::VB;
        for (int v = 0; v < Cl::NVT; ++v) {
          const int b0 = first + v * Cl::VB;
          if (b0 < 0 || b0 + Cl::VB > win || b0 / Cl::BOXB != (b0 + Cl::VB - 1) / Cl::BOXB)
            return fail("vector read", lane, b0);
        }
        const int blk0 = strip * Cl::SBLK + lane * Cl::NB, px0 = blk0 * Cl::Q;
        if (blk0 * PH >= jd.OW || wrap) continue;
        if (nar && (lane >= Cl::NPN || (px0 - Cl::LH) * Cl::C - xw < 0 ||
                    (px0 + Cl::NB * Cl::Q + Cl::RH) * Cl::C - xw > win / Cl::SZ))
          return fail("narrow lane's pixels outside its window", lane, px0);
        for (int px = px0 - Cl::LH; px < px0 + Cl::NB * Cl::Q + Cl::RH; ++px) {
          if (px < 0 && !(px >= fx.l_lo && fx.nl > 0)) return fail("left border pixel not fixed", lane, px);
          if (px >= jd.W && !(px >= fx.r_lo && px < fx.r_lo + fx.nr / Cl::C)) return fail("right border pixel not fixed", lane, px);
        }
      }
      // replay of the stream and window on frame-row indices: stage s holds
      // frame rows ystream + s*SR .. + SR - 1
      const int nst = Cl::STG0 + ((nblk + Cl::VBLK) * Q + Cl::SRR - 1) / Cl::SRR;
      const int ystream = ys + Cl::YOFF;
      int wrow[64];
      int sr = 0;  // rows consumed from the stream, checked against their position
      auto take = [&](int s, int r, int i) -> std::string {
        if (s >= nst) return fail("stage beyond the tile", s, nst);
        wrow[i] = ystream + s * Cl::SRR + r + (s == 0 ? Cl::S0SHIFT : 0);
        if (wrap) wrow[i] = wrapped(wrow[i]);
        ++sr;
        return std::string();
      };
      for (int ps = 0; ps < (Cl::PRO ? 0 : Cl::NPS); ++ps)
        for (int r = 0; r < Cl::SRR; ++r) {
          const int i = ps == 0 ? r - Cl::EXTRA + Cl::S0SHIFT : ps * Cl::SRR + r - Cl::EXTRA;
          if (i < 0 || (ps == 0 && r >= Cl::SRR - Cl::S0SHIFT)) continue;
          const int y = ys + i;
          if (y < 0 && !wrap) continue;
          if (i > 0 && y >= jd.H && !wrap) { wrow[i] = wrow[i - 1]; continue; }
          std::string e = take(ps, r, i);
          if (!e.empty()) return e;
          if (wrow[i] != (wrap ? wrapped(y) : y)) return fail("prologue row mismatch", i, wrow[i]);
        }
      if (ys < 0 && !Cl::PRO && !wrap)
        for (int i = 0; i < Cl::LHV; ++i) wrow[i] = wrow[Cl::LHV];
      const int nunits = (nblk + Cl::VBLK + Cl::UBLK - 1) / Cl::UBLK;
      for (int u = 0; u < nunits; ++u)
        for (int st = 0; st < Cl::USTG; ++st) {
          const int s = Cl::STG0 + u * Cl::USTG + st;
          if (s >= nst) break;
          for (int r = 0; r < Cl::SRR; ++r) {
            const int ru = st * Cl::SRR + r, bq = ru / Q, q = ru - bq * Q, m = u * Cl::UBLK + bq - Cl::VBLK;
            if (m >= nblk) continue;
            const int i = L - Q + q, y = ys + m * Q + i;
            if (y >= jd.H && !wrap) wrow[i] = wrow[i - 1];
            else {
              std::string e = take(s, r, i);
              if (!e.empty()) return e;
              if (wrow[i] != (wrap ? wrapped(y) : y)) return fail("stream row mismatch", i, wrow[i]);
            }
            if (q != Q - 1) continue;
            if (m < 0) {  // a lead block: no outputs, the window moves on
              for (int i2 = 0; i2 < L - Q; ++i2) wrow[i2] = wrow[i2 + Q];
              if (m == -1 && ys < 0 && !wrap)
                for (int i2 = 0; i2 < Cl::LHV; ++i2) wrow[i2] = wrow[Cl::LHV];
              continue;
            }
            const int rr = rb0 + m;
            for (int i2 = 0; i2 < L; ++i2) {
              int want = rr * Q + Cl::BMINV + i2;
              want = wrap ? wrapped(want) : (want < 0 ? 0 : (want > jd.H - 1 ? jd.H - 1 : want));
              if (wrow[i2] != want) return fail("window row mismatch", i2, wrow[i2]);
            }
            for (int lane = 0; lane < lps; ++lane) {
              const int blk0 = strip * Cl::SBLK + lane * Cl::NB;
              if (blk0 * PH >= jd.OW) continue;
              const int nv = std::min(Cl::NOUT, jd.OW * Cl::C - blk0 * PH * Cl::C);
              for (int jv = 0; jv < P; ++jv) {
                const int oy = rr * P + jv;
                if (oy >= jd.OH) continue;
                for (int k = 0; k < nv; ++k) written[((size_t)oy * jd.OW) * Cl::C + (size_t)blk0 * PH * Cl::C + k]++;
              }
            }
            for (int i2 = 0; i2 < L - Q; ++i2) wrow[i2] = wrow[i2 + Q];
          }
        }
      // with lead blocks every stream row above the frame's end is filtered (those above row 0 too)
      const int want_rows = wrap ? (Cl::PRO ? ye - ystream : ye - ys) : (Cl::PRO ? std::min(ye, jd.H) - ystream : nrow);
      if (sr != want_rows) return fail("stream rows left over", sr, want_rows);
    }
  }
  }
  for (size_t i = 0; i < written.size(); ++i)
    if (written[i] != 1) return fail("output element written != 1 times", (int)i, written[i]);
  return std::string();
}

template <class Cl>
int narrow_fix_elems(int strip, int W, int OW) {
  const EdgeFix f = edge_fix<Cl>(strip, W, OW);
  return 4 * (f.nl + f.nr);
}

// with_wrap: also compile the class for modular tilers (tile shape 0 only:
// the clamp kernels are the ones the tuner chooses among)
template <class Cl, bool WITH_WRAP>
RowsEntry make_entry() {
  RowsEntry e{true, WITH_WRAP, host_geom<Cl>(), rows_info<Cl, false>(true), rows_info<Cl, false>(false),
              KernelInfo{nullptr, 0, 0}, KernelInfo{nullptr, 0, 0}, &check_rows<Cl>,
              Cl::NB, Cl::SRR, Cl::NST, Cl::WPC, Cl::MINB, &narrow_fix_elems<Cl>};
  if constexpr (WITH_WRAP) {
    e.few_wrap = rows_info<Cl, true>(true);
    e.many_wrap = rows_info<Cl, true>(false);
  }
  return e;
}

// Tile shapes compiled per class, and the table of every (class, shape).
constexpr int kShapes = 2;
using RowsTable = RowsEntry[kFcCount][kShapes];
// each rows_*.cu registers its classes
void register_f32(RowsTable& t);
void register_f16(RowsTable& t);
void register_u8rgb(RowsTable& t);
void register_u8c1(RowsTable& t);
void register_cif(RowsTable& t);

}  // namespace rows
}  // namespace ds

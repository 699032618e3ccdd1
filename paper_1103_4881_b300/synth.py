"""Seeded synthetic inputs for the downscaler workloads.

Frames only: this module holds none of the filter's arithmetic.  The paper
measures on its own 2000-frame CIF video (Sec. 3), which is not available;
these generators stand in for it with the shapes, value ranges and seeds of
the workload table below (numpy PCG64 streams, so the CUDA tests, the
benchmark and the CPU oracle all see the same pixels).
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

DS_F32, DS_F16, DS_U8, DS_U8_RGB = 0, 1, 2, 3
NP_DTYPE = {DS_F32: np.float32, DS_F16: np.float16, DS_U8: np.uint8, DS_U8_RGB: np.uint8}
CHANNELS = {DS_F32: 1, DS_F16: 1, DS_U8: 1, DS_U8_RGB: 3}


@dataclass(frozen=True)
class Workload:
    name: str
    frames: int
    height: int
    width: int
    ratio: tuple
    taps: int
    dtype: int
    seed: int
    content: str  # "uniform", "gradient", "bytes", "noisy_half"
    ratio_v: tuple = None   # vertical ratio and taps when they differ from the horizontal ones
    taps_v: int = 0
    planes: tuple = ()      # planar formats: ((h, w), ...) per plane; () = one plane height x width

    @property
    def channels(self) -> int:
        return CHANNELS[self.dtype]

    @property
    def vratio(self) -> tuple:
        return self.ratio_v if self.ratio_v else self.ratio

    @property
    def vtaps(self) -> int:
        return self.taps_v if self.taps_v else self.taps

    @property
    def out_height(self) -> int:
        return self.height * self.vratio[0] // self.vratio[1]

    @property
    def out_width(self) -> int:
        return self.width * self.ratio[0] // self.ratio[1]

    def plane_shapes(self):
        return list(self.planes) if self.planes else [(self.height, self.width)]

    def plane_out_shape(self, hw):
        oh, ow = hw[0] * self.vratio[0] // self.vratio[1], hw[1] * self.ratio[0] // self.ratio[1]
        return (oh, ow) if self.channels == 1 else (oh, ow, self.channels)

    def frame_shape(self):
        return (self.height, self.width) if self.channels == 1 else (self.height, self.width, self.channels)

    def out_frame_shape(self):
        return self.plane_out_shape((self.height, self.width))

    def bytes_per_frame(self) -> int:
        """Algorithmic bytes: input read once plus output written once (all planes)."""
        isz = np.dtype(NP_DTYPE[self.dtype]).itemsize
        tot = 0
        for hw in self.plane_shapes():
            oh, ow = self.plane_out_shape(hw)[:2]
            tot += (hw[0] * hw[1] + oh * ow) * self.channels * isz
        return tot


WORKLOADS = {
    # one 480x640 fp32 frame, uniform [0,1), 3/8 with 8 taps
    "plain_480x640_f32": Workload("plain_480x640_f32", 1, 480, 640, (3, 8), 8, DS_F32, 1001, "uniform"),
    # 64 fp32 1080x1920 frames, uniform plus a seeded smooth gradient, 3/8 K=8
    "batch64_1080x1920_f32": Workload("batch64_1080x1920_f32", 64, 1080, 1920, (3, 8), 8, DS_F32, 2000, "gradient"),
    # 300 uint8 RGB 1080x1920x3 frames, uniform bytes, 1/2 K=6, Q14 taps
    "rgb300_1080x1920_u8": Workload("rgb300_1080x1920_u8", 300, 1080, 1920, (1, 2), 6, DS_U8_RGB, 3000, "bytes"),
    # 128 fp16 2160x3840 frames, uniform + N(0, 0.05) clipped, 3/8 K=8
    "uhd128_2160x3840_f16": Workload("uhd128_2160x3840_f16", 128, 2160, 3840, (3, 8), 8, DS_F16, 4000, "noisy_half"),
    # the paper's case (Sec. 3): 2000 CIF frames, 24-bit RGB 352x288 -> 132x128,
    # horizontal 3/8 and vertical 4/9, K=8 on both axes; uniform bytes
    "cif2000_352x288_u8rgb": Workload("cif2000_352x288_u8rgb", 2000, 288, 352, (3, 8), 8, DS_U8_RGB, 7000, "bytes",
                                      ratio_v=(4, 9), taps_v=8),
    # the same as planar YUV 4:2:0: Y 352x288, U and V 176x144 (outputs 132x128, 66x64)
    "cif2000_yuv420_u8": Workload("cif2000_yuv420_u8", 2000, 288, 352, (3, 8), 8, DS_U8, 8000, "bytes",
                                  ratio_v=(4, 9), taps_v=8, planes=((288, 352), (144, 176), (144, 176))),
}


def frame(w: Workload, i: int) -> np.ndarray:
    """Frame i of workload w (i is also the seed offset)."""
    if w.content == "uniform":
        rng = np.random.default_rng(w.seed + i)
        return rng.random(w.frame_shape(), dtype=np.float32)
    if w.content == "gradient":
        rng = np.random.default_rng(w.seed + i)
        u = rng.random((w.height, w.width), dtype=np.float32)
        alpha, beta = rng.random(2)
        gx = np.arange(w.width, dtype=np.float64) / max(1, w.width - 1)
        gy = np.arange(w.height, dtype=np.float64) / max(1, w.height - 1)
        v = (u + alpha * gx[None, :] + beta * gy[:, None]) / (1.0 + alpha + beta)
        return v.astype(np.float32)
    if w.content == "bytes":
        rng = np.random.default_rng(w.seed + i)
        return rng.integers(0, 256, w.frame_shape(), dtype=np.uint8)
    if w.content == "noisy_half":
        rng = np.random.default_rng(w.seed + i)
        u = rng.random(w.frame_shape(), dtype=np.float32)
        n = rng.normal(0.0, 0.05, w.frame_shape()).astype(np.float32)
        return np.clip(u + n, 0.0, 1.0).astype(np.float16)
    raise ValueError(w.content)


def _each(fn, idx):
    """[fn(i) for i in idx], on several threads for long lists (every frame has
    its own generator, and numpy's fills run without the interpreter lock, so
    the frames are the same whatever the thread count)."""
    idx = list(idx)
    if len(idx) < 8:
        return [fn(i) for i in idx]
    with ThreadPoolExecutor(max(1, min(16, os.cpu_count() or 1))) as ex:
        return list(ex.map(fn, idx))


def frames(w: Workload, idx=None) -> np.ndarray:
    """Frames idx (default: all) stacked as (n, H, W[, C]) (the first plane)."""
    idx = range(w.frames) if idx is None else idx
    return np.stack(_each(lambda i: frame(w, i), idx))


def plane_frames(w: Workload, idx=None):
    """Frames idx of every plane: a list with one (n, h, w[, C]) array per plane."""
    if not w.planes:
        return [frames(w, idx)]
    idx = range(w.frames) if idx is None else idx
    out = []
    for k, (h, ww) in enumerate(w.planes):
        shape = (h, ww) if w.channels == 1 else (h, ww, w.channels)
        out.append(np.stack(_each(
            lambda i: np.random.default_rng(w.seed + 1_000_003 * k + i).integers(0, 256, shape, dtype=np.uint8), idx)))
    return out


def random_frames(shape, dtype: int, seed: int) -> np.ndarray:
    """Generic seeded frames for tests: floats uniform [0,1), bytes uniform 0..255."""
    rng = np.random.default_rng(seed)
    if dtype in (DS_U8, DS_U8_RGB):
        return rng.integers(0, 256, shape, dtype=np.uint8)
    x = rng.random(shape, dtype=np.float32)
    return x.astype(NP_DTYPE[dtype])


# --------------------------------------------------------------------------
# serving mix: 2000 requests, Poisson arrivals at 5000/s
# --------------------------------------------------------------------------
SERVE_SIZES = ((480, 640), (720, 1280), (1080, 1920), (2160, 3840))
SERVE_RATIOS = (((1, 2), 6), ((3, 8), 8), ((2, 3), 6))
SERVE_DTYPES = (DS_U8_RGB, DS_F16, DS_F32)


@dataclass(frozen=True)
class Request:
    rid: int
    arrival_s: float
    height: int
    width: int
    ratio: tuple
    taps: int
    dtype: int


def serving_requests(n: int = 2000, rate_hz: float = 5000.0, seed_arrivals: int = 5000,
                     seed_shapes: int = 5001):
    """Requests with exponential inter-arrival times (mean 1/rate) and uniformly
    drawn size, ratio and dtype."""
    ra = np.random.default_rng(seed_arrivals)
    t = np.cumsum(ra.exponential(1.0 / rate_hz, n))
    rs = np.random.default_rng(seed_shapes)
    si = rs.integers(0, len(SERVE_SIZES), n)
    ri = rs.integers(0, len(SERVE_RATIOS), n)
    di = rs.integers(0, len(SERVE_DTYPES), n)
    out = []
    for k in range(n):
        (h, w), (ratio, taps), dt = SERVE_SIZES[si[k]], SERVE_RATIOS[ri[k]], SERVE_DTYPES[di[k]]
        out.append(Request(k, float(t[k]), h, w, ratio, taps, dt))
    return out


def request_content(height: int, width: int, dtype: int, seed: int) -> np.ndarray:
    """One request frame with the content recipe of the batch workload of its
    dtype: fp32 uniform plus a smooth gradient (as the 1080p fp32 batch), fp16
    uniform plus N(0, 0.05) clipped (as the 4K fp16 batch), uint8 uniform
    bytes (as the RGB batch)."""
    content = {DS_F32: "gradient", DS_F16: "noisy_half", DS_U8: "bytes", DS_U8_RGB: "bytes"}[dtype]
    w = Workload("request", 1, height, width, (1, 2), 6, dtype, seed, content)
    return frame(w, 0)


def request_frame(req: Request) -> np.ndarray:
    """Pixel content of a request, seeded by its id."""
    return request_content(req.height, req.width, req.dtype, 6000 + req.rid)

"""Recipes for the five workloads (sizes, value distributions, structure).

* Smooth field S(s): white N(0,1) noise, filtered with a periodic Gaussian of
  standard deviation s pixels (FFT), normalised to [0, 1] by min/max.
* Edges: K random half-planes (uniform angle, offset uniform over the image),
  each adding +-U(0.1, 0.3).
* Images: "smooth + edges" clipped to [0, 1] and scaled to 8 bits (integers),
  to 255 on the 2^-16 grid (float32, exact), or "uniform noise + smooth" to 16 bits.
* Scales: paper scales a_k (Sec. 7) drawn as lo + (hi - lo) S(s), four independent
  fields; or ellipse fields (sigma, elongation, cos theta, sin theta) with
  sigma = 1 + 23 S(64), elongation = 1 + 5 S(64), theta = pi frac(4 S(96)).

* 1-D signals (Sec. 3 filter): rows of smooth + step noise, each row its own
  smooth field along its length (Gaussian of s samples, FFT per row) plus K
  random steps, on the 2^-16 grid (float32); scales a = lo + (hi - lo) S(s)
  per sample.

Every draw uses numpy's PCG64 generator seeded from SEED_BASE + a workload
index (+ an image index).
"""
import numpy as np

SEED_BASE = 908386


def smooth_field(rng, shape, sigma, dtype=np.float64):
    h, w = shape
    noise = rng.standard_normal((h, w))
    fy = np.fft.fftfreq(h)[:, None]
    fx = np.fft.rfftfreq(w)[None, :]
    gain = np.exp(-2.0 * (np.pi * sigma) ** 2 * (fx * fx + fy * fy))
    out = np.fft.irfft2(np.fft.rfft2(noise) * gain, s=(h, w))
    lo, hi = out.min(), out.max()
    out = (out - lo) / (hi - lo if hi > lo else 1.0)
    return out.astype(dtype)


def edge_field(rng, shape, k):
    h, w = shape
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    out = np.zeros(shape)
    for _ in range(k):
        ang = rng.uniform(0, 2 * np.pi)
        cx, cy = rng.uniform(0, w), rng.uniform(0, h)
        amp = rng.uniform(0.1, 0.3) * (1 if rng.uniform() < 0.5 else -1)
        side = (xx - cx) * np.cos(ang) + (yy - cy) * np.sin(ang) > 0
        out += amp * side
    return out


def image_c1(rng, shape=(256, 256), smooth=12.0, edges=6):
    """Integers in [0, 255] (returned as float64, as the workload states)."""
    v = np.clip(0.7 * smooth_field(rng, shape, smooth) + edge_field(rng, shape, edges), 0, 1)
    return np.round(255.0 * v).astype(np.float64)


def image_f32_grid(rng, shape, smooth=24.0, edges=12, frac_bits=16):
    """255 * clip(0.7 S + edges) rounded to the 2^-frac_bits grid, float32 (exact)."""
    v = np.clip(0.7 * smooth_field(rng, shape, smooth) + edge_field(rng, shape, edges), 0, 1)
    q = float(1 << frac_bits)
    return (np.round(255.0 * v * q) / q).astype(np.float32)


def image_c2(rng, shape=(2048, 2048)):
    return image_f32_grid(rng, shape, 24.0, 12, 16)


def image_c3(rng, shape=(8192, 8192), smooth=48.0):
    """uint16: round(65535 clip(0.5 U(0,1) + 0.5 S(48)))."""
    v = np.clip(0.5 * rng.uniform(0, 1, shape) + 0.5 * smooth_field(rng, shape, smooth), 0, 1)
    return np.round(65535.0 * v).astype(np.uint16)


def scales_a4(rng, shape, lo, hi, smooth):
    """Four independent smooth fields mapped affinely to [lo, hi]; (H, W, 4) float32."""
    return np.stack([lo + (hi - lo) * smooth_field(rng, shape, smooth) for _ in range(4)],
                    axis=-1).astype(np.float32)


def ellipse_field(rng, shape, sig=(1.0, 24.0), elong=(1.0, 6.0)):
    """(H, W, 4) float32: sigma, elongation, cos theta, sin theta."""
    s = sig[0] + (sig[1] - sig[0]) * smooth_field(rng, shape, 64.0)
    e = elong[0] + (elong[1] - elong[0]) * smooth_field(rng, shape, 64.0)
    th = np.pi * np.mod(4.0 * smooth_field(rng, shape, 96.0), 1.0)
    return np.stack([s, e, np.cos(th), np.sin(th)], axis=-1).astype(np.float32)


def workload(name, shape=None, seed_offset=0):
    """Inputs of one named workload.  Returns a dict with the image, its
    dtype / fraction bits, the raw scale field and its kind, order n and Q.
    ``shape`` overrides the size (parity tests use smaller sizes with the same
    recipe)."""
    if name == "c1":  # 256x256 integer image, n=1, a_k in [1, 8]
        rng = np.random.default_rng(SEED_BASE + 0 + seed_offset)
        shape = shape or (256, 256)
        img = image_c1(rng, shape)
        sc = scales_a4(rng, shape, 1.0, 8.0, 32.0)
        return dict(image=img, frac_bits=0, scale_kind="a4", scales=sc, n=1, q_bits=8,
                    cmax=8.0, value_bound=255.0)
    if name == "c2":  # 2048x2048 float32, n=2, ellipse fields
        rng = np.random.default_rng(SEED_BASE + 1 + seed_offset)
        shape = shape or (2048, 2048)
        img = image_c2(rng, shape)
        sc = ellipse_field(rng, shape)
        return dict(image=img, frac_bits=16, scale_kind="ellipse", scales=sc, n=2, q_bits=8,
                    cmax=150.0, value_bound=255.0, sigma_max=24.0, e_max=6.0)
    if name == "c3":  # 8192x8192 uint16, n=3, a_k in [1, 48]
        rng = np.random.default_rng(SEED_BASE + 2 + seed_offset)
        shape = shape or (8192, 8192)
        img = image_c3(rng, shape)
        sc = scales_a4(rng, shape, 1.0, 48.0, 128.0)
        return dict(image=img, frac_bits=0, scale_kind="a4", scales=sc, n=3, q_bits=8,
                    cmax=48.0, value_bound=65535.0)
    raise ValueError(name)


def batch_workload(count=64, lo=128, hi=2048, seed_offset=0):
    """64 images of uneven size: sides U{lo..hi}, n U{1,2,3}, float32 on the
    2^-16 grid, paper scales a_k in [1, 32] from S(32) fields."""
    rng = np.random.default_rng(SEED_BASE + 3 + seed_offset)
    jobs = []
    for i in range(count):
        h, w = int(rng.integers(lo, hi + 1)), int(rng.integers(lo, hi + 1))
        n = int(rng.integers(1, 4))
        r = np.random.default_rng(SEED_BASE + 3 + seed_offset + 1000 * (i + 1))
        img = image_f32_grid(r, (h, w), 24.0, 12, 16)
        sc = scales_a4(r, (h, w), 1.0, 32.0, 32.0)
        jobs.append(dict(image=img, frac_bits=16, scale_kind="a4", scales=sc, n=n, q_bits=8,
                         cmax=32.0, value_bound=255.0))
    return jobs


def smooth_rows(rng, count, length, sigma):
    """Each row an independent smooth field along its length, in [0, 1]."""
    noise = rng.standard_normal((count, length))
    fx = np.fft.rfftfreq(length)[None, :]
    gain = np.exp(-2.0 * (np.pi * sigma) ** 2 * fx * fx)
    out = np.fft.irfft(np.fft.rfft(noise, axis=1) * gain, n=length, axis=1)
    lo, hi = out.min(axis=1, keepdims=True), out.max(axis=1, keepdims=True)
    return (out - lo) / np.where(hi > lo, hi - lo, 1.0)


def signals_1d(rng, count, length, smooth=64.0, steps=8, frac_bits=16):
    """255 clip(0.7 S + steps) on the 2^-frac_bits grid, float32 rows."""
    v = 0.7 * smooth_rows(rng, count, length, smooth)
    for _ in range(steps):
        at = rng.integers(0, length, count)
        amp = rng.uniform(0.1, 0.3, count) * np.where(rng.uniform(size=count) < 0.5, 1.0, -1.0)
        v += amp[:, None] * (np.arange(length)[None, :] >= at[:, None])
    q = float(1 << frac_bits)
    return (np.round(255.0 * np.clip(v, 0, 1) * q) / q).astype(np.float32)


def scales_1d(rng, count, length, lo, hi, smooth):
    return (lo + (hi - lo) * smooth_rows(rng, count, length, smooth)).astype(np.float32)


def workload_1d(count=2048, length=65536, seed_offset=0):
    """The 1-D filter workload: float32 signals on the 2^-16 grid, model degree
    n1 = 1, analysis degree n2 = 3, scales a in [1, 64] varying smoothly
    (S(2048)) along each signal, Q = 8."""
    rng = np.random.default_rng(SEED_BASE + 5 + seed_offset)
    f = signals_1d(rng, count, length)
    a = scales_1d(rng, count, length, 1.0, 64.0, 2048.0)
    return dict(signals=f, scales=a, n1=1, n2=3, q_bits=8, frac_bits=16, max_scale=64.0, value_bound=255.0)

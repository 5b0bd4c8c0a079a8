"""Helpers for GPU parity tests: run the CUDA path through the C ABI and
compare with the oracle."""
import numpy as np

from oracle import scales as oscales

TORCH_IN = {"float64": "float64", "float32": "float32", "uint8": "uint8", "uint16": "uint16"}


def torch_dtype(np_dtype):
    import torch
    return {np.dtype(np.float64): torch.float64, np.dtype(np.float32): torch.float32,
            np.dtype(np.uint8): torch.uint8, np.dtype(np.uint16): torch.uint16}[np.dtype(np_dtype)]


def to_device(arr, dev):
    import torch
    if arr.dtype == np.uint16:
        return torch.from_numpy(arr.view(np.int16).copy()).to(dev).view(torch.uint16)
    return torch.from_numpy(np.ascontiguousarray(arr)).to(dev)


def run_exact(w, dev="cuda:0", out="f64", max_scale_product=0.0, want=("s", "num", "C"), debug_bounds=False):
    """Run abf_integrate + abf_filter (+ numerators, prepared scales) for a
    workload dict; returns numpy results and the filter object."""
    import torch
    from paper_0908_3861_gb300 import AdaptiveFilter
    img, sc = w["image"], w["scales"]
    H, W = img.shape
    filt = AdaptiveFilter(W, H, w["n"], torch_dtype(img.dtype), scale_kind=w["scale_kind"], q_bits=w["q_bits"],
                          frac_bits=w["frac_bits"], max_scale=w["cmax"], out=out,
                          value_bound=w.get("value_bound", 0.0), max_scale_product=max_scale_product,
                          min_scale=w.get("min_scale", 0.0), device=dev, debug_bounds=debug_bounds)
    f_t = to_device(img, dev)
    s_t = to_device(sc.astype(np.float32), dev)
    res = {}
    filt.integrate(f_t)
    if "s" in want:
        res["s"] = filt.filter(s_t).cpu().numpy()
    if "num" in want:
        res["num"] = filt.numerators(s_t).cpu().numpy().astype(np.uint64)
    if "C" in want:
        res["C"] = filt.prepare_scales(s_t).cpu().numpy()
    if "g" in want:
        res["g"] = filt.integrated().cpu().numpy().astype(np.uint64)
    torch.cuda.synchronize()
    res["status"] = filt.device_status()
    res["limbs"] = filt.limbs
    res["halo"] = filt.info["halo_lrbt"]
    res["filt"] = filt
    return res


def wide_to_int(num, L):
    """(..., L) uint64 limbs -> Python ints modulo 2^(64 L)."""
    flat = num.reshape(-1, L)
    return [sum(int(v[i]) << (64 * i) for i in range(L)) for v in flat]


def oracle_C(w):
    return oscales.scales_to_C(w["scale_kind"], w["scales"], w["n"], w["q_bits"], w["cmax"])


def f_int(w):
    img = w["image"]
    if img.dtype in (np.float32, np.float64):
        v = img.astype(np.float64) * float(1 << w["frac_bits"])
        assert np.all(v == np.rint(v))
        return v.astype(np.int64)
    return img.astype(np.int64)


def assert_close_f64(got, ref, rel=1e-13, absol=0.0):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    err = np.abs(got - ref)
    tol = rel * np.abs(ref) + absol
    bad = np.argwhere(err > tol)
    assert bad.size == 0, "max err %g at %s (got %r ref %r)" % (
        err.max(), bad[0], got[tuple(bad[0])], ref[tuple(bad[0])])


# ------------------------------------------------------ oracle on many pixels

_POOL_CACHE = {}


def _pool_init(name, shape):
    """Worker set-up: the workload regenerated from its seed (the same bytes as
    the parent's), its integer image and its integer steps."""
    import synthetic
    w = synthetic.workload(name, shape=shape)
    _POOL_CACHE["w"] = w
    _POOL_CACHE["fi"] = f_int(w)
    _POOL_CACHE["C"] = oracle_C(w)


def _pool_chunk(pix):
    from oracle import paper
    w = _POOL_CACHE["w"]
    S, s = paper.filter_pixels(_POOL_CACHE["fi"], _POOL_CACHE["C"], w["n"], w["q_bits"], w["frac_bits"], pix)
    return S, list(s)


def oracle_pixels_parallel(name, shape, pix, chunk=256, procs=None):
    """paper.filter_pixels on many pixels of a named workload, in a pool of
    spawned processes (one per host core), each regenerating the workload from
    its seed: returns (S list, s list) in the order of pix."""
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor
    procs = procs or os.cpu_count() or 1
    jobs = [pix[i:i + chunk] for i in range(0, len(pix), chunk)]
    S, s = [], []
    with ProcessPoolExecutor(max_workers=procs, mp_context=mp.get_context("spawn"), initializer=_pool_init,
                             initargs=(name, shape)) as ex:
        for S_part, s_part in ex.map(_pool_chunk, jobs):
            S.extend(S_part)
            s.extend(s_part)
    return S, s

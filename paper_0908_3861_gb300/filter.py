"""Convenience wrapper over the C ABI: one plan, its device buffers (allocated
with PyTorch), and the two steps of Sec. 7.  Marshalling and allocation only;
the computation is the library's."""
import torch

from . import _abf as C

_DT = {torch.uint8: C.ABF_U8, torch.uint16: C.ABF_U16, torch.float32: C.ABF_F32, torch.float64: C.ABF_F64}
_OUT = {"f32": (C.ABF_F32, torch.float32), "f64": (C.ABF_F64, torch.float64)}


class AdaptiveFilter:
    """s = adaptive box-spline filter of f (abf_integrate + abf_filter)."""

    def __init__(self, width, height, n, in_dtype, scale_kind="c4", q_bits=8, frac_bits=0, max_scale=8.0,
                 out="f64", form="exact", min_scale=0.0, value_bound=0.0, max_scale_product=0.0, device=None,
                 directions=4, model_boxes=0, debug_bounds=False):
        """debug_bounds: check every tap's reads against the lattice box
        (ABF_FLAG_DEBUG_BOUNDS; see bounds_violation)."""
        self.device = torch.device(device or "cuda")
        self.W, self.H, self.n = int(width), int(height), int(n)
        self.in_dtype = in_dtype
        self.out_code, self.out_dtype = _OUT[out]
        d = C.abf_desc()
        d.width, d.height, d.order_n = self.W, self.H, self.n
        d.in_dtype = _DT[in_dtype]
        d.out_dtype = self.out_code
        d.form = C.FORMS[form]
        d.scale_kind = C.SCALE_KINDS[scale_kind]
        d.q_bits = int(q_bits)
        d.in_frac_bits = int(frac_bits)
        d.flags = C.ABF_FLAG_DEBUG_BOUNDS if debug_bounds else 0
        d.max_scale = float(max_scale)
        d.min_scale = float(min_scale)
        d.value_bound = float(value_bound)
        d.max_scale_product = float(max_scale_product)
        d.directions = int(directions)
        d.model_boxes = int(model_boxes)
        self.desc = d
        with torch.cuda.device(self.device):
            self.plan = C.abf_plan_create(d)
        q = C.abf_plan_query(self.plan)
        self.info = q
        self.limbs = q["limbs"]
        self.g = torch.empty(max(q["integrated_bytes"], 16), dtype=torch.uint8, device=self.device)
        self.ws = torch.empty(max(q["workspace_bytes"], 16), dtype=torch.uint8, device=self.device)

    def close(self):
        if self.plan is not None:
            C.abf_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check_f(self, f):
        assert f.is_cuda and f.dtype == self.in_dtype and f.shape == (self.H, self.W) and f.is_contiguous()
        return f.shape[1] * f.element_size()

    def _check_scales(self, sc):
        assert sc.is_cuda and sc.dtype == torch.float32 and sc.shape == (self.H, self.W, 4) and sc.is_contiguous()
        return self.W * 16

    @property
    def exact(self):
        return self.desc.form == C.ABF_FORM_EXACT

    def integrate(self, f, stream=None):
        """Exact form: the non-adaptive step into the plan's integrated image."""
        C.abf_integrate(self.plan, f, self._check_f(f), self.g, self.ws, stream)

    def filter(self, scales, out=None, stream=None, f=None):
        """Adaptive step.  Exact form: from the integrated image; tile forms:
        from the image f (the running sums are restarted per tile)."""
        sp = self._check_scales(scales)
        if out is None:
            out = torch.empty((self.H, self.W), dtype=self.out_dtype, device=self.device)
        if self.exact:
            C.abf_filter(self.plan, self.g, 0, scales, sp, out, self.W * out.element_size(), self.ws, stream)
        else:
            C.abf_filter(self.plan, f, self._check_f(f), scales, sp, out, self.W * out.element_size(), self.ws,
                         stream)
        return out

    def __call__(self, f, scales, out=None, stream=None):
        if self.exact:
            self.integrate(f, stream)
            return self.filter(scales, out, stream)
        return self.filter(scales, out, stream, f=f)

    def autotune(self, scales, out=None, stream=None):
        """Exact form: time 4, 8 and 16 rows per CTA on the integrated image and
        these scales, keep the fastest; returns (rows, [ms x 3])."""
        sp = self._check_scales(scales)
        if out is None:
            out = torch.empty((self.H, self.W), dtype=self.out_dtype, device=self.device)
        return C.abf_plan_autotune(self.plan, self.g, scales, sp, out, self.W * out.element_size(), stream)

    def numerators(self, scales, stream=None):
        sp = self._check_scales(scales)
        num = torch.empty((self.H, self.W, self.limbs), dtype=torch.int64, device=self.device)
        C.abf_filter_numerator(self.plan, self.g, scales, sp, num, self.W * 8 * self.limbs, self.ws, stream)
        return num

    def prepare_scales(self, scales, stream=None):
        sp = self._check_scales(scales)
        out = torch.empty((self.H, self.W, 4), dtype=torch.int32, device=self.device)
        C.abf_prepare_scales(self.plan, scales, sp, out, self.W * 16, stream)
        return out

    def integrated(self):
        """The integrated image as (rows, pitch, limbs) int64 (a view of the buffer)."""
        rows = self.H + self.info["halo_lrbt"][3]
        pitch = self.info["g_pitch"]
        return self.g[: rows * pitch * self.limbs * 8].view(torch.int64).view(rows, pitch, self.limbs)

    def denominator(self):
        return C.abf_plan_denominator(self.plan)

    def device_status(self):
        return C.abf_last_device_status(self.plan)

    def launch_rows(self):
        """Rows (warps) per CTA of the adaptive step (8 by default; set by
        autotune, or from a tuning kept under ABF_TUNE_CACHE)."""
        return C.abf_plan_rows(self.plan)

    def bounds_violation(self):
        """First pixel index (y W + x) whose taps would have left the lattice
        box, or -1; only for filters created with debug_bounds=True."""
        return C.abf_debug_bounds_violation(self.plan)


class Batch:
    """Many exact-form filters run as one batch: the non-adaptive step of all
    images in one launch per pass and (limbs, order, input type) group
    (abf_integrate_batch), then one persistent launch of the adaptive step per
    (order, limbs) group over all images (abf_filter_batch)."""

    def __init__(self, filters, device=None):
        self.filters = list(filters)
        self.device = torch.device(device or "cuda")
        self.ws = torch.zeros(256, dtype=torch.uint8, device=self.device)
        self.ws_int = torch.zeros(256, dtype=torch.uint8, device=self.device)

    def integrate(self, images, stream=None):
        jobs = []
        for flt, f in zip(self.filters, images):
            jobs.append(C.abf_integrate_job(flt.plan.value, f.data_ptr(), flt._check_f(f), flt.g.data_ptr(),
                                            flt.ws.data_ptr()))
        C.abf_integrate_batch(jobs, self.ws_int, stream)

    def __call__(self, images, scales, outs, stream=None):
        self.integrate(images, stream)
        jobs = []
        for flt, sc, o in zip(self.filters, scales, outs):
            flt._check_scales(sc)
            jobs.append(C.abf_job(flt.plan.value, flt.g.data_ptr(), sc.data_ptr(), flt.W * 16, o.data_ptr(),
                                  flt.W * o.element_size()))
        C.abf_filter_batch(jobs, self.ws, stream)
        return outs

    def autotune(self, images, scales, outs, stream=None):
        """Integrate, then time the batch launch at 4, 8 and 16 rows per CTA and
        cache the fastest for batches of this composition; returns (rows, [ms x 3])."""
        self.integrate(images, stream)
        jobs = []
        for flt, sc, o in zip(self.filters, scales, outs):
            flt._check_scales(sc)
            jobs.append(C.abf_job(flt.plan.value, flt.g.data_ptr(), sc.data_ptr(), flt.W * 16, o.data_ptr(),
                                  flt.W * o.element_size()))
        return C.abf_batch_autotune(jobs, self.ws, stream)


def make_desc(width, height, n, in_dtype, scale_kind="c4", q_bits=8, frac_bits=0, max_scale=8.0, out="f64",
              form="exact", min_scale=0.0, value_bound=0.0, max_scale_product=0.0, directions=4, model_boxes=0):
    d = C.abf_desc()
    d.width, d.height, d.order_n = int(width), int(height), int(n)
    d.in_dtype = _DT[in_dtype]
    d.out_dtype = _OUT[out][0]
    d.form = C.FORMS[form]
    d.scale_kind = C.SCALE_KINDS[scale_kind]
    d.q_bits = int(q_bits)
    d.in_frac_bits = int(frac_bits)
    d.flags = 0
    d.max_scale = float(max_scale)
    d.min_scale = float(min_scale)
    d.value_bound = float(value_bound)
    d.max_scale_product = float(max_scale_product)
    d.directions = int(directions)
    d.model_boxes = int(model_boxes)
    return d


class Server:
    """The library's request loop (abf_server_*): jobs from host memory,
    admitted by device-memory footprint, run concurrently on their own streams,
    integrated images optionally kept resident by image id."""

    def __init__(self, hbm_budget, max_inflight=4, device=None, group_mesh=False):
        """group_mesh: jobs admitted together share one batched launch of the
        adaptive step (ABF_SERVER_GROUP_MESH)."""
        self.device = torch.device(device or "cuda")
        with torch.cuda.device(self.device):
            self.h = C.abf_server_create(hbm_budget, max_inflight,
                                         C.ABF_SERVER_GROUP_MESH if group_mesh else 0)
        self.keep = {}

    def submit(self, desc, f, scales, out, image_id=0):
        """f, scales, out: CPU tensors (pinned for overlapping copies); f may be
        None when the image is resident under image_id."""
        req = C.abf_request()
        req.desc = desc
        req.h_f = f.data_ptr() if f is not None else None
        req.f_pitch = desc.width * (f.element_size() if f is not None else 0)
        req.h_scales = scales.data_ptr()
        req.scale_pitch = desc.width * 16
        req.h_s = out.data_ptr()
        req.s_pitch = desc.width * out.element_size()
        req.image_id = int(image_id)
        t = C.abf_submit(self.h, req)
        self.keep[t] = (f, scales, out)
        return t

    def wait(self, ticket, timeout_s=None):
        st = C.abf_wait(self.h, ticket, -1 if timeout_s is None else int(timeout_s * 1e6))
        self.keep.pop(ticket, None)
        return dict(t_submit_us=st.t_submit_us, t_admit_us=st.t_admit_us, t_done_us=st.t_done_us,
                    resident_hit=st.resident_hit, status=st.status, device_status=st.device_status,
                    t_gpu_start_us=st.t_gpu_start_us, t_gpu_end_us=st.t_gpu_end_us)

    def poll(self, ticket):
        done, st = C.abf_poll(self.h, ticket)
        return done

    def pause(self, paused=True):
        C.abf_server_pause(self.h, paused)

    def stats(self):
        return C.abf_server_stats(self.h)

    def close(self):
        if self.h is not None:
            C.abf_server_destroy(self.h)
            self.h = None


class AdaptiveFilter1D:
    """The 1-D scale-adaptive B-spline filter of Sec. 3 on `count` signals of
    `length` samples (abf1d_integrate + abf1d_filter).  n1 is the degree of
    the signal model (0..5; from 2 on the samples are interpolated, c = f *
    (b^{n1})^-1 rounded to the 2^-frac_bits grid), n2 that of the analysis
    B-spline (0..3)."""

    def __init__(self, length, count, n1, n2, in_dtype, q_bits=8, frac_bits=0, max_scale=8.0, value_bound=0.0,
                 out="f64", device=None):
        self.device = torch.device(device or "cuda")
        self.length, self.count = int(length), int(count)
        self.in_dtype = in_dtype
        self.out_code, self.out_dtype = _OUT[out]
        d = C.abf1d_desc()
        d.length, d.count, d.n1, d.n2 = self.length, self.count, int(n1), int(n2)
        d.in_dtype, d.out_dtype = _DT[in_dtype], self.out_code
        d.q_bits, d.in_frac_bits = int(q_bits), int(frac_bits)
        d.max_scale, d.value_bound = float(max_scale), float(value_bound)
        self.desc = d
        self.plan = None
        with torch.cuda.device(self.device):
            self.plan = C.abf1d_plan_create(d)
        self.info = C.abf1d_plan_query(self.plan)
        self.limbs = self.info["limbs"]
        self.g = torch.empty(max(self.info["integrated_bytes"], 16), dtype=torch.uint8, device=self.device)

    def close(self):
        if self.plan is not None:
            C.abf1d_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, t, dtype, what):
        if t.device != self.device or t.dtype != dtype or tuple(t.shape) != (self.count, self.length) \
                or t.stride(1) != 1:
            raise ValueError("%s must be a (%d, %d) %s tensor on %s" % (what, self.count, self.length, dtype,
                                                                        self.device))

    def integrate(self, f, stream=None):
        self._check(f, self.in_dtype, "f")
        C.abf1d_integrate(self.plan, f, f.stride(0) * f.element_size(), self.g, stream)

    def filter(self, a, out=None, stream=None):
        self._check(a, torch.float32, "a")
        if out is None:
            out = torch.empty((self.count, self.length), dtype=self.out_dtype, device=self.device)
        C.abf1d_filter(self.plan, self.g, a, a.stride(0) * 4, out, out.stride(0) * out.element_size(), stream)
        return out

    def __call__(self, f, a, out=None, stream=None):
        self.integrate(f, stream)
        return self.filter(a, out, stream)

    def numerators(self, a, stream=None):
        self._check(a, torch.float32, "a")
        num = torch.empty((self.count, self.length, self.limbs), dtype=torch.int64, device=self.device)
        C.abf1d_filter_numerator(self.plan, self.g, a, a.stride(0) * 4, num, self.length * self.limbs * 8, stream)
        return num

    def integrated(self):
        """g as (count, pitch, limbs) int64 (a view of the buffer); element i
        holds g at signal position i - info["left"]."""
        pitch = self.info["g_pitch"]
        return self.g[: self.count * pitch * self.limbs * 8].view(torch.int64).view(self.count, pitch, self.limbs)

    def device_status(self):
        return C.abf1d_last_device_status(self.plan)


def estimate_ellipses(f, rho=2.0, sigma0=4.0, e_max=4.0, stream=None):
    """Per-pixel ellipses (sigma, elongation, cos t, sin t) from the image's
    structure tensor (abf_estimate_ellipses): an (H, W, 4) float32 tensor for
    the filter's "ellipse" scale kind."""
    if f.dim() != 2 or f.stride(1) != 1:
        raise ValueError("f must be a 2-D row-major tensor")
    H, W = f.shape
    ws = torch.empty(max(C.abf_ellipse_ws_bytes(W, H), 16), dtype=torch.uint8, device=f.device)
    out = torch.empty((H, W, 4), dtype=torch.float32, device=f.device)
    C.abf_estimate_ellipses(f, f.stride(0) * f.element_size(), _DT[f.dtype], W, H, float(rho), float(sigma0),
                            float(e_max), ws, out, W * 16, stream)
    return out


def ellipse_product_bound(sigma_max, e_max, n, q_bits=8, max_scale=150.0, device=None, margin=1.01):
    """An upper bound on c1 c2 c3 c4 for every ellipse with sigma <= sigma_max
    and elongation in [1, e_max] (any orientation), for abf_desc's
    max_scale_product: the library's own moment rule measured
    (abf_measure_scales) over a grid of the parameter range at sigma_max (every
    step grows with sigma), times a margin for the space between grid points.
    It depends on the parameter range only, not on an image's scale field;
    the filter still checks every pixel's numerator bound and flags a pixel
    that exceeds it (ABF_DEV_RANGE), so a bound that is too small is never
    silently wrong."""
    import math
    dev = torch.device(device or "cuda")
    ne, nt = 64, 1024
    e = torch.linspace(1.0, float(e_max), ne, dtype=torch.float64)
    th = torch.arange(nt, dtype=torch.float64) * (math.pi / nt)
    f = torch.empty((ne, nt, 4), dtype=torch.float32)
    f[..., 0] = float(sigma_max)
    f[..., 1] = e[:, None].to(torch.float32)
    f[..., 2] = torch.cos(th)[None, :].to(torch.float32)
    f[..., 3] = torch.sin(th)[None, :].to(torch.float32)
    d = C.abf_desc()
    d.width, d.height, d.order_n = nt, ne, int(n)
    d.scale_kind = C.ABF_SCALES_ELLIPSE
    d.q_bits, d.max_scale = int(q_bits), float(max_scale)
    _, prod = C.abf_measure_scales(d, f.to(dev), nt * 16)
    return prod * margin

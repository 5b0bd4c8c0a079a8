"""ctypes binding of libabf (include/abf.h): the same entry points, argument
marshalling only.  Every step of the filter runs in the library's CUDA
kernels; there is no Python or CPU implementation behind these functions.

Loading fails loudly when libabf.so has not been built (``build()`` in
``paper_0908_3861_gb300.build`` or ``__graft_entry__.build()``).
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libabf.so")

ABF_OK, ABF_ERR_INVALID, ABF_ERR_OOM, ABF_ERR_CUDA, ABF_ERR_UNSUPPORTED = 0, 1, 2, 3, 4
ABF_ERR_RANGE, ABF_ERR_TIMEOUT, ABF_ERR_BUSY = 5, 6, 7
STATUS_NAMES = {0: "ABF_OK", 1: "ABF_ERR_INVALID", 2: "ABF_ERR_OOM", 3: "ABF_ERR_CUDA",
                4: "ABF_ERR_UNSUPPORTED", 5: "ABF_ERR_RANGE", 6: "ABF_ERR_TIMEOUT", 7: "ABF_ERR_BUSY"}
ABF_U8, ABF_U16, ABF_F32, ABF_F64 = 0, 1, 2, 3
ABF_FORM_EXACT, ABF_FORM_PLAIN_F64, ABF_FORM_TILE_F32 = 0, 1, 2
ABF_SCALES_C4, ABF_SCALES_A4, ABF_SCALES_ELLIPSE = 0, 1, 2
ABF_DEV_BAD_SCALE, ABF_DEV_RANGE, ABF_DEV_TIMEOUT, ABF_DEV_BAD_INPUT, ABF_DEV_PRECISION = 1, 2, 4, 8, 16
ABF_DEV_BOUNDS = 32
ABF_FLAG_DEBUG_BOUNDS = 1
ABF_FAULT_ALLOC, ABF_FAULT_QUEUE_STALL, ABF_FAULT_BAD_DESC = 1, 2, 3

SCALE_KINDS = {"c4": ABF_SCALES_C4, "a4": ABF_SCALES_A4, "ellipse": ABF_SCALES_ELLIPSE}
FORMS = {"exact": ABF_FORM_EXACT, "plain_f64": ABF_FORM_PLAIN_F64, "tile_f32": ABF_FORM_TILE_F32}


class AbfError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s: %s" % (where, STATUS_NAMES.get(status, status)))


class abf_integrate_job(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("d_f", ctypes.c_void_p), ("f_pitch", ctypes.c_size_t),
                ("d_g", ctypes.c_void_p), ("d_ws", ctypes.c_void_p)]


class abf_job(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("d_g", ctypes.c_void_p), ("d_scales", ctypes.c_void_p),
                ("scale_pitch", ctypes.c_size_t), ("d_s", ctypes.c_void_p), ("s_pitch", ctypes.c_size_t)]


class abf_desc(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("order_n", ctypes.c_int32),
                ("in_dtype", ctypes.c_int32), ("out_dtype", ctypes.c_int32), ("form", ctypes.c_int32),
                ("scale_kind", ctypes.c_int32), ("q_bits", ctypes.c_int32),
                ("in_frac_bits", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("max_scale", ctypes.c_double), ("min_scale", ctypes.c_double),
                ("value_bound", ctypes.c_double), ("max_scale_product", ctypes.c_double),
                ("directions", ctypes.c_int32), ("model_boxes", ctypes.c_int32)]


class abf1d_desc(ctypes.Structure):
    _fields_ = [("length", ctypes.c_int32), ("count", ctypes.c_int32), ("n1", ctypes.c_int32),
                ("n2", ctypes.c_int32), ("in_dtype", ctypes.c_int32), ("out_dtype", ctypes.c_int32),
                ("q_bits", ctypes.c_int32), ("in_frac_bits", ctypes.c_int32),
                ("max_scale", ctypes.c_double), ("value_bound", ctypes.c_double)]


class abf_server_cfg(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("max_inflight", ctypes.c_int32), ("flags", ctypes.c_int32)]


class abf_request(ctypes.Structure):
    _fields_ = [("desc", abf_desc), ("h_f", ctypes.c_void_p), ("f_pitch", ctypes.c_size_t),
                ("h_scales", ctypes.c_void_p), ("scale_pitch", ctypes.c_size_t), ("h_s", ctypes.c_void_p),
                ("s_pitch", ctypes.c_size_t), ("image_id", ctypes.c_uint64)]


class abf_job_stats(ctypes.Structure):
    _fields_ = [("t_submit_us", ctypes.c_double), ("t_admit_us", ctypes.c_double), ("t_done_us", ctypes.c_double),
                ("resident_hit", ctypes.c_int32), ("status", ctypes.c_int32), ("device_status", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("t_gpu_start_us", ctypes.c_double),
                ("t_gpu_end_us", ctypes.c_double)]


_lib = None


def signatures():
    """name -> (argtypes, restype) of every C entry point (include/abf.h)."""
    vp, sz, i32, st = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32, ctypes.c_int
    P = ctypes.POINTER
    return {
        "abf_plan_create": ([P(abf_desc), P(vp)], st),
        "abf_plan_destroy": ([vp], st),
        "abf_plan_query": ([vp, P(sz), P(sz), P(i32), P(i32), P(ctypes.c_int64)], st),
        "abf_integrate": ([vp, vp, sz, vp, vp, vp], st),
        "abf_integrate_noalloc": ([vp, vp, sz, vp, vp], st),
        "abf_filter": ([vp, vp, sz, vp, sz, vp, sz, vp, vp], st),
        "abf_filter_numerator": ([vp, vp, vp, sz, vp, sz, vp, vp], st),
        "abf_prepare_scales": ([vp, vp, sz, vp, sz, vp], st),
        "abf_plan_denominator": ([vp, P(ctypes.c_uint32)], st),
        "abf_last_device_status": ([vp, P(i32)], st),
        "abf_debug_bounds_violation": ([vp, P(ctypes.c_int64)], st),
        "abf_debug_inject_fault": ([i32, i32], st),
        "abf_plan_rows": ([vp, P(i32)], st),
        "abf_measure_scales": ([P(abf_desc), vp, sz, P(ctypes.c_double), P(ctypes.c_double), vp], st),
        "abf_weight_table_host": ([i32, i32, vp, sz, P(sz), P(i32), P(ctypes.c_uint32)], st),
        "abf_filter_batch": ([P(abf_job), i32, vp, sz, vp], st),
        "abf_integrate_batch": ([P(abf_integrate_job), i32, vp, sz, vp], st),
        "abf_integrate_batch_max_jobs": ([], i32),
        "abf_probe_alu": ([i32, P(ctypes.c_double)], st),
        "abf_general_table_host": ([i32, i32, i32, i32, vp, sz, P(sz), P(i32), P(i32), P(i32), P(ctypes.c_uint32)],
                                   st),
        "abf_batch_max_jobs": ([], i32),
        "abf_plan_autotune": ([vp, vp, vp, sz, vp, sz, vp, P(i32), P(ctypes.c_float)], st),
        "abf_batch_autotune": ([P(abf_job), i32, vp, sz, vp, P(i32), P(ctypes.c_float)], st),
        "abf_server_create": ([P(abf_server_cfg), P(vp)], st),
        "abf_submit": ([vp, P(abf_request), P(ctypes.c_uint64)], st),
        "abf_poll": ([vp, ctypes.c_uint64, P(i32), P(abf_job_stats)], st),
        "abf_wait": ([vp, ctypes.c_uint64, ctypes.c_int64, P(abf_job_stats)], st),
        "abf_server_pause": ([vp, i32], st),
        "abf_server_stats": ([vp, P(sz), P(sz), P(i32), P(i32), P(i32)], st),
        "abf_server_destroy": ([vp], st),
        "abf1d_plan_create": ([P(abf1d_desc), P(vp)], st),
        "abf1d_plan_destroy": ([vp], st),
        "abf1d_plan_query": ([vp, P(sz), P(i32), P(i32), P(i32), P(ctypes.c_int64)], st),
        "abf1d_integrate": ([vp, vp, sz, vp, vp], st),
        "abf1d_filter": ([vp, vp, vp, sz, vp, sz, vp], st),
        "abf1d_filter_numerator": ([vp, vp, vp, sz, vp, sz, vp], st),
        "abf1d_last_device_status": ([vp, P(i32)], st),
        "abf1d_prefilter_host": ([i32, P(i32), P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double)], st),
        "abf1d_weight_table_host": ([i32, i32, i32, P(ctypes.c_uint64), sz, P(sz), P(i32), P(i32),
                                     P(ctypes.c_uint64)], st),
        "abf_ellipse_ws_bytes": ([i32, i32], sz),
        "abf_estimate_ellipses": ([vp, sz, i32, i32, i32, ctypes.c_double, ctypes.c_double, ctypes.c_double, vp, sz,
                                   vp, sz, vp], st),
        "abf_debug_starved_lookback": ([vp, vp, vp, vp], st),
        "abf_status_str": ([st], ctypes.c_char_p),
        "abf_version": ([], i32),
    }


def lib():
    """The loaded libabf (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libabf.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    sigs = signatures()
    for name, (args, res) in sigs.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _check(status, where):
    if status != ABF_OK:
        raise AbfError(status, where)


def _stream(stream):
    """cudaStream_t of a torch stream (None: torch's current stream)."""
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


# ----------------------------------------------------------- entry points

def abf_plan_create(desc):
    h = ctypes.c_void_p()
    _check(lib().abf_plan_create(ctypes.byref(desc), ctypes.byref(h)), "abf_plan_create")
    return h


def abf_plan_destroy(plan):
    _check(lib().abf_plan_destroy(plan), "abf_plan_destroy")


def abf_plan_query(plan):
    gb, wb = ctypes.c_size_t(), ctypes.c_size_t()
    halo = (ctypes.c_int32 * 4)()
    limbs = ctypes.c_int32()
    pitch = ctypes.c_int64()
    _check(lib().abf_plan_query(plan, ctypes.byref(gb), ctypes.byref(wb), halo, ctypes.byref(limbs),
                                ctypes.byref(pitch)), "abf_plan_query")
    return dict(integrated_bytes=gb.value, workspace_bytes=wb.value, halo_lrbt=list(halo),
                limbs=limbs.value, g_pitch=pitch.value)


def abf_integrate(plan, f, f_pitch, g, ws, stream=None):
    _check(lib().abf_integrate(plan, _ptr(f), f_pitch, _ptr(g), _ptr(ws), _stream(stream)), "abf_integrate")


def abf_integrate_noalloc(plan, f, f_pitch, g, stream=None):
    """abf_integrate with the library's fixed scratch (no workspace argument)."""
    _check(lib().abf_integrate_noalloc(plan, _ptr(f), f_pitch, _ptr(g), _stream(stream)), "abf_integrate_noalloc")


def abf_filter(plan, src, src_pitch, scales, scale_pitch, s, s_pitch, ws, stream=None):
    _check(lib().abf_filter(plan, _ptr(src), src_pitch, _ptr(scales), scale_pitch, _ptr(s), s_pitch, _ptr(ws),
                            _stream(stream)), "abf_filter")


def abf_filter_numerator(plan, g, scales, scale_pitch, num, num_pitch, ws, stream=None):
    _check(lib().abf_filter_numerator(plan, _ptr(g), _ptr(scales), scale_pitch, _ptr(num), num_pitch, _ptr(ws),
                                      _stream(stream)), "abf_filter_numerator")


def abf_prepare_scales(plan, scales, scale_pitch, C, C_pitch, stream=None):
    _check(lib().abf_prepare_scales(plan, _ptr(scales), scale_pitch, _ptr(C), C_pitch, _stream(stream)),
           "abf_prepare_scales")


def abf_plan_denominator(plan):
    w = (ctypes.c_uint32 * 4)()
    _check(lib().abf_plan_denominator(plan, w), "abf_plan_denominator")
    return sum(int(w[i]) << (32 * i) for i in range(4))


def abf_last_device_status(plan):
    c = ctypes.c_int32()
    _check(lib().abf_last_device_status(plan, ctypes.byref(c)), "abf_last_device_status")
    return c.value


def abf_debug_bounds_violation(plan):
    """The first pixel (y W + x) whose taps would have read outside the lattice
    box, or -1 (plans created with ABF_FLAG_DEBUG_BOUNDS; clears the record)."""
    v = ctypes.c_int64()
    _check(lib().abf_debug_bounds_violation(plan, ctypes.byref(v)), "abf_debug_bounds_violation")
    return v.value


def abf_plan_rows(plan):
    """Rows (warps) per CTA the plan's adaptive step launches with."""
    r = ctypes.c_int32()
    _check(lib().abf_plan_rows(plan, ctypes.byref(r)), "abf_plan_rows")
    return r.value


def abf_debug_inject_fault(kind, count):
    """Arm (count > 0) or disarm (0) a host-side fault: ABF_FAULT_ALLOC,
    ABF_FAULT_QUEUE_STALL or ABF_FAULT_BAD_DESC."""
    _check(lib().abf_debug_inject_fault(int(kind), int(count)), "abf_debug_inject_fault")


def abf_measure_scales(desc, scales, scale_pitch, stream=None):
    """(max step, max product c1 c2 c3 c4) of a scale field (synchronises)."""
    a, p = ctypes.c_double(), ctypes.c_double()
    _check(lib().abf_measure_scales(ctypes.byref(desc), _ptr(scales), scale_pitch, ctypes.byref(a),
                                    ctypes.byref(p), _stream(stream)), "abf_measure_scales")
    return a.value, p.value


def abf_weight_table_host(n, q_bits):
    """(bytes, word_bytes, D) of the host-generated ZP^{*n} table."""
    need, wb = ctypes.c_size_t(), ctypes.c_int32()
    d = (ctypes.c_uint32 * 4)()
    _check(lib().abf_weight_table_host(n, q_bits, None, 0, ctypes.byref(need), ctypes.byref(wb), d),
           "abf_weight_table_host")
    buf = ctypes.create_string_buffer(need.value)
    _check(lib().abf_weight_table_host(n, q_bits, buf, need.value, None, None, None), "abf_weight_table_host")
    return buf.raw, wb.value, sum(int(d[i]) << (32 * i) for i in range(4))


def abf_integrate_batch(jobs, ws, stream=None):
    """jobs: list of abf_integrate_job structures."""
    arr = (abf_integrate_job * len(jobs))(*jobs)
    _check(lib().abf_integrate_batch(arr, len(jobs), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)),
           "abf_integrate_batch")


def abf_general_table_host(directions, n, model_boxes, q_bits, with_weights=True):
    """The generalised interpolation table on the host: returns (weights as
    a list of rows of Python ints, stencil [(dx, dy)], D, wbytes)."""
    need, wb, R = ctypes.c_size_t(), ctypes.c_int32(), ctypes.c_int32()
    st = (ctypes.c_int32 * 512)()
    D4 = (ctypes.c_uint32 * 4)()
    _check(lib().abf_general_table_host(directions, n, model_boxes, q_bits, None, 0, ctypes.byref(need),
                                        ctypes.byref(wb), ctypes.byref(R), st, D4), "abf_general_table_host")
    stencil = [(st[2 * i], st[2 * i + 1]) for i in range(R.value)]
    D = sum(int(D4[i]) << (32 * i) for i in range(4))
    rows = None
    if with_weights:
        buf = (ctypes.c_uint8 * need.value)()
        _check(lib().abf_general_table_host(directions, n, model_boxes, q_bits, buf, need.value, None, None, None,
                                            None, None), "abf_general_table_host")
        raw = bytes(buf)
        w, Rv = wb.value, R.value
        rows = [[int.from_bytes(raw[(r * Rv + c) * w:(r * Rv + c + 1) * w], "little") for c in range(Rv)]
                for r in range(need.value // (w * Rv))]
    return rows, stencil, D, wb.value


def abf_probe_alu(kind):
    v = ctypes.c_double()
    _check(lib().abf_probe_alu(int(kind), ctypes.byref(v)), "abf_probe_alu")
    return v.value


def abf_integrate_batch_max_jobs():
    return lib().abf_integrate_batch_max_jobs()


def abf_filter_batch(jobs, ws, stream=None):
    """jobs: list of abf_job structures."""
    arr = (abf_job * len(jobs))(*jobs)
    _check(lib().abf_filter_batch(arr, len(jobs), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)),
           "abf_filter_batch")


def abf_batch_max_jobs():
    return lib().abf_batch_max_jobs()


ABF_SERVER_GROUP_MESH = 1


def abf_server_create(hbm_budget, max_inflight, flags=0):
    cfg = abf_server_cfg(int(hbm_budget), int(max_inflight), int(flags))
    h = ctypes.c_void_p()
    _check(lib().abf_server_create(ctypes.byref(cfg), ctypes.byref(h)), "abf_server_create")
    return h


def abf_submit(server, req):
    t = ctypes.c_uint64()
    _check(lib().abf_submit(server, ctypes.byref(req), ctypes.byref(t)), "abf_submit")
    return t.value


def abf_poll(server, ticket):
    done = ctypes.c_int32()
    st = abf_job_stats()
    _check(lib().abf_poll(server, ticket, ctypes.byref(done), ctypes.byref(st)), "abf_poll")
    return bool(done.value), st


def abf_wait(server, ticket, timeout_us=-1):
    st = abf_job_stats()
    _check(lib().abf_wait(server, ticket, int(timeout_us), ctypes.byref(st)), "abf_wait")
    return st


def abf_server_pause(server, paused):
    _check(lib().abf_server_pause(server, 1 if paused else 0), "abf_server_pause")


def abf_server_stats(server):
    u, p = ctypes.c_size_t(), ctypes.c_size_t()
    i, q, r = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().abf_server_stats(server, ctypes.byref(u), ctypes.byref(p), ctypes.byref(i), ctypes.byref(q),
                                  ctypes.byref(r)), "abf_server_stats")
    return dict(used=u.value, peak=p.value, inflight=i.value, queued=q.value, resident=r.value)


def abf_server_destroy(server):
    _check(lib().abf_server_destroy(server), "abf_server_destroy")


def abf_status_str(s):
    return lib().abf_status_str(s).decode()


def abf_version():
    return lib().abf_version()


# ------------------------------------------------------ 1-D filter (Sec. 3)

def abf1d_plan_create(desc):
    h = ctypes.c_void_p()
    _check(lib().abf1d_plan_create(ctypes.byref(desc), ctypes.byref(h)), "abf1d_plan_create")
    return h


def abf1d_plan_destroy(plan):
    _check(lib().abf1d_plan_destroy(plan), "abf1d_plan_destroy")


def abf1d_plan_query(plan):
    gb, left, right = ctypes.c_size_t(), ctypes.c_int32(), ctypes.c_int32()
    limbs, pitch = ctypes.c_int32(), ctypes.c_int64()
    _check(lib().abf1d_plan_query(plan, ctypes.byref(gb), ctypes.byref(left), ctypes.byref(right),
                                  ctypes.byref(limbs), ctypes.byref(pitch)), "abf1d_plan_query")
    return dict(integrated_bytes=gb.value, left=left.value, right=right.value, limbs=limbs.value,
                g_pitch=pitch.value)


def abf1d_integrate(plan, f, f_pitch, g, stream=None):
    _check(lib().abf1d_integrate(plan, _ptr(f), f_pitch, _ptr(g), _stream(stream)), "abf1d_integrate")


def abf1d_filter(plan, g, a, a_pitch, s, s_pitch, stream=None):
    _check(lib().abf1d_filter(plan, _ptr(g), _ptr(a), a_pitch, _ptr(s), s_pitch, _stream(stream)), "abf1d_filter")


def abf1d_filter_numerator(plan, g, a, a_pitch, num, num_pitch, stream=None):
    _check(lib().abf1d_filter_numerator(plan, _ptr(g), _ptr(a), a_pitch, _ptr(num), num_pitch, _stream(stream)),
           "abf1d_filter_numerator")


def abf1d_last_device_status(plan):
    v = ctypes.c_int32()
    _check(lib().abf1d_last_device_status(plan, ctypes.byref(v)), "abf1d_last_device_status")
    return v.value


# ----------------------------------------------------------------- autotuner

def abf_plan_autotune(plan, g, scales, scale_pitch, s, s_pitch, stream=None):
    """Times 4, 8 and 16 rows per CTA on this data; returns (choice, [ms x 3])."""
    w, ms = ctypes.c_int32(), (ctypes.c_float * 3)()
    _check(lib().abf_plan_autotune(plan, _ptr(g), _ptr(scales), scale_pitch, _ptr(s), s_pitch, _stream(stream),
                                   ctypes.byref(w), ms), "abf_plan_autotune")
    return w.value, list(ms)


def abf_batch_autotune(jobs, ws, stream=None):
    arr = (abf_job * len(jobs))(*jobs)
    w, ms = ctypes.c_int32(), (ctypes.c_float * 3)()
    _check(lib().abf_batch_autotune(arr, len(jobs), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream),
                                    ctypes.byref(w), ms), "abf_batch_autotune")
    return w.value, list(ms)


def abf1d_prefilter_host(n1):
    """(z, A, hnorm): poles and weights of the inverse interpolation filter."""
    npoles = ctypes.c_int32()
    z, A, hn = (ctypes.c_double * 2)(), (ctypes.c_double * 2)(), ctypes.c_double()
    _check(lib().abf1d_prefilter_host(n1, ctypes.byref(npoles), z, A, ctypes.byref(hn)), "abf1d_prefilter_host")
    return list(z[: npoles.value]), list(A[: npoles.value]), hn.value


def abf1d_weight_table_host(n1, n2, q_bits):
    """(rows x K table as a list of lists, dmin, D) of the 1-D B-spline weights."""
    need, K, dmin, D = ctypes.c_size_t(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_uint64()
    _check(lib().abf1d_weight_table_host(n1, n2, q_bits, None, 0, ctypes.byref(need), ctypes.byref(K),
                                         ctypes.byref(dmin), ctypes.byref(D)), "abf1d_weight_table_host")
    buf = (ctypes.c_uint64 * need.value)()
    _check(lib().abf1d_weight_table_host(n1, n2, q_bits, buf, need.value, None, None, None, None),
           "abf1d_weight_table_host")
    k = K.value
    vals = list(buf)
    return [vals[i:i + k] for i in range(0, len(vals), k)], dmin.value, D.value


# ---------------------------------------------------- scale-map estimation

def abf_ellipse_ws_bytes(width, height):
    return lib().abf_ellipse_ws_bytes(width, height)


def abf_estimate_ellipses(f, f_pitch, in_dtype, width, height, rho, sigma0, e_max, ws, out, out_pitch, stream=None):
    _check(lib().abf_estimate_ellipses(_ptr(f), f_pitch, in_dtype, width, height, rho, sigma0, e_max, _ptr(ws),
                                       ws.numel() * ws.element_size(), _ptr(out), out_pitch, _stream(stream)),
           "abf_estimate_ellipses")


def abf_debug_starved_lookback(plan, g, ws, stream=None):
    _check(lib().abf_debug_starved_lookback(plan, _ptr(g), _ptr(ws), _stream(stream)), "abf_debug_starved_lookback")

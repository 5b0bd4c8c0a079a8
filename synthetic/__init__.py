"""Seeded synthetic inputs for the adaptive box-spline filter.

This module holds none of the filter's arithmetic: it only draws images and
raw per-pixel scale fields (paper scales a_k, or ellipse parameters), and
1-D signals with per-sample scales.  Both the
oracle and the CUDA path consume its output; each applies the scale readings
itself.
"""
from .workloads import (smooth_field, edge_field, image_c1, image_c2, image_c3,
                        image_f32_grid, scales_a4, ellipse_field, workload,
                        batch_workload, smooth_rows, signals_1d, scales_1d,
                        workload_1d, SEED_BASE)

__all__ = ["smooth_field", "edge_field", "image_c1", "image_c2", "image_c3",
           "image_f32_grid", "scales_a4", "ellipse_field", "workload",
           "batch_workload", "smooth_rows", "signals_1d", "scales_1d",
           "workload_1d", "SEED_BASE"]

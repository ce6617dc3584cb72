"""Seeded synthetic workloads for continuous-component normal integration.

This package only synthesises inputs: analytic depth maps, their normal maps
(computed from closed-form surface derivatives), masks and camera intrinsics.
It holds none of the integration method's arithmetic, so both the FP64 CPU
oracle (through the tests) and the CUDA path consume the same arrays.
"""
from .generators import (  # noqa: F401
    Workload, make_workload, workload_names, c1_map, c2_type_map, c3_map, c5_map,
    random_normal_field, plane_map, sphere_map,
)

"""SEPSO planner for GB300 (sm_103a): hand-written CUDA behind a C ABI.

Self-Evolving Particle Swarm Optimization for real-time path planning in dynamic
scenes (Xin, Li, Zhang, Li; arXiv 2308.10169).  ``Planner`` drives the library
``libsepso.so`` (include/sepso.h); ``inputs`` draws seeded synthetic workloads.
The CUDA library is required: nothing here falls back to a CPU implementation.
"""
from .inputs import (AT_OFF, AT_STALL, AT_STD_WINDOW, TABLE_HYPER8, TABLE_HYPER8_PATH, Scene,
                     SepsoConfig, dynamic_workload, sample_hyper, static_workload)

__all__ = ["Planner", "BatchPlanner", "BFPlanner", "Server", "Prior", "SepsoConfig", "Scene", "static_workload", "dynamic_workload",
           "sample_hyper", "TABLE_HYPER8", "TABLE_HYPER8_PATH", "AT_OFF", "AT_STALL",
           "AT_STD_WINDOW"]


def __getattr__(name):
    if name == "Planner":
        from .planner import Planner
        return Planner
    if name == "Server":
        from .planner import Server
        return Server
    if name == "Prior":
        from .prior import Prior
        return Prior
    if name == "BatchPlanner":
        from .planner import BatchPlanner
        return BatchPlanner
    if name == "BFPlanner":
        from .planner import BFPlanner
        return BFPlanner
    raise AttributeError(name)

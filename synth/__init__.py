"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This package draws point clouds, depth frames, agent sets and request streams.
It holds none of the planning method's arithmetic: no voxelisation, no force
law, no integration and no cost.  Both the CUDA path and the oracle receive the
arrays it returns as plain data.
"""

from .scenes import (  # noqa: F401
    sphere_cloud,
    tabletop_scene,
    render_depth_frame,
    camera_pose,
    agent_set,
)
from .workloads import (  # noqa: F401
    PhysicsParams,
    Workspace,
    sphere_workload,
    tabletop_workload,
    batch_workloads,
    adjoint_workload,
    serve_stream,
    ensemble_agents,
    multi_sensor_frames,
)

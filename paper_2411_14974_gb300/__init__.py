"""GB300-native (sm_103a) differentiable tile rasterizer for 3D smooth convexes.

3D Convex Splatting (arXiv 2411.14974), Sec. 3.2: convexes given as K free 3D points are
projected (Eq. 4), their 2D hull becomes lines, delta/sigma are scaled by the camera distance
(Eq. S1/S2), and pixels composite the smooth indicators front to back (Eq. 5).  The compute runs
in the CUDA library behind include/convex_splat.h; this package only marshals arguments.
"""
from .rasterizer import (ARRAYS, PARAMS, WORK_FIELDS, Context, RefineSettings, SceneTensors, Server,  # noqa: F401
                         alu_rates,
                         Settings, State, TrainConfig, Trainer, adam_step, backward, camera_struct, forward,
                         launch_count, loss_l1_dssim, profile_enable, profile_read, refine, render, step_host,
                         step_host_submit, step_host_wait, work_counts)

// Launch shape of collision_kernel<T, N>: thread-block cluster size, plane groups per CTA and
// the CTAs per SM the registers are sized for.  Written by paper_1903_03056_gb300/tune.py from
// timings on the device (record: tuned_shapes.json); edit by re-running the tuner.
#pragma once

DGFS_SHAPE(float, 4, 1, 4)
DGFS_SHAPE(float, 6, 1, 6)
DGFS_SHAPE(float, 8, 1, 8)
DGFS_SHAPE(float, 12, 1, 12)
DGFS_SHAPE3(float, 16, 1, 8, 3)
DGFS_SHAPE3(float, 24, 1, 8, 2)
DGFS_SHAPE3(float, 32, 8, 4, 3)
DGFS_SHAPE3(float, 48, 2, 4, 1)
DGFS_SHAPE(double, 4, 1, 4)
DGFS_SHAPE(double, 6, 1, 6)
DGFS_SHAPE(double, 8, 1, 8)
DGFS_SHAPE(double, 12, 1, 12)
DGFS_SHAPE(double, 16, 1, 8)
DGFS_SHAPE(double, 24, 2, 6)
DGFS_SHAPE(double, 32, 4, 4)
DGFS_SHAPE(double, 48, 4, 1)

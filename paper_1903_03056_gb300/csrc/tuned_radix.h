// Radix schedule of the register line transform per (precision, N): the decimal digits of the
// code, first stage first (442 = radix 4, 4, then 2).  Written by
// paper_1903_03056_gb300/tune.py --radix from timings on the device (record:
// tuned_shapes.json, keys "radix/..."); edit by re-running the tuner.
#pragma once

DGFS_RADIX(float, 4, 4)
DGFS_RADIX(float, 6, 23)
DGFS_RADIX(float, 8, 42)
DGFS_RADIX(float, 12, 43)
DGFS_RADIX(float, 16, 28)
DGFS_RADIX(float, 24, 38)
DGFS_RADIX(float, 32, 228)
DGFS_RADIX(float, 48, 344)
DGFS_RADIX(double, 4, 4)
DGFS_RADIX(double, 6, 23)
DGFS_RADIX(double, 8, 42)
DGFS_RADIX(double, 12, 43)
DGFS_RADIX(double, 16, 44)
DGFS_RADIX(double, 24, 423)
DGFS_RADIX(double, 32, 442)
DGFS_RADIX(double, 48, 443)

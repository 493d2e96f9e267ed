// Mixed form, slices of width 32 < W <= 64 (the two-chain sweep, two rows per lane).
#include "solve_device.cuh"

DY_SOLVE_VARIANT(float, 64)

// Mixed form, slices of width 16 < W <= 32 (the two-chain single-warp sweep).
#include "solve_device.cuh"

DY_SOLVE_VARIANT(float, 32)

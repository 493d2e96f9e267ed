// FP64 form (complex128 sweeps): the 8-warp sweep for W <= 64 and the
// row-chunked sweep for W > 64; a translation unit of its own so it compiles
// in parallel with the mixed form's variants.
#include "solve_device.cuh"

DY_SOLVE_VARIANT(double, 0)
DY_SOLVE_VARIANT(double, 64)

template <>
cudaError_t launch_xmatvec<double>(const Geo& g, const Bufs& b, int K, int j, int mixed, int ncols, cudaStream_t st) {
  if (sweep_form<double>(g) == 0) return run_xmatvec<double, 0>(g, b, K, j, mixed, ncols, st);
  return run_xmatvec<double, 64>(g, b, K, j, mixed, ncols, st);
}

template <>
cudaError_t launch_bsolve<double>(const Geo& g, const Bufs& b, int K, const cxd* q_dd, cxd* w_dd,
                                  cudaStream_t st) {
  if (sweep_form<double>(g) == 0) return run_bsolve<double, 0>(g, b, K, q_dd, w_dd, st);
  return run_bsolve<double, 64>(g, b, K, q_dd, w_dd, st);
}

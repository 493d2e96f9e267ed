// Mixed form (complex64 sweeps): the dispatch over sweep forms and the
// W > 64 (row-chunked) and W <= 16 variants.  The W <= 32 and W <= 64
// variants are compiled in k_xmatvec_c64_w32.cu and k_xmatvec_c64_w64.cu.
#include "solve_device.cuh"

DY_SOLVE_VARIANT(float, 0)
DY_SOLVE_VARIANT(float, 16)

template <>
cudaError_t launch_xmatvec<float>(const Geo& g, const Bufs& b, int K, int j, int mixed, int ncols, cudaStream_t st) {
  switch (sweep_form<float>(g)) {
    case 0: return run_xmatvec<float, 0>(g, b, K, j, mixed, ncols, st);
    case 16: return run_xmatvec<float, 16>(g, b, K, j, mixed, ncols, st);
    case 32: return run_xmatvec<float, 32>(g, b, K, j, mixed, ncols, st);
    default: return run_xmatvec<float, 64>(g, b, K, j, mixed, ncols, st);
  }
}

template <>
cudaError_t launch_bsolve<float>(const Geo& g, const Bufs& b, int K, const cxd* q_dd, cxd* w_dd,
                                 cudaStream_t st) {
  switch (sweep_form<float>(g)) {
    case 0: return run_bsolve<float, 0>(g, b, K, q_dd, w_dd, st);
    case 16: return run_bsolve<float, 16>(g, b, K, q_dd, w_dd, st);
    case 32: return run_bsolve<float, 32>(g, b, K, q_dd, w_dd, st);
    default: return run_bsolve<float, 64>(g, b, K, q_dd, w_dd, st);
  }
}

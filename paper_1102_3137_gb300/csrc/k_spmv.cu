// Batched lattice-stencil product y = H(i w_k) x for K frequencies at once
// (Eq. 1: H_ij = t on nearest neighbours, H_ii = i w + mu - V_i - Sigma_i).
// H is never stored: the diagonal is rebuilt from V, Sigma and w on the fly.
// Natural site order, x fastest; one thread per site, grid-stride, so a warp
// reads 32 consecutive x (and its +-1, +-Lx, +-Lx*Ly neighbours) coalesced.
#include "dyson_common.cuh"

namespace {

template <typename R>
__global__ void __launch_bounds__(DY_THREADS) k_spmv(Geo g, const double* __restrict__ V,
                                                     const double* __restrict__ omega,
                                                     const cxd* __restrict__ sigma,
                                                     const cx<R>* __restrict__ x,
                                                     cx<R>* __restrict__ y) {
  const int kf = blockIdx.y;
  const int N = g.N, Lx = g.Lx, Ly = g.Ly, Lz = g.Lz, LxLy = Lx * Ly;
  const cx<R>* xk = x + (size_t)kf * N;
  cx<R>* yk = y + (size_t)kf * N;
  const cxd* sk = sigma + (size_t)kf * N;
  const double w = omega[kf];
  const R t = (R)g.t;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
    const int xi = n % Lx, rest = n / Lx, yi = rest % Ly, zi = rest / Ly;
    const cxd s = sk[n];
    const cx<R> d = g.eta > 0.0 ? cx<R>{(R)(w + g.mu - V[n] - s.x), (R)(g.eta - s.y)}
                                : cx<R>{(R)(g.mu - V[n] - s.x), (R)(w - s.y)};
    cx<R> nb = {0, 0};
    if (xi > 0) nb = nb + xk[n - 1];
    if (xi < Lx - 1) nb = nb + xk[n + 1];
    if (yi > 0) nb = nb + xk[n - Lx];
    if (yi < Ly - 1) nb = nb + xk[n + Lx];
    if (zi > 0) nb = nb + xk[n - LxLy];
    if (zi < Lz - 1) nb = nb + xk[n + LxLy];
    yk[n] = d * xk[n] + t * nb;
  }
}

}  // namespace

template <typename R>
cudaError_t launch_spmv(const Geo& g, const double* V, const double* omega, const cxd* sigma,
                        const cx<R>* x, cx<R>* y, int K, cudaStream_t st) {
  int bx = (g.N + DY_THREADS - 1) / DY_THREADS;
  k_spmv<R><<<dim3(bx, K), DY_THREADS, 0, st>>>(g, V, omega, sigma, x, y);
  return cudaGetLastError();
}
template cudaError_t launch_spmv<double>(const Geo&, const double*, const double*, const cxd*,
                                         const cxd*, cxd*, int, cudaStream_t);
template cudaError_t launch_spmv<float>(const Geo&, const double*, const double*, const cxd*,
                                        const cxf*, cxf*, int, cudaStream_t);

// Batched lattice-stencil product y = H(i w_k) x for K frequencies at once
// (Eq. 1: H_ij = t on nearest neighbours, H_ii = i w + mu - V_i - Sigma_i; on
// the real axis i w -> w + i eta).  H is never stored: the diagonal is
// rebuilt from V, Sigma and w on the fly.  Natural site order, x fastest.
//
// Thread (tx, ty) of a block takes two consecutive x sites of one lattice
// row (row = y + Ly z): the x pair, its two x neighbours and the pairs one
// row and one plane away are 16-byte or 8-byte loads, coalesced over tx, and
// the grid (x pairs, rows, frequencies) needs no per-site division.  The
// FP64 inputs (Sigma, V) are converted first and the diagonal is formed in
// R; in the complex64 form the conversions are integer operations on the bit
// patterns (d2f_bits), so nothing runs on the FP64 pipe (1/64 of FP32 here).
#include "dyson_common.cuh"

namespace {

template <typename R>
__global__ void __launch_bounds__(256) k_spmv(Geo g, const double* __restrict__ V,
                                              const double* __restrict__ omega,
                                              const cxd* __restrict__ sigma,
                                              const cx<R>* __restrict__ x, cx<R>* __restrict__ y,
                                              bool vec) {
  using C = cx<R>;
  const int kf = blockIdx.z;
  const int Lx = g.Lx, Ly = g.Ly, Lz = g.Lz, LxLy = Lx * Ly, N = g.N;
  const int xs = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int row = blockIdx.y * blockDim.y + threadIdx.y;
  if (xs >= Lx || row >= Ly * Lz) return;
  const int yi = row % Ly, zi = row / Ly;
  const int n = xs + Lx * row;
  const bool two = xs + 1 < Lx;
  const C* xk = x + (size_t)kf * N;
  const cxd* sk = sigma + (size_t)kf * N;
  auto cvt = [](double v) -> R {
    if constexpr (sizeof(R) == 4) return d2f_bits(v);   // integer unit, not the FP64 pipe
    else return v;
  };
  const R t = cvt(g.t), wr = cvt(omega[kf]), er = cvt(g.eta), mur = cvt(g.mu);
  const bool real_axis = g.real_axis != 0;
  // vec (complex64, Lx even, x and y 16-byte aligned): every pair starts on a
  // 16-byte boundary (n is even)
  auto ld2 = [&](int m, C& p0, C& p1) {
    if (vec) {
      const float4 v = *reinterpret_cast<const float4*>(xk + m);
      p0 = C{(R)v.x, (R)v.y};
      p1 = C{(R)v.z, (R)v.w};
    } else {
      p0 = xk[m];
      p1 = two ? xk[m + 1] : C{0, 0};
    }
  };
  C x0, x1;
  ld2(n, x0, x1);
  C a0 = {0, 0}, a1 = {0, 0};
  if (xs > 0) a0 = a0 + xk[n - 1];
  a0 = a0 + x1;
  a1 = a1 + x0;
  if (xs + 2 < Lx) a1 = a1 + xk[n + 2];
  auto pair = [&](int m) {
    C p0, p1;
    ld2(m, p0, p1);
    a0 = a0 + p0;
    a1 = a1 + p1;
  };
  if (yi > 0) pair(n - Lx);
  if (yi < Ly - 1) pair(n + Lx);
  if (zi > 0) pair(n - LxLy);
  if (zi < Lz - 1) pair(n + LxLy);
  auto diag = [&](int m) {
    const cxd s = sk[m];
    const R vr = cvt(V[m]), sr = cvt(s.x), si = cvt(s.y);
    return real_axis ? C{wr + mur - vr - sr, er - si} : C{mur - vr - sr, wr - si};
  };
  C* yk = y + (size_t)kf * N;
  const C y0 = diag(n) * x0 + t * a0;
  if (vec) {
    const C y1 = diag(n + 1) * x1 + t * a1;
    *reinterpret_cast<float4*>(yk + n) = make_float4((float)y0.x, (float)y0.y, (float)y1.x, (float)y1.y);
  } else {
    yk[n] = y0;
    if (two) yk[n + 1] = diag(n + 1) * x1 + t * a1;
  }
}

}  // namespace

template <typename R>
cudaError_t launch_spmv(const Geo& g, const double* V, const double* omega, const cxd* sigma,
                        const cx<R>* x, cx<R>* y, int K, cudaStream_t st) {
  const int rows = g.Ly * g.Lz;
  const int pairs = (g.Lx + 1) / 2;
  const int tx = pairs >= 32 ? 32 : (pairs >= 16 ? 16 : 8);
  const dim3 block(tx, 256 / tx);
  const dim3 grid((pairs + tx - 1) / tx, (rows + block.y - 1) / block.y, K);
  if (grid.y > 65535 || K > 65535) return cudaErrorInvalidConfiguration;
  const bool vec = sizeof(R) == 4 && (g.Lx % 2) == 0 && (reinterpret_cast<uintptr_t>(x) % 16) == 0 &&
                   (reinterpret_cast<uintptr_t>(y) % 16) == 0;
  k_spmv<R><<<grid, block, 0, st>>>(g, V, omega, sigma, x, y, vec);
  return cudaGetLastError();
}
template cudaError_t launch_spmv<double>(const Geo&, const double*, const double*, const cxd*,
                                         const cxd*, cxd*, int, cudaStream_t);
template cudaError_t launch_spmv<float>(const Geo&, const double*, const double*, const cxd*,
                                        const cxf*, cxf*, int, cudaStream_t);

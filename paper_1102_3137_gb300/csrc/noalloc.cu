// dyson_subdomain_diag_noalloc: diag(blkdiag(B^-1, 0)) for callers that cannot
// allocate device memory.
//
// Some callers must not call cudaMalloc at all: code running inside a
// captured or replayed CUDA graph that must stay allocation-free, hosts with a
// fixed memory budget that is reserved up front, and embedders that hand the
// library only the buffers they own.  This entry point serves them: it takes
// the caller's device inputs and output and keeps everything else (the dd
// index map, the subdomain slice factors and the subdomain-first diagonal) in
// one file-scope device array of fixed size.
//
// Every GPU that loads this library holds that array until the process exits.
// All calls share it and it keeps the last call's contents; calls whose work
// overlaps on the GPU (two streams, two threads) race on it and must be
// serialised by the caller.  Nothing in it needs clearing between calls: each
// call writes every byte it later reads.
#include <cstring>
#include <mutex>
#include <string>

#include "dyson.h"
#include "dyson_common.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)DYSON_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[DYSON_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_scratch_mu;
void* g_scratch_dev[kMaxDevices] = {};

// Device address of the scratch array on device `dev` (the current device).
// The host-side name of the array is only a stand-in; kernels need this address.
cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return cudaSuccess;
}

// natural index of every subdomain-first slot (-1 on padding), from the geometry
__global__ void k_dd2nat(Geo g, int* dd2nat) {
  const size_t nsub = (size_t)g.Lx * g.W;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < (size_t)g.Ndd;
       k += (size_t)gridDim.x * blockDim.x) {
    int v = -1;
    if (k < (size_t)g.ifc_off) {
      const int i = (int)(k / nsub);
      const int rem = (int)(k - i * nsub);
      const int s = rem / g.W, j = rem - s * g.W;
      if (j < g.T * g.h[i]) v = sub_nat(g, i, s, j);
    } else {
      const size_t o = k - g.ifc_off;
      const int l = (int)(o / g.A), a = (int)(o - (size_t)l * g.A);
      v = a + g.A * g.ylayer[l];
    }
    dd2nat[k] = v;
  }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" int dyson_subdomain_diag_noalloc(const dyson_geometry* geom, int K, const double* omega,
                                            const double* V, const double* sigma, double* diagB,
                                            void* stream) {
  if (!geom || !omega || !V || !sigma || !diagB || K < 1)
    return dyson_internal_fail(DYSON_E_BAD_ARG, "noalloc: NULL pointer or K < 1");
  if (geom->precision != DYSON_FP64)
    return dyson_internal_fail(DYSON_E_BAD_ARG, "noalloc: only the FP64 form is available");
  int heights[DY_MAXP] = {0};
  int m = 0, ndd = 0;
  int rc = dyson_partition(geom, heights, &m, &ndd, nullptr);
  if (rc) return rc;
  Geo g;
  std::memset(&g, 0, sizeof(g));
  g.dim = geom->dim;
  g.Lx = geom->L[0];
  g.Ly = geom->L[1];
  g.Lz = geom->dim == 3 ? geom->L[2] : 1;
  g.N = g.Lx * g.Ly * g.Lz;
  g.p = geom->p;
  g.T = geom->dim == 3 ? g.Ly : 1;
  g.A = g.Lx * g.T;
  g.Ls = geom->dim == 3 ? g.Lz : g.Ly;
  int c = 0, hmax = 0;
  for (int i = 0; i < g.p; ++i) {
    g.h[i] = heights[i];
    g.s0[i] = c;
    c += g.h[i];
    if (g.h[i] > hmax) hmax = g.h[i];
    if (i < g.p - 1) g.ylayer[i] = c++;
  }
  g.W = (g.T * hmax + 3) & ~3;
  if (g.W > DY_MAXW_SMEM)
    return dyson_internal_fail(DYSON_E_UNSUPPORTED, "noalloc: slice width above 64");
  g.Ndd = ndd;
  g.ifc_off = g.p * g.Lx * g.W;
  g.t = geom->t;
  g.mu = geom->mu;
  if (!(geom->eta >= 0.0)) return dyson_internal_fail(DYSON_E_BAD_ARG, "noalloc: eta must be >= 0");
  g.eta = geom->eta;
  g.real_axis = geom->eta > 0.0 ? 1 : 0;
  g.nb = 1;
  const size_t b_map = align256((size_t)ndd * sizeof(int));
  const size_t b_diag = align256((size_t)K * ndd * sizeof(cxd));
  const size_t b_g = align256((size_t)K * g.p * g.Lx * g.W * g.W * sizeof(cxd));
  const size_t need = b_map + b_diag + b_g;
  if (need > kScratchBytes)
    return dyson_internal_fail(
        DYSON_E_BUDGET, "noalloc: this geometry and K need " + std::to_string(need) +
                            " bytes of scratch; the fixed scratch holds " +
                            std::to_string(kScratchBytes) + " (use fewer frequencies per call)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return dyson_internal_fail(DYSON_E_CUDA, "noalloc: no usable current device");
  void* base = nullptr;
  e = scratch_address(dev, &base);
  if (e != cudaSuccess)
    return dyson_internal_fail(DYSON_E_CUDA, std::string("noalloc: cudaGetSymbolAddress: ") +
                                                 cudaGetErrorString(e));
  unsigned char* sc = static_cast<unsigned char*>(base);
  Bufs b;
  std::memset(&b, 0, sizeof(b));
  b.V = V;
  b.omega = omega;
  b.sigma = reinterpret_cast<const cxd*>(sigma);
  int* dd2nat = reinterpret_cast<int*>(sc);
  b.dd2nat = dd2nat;
  b.diagB = reinterpret_cast<cxd*>(sc + b_map);
  b.g = sc + b_map + b_diag;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int bx = (ndd + 255) / 256;
  if (bx > 1024) bx = 1024;
  k_dd2nat<<<bx, 256, 0, st>>>(g, dd2nat);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_factor<double, double>(g, b, K, st);
  if (e == cudaSuccess) e = launch_scatter(g, b, K, b.diagB, reinterpret_cast<cxd*>(diagB), ndd, st);
  if (e != cudaSuccess)
    return dyson_internal_fail(DYSON_E_CUDA, std::string("noalloc: launch: ") + cudaGetErrorString(e));
  return DYSON_OK;
}

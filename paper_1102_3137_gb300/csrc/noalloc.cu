// dyson_subdomain_diag_noalloc: diag(blkdiag(B^-1, 0)) for callers that cannot
// allocate device memory.
//
// Some host programs hand the solver no allocator at all: a simulation that
// carves all of its device memory out of one pool at start-up and treats any
// later cudaMalloc as a failure (the pool may leave nothing free, and an
// allocation can stall the device), or a plugin living inside another
// framework that owns every device buffer and only lends it input and output
// arrays.  This entry point serves them: it takes the caller's device inputs
// and output and keeps everything else (the index map from the internal
// subdomain-first layout to natural order, the subdomain slice factors and
// the subdomain-first diagonal) in one file-scope device array of fixed size.
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

// The fields of Geo this path reads, from the caller's geometry, with the
// checks they need and nothing allocated: heights of the p strips/slabs along
// the slow axis (the first (L_slow - p + 1) mod p one layer taller), the
// interface layers between them, the padded slice width and the
// subdomain-first vector length.  Only dim, L, t, mu, p, precision and eta
// are read; the other fields of the geometry play no part here.
int noalloc_geo(const dyson_geometry* in, Geo* out) {
  if (in->precision != DYSON_FP64)
    return dyson_internal_fail(DYSON_E_BAD_ARG, "noalloc: only the FP64 form is available");
  if (in->dim != 2 && in->dim != 3) return dyson_internal_fail(DYSON_E_BAD_ARG, "noalloc: dim must be 2 or 3");
  Geo g;
  std::memset(&g, 0, sizeof(g));
  g.dim = in->dim;
  g.Lx = in->L[0];
  g.Ly = in->L[1];
  g.Lz = in->dim == 3 ? in->L[2] : 1;
  if (g.Lx < 1 || g.Ly < 1 || g.Lz < 1)
    return dyson_internal_fail(DYSON_E_BAD_ARG, "noalloc: lattice extents must be >= 1");
  const long long N = (long long)g.Lx * g.Ly * g.Lz;
  if (N > (1LL << 30)) return dyson_internal_fail(DYSON_E_UNSUPPORTED, "noalloc: lattice too large");
  g.N = (int)N;
  g.p = in->p;
  if (g.p < 1 || g.p > DY_MAXP) return dyson_internal_fail(DYSON_E_BAD_ARG, "noalloc: p must be in 1..16");
  g.T = in->dim == 3 ? g.Ly : 1;
  g.A = g.Lx * g.T;
  g.Ls = in->dim == 3 ? g.Lz : g.Ly;
  if (g.Ls - (g.p - 1) < g.p)
    return dyson_internal_fail(DYSON_E_BAD_ARG, "noalloc: too many subdomains for the slow axis");
  const int base = (g.Ls - (g.p - 1)) / g.p, extra = (g.Ls - (g.p - 1)) % g.p;
  int c = 0, hmax = 0;
  for (int i = 0; i < g.p; ++i) {
    g.h[i] = base + (i < extra ? 1 : 0);
    g.s0[i] = c;
    c += g.h[i];
    if (g.h[i] > hmax) hmax = g.h[i];
    if (i < g.p - 1) g.ylayer[i] = c++;
  }
  g.W = (g.T * hmax + 3) & ~3;
  if (g.W > DY_MAXW_SMEM)
    return dyson_internal_fail(DYSON_E_UNSUPPORTED, "noalloc: slice width above 64");
  const long long ndd = (long long)g.p * g.Lx * g.W + (long long)(g.p - 1) * g.A;
  if (ndd > (1LL << 30)) return dyson_internal_fail(DYSON_E_UNSUPPORTED, "noalloc: lattice too large");
  g.Ndd = (int)ndd;
  g.ifc_off = g.p * g.Lx * g.W;
  g.t = in->t;
  g.mu = in->mu;
  if (!(in->eta >= 0.0)) return dyson_internal_fail(DYSON_E_BAD_ARG, "noalloc: eta must be >= 0");
  g.eta = in->eta;
  g.real_axis = in->eta > 0.0 ? 1 : 0;
  g.nb = 1;
  *out = g;
  return DYSON_OK;
}

// A caller's pointer must be device (or managed) memory of the current device:
// the kernels run there and dereference it.
int check_device_ptr(const void* ptr, int dev, const char* what) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return dyson_internal_fail(DYSON_E_BAD_ARG, std::string("noalloc: cannot query ") + what);
  }
  if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev)
    return dyson_internal_fail(DYSON_E_BAD_ARG, std::string("noalloc: ") + what +
                                                    " is not device memory of the current device");
  return DYSON_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" int dyson_subdomain_diag_noalloc(const dyson_geometry* geom, int K, const double* omega,
                                            const double* V, const double* sigma, double* diagB,
                                            void* stream) {
  if (!geom || !omega || !V || !sigma || !diagB || K < 1)
    return dyson_internal_fail(DYSON_E_BAD_ARG, "noalloc: NULL pointer or K < 1");
  Geo g;
  int rc = noalloc_geo(geom, &g);
  if (rc) return rc;
  if (K > 65535)   // frequencies run on gridDim.y of the factor launch
    return dyson_internal_fail(DYSON_E_BAD_ARG, "noalloc: K must be at most 65535");
  const int ndd = g.Ndd;
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
  {
    const void* ptrs[4] = {omega, V, sigma, diagB};
    const char* names[4] = {"omega", "V", "sigma", "diagB"};
    for (int k = 0; k < 4; ++k) {
      int rc2 = check_device_ptr(ptrs[k], dev, names[k]);
      if (rc2) return rc2;
    }
  }
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

// Host side of the C ABI declared in include/dyson.h: argument checks, the
// domain-decomposition maps (Sec. 2.2, Fig. 1 right), the plan's device
// arena, and the solve sequence replayed from a captured CUDA graph:
//   init -> factor (diag(B^-1), g_s) -> preconditioner ->
//   k x [X-matvec -> Lanczos step + assembly] -> diag(G) out.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "dyson.h"
#include "dyson_common.cuh"
#include "host_internal.h"

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CK(call)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess)                                                        \
      return fail(DYSON_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct Part {
  Geo g;
  std::vector<int> dd2nat;
  int m;
};

// Validate a geometry and build the subdomain-first ordering.
int build_part(const dyson_geometry* in, Part* out, bool gpu) {
  if (!in) return fail(DYSON_E_BAD_ARG, "geometry is NULL");
  Geo g;
  std::memset(&g, 0, sizeof(g));
  if (in->dim != 2 && in->dim != 3) return fail(DYSON_E_BAD_ARG, "dim must be 2 or 3");
  g.dim = in->dim;
  g.Lx = in->L[0];
  g.Ly = in->L[1];
  g.Lz = in->dim == 3 ? in->L[2] : 1;
  if (g.Lx < 1 || g.Ly < 1 || g.Lz < 1) return fail(DYSON_E_BAD_ARG, "lattice extents must be >= 1");
  long long N = (long long)g.Lx * g.Ly * g.Lz;
  if (N > (1LL << 30)) return fail(DYSON_E_UNSUPPORTED, "lattice too large");
  g.N = (int)N;
  g.p = in->p;
  g.T = in->dim == 3 ? g.Ly : 1;
  g.A = g.Lx * g.T;
  g.Ls = in->dim == 3 ? g.Lz : g.Ly;
  if (g.p < 1 || g.p > DY_MAXP) return fail(DYSON_E_BAD_ARG, "p must be in 1..16");
  if (g.Ls - (g.p - 1) < g.p) return fail(DYSON_E_BAD_ARG, "too many subdomains for the slow axis");
  const int base = (g.Ls - (g.p - 1)) / g.p, extra = (g.Ls - (g.p - 1)) % g.p;
  int c = 0, hmax = 0;
  for (int i = 0; i < g.p; ++i) {
    g.h[i] = base + (i < extra ? 1 : 0);
    g.s0[i] = c;
    c += g.h[i];
    if (g.h[i] > hmax) hmax = g.h[i];
    if (i < g.p - 1) g.ylayer[i] = c++;
  }
  g.W = (g.T * hmax + 3) & ~3;   // multiple of 4: 16-byte aligned rows and bulk copies
  if (gpu && g.W > DY_MAXW)
    return fail(DYSON_E_UNSUPPORTED, "slice width " + std::to_string(g.W) + " exceeds " +
                                         std::to_string(DY_MAXW));
  long long ndd = (long long)g.p * g.Lx * g.W + (long long)(g.p - 1) * g.A;
  if (ndd > (1LL << 30)) return fail(DYSON_E_UNSUPPORTED, "lattice too large");
  g.Ndd = (int)ndd;
  g.ifc_off = g.p * g.Lx * g.W;
  g.penta = (g.T == 1 && g.W <= DY_MAXW_SMEM) ? 1 : 0;
  if (in->precond < DYSON_PRECOND_AUTO || in->precond > DYSON_PRECOND_LAYER)
    return fail(DYSON_E_BAD_ARG, "precond must be DYSON_PRECOND_AUTO, _BANDED or _LAYER");
  {
    // 2D strips: lines up to 160 sites (shared memory) or up to 1024 with slices of 32;
    // 3D slabs: layers of A = Lx Ly <= 1024 sites with slices wider than 64 (their
    // factorization is the one-sided global-memory one the surface recursion reads)
    const bool fits2 = g.T == 1 && g.p > 1 && g.W <= DY_LPRE_MAXW &&
                       (g.Lx <= DY_LPRE_MAXLX || (g.Lx <= DY_LPRE_MAXLX_G && g.W == DY_LPRE_MAXW));
    const bool fits3 = g.T > 1 && g.p > 1 && g.W > DY_MAXW_SMEM && g.A <= DY_LPRE_MAXLX_G;
    const bool fits = fits2 || fits3;
    if (in->precond == DYSON_PRECOND_LAYER && !fits)
      return fail(DYSON_E_UNSUPPORTED, "exact layer preconditioner: p > 1 and either 2D strips with Lx <= " +
                                           std::to_string(DY_LPRE_MAXLX) + " and slice width <= " +
                                           std::to_string(DY_LPRE_MAXW) + ", or Lx <= " +
                                           std::to_string(DY_LPRE_MAXLX_G) + " and slice width " +
                                           std::to_string(DY_LPRE_MAXW) + ", or 3D slabs with Lx Ly <= " +
                                           std::to_string(DY_LPRE_MAXLX_G) + " and slice width > " +
                                           std::to_string(DY_MAXW_SMEM));
    g.lpre = (fits && in->precond != DYSON_PRECOND_BANDED) ? 1 : 0;
  }
  g.k_max = in->k_max;
  if (g.k_max < 1 || g.k_max > 256) return fail(DYSON_E_BAD_ARG, "k_max must be in 1..256");
  g.nb = in->block_size > 1 ? in->block_size : 1;
  g.qsplit = (in->precision == DYSON_MIXED && g.nb == 1 && g.k_max <= 64) ? 1 : 0;
  if (in->block_size < 0 || g.nb > DY_MAXNB)
    return fail(DYSON_E_BAD_ARG, "block_size must be in 0.." + std::to_string(DY_MAXNB));
  if (g.nb > 1 && (g.k_max % g.nb || g.k_max * g.nb > DY_BLOCK_H))
    return fail(DYSON_E_BAD_ARG, "block plans need k_max a multiple of block_size and k_max * block_size <= " +
                                     std::to_string(DY_BLOCK_H));
  if (in->precision != DYSON_FP64 && in->precision != DYSON_MIXED)
    return fail(DYSON_E_BAD_ARG, "precision must be DYSON_FP64 or DYSON_MIXED");
  const bool mixed = in->precision == DYSON_MIXED;
  // a single subdomain needs no sweeps (X = 0: the solve is the recursion alone)
  if (gpu && g.p > 1 && dyson_internal_sweep_smem(g, mixed) == 0)
    return fail(DYSON_E_UNSUPPORTED, "slice width " + std::to_string(g.W) + " with Lx = " +
                                         std::to_string(g.Lx) +
                                         ": the sweep row buffer does not fit shared memory");
  g.t = in->t;
  g.mu = in->mu;
  if (!(in->eta >= 0.0)) return fail(DYSON_E_BAD_ARG, "eta must be >= 0 (0: Matsubara axis)");
  g.eta = in->eta;
  g.real_axis = in->eta > 0.0 ? 1 : 0;
  g.krylov_tol = in->krylov_tol > 0 ? in->krylov_tol : (mixed ? 1e-5 : 1e-13);
  g.krylov_maxit = in->krylov_maxit > 0 ? in->krylov_maxit : 1000;
  g.refine_tol = in->refine_tol > 0 ? in->refine_tol : 1e-13;   // the FP64 form's krylov_tol
  g.refine_max = in->refine_max > 0 ? in->refine_max : 6;
  if (in->freq_groups < 0) return fail(DYSON_E_BAD_ARG, "freq_groups must be >= 0 (0: default)");
  if (in->max_freqs < 1 || (long long)in->max_freqs * g.nb > 65535)
    return fail(DYSON_E_BAD_ARG, "max_freqs (times block_size) must be in 1..65535");
  out->dd2nat.assign(g.Ndd, -1);
  for (int i = 0; i < g.p; ++i) {
    const int w = g.T * g.h[i];
    for (int s = 0; s < g.Lx; ++s)
      for (int j = 0; j < w; ++j) {
        int tr = j % g.T, sl = j / g.T;
        out->dd2nat[(size_t)i * g.Lx * g.W + (size_t)s * g.W + j] =
            s + g.Lx * tr + g.A * (g.s0[i] + sl);
      }
  }
  for (int l = 0; l < g.p - 1; ++l)
    for (int a = 0; a < g.A; ++a) out->dd2nat[(size_t)g.ifc_off + (size_t)l * g.A + a] = a + g.A * g.ylayer[l];
  out->m = (g.p - 1) * g.A;
  out->g = g;
  return DYSON_OK;
}

enum {
  B_V, B_OMEGA, B_SIGMA, B_Q1, B_DD2NAT, B_G, B_G64, B_DIAGB, B_Q, B_ACC, B_U, B_V1, B_V2, B_V3,
  B_YSCR, B_BND, B_IFV, B_PRE, B_LAN, B_MAXT, B_ST, B_OUT, B_STATUS, B_SWEEPS, B_FWORK, B_OFFB, B_OFF2,
  B_LPT, B_LPM, B_LPG, B_LPV, B_HDIAG, B_LPW, B_GRAM, B_COUNT
};

size_t layout(const Geo& g, int K, bool mixed, size_t off[B_COUNT]) {
  const size_t cs = mixed ? sizeof(cxf) : sizeof(cxd);
  const size_t Kz = (size_t)K, Ndd = g.Ndd, nsub = (size_t)g.Lx * g.W;
  const size_t Ks = Kz * g.nb;     // work slots: one per (frequency, block column)
  size_t sz[B_COUNT];
  sz[B_V] = g.N * sizeof(double);
  sz[B_OMEGA] = Kz * sizeof(double);
  sz[B_SIGMA] = Kz * g.N * sizeof(cxd);
  sz[B_Q1] = (size_t)g.nb * g.N * sizeof(double);
  sz[B_DD2NAT] = Ndd * sizeof(int);
  sz[B_G] = Kz * g.p * nsub * g.W * cs;
  sz[B_G64] = mixed ? Kz * g.p * nsub * g.W * sizeof(cxd) : 0;
  sz[B_DIAGB] = Kz * Ndd * sizeof(cxd);
  sz[B_Q] = Kz * (g.k_max + g.nb) * Ndd * sizeof(cxd);
  sz[B_ACC] = Kz * Ndd * sizeof(cxd);
  sz[B_U] = Ks * Ndd * sizeof(cxd);
  sz[B_V1] = mixed ? Ks * Ndd * sizeof(cxd) : 0;
  sz[B_V2] = sz[B_V1];
  sz[B_V3] = sz[B_V1];
  sz[B_YSCR] = Ks * g.p * nsub * cs;
  sz[B_BND] = Ks * g.p * 2 * g.A * sizeof(cxd);
  sz[B_IFV] = Ks * IF_N * nifc(g) * sizeof(cxd);
  sz[B_PRE] = Kz * nifc(g) * 3 * sizeof(cxd);
  sz[B_LAN] = Kz * (g.k_max + g.nb) * 2 * g.nb * sizeof(cxd);
  sz[B_MAXT] = Kz * sizeof(double);
  sz[B_ST] = Kz * ST_N * sizeof(int);
  sz[B_OUT] = Kz * g.N * sizeof(cxd);
  sz[B_STATUS] = Kz * sizeof(int);
  sz[B_SWEEPS] = Ks * g.p * sizeof(unsigned long long);
  sz[B_FWORK] = g.W > DY_MAXW_SMEM ? (size_t)DY_FACTOR_CTAS * 2 * g.W * g.W * sizeof(cxd) : 0;
  sz[B_OFFB] = Kz * g.p * nsub * sizeof(cxd);
  sz[B_OFF2] = g.penta ? Kz * g.p * nsub * sizeof(cxd) : 0;
  const size_t A2 = (size_t)g.A * g.A;   // layer blocks (A = Lx in 2D)
  sz[B_LPT] = g.lpre ? Kz * g.p * 2 * A2 * sizeof(cxf) : 0;
  sz[B_LPM] = g.lpre ? Kz * (g.p - 1) * A2 * cs : 0;
  sz[B_LPG] = (g.lpre && g.T == 1) ? Kz * g.p * nsub * g.W * sizeof(cxf) : 0;
  sz[B_LPV] = (g.lpre && g.T == 1 && g.Lx > DY_LPRE_MAXLX) ? Kz * g.p * 2 * (size_t)g.Lx * g.W * sizeof(cxf) : 0;
  sz[B_LPW] = (g.lpre && g.T > 1) ? (size_t)DY_FACTOR_CTAS * 2 * g.W * 2 * (size_t)g.Lx * g.T * sizeof(cxf) : 0;
  sz[B_HDIAG] = mixed ? Kz * Ndd * sizeof(cxd) : 0;
  sz[B_GRAM] = g.qsplit ? Kz * (size_t)(g.k_max + 1) * (g.k_max + 1) * sizeof(cxd) : 0;
  size_t o = 0;
  for (int k = 0; k < B_COUNT; ++k) {
    off[k] = o;
    o += (sz[k] + 255) & ~(size_t)255;
  }
  return o;
}

}  // namespace

int dyson_internal_fail(int code, const std::string& msg) { return fail(code, msg); }

cudaError_t raise_smem_limit(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> cur;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  size_t& have = cur[{dev, func}];
  if (bytes <= have || bytes <= 48 * 1024) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) have = bytes;
  return e;
}

struct dyson_plan_s {
  dyson_geometry gi;
  Geo g;
  bool mixed;
  int Kcap;
  int device;
  char* arena;
  size_t bytes;
  size_t off[B_COUNT];
  Bufs b;
  int* status_d;
  cudaStream_t cap;
  std::map<int, cudaGraphExec_t> graphs;
  bool use_graph;
  bool profile;                    // bracket every kernel with timing events
  bool tuned;                      // the copy-ring configuration has been timed
  int tune_candidates;             // configurations timed
  float tune_ms_heuristic, tune_ms_best;   // one X-matvec launch with each
  std::vector<cudaEvent_t> evs;    // 2 per profiled kernel
  std::vector<int> ev_kind;        // DYSON_KERNEL_* of each profiled kernel
  int n_prof;                      // profiled kernels in the last enqueued sequence
  int ngroups;                     // frequency groups run as parallel graph branches
  std::vector<cudaStream_t> gs;    // one stream per group (group 0 highest priority)
  std::vector<cudaEvent_t> gev;    // fork + one join event per group
};

namespace {

template <typename T>
T* at(dyson_plan p, int k) { return reinterpret_cast<T*>(p->arena + p->off[k]); }

int check_plan(dyson_plan p) {
  if (!p) return fail(DYSON_E_BAD_ARG, "plan is NULL");
  cudaError_t e = cudaSetDevice(p->device);
  if (e != cudaSuccess) return fail(DYSON_E_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  return DYSON_OK;
}

// the entry points that sweep the subdomains (every geometry with p > 1 passed
// this at plan creation)
int check_sweeps(dyson_plan p) {
  if (dyson_internal_sweep_smem(p->g, p->mixed) == 0)
    return fail(DYSON_E_UNSUPPORTED, "slice width " + std::to_string(p->g.W) + " with Lx = " +
                                         std::to_string(p->g.Lx) +
                                         ": the sweep row buffer does not fit shared memory");
  return DYSON_OK;
}

int check_K(dyson_plan p, int K) {
  if (K < 1 || K > p->Kcap)
    return fail(DYSON_E_BAD_ARG, "K must be in 1..max_freqs (" + std::to_string(p->Kcap) + ")");
  return DYSON_OK;
}

int check_mem(int mem_kind) {
  if (mem_kind != DYSON_MEM_HOST && mem_kind != DYSON_MEM_DEVICE)
    return fail(DYSON_E_BAD_ARG, "mem_kind must be DYSON_MEM_HOST or DYSON_MEM_DEVICE");
  return DYSON_OK;
}

// copy omega, V, sigma (and q1) into the plan's input buffers
int stage_inputs(dyson_plan p, int K, const double* omega, const double* V, const double* sigma,
                 const double* q1, cudaStream_t s) {
  if (!omega || !V || !sigma) return fail(DYSON_E_BAD_ARG, "omega, V and sigma must not be NULL");
  const Geo& g = p->g;
  CK(cudaMemcpyAsync(at<double>(p, B_OMEGA), omega, K * sizeof(double), cudaMemcpyDefault, s));
  CK(cudaMemcpyAsync(at<double>(p, B_V), V, g.N * sizeof(double), cudaMemcpyDefault, s));
  CK(cudaMemcpyAsync(at<cxd>(p, B_SIGMA), sigma, (size_t)K * g.N * sizeof(cxd), cudaMemcpyDefault, s));
  if (q1)
    CK(cudaMemcpyAsync(at<double>(p, B_Q1), q1, (size_t)g.nb * g.N * sizeof(double), cudaMemcpyDefault, s));
  return DYSON_OK;
}

int finish(int mem_kind, cudaStream_t s) {
  if (mem_kind == DYSON_MEM_HOST) CK(cudaStreamSynchronize(s));
  else CK(cudaGetLastError());
  return DYSON_OK;
}

#define LK(call)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return fail(DYSON_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

int enqueue_factor(dyson_plan p, int K, cudaStream_t s) {
  if (p->mixed) LK((launch_factor<dfl, float>(p->g, p->b, K, s)));
  else LK((launch_factor<double, double>(p->g, p->b, K, s)));
  return DYSON_OK;
}

// Record a timing event on s; inside a stream capture it becomes an event-record
// node of the graph, so replays time every kernel on the stream they run on.
cudaError_t prof_event(dyson_plan p, int idx, cudaStream_t s, bool capturing) {
  while ((int)p->evs.size() <= idx) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    p->evs.push_back(e);
  }
  return capturing ? cudaEventRecordWithFlags(p->evs[idx], s, cudaEventRecordExternal)
                   : cudaEventRecord(p->evs[idx], s);
}

template <typename F>
int run_kernel(dyson_plan p, int kind, cudaStream_t s, bool cap, const char* what, F&& f) {
  if (p->profile) {
    const int k = p->n_prof;
    if ((int)p->ev_kind.size() <= k) p->ev_kind.resize(k + 1);
    p->ev_kind[k] = kind;
    LK(prof_event(p, 2 * k, s, cap));
  }
  cudaError_t e = f();
  if (e != cudaSuccess) return fail(DYSON_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  if (p->profile) {
    LK(prof_event(p, 2 * p->n_prof + 1, s, cap));
    p->n_prof++;
  }
  return DYSON_OK;
}

#define RUN(kind, what, expr) \
  do {                       \
    int rc_ = run_kernel(p, kind, s, cap, what, [&]() { return (expr); }); \
    if (rc_) return rc_;     \
  } while (0)

// The plan's buffers seen from frequency k0 on: every per-frequency array
// advanced by k0 frequencies, every per-slot array by k0 * nb slots (byte
// strides of the form's precision where the kernels read the buffer in it).
// Kernels index frequencies from blockIdx.y, so a launch over this view with K
// frequencies works on frequencies k0 .. k0 + K - 1 of the plan.
Bufs sub_bufs(const Geo& g, const Bufs& b, bool mixed, int k0) {
  if (k0 == 0) return b;
  Bufs s = b;
  const size_t K0 = (size_t)k0, S0 = K0 * g.nb, Ndd = g.Ndd, nsub = (size_t)g.Lx * g.W;
  const size_t cs = mixed ? sizeof(cxf) : sizeof(cxd), Lx2 = (size_t)g.Lx * g.Lx;
  auto adv = [](auto* ptr, size_t bytes) {
    using T = std::remove_pointer_t<decltype(ptr)>;
    return ptr ? reinterpret_cast<T*>(reinterpret_cast<char*>(const_cast<std::remove_const_t<T>*>(ptr)) + bytes)
               : ptr;
  };
  s.omega = b.omega + K0;
  s.sigma = b.sigma + K0 * g.N;
  s.g = adv(reinterpret_cast<char*>(b.g), K0 * g.p * nsub * g.W * cs);
  s.g64 = b.g64 ? b.g64 + K0 * g.p * nsub * g.W : nullptr;
  s.diagB = b.diagB + K0 * Ndd;
  s.hdiag = b.hdiag ? b.hdiag + K0 * Ndd : nullptr;
  s.offB = b.offB ? b.offB + K0 * g.p * nsub : nullptr;
  s.off2 = b.off2 ? b.off2 + K0 * g.p * nsub : nullptr;
  s.Q = b.Q + K0 * (g.k_max + g.nb) * Ndd;
  s.acc = b.acc + K0 * Ndd;
  s.u = b.u + S0 * Ndd;
  s.v1 = b.v1 ? b.v1 + S0 * Ndd : nullptr;
  s.v2 = b.v2 ? b.v2 + S0 * Ndd : nullptr;
  s.v3 = b.v3 ? b.v3 + S0 * Ndd : nullptr;
  s.yscr = adv(reinterpret_cast<char*>(b.yscr), S0 * g.p * nsub * cs);
  s.bnd = adv(b.bnd, S0 * g.p * 2 * g.A * cs);
  s.ifv = adv(b.ifv, S0 * IF_N * nifc(g) * cs);
  s.pre = adv(b.pre, K0 * nifc(g) * 3 * cs);
  s.lan = b.lan + K0 * (g.k_max + g.nb) * 2 * g.nb;
  s.maxT = b.maxT + K0;
  s.st = b.st + K0 * ST_N;
  s.out = b.out + K0 * g.N;
  s.sweeps = b.sweeps ? b.sweeps + S0 * g.p : nullptr;
  const size_t A2 = (size_t)g.A * g.A;
  s.lpt = b.lpt ? b.lpt + K0 * g.p * 2 * A2 : nullptr;
  s.lpm = adv(reinterpret_cast<char*>(b.lpm), K0 * (g.p > 1 ? g.p - 1 : 0) * A2 * cs);
  s.lpg = b.lpg ? b.lpg + K0 * g.p * nsub * g.W : nullptr;
  s.lpv = b.lpv ? b.lpv + K0 * g.p * 2 * (size_t)g.Lx * g.W : nullptr;
  s.gram = b.gram ? b.gram + K0 * (size_t)(g.k_max + 1) * (g.k_max + 1) : nullptr;
  return s;
}

// One batch of K frequencies (from the view b) on stream s.  (Running the
// layer preconditioner's build beside the factorization on a second branch
// was measured slower: the two kernels compete for issue slots.)
int enqueue_range(dyson_plan p, const Bufs& b, int K, int* status, cudaStream_t s, bool cap) {
  const Geo& g = p->g;
  if (g.nb > 1) RUN(DYSON_KERNEL_INIT, "init", launch_init_block(g, b, K, s));
  else RUN(DYSON_KERNEL_INIT, "init", launch_init(g, b, K, s));
  if (p->mixed) RUN(DYSON_KERNEL_FACTOR, "factor", (launch_factor<dfl, float>(g, b, K, s)));
  else RUN(DYSON_KERNEL_FACTOR, "factor", (launch_factor<double, double>(g, b, K, s)));
  if (g.p > 1) {
    if (p->mixed) RUN(DYSON_KERNEL_PRECOND, "precond", launch_precond<float>(g, b, K, s));
    else RUN(DYSON_KERNEL_PRECOND, "precond", launch_precond<double>(g, b, K, s));
  }
  if (g.p > 1) {
    for (int j = 0; j < g.k_max / g.nb; ++j) {      // (block) Lanczos steps
      if (p->mixed) RUN(DYSON_KERNEL_XMATVEC, "xmatvec", launch_xmatvec<float>(g, b, K, j, 1, g.nb, s));
      else RUN(DYSON_KERNEL_XMATVEC, "xmatvec", launch_xmatvec<double>(g, b, K, j, 0, g.nb, s));
      if (g.nb > 1) RUN(DYSON_KERNEL_LANCZOS, "lanczos", launch_block_lanczos(g, b, K, j, s));
      else if (p->mixed && g.k_max <= 64) RUN(DYSON_KERNEL_LANCZOS, "lanczos", launch_lanczos_dd(g, b, K, j, s));
      else RUN(DYSON_KERNEL_LANCZOS, "lanczos", launch_lanczos(g, b, K, j, s));
    }
  }
  RUN(DYSON_KERNEL_FINALIZE, "finalize", launch_finalize(g, b, K, s));
  RUN(DYSON_KERNEL_STATUS, "status", launch_status(g, b, K, status, s));
  return DYSON_OK;
}

// Groups a batch of K frequencies is split into (at least two frequencies each).
int groups_for(dyson_plan p, int K) {
  int G = p->ngroups;
  while (G > 1 && K < 2 * G) --G;
  return G;
}

// The whole solve.  With frequency groups, contiguous index ranges run as
// parallel branches (forked from and joined back into s): a launch of one
// group waits only for that group's previous step, so the slowest frequency's
// chain of X-matvecs is not held back by every frequency's Lanczos step and
// factorization, and the faster groups fill the SMs it leaves idle.
int enqueue_solve(dyson_plan p, int K, cudaStream_t s, bool cap) {
  p->n_prof = 0;
  const int G = groups_for(p, K);
  if (G <= 1) return enqueue_range(p, p->b, K, p->status_d, s, cap);
  CK(cudaEventRecord(p->gev[0], s));
  int k0 = 0;
  for (int gi = 0; gi < G; ++gi) {
    const int Kg = K / G + (gi < K % G ? 1 : 0);
    CK(cudaStreamWaitEvent(p->gs[gi], p->gev[0], 0));
    const Bufs sb = sub_bufs(p->g, p->b, p->mixed, k0);
    int rc = enqueue_range(p, sb, Kg, p->status_d + k0, p->gs[gi], cap);
    if (rc) return rc;
    CK(cudaEventRecord(p->gev[1 + gi], p->gs[gi]));
    CK(cudaStreamWaitEvent(s, p->gev[1 + gi], 0));
    k0 += Kg;
  }
  return DYSON_OK;
}

// Autotuner (batched kernels' tile choice): at the first solve of a plan with
// an interface, on the caller's staged inputs, run init, factorization and
// preconditioner once, then time one X-matvec launch (after one untimed) for
// each copy-ring configuration the geometry admits (ring slots; chunk height
// for W > 64) and keep the fastest for every later launch and captured graph.
int autotune(dyson_plan p, int K, cudaStream_t s) {
  p->tuned = true;
  if (p->g.p < 2) return DYSON_OK;
  int S[32], CR[32], NT[32];
  const int n = dyson_internal_ring_candidates(p->g, p->mixed, S, CR, NT, 32);
  p->tune_candidates = n;
  if (n < 2) return DYSON_OK;
  Geo& g = p->g;
  if (g.nb > 1) LK(launch_init_block(g, p->b, K, s));
  else LK(launch_init(g, p->b, K, s));
  if (p->mixed) LK((launch_factor<dfl, float>(g, p->b, K, s)));
  else LK((launch_factor<double, double>(g, p->b, K, s)));
  if (p->mixed) LK(launch_precond<float>(g, p->b, K, s));
  else LK(launch_precond<double>(g, p->b, K, s));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int best = 0;
  float best_ms = 0.f;
  int rc = DYSON_OK;
  for (int c = 0; c < n && rc == DYSON_OK; ++c) {
    g.ring_S = S[c];
    g.ring_CR = CR[c];
    g.xm_nt = NT[c];
    cudaError_t e = p->mixed ? launch_xmatvec<float>(g, p->b, K, 0, 1, g.nb, s)
                             : launch_xmatvec<double>(g, p->b, K, 0, 0, g.nb, s);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess)
      e = p->mixed ? launch_xmatvec<float>(g, p->b, K, 0, 1, g.nb, s)
                   : launch_xmatvec<double>(g, p->b, K, 0, 0, g.nb, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      rc = fail(DYSON_E_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
      break;
    }
    if (c == 0) p->tune_ms_heuristic = ms;
    if (c == 0 || ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g.ring_S = S[best];
  g.ring_CR = CR[best];
  g.xm_nt = NT[best];
  p->tune_ms_best = best_ms;
  return rc;
}

int get_graph(dyson_plan p, int K, cudaGraphExec_t* out) {
  auto it = p->graphs.find(K);
  if (it != p->graphs.end()) {
    *out = it->second;
    return DYSON_OK;
  }
  CK(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeRelaxed));
  int rc = enqueue_solve(p, K, p->cap, true);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(p->cap, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return fail(DYSON_E_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
  cudaGraphExec_t exec;
  // kernel nodes keep the priority of the stream they were captured from
  e = cudaGraphInstantiate(&exec, graph, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(DYSON_E_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  p->graphs[K] = exec;
  *out = exec;
  return DYSON_OK;
}

}  // namespace

extern "C" {

const char* dyson_version(void) { return "paper_1102_3137_gb300 0.1 (sm_103a)"; }

const char* dyson_last_error(void) { return g_err.c_str(); }

int dyson_partition(const dyson_geometry* geom, int* heights, int* m, int* ndd, int* dd2nat) {
  Part part;
  int rc = build_part(geom, &part, false);
  if (rc) return rc;
  if (heights)
    for (int i = 0; i < part.g.p; ++i) heights[i] = part.g.h[i];
  if (m) *m = part.m;
  if (ndd) *ndd = part.g.Ndd;
  if (dd2nat) std::memcpy(dd2nat, part.dd2nat.data(), part.dd2nat.size() * sizeof(int));
  return DYSON_OK;
}

int dyson_plan_footprint(const dyson_geometry* geom, size_t* bytes) {
  Part part;
  int rc = build_part(geom, &part, true);
  if (rc) return rc;
  if (!bytes) return fail(DYSON_E_BAD_ARG, "bytes is NULL");
  size_t off[B_COUNT];
  *bytes = layout(part.g, geom->max_freqs, geom->precision == DYSON_MIXED, off);
  return DYSON_OK;
}

int dyson_plan_create(const dyson_geometry* geom, dyson_plan* out) {
  if (!out) return fail(DYSON_E_BAD_ARG, "out is NULL");
  *out = nullptr;
  Part part;
  int rc = build_part(geom, &part, true);
  if (rc) return rc;
  dyson_plan p = new dyson_plan_s();
  p->gi = *geom;
  p->g = part.g;
  p->mixed = geom->precision == DYSON_MIXED;
  p->Kcap = geom->max_freqs;
  p->use_graph = !(getenv("DYSON_NO_GRAPH") && getenv("DYSON_NO_GRAPH")[0] == '1');
  cudaGetDevice(&p->device);
  p->bytes = layout(p->g, p->Kcap, p->mixed, p->off);
  cudaError_t e = cudaMalloc(&p->arena, p->bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return fail(DYSON_E_OOM, "cudaMalloc of " + std::to_string(p->bytes) + " bytes failed: " +
                                 cudaGetErrorString(e));
  }
  e = cudaMemset(p->arena, 0, p->bytes);
  if (e == cudaSuccess)
    e = cudaMemcpy(at<int>(p, B_DD2NAT), part.dd2nat.data(), part.dd2nat.size() * sizeof(int),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaFree(p->arena);
    delete p;
    return fail(DYSON_E_CUDA, std::string("plan set-up: ") + cudaGetErrorString(e));
  }
  Bufs& b = p->b;
  b.V = at<double>(p, B_V);
  b.omega = at<double>(p, B_OMEGA);
  b.sigma = at<cxd>(p, B_SIGMA);
  b.q1 = at<double>(p, B_Q1);
  b.dd2nat = at<int>(p, B_DD2NAT);
  b.g = at<void>(p, B_G);
  b.g64 = p->mixed ? at<cxd>(p, B_G64) : nullptr;
  b.diagB = at<cxd>(p, B_DIAGB);
  b.hdiag = p->mixed ? at<cxd>(p, B_HDIAG) : nullptr;
  b.Q = at<cxd>(p, B_Q);
  b.acc = at<cxd>(p, B_ACC);
  b.u = at<cxd>(p, B_U);
  b.v1 = p->mixed ? at<cxd>(p, B_V1) : nullptr;
  b.v2 = p->mixed ? at<cxd>(p, B_V2) : nullptr;
  b.v3 = p->mixed ? at<cxd>(p, B_V3) : nullptr;
  b.yscr = at<void>(p, B_YSCR);
  b.bnd = at<cxd>(p, B_BND);
  b.ifv = at<cxd>(p, B_IFV);
  b.pre = at<cxd>(p, B_PRE);
  b.lan = at<cxd>(p, B_LAN);
  b.maxT = at<double>(p, B_MAXT);
  b.st = at<int>(p, B_ST);
  b.out = at<cxd>(p, B_OUT);
  b.sweeps = at<unsigned long long>(p, B_SWEEPS);
  b.fwork = p->g.W > DY_MAXW_SMEM ? at<cxd>(p, B_FWORK) : nullptr;
  b.offB = at<cxd>(p, B_OFFB);
  b.off2 = p->g.penta ? at<cxd>(p, B_OFF2) : nullptr;
  b.lpt = p->g.lpre ? at<cxf>(p, B_LPT) : nullptr;
  b.lpm = p->g.lpre ? (void*)at<char>(p, B_LPM) : nullptr;
  b.lpg = p->g.lpre ? at<cxf>(p, B_LPG) : nullptr;
  b.lpv = (p->g.lpre && p->g.T == 1 && p->g.Lx > DY_LPRE_MAXLX) ? at<cxf>(p, B_LPV) : nullptr;
  b.lpw = (p->g.lpre && p->g.T > 1) ? at<cxf>(p, B_LPW) : nullptr;
  b.gram = p->g.qsplit ? at<cxd>(p, B_GRAM) : nullptr;
  p->status_d = at<int>(p, B_STATUS);
  p->profile = false;
  p->tuned = false;
  p->tune_candidates = 0;
  p->tune_ms_heuristic = p->tune_ms_best = 0.f;
  p->n_prof = 0;
  // X-matvec CTA size (complex64 two-chain form): 128 threads, four CTAs per SM,
  // when the solve's clusters would not all fit at two CTAs per SM; the
  // autotuner may revise it at the first solve
  if (p->mixed && p->g.W <= DY_MAXW_SMEM && p->g.p > 1) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    const long long ctas = (long long)p->g.p * p->Kcap * p->g.nb;
    p->g.xm_nt = (sms > 0 && ctas > 2LL * sms) ? 128 : 256;
  }
  // frequency groups: not with the shared wide-slice factor workspace
  p->ngroups = 1;
  if (p->g.p > 1 && !b.fwork) {
    // default: one group per 16 frequencies of the plan's capacity in the mixed form, per 8
    // in FP64, at most DY_FREQ_GROUPS (512^2 x 32: mixed 1346 ms in 2 groups, 1370 in 4,
    // 1373 in 8; FP64 3386 ms in 4 groups, 3545 in 2)
    const int per = p->mixed ? 16 : 8;
    const int dflt = p->Kcap / per < 1 ? 1 : (p->Kcap / per > DY_FREQ_GROUPS ? DY_FREQ_GROUPS : p->Kcap / per);
    p->ngroups = geom->freq_groups > 0 ? geom->freq_groups : dflt;
    if (p->ngroups > DY_MAX_GROUPS) p->ngroups = DY_MAX_GROUPS;
  }
  if (p->ngroups > 1) {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);      // hi: the greatest priority (numerically lowest)
    for (int gi = 0; gi < p->ngroups && e == cudaSuccess; ++gi) {
      cudaStream_t st;
      const int prio = gi == 0 ? hi : (gi == 1 && hi < lo ? hi + 1 : lo);
      e = cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio);
      if (e == cudaSuccess) p->gs.push_back(st);
    }
    for (int gi = 0; gi <= p->ngroups && e == cudaSuccess; ++gi) {
      cudaEvent_t ev;
      e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e == cudaSuccess) p->gev.push_back(ev);
    }
  }
  if (e != cudaSuccess) {
    dyson_plan_destroy(p);
    return fail(DYSON_E_CUDA, std::string("plan streams: ") + cudaGetErrorString(e));
  }
  *out = p;
  return DYSON_OK;
}

int dyson_plan_destroy(dyson_plan p) {
  if (!p) return DYSON_OK;
  cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  for (auto& kv : p->graphs) cudaGraphExecDestroy(kv.second);
  for (auto e : p->evs) cudaEventDestroy(e);
  for (auto e : p->gev) cudaEventDestroy(e);
  for (auto st : p->gs) cudaStreamDestroy(st);
  cudaStreamDestroy(p->cap);
  cudaFree(p->arena);
  delete p;
  return DYSON_OK;
}

}  // extern "C"

// Enqueue a whole solve on `stream` (inputs in, graph, outputs out) without
// waiting for it; the serving loop uses this directly.
int dyson_internal_solve_enqueue(dyson_plan p, int K, const double* omega, const double* V,
                                 const double* sigma, const double* q1, double* diagG, int* status,
                                 int mem_kind, void* stream) {
  int rc;
  if ((rc = check_plan(p)) || (rc = check_K(p, K)) || (rc = check_mem(mem_kind))) return rc;
  if (!q1 || !diagG) return fail(DYSON_E_BAD_ARG, "q1 and diagG must not be NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = stage_inputs(p, K, omega, V, sigma, q1, s))) return rc;
  if (!p->tuned && (rc = autotune(p, K, s))) return rc;
  if (p->use_graph) {
    cudaGraphExec_t ex;
    if ((rc = get_graph(p, K, &ex))) return rc;
    CK(cudaGraphLaunch(ex, s));
  } else if ((rc = enqueue_solve(p, K, s, false))) {
    return rc;
  }
  CK(cudaMemcpyAsync(diagG, p->b.out, (size_t)K * p->g.N * sizeof(cxd), cudaMemcpyDefault, s));
  if (status) CK(cudaMemcpyAsync(status, p->status_d, K * sizeof(int), cudaMemcpyDefault, s));
  return DYSON_OK;
}

int dyson_internal_solve_enqueue_segs(dyson_plan p, int nseg, const SolveSeg* segs, const double* V,
                                      const double* q1, int mem_kind, void* stream) {
  int rc;
  if ((rc = check_plan(p)) || (rc = check_mem(mem_kind))) return rc;
  if (nseg < 1 || !segs || !V || !q1) return fail(DYSON_E_BAD_ARG, "fused solve: no segments, V or q1");
  int K = 0;
  for (int n = 0; n < nseg; ++n) {
    if (segs[n].K < 1 || !segs[n].omega || !segs[n].sigma || !segs[n].diagG)
      return fail(DYSON_E_BAD_ARG, "fused solve: a segment without frequencies or buffers");
    K += segs[n].K;
  }
  if ((rc = check_K(p, K))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const Geo& g = p->g;
  const size_t N = g.N;
  for (int n = 0, k0 = 0; n < nseg; k0 += segs[n].K, ++n) {
    CK(cudaMemcpyAsync(at<double>(p, B_OMEGA) + k0, segs[n].omega, segs[n].K * sizeof(double),
                       cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(at<cxd>(p, B_SIGMA) + (size_t)k0 * N, segs[n].sigma, (size_t)segs[n].K * N * sizeof(cxd),
                       cudaMemcpyDefault, s));
  }
  CK(cudaMemcpyAsync(at<double>(p, B_V), V, N * sizeof(double), cudaMemcpyDefault, s));
  CK(cudaMemcpyAsync(at<double>(p, B_Q1), q1, (size_t)g.nb * N * sizeof(double), cudaMemcpyDefault, s));
  if (!p->tuned && (rc = autotune(p, K, s))) return rc;
  if (p->use_graph) {
    cudaGraphExec_t ex;
    if ((rc = get_graph(p, K, &ex))) return rc;
    CK(cudaGraphLaunch(ex, s));
  } else if ((rc = enqueue_solve(p, K, s, false))) {
    return rc;
  }
  for (int n = 0, k0 = 0; n < nseg; k0 += segs[n].K, ++n) {
    CK(cudaMemcpyAsync(segs[n].diagG, p->b.out + (size_t)k0 * N, (size_t)segs[n].K * N * sizeof(cxd),
                       cudaMemcpyDefault, s));
    if (segs[n].status)
      CK(cudaMemcpyAsync(segs[n].status, p->status_d + k0, segs[n].K * sizeof(int), cudaMemcpyDefault, s));
  }
  return DYSON_OK;
}

size_t dyson_internal_plan_bytes(dyson_plan p) { return p ? p->bytes : 0; }

int dyson_internal_plan_dev(dyson_plan p, PlanDev* out) {
  int rc;
  if ((rc = check_plan(p))) return rc;
  out->omega = at<double>(p, B_OMEGA);
  out->V = at<double>(p, B_V);
  out->sigma = at<double>(p, B_SIGMA);
  out->q1 = at<double>(p, B_Q1);
  out->acc = reinterpret_cast<const double*>(p->b.acc);
  out->diagB = reinterpret_cast<const double*>(p->b.diagB);
  out->dd2nat = p->b.dd2nat;
  out->status = p->status_d;
  out->Ndd = p->g.Ndd;
  out->N = p->g.N;
  return DYSON_OK;
}

int dyson_internal_solve_resident(dyson_plan p, int K, void* stream) {
  int rc;
  if ((rc = check_plan(p)) || (rc = check_K(p, K))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (!p->tuned && (rc = autotune(p, K, s))) return rc;
  if (p->use_graph) {
    cudaGraphExec_t ex;
    if ((rc = get_graph(p, K, &ex))) return rc;
    CK(cudaGraphLaunch(ex, s));
    return DYSON_OK;
  }
  return enqueue_solve(p, K, s, false);
}

int dyson_internal_factor_resident(dyson_plan p, int K, void* stream) {
  int rc;
  if ((rc = check_plan(p)) || (rc = check_K(p, K))) return rc;
  return enqueue_factor(p, K, (cudaStream_t)stream);
}

extern "C" {

int dyson_solve(dyson_plan p, int K, const double* omega, const double* V, const double* sigma,
                const double* q1, double* diagG, int* status, int mem_kind, void* stream) {
  int rc = dyson_internal_solve_enqueue(p, K, omega, V, sigma, q1, diagG, status, mem_kind, stream);
  if (rc) return rc;
  return finish(mem_kind, (cudaStream_t)stream);
}

int dyson_plan_tuning(dyson_plan p, int* ring_slots, int* chunk_rows, int* candidates,
                      float* ms_heuristic, float* ms_best, int* threads) {
  int rc;
  if ((rc = check_plan(p))) return rc;
  int S = 0, CR = 0, NT = 0;
  dyson_internal_ring_plan(p->g, p->mixed, &S, &CR, &NT);
  if (threads) *threads = NT;
  if (ring_slots) *ring_slots = S;
  if (chunk_rows) *chunk_rows = CR;
  if (candidates) *candidates = p->tuned ? p->tune_candidates : 0;
  if (ms_heuristic) *ms_heuristic = p->tune_ms_heuristic;
  if (ms_best) *ms_best = p->tune_ms_best;
  return DYSON_OK;
}

int dyson_solve_info(dyson_plan p, int K, double* alpha_beta, int* steps, int* iters, int* refines) {
  int rc;
  if ((rc = check_plan(p)) || (rc = check_K(p, K))) return rc;
  CK(cudaDeviceSynchronize());
  const Geo& g = p->g;
  std::vector<int> st((size_t)K * ST_N);
  CK(cudaMemcpy(st.data(), p->b.st, st.size() * sizeof(int), cudaMemcpyDeviceToHost));
  for (int k = 0; k < K; ++k) {
    if (steps) steps[k] = st[(size_t)k * ST_N + ST_STEPS];
    if (iters) iters[k] = st[(size_t)k * ST_N + ST_ITERS];
    if (refines) refines[k] = st[(size_t)k * ST_N + ST_REFINE];
  }
  if (alpha_beta && g.nb > 1)
    return fail(DYSON_E_BAD_ARG, "block plan: alpha_beta must be NULL (dyson_block_info has T)");
  if (alpha_beta) {
    std::vector<cxd> lan((size_t)K * (g.k_max + 1) * 2);
    CK(cudaMemcpy(lan.data(), p->b.lan, lan.size() * sizeof(cxd), cudaMemcpyDeviceToHost));
    for (int k = 0; k < K; ++k)
      for (int j = 0; j < g.k_max; ++j)
        for (int c = 0; c < 2; ++c) {
          cxd v = lan[((size_t)k * (g.k_max + 1) + j) * 2 + c];
          double* o = alpha_beta + (((size_t)k * g.k_max + j) * 2 + c) * 2;
          o[0] = v.x;
          o[1] = v.y;
        }
  }
  return DYSON_OK;
}

int dyson_block_info(dyson_plan p, int K, double* AB, int* steps) {
  int rc;
  if ((rc = check_plan(p)) || (rc = check_K(p, K))) return rc;
  const Geo& g = p->g;
  if (g.nb < 2) return fail(DYSON_E_BAD_ARG, "not a block plan (block_size < 2)");
  CK(cudaDeviceSynchronize());
  if (steps) {
    std::vector<int> st((size_t)K * ST_N);
    CK(cudaMemcpy(st.data(), p->b.st, st.size() * sizeof(int), cudaMemcpyDeviceToHost));
    for (int k = 0; k < K; ++k) steps[k] = st[(size_t)k * ST_N + ST_STEPS];
  }
  if (AB) {
    // device: [K][k_max/nb + 1][2][nb][nb]; caller: [K][k_max/nb][2][nb][nb]
    const size_t per = (size_t)(g.k_max + g.nb) * 2 * g.nb, keep = (size_t)g.k_max * 2 * g.nb;
    std::vector<cxd> lan((size_t)K * per);
    CK(cudaMemcpy(lan.data(), p->b.lan, lan.size() * sizeof(cxd), cudaMemcpyDeviceToHost));
    for (int k = 0; k < K; ++k)
      std::memcpy(AB + (size_t)k * keep * 2, lan.data() + (size_t)k * per, keep * sizeof(cxd));
  }
  return DYSON_OK;
}

int dyson_plan_set_profiling(dyson_plan p, int on) {
  int rc;
  if ((rc = check_plan(p))) return rc;
  if (p->profile != (on != 0)) {
    CK(cudaDeviceSynchronize());
    for (auto& kv : p->graphs) cudaGraphExecDestroy(kv.second);
    p->graphs.clear();
    p->profile = on != 0;
  }
  return DYSON_OK;
}

int dyson_profile_read(dyson_plan p, int max_kernels, int* kinds, float* ms, int* n) {
  int rc;
  if ((rc = check_plan(p))) return rc;
  if (!n) return fail(DYSON_E_BAD_ARG, "n is NULL");
  if (!p->profile) return fail(DYSON_E_BAD_ARG, "profiling is off for this plan");
  CK(cudaDeviceSynchronize());
  *n = p->n_prof;
  for (int k = 0; k < p->n_prof && k < max_kernels; ++k) {
    if (kinds) kinds[k] = p->ev_kind[k];
    if (ms) CK(cudaEventElapsedTime(&ms[k], p->evs[2 * k], p->evs[2 * k + 1]));
  }
  return DYSON_OK;
}

int dyson_profile_spans(dyson_plan p, int max_kernels, float* start_ms, float* end_ms, int* n) {
  int rc;
  if ((rc = check_plan(p))) return rc;
  if (!n) return fail(DYSON_E_BAD_ARG, "n is NULL");
  if (!p->profile) return fail(DYSON_E_BAD_ARG, "profiling is off for this plan");
  CK(cudaDeviceSynchronize());
  *n = p->n_prof;
  // offsets from the earliest start event of the sequence (kernels of different
  // frequency groups run concurrently, so launch order is not time order)
  int first = 0;
  for (int k = 1; k < p->n_prof; ++k) {
    float d = 0.f;
    CK(cudaEventElapsedTime(&d, p->evs[2 * first], p->evs[2 * k]));
    if (d < 0.f) first = k;
  }
  for (int k = 0; k < p->n_prof && k < max_kernels; ++k) {
    if (start_ms) CK(cudaEventElapsedTime(&start_ms[k], p->evs[2 * first], p->evs[2 * k]));
    if (end_ms) CK(cudaEventElapsedTime(&end_ms[k], p->evs[2 * first], p->evs[2 * k + 1]));
  }
  return DYSON_OK;
}

int dyson_lanczos_basis(dyson_plan p, int k, int nvec, double* Q) {
  int rc;
  if ((rc = check_plan(p))) return rc;
  const Geo& g = p->g;
  if (k < 0 || k >= p->Kcap) return fail(DYSON_E_BAD_ARG, "frequency index out of range");
  if (nvec < 1 || nvec > g.k_max + g.nb) return fail(DYSON_E_BAD_ARG, "nvec must be in 1..k_max+block_size");
  if (!Q) return fail(DYSON_E_BAD_ARG, "Q is NULL");
  CK(cudaDeviceSynchronize());
  const size_t bytes = (size_t)nvec * g.N * sizeof(cxd);
  cxd* tmp = nullptr;
  CK(cudaMalloc(&tmp, bytes));
  const cxd* src = p->b.Q + (size_t)k * (g.k_max + g.nb) * g.Ndd;
  cudaError_t e = launch_scatter(g, p->b, nvec, src, tmp, g.Ndd, 0);
  if (e == cudaSuccess) e = cudaMemcpy(Q, tmp, bytes, cudaMemcpyDeviceToHost);
  cudaFree(tmp);
  if (e != cudaSuccess) return fail(DYSON_E_CUDA, std::string("basis copy: ") + cudaGetErrorString(e));
  if (g.qsplit) {                          // double-float entries {re.hi, re.lo, im.hi, im.lo}: widen
    const size_t n = (size_t)nvec * g.N;
    for (size_t e2 = 0; e2 < n; ++e2) {
      float f[4];
      std::memcpy(f, Q + 2 * e2, sizeof(f));
      Q[2 * e2] = (double)f[0] + (double)f[1];
      Q[2 * e2 + 1] = (double)f[2] + (double)f[3];
    }
  }
  return DYSON_OK;
}

int dyson_wait_selftest(double limit_s, int* timed_out, double* waited_s) {
  if (!(limit_s >= 1e-6 && limit_s <= 10.0)) return fail(DYSON_E_BAD_ARG, "limit_s must be in [1e-6, 10]");
  if (!timed_out) return fail(DYSON_E_BAD_ARG, "timed_out is NULL");
  int* d = nullptr;
  CK(cudaMalloc(&d, 2 * sizeof(int)));
  int h[2] = {-1, 0};
  cudaError_t e = launch_wait_selftest((unsigned long long)(limit_s * 1e9), d, 0);
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return fail(DYSON_E_CUDA, std::string("wait self-test: ") + cudaGetErrorString(e));
  *timed_out = h[0] == DYSON_ST_WAIT_TIMEOUT ? 1 : 0;
  if (waited_s) *waited_s = h[1] * 1e-6;
  return DYSON_OK;
}

int dyson_work_counters(dyson_plan p, int K, unsigned long long* sweeps) {
  int rc;
  if ((rc = check_plan(p)) || (rc = check_K(p, K))) return rc;
  if (!sweeps) return fail(DYSON_E_BAD_ARG, "sweeps is NULL");
  CK(cudaDeviceSynchronize());
  const int nb = p->g.nb, P = p->g.p;
  std::vector<unsigned long long> per((size_t)K * nb * P);
  CK(cudaMemcpy(per.data(), p->b.sweeps, per.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
  for (int k = 0; k < K; ++k)
    for (int i = 0; i < P; ++i) {
      unsigned long long t = 0;
      for (int c = 0; c < nb; ++c) t += per[((size_t)k * nb + c) * P + i];
      sweeps[(size_t)k * P + i] = t;
    }
  return DYSON_OK;
}

int dyson_apply_H(dyson_plan p, int K, const double* omega, const double* V, const double* sigma,
                  const double* x, double* y, int mem_kind, void* stream) {
  int rc;
  if ((rc = check_plan(p)) || (rc = check_mem(mem_kind))) return rc;
  // device buffers are read in place, so K is not bounded by the plan's capacity
  if (K < 1 || (mem_kind == DYSON_MEM_HOST && K > p->Kcap))
    return fail(DYSON_E_BAD_ARG, "K must be >= 1 (and <= max_freqs with host buffers)");
  if (!x || !y) return fail(DYSON_E_BAD_ARG, "x and y must not be NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)K * p->g.N * sizeof(cxd);
  const cxd* xd = reinterpret_cast<const cxd*>(x);
  cxd* yd = reinterpret_cast<cxd*>(y);
  const double *Vd = V, *wd = omega;
  const cxd* sd = reinterpret_cast<const cxd*>(sigma);
  if (mem_kind == DYSON_MEM_HOST) {          // stage into the plan; device inputs are read in place
    if ((rc = stage_inputs(p, K, omega, V, sigma, nullptr, s))) return rc;
    CK(cudaMemcpyAsync(p->b.u, x, bytes, cudaMemcpyHostToDevice, s));
    xd = p->b.u;
    yd = p->b.out;
    Vd = p->b.V;
    wd = p->b.omega;
    sd = p->b.sigma;
  } else if (!omega || !V || !sigma) {
    return fail(DYSON_E_BAD_ARG, "omega, V and sigma must not be NULL");
  }
  LK(launch_spmv<double>(p->g, Vd, wd, sd, xd, yd, K, s));
  if (mem_kind == DYSON_MEM_HOST) CK(cudaMemcpyAsync(y, yd, bytes, cudaMemcpyDeviceToHost, s));
  return finish(mem_kind, s);
}

int dyson_apply_H_c64(dyson_plan p, int K, const double* omega, const double* V,
                      const double* sigma, const float* x, float* y, int mem_kind, void* stream) {
  int rc;
  if ((rc = check_plan(p)) || (rc = check_mem(mem_kind))) return rc;
  // device buffers are read in place, so K is not bounded by the plan's capacity
  if (K < 1 || (mem_kind == DYSON_MEM_HOST && K > p->Kcap))
    return fail(DYSON_E_BAD_ARG, "K must be >= 1 (and <= max_freqs with host buffers)");
  if (!x || !y) return fail(DYSON_E_BAD_ARG, "x and y must not be NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)K * p->g.N * sizeof(cxf);
  const cxf* xd = reinterpret_cast<const cxf*>(x);
  cxf* yd = reinterpret_cast<cxf*>(y);
  const double *Vd = V, *wd = omega;
  const cxd* sd = reinterpret_cast<const cxd*>(sigma);
  if (mem_kind == DYSON_MEM_HOST) {          // stage into the plan; device inputs are read in place
    if ((rc = stage_inputs(p, K, omega, V, sigma, nullptr, s))) return rc;
    CK(cudaMemcpyAsync(p->b.u, x, bytes, cudaMemcpyHostToDevice, s));
    xd = reinterpret_cast<const cxf*>(p->b.u);
    yd = reinterpret_cast<cxf*>(p->b.out);
    Vd = p->b.V;
    wd = p->b.omega;
    sd = p->b.sigma;
  } else if (!omega || !V || !sigma) {
    return fail(DYSON_E_BAD_ARG, "omega, V and sigma must not be NULL");
  }
  LK(launch_spmv<float>(p->g, Vd, wd, sd, xd, yd, K, s));
  if (mem_kind == DYSON_MEM_HOST) CK(cudaMemcpyAsync(y, yd, bytes, cudaMemcpyDeviceToHost, s));
  return finish(mem_kind, s);
}

int dyson_subdomain_diag(dyson_plan p, int K, const double* omega, const double* V,
                         const double* sigma, double* diagB, int mem_kind, void* stream) {
  int rc;
  if ((rc = check_plan(p)) || (rc = check_K(p, K)) || (rc = check_mem(mem_kind))) return rc;
  if (!diagB) return fail(DYSON_E_BAD_ARG, "diagB must not be NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = stage_inputs(p, K, omega, V, sigma, nullptr, s))) return rc;
  if ((rc = enqueue_factor(p, K, s))) return rc;
  cxd* dst = mem_kind == DYSON_MEM_HOST ? p->b.out : reinterpret_cast<cxd*>(diagB);
  LK(launch_scatter(p->g, p->b, K, p->b.diagB, dst, p->g.Ndd, s));
  if (mem_kind == DYSON_MEM_HOST)
    CK(cudaMemcpyAsync(diagB, dst, (size_t)K * p->g.N * sizeof(cxd), cudaMemcpyDeviceToHost, s));
  return finish(mem_kind, s);
}

int dyson_subdomain_solve(dyson_plan p, int K, const double* omega, const double* V,
                          const double* sigma, const double* q, double* w, int mem_kind,
                          void* stream) {
  int rc;
  if ((rc = check_plan(p)) || (rc = check_K(p, K)) || (rc = check_mem(mem_kind))) return rc;
  if ((rc = check_sweeps(p))) return rc;
  if (!q || !w) return fail(DYSON_E_BAD_ARG, "q and w must not be NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = stage_inputs(p, K, omega, V, sigma, nullptr, s))) return rc;
  const size_t bytes = (size_t)K * p->g.N * sizeof(cxd);
  const cxd* qn = reinterpret_cast<const cxd*>(q);
  if (mem_kind == DYSON_MEM_HOST) {
    CK(cudaMemcpyAsync(p->b.out, q, bytes, cudaMemcpyHostToDevice, s));
    qn = p->b.out;
  }
  if ((rc = enqueue_factor(p, K, s))) return rc;
  LK(launch_gather(p->g, p->b, K, qn, p->b.acc, p->g.Ndd, s));
  if (p->mixed) LK(launch_bsolve<float>(p->g, p->b, K, p->b.acc, p->b.u, s));
  else LK(launch_bsolve<double>(p->g, p->b, K, p->b.acc, p->b.u, s));
  cxd* dst = mem_kind == DYSON_MEM_HOST ? p->b.out : reinterpret_cast<cxd*>(w);
  LK(launch_scatter(p->g, p->b, K, p->b.u, dst, p->g.Ndd, s));
  if (mem_kind == DYSON_MEM_HOST) CK(cudaMemcpyAsync(w, dst, bytes, cudaMemcpyDeviceToHost, s));
  return finish(mem_kind, s);
}

int dyson_xmatvec(dyson_plan p, int K, const double* omega, const double* V, const double* sigma,
                  const double* q, double* u, int mem_kind, void* stream) {
  int rc;
  if ((rc = check_plan(p)) || (rc = check_K(p, K)) || (rc = check_mem(mem_kind))) return rc;
  if ((rc = check_sweeps(p))) return rc;
  if (!q || !u) return fail(DYSON_E_BAD_ARG, "q and u must not be NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = stage_inputs(p, K, omega, V, sigma, nullptr, s))) return rc;
  const Geo& g = p->g;
  const size_t bytes = (size_t)K * g.N * sizeof(cxd);
  const cxd* qn = reinterpret_cast<const cxd*>(q);
  if (mem_kind == DYSON_MEM_HOST) {
    CK(cudaMemcpyAsync(p->b.out, q, bytes, cudaMemcpyHostToDevice, s));
    qn = p->b.out;
  }
  if ((rc = enqueue_factor(p, K, s))) return rc;
  if (p->mixed) LK(launch_precond<float>(g, p->b, K, s));
  else LK(launch_precond<double>(g, p->b, K, s));
  // one vector per frequency: column 0 of block 0, result in the frequency's first slot
  LK(launch_gather(g, p->b, K, qn, p->b.Q, (size_t)(g.k_max + g.nb) * g.Ndd, s));
  LK(launch_qsplit(g, p->b, K, s));
  CK(cudaMemsetAsync(p->b.st, 0, (size_t)K * ST_N * sizeof(int), s));
  if (g.p > 1) {
    if (p->mixed) LK(launch_xmatvec<float>(g, p->b, K, 0, 1, 1, s));
    else LK(launch_xmatvec<double>(g, p->b, K, 0, 0, 1, s));
  } else {
    CK(cudaMemsetAsync(p->b.u, 0, (size_t)K * g.nb * g.Ndd * sizeof(cxd), s));
  }
  cxd* dst = mem_kind == DYSON_MEM_HOST ? p->b.out : reinterpret_cast<cxd*>(u);
  LK(launch_scatter(g, p->b, K, p->b.u, dst, (size_t)g.nb * g.Ndd, s));
  if (mem_kind == DYSON_MEM_HOST) CK(cudaMemcpyAsync(u, dst, bytes, cudaMemcpyDeviceToHost, s));
  return finish(mem_kind, s);
}

}  // extern "C"

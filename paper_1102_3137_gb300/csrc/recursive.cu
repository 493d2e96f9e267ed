// Recursive decomposition of the low-rank correction method (Sec. 2.3, last
// paragraph): the domain is cut in two by one interface line, each half is cut
// again across the other axis, and so on, the number of domains alternating
// (d_x, d_y) = (2, 1), (1, 2), (2, 1), ... level by level.
//
// Reading of the recursion taken here (the paper states only the alternation):
// a box of the lattice is the principal submatrix H_box of H on its sites, open
// at the box edges.  Its diagonal is
//
//   diag(H_box^-1) ~ [diag of each half's inverse, by the same rule one level
//                     down; 0 on the cut line] + diag(Q_k T_k Q_k^T),
//
// Q_k T_k Q_k^T the rank-k complex-symmetric Lanczos approximation (Eq. 10) of
// X_box = H_box^-1 - blkdiag(H_1^-1, H_2^-1, 0) (Eqs. 5-8 on the box), started
// from the caller's q1 restricted to the box.  The line sits at the middle of
// the cut axis, the half before it one site shorter when the box has an even
// extent there; an axis shorter than 3 sites cannot be cut and the other is
// cut instead; boxes of at most min_sites sites (or too thin along both axes)
// are inverted exactly.  Hence diag(G) at a site is the exact diagonal of its
// leaf box plus the correction of every box above it.
//
// GPU form.  Every box is one two-strip (p = 2) low-rank solve of an ordinary
// plan and every leaf the slice recursion of a p = 1 plan, all frequencies of
// the call batched in each.  A box is gathered into its plan's input buffers
// oriented so that the cut line runs along the plan's fast axis (transposed
// when the cut is across x) and reflected along the slow axis when the plan's
// partition would put the line one row off the middle rule above (the plan
// makes the first strip the taller one).  After a box's solve its correction
// diag(Q T Q^T), still in the plan's subdomain-first layout, is added into the
// output at the box's sites; a leaf's exact diagonal is added likewise.  The
// boxes of one level are disjoint, so they run on several streams (each with
// its own plans) without racing on the output; levels run one after another
// in a fixed order, so results are bitwise repeatable.
#include <algorithm>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "dyson.h"
#include "dyson_common.cuh"
#include "host_internal.h"

namespace {

struct RBox {
  int x0, y0, nx, ny;   // origin and extents in the lattice
  int leaf;             // 1: inverted exactly; 0: cut in two
  int transpose;        // the plan's fast axis is the lattice's y axis
  int reflect;          // the plan's slow axis runs backwards
  int Lf, Ls;           // the plan's fast and slow extents
  int plan;             // index into the plan table
};

// Where a box site of the plan's natural order lands in the lattice.
struct RMap {
  int x0, y0, Lf, Ls, transpose, reflect, Lx;
  __device__ __forceinline__ int site(int nat) const {
    const int xf = nat % Lf, ys = nat / Lf;
    const int s = reflect ? Ls - 1 - ys : ys;
    const int gx = transpose ? x0 + s : x0 + xf;
    const int gy = transpose ? y0 + xf : y0 + s;
    return gx + Lx * gy;
  }
};

// The box's share of V, sigma (all K frequencies) and q1, in the plan's order.
__global__ void k_rec_gather(RMap m, int N, const double* V, const cxd* sigma, const double* q1,
                             double* Vb, cxd* sigmab, double* q1b) {
  const int kf = blockIdx.y;
  const int Nb = m.Lf * m.Ls;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Nb; i += gridDim.x * blockDim.x) {
    const int gi = m.site(i);
    sigmab[(size_t)kf * Nb + i] = sigma[(size_t)kf * N + gi];
    if (kf == 0) {
      Vb[i] = V[gi];
      q1b[i] = q1[gi];
    }
  }
}

// out += src at the box's sites (src in the plan's subdomain-first layout), and
// the box's status flags folded into the running ones: every flag but
// TERMINATED OR-ed, TERMINATED AND-ed (the result is exact only when every box
// closed its Krylov space).  The boxes of a level are disjoint, so the adds never
// meet; the flags are shared by all of them and folded atomically.
__global__ void k_rec_add(RMap m, int N, int Ndd, const int* dd2nat, const cxd* src, cxd* out,
                          const int* st_box, int* st_or, int* st_and) {
  const int kf = blockIdx.y;
  if (st_box && blockIdx.x == 0 && threadIdx.x == 0) {   // boxes of a level run concurrently
    const int s = st_box[kf];
    atomicOr(st_or + kf, s & ~DYSON_ST_TERMINATED);
    atomicAnd(st_and + kf, s);
  }
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < Ndd; k += gridDim.x * blockDim.x) {
    const int nat = dd2nat[k];
    if (nat < 0) continue;
    const size_t o = (size_t)kf * N + m.site(nat);
    const cxd a = out[o], b = src[(size_t)kf * Ndd + k];
    out[o] = cxd{a.x + b.x, a.y + b.y};
  }
}

__global__ void k_rec_init(int K, int N, cxd* out, int* st_or, int* st_and) {
  const int kf = blockIdx.y;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st_or[kf] = 0;
    st_and[kf] = DYSON_ST_TERMINATED;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
    out[(size_t)kf * N + i] = cxd{0.0, 0.0};
}

__global__ void k_rec_status(int K, const int* st_or, const int* st_and, int* status) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x)
    status[k] = st_or[k] | (st_and[k] & DYSON_ST_TERMINATED);
}

int grid_for(int n) { return std::max(1, std::min((n + 255) / 256, 1024)); }

}  // namespace

struct dyson_rplan_s {
  dyson_geometry gi;
  int Lx, Ly, N, Kcap, min_sites, first_cut;
  int device;
  int nstreams;
  std::vector<std::vector<RBox>> levels;   // boxes of each level, leaves included
  struct Shape {
    int Lf, Ls, leaf;
  };
  std::vector<Shape> shapes;
  std::vector<dyson_plan> plans;           // [stream][shape], NULL where unused
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> ev;             // fork + one join per stream
  size_t bytes;                            // box plans + the staging below
  char* arena;                             // inputs and outputs of host-memory calls, status words
  double *omega_h, *V_h, *q1_h;
  cxd *sigma_h, *out_h;
  int *st_or, *st_and, *status_h;
  int n_internal, n_leaves;
};

namespace {

int rfail(int code, const std::string& msg) { return dyson_internal_fail(code, "recursive: " + msg); }

#define RCK(call)                                                                       \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return rfail(DYSON_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// The box tree, level by level, by the rule in the file comment.
void build_tree(std::vector<std::vector<RBox>>& levels, int min_sites, int x0, int x1, int y0, int y1,
                int cut_y, int level) {
  const int nx = x1 - x0 + 1, ny = y1 - y0 + 1;
  if ((int)levels.size() <= level) levels.resize(level + 1);
  RBox b;
  std::memset(&b, 0, sizeof(b));
  b.x0 = x0;
  b.y0 = y0;
  b.nx = nx;
  b.ny = ny;
  const long long size = (long long)nx * ny;
  if (size <= min_sites || (!cut_y && nx < 3) || (cut_y && ny < 3)) {
    if (size <= min_sites || (nx < 3 && ny < 3)) {
      // leaf: the slice recursion runs along the longer axis (narrower slices)
      b.leaf = 1;
      b.transpose = ny > nx ? 1 : 0;
      b.Lf = b.transpose ? ny : nx;
      b.Ls = b.transpose ? nx : ny;
      levels[level].push_back(b);
      return;
    }
    cut_y = !cut_y;
  }
  b.transpose = cut_y ? 0 : 1;
  b.Lf = cut_y ? nx : ny;
  b.Ls = cut_y ? ny : nx;
  b.reflect = (b.Ls % 2 == 0) ? 1 : 0;
  levels[level].push_back(b);
  if (cut_y) {
    const int ym = (y0 + y1) / 2;
    build_tree(levels, min_sites, x0, x1, y0, ym - 1, 0, level + 1);
    build_tree(levels, min_sites, x0, x1, ym + 1, y1, 0, level + 1);
  } else {
    const int xm = (x0 + x1) / 2;
    build_tree(levels, min_sites, x0, xm - 1, y0, y1, 1, level + 1);
    build_tree(levels, min_sites, xm + 1, x1, y0, y1, 1, level + 1);
  }
}

int check_tree_args(const dyson_geometry* geom, int min_sites, int first_cut) {
  if (geom->dim != 2) return rfail(DYSON_E_BAD_ARG, "the recursion is defined for 2D lattices (dim = 2)");
  if (geom->L[0] < 1 || geom->L[1] < 1) return rfail(DYSON_E_BAD_ARG, "lattice extents must be >= 1");
  if ((long long)geom->L[0] * geom->L[1] > (1LL << 30)) return rfail(DYSON_E_UNSUPPORTED, "lattice too large");
  if (min_sites < 1) return rfail(DYSON_E_BAD_ARG, "min_sites must be >= 1");
  if (first_cut != DYSON_CUT_X && first_cut != DYSON_CUT_Y)
    return rfail(DYSON_E_BAD_ARG, "first_cut must be DYSON_CUT_X or DYSON_CUT_Y");
  return DYSON_OK;
}

int shape_index(dyson_rplan_s* r, int Lf, int Ls, int leaf) {
  for (size_t k = 0; k < r->shapes.size(); ++k)
    if (r->shapes[k].Lf == Lf && r->shapes[k].Ls == Ls && r->shapes[k].leaf == leaf) return (int)k;
  r->shapes.push_back({Lf, Ls, leaf});
  return (int)r->shapes.size() - 1;
}

dyson_plan& plan_at(dyson_rplan_s* r, int stream, int shape) {
  return r->plans[(size_t)stream * r->shapes.size() + shape];
}

void destroy(dyson_rplan_s* r) {
  if (!r) return;
  cudaSetDevice(r->device);
  for (dyson_plan p : r->plans)
    if (p) dyson_plan_destroy(p);
  for (cudaStream_t s : r->streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : r->ev) cudaEventDestroy(e);
  cudaFree(r->arena);
  delete r;
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// With device buffers the kernels of every box dereference the caller's pointers
// on the plan's device: anything else is refused before work is enqueued.
int check_dev_ptr(const void* ptr, int dev, const char* what) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return rfail(DYSON_E_BAD_ARG, std::string("cannot query ") + what);
  }
  if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev)
    return rfail(DYSON_E_BAD_ARG, std::string(what) + " is not device memory of the plan's device");
  return DYSON_OK;
}

// one box: gather, solve (or factor a leaf), add its share into out
int run_box(dyson_rplan_s* r, const RBox& b, int si, int K, const double* omega, const double* V,
            const cxd* sigma, const double* q1, cxd* out) {
  dyson_plan p = plan_at(r, si, b.plan);
  cudaStream_t s = r->streams[si];
  PlanDev d;
  int rc = dyson_internal_plan_dev(p, &d);
  if (rc) return rc;
  RMap m{b.x0, b.y0, b.Lf, b.Ls, b.transpose, b.reflect, r->Lx};
  RCK(cudaMemcpyAsync(d.omega, omega, K * sizeof(double), cudaMemcpyDeviceToDevice, s));
  k_rec_gather<<<dim3(grid_for(d.N), K), 256, 0, s>>>(m, r->N, V, sigma, q1, d.V,
                                                      reinterpret_cast<cxd*>(d.sigma), d.q1);
  RCK(cudaGetLastError());
  if (b.leaf) {
    if ((rc = dyson_internal_factor_resident(p, K, s))) return rc;
  } else if ((rc = dyson_internal_solve_resident(p, K, s))) {
    return rc;
  }
  const cxd* src = reinterpret_cast<const cxd*>(b.leaf ? d.diagB : d.acc);
  k_rec_add<<<dim3(grid_for(d.Ndd), K), 256, 0, s>>>(m, r->N, d.Ndd, d.dd2nat, src, out,
                                                     b.leaf ? nullptr : d.status, r->st_or, r->st_and);
  RCK(cudaGetLastError());
  return DYSON_OK;
}

}  // namespace

extern "C" {

int dyson_recursive_plan_create(const dyson_geometry* geom, int min_sites, int first_cut, int streams,
                                dyson_rplan* out) {
  if (!geom || !out) return rfail(DYSON_E_BAD_ARG, "geometry or output handle is NULL");
  *out = nullptr;
  int rc0 = check_tree_args(geom, min_sites, first_cut);
  if (rc0) return rc0;
  if (geom->block_size > 1) return rfail(DYSON_E_BAD_ARG, "the recursion runs the scalar Lanczos recurrence (block_size 0 or 1)");
  if (streams < 0 || streams > 16) return rfail(DYSON_E_BAD_ARG, "streams must be in 0..16 (0: 4)");
  if (geom->max_freqs < 1 || geom->max_freqs > 65535) return rfail(DYSON_E_BAD_ARG, "max_freqs must be in 1..65535");
  if (geom->k_max < 1 || geom->k_max > 256) return rfail(DYSON_E_BAD_ARG, "k_max must be in 1..256");
  dyson_rplan_s* r = new dyson_rplan_s();
  r->gi = *geom;
  r->Lx = geom->L[0];
  r->Ly = geom->L[1];
  r->N = r->Lx * r->Ly;
  r->Kcap = geom->max_freqs;
  r->min_sites = min_sites;
  r->first_cut = first_cut;
  r->arena = nullptr;
  cudaGetDevice(&r->device);
  build_tree(r->levels, min_sites, 0, r->Lx - 1, 0, r->Ly - 1, first_cut == DYSON_CUT_Y ? 1 : 0, 0);
  size_t widest = 1;
  r->n_internal = r->n_leaves = 0;
  for (auto& lv : r->levels) {
    widest = std::max(widest, lv.size());
    for (RBox& b : lv) {
      b.plan = shape_index(r, b.Lf, b.Ls, b.leaf);
      (b.leaf ? r->n_leaves : r->n_internal)++;
    }
  }
  r->nstreams = (int)std::min<size_t>(widest, streams > 0 ? streams : 4);
  r->plans.assign((size_t)r->nstreams * r->shapes.size(), nullptr);
  r->bytes = 0;
  int rc = DYSON_OK;
  // plans: box j of a level runs on stream j mod nstreams
  for (auto& lv : r->levels) {
    for (size_t j = 0; j < lv.size() && rc == DYSON_OK; ++j) {
      const RBox& b = lv[j];
      dyson_plan& p = plan_at(r, (int)(j % r->nstreams), b.plan);
      if (p) continue;
      dyson_geometry g = *geom;
      g.dim = 2;
      g.L[0] = b.Lf;
      g.L[1] = b.Ls;
      g.L[2] = 1;
      g.p = b.leaf ? 1 : 2;
      g.k_max = b.leaf ? 1 : geom->k_max;
      g.block_size = 0;
      rc = dyson_plan_create(&g, &p);
      if (rc == DYSON_OK) r->bytes += dyson_internal_plan_bytes(p);
      else
        dyson_internal_fail(rc, std::string("recursive: plan of a ") + std::to_string(b.Lf) + " x " +
                                    std::to_string(b.Ls) + (b.leaf ? " leaf" : " box") + ": " + dyson_last_error());
    }
  }
  if (rc == DYSON_OK) {
    const size_t K = r->Kcap, N = r->N;
    const size_t sz = al256(K * sizeof(double)) + 2 * al256(N * sizeof(double)) + 2 * al256(K * N * sizeof(cxd)) +
                      3 * al256(K * sizeof(int));
    cudaError_t e = cudaMalloc(&r->arena, sz);
    if (e != cudaSuccess) {
      cudaGetLastError();
      r->arena = nullptr;
      rc = rfail(DYSON_E_OOM, "staging buffers: " + std::string(cudaGetErrorString(e)));
    } else {
      r->bytes += sz;
      char* c = r->arena;
      r->omega_h = reinterpret_cast<double*>(c);
      c += al256(K * sizeof(double));
      r->V_h = reinterpret_cast<double*>(c);
      c += al256(N * sizeof(double));
      r->q1_h = reinterpret_cast<double*>(c);
      c += al256(N * sizeof(double));
      r->sigma_h = reinterpret_cast<cxd*>(c);
      c += al256(K * N * sizeof(cxd));
      r->out_h = reinterpret_cast<cxd*>(c);
      c += al256(K * N * sizeof(cxd));
      r->st_or = reinterpret_cast<int*>(c);
      c += al256(K * sizeof(int));
      r->st_and = reinterpret_cast<int*>(c);
      c += al256(K * sizeof(int));
      r->status_h = reinterpret_cast<int*>(c);
    }
  }
  for (int k = 0; k < r->nstreams && rc == DYSON_OK; ++k) {
    cudaStream_t s;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) rc = rfail(DYSON_E_CUDA, std::string("stream: ") + cudaGetErrorString(e));
    else r->streams.push_back(s);
  }
  for (int k = 0; k <= r->nstreams && rc == DYSON_OK; ++k) {
    cudaEvent_t e;
    cudaError_t c = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    if (c != cudaSuccess) rc = rfail(DYSON_E_CUDA, std::string("event: ") + cudaGetErrorString(c));
    else r->ev.push_back(e);
  }
  if (rc) {
    std::string msg = dyson_last_error();
    destroy(r);
    return dyson_internal_fail(rc, msg);
  }
  *out = r;
  return DYSON_OK;
}

int dyson_recursive_boxes(const dyson_geometry* geom, int min_sites, int first_cut, int* n, int* boxes) {
  if (!geom || !n) return rfail(DYSON_E_BAD_ARG, "geometry or n is NULL");
  int rc = check_tree_args(geom, min_sites, first_cut);
  if (rc) return rc;
  std::vector<std::vector<RBox>> levels;
  build_tree(levels, min_sites, 0, geom->L[0] - 1, 0, geom->L[1] - 1, first_cut == DYSON_CUT_Y ? 1 : 0, 0);
  int k = 0;
  for (size_t l = 0; l < levels.size(); ++l)
    for (const RBox& b : levels[l]) {
      if (boxes) {
        int* o = boxes + 8 * (size_t)k;
        o[0] = b.x0;
        o[1] = b.y0;
        o[2] = b.nx;
        o[3] = b.ny;
        o[4] = (int)l;
        o[5] = b.leaf;
        // the cut line's coordinate along the cut axis (-1 for a leaf), from the
        // orientation the box's plan uses: its interface row (the taller strip
        // first) mapped back through the reflection
        int line = -1;
        if (!b.leaf) {
          const int row = b.Ls / 2;   // the first strip has ceil((Ls - 1) / 2) rows, then the line
          const int s = b.reflect ? b.Ls - 1 - row : row;
          line = (b.transpose ? b.x0 : b.y0) + s;
        }
        o[6] = b.leaf ? -1 : (b.transpose ? 0 : 1);
        o[7] = line;
      }
      ++k;
    }
  *n = k;
  return DYSON_OK;
}

int dyson_recursive_plan_destroy(dyson_rplan r) {
  if (!r) return rfail(DYSON_E_BAD_ARG, "plan is NULL");
  destroy(r);
  return DYSON_OK;
}

int dyson_recursive_plan_info(dyson_rplan r, int* levels, int* boxes, int* leaves, int* plans,
                              size_t* bytes) {
  if (!r) return rfail(DYSON_E_BAD_ARG, "plan is NULL");
  if (levels) *levels = (int)r->levels.size();
  if (boxes) *boxes = r->n_internal;
  if (leaves) *leaves = r->n_leaves;
  if (plans) {
    int n = 0;
    for (dyson_plan p : r->plans) n += p ? 1 : 0;
    *plans = n;
  }
  if (bytes) *bytes = r->bytes;
  return DYSON_OK;
}

int dyson_recursive_solve(dyson_rplan r, int K, const double* omega, const double* V, const double* sigma,
                          const double* q1, double* diagG, int* status, int mem_kind, void* stream) {
  if (!r) return rfail(DYSON_E_BAD_ARG, "plan is NULL");
  if (K < 1 || K > r->Kcap) return rfail(DYSON_E_BAD_ARG, "K must be in 1..max_freqs (" + std::to_string(r->Kcap) + ")");
  if (!omega || !V || !sigma || !q1 || !diagG) return rfail(DYSON_E_BAD_ARG, "omega, V, sigma, q1 and diagG must not be NULL");
  if (mem_kind != DYSON_MEM_HOST && mem_kind != DYSON_MEM_DEVICE)
    return rfail(DYSON_E_BAD_ARG, "mem_kind must be DYSON_MEM_HOST or DYSON_MEM_DEVICE");
  RCK(cudaSetDevice(r->device));
  if (mem_kind == DYSON_MEM_DEVICE) {
    const void* ptrs[6] = {omega, V, sigma, q1, diagG, status};
    const char* names[6] = {"omega", "V", "sigma", "q1", "diagG", "status"};
    for (int k = 0; k < 6; ++k) {
      if (!ptrs[k]) continue;
      int rc = check_dev_ptr(ptrs[k], r->device, names[k]);
      if (rc) return rc;
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t N = r->N;
  const double *om = omega, *Vd = V, *q1d = q1;
  const cxd* sg = reinterpret_cast<const cxd*>(sigma);
  cxd* out = reinterpret_cast<cxd*>(diagG);
  if (mem_kind == DYSON_MEM_HOST) {
    RCK(cudaMemcpyAsync(r->omega_h, omega, K * sizeof(double), cudaMemcpyHostToDevice, s));
    RCK(cudaMemcpyAsync(r->V_h, V, N * sizeof(double), cudaMemcpyHostToDevice, s));
    RCK(cudaMemcpyAsync(r->q1_h, q1, N * sizeof(double), cudaMemcpyHostToDevice, s));
    RCK(cudaMemcpyAsync(r->sigma_h, sigma, K * N * sizeof(cxd), cudaMemcpyHostToDevice, s));
    om = r->omega_h;
    Vd = r->V_h;
    q1d = r->q1_h;
    sg = r->sigma_h;
    out = r->out_h;
  }
  k_rec_init<<<dim3(grid_for(r->N), K), 256, 0, s>>>(K, r->N, out, r->st_or, r->st_and);
  RCK(cudaGetLastError());
  for (auto& lv : r->levels) {
    const int ns = (int)std::min<size_t>(lv.size(), r->nstreams);
    RCK(cudaEventRecord(r->ev[0], s));
    for (int k = 0; k < ns; ++k) RCK(cudaStreamWaitEvent(r->streams[k], r->ev[0], 0));
    for (size_t j = 0; j < lv.size(); ++j) {
      int rc = run_box(r, lv[j], (int)(j % r->nstreams), K, om, Vd, sg, q1d, out);
      if (rc) return rc;
    }
    for (int k = 0; k < ns; ++k) {
      RCK(cudaEventRecord(r->ev[1 + k], r->streams[k]));
      RCK(cudaStreamWaitEvent(s, r->ev[1 + k], 0));
    }
  }
  int* st = (mem_kind == DYSON_MEM_DEVICE && status) ? status : r->status_h;
  k_rec_status<<<1, 256, 0, s>>>(K, r->st_or, r->st_and, st);
  RCK(cudaGetLastError());
  if (mem_kind == DYSON_MEM_HOST) {
    RCK(cudaMemcpyAsync(diagG, r->out_h, K * N * sizeof(cxd), cudaMemcpyDeviceToHost, s));
    if (status) RCK(cudaMemcpyAsync(status, r->status_h, K * sizeof(int), cudaMemcpyDeviceToHost, s));
    RCK(cudaStreamSynchronize(s));
  }
  return DYSON_OK;
}

}  // extern "C"

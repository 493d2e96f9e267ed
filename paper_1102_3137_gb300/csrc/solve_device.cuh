// Lanczos-based low-rank correction: device code shared by the per-step
// kernels (included by k_solve.cu and the two k_xmatvec_*.cu units).
//
// Every kernel here runs one thread-block cluster per frequency with one CTA
// per subdomain (cluster = p CTAs, grid = p x K).  CTA i owns subdomain i's
// slice block of every DD-layout vector and interface layer i (i < p-1).
// Reductions over a frequency's lattice are two-level: a fixed-order
// block reduction, then every CTA reads the p partials from distributed
// shared memory in rank order, so all CTAs of a cluster hold bit-identical
// scalars and take identical branch decisions (no CTA can leave a cluster
// barrier behind).  Every kernel that reads peers' shared memory ends with a
// cluster barrier, so no CTA exits while a peer may still be reading it.
//
// X-"matvec" (Sec. 2.3, Eqs. 6-8).  The paper defines u = v - w with
// H v = q and w = blkdiag(B^-1, 0) q.  Eliminating the subdomain unknowns
// of H v = q gives, without ever forming S = C - E^T B^-1 E (Eq. 4),
//     y   = S^-1 (E^T B^-1 q_B - q_C),
//     u_B = B^-1 E y,   u_C = -y,
// which is exactly v - w with no cancellation.  S y = r is solved by COCG
// (conjugate orthogonal CG: CG in the bilinear form, valid for complex
// symmetric S) whose S-products are subdomain solves with boundary-only
// right-hand sides.
#pragma once
#include <cooperative_groups.h>

#include "dyson.h"
#include "dyson_common.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr double TERM_TOL = 1e-12;    // ||r||_2 <= TERM_TOL * max|T|: invariant subspace
constexpr double BRK_TOL = 1e-14;     // |r^T r| <= BRK_TOL * ||r||^2: breakdown
constexpr int KMAX_SMEM = 256;        // largest Lanczos rank cap
// refinement stops early once a pass no longer shrinks the squared FP64
// residual 16-fold (the residual has reached its rounding floor)
constexpr double REFINE_STALL = 1.0 / 16.0;

__device__ __forceinline__ size_t own_idx(const Geo& g, int i, int e, int nsub) {
  return e < nsub ? (size_t)i * nsub + e : (size_t)g.ifc_off + (size_t)i * g.A + (e - nsub);
}
__device__ __forceinline__ int own_count(const Geo& g, int i) {
  return g.Lx * g.W + (i < g.p - 1 ? g.A : 0);
}

// ---------------------------------------------------------------- reductions
struct RedSmem {
  cxd wred[DY_WARPS * 8];
  cxd slot[2 * 8];
  cxd res[8];
};

__device__ __forceinline__ cxd warp_sum(cxd v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
  }
  return v;
}

// Sum NV complex partials over the whole cluster; every thread gets the totals.
template <int NV>
__device__ void cluster_sum(cg::cluster_group& cl, RedSmem& rs, int& phase, int p, cxd (&v)[NV]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) rs.wred[wid * 8 + k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    cxd s = {0, 0};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = s + rs.wred[w * 8 + threadIdx.x];
    rs.slot[phase * 8 + threadIdx.x] = s;
  }
  cl.sync();
  if (threadIdx.x < NV) {
    cxd s = {0, 0};
    for (int r = 0; r < p; ++r) {
      const cxd* rem = cl.map_shared_rank(rs.slot, r);
      s = s + rem[phase * 8 + threadIdx.x];
    }
    rs.res[threadIdx.x] = s;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = rs.res[k];
  phase ^= 1;
}

// CTA-local sum (no cluster exchange)
template <int NV>
__device__ void block_sum(RedSmem& rs, cxd (&v)[NV]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) rs.wred[wid * 8 + k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    cxd s = {0, 0};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = s + rs.wred[w * 8 + threadIdx.x];
    rs.res[threadIdx.x] = s;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = rs.res[k];
  __syncthreads();
}

// ---------------------------------------------------------------- async copies
// g_s blocks stream from HBM into a ring of shared-memory slots with 1D bulk
// copies (cp.async.bulk, completion counted on an mbarrier per slot).  Every
// wait is bounded by the global timer: on time-out the kernel records
// DYSON_ST_WAIT_TIMEOUT and goes on (no CTA may leave its cluster's barriers);
// the thread then waits on the ring no more in that sweep, and no thread of the
// CTA waits in its later sweeps.
constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;   // 2 s
constexpr int ST_WAIT_TIMEOUT = DYSON_ST_WAIT_TIMEOUT;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_wait_for(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  return mbar_wait_for(bar, parity, WAIT_LIMIT_NS);
}
// A copy-ring wait that gives up for good: once one of this thread's waits has
// run out (dead, a register flag, seeded from the CTA's shared flag at the start
// of each sweep), its later waits return at once, so a lost copy costs the
// kernel one wait limit per thread and sweep instead of one per slice step.
__device__ __forceinline__ void ring_wait(uint64_t* bar, uint32_t parity, bool& dead, int* err) {
  if (dead) return;
  if (!mbar_wait(bar, parity)) {
    dead = true;
    *err = 1;
  }
}

// Per-CTA copy pipeline: S slots of one W x W block each, one mbarrier per slot.
struct Pipe {
  uint64_t* bar;   // [S] in static shared memory
  void* ring;      // S slots in dynamic shared memory
  void* ybuf;      // forward intermediates in shared memory, or null (global scratch)
  int S;
  int CR;          // rows of a slice block per streamed chunk (= W unless W > 64)
  unsigned seq;    // blocks issued (= consumed) so far by this CTA (left chain of the two-chain form)
  unsigned seq2;   // the same for the right chain of the two-chain form
  int* err;        // shared flag: a bounded wait ran out
};

constexpr int MAX_STAGES = 8;

__device__ void pipe_init(Pipe& pp) {
  if (threadIdx.x == 0) {
    for (int k = 0; k < pp.S; ++k) mbar_init(pp.bar + k, 1);
    *pp.err = 0;
    fence_mbar_init();
  }
  __syncthreads();
}

// ---------------------------------------------------------------- block sweep
// Solve B_i x = rhs by block forward/back substitution with the stored
// left-connected inverses g_s (Eq. 7 and the S-products):
//   forward  y_s = g_s (rhs_s - t y_{s-1})
//   backward x_s = y_s - t g_s x_{s+1}
// The right-hand side is either a full DD block (src) or boundary-only,
// t times an interface-layer vector on the first/last slow rows (E y).
// The 2 Lx - 1 blocks the two passes read stream through the copy ring.
template <typename R>
struct SweepArgs {
  const cx<R>* g;      // [Lx][W][W] this subdomain's factors
  cx<R>* y;            // [Lx][W] scratch for the forward intermediates
  const cxd* src;      // full right-hand side (subdomain block) or null
  const cx<R>* lay_lo; // interface layer below (i-1), boundary mode
  const cx<R>* lay_hi; // interface layer above (i), boundary mode
  cxd* dst;            // full solution out (subdomain block) or null
  int dst_op;          // 0 store, 1 add, 2 subtract, 3 store negated
  double in_scale;     // src is multiplied by this when rounded to R
  double out_scale;    // x is multiplied by this when written to dst
  cx<R>* bnd_lo;       // solution on the lowest slow row, layer layout (or null)
  cx<R>* bnd_hi;       // solution on the highest slow row
};

// Thread layout of the block products y = g_s z (g_s complex symmetric, so its
// row r is also its column r and rows are read contiguously): warp w owns rows
// [w*RPW, (w+1)*RPW); inside the warp lane = rr*G + cg, row group rr, column
// class cg (columns cg, cg+G, ...: CPG of them); the G partial sums of a row
// are added with log2(G) butterfly shuffles and lane rr*G finishes the row.
struct SweepLayout {
  int RPW, G, CPG;
};
__host__ __device__ inline SweepLayout sweep_layout(int rows, int W) {
  int rpw = (rows + DY_WARPS - 1) / DY_WARPS, p2 = 1;
  while (p2 < rpw) p2 <<= 1;
  SweepLayout L;
  L.RPW = p2;
  L.G = 32 / p2;
  L.CPG = (W + L.G - 1) / L.G;
  return L;
}

// The sequential slice loop touches only shared memory (or the per-unit
// scratch) and R-precision registers: a parallel pre-pass converts the
// right-hand side into the row buffer yb (rhs_s in row s), the forward pass
// overwrites row s with y_s, the backward pass with x_s, and a parallel
// post-pass converts the rows to FP64 and writes the requested outputs.  On
// GB300 FP64 issue is ~1/64 of FP32, so keeping conversions out of the
// dependent chain matters as much as keeping global loads out of it.
template <typename R>
__device__ void sweep_chunked(const Geo& g, int i, const SweepArgs<R>& a, cx<R>* sm, Pipe& pp,
                              unsigned long long* cnt);

// Pre-pass of a sweep (all threads): the right-hand side rows in precision R
// into the row buffer yb [Lx][W] (zero on padding columns).
// In complex64 the FP64 right-hand side is converted by integer operations
// (d2f_bits) and scaled in FP32, so the pass issues nothing on the FP64 pipe;
// the scale only keeps the values inside the FP32 range, so its product is
// taken in FP32 whenever it is itself well inside that range.
template <typename R>
__device__ __forceinline__ void sweep_prepass(const Geo& g, int i, const SweepArgs<R>& a, cx<R>* yb) {
  const int W = g.W, Lx = g.Lx, T = g.T, w = T * g.h[i], nrow = Lx * W;
  const R t = (R)g.t;
  const double as = fabs(a.in_scale);
  const bool fast = sizeof(R) == 4 && as > 1e-30 && as < 1e30;
  const R scf = (R)a.in_scale;
  if constexpr (sizeof(R) == 4) {
    if (a.src && fast) {                 // the common case: PU rows' loads in flight per thread
      constexpr int PU = 4;
      const int nt = (int)blockDim.x;
      for (int e0 = threadIdx.x; e0 < nrow; e0 += PU * nt) {
        cxd v[PU];
        bool on[PU];
#pragma unroll
        for (int u = 0; u < PU; ++u) {
          const int e = e0 + u * nt, j = e % W;
          on[u] = e < nrow && j < w;
          v[u] = on[u] ? a.src[e] : cxd{0, 0};
        }
#pragma unroll
        for (int u = 0; u < PU; ++u) {
          const int e = e0 + u * nt;
          if (e < nrow) yb[e] = on[u] ? scf * c2f_bits(v[u]) : cx<R>{0, 0};
        }
      }
      return;
    }
  }
  for (int e = threadIdx.x; e < nrow; e += (int)blockDim.x) {
    const int s = e / W, j = e - s * W;
    cxd v = {0, 0};
    if (j < w) {
      if (a.src && fast) {
        if constexpr (sizeof(R) == 4) yb[e] = scf * c2f_bits(a.src[e]);
        continue;
      } else if (a.src) {
        v = a.in_scale * a.src[e];
      } else {
        cx<R> u = {0, 0};
        if (a.lay_lo && j < T) u = u + t * a.lay_lo[s + Lx * j];
        if (a.lay_hi && j >= w - T) u = u + t * a.lay_hi[s + Lx * (j - (w - T))];
        yb[e] = u;
        continue;
      }
    }
    yb[e] = cconv<R>(v);
  }
}

// Post-pass of a sweep (all threads): the solution rows x_s in yb to the FP64
// outputs and the boundary-row copies.
// In complex64 the scale is applied in FP32 and the value widened by integer
// operations (f2d_bits); only the accumulating add/subtract into the FP64
// output runs on the FP64 pipe.
template <typename R>
__device__ __forceinline__ void sweep_postpass(const Geo& g, int i, const SweepArgs<R>& a,
                                               const cx<R>* yb) {
  const int W = g.W, Lx = g.Lx, T = g.T, w = T * g.h[i], nrow = Lx * W;
  const double os = fabs(a.out_scale);
  const bool fast = sizeof(R) == 4 && os > 1e-30 && os < 1e30;
  const R scf = (R)a.out_scale;
  if constexpr (sizeof(R) == 4) {
    if (a.dst && fast) {                 // the common case: PU rows' loads in flight per thread
      constexpr int PU = 4;
      const int nt = (int)blockDim.x;
      const bool rd = a.dst_op == 1 || a.dst_op == 2;
      for (int e0 = threadIdx.x; e0 < nrow; e0 += PU * nt) {
        cx<R> xr[PU];
        cxd dv[PU];
        bool on[PU];
#pragma unroll
        for (int u = 0; u < PU; ++u) {
          const int e = e0 + u * nt, j = e % W;
          on[u] = e < nrow && j < w;
          xr[u] = on[u] ? yb[e] : cx<R>{0, 0};
          dv[u] = (on[u] && rd) ? a.dst[e] : cxd{0, 0};
        }
#pragma unroll
        for (int u = 0; u < PU; ++u) {
          if (!on[u]) continue;
          const int e = e0 + u * nt, s = e / W, j = e - s * W;
          const cxd xd = c2d_bits(scf * xr[u]);
          cxd* d = a.dst + e;
          if (a.dst_op == 0) *d = xd;
          else if (a.dst_op == 1) *d = dv[u] + xd;
          else if (a.dst_op == 2) *d = dv[u] - xd;
          else *d = -xd;
          if (a.bnd_lo && j < T) a.bnd_lo[s + Lx * j] = xr[u];
          if (a.bnd_hi && j >= w - T) a.bnd_hi[s + Lx * (j - (w - T))] = xr[u];
        }
      }
      return;
    }
  }
  for (int e = threadIdx.x; e < nrow; e += (int)blockDim.x) {
    const int s = e / W, j = e - s * W;
    if (j >= w) continue;
    const cx<R> xr = yb[e];
    if (a.dst) {
      cxd xd;
      if constexpr (sizeof(R) == 4) {
        if (fast) xd = c2d_bits(scf * xr);
        else xd = a.out_scale * cconv<double>(xr);
      } else {
        xd = a.out_scale * cconv<double>(xr);
      }
      cxd* d = a.dst + e;
      if (a.dst_op == 0) *d = xd;
      else if (a.dst_op == 1) *d = *d + xd;
      else if (a.dst_op == 2) *d = *d - xd;
      else *d = -xd;
    }
    if (a.bnd_lo && j < T) a.bnd_lo[s + Lx * j] = xr;
    if (a.bnd_hi && j >= w - T) a.bnd_hi[s + Lx * (j - (w - T))] = xr;
  }
}

// y = g z for one slice block of the complex64 two-sided factors, by one warp:
// lane r owns rows r (and r + 32 when WF = 64).  The block is stored with
// column pairs interleaved, so row r's columns 2k, 2k+1 are one 16-byte load
// at pair index k W + r (contiguous over the warp, conflict-free), against the
// broadcast pair z[2k], z[2k+1].  Loads are plain (an inline-asm load with a
// memory clobber ordered every load behind the previous one: 2.6x slower per
// slice) and issued four pairs at a time, so a batch's loads are in flight
// together; 8 (4 at WF = 64) accumulators per row keep the FMA chains short.
template <int WF>
__device__ __forceinline__ void pair_product(const cxf* blk, const cxf* z, int W, int lane, cxf& m0,
                                             cxf& m1) {
  const float4* g4 = reinterpret_cast<const float4*>(blk);
  const float4* z4 = reinterpret_cast<const float4*>(z);
  const int r0 = lane, r1 = lane + 32;
  const bool v0 = r0 < W, v1 = WF > 32 && r1 < W;
  constexpr int NA = WF <= 32 ? 8 : 4;
  constexpr int NB = WF <= 32 ? WF / 8 : 1;        // batches unrolled (one at a time at WF = 64)
  cxf a[NA], c[NA];
#pragma unroll
  for (int u = 0; u < NA; ++u) a[u] = c[u] = cxf{0.f, 0.f};
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll NB
  for (int k0 = 0; k0 < WF / 2; k0 += 4) {
    float4 zz[4], ga[4], gb[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      // pairs past W and rows past W read in-range entries (pair 0, row 0) and
      // the z pair is zeroed, so they add nothing; such rows are not written
      const int k = k0 + q;
      const bool on = 2 * k < W;
      const int kk = on ? k : 0;
      zz[q] = on ? z4[kk] : zero;
      ga[q] = g4[(size_t)kk * W + (v0 ? r0 : 0)];
      if (WF > 32) gb[q] = g4[(size_t)kk * W + (v1 ? r1 : 0)];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int u = (2 * q) & (NA - 1);
      const cxf za = {zz[q].x, zz[q].y}, zb = {zz[q].z, zz[q].w};
      a[u] = cfma(cxf{ga[q].x, ga[q].y}, za, a[u]);
      a[u + 1] = cfma(cxf{ga[q].z, ga[q].w}, zb, a[u + 1]);
      if (WF > 32) {
        c[u] = cfma(cxf{gb[q].x, gb[q].y}, za, c[u]);
        c[u + 1] = cfma(cxf{gb[q].z, gb[q].w}, zb, c[u + 1]);
      }
    }
  }
  if constexpr (NA == 8) {
    m0 = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    m1 = ((c[0] + c[1]) + (c[2] + c[3])) + ((c[4] + c[5]) + (c[6] + c[7]));
  } else {
    m0 = (a[0] + a[1]) + (a[2] + a[3]);
    m1 = (c[0] + c[1]) + (c[2] + c[3]);
  }
}

// complex64 sweep for W <= 64 on the two-sided factors (k_factor, mixed form),
// with m = Lx / 2:
//   left chain, warp 0:   y_s = g_s (rhs_s - t y_{s-1})        s = 0 .. m-1
//   right chain, warp 1:  y_s = g_s (rhs_s - t y_{s+1})        s = Lx-1 .. m+1
//   middle, warp 0:       x_m = G_mm (rhs_m - t y_{m-1} - t y_{m+1})
//   back-substitution:    x_s = y_s - t g_s x_{s+1}  (warp 0, s = m-1 .. 0)
//                         x_s = y_s - t g_s x_{s-1}  (warp 1, s = m+1 .. Lx-1)
// so the dependent chain is ~Lx slices instead of 2 Lx - 1, and each slice
// is one warp's work: in complex64 a W x W product is far cheaper than a CTA
// barrier plus a cross-warp reduction, which is what a slice cost when eight
// warps shared it.  Each chain streams its own blocks through its half of the
// copy ring and its lane 0 refills a slot as soon as the warp has read it.
// Rows of the right-hand side (forward) and of y (backward) are read two
// slices ahead into registers, which hides the latency when the row buffer is
// the global scratch.  The other warps join for the pre- and post-passes.
template <int WF>
__device__ void sweep_pair(const Geo& g, int i, const SweepArgs<float>& a, cxf* sm, Pipe& pp,
                           unsigned long long* cnt) {
  using C = cxf;
  bool dead = *pp.err != 0;              // an earlier wait of this CTA ran out
  const int W = g.W, Lx = g.Lx, m = Lx / 2, qR = Lx - 1 - m;
  const int NLL = 2 * m + 1, NLR = 2 * qR;
  C* zL = sm;                            // [2][W] left chain z
  C* zR = sm + 2 * W;                    // [2][W] right chain z
  C* zM = sm + 4 * W;                    // [2][W] partial middle z from the left / right chain
  C* ring = reinterpret_cast<C*>(pp.ring);
  C* yb = pp.ybuf ? reinterpret_cast<C*>(pp.ybuf) : a.y;   // [Lx][W] row buffer
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const float t = (float)g.t;
  const int WW = W * W;
  const uint32_t bytes = (uint32_t)(WW * sizeof(C));
  const int SL = pp.S / 2, SR = pp.S - SL;
  const int r0 = lane, r1 = lane + 32;
  const bool v0 = r0 < W, v1 = WF > 32 && r1 < W;
  auto sliceL = [&](int n) { return n <= m ? n : 2 * m - n; };
  auto sliceR = [&](int n) { return n < qR ? Lx - 1 - n : m + 1 + (n - qR); };
  // the chains consume their blocks in order: slot and phase parity advance
  // by one step at a time (no division on the critical path); the block of
  // step n + S_c reuses the slot of step n
  int curL = (int)(pp.seq % (unsigned)SL), curR = SL + (int)(pp.seq2 % (unsigned)SR);
  uint32_t phL = (pp.seq / (unsigned)SL) & 1u, phR = (pp.seq2 / (unsigned)SR) & 1u;
  auto issue_at = [&](int slot, int slice) {
    bulk_load(ring + (size_t)slot * WW, a.g + (size_t)slice * WW, bytes, pp.bar + slot);
  };
  // Wait for the block of step n, product with z, refill the slot.  The
  // slot's loads have completed (their values are in p0, p1) before the warp
  // barrier, so the copy that overwrites it needs no proxy fence.
  auto stepL = [&](int n, const C* z, C& p0, C& p1) {
    const int sl = curL;
    ring_wait(pp.bar + sl, phL, dead, pp.err);
    pair_product<WF>(ring + (size_t)sl * WW, z, W, lane, p0, p1);
    __syncwarp();
    if (lane == 0 && n + SL < NLL) issue_at(sl, sliceL(n + SL));
    if (++curL == SL) {
      curL = 0;
      phL ^= 1u;
    }
  };
  auto stepR = [&](int n, const C* z, C& p0, C& p1) {
    const int sl = curR;
    ring_wait(pp.bar + sl, phR, dead, pp.err);
    pair_product<WF>(ring + (size_t)sl * WW, z, W, lane, p0, p1);
    __syncwarp();
    if (lane == 0 && n + SR < NLR) issue_at(sl, sliceR(n + SR));
    if (++curR == SL + SR) {
      curR = SL;
      phR ^= 1u;
    }
  };
  auto rd = [&](int s, int r) { return yb[(size_t)s * W + r]; };


  __syncthreads();                       // previous users of ring, z buffers and yb are done
  if (tid == 0) {
    fence_proxy_async();
    for (int n = 0; n < SL && n < NLL; ++n) issue_at((int)((pp.seq + n) % (unsigned)SL), sliceL(n));
    for (int n = 0; n < SR && n < NLR; ++n) issue_at(SL + (int)((pp.seq2 + n) % (unsigned)SR), sliceR(n));
  }
  sweep_prepass<float>(g, i, a, yb);
  __syncthreads();

  // ---- forward chains
  if (wid == 0) {
    C fA0 = {0, 0}, fA1 = {0, 0}, fB0 = {0, 0}, fB1 = {0, 0};   // rhs_{s+1}, s even / odd
    if (v0) zL[r0] = rd(0, r0);
    if (v1) zL[r1] = rd(0, r1);
    if (m >= 1) {
      if (v0) fA0 = rd(1, r0);
      if (v1) fA1 = rd(1, r1);
    }
    if (m >= 2) {
      if (v0) fB0 = rd(2, r0);
      if (v1) fB1 = rd(2, r1);
    }
    __syncwarp();
    auto fwd = [&](int s, C& f0, C& f1) {
      C y0, y1;
      stepL(s, zL + (s & 1) * W, y0, y1);
      C* zn = (s + 1 < m) ? zL + ((s + 1) & 1) * W : zM;   // z_{s+1}, or the middle partial
      if (v0) {
        yb[(size_t)s * W + r0] = y0;
        zn[r0] = f0 - t * y0;
        if (s + 3 <= m) f0 = rd(s + 3, r0);
      }
      if (v1) {
        yb[(size_t)s * W + r1] = y1;
        zn[r1] = f1 - t * y1;
        if (s + 3 <= m) f1 = rd(s + 3, r1);
      }
      __syncwarp();
    };
    for (int s = 0; s < m; s += 2) {
      fwd(s, fA0, fA1);
      if (s + 1 < m) fwd(s + 1, fB0, fB1);
    }
    if (m == 0) {                        // no left chain: the middle starts from rhs_0
      if (v0) zM[r0] = rd(0, r0);
      if (v1) zM[r1] = rd(0, r1);
    }
  } else if (wid == 1 && qR > 0) {
    C fA0 = {0, 0}, fA1 = {0, 0}, fB0 = {0, 0}, fB1 = {0, 0};   // rhs_{s-1}, step n even / odd
    if (v0) zR[r0] = rd(Lx - 1, r0);
    if (v1) zR[r1] = rd(Lx - 1, r1);
    if (Lx - 2 > m) {
      if (v0) fA0 = rd(Lx - 2, r0);
      if (v1) fA1 = rd(Lx - 2, r1);
    }
    if (Lx - 3 > m) {
      if (v0) fB0 = rd(Lx - 3, r0);
      if (v1) fB1 = rd(Lx - 3, r1);
    }
    __syncwarp();
    auto fwd = [&](int n, C& f0, C& f1) {
      const int s = Lx - 1 - n;
      C y0, y1;
      stepR(n, zR + (n & 1) * W, y0, y1);
      const bool inner = s - 1 > m;
      C* zn = inner ? zR + ((n + 1) & 1) * W : zM + W;
      if (v0) {
        yb[(size_t)s * W + r0] = y0;
        zn[r0] = inner ? f0 - t * y0 : -(t * y0);
        if (s - 3 > m) f0 = rd(s - 3, r0);
      }
      if (v1) {
        yb[(size_t)s * W + r1] = y1;
        zn[r1] = inner ? f1 - t * y1 : -(t * y1);
        if (s - 3 > m) f1 = rd(s - 3, r1);
      }
      __syncwarp();
    };
    for (int n = 0; n < qR; n += 2) {
      fwd(n, fA0, fA1);
      if (n + 1 < qR) fwd(n + 1, fB0, fB1);
    }
  }
  __syncthreads();                       // both chains' partials of the middle z written

  // ---- middle block
  if (wid == 0) {
    C* zc = zL + (m & 1) * W;
    if (v0) zc[r0] = qR > 0 ? zM[r0] + zM[W + r0] : zM[r0];
    if (v1) zc[r1] = qR > 0 ? zM[r1] + zM[W + r1] : zM[r1];
    __syncwarp();
    C x0, x1;
    stepL(m, zc, x0, x1);
    C* znL = zL + ((m + 1) & 1) * W;
    C* znR = zR + (qR & 1) * W;
    if (v0) {
      yb[(size_t)m * W + r0] = x0;
      znL[r0] = x0;
      znR[r0] = x0;
    }
    if (v1) {
      yb[(size_t)m * W + r1] = x1;
      znL[r1] = x1;
      znR[r1] = x1;
    }
  }
  __syncthreads();                       // x_m visible to the right chain

  // ---- back-substitution
  if (wid == 0 && m > 0) {
    C yA0 = {0, 0}, yA1 = {0, 0}, yB0 = {0, 0}, yB1 = {0, 0};   // y_s, step parity
    if (v0) yA0 = rd(m - 1, r0);
    if (v1) yA1 = rd(m - 1, r1);
    if (m >= 2) {
      if (v0) yB0 = rd(m - 2, r0);
      if (v1) yB1 = rd(m - 2, r1);
    }
    auto bwd = [&](int n, C& y0v, C& y1v) {
      const int s = 2 * m - n;
      C p0, p1;
      stepL(n, zL + (n & 1) * W, p0, p1);
      C* zn = zL + ((n + 1) & 1) * W;
      if (v0) {
        const C xv = y0v - t * p0;
        yb[(size_t)s * W + r0] = xv;
        zn[r0] = xv;
        if (s >= 2) y0v = rd(s - 2, r0);
      }
      if (v1) {
        const C xv = y1v - t * p1;
        yb[(size_t)s * W + r1] = xv;
        zn[r1] = xv;
        if (s >= 2) y1v = rd(s - 2, r1);
      }
      __syncwarp();
    };
    for (int n = m + 1; n < NLL; n += 2) {
      bwd(n, yA0, yA1);
      if (n + 1 < NLL) bwd(n + 1, yB0, yB1);
    }
  } else if (wid == 1 && qR > 0) {
    C yA0 = {0, 0}, yA1 = {0, 0}, yB0 = {0, 0}, yB1 = {0, 0};
    if (v0) yA0 = rd(m + 1, r0);
    if (v1) yA1 = rd(m + 1, r1);
    if (m + 2 < Lx) {
      if (v0) yB0 = rd(m + 2, r0);
      if (v1) yB1 = rd(m + 2, r1);
    }
    auto bwd = [&](int n, C& y0v, C& y1v) {
      const int s = m + 1 + (n - qR);
      C p0, p1;
      stepR(n, zR + (n & 1) * W, p0, p1);
      C* zn = zR + ((n + 1) & 1) * W;
      if (v0) {
        const C xv = y0v - t * p0;
        yb[(size_t)s * W + r0] = xv;
        zn[r0] = xv;
        if (s + 2 < Lx) y0v = rd(s + 2, r0);
      }
      if (v1) {
        const C xv = y1v - t * p1;
        yb[(size_t)s * W + r1] = xv;
        zn[r1] = xv;
        if (s + 2 < Lx) y1v = rd(s + 2, r1);
      }
      __syncwarp();
    };
    for (int n = qR; n < NLR; n += 2) {
      bwd(n, yA0, yA1);
      if (n + 1 < NLR) bwd(n + 1, yB0, yB1);
    }
  }
  __syncthreads();                       // yb complete for the post-pass
  sweep_postpass<float>(g, i, a, yb);
  pp.seq += NLL;
  pp.seq2 += NLR;
  if (tid == 0 && cnt) *cnt += 1;
}

// WF selects the sweep form at compile time, so each kernel carries only its
// own: 0 = row-chunked (W > 64); otherwise W <= WF <= 64, the two-chain
// single-warp form in complex64 and the 8-warp form in FP64.
template <typename R, int WF>
__device__ void sweep(const Geo& g, int i, const SweepArgs<R>& a, cx<R>* sm, Pipe& pp,
                      unsigned long long* cnt) {
  if constexpr (WF == 0) {
    sweep_chunked<R>(g, i, a, sm, pp, cnt);
    return;
  } else if constexpr (sizeof(R) == 4) {
    sweep_pair<WF>(g, i, a, sm, pp, cnt);
    return;
  }
  bool dead = *pp.err != 0;              // an earlier wait of this CTA ran out
  const int W = g.W, Lx = g.Lx;
  const SweepLayout L = sweep_layout(W, W);
  cx<R>* zbuf = sm;                      // [2][W]: z of the current and of the next slice
  cx<R>* ring = reinterpret_cast<cx<R>*>(pp.ring);
  cx<R>* yb = pp.ybuf ? reinterpret_cast<cx<R>*>(pp.ybuf) : a.y;   // [Lx][W] row buffer
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int rr = lane / L.G, cg = lane - rr * L.G;
  const int row = wid * L.RPW + rr;      // the row this lane works on
  const bool rvalid = row < W;
  const bool owner = rvalid && cg == 0;  // finishes the row
  // rows of one warp are W entries apart, i.e. in the same banks; starting each
  // row group at a different multiple of G spreads a warp's accesses over all banks
  const int rot = (W % L.G == 0) ? (rr * L.G) % W : 0;
  const R t = (R)g.t;
  const int WW = W * W;
  const uint32_t bytes = (uint32_t)(WW * sizeof(cx<R>));
  const int NL = 2 * Lx - 1;
  const int S = pp.S;
  auto slice_of = [&](int n) { return n < Lx ? n : 2 * Lx - 2 - n; };
  auto issue = [&](int n) {
    const unsigned q = pp.seq + n;
    const int slot = (int)(q % S);
    bulk_load(ring + (size_t)slot * WW, a.g + (size_t)slice_of(n) * WW, bytes, pp.bar + slot);
  };

  __syncthreads();                       // previous users of ring, zbuf and yb are done
  if (tid == 0) {
    fence_proxy_async();
    for (int n = 0; n < S && n < NL; ++n) issue(n);
  }
  sweep_prepass<R>(g, i, a, yb);
  __syncthreads();
  if (owner) zbuf[row] = yb[row];
  // Rows are read two slices ahead into ping-pong registers: with yb in shared
  // memory this costs nothing, with the global scratch it hides the latency.
  cx<R> fA = {0, 0}, fB = {0, 0};
  if (owner) {
    if (Lx > 1) fA = yb[W + row];
    if (Lx > 2) fB = yb[2 * W + row];
  }
  __syncthreads();

  // one slice of either pass: wait for g_s, row products, butterfly
  auto product = [&](int n) -> cx<R> {
    const unsigned q = pp.seq + n;
    const int slot = (int)(q % S);
    ring_wait(pp.bar + slot, (q / S) & 1u, dead, pp.err);
    const cx<R>* grow = ring + (size_t)slot * WW + (size_t)row * W;
    const cx<R>* zc = zbuf + (n & 1) * W;
    cx<R> acc = {0, 0};
    if (rvalid) {
#pragma unroll 4
      for (int k = 0; k < L.CPG; ++k) {
        const int base = cg + L.G * k;   // columns interleaved over the group's lanes
        if (base < W) {
          int col = base + rot;          // rotated per row group: no bank conflicts
          if (col >= W) col -= W;
          acc = cfma(grow[col], zc[col], acc);
        }
      }
    }
    for (int off = L.G >> 1; off > 0; off >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
    }
    return acc;
  };
  auto finish = [&](int n) {
    __syncthreads();                     // slot n and z of slice n fully read; z of n+1 written
    if (tid == 0 && n + S < NL) {
      fence_proxy_async();
      issue(n + S);
    }
  };
  // forward: y_s = g_s (rhs_s - t y_{s-1}); row s of yb becomes y_s
  auto fwd = [&](int s, cx<R>& f) {
    const cx<R> m = product(s);
    if (owner) {
      cx<R>* zn = zbuf + ((s + 1) & 1) * W;
      yb[(size_t)s * W + row] = m;
      zn[row] = (s + 1 < Lx) ? f - t * m : m;   // x_{Lx-1} = y_{Lx-1}
      if (s + 3 < Lx) f = yb[(size_t)(s + 3) * W + row];
    }
    finish(s);
  };
  for (int s = 0; s < Lx; s += 2) {
    fwd(s, fA);
    if (s + 1 < Lx) fwd(s + 1, fB);
  }
  // backward: x_s = y_s - t g_s x_{s+1}; row s of yb becomes x_s
  cx<R> yA = {0, 0}, yB = {0, 0};
  if (owner && Lx > 1) {
    yA = yb[(size_t)(Lx - 2) * W + row];
    if (Lx > 2) yB = yb[(size_t)(Lx - 3) * W + row];
  }
  auto bwd = [&](int s, cx<R>& yv) {
    const int n = 2 * Lx - 2 - s;
    const cx<R> m = product(n);
    if (owner) {
      cx<R>* zn = zbuf + ((n + 1) & 1) * W;
      const cx<R> xv = yv - t * m;
      yb[(size_t)s * W + row] = xv;
      zn[row] = xv;
      if (s >= 2) yv = yb[(size_t)(s - 2) * W + row];
    }
    finish(n);
  };
  for (int s = Lx - 2; s >= 0; s -= 2) {
    bwd(s, yA);
    if (s - 1 >= 0) bwd(s - 1, yB);
  }
  sweep_postpass<R>(g, i, a, yb);
  pp.seq += NL;
  if (tid == 0 && cnt) *cnt += 1;
}

// Wide slices (W > 64, 3D slabs): a slice block streams as NC = W / CR chunks
// of CR rows (NC = 1 when whole blocks leave enough ring slots); each chunk's
// rows are finished as soon as it arrives and its slot is released after a
// barrier.  The row buffer yb is always on chip on this path.
template <typename R>
__device__ void sweep_chunked(const Geo& g, int i, const SweepArgs<R>& a, cx<R>* sm, Pipe& pp,
                              unsigned long long* cnt) {
  bool dead = *pp.err != 0;              // an earlier wait of this CTA ran out
  const int W = g.W, Lx = g.Lx, T = g.T, w = T * g.h[i];
  const int CR = pp.CR, NC = W / CR;
  const SweepLayout L = sweep_layout(CR, W);
  cx<R>* zbuf = sm;
  cx<R>* ring = reinterpret_cast<cx<R>*>(pp.ring);
  cx<R>* yb = reinterpret_cast<cx<R>*>(pp.ybuf);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int rr = lane / L.G, cg = lane - rr * L.G;
  const int lrow = wid * L.RPW + rr;     // row inside a chunk
  const bool rvalid = lrow < CR;
  const bool owner = rvalid && cg == 0;
  const int rot = (W % L.G == 0) ? (rr * L.G) % W : 0;
  const R t = (R)g.t;
  const int WW = W * W, CW = CR * W;
  const uint32_t bytes = (uint32_t)(CW * sizeof(cx<R>));
  const int NL = 2 * Lx - 1, NQ = NL * NC;
  const int S = pp.S;
  const int nrow = Lx * W;
  auto slice_of = [&](int n) { return n < Lx ? n : 2 * Lx - 2 - n; };
  auto issue = [&](int q) {
    const unsigned qq = pp.seq + q;
    const int slot = (int)(qq % S);
    const int n = q / NC, c = q - n * NC;
    bulk_load(ring + (size_t)slot * CW, a.g + (size_t)slice_of(n) * WW + (size_t)c * CW, bytes,
              pp.bar + slot);
  };

  __syncthreads();
  if (tid == 0) {
    fence_proxy_async();
    for (int q = 0; q < S && q < NQ; ++q) issue(q);
  }
  for (int e = tid; e < nrow; e += (int)blockDim.x) {
    const int s = e / W, j = e - s * W;
    cxd v = {0, 0};
    if (j < w) {
      if (a.src) {
        v = a.in_scale * a.src[e];
      } else {
        cx<R> u = {0, 0};
        if (a.lay_lo && j < T) u = u + t * a.lay_lo[s + Lx * j];
        if (a.lay_hi && j >= w - T) u = u + t * a.lay_hi[s + Lx * (j - (w - T))];
        yb[e] = u;
        continue;
      }
    }
    yb[e] = cconv<R>(v);
  }
  __syncthreads();
  for (int e = tid; e < W; e += (int)blockDim.x) zbuf[e] = yb[e];
  __syncthreads();
  for (int n = 0; n < NL; ++n) {
    const int s = slice_of(n);
    const cx<R>* zc = zbuf + (n & 1) * W;
    cx<R>* zn = zbuf + ((n + 1) & 1) * W;
    for (int c = 0; c < NC; ++c) {
      const int q = n * NC + c;
      const unsigned qq = pp.seq + q;
      const int slot = (int)(qq % S);
      ring_wait(pp.bar + slot, (qq / S) & 1u, dead, pp.err);
      const cx<R>* grow = ring + (size_t)slot * CW + (size_t)lrow * W;
      cx<R> acc = {0, 0};
      if (rvalid) {
#pragma unroll 4
        for (int k = 0; k < L.CPG; ++k) {
          const int base = cg + L.G * k;
          if (base < W) {
            int col = base + rot;
            if (col >= W) col -= W;
            acc = cfma(grow[col], zc[col], acc);
          }
        }
      }
      for (int off = L.G >> 1; off > 0; off >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
      }
      if (owner) {
        const int row = c * CR + lrow;
        if (n < Lx) {                    // forward: row s of yb becomes y_s
          yb[(size_t)s * W + row] = acc;
          zn[row] = (s + 1 < Lx) ? yb[(size_t)(s + 1) * W + row] - t * acc : acc;
        } else {                         // backward: row s of yb becomes x_s
          const cx<R> xv = yb[(size_t)s * W + row] - t * acc;
          yb[(size_t)s * W + row] = xv;
          zn[row] = xv;
        }
      }
      __syncthreads();                   // chunk slot released; rows of z for n+1 written
      if (tid == 0 && q + S < NQ) {
        fence_proxy_async();
        issue(q + S);
      }
    }
  }
  for (int e = tid; e < nrow; e += (int)blockDim.x) {
    const int s = e / W, j = e - s * W;
    if (j >= w) continue;
    const cx<R> xr = yb[e];
    if (a.dst) {
      const cxd xd = a.out_scale * cconv<double>(xr);
      cxd* d = a.dst + e;
      if (a.dst_op == 0) *d = xd;
      else if (a.dst_op == 1) *d = *d + xd;
      else if (a.dst_op == 2) *d = *d - xd;
      else *d = -xd;
    }
    if (a.bnd_lo && j < T) a.bnd_lo[s + Lx * j] = xr;
    if (a.bnd_hi && j >= w - T) a.bnd_hi[s + Lx * (j - (w - T))] = xr;
  }
  pp.seq += NQ;
  if (tid == 0 && cnt) *cnt += 1;
}

template <typename R>
__device__ __forceinline__ SweepArgs<R> sweep_base(const Geo& g, const Bufs& b, int vs, int i) {
  SweepArgs<R> a;
  const size_t nsub = (size_t)g.Lx * g.W;
  a.g = reinterpret_cast<const cx<R>*>(b.g) + ((size_t)slot_freq(g, vs) * g.p + i) * nsub * g.W;
  a.y = reinterpret_cast<cx<R>*>(b.yscr) + ((size_t)vs * g.p + i) * nsub;
  a.src = nullptr;
  a.lay_lo = a.lay_hi = nullptr;
  a.dst = nullptr;
  a.dst_op = 0;
  a.in_scale = a.out_scale = 1.0;
  a.bnd_lo = a.bnd_hi = nullptr;
  return a;
}

__device__ __forceinline__ unsigned long long* sweep_cnt(const Geo& g, const Bufs& b, int vs, int i) {
  return b.sweeps ? b.sweeps + (size_t)vs * g.p + i : nullptr;
}
// boundary-row values and interface vectors are kept in the sweep precision R
// (their buffers are sized for complex128, so either precision fits)
template <typename R>
__device__ __forceinline__ cx<R>* bnd_ptr(const Geo& g, const Bufs& b, int vs, int i, int hi) {
  return reinterpret_cast<cx<R>*>(b.bnd) + (((size_t)vs * g.p + i) * 2 + hi) * g.A;
}
template <typename R>
__device__ __forceinline__ cx<R>* ifv_ptr(const Geo& g, const Bufs& b, int vs, int slot) {
  return reinterpret_cast<cx<R>*>(b.ifv) + ((size_t)vs * IF_N + slot) * nifc(g);
}

// ---------------------------------------------------------------- interface pieces
template <typename R>
__device__ __forceinline__ cx<R> shfl_up_c(cx<R> v, int d) {
  return {__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d)};
}
template <typename R>
__device__ __forceinline__ cx<R> shfl_down_c(cx<R> v, int d) {
  return {__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d)};
}

// Affine map on a pair of complex values: (s0, s1) -> (a s0 + b s1 + u, c s0 + d s1 + v).
template <typename R>
struct Aff2 {
  cx<R> a, b, c, d, u, v;
};
template <typename R>
__device__ __forceinline__ Aff2<R> aff_id() {
  return {{1, 0}, {0, 0}, {0, 0}, {1, 0}, {0, 0}, {0, 0}};
}
// o after in
template <typename R>
__device__ __forceinline__ Aff2<R> aff_after(const Aff2<R>& o, const Aff2<R>& in) {
  return {o.a * in.a + o.b * in.c, o.a * in.b + o.b * in.d, o.c * in.a + o.d * in.c,
          o.c * in.b + o.d * in.d, o.a * in.u + o.b * in.v + o.u, o.c * in.u + o.d * in.v + o.v};
}
template <typename R>
__device__ __forceinline__ Aff2<R> aff_shfl_up(const Aff2<R>& f, int d) {
  return {shfl_up_c(f.a, d), shfl_up_c(f.b, d), shfl_up_c(f.c, d),
          shfl_up_c(f.d, d), shfl_up_c(f.u, d), shfl_up_c(f.v, d)};
}
template <typename R>
__device__ __forceinline__ Aff2<R> aff_shfl_down(const Aff2<R>& f, int d) {
  return {shfl_down_c(f.a, d), shfl_down_c(f.b, d), shfl_down_c(f.c, d),
          shfl_down_c(f.d, d), shfl_down_c(f.u, d), shfl_down_c(f.v, d)};
}

// Apply the banded interface preconditioner along the x lines of layer i:
// z = M^-1 r with M = L D L^T (complex symmetric, no conjugation; L unit lower
// with sub-diagonals l1, l2, l2 = 0 where only the tridiagonal part is kept):
//   forward   y_x = r_x - l1_x y_{x-1} - l2_x y_{x-2},   w_x = y_x / d_x
//   backward  z_x = w_x - l1_{x+1} z_{x+1} - l2_{x+2} z_{x+2}
// Each recurrence is a chain of affine maps on the pair state (y_x, y_{x-1})
// (resp. (z_x, z_{x+1})): one warp per line, 128 sites (4 per lane) per pass
// with the state carried from pass to pass; each lane composes its 4 sites'
// maps, a 5-step warp scan composes across lanes, then the lanes finish
// their sites.  Factors per site: 1/d_x, l1_x, l2_x.
//
// r is the COCG residual, rewritten in this kernel between calls: it must be
// read through the coherent path, never as const __restrict__ (which lets the
// compiler use non-coherent loads whose cached lines can be stale by the next
// iteration).  The preconditioner factors are read-only for the kernel's life.
//
// Not inlined: the scan's state would otherwise compete for registers with the
// whole X-matvec kernel (capped at 128 per thread for two CTAs per SM) and
// spill inside the sweeps.
template <typename R>
__device__ __noinline__ void precond_apply(const Geo& g, const Bufs& b, int vs, int i, const cx<R>* r,
                                           cx<R>* z) {
  using C = cx<R>;
  constexpr int E = 4, CH = 32 * E;
  const int Lx = g.Lx, A = g.A;
  const C* __restrict__ pre =
      reinterpret_cast<const C*>(b.pre) + ((size_t)slot_freq(g, vs) * nifc(g) + (size_t)i * A) * 3;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const C zero = {0, 0};
  for (int tr = wid; tr < g.T; tr += (int)(blockDim.x >> 5)) {
    const int o = Lx * tr;
    const C* invd = pre + o;
    const C* l1 = pre + A + o;
    const C* l2 = pre + 2 * A + o;
    C c0v = zero, c1v = zero;              // (y, y_prev) entering the pass
    for (int c0 = 0; c0 < Lx; c0 += CH) {
      const int x0 = c0 + lane * E;
      // site x: (s0, s1) -> (-l1_x s0 - l2_x s1 + r_x, s0); the coefficients are
      // re-read in the apply pass rather than held in registers
      Aff2<R> P = aff_id<R>();
#pragma unroll
      for (int k = 0; k < E; ++k) {
        const int x = x0 + k;
        if (x < Lx) P = aff_after(Aff2<R>{-l1[x], -l2[x], {1, 0}, zero, r[o + x], zero}, P);
      }
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {   // inclusive scan: lanes l-d.. then l
        const Aff2<R> q = aff_shfl_up(P, d);
        if (lane >= d) P = aff_after(P, q);
      }
      // state entering this lane: the previous lane's prefix applied to the carry
      C s0 = P.a * c0v + P.b * c1v + P.u, s1 = P.c * c0v + P.d * c1v + P.v;
      s0 = shfl_up_c(s0, 1);
      s1 = shfl_up_c(s1, 1);
      if (lane == 0) {
        s0 = c0v;
        s1 = c1v;
      }
#pragma unroll
      for (int k = 0; k < E; ++k) {
        const int x = x0 + k;
        if (x < Lx) {
          const C y = r[o + x] - l1[x] * s0 - l2[x] * s1;
          s1 = s0;
          s0 = y;
          z[o + x] = y * invd[x];
        }
      }
      c0v = cx<R>{__shfl_sync(0xffffffffu, s0.x, 31), __shfl_sync(0xffffffffu, s0.y, 31)};
      c1v = cx<R>{__shfl_sync(0xffffffffu, s1.x, 31), __shfl_sync(0xffffffffu, s1.y, 31)};
    }
    __syncwarp();
    C e0v = zero, e1v = zero;              // (z, z_next) entering the pass from the right
    const int nch = (Lx + CH - 1) / CH;
    for (int c = nch - 1; c >= 0; --c) {
      const int x0 = c * CH + lane * E;
      // site x: (s0, s1) -> (-l1_{x+1} s0 - l2_{x+2} s1 + w_x, s0)
      auto m1 = [&](int x) { return (x + 1 < Lx) ? l1[x + 1] : zero; };
      auto m2 = [&](int x) { return (x + 2 < Lx) ? l2[x + 2] : zero; };
      Aff2<R> Q = aff_id<R>();
#pragma unroll
      for (int k = E - 1; k >= 0; --k) {
        const int x = x0 + k;
        if (x < Lx) Q = aff_after(Aff2<R>{-m1(x), -m2(x), {1, 0}, zero, z[o + x], zero}, Q);
      }
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {   // inclusive suffix scan: lanes l+d.. then l
        const Aff2<R> q = aff_shfl_down(Q, d);
        if (lane + d < 32) Q = aff_after(Q, q);
      }
      C s0 = Q.a * e0v + Q.b * e1v + Q.u, s1 = Q.c * e0v + Q.d * e1v + Q.v;
      s0 = shfl_down_c(s0, 1);
      s1 = shfl_down_c(s1, 1);
      if (lane == 31) {
        s0 = e0v;
        s1 = e1v;
      }
#pragma unroll
      for (int k = E - 1; k >= 0; --k) {
        const int x = x0 + k;
        if (x < Lx) {
          const C v = z[o + x] - m1(x) * s0 - m2(x) * s1;
          s1 = s0;
          s0 = v;
          z[o + x] = v;
        }
      }
      e0v = cx<R>{__shfl_sync(0xffffffffu, s0.x, 0), __shfl_sync(0xffffffffu, s0.y, 0)};
      e1v = cx<R>{__shfl_sync(0xffffffffu, s1.x, 0), __shfl_sync(0xffffffffu, s1.y, 0)};
    }
  }
}

// (C p)[a] on layer l: the Dyson matrix restricted to the interface layer,
// with its diagonal d_C precomputed in R precision.
template <typename R>
__device__ __forceinline__ cx<R> layer_C_apply(const Geo& g, const cx<R>* dC, const cx<R>* pv, int a) {
  const int Lx = g.Lx, x = a % Lx, tr = a / Lx;
  cx<R> nb = {0, 0};
  if (x > 0) nb = nb + pv[a - 1];
  if (x < Lx - 1) nb = nb + pv[a + 1];
  if (tr > 0) nb = nb + pv[a - Lx];
  if (tr < g.T - 1) nb = nb + pv[a + Lx];
  return dC[a] * pv[a] + (R)g.t * nb;
}

// ---------------------------------------------------------------- reductions in R
template <typename R>
__device__ __forceinline__ cx<R> warp_sum_r(cx<R> v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
  }
  return v;
}
// Cluster-wide sums in R precision (partials exchanged through the same
// shared slots as cluster_sum, widened to double there).
template <typename R, int NV>
__device__ void cluster_sum_r(cg::cluster_group& cl, RedSmem& rs, int& phase, int p, cx<R> (&v)[NV]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum_r(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) rs.wred[wid * 8 + k] = cconv<double>(v[k]);
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    cxd s = {0, 0};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = s + rs.wred[w * 8 + threadIdx.x];
    rs.slot[phase * 8 + threadIdx.x] = s;
  }
  cl.sync();
  if (threadIdx.x < NV) {
    cxd s = {0, 0};
    for (int r = 0; r < p; ++r) {
      const cxd* rem = cl.map_shared_rank(rs.slot, r);
      s = s + rem[phase * 8 + threadIdx.x];
    }
    rs.res[threadIdx.x] = s;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = cconv<R>(rs.res[k]);
  phase ^= 1;
}

// COCG for S y = b on the interface (S = C - E^T B^-1 E never formed), all in
// precision R: the FP64 form solves to krylov_tol in FP64; the mixed form's
// inner solves (refined in FP64 one level up) run entirely in complex64.
// z = M_l^-1 r on interface line i with the exact layer block of S (2D
// strips): a dense symmetric product, thread a owning output a; the stored
// inverse is symmetric, so column a is read contiguously across threads.
// r must be complete (a barrier after its writers) before the call.
template <typename R>
__device__ __noinline__ void lpre_apply(const Geo& g, const Bufs& b, int vs, int i, const cx<R>* r,
                                        cx<R>* z) {
  using C = cx<R>;
  const int Lx = g.A;               // the layer's sites (Lx in 2D, Lx Ly in 3D)
  const C* rsh = r;                 // every thread reads all of r: served by L1
  const C* M = reinterpret_cast<const C*>(b.lpm) + ((size_t)slot_freq(g, vs) * (g.p - 1) + i) * (size_t)Lx * Lx;
  // eight entries of the column in flight per thread before any is used: M is
  // read from HBM on every application (long lines keep 2 MB per line), so the
  // product is bound by how many loads each thread keeps outstanding
  constexpr int U = 8;
  for (int a = threadIdx.x; a < Lx; a += (int)blockDim.x) {
    C acc[4] = {};
    const C* col = M + a;
    int c = 0;
    for (; c + U <= Lx; c += U) {
      C mv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) mv[u] = col[(size_t)(c + u) * Lx];
#pragma unroll
      for (int u = 0; u < U; ++u) acc[u & 3] = cfma(mv[u], rsh[c + u], acc[u & 3]);
    }
    for (; c < Lx; ++c) acc[0] = cfma(col[(size_t)c * Lx], rsh[c], acc[0]);
    z[a] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
  }
}

template <typename R>
__device__ __forceinline__ void interface_precond(const Geo& g, const Bufs& b, int vs, int i, const cx<R>* r,
                                                  cx<R>* z) {
  if (g.lpre) lpre_apply<R>(g, b, vs, i, r, z);
  else precond_apply<R>(g, b, vs, i, r, z);
}

// Right-hand side in IF_B, solution in IF_X.  Returns the iteration count;
// *conv is set to 0 if the cap was hit.
template <typename R, int WF>
__device__ int schur_cocg(cg::cluster_group& cl, RedSmem& rs, int& phase, const Geo& g,
                          const Bufs& b, int vs, int i, double tol, cx<R>* sm, Pipe& pp,
                          int* conv) {
  using C = cx<R>;
  const int p = g.p, A = g.A;
  const bool has = i < p - 1;
  C* X = ifv_ptr<R>(g, b, vs, IF_X);
  C* Rv = ifv_ptr<R>(g, b, vs, IF_R);
  C* Z = ifv_ptr<R>(g, b, vs, IF_Z);
  C* P = ifv_ptr<R>(g, b, vs, IF_P);
  C* SP = ifv_ptr<R>(g, b, vs, IF_SP);
  const C* Bv = ifv_ptr<R>(g, b, vs, IF_B);
  const C* dC = ifv_ptr<R>(g, b, vs, IF_D) + (size_t)i * A;
  const size_t o = (size_t)i * A;
  const C* bl_i = bnd_ptr<R>(g, b, vs, i, 1);
  const C* bl_n = has ? bnd_ptr<R>(g, b, vs, i + 1, 0) : nullptr;
  const R tr = (R)g.t;

  if (has) {
    for (int a = threadIdx.x; a < A; a += (int)blockDim.x) {
      X[o + a] = C{0, 0};
      Rv[o + a] = Bv[o + a];
    }
  }
  __syncthreads();
  if (has) interface_precond<R>(g, b, vs, i, Rv + o, Z + o);
  __syncthreads();
  C v2[2] = {{0, 0}, {0, 0}};
  if (has) {
    for (int a = threadIdx.x; a < A; a += (int)blockDim.x) {
      C zz = Z[o + a], r = Rv[o + a];
      P[o + a] = zz;
      v2[0] = cfma(r, zz, v2[0]);
      v2[1].x += cabs2(r);
    }
  }
  cluster_sum_r<R, 2>(cl, rs, phase, p, v2);
  C rho = v2[0];
  const R bn = v2[1].x;
  *conv = 1;
  if (bn == (R)0) return 0;
  SweepArgs<R> sa = sweep_base<R>(g, b, vs, i);
  sa.lay_lo = (i > 0) ? P + (size_t)(i - 1) * A : nullptr;
  sa.lay_hi = has ? P + o : nullptr;
  sa.bnd_lo = bnd_ptr<R>(g, b, vs, i, 0);
  sa.bnd_hi = bnd_ptr<R>(g, b, vs, i, 1);
  const R tol2 = (R)(tol * tol);
  int it = 0;
  for (;;) {
    if (it >= g.krylov_maxit) {
      *conv = 0;
      break;
    }
    ++it;
    cl.sync();                                  // P of both neighbour layers is final
    sweep<R, WF>(g, i, sa, sm, pp, sweep_cnt(g, b, vs, i));   // B^-1 E p on this subdomain
    cl.sync();                                  // boundary values of every subdomain written
    C v1[1] = {{0, 0}};
    if (has) {
      for (int a = threadIdx.x; a < A; a += (int)blockDim.x) {
        C sp = layer_C_apply<R>(g, dC, P + o, a) - tr * (bl_i[a] + bl_n[a]);
        SP[o + a] = sp;
        v1[0] = cfma(P[o + a], sp, v1[0]);
      }
    }
    cluster_sum_r<R, 1>(cl, rs, phase, p, v1);
    const C alpha = cdiv(rho, v1[0]);
    if (has) {
      for (int a = threadIdx.x; a < A; a += (int)blockDim.x) {
        X[o + a] = X[o + a] + alpha * P[o + a];
        Rv[o + a] = Rv[o + a] - alpha * SP[o + a];
      }
    }
    __syncthreads();
    if (has) interface_precond<R>(g, b, vs, i, Rv + o, Z + o);
    __syncthreads();
    v2[0] = v2[1] = C{0, 0};
    if (has) {
      for (int a = threadIdx.x; a < A; a += (int)blockDim.x) {
        C zz = Z[o + a], r = Rv[o + a];
        v2[0] = cfma(r, zz, v2[0]);
        v2[1].x += cabs2(r);
      }
    }
    cluster_sum_r<R, 2>(cl, rs, phase, p, v2);
    if (v2[1].x <= tol2 * bn) break;
    const C beta = cdiv(v2[0], rho);
    rho = v2[0];
    if (has) {
      for (int a = threadIdx.x; a < A; a += (int)blockDim.x) P[o + a] = Z[o + a] + beta * P[o + a];
    }
  }
  return it;
}

// Layer diagonal d_C = i w + mu - V - Sigma on this CTA's interface layer, in
// precision R, computed once per launch for the interface products.
template <typename R>
__device__ void layer_diag(const Geo& g, const Bufs& b, int vs, int i) {
  if (i >= g.p - 1) return;
  cx<R>* dC = ifv_ptr<R>(g, b, vs, IF_D) + (size_t)i * g.A;
  const int f = slot_freq(g, vs);
  const cxd* hd = b.hdiag ? b.hdiag + (size_t)f * g.Ndd + g.ifc_off + (size_t)i * g.A : nullptr;
  for (int a = threadIdx.x; a < g.A; a += (int)blockDim.x)
    dC[a] = cconv<R>(hd ? hd[a] : dyson_diag(g, b, f, a + g.A * g.ylayer[i]));
}

// res = rhs - H x (mode 0: full H; mode 1: B only, no interface coupling),
// FP64, on this CTA's entries.  Returns partials (||res||^2, ||rhs||^2).
// H_ii comes from the per-solve DD-layout copy (coalesced); each thread takes
// RU sites per pass and issues all their loads before any store, so the loads
// of a pass are in flight together; every term enters by one fused
// multiply-add (the FP64 pipe is what bounds this pass when all frequencies
// run it together).
__device__ __noinline__ void residual_H(const Geo& g, const Bufs& b, int vs, int i, const cxd* rhs,
                                        const cxd* x, cxd* res, int mode, double* rn, double* qn) {
  constexpr int RU = 4;
  const int W = g.W, Lx = g.Lx, T = g.T, h = g.h[i], w = T * h, A = g.A;
  const int nsub = Lx * W, nt = (int)blockDim.x;
  const cxd* xs = x + (size_t)i * nsub;
  const cxd* rs_ = rhs + (size_t)i * nsub;
  cxd* ro = res + (size_t)i * nsub;
  const double t = g.t;
  const int f = slot_freq(g, vs);
  const cxd* hd = b.hdiag + (size_t)f * g.Ndd;
  const cxd* hs = hd + (size_t)i * nsub;
  const cxd* xlo = (mode == 0 && i > 0) ? x + g.ifc_off + (size_t)(i - 1) * A : nullptr;
  const cxd* xhi = (mode == 0 && i < g.p - 1) ? x + g.ifc_off + (size_t)i * A : nullptr;
  double sr = 0, sq = 0;
  const double mt = -t;
  for (int e0 = threadIdx.x; e0 < nsub; e0 += RU * nt) {
    cxd q[RU], rr[RU];
    bool on[RU];
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      const int e = e0 + u * nt;
      const int s = e / W, j = e - s * W;
      on[u] = e < nsub && j < w;
      q[u] = rr[u] = cxd{0, 0};
      if (on[u]) {
        const int tr = j % T, sl = j / T;
        const cxd dv = hs[e], xc = xs[e];
        cxd r = rs_[e];
        q[u] = r;
        // r = q - t (sum of neighbours) - H_ii x, one fused multiply-add per term
        auto sub = [&](cxd v) {
          r.x = fma(mt, v.x, r.x);
          r.y = fma(mt, v.y, r.y);
        };
        if (s > 0) sub(xs[e - W]);
        if (s < Lx - 1) sub(xs[e + W]);
        if (tr > 0) sub(xs[e - 1]);
        if (tr < T - 1) sub(xs[e + 1]);
        if (sl > 0) sub(xs[e - T]);
        if (sl < h - 1) sub(xs[e + T]);
        if (sl == 0 && xlo) sub(xlo[s + Lx * tr]);
        if (sl == h - 1 && xhi) sub(xhi[s + Lx * tr]);
        r.x = fma(-dv.x, xc.x, fma(dv.y, xc.y, r.x));
        r.y = fma(-dv.x, xc.y, fma(-dv.y, xc.x, r.y));
        rr[u] = r;
      }
    }
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      if (!on[u]) continue;
      ro[e0 + u * nt] = rr[u];
      sr += cabs2(rr[u]);
      sq += cabs2(q[u]);
    }
  }
  if (mode == 0 && i < g.p - 1) {
    const size_t o = g.ifc_off + (size_t)i * A;
    const cxd* xl = x + o;
    const cxd* xb = x + (size_t)i * nsub;         // subdomain i: its top row touches layer i
    const cxd* xa = x + (size_t)(i + 1) * nsub;   // subdomain i+1: its bottom row touches layer i
    const int hi = T * (g.h[i] - 1);
    for (int a = threadIdx.x; a < A; a += nt) {
      const int xx = a % Lx, tr = a / Lx;
      cxd nb = {0, 0};
      if (xx > 0) nb = nb + xl[a - 1];
      if (xx < Lx - 1) nb = nb + xl[a + 1];
      if (tr > 0) nb = nb + xl[a - Lx];
      if (tr < T - 1) nb = nb + xl[a + Lx];
      cxd hv = hd[o + a] * xl[a] + t * nb;
      hv = hv + t * (xb[(size_t)xx * W + hi + tr] + xa[(size_t)xx * W + tr]);
      cxd q = rhs[o + a];
      cxd rr = q - hv;
      res[o + a] = rr;
      sr += cabs2(rr);
      sq += cabs2(q);
    }
  }
  *rn = sr;
  *qn = sq;
}

// x = H^-1 rhs by elimination of the subdomain unknowns, sweeps and the
// interface solve in precision R:
//   z = B^-1 rhs_B;  y = S^-1 (rhs_C - E^T z);  x_B = z - B^-1 E y;  x_C = y.
// zero_B: rhs_B = 0 is known, so z = 0 and its sweep is skipped.
// sc: the solve runs on rhs / sc and its result is scaled back by sc, so the
// R-precision recurrences work on O(1) numbers (the squared norms of the
// shrinking refinement residuals would leave float range otherwise).
template <typename R, int WF>
__device__ int solve_H(cg::cluster_group& cl, RedSmem& rs, int& phase, const Geo& g,
                       const Bufs& b, int vs, int i, const cxd* rhs, cxd* xout, bool zero_B,
                       double sc, double tol, cx<R>* sm, Pipe& pp, int* conv) {
  const int A = g.A;
  const bool has = i < g.p - 1;
  const size_t nsub = (size_t)g.Lx * g.W;
  cx<R>* Bv = ifv_ptr<R>(g, b, vs, IF_B);
  const cxd* rc = rhs + g.ifc_off + (size_t)i * A;
  const R tr = (R)g.t;
  const double isc = 1.0 / sc;
  if (!zero_B) {
    SweepArgs<R> sa = sweep_base<R>(g, b, vs, i);
    sa.src = rhs + i * nsub;
    sa.in_scale = isc;
    sa.dst = xout + i * nsub;
    sa.out_scale = sc;
    sa.dst_op = 0;
    sa.bnd_lo = bnd_ptr<R>(g, b, vs, i, 0);
    sa.bnd_hi = bnd_ptr<R>(g, b, vs, i, 1);
    sweep<R, WF>(g, i, sa, sm, pp, sweep_cnt(g, b, vs, i));
    cl.sync();
    if (has) {
      const cx<R>* bl_i = bnd_ptr<R>(g, b, vs, i, 1);
      const cx<R>* bl_n = bnd_ptr<R>(g, b, vs, i + 1, 0);
      for (int a = threadIdx.x; a < A; a += (int)blockDim.x)
        Bv[(size_t)i * A + a] = cconv<R>(isc * rc[a]) - tr * (bl_i[a] + bl_n[a]);
    }
  } else if (has) {
    for (int a = threadIdx.x; a < A; a += (int)blockDim.x) Bv[(size_t)i * A + a] = cconv<R>(isc * rc[a]);
  }
  __syncthreads();
  int it = schur_cocg<R, WF>(cl, rs, phase, g, b, vs, i, tol, sm, pp, conv);
  cl.sync();
  const cx<R>* X = ifv_ptr<R>(g, b, vs, IF_X);
  SweepArgs<R> sb = sweep_base<R>(g, b, vs, i);
  sb.lay_lo = (i > 0) ? X + (size_t)(i - 1) * A : nullptr;
  sb.lay_hi = has ? X + (size_t)i * A : nullptr;
  sb.dst = xout + i * nsub;
  sb.out_scale = sc;
  sb.dst_op = zero_B ? 3 : 2;
  sweep<R, WF>(g, i, sb, sm, pp, sweep_cnt(g, b, vs, i));
  if (has) {
    cxd* xc = xout + g.ifc_off + (size_t)i * A;
    for (int a = threadIdx.x; a < A; a += (int)blockDim.x) xc[a] = sc * cconv<double>(X[(size_t)i * A + a]);
  }
  return it;
}

constexpr size_t YBUF_MAX = 64 * 1024;   // forward intermediates kept on chip up to this size

// Shared-memory plan of a sweep: ring of S slots of CR x W entries (CR = W when
// a whole slice block fits a slot, the W <= 64 strips; row chunks otherwise),
// zw entries of z vectors (2 W; 6 W for the two-chain complex64 form, whose
// ring is split evenly between its chains), and the on-chip row buffer when
// it fits.  per_sm is the number of CTAs per SM the budget is shared by: 2
// (256 threads, ~100 KB each) or, for the complex64 two-chain form, 4 (128
// threads, ~52 KB each, the row buffer on chip only up to 16 KB).
struct RingPlan {
  int CR, S, zw;
  size_t ybuf, smem;
};
constexpr size_t CTA4_BUDGET = 52 * 1024;   // dynamic shared memory per CTA at four CTAs per SM
constexpr size_t CTA4_YBUF_MAX = 16 * 1024;
template <typename R>
__host__ __device__ inline RingPlan ring_plan(int W, int Lx, int per_sm = 2) {
  RingPlan rp;
  const size_t cs = sizeof(cx<R>);
  const size_t yb = (size_t)Lx * W * cs;
  if (W <= DY_MAXW_SMEM) {
    const bool pair = sizeof(R) == 4;
    const bool four = pair && per_sm == 4;
    rp.zw = pair ? 6 * W : 2 * W;
    rp.ybuf = yb <= (four ? CTA4_YBUF_MAX : YBUF_MAX) ? yb : 0;
    rp.CR = W;
    const long budget = four ? (long)CTA4_BUDGET : (long)100 * 1024;
    long S = (budget - (long)rp.ybuf - (long)(rp.zw * cs)) / (long)(W * W * cs);
    if (S > MAX_STAGES) S = MAX_STAGES;
    if (S < 2) S = 2;
    if (pair) S &= ~1L;
    rp.S = (int)S;
  } else {
    rp.zw = 2 * W;
    rp.ybuf = yb;                                                       // one CTA per SM
    const long budget = (long)200 * 1024 - (long)yb - (long)(2 * W * cs);
    // largest divisor of W whose chunks leave >= 4 ring slots (>= 2 as a last
    // resort); a chunk row is W entries, a multiple of 32 bytes, so any row count
    // keeps the bulk copies 16-byte aligned
    rp.CR = 0;
    rp.S = 0;
    for (int want = 4; want >= 2 && !rp.CR; want -= 2)
      for (int cr = W; cr >= 1; --cr) {
        if (W % cr) continue;
        const long S = budget / (long)((size_t)cr * W * cs);
        if (S >= want) {
          rp.CR = cr;
          rp.S = (int)(S > MAX_STAGES ? MAX_STAGES : S);
          break;
        }
      }
  }
  rp.smem = rp.CR ? (size_t)rp.S * rp.CR * W * cs + (size_t)rp.zw * cs + rp.ybuf : 0;
  return rp;
}
// threads per CTA of the X-matvec of a geometry in precision R: 128 (four CTAs
// per SM) for the complex64 two-chain form when the plan chose it, else 256
template <typename R>
__host__ __device__ inline int xm_threads(const Geo& g) {
  return (sizeof(R) == 4 && g.W <= DY_MAXW_SMEM && g.xm_nt == 128) ? 128 : 256;
}
// The plan of a geometry: the heuristic above, or the autotuner's choice of
// slots (and chunk rows for W > 64) with the same row buffer and z area.
constexpr size_t SMEM_LIMIT = 225 * 1024;   // dynamic shared memory per CTA, below the 227 KB cap
template <typename R>
__host__ __device__ inline RingPlan ring_plan(const Geo& g) {
  RingPlan rp = ring_plan<R>(g.W, g.Lx, xm_threads<R>(g) == 128 ? 4 : 2);
  if (g.ring_S > 0 && rp.CR > 0) {
    rp.S = g.ring_S;
    if (g.W > DY_MAXW_SMEM && g.ring_CR > 0) rp.CR = g.ring_CR;
    rp.smem = (size_t)rp.S * rp.CR * g.W * sizeof(cx<R>) + (size_t)rp.zw * sizeof(cx<R>) + rp.ybuf;
  }
  return rp;
}
// Configurations the autotuner times: the heuristic's first, then every slot
// count 2..MAX_STAGES (even in the two-chain complex64 form) that fits, and
// for W > 64 the chunk heights (divisors of W) with the most slots that fit;
// the complex64 two-chain form adds the same slot counts at 128 threads per
// CTA (four CTAs per SM).  NT[] receives each configuration's threads per CTA.
template <typename R>
inline int ring_candidates(const Geo& g, int* S, int* CR, int* NT, int max) {
  const int nt0 = xm_threads<R>(g);
  const RingPlan h = ring_plan<R>(g.W, g.Lx, nt0 == 128 ? 4 : 2);
  if (h.CR == 0 || max < 1) return 0;
  int n = 0;
  S[n] = h.S;
  CR[n] = h.CR;
  NT[n] = nt0;
  ++n;
  const size_t cs = sizeof(cx<R>);
  auto fits = [&](int s, int cr, int nt) {
    const RingPlan b = ring_plan<R>(g.W, g.Lx, nt == 128 ? 4 : 2);
    const size_t fixed = (size_t)b.zw * cs + b.ybuf;
    return (size_t)s * cr * g.W * cs + fixed <= (nt == 128 ? CTA4_BUDGET : SMEM_LIMIT);
  };
  auto add = [&](int s, int cr, int nt) {
    for (int k = 0; k < n; ++k)
      if (S[k] == s && CR[k] == cr && NT[k] == nt) return;
    if (n < max && fits(s, cr, nt)) {
      S[n] = s;
      CR[n] = cr;
      NT[n] = nt;
      ++n;
    }
  };
  if (g.W <= DY_MAXW_SMEM) {
    const int step = sizeof(R) == 4 ? 2 : 1;        // two chains split the ring evenly
    for (int s = 2; s <= MAX_STAGES; s += step) add(s, g.W, 256);
    if (sizeof(R) == 4)
      for (int s = 2; s <= MAX_STAGES; s += step) add(s, g.W, 128);
  } else {
    for (int cr = g.W; cr >= 1; --cr) {
      if (g.W % cr) continue;
      int best = 0;
      for (int s = MAX_STAGES; s >= 2; --s)
        if (fits(s, cr, 256)) {
          best = s;
          break;
        }
      if (best >= 3) add(best, cr, 256);
      if (n >= max) break;
    }
  }
  return n;
}

// ---------------------------------------------------------------- kernels
// u = X q_j  (Sec. 2.3 Eqs. 6-8), with u = v - w computed as the solution of
// H u = q - H w = [0; q_C - E^T w_B]  (w = blkdiag(B^-1, 0) q, so B w_B = q_B),
// i.e. y = S^-1 (E^T w_B - q_C), u_B = B^-1 E y, u_C = -y: no cancellation.
//   mixed = 0: every sweep in R (= double), the interface solve to krylov_tol.
//   mixed = 1: sweeps in complex64 (R = float).  w_B is refined against FP64
//              residuals of B, u against FP64 residuals of H, each until the
//              relative residual is below refine_tol.
template <typename R, int WF, int NT>
__global__ void __launch_bounds__(NT, NT == 128 ? 4 : 2) k_xmatvec(Geo g, Bufs b, int j, int mixed, int ncols) {
  cg::cluster_group cl = cg::this_cluster();
  __shared__ RedSmem rs;
  __shared__ __align__(8) uint64_t bars[MAX_STAGES];
  __shared__ int err;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // one cluster per (frequency, block column): slot vs = f * nb + c
  const int i = blockIdx.x, vs = blockIdx.y, p = g.p, A = g.A;
  const int f = slot_freq(g, vs), c = vs - f * g.nb;
  if (c >= ncols) return;                  // same values in every CTA of the cluster
  int* st = b.st + (size_t)f * ST_N;
  if (st[ST_DONE]) return;
  Pipe pp;
  pp.bar = bars;
  const RingPlan rp = ring_plan<R>(g);
  pp.S = rp.S;
  pp.CR = rp.CR;
  pp.ring = smem_raw;
  pp.seq = 0;
  pp.seq2 = 0;
  pp.err = &err;
  pipe_init(pp);
  cx<R>* sm = reinterpret_cast<cx<R>*>(smem_raw + (size_t)rp.S * rp.CR * g.W * sizeof(cx<R>));
  pp.ybuf = rp.ybuf ? (void*)(sm + rp.zw) : nullptr;
  layer_diag<R>(g, b, vs, i);
  int phase = 0;
  const bool has = i < p - 1;
  const size_t Ndd = g.Ndd, nsub = (size_t)g.Lx * g.W;
  const cxd* q = b.Q + ((size_t)f * (g.k_max + g.nb) + (size_t)j * g.nb + c) * Ndd;
  cxd* u = b.u + (size_t)vs * Ndd;
  if (g.qsplit) {
    // the basis is stored as double-floats: widen this CTA's entries of q_j into u,
    // which is free until the first H solve writes it, and read q_j from there
    const cdfl* qs = reinterpret_cast<const cdfl*>(q);
    const int n = own_count(g, i);
    for (int e = threadIdx.x; e < n; e += (int)blockDim.x) {
      const size_t k = own_idx(g, i, e, (int)nsub);
      u[k] = cwiden(qs[k]);
    }
    __syncthreads();
    q = u;
  }
  int iters = 0, solves = 0, refines = 0, conv_all = 1, conv = 1;

  if (!mixed) {
    // w = B^-1 q_B, only its boundary rows are needed: E^T w
    SweepArgs<R> sa = sweep_base<R>(g, b, vs, i);
    sa.src = q + i * nsub;
    sa.bnd_lo = bnd_ptr<R>(g, b, vs, i, 0);
    sa.bnd_hi = bnd_ptr<R>(g, b, vs, i, 1);
    sweep<R, WF>(g, i, sa, sm, pp, sweep_cnt(g, b, vs, i));
    cl.sync();
    cx<R>* Bv = ifv_ptr<R>(g, b, vs, IF_B);
    if (has) {
      const cx<R>* bl_i = bnd_ptr<R>(g, b, vs, i, 1);
      const cx<R>* bl_n = bnd_ptr<R>(g, b, vs, i + 1, 0);
      const cxd* qc = q + g.ifc_off + (size_t)i * A;
      for (int a = threadIdx.x; a < A; a += (int)blockDim.x)
        Bv[(size_t)i * A + a] = (R)g.t * (bl_i[a] + bl_n[a]) - cconv<R>(qc[a]);
    }
    __syncthreads();
    iters += schur_cocg<R, WF>(cl, rs, phase, g, b, vs, i, g.krylov_tol, sm, pp, &conv);
    conv_all &= conv;
    solves = 1;
    cl.sync();
    const cx<R>* X = ifv_ptr<R>(g, b, vs, IF_X);
    SweepArgs<R> sb = sweep_base<R>(g, b, vs, i);
    sb.lay_lo = (i > 0) ? X + (size_t)(i - 1) * A : nullptr;
    sb.lay_hi = has ? X + (size_t)i * A : nullptr;
    sb.dst = u + i * nsub;
    sb.dst_op = 0;
    sweep<R, WF>(g, i, sb, sm, pp, sweep_cnt(g, b, vs, i));
    if (has) {
      cxd* uc = u + g.ifc_off + (size_t)i * A;
      for (int a = threadIdx.x; a < A; a += (int)blockDim.x) uc[a] = -cconv<double>(X[(size_t)i * A + a]);
    }
  } else {
    cxd* wv = b.v1 + (size_t)vs * Ndd;   // w_B, later the refinement corrections
    cxd* rv = b.v2 + (size_t)vs * Ndd;   // FP64 residuals
    cxd* hr = b.v3 + (size_t)vs * Ndd;   // right-hand side [0; q_C - E^T w_B]
    // ---- w_B = B^-1 q_B, refined against FP64 residuals of B (subdomain-local)
    {
      SweepArgs<R> sa = sweep_base<R>(g, b, vs, i);
      sa.src = q + i * nsub;
      sa.dst = wv + i * nsub;
      sa.dst_op = 0;
      sweep<R, WF>(g, i, sa, sm, pp, sweep_cnt(g, b, vs, i));
      double prev = INFINITY;
      for (int r = 0; r < g.refine_max; ++r) {
        __syncthreads();
        double rn, qn;
        residual_H(g, b, vs, i, q, wv, rv, 1, &rn, &qn);
        cxd v2[2] = {{rn, 0}, {qn, 0}};
        block_sum<2>(rs, v2);
        if (v2[0].x <= g.refine_tol * g.refine_tol * v2[1].x) break;
        if (v2[0].x > REFINE_STALL * prev) break;        // at the FP64 rounding floor
        prev = v2[0].x;
        SweepArgs<R> sc = sweep_base<R>(g, b, vs, i);
        sc.src = rv + i * nsub;
        sc.dst = wv + i * nsub;
        sc.dst_op = 1;
        sweep<R, WF>(g, i, sc, sm, pp, sweep_cnt(g, b, vs, i));
      }
    }
    cl.sync();                             // w_B of the neighbour subdomains is final
    {
      const int n = own_count(g, i);
      const int hi = g.T * (g.h[i] - 1);
      for (int e = threadIdx.x; e < n; e += (int)blockDim.x) {
        size_t k = own_idx(g, i, e, (int)nsub);
        cxd v = {0, 0};
        if (e >= (int)nsub) {
          const int a = e - (int)nsub, xx = a % g.Lx, tr = a / g.Lx;
          const cxd ew = wv[i * nsub + (size_t)xx * g.W + hi + tr] +
                         wv[(i + 1) * nsub + (size_t)xx * g.W + tr];
          v = q[k] - g.t * ew;
        }
        hr[k] = v;
      }
    }
    __syncthreads();                       // interface entries of hr are written by other threads
    double hn;
    {
      cxd v1[1] = {{0, 0}};
      if (has)
        for (int a = threadIdx.x; a < A; a += (int)blockDim.x)
          v1[0].x += cabs2(hr[g.ifc_off + (size_t)i * A + a]);
      cluster_sum<1>(cl, rs, phase, p, v1);   // also: every CTA has read w_B before it is reused
      hn = sqrt(v1[0].x);
    }
    if (hn > 0.0) {
      iters += solve_H<R, WF>(cl, rs, phase, g, b, vs, i, hr, u, true, hn, g.krylov_tol, sm, pp, &conv);
      conv_all &= conv;
      ++solves;
    } else {
      const int n = own_count(g, i);
      for (int e = threadIdx.x; e < n; e += (int)blockDim.x) u[own_idx(g, i, e, (int)nsub)] = cxd{0, 0};
    }
    double prev = INFINITY;
    for (int r = 0; r < g.refine_max && hn > 0.0; ++r) {
      cl.sync();
      double rn, qn;
      residual_H(g, b, vs, i, hr, u, rv, 0, &rn, &qn);
      cxd v2[2] = {{rn, 0}, {qn, 0}};
      cluster_sum<2>(cl, rs, phase, p, v2);
      if (v2[0].x <= g.refine_tol * g.refine_tol * v2[1].x) break;
      if (v2[0].x > REFINE_STALL * prev) break;          // at the FP64 rounding floor
      prev = v2[0].x;
      ++refines;
      iters += solve_H<R, WF>(cl, rs, phase, g, b, vs, i, rv, wv, false, sqrt(v2[0].x), g.krylov_tol, sm,
                          pp, &conv);
      conv_all &= conv;
      ++solves;
      __syncthreads();
      const int n = own_count(g, i), nt = (int)blockDim.x;
      for (int e0 = threadIdx.x; e0 < n; e0 += 4 * nt) {   // four entries' loads in flight
        cxd a4[4], b4[4];
        size_t k4[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int e = e0 + m * nt;
          k4[m] = e < n ? own_idx(g, i, e, (int)nsub) : 0;
          a4[m] = e < n ? u[k4[m]] : cxd{0, 0};
          b4[m] = e < n ? wv[k4[m]] : cxd{0, 0};
        }
#pragma unroll
        for (int m = 0; m < 4; ++m)
          if (e0 + m * nt < n) u[k4[m]] = a4[m] + b4[m];
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && err) atomicOr(st + ST_STATUS, ST_WAIT_TIMEOUT);
  if (i == 0 && threadIdx.x == 0) {       // the nb clusters of a frequency share its counters
    atomicAdd(st + ST_ITERS, iters);
    atomicAdd(st + ST_SOLVES, solves);
    atomicAdd(st + ST_REFINE, refines);
    if (!conv_all) atomicOr(st + ST_STATUS, 4);
  }
  cl.sync();          // no CTA exits while a peer may still read its shared memory
}

// w = blkdiag(B^-1, 0) q for DD-layout vectors (Eq. 7), one CTA per subdomain.
template <typename R, int WF>
__global__ void __launch_bounds__(DY_THREADS, 2) k_bsolve(Geo g, Bufs b, const cxd* q, cxd* w) {
  __shared__ __align__(8) uint64_t bars[MAX_STAGES];
  __shared__ int err;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int i = blockIdx.x, kf = blockIdx.y, vs = kf * g.nb;   // scratch of the frequency's first slot
  const size_t nsub = (size_t)g.Lx * g.W;
  Pipe pp;
  pp.bar = bars;
  const RingPlan rp = ring_plan<R>(g);
  pp.S = rp.S;
  pp.CR = rp.CR;
  pp.ring = smem_raw;
  pp.seq = 0;
  pp.seq2 = 0;
  pp.err = &err;
  pipe_init(pp);
  cx<R>* sm = reinterpret_cast<cx<R>*>(smem_raw + (size_t)rp.S * rp.CR * g.W * sizeof(cx<R>));
  pp.ybuf = rp.ybuf ? (void*)(sm + rp.zw) : nullptr;
  SweepArgs<R> sa = sweep_base<R>(g, b, vs, i);
  sa.src = q + (size_t)kf * g.Ndd + i * nsub;
  sa.dst = w + (size_t)kf * g.Ndd + i * nsub;
  sa.dst_op = 0;
  sweep<R, WF>(g, i, sa, sm, pp, sweep_cnt(g, b, vs, i));
  if (i < g.p - 1)
    for (int a = threadIdx.x; a < g.A; a += (int)blockDim.x)
      w[(size_t)kf * g.Ndd + g.ifc_off + (size_t)i * g.A + a] = cxd{0, 0};
  __syncthreads();
  if (threadIdx.x == 0 && err) atomicOr(b.st + (size_t)kf * ST_N + ST_STATUS, ST_WAIT_TIMEOUT);
}

template <typename Kern, typename... Args>
cudaError_t launch_cluster_nt(Kern kern, dim3 grid, int cx_, int threads, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaError_t e = raise_smem_limit((const void*)kern, smem);
  if (e != cudaSuccess) return e;
  if (cx_ > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cx_;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <typename Kern, typename... Args>
cudaError_t launch_cluster(Kern kern, dim3 grid, int cx_, size_t smem, cudaStream_t st, Args... args) {
  return launch_cluster_nt(kern, grid, cx_, DY_THREADS, smem, st, args...);
}

template <typename R>
size_t sweep_smem(const Geo& g) { return ring_plan<R>(g).smem; }
// the WF of the kernels for this geometry: every slice wider than 64 takes the
// streamed form (CR may equal W there); the complex64 two-chain form is
// compiled for W <= 16, 32 and 64 (fully unrolled block products); the FP64
// 8-warp form needs no width class
template <typename R>
int sweep_form(const Geo& g) {
  if (g.W > DY_MAXW_SMEM) return 0;
  if (sizeof(R) == 8) return 64;
  return g.W <= 16 ? 16 : (g.W <= 32 ? 32 : 64);
}

}  // namespace

// One X-matvec / subdomain-solve variant (precision R, sweep form WF) per
// entry point; each is defined by DY_SOLVE_VARIANT in the translation unit
// that compiles it, so the variants build in parallel.
template <typename R, int WF>
cudaError_t run_xmatvec(const Geo& g, const Bufs& b, int K, int j, int mixed, int ncols, cudaStream_t st);
template <typename R, int WF>
cudaError_t run_bsolve(const Geo& g, const Bufs& b, int K, const cxd* q_dd, cxd* w_dd, cudaStream_t st);

#define DY_SOLVE_VARIANT(R, WF)                                                                   \
  template <>                                                                                     \
  cudaError_t run_xmatvec<R, WF>(const Geo& g, const Bufs& b, int K, int j, int mixed, int ncols, \
                                 cudaStream_t st) {                                               \
    if (sizeof(R) == 4 && xm_threads<R>(g) == 128)                                                \
      return launch_cluster_nt(k_xmatvec<R, WF, (sizeof(R) == 4 ? 128 : 256)>, dim3(g.p, K * g.nb), \
                               g.p, 128, sweep_smem<R>(g), st, g, b, j, mixed, ncols);           \
    return launch_cluster_nt(k_xmatvec<R, WF, 256>, dim3(g.p, K * g.nb), g.p, 256,                \
                             sweep_smem<R>(g), st, g, b, j, mixed, ncols);                        \
  }                                                                                               \
  template <>                                                                                     \
  cudaError_t run_bsolve<R, WF>(const Geo& g, const Bufs& b, int K, const cxd* q_dd, cxd* w_dd,   \
                                cudaStream_t st) {                                                \
    const size_t smem = sweep_smem<R>(g);                                                         \
    cudaError_t e = raise_smem_limit((const void*)k_bsolve<R, WF>, smem);                         \
    if (e != cudaSuccess) return e;                                                               \
    k_bsolve<R, WF><<<dim3(g.p, K), DY_THREADS, smem, st>>>(g, b, q_dd, w_dd);                    \
    return cudaGetLastError();                                                                    \
  }

// Exact interface-layer preconditioner for 2D strips: M = blkdiag_l(S_ll),
// the diagonal blocks of the Schur complement S = C - E^T B^-1 E (Eq. 4) on
// each interface line, inverted once per solve.  The paper leaves the
// interface solver open and credits ARMS-type approximate Schur complements;
// here S_ll is formed without approximation,
//
//   S_ll = C_ll - t^2 (P_top(l) + P_bot(l+1)),
//
// P_top(i) / P_bot(i) the restriction of B_i^-1 to the top / bottom row of
// strip i, its "surface" Green's function along the row.  Only the coupling
// between different lines (through a whole strip) is left out, which is
// small, so COCG on S needs one or two iterations.  S itself is never formed.
//
// The preconditioner may be inexact, so everything here runs in complex64:
//   k_surface    per (strip, frequency): the left-connected slice recursion
//                along x, g_s = (D_s - t^2 g_{s-1})^-1, then backward
//                G_ss = g_s + t^2 g_s G_{s+1,s+1} g_s and, for every s' > s,
//                G_{s,s'} = -t g_s G_{s+1,s'} applied to the boundary columns
//                of G_{s',s'} (kept in shared memory); P[s][s'] is their
//                boundary entry.
//   k_layer_inv  per (interface line, frequency): S_ll and its inverse by the
//                sweep operator, symmetrised so that COCG sees a complex
//                symmetric M^-1.
// Lines longer than DY_LPRE_MAXLX (160) do not fit shared memory; there
//   k_surface_g  keeps the boundary columns of G_{s,s'} in global memory
//                (one warp per column, the column broadcast through shared
//                memory), and
//   k_layer_inv_g forms S_ll in place of P_top(l) and inverts it there by
//                block Gauss-Jordan on 32 x 32 blocks (pivot block by the sweep
//                operator in shared memory, row panel, rank-32 update of the
//                rest, column panel), then writes the symmetrised inverse.
// 3D slabs (slice width W = T h, T = Ly > 1) have interface layers of
// A = Lx T sites, S_ll is A x A (in-plane hopping along x and y), and
//   k_surface_3d forms P_bot(i), P_top(i) from the factorization's
//                left-connected g_s (read in binary64), by the backward
//                recursion G_ss = g_s + t^2 g_s G_{s+1,s+1} g_s and the chains
//                G_{s,c} = -t g_s G_{s+1,c} carried on the T boundary columns
//                of each slice c, with 32 x 32 tiles through shared memory
//                multiplied on the tensor cores (3xTF32; persistent grid, one
//                (slab, frequency) at a time per CTA);
//   k_layer_inv_g  inverts the A x A blocks as above (A <= 1024).
#include <type_traits>

#include "solve_device.cuh"
#include "tc_tf32.cuh"

namespace {

using cxf_ = cx<float>;

// In-place inverse of an n x n complex64 matrix (row stride n) in shared
// memory by the sweep operator on the full matrix (pivots on the diagonal;
// Im of the Dyson diagonal keeps them away from zero).  Thread t owns column
// t % n and every (256 / n)-th row from t / n.
__device__ __forceinline__ void sweep_invert_f(cxf_* A, int n, cxf_* prow, cxf_* fcol) {
  const int nrp = DY_THREADS / n;
  const int c = threadIdx.x % n, r0 = threadIdx.x / n;
  const bool act = r0 < nrp;
  for (int k = 0; k < n; ++k) {
    __syncthreads();
    for (int e = threadIdx.x; e < n; e += DY_THREADS) {
      const cxf_ piv = cinv(A[k * n + k]);
      prow[e] = A[k * n + e];
      fcol[e] = (e == k) ? cxf_{-piv.x, -piv.y} : A[e * n + k] * piv;
    }
    __syncthreads();
    if (act) {
      const cxf_ pc = prow[c];
      for (int r = r0; r < n; r += nrp) {
        cxf_& a = A[r * n + c];
        if (c == k) a = fcol[r];                                    // a_rk / a_kk; -1 / a_kk at r = k
        else if (r == k) a = pc * cxf_{-fcol[k].x, -fcol[k].y};     // a_kc / a_kk
        else a = cfma(cxf_{-fcol[r].x, -fcol[r].y}, pc, a);         // a_rc - a_rk a_kc / a_kk
      }
    }
  }
  __syncthreads();
  // the sweep ends at -A^-1
  for (int e = threadIdx.x; e < n * n; e += DY_THREADS) A[e] = cxf_{-A[e].x, -A[e].y};
  __syncthreads();
}

// C = alpha X Y + beta D for W x W shared matrices (D may alias nothing, may be null)
__device__ __forceinline__ void small_matmul(cxf_* C, const cxf_* X, const cxf_* Y, int W, float alpha,
                                             const cxf_* D) {
  for (int e = threadIdx.x; e < W * W; e += DY_THREADS) {
    const int r = e / W, c = e - r * W;
    cxf_ acc = {0.f, 0.f};
    for (int k = 0; k < W; ++k) acc = cfma(X[r * W + k], Y[k * W + c], acc);
    acc = cxf_{alpha * acc.x, alpha * acc.y};
    if (D) acc = acc + D[e];
    C[e] = acc;
  }
}

// The same for W = 32 with four rows per thread sharing each load of Y:
// lane = column, warp = first row, rows warp + 8 j.
__device__ __forceinline__ void small_matmul32(cxf_* C, const cxf_* X, const cxf_* Y, float alpha,
                                               const cxf_* D) {
  constexpr int W = 32;
  const int c = threadIdx.x & 31, r0 = threadIdx.x >> 5;
  cxf_ acc[4] = {};
#pragma unroll 8
  for (int k = 0; k < W; ++k) {
    const cxf_ y = Y[k * W + c];
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] = cfma(X[(r0 + 8 * j) * W + k], y, acc[j]);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int e = (r0 + 8 * j) * W + c;
    cxf_ v = cxf_{alpha * acc[j].x, alpha * acc[j].y};
    if (D) v = v + D[e];
    C[e] = v;
  }
}

constexpr int SURF_MAXW = 32;
constexpr int SURF_NG = DY_THREADS / 32;                             // column groups (one per warp)
constexpr int SURF_NCOL = (DY_LPRE_MAXLX + SURF_NG - 1) / SURF_NG;   // columns per thread at most

__host__ __device__ __forceinline__ int surf_ldv(int Lx) { return Lx | 1; }   // odd stride: no bank conflicts

// WT: the slice width at compile time (32, the common 2D strip), or 0 for any
// width up to 32 read from the geometry
template <int WT>
__global__ void __launch_bounds__(DY_THREADS, 2) k_surface(Geo g, Bufs b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int i = blockIdx.x, f = blockIdx.y;
  const int W = WT ? WT : g.W, Lx = g.Lx, w = g.h[i], n = W * W, ldv = surf_ldv(Lx);
  const bool need_top = i < g.p - 1, need_bot = i > 0;
  cxf_* Gs = reinterpret_cast<cxf_*>(smem_raw);   // g_s
  cxf_* Gd = Gs + n;                              // G_ss
  cxf_* Tm = Gd + n;
  cxf_* prow = Tm + n;
  cxf_* fcol = prow + W;
  cxf_* Vt = fcol + W;                            // [W][ldv] boundary columns of G_{s,s'}, top row
  cxf_* Vb = Vt + (size_t)W * ldv;                // same for the bottom row
  cxf_* gsv = b.lpg + ((size_t)f * g.p + i) * (size_t)Lx * n;   // own scratch: runs beside the factorization
  cxf_* Pt = b.lpt + (((size_t)f * g.p + i) * 2 + 0) * (size_t)Lx * Lx;
  cxf_* Pb = b.lpt + (((size_t)f * g.p + i) * 2 + 1) * (size_t)Lx * Lx;
  const float t = d2f_bits(g.t), t2 = t * t;
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;

  // forward: g_s = (D_s - t^2 g_{s-1})^-1, padding rows/columns carry the identity
  for (int s = 0; s < Lx; ++s) {
    for (int e = threadIdx.x; e < n; e += DY_THREADS) {
      const int r = e / W, c = e - r * W;
      cxf_ v = {0.f, 0.f};
      if (r < w && c < w) {
        if (r == c) {
          const cxd d = dyson_diag(g, b, f, sub_nat(g, i, s, r));
          v = cxf_{d2f_bits(d.x), d2f_bits(d.y)};
        } else if (r == c + 1 || c == r + 1) {
          v = cxf_{t, 0.f};
        }
        if (s > 0) v = cfma(cxf_{-t2, 0.f}, Gs[e], v);
      } else if (r == c) {
        v = cxf_{1.f, 0.f};
      }
      Gs[e] = v;
    }
    sweep_invert_f(Gs, W, prow, fcol);
    for (int e = threadIdx.x; e < n; e += DY_THREADS) {
      const int r = e / W, c = e - r * W;
      if (r >= w || c >= w) Gs[e] = cxf_{0.f, 0.f};
      gsv[(size_t)s * n + e] = Gs[e];
    }
    __syncthreads();
  }
  // backward: G_ss, and for every s' > s the boundary columns of
  // G_{s,s'} = -t g_s G_{s+1,s'}; lane = row, warp = column group
  for (int s = Lx - 1; s >= 0; --s) {
    for (int e = threadIdx.x; e < n; e += DY_THREADS) Gs[e] = gsv[(size_t)s * n + e];
    __syncthreads();
    if (s == Lx - 1) {
      for (int e = threadIdx.x; e < n; e += DY_THREADS) Gd[e] = Gs[e];
    } else {
      if constexpr (WT == 32) {
        small_matmul32(Tm, Gs, Gd, 1.f, nullptr);          // g_s G_{s+1,s+1}
        __syncthreads();
        small_matmul32(Gd, Tm, Gs, t2, Gs);                 // g_s + t^2 g_s G g_s
      } else {
        small_matmul(Tm, Gs, Gd, W, 1.f, nullptr);
        __syncthreads();
        small_matmul(Gd, Tm, Gs, W, t2, Gs);
      }
      cxf_ gr[SURF_MAXW];                                  // row `lane` of g_s (symmetric)
#pragma unroll
      for (int k = 0; k < SURF_MAXW; ++k) gr[k] = (lane < W && k < W) ? Gs[k * W + lane] : cxf_{0.f, 0.f};
      for (int side = 0; side < 2; ++side) {
        if (side == 0 ? !need_top : !need_bot) continue;
        cxf_* V = side == 0 ? Vt : Vb;
        cxf_ out[SURF_NCOL];
#pragma unroll
        for (int j = 0; j < SURF_NCOL; ++j) {
          const int c = s + 1 + grp + SURF_NG * j;
          cxf_ acc = {0.f, 0.f};
          if (c < Lx) {
#pragma unroll
            for (int k = 0; k < SURF_MAXW; ++k)
              if (k < W) acc = cfma(gr[k], V[k * ldv + c], acc);
          }
          out[j] = cxf_{-t * acc.x, -t * acc.y};
        }
        __syncthreads();                                   // every column read before any is rewritten
        cxf_* P = side == 0 ? Pt : Pb;
        const int rb = side == 0 ? w - 1 : 0;
#pragma unroll
        for (int j = 0; j < SURF_NCOL; ++j) {
          const int c = s + 1 + grp + SURF_NG * j;
          if (c < Lx && lane < W) {
            V[lane * ldv + c] = out[j];
            if (lane == rb) {
              P[(size_t)s * Lx + c] = out[j];
              P[(size_t)c * Lx + s] = out[j];
            }
          }
        }
      }
    }
    __syncthreads();
    // start the chain of column s' = s: the boundary columns of G_ss
    for (int r = threadIdx.x; r < W; r += DY_THREADS) {
      Vt[r * ldv + s] = Gd[r * W + (w - 1)];
      Vb[r * ldv + s] = Gd[r * W + 0];
    }
    if (threadIdx.x == 0) {
      Pt[(size_t)s * Lx + s] = Gd[(w - 1) * W + (w - 1)];
      Pb[(size_t)s * Lx + s] = Gd[0];
    }
    __syncthreads();
  }
}

// The same surface Green's functions for lines longer than the shared-memory
// form takes (Lx > DY_LPRE_MAXLX, slice width 32): the boundary columns
// V[c][r] of G_{s,c}, c > s, live in global memory (b.lpv), column-major, and
// the update V[:, c] <- -t g_s V[:, c] runs one warp per column: the warp
// reads its column, broadcasts it through shared memory and lane r forms row
// r of the product from its register copy of row r of g_s.  Only that warp
// touches column c within a step, so the in-place update needs no barrier.
__global__ void __launch_bounds__(DY_THREADS) k_surface_g(Geo g, Bufs b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int W = 32, n = W * W;
  const int i = blockIdx.x, f = blockIdx.y;
  const int Lx = g.Lx, w = g.h[i];
  const bool need_top = i < g.p - 1, need_bot = i > 0;
  cxf_* Gs = reinterpret_cast<cxf_*>(smem_raw);   // g_s
  cxf_* Gd = Gs + n;                              // G_ss
  cxf_* Tm = Gd + n;
  cxf_* prow = Tm + n;
  cxf_* fcol = prow + W;
  cxf_* colb = fcol + W;                          // [8 warps][W] column broadcast
  cxf_* gsv = b.lpg + ((size_t)f * g.p + i) * (size_t)Lx * n;
  cxf_* Pt = b.lpt + (((size_t)f * g.p + i) * 2 + 0) * (size_t)Lx * Lx;
  cxf_* Pb = b.lpt + (((size_t)f * g.p + i) * 2 + 1) * (size_t)Lx * Lx;
  cxf_* Vt = b.lpv + (((size_t)f * g.p + i) * 2 + 0) * (size_t)Lx * W;   // [Lx][W]
  cxf_* Vb = b.lpv + (((size_t)f * g.p + i) * 2 + 1) * (size_t)Lx * W;
  const float t = d2f_bits(g.t), t2 = t * t;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;

  // forward: g_s = (D_s - t^2 g_{s-1})^-1, padding rows/columns carry the identity
  for (int s = 0; s < Lx; ++s) {
    for (int e = threadIdx.x; e < n; e += DY_THREADS) {
      const int r = e / W, c = e - r * W;
      cxf_ v = {0.f, 0.f};
      if (r < w && c < w) {
        if (r == c) {
          const cxd d = dyson_diag(g, b, f, sub_nat(g, i, s, r));
          v = cxf_{d2f_bits(d.x), d2f_bits(d.y)};
        } else if (r == c + 1 || c == r + 1) {
          v = cxf_{t, 0.f};
        }
        if (s > 0) v = cfma(cxf_{-t2, 0.f}, Gs[e], v);
      } else if (r == c) {
        v = cxf_{1.f, 0.f};
      }
      Gs[e] = v;
    }
    sweep_invert_f(Gs, W, prow, fcol);
    for (int e = threadIdx.x; e < n; e += DY_THREADS) {
      const int r = e / W, c = e - r * W;
      if (r >= w || c >= w) Gs[e] = cxf_{0.f, 0.f};
      gsv[(size_t)s * n + e] = Gs[e];
    }
    __syncthreads();
  }
  // backward: G_ss, and for every c > s the boundary columns of G_{s,c} = -t g_s G_{s+1,c}
  cxf_* cb = colb + wid * W;
  for (int s = Lx - 1; s >= 0; --s) {
    for (int e = threadIdx.x; e < n; e += DY_THREADS) Gs[e] = gsv[(size_t)s * n + e];
    __syncthreads();
    if (s == Lx - 1) {
      for (int e = threadIdx.x; e < n; e += DY_THREADS) Gd[e] = Gs[e];
    } else {
      small_matmul32(Tm, Gs, Gd, 1.f, nullptr);          // g_s G_{s+1,s+1}
      __syncthreads();
      small_matmul32(Gd, Tm, Gs, t2, Gs);                 // g_s + t^2 g_s G g_s
      cxf_ gr[W];                                         // row `lane` of g_s (symmetric)
#pragma unroll
      for (int k = 0; k < W; ++k) gr[k] = Gs[k * W + lane];
      for (int side = 0; side < 2; ++side) {
        if (side == 0 ? !need_top : !need_bot) continue;
        cxf_* V = side == 0 ? Vt : Vb;
        cxf_* P = side == 0 ? Pt : Pb;
        const int rb = side == 0 ? w - 1 : 0;
        for (int c = s + 1 + wid; c < Lx; c += DY_WARPS) {
          cb[lane] = V[(size_t)c * W + lane];
          __syncwarp();
          cxf_ acc0 = {0.f, 0.f}, acc1 = {0.f, 0.f};
#pragma unroll
          for (int k = 0; k < W; k += 2) {
            acc0 = cfma(gr[k], cb[k], acc0);
            acc1 = cfma(gr[k + 1], cb[k + 1], acc1);
          }
          const cxf_ acc = acc0 + acc1;
          const cxf_ out = {-t * acc.x, -t * acc.y};
          __syncwarp();                                   // the column is read before it is rewritten
          V[(size_t)c * W + lane] = out;
          if (lane == rb) {
            P[(size_t)s * Lx + c] = out;
            P[(size_t)c * Lx + s] = out;
          }
        }
      }
    }
    __syncthreads();
    // start the chain of column c = s: the boundary columns of G_ss
    for (int r = threadIdx.x; r < W; r += DY_THREADS) {
      Vt[(size_t)s * W + r] = Gd[r * W + (w - 1)];
      Vb[(size_t)s * W + r] = Gd[r * W + 0];
    }
    if (threadIdx.x == 0) {
      Pt[(size_t)s * Lx + s] = Gd[(w - 1) * W + (w - 1)];
      Pb[(size_t)s * Lx + s] = Gd[0];
    }
    __syncthreads();
  }
}

// S_ll and its inverse for lines longer than the shared-memory form takes, in
// place of P_top(l) (only line l reads it): A = S_ll, then block Gauss-Jordan
// with NB x NB blocks,
//   P = A_kk^-1;  A_kj <- P A_kj;  A_ij <- A_ij - A_ik A_kj;  A_ik <- -A_ik P;  A_kk <- P
// (i, j != k), which leaves A^-1; pivots come from the sweep operator on the
// diagonal block (Im S_ll > 0 keeps them away from zero).  The symmetrised
// inverse is written in the form's precision.
// C (M x N, row stride ldc) = alpha X Y (+ D), X: M x K, Y: K x N, D: M x N, all in
// global memory in any of binary64 / complex64 (converted to complex64 on load),
// 32 x 32 tiles staged through shared memory and multiplied on the tensor cores
// (3xTF32, binary32 accuracy): warp w forms the 16 x 8 sub-tile at rows 16 (w / 4),
// columns 8 (w % 4) of each output tile.  Callers keep C apart from X, Y.
template <typename TX, typename TY, typename TD>
__device__ void gmm_c64(cxf_* C, int ldc, const TX* X, int ldx, const TY* Y, int ldy, const TD* D, int ldd,
                        int M, int N, int K, float alpha, cxf_ (&tx)[32][32], cxf_ (&ty)[32][32]) {
  auto f32 = [](auto v) -> cxf_ {
    using V = decltype(v);
    if constexpr (std::is_same_v<V, cxd>) return cxf_{d2f_bits(v.x), d2f_bits(v.y)};
    else if constexpr (std::is_same_v<V, cx<dfl>>) return cxf_{v.x.hi + v.x.lo, v.y.hi + v.y.lo};
    else return v;
  };
  static_assert(DY_THREADS == 256, "eight 16 x 8 tensor-core tiles per 32 x 32 output tile");
  const int lr = threadIdx.x >> 5, lc = threadIdx.x & 31;
  const int tm = 16 * (lr >> 2), tn = 8 * (lr & 3);
  for (int r0 = 0; r0 < M; r0 += 32)
    for (int c0 = 0; c0 < N; c0 += 32) {
      tc::CTile acc = {};
      for (int k0 = 0; k0 < K; k0 += 32) {
        __syncthreads();                     // previous tiles fully read
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int r = lr + 8 * m;
          tx[r][lc] = (r0 + r < M && k0 + lc < K) ? f32(X[(size_t)(r0 + r) * ldx + k0 + lc]) : cxf_{0.f, 0.f};
          ty[r][lc] = (k0 + r < K && c0 + lc < N) ? f32(Y[(size_t)(k0 + r) * ldy + c0 + lc]) : cxf_{0.f, 0.f};
        }
        __syncthreads();
        tc::cgemm_tile_3xtf32(acc, &tx[0][0], &ty[0][0], 32, tm, tn);
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        int r, c;
        tc::tile_pos(e, tm, tn, r, c);
        if (r0 + r < M && c0 + c < N) {
          cxf_ v = {alpha * acc.re[e], alpha * acc.im[e]};
          if (D) v = v + f32(D[(size_t)(r0 + r) * ldd + c0 + c]);
          C[(size_t)(r0 + r) * ldc + c0 + c] = v;
        }
      }
    }
  __syncthreads();
}

// Surface Green's functions of 3D slabs (see the top of the file).  Chains are kept
// as one W x NV matrix per CTA, NV = 2 Lx T columns: [side][slice c][boundary column b]
// (side 0 top, 1 bottom), updated by one product per step into the other half of
// the ping-pong pair.  G_{s+1,s+1} and the product g_s G_{s+1,s+1} (complex64) use
// the factor's per-CTA workspace, free once the factorization has run.
template <typename FT>   // the factors' element: binary64 (FP64 form) or double-float (mixed)
__global__ void __launch_bounds__(DY_THREADS) k_surface_3d(Geo g, Bufs b, int K) {
  __shared__ __align__(16) cxf_ tx[32][32];
  __shared__ __align__(16) cxf_ ty[32][32];
  const int W = g.W, Lx = g.Lx, T = g.T, A = g.A;
  const size_t n = (size_t)W * W, NV = (size_t)2 * Lx * T;
  cxf_* Gd = reinterpret_cast<cxf_*>(b.fwork + (size_t)blockIdx.x * 2 * n);   // G_{s+1,s+1}
  cxf_* Tm = Gd + n;
  cxf_* Va = b.lpw + (size_t)blockIdx.x * 2 * W * NV;
  cxf_* Vb = Va + (size_t)W * NV;
  const float t = d2f_bits(g.t), t2 = t * t;
  for (int unit = blockIdx.x; unit < g.p * K; unit += gridDim.x) {
    const int i = unit % g.p, f = unit / g.p, w = T * g.h[i];
    const FT* gs = reinterpret_cast<const FT*>(b.g64 ? (const void*)b.g64 : b.g) + ((size_t)f * g.p + i) * (size_t)Lx * n;
    cxf_* P[2] = {b.lpt + (((size_t)f * g.p + i) * 2 + 0) * (size_t)A * A,
                  b.lpt + (((size_t)f * g.p + i) * 2 + 1) * (size_t)A * A};
    const bool need[2] = {i < g.p - 1, i > 0};
    // boundary row / column j of slice for side sd and in-plane index b: top rows
    // (slow row h-1) and bottom rows (slow row 0); its layer index is x + Lx b
    auto bj = [&](int sd, int bb) { return sd == 0 ? w - T + bb : bb; };
    cxf_* V = Va;
    cxf_* Vn = Vb;
    for (int s = Lx - 1; s >= 0; --s) {
      const FT* g_s = gs + (size_t)s * n;
      if (s < Lx - 1) {
        // G_{s,c}[:, bnd(c)] = -t g_s G_{s+1,c}[:, bnd(c)] for every c > s, both sides
        const int c0 = (s + 1) * T, nc = (Lx - 1 - s) * T;
        for (int sd = 0; sd < 2; ++sd) {
          if (!need[sd]) continue;
          const size_t off = (size_t)sd * Lx * T + c0;
          gmm_c64(Vn + off, (int)NV, g_s, W, V + off, (int)NV, (const cxf_*)nullptr, 0, W, nc, W, -t, tx, ty);
        }
        cxf_* tmp = V;
        V = Vn;
        Vn = tmp;
        // P[s][c] = rows bnd(s) of the chains, and its mirror (G is complex symmetric)
        for (int sd = 0; sd < 2; ++sd) {
          if (!need[sd]) continue;
          for (int e = threadIdx.x; e < T * nc; e += DY_THREADS) {
            const int ra = e / nc, q = e - ra * nc;            // row b_s, chain column (c, b_c)
            const int c = s + 1 + q / T, bc = q % T;
            const cxf_ v = V[(size_t)bj(sd, ra) * NV + (size_t)sd * Lx * T + c0 + q];
            const size_t a = (size_t)s + (size_t)Lx * ra, a2 = (size_t)c + (size_t)Lx * bc;
            P[sd][a * A + a2] = v;
            P[sd][a2 * A + a] = v;
          }
        }
      }
      // G_ss = g_s + t^2 g_s G_{s+1,s+1} g_s  (g_{Lx-1} itself at the end of the slab)
      if (s == Lx - 1) {
        for (size_t e = threadIdx.x; e < n; e += DY_THREADS) {
          if constexpr (std::is_same_v<FT, cxd>) Gd[e] = cxf_{d2f_bits(g_s[e].x), d2f_bits(g_s[e].y)};
          else Gd[e] = cxf_{g_s[e].x.hi + g_s[e].x.lo, g_s[e].y.hi + g_s[e].y.lo};
        }
        __syncthreads();
      } else {
        gmm_c64(Tm, W, g_s, W, Gd, W, (const cxf_*)nullptr, 0, W, W, W, 1.f, tx, ty);
        gmm_c64(Gd, W, Tm, W, g_s, W, g_s, W, W, W, W, t2, tx, ty);
      }
      // start the chains of column c = s, and the diagonal block P[s][s]
      for (int sd = 0; sd < 2; ++sd) {
        if (!need[sd]) continue;
        for (int e = threadIdx.x; e < W * T; e += DY_THREADS) {
          const int r = e / T, bc = e - r * T;
          V[(size_t)r * NV + (size_t)sd * Lx * T + (size_t)s * T + bc] = Gd[(size_t)r * W + bj(sd, bc)];
        }
        for (int e = threadIdx.x; e < T * T; e += DY_THREADS) {
          const int ra = e / T, bc = e - ra * T;
          P[sd][((size_t)s + (size_t)Lx * ra) * A + (size_t)s + (size_t)Lx * bc] = Gd[(size_t)bj(sd, ra) * W + bj(sd, bc)];
        }
      }
      __syncthreads();
    }
  }
}

constexpr int LINV_NB = 32;
template <typename R>
__global__ void __launch_bounds__(DY_THREADS) k_layer_inv_g(Geo g, Bufs b) {
  __shared__ __align__(16) cxf_ Pk[LINV_NB * LINV_NB];
  __shared__ __align__(16) cxf_ X[LINV_NB * LINV_NB];
  __shared__ __align__(16) cxf_ Y[LINV_NB * LINV_NB];
  __shared__ cxf_ prow[LINV_NB], fcol[LINV_NB];
  constexpr int NB = LINV_NB;
  // the layer has A = Lx T sites (T = 1 in 2D), layer index a = x + Lx y; below,
  // "Lx" is the matrix dimension A
  const int l = blockIdx.x, f = blockIdx.y, Lx = g.A, lx = g.Lx;
  const size_t n2 = (size_t)Lx * Lx;
  cxf_* A = b.lpt + (((size_t)f * g.p + l) * 2 + 0) * n2;          // P_top(l), overwritten
  const cxf_* Pb = b.lpt + (((size_t)f * g.p + l + 1) * 2 + 1) * n2;
  const float t = d2f_bits(g.t), t2 = t * t;
  for (size_t e = threadIdx.x; e < n2; e += DY_THREADS) {
    const int r = (int)(e / Lx), c = (int)(e - (size_t)r * Lx);
    cxf_ v = {0.f, 0.f};
    if (r == c) {
      const cxd d = dyson_diag(g, b, f, r + g.A * g.ylayer[l]);
      v = cxf_{d2f_bits(d.x), d2f_bits(d.y)};
    } else if (((r == c + 1 || c == r + 1) && r / lx == c / lx) || r == c + lx || c == r + lx) {
      v = cxf_{t, 0.f};                                             // in-plane neighbours along x and y
    }
    A[e] = cfma(cxf_{-t2, 0.f}, A[e] + Pb[e], v);
  }
  const int nbk = (Lx + NB - 1) / NB;
  // load / store a block (rows r0.., cols c0..), zero-padded past Lx (identity on the diagonal pad)
  auto ld = [&](cxf_* T, int r0, int c0, bool diag) {
    for (int e = threadIdx.x; e < NB * NB; e += DY_THREADS) {
      const int r = e / NB, c = e - r * NB;
      cxf_ v = {0.f, 0.f};
      if (r0 + r < Lx && c0 + c < Lx) v = A[(size_t)(r0 + r) * Lx + c0 + c];
      else if (diag && r == c) v = cxf_{1.f, 0.f};
      T[e] = v;
    }
  };
  auto st = [&](const cxf_* T, int r0, int c0) {
    for (int e = threadIdx.x; e < NB * NB; e += DY_THREADS) {
      const int r = e / NB, c = e - r * NB;
      if (r0 + r < Lx && c0 + c < Lx) A[(size_t)(r0 + r) * Lx + c0 + c] = T[e];
    }
  };
  // C(r0, c0) <- C + alpha * (Xm Ym) or alpha * (Xm Ym) (overwrite), 32 x 32 x 32 on
  // the tensor cores (3xTF32, binary32 accuracy): warp w computes the 16 x 8 tile
  // at rows 16 (w / 4), columns 8 (w % 4)
  auto mm = [&](const cxf_* Xm, const cxf_* Ym, int r0, int c0, float alpha, bool accumulate) {
    const int wq = threadIdx.x >> 5, tm = 16 * (wq >> 2), tn = 8 * (wq & 3);
    tc::CTile acc = {};
    tc::cgemm_tile_3xtf32(acc, Xm, Ym, NB, tm, tn);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int r, c;
      tc::tile_pos(e, tm, tn, r, c);
      if (r0 + r < Lx && c0 + c < Lx) {
        cxf_& o = A[(size_t)(r0 + r) * Lx + c0 + c];
        const cxf_ v = {alpha * acc.re[e], alpha * acc.im[e]};
        o = accumulate ? o + v : v;
      }
    }
  };
  static_assert(LINV_NB == 32 && DY_THREADS == 256, "eight 16 x 8 tensor-core tiles per 32 x 32 block");
  for (int kb = 0; kb < nbk; ++kb) {
    const int k0 = kb * NB;
    __syncthreads();
    ld(Pk, k0, k0, true);
    sweep_invert_f(Pk, NB, prow, fcol);                   // Pk = A_kk^-1
    // row panel A_kj <- Pk A_kj
    for (int jb = 0; jb < nbk; ++jb) {
      if (jb == kb) continue;
      __syncthreads();
      ld(Y, k0, jb * NB, false);
      __syncthreads();
      mm(Pk, Y, k0, jb * NB, 1.f, false);
    }
    // rank-NB update of the rest with the old column panel
    for (int ib = 0; ib < nbk; ++ib) {
      if (ib == kb) continue;
      __syncthreads();
      ld(X, ib * NB, k0, false);
      for (int jb = 0; jb < nbk; ++jb) {
        if (jb == kb) continue;
        __syncthreads();
        ld(Y, k0, jb * NB, false);
        __syncthreads();
        mm(X, Y, ib * NB, jb * NB, -1.f, true);
      }
      // column panel of this block row: A_ik <- -A_ik Pk (X still holds the old A_ik)
      __syncthreads();
      mm(X, Pk, ib * NB, k0, -1.f, false);
    }
    __syncthreads();
    st(Pk, k0, k0);
  }
  __syncthreads();
  cx<R>* M = reinterpret_cast<cx<R>*>(b.lpm) + ((size_t)f * (g.p - 1) + l) * n2;
  for (size_t e = threadIdx.x; e < n2; e += DY_THREADS) {
    const int r = (int)(e / Lx), c = (int)(e - (size_t)r * Lx);
    const cxf_ a = A[e], at = A[(size_t)c * Lx + r];
    M[e] = cx<R>{(R)(0.5f * (a.x + at.x)), (R)(0.5f * (a.y + at.y))};
  }
}

// S_ll = C_ll - t^2 (P_top(l) + P_bot(l+1)) and M_l^-1, symmetrised, in the form's precision.
template <typename R>
__global__ void __launch_bounds__(DY_THREADS) k_layer_inv(Geo g, Bufs b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int l = blockIdx.x, f = blockIdx.y, Lx = g.Lx, n = Lx * Lx;
  cxf_* S = reinterpret_cast<cxf_*>(smem_raw);
  cxf_* prow = S + n;
  cxf_* fcol = prow + Lx;
  const cxf_* Pt = b.lpt + (((size_t)f * g.p + l) * 2 + 0) * (size_t)n;
  const cxf_* Pb = b.lpt + (((size_t)f * g.p + l + 1) * 2 + 1) * (size_t)n;
  const float t = d2f_bits(g.t), t2 = t * t;
  for (int e = threadIdx.x; e < n; e += DY_THREADS) {
    const int r = e / Lx, c = e - r * Lx;
    cxf_ v = {0.f, 0.f};
    if (r == c) {
      const cxd d = dyson_diag(g, b, f, r + g.A * g.ylayer[l]);
      v = cxf_{d2f_bits(d.x), d2f_bits(d.y)};
    } else if (r == c + 1 || c == r + 1) {
      v = cxf_{t, 0.f};
    }
    S[e] = cfma(cxf_{-t2, 0.f}, Pt[e] + Pb[e], v);
  }
  sweep_invert_f(S, Lx, prow, fcol);
  cx<R>* M = reinterpret_cast<cx<R>*>(b.lpm) + ((size_t)f * (g.p - 1) + l) * (size_t)n;
  for (int e = threadIdx.x; e < n; e += DY_THREADS) {
    const int r = e / Lx, c = e - r * Lx;
    const cxf_ a = S[e], at = S[c * Lx + r];
    const cxf_ v = {0.5f * (a.x + at.x), 0.5f * (a.y + at.y)};
    M[e] = cx<R>{(R)v.x, (R)v.y};
  }
}

}  // namespace

size_t dyson_internal_surface_smem(const Geo& g) {
  return (3 * (size_t)g.W * g.W + 2 * (size_t)g.W + 2 * (size_t)g.W * surf_ldv(g.Lx)) * sizeof(cxf_);
}

size_t dyson_internal_layer_inv_smem(const Geo& g) {
  if (g.Lx > DY_LPRE_MAXLX) return 0;                      // global-memory form
  return ((size_t)g.Lx * g.Lx + 2 * (size_t)g.Lx) * sizeof(cxf_);
}

static size_t surface_g_smem() { return (3 * 32 * 32 + 2 * 32 + DY_WARPS * 32) * sizeof(cxf_); }

cudaError_t launch_surface(const Geo& g, const Bufs& b, int K, cudaStream_t st) {
  if (!g.lpre) return cudaSuccess;
  if (g.T > 1) {                           // 3D slabs: persistent grid over (slab, frequency)
    if (!b.lpw || !b.fwork || g.W <= DY_MAXW_SMEM || g.A > DY_LPRE_MAXLX_G) return cudaErrorInvalidValue;
    const int units = g.p * K;
    const int grid = units < DY_FACTOR_CTAS ? units : DY_FACTOR_CTAS;
    if (b.g64) k_surface_3d<cx<dfl>><<<grid, DY_THREADS, 0, st>>>(g, b, K);   // mixed: double-float factors
    else k_surface_3d<cxd><<<grid, DY_THREADS, 0, st>>>(g, b, K);
    return cudaGetLastError();
  }
  if (g.W > SURF_MAXW || g.Lx > DY_LPRE_MAXLX_G) return cudaErrorInvalidValue;
  if (g.Lx > DY_LPRE_MAXLX) {
    if (g.W != 32 || !b.lpv) return cudaErrorInvalidValue;
    k_surface_g<<<dim3(g.p, K), DY_THREADS, surface_g_smem(), st>>>(g, b);
    return cudaGetLastError();
  }
  const size_t smem = dyson_internal_surface_smem(g);
  if (g.W == 32) {
    cudaError_t e = raise_smem_limit((const void*)k_surface<32>, smem);
    if (e != cudaSuccess) return e;
    k_surface<32><<<dim3(g.p, K), DY_THREADS, smem, st>>>(g, b);
  } else {
    cudaError_t e = raise_smem_limit((const void*)k_surface<0>, smem);
    if (e != cudaSuccess) return e;
    k_surface<0><<<dim3(g.p, K), DY_THREADS, smem, st>>>(g, b);
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_layer_inv(const Geo& g, const Bufs& b, int K, cudaStream_t st) {
  if (!g.lpre) return cudaSuccess;
  if (g.T > 1 || g.Lx > DY_LPRE_MAXLX) {
    k_layer_inv_g<R><<<dim3(g.p - 1, K), DY_THREADS, 0, st>>>(g, b);
    return cudaGetLastError();
  }
  const size_t smem = dyson_internal_layer_inv_smem(g);
  cudaError_t e = raise_smem_limit((const void*)k_layer_inv<R>, smem);
  if (e != cudaSuccess) return e;
  k_layer_inv<R><<<dim3(g.p - 1, K), DY_THREADS, smem, st>>>(g, b);
  return cudaGetLastError();
}
template cudaError_t launch_layer_inv<float>(const Geo&, const Bufs&, int, cudaStream_t);
template cudaError_t launch_layer_inv<double>(const Geo&, const Bufs&, int, cudaStream_t);

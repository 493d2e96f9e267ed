// Subdomain factorization: diag(B^-1) and the slice factors used by every
// subdomain solve (Sec. 2.3: "the diagonal of B^-1 ... needs to be
// calculated only once at the very beginning of the Lanczos steps"; Eq. 7).
//
// One CTA per (subdomain, frequency).  B_i is block tridiagonal along x with
// slice blocks D_s (diag(H_jj) + t * in-slice hopping) and couplings t*I:
//   forward   g_s  = (D_s - t^2 g_{s-1})^-1          (left-connected inverse)
//   backward  G_ss = g_s + t^2 g_s G_{s+1,s+1} g_s
// The g_s are stored for the block forward/back substitutions; diag(G_ss) is
// diag(B^-1) on that slice.  Matrices live in shared memory (W <= 64);
// inversion is in-place Gauss-Jordan without pivoting, which is safe here
// because every pivot block has a positive-definite imaginary part
// (Im H_jj >= w_0 > 0 and -t^2 Im g_{s-1} is positive semi-definite), so
// all Schur complements stay non-singular.
#include "dyson_common.cuh"

namespace {

template <typename R>
__device__ __forceinline__ bool slice_adjacent(int r, int c, int T) {
  int tr_r = r % T, sl_r = r / T, tr_c = c % T, sl_c = c / T;
  if (sl_r == sl_c) return abs(tr_r - tr_c) == 1;
  return tr_r == tr_c && abs(sl_r - sl_c) == 1;
}

// In-place inverse of the complex symmetric W x W matrix A (row-major, shared)
// by the symmetric sweep operator (symmetric Gauss-Jordan): sweeping pivot k
// maps a_kk -> -1/a_kk, a_rk, a_kr -> a_rk / a_kk and the rest to
// a_rc - a_rk a_kc / a_kk, which keeps the matrix symmetric, so only the upper
// triangle is updated (W^2/2 complex FMAs per step, half of plain
// Gauss-Jordan); after all W pivots it holds -A^-1.  Step k: W threads cache
// column k unscaled in prow and scaled by the pivot inverse in fcol (with
// -1/a_kk at fcol[k]); every other entry has one owner thread.  Every block
// inverted here is complex symmetric (D_s and the g_s are), without pivoting
// because Im A is positive definite (leading minors never vanish).
template <typename R>
__device__ void gj_invert(cx<R>* A, int W, cx<R>* prow, cx<R>* fcol) {
  const int n = W * W;
  for (int k = 0; k < W; ++k) {
    __syncthreads();                         // step k-1 finished by every thread
    for (int e = threadIdx.x; e < W; e += DY_THREADS) {
      const cx<R> piv = cinv(A[k * W + k]);
      const cx<R> a = (e < k) ? A[e * W + k] : A[k * W + e];   // a_ek from the upper triangle
      prow[e] = a;
      fcol[e] = (e == k) ? -piv : a * piv;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n; e += DY_THREADS) {
      const int r = e / W, c = e - r * W;
      if (c < r) continue;
      if (r == k || c == k) A[e] = fcol[r == k ? c : r];
      else A[e] = cfma(-fcol[r], prow[c], A[e]);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += DY_THREADS) {   // -(-A^-1), upper triangle
    const int r = e / W, c = e - r * W;
    if (c >= r) A[e] = -A[e];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += DY_THREADS) {   // mirror to the lower triangle
    const int r = e / W, c = e - r * W;
    if (c < r) A[e] = A[c * W + r];
  }
  __syncthreads();
}

// C = X * Y for W x W shared matrices
template <typename R>
__device__ __forceinline__ void smem_matmul(cx<R>* C, const cx<R>* X, const cx<R>* Y, int W) {
  const int n = W * W;
  for (int e = threadIdx.x; e < n; e += DY_THREADS) {
    int r = e / W, c = e - r * W;
    cx<R> acc = {0, 0};
    const cx<R>* xr = X + r * W;
    for (int k = 0; k < W; ++k) acc = cfma(xr[k], Y[k * W + c], acc);
    C[e] = acc;
  }
}

// R: arithmetic of the recursion; S: storage of the g_s handed to the sweeps.
//
// FP64 form (S == R): one-sided recursion, g_s left-connected for every s,
// stored row-major for the 8-warp sweeps.
//
// Mixed form (S != R): two-sided recursion, so that the complex64 sweeps can
// run two chains at once (one from each end).  With m = Lx / 2:
//   left   g_s = (D_s - t^2 g_{s-1})^-1            s < m
//   right  g_s = (D_s - t^2 g_{s+1})^-1            s > m
//   middle G_mm = (D_m - t^2 g_{m-1} - t^2 g_{m+1})^-1
//   G_ss = g_s + t^2 g_s G_{s+1,s+1} g_s  (s < m),  g_s + t^2 g_s G_{s-1,s-1} g_s  (s > m)
// Slot s holds g_s, or G_mm for s = m.  The recursion runs in R (FP64) with
// the factors kept in b.g64; the complex64 copy in b.g is written with column
// pairs interleaved: entry (r, c) of a block at ((c / 2) W + r) 2 + c % 2, so
// that the lane owning row r reads columns 2k, 2k+1 as one 16-byte word.
template <typename R, typename S>
__global__ void __launch_bounds__(DY_THREADS) k_factor(Geo g, Bufs b) {
  using C = cx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int i = blockIdx.x, kf = blockIdx.y;
  const int W = g.W, Lx = g.Lx, T = g.T, w = T * g.h[i];
  const int n = W * W;
  C* A = reinterpret_cast<C*>(smem_raw);
  C* Bm = A + n;
  C* Cm = Bm + n;
  C* prow = Cm + n;                          // Gauss-Jordan pivot row / column caches
  C* fcol = prow + W;
  C* Gprev = fcol + W;                       // [2][W] columns of the last off-diagonal block at the boundary rows
  C* Gmid = Gprev + 2 * W;                   // [2][W] rows of G_{m+1,m} at the boundary rows (two-sided)
  constexpr bool two = sizeof(S) != sizeof(R);
  const size_t uoff = ((size_t)kf * g.p + i) * (size_t)Lx * n;
  C* gout = reinterpret_cast<C*>(two ? b.g64 : b.g) + uoff;
  cx<S>* gsw = reinterpret_cast<cx<S>*>(b.g) + uoff;
  cxd* dB = b.diagB + (size_t)kf * g.Ndd + (size_t)i * Lx * W;
  const R t = (R)g.t, t2 = (R)(g.t * g.t);

  // A = D_s - t^2 (pa + pb); pa may be A itself (each entry is read and
  // written by the same thread), either may be null
  auto form = [&](int s, const C* pa, const C* pb) {
    for (int e = threadIdx.x; e < n; e += DY_THREADS) {
      int r = e / W, c = e - r * W;
      C v = {0, 0};
      if (pa) v = v - t2 * pa[e];
      if (pb) v = v - t2 * pb[e];
      if (r < w && c < w) {
        if (r == c) {
          cxd d = dyson_diag(g, b, kf, sub_nat(g, i, s, r));
          v = v + cconv<R>(d);
        } else if (slice_adjacent<R>(r, c, T)) {
          v.x += t;
        }
      } else {
        v = (r == c) ? C{1, 0} : C{0, 0};
      }
      A[e] = v;
    }
  };
  // invert A in place, zero its padding and store it in slot s
  auto invert_store = [&](int s) {
    gj_invert<R>(A, W, prow, fcol);
    for (int e = threadIdx.x; e < n; e += DY_THREADS) {
      int r = e / W, c = e - r * W;
      C v = A[e];
      if (r >= w || c >= w) v = C{0, 0};
      A[e] = v;
      gout[(size_t)s * n + e] = v;
      if (two) gsw[(size_t)s * n + ((size_t)(c >> 1) * W + r) * 2 + (c & 1)] = cconv<S>(v);
    }
    __syncthreads();
  };
  auto diag_out = [&](int s) {
    for (int r = threadIdx.x; r < W; r += DY_THREADS)
      dB[(size_t)s * W + r] = (r < w) ? cconv<double>(A[r * W + r]) : cxd{0, 0};
  };
  cxd* oB = b.offB ? b.offB + ((size_t)kf * g.p + i) * (size_t)Lx * W : nullptr;
  // distance-2 couplings on the two boundary rows (2D strips: row 0 below,
  // row w-1 above): G_{s,s2} = -t g_s G_{sn,s2} with s2 = 2 sn - s, from the
  // columns of the previous step's off-diagonal block G_{sn,s2}
  cxd* o2 = (b.off2 && T == 1) ? b.off2 + ((size_t)kf * g.p + i) * (size_t)Lx * W : nullptr;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // A <- g_s + t^2 g_s A g_s with g_s from slot s (A = G of the neighbour toward
  // the start, slice sn); -t g_s A is the off-diagonal block G_{s,sn}, whose
  // diagonal the interface preconditioner uses (stored at min(s, sn)).
  // prevc: boundary columns of G_{sn,s2} (null if s2 is outside the strip);
  // mid: also keep the boundary rows of G_{s,sn} in Gmid
  auto grow_G = [&](int s, int sn, const C* prevc, bool mid) {
    for (int e = threadIdx.x; e < n; e += DY_THREADS) Bm[e] = gout[(size_t)s * n + e];
    __syncthreads();
    smem_matmul<R>(Cm, Bm, A, W);
    __syncthreads();
    if (oB)
      for (int r = threadIdx.x; r < W; r += DY_THREADS)
        oB[(size_t)(s < sn ? s : sn) * W + r] = (r < w) ? cconv<double>((-t) * Cm[r * W + r]) : cxd{0, 0};
    if (o2) {
      const int s2 = 2 * sn - s;
      if (prevc && wid < 2) {                // warp jj: boundary row jj ? w-1 : 0
        const int j = wid ? w - 1 : 0;
        C acc = {0, 0};
        for (int c = lane; c < W; c += 32) acc = cfma(Bm[j * W + c], prevc[wid * W + c], acc);
        for (int off = 16; off > 0; off >>= 1) {
          acc.x += shfl_xor_any(acc.x, off);
          acc.y += shfl_xor_any(acc.y, off);
        }
        if (lane == 0) o2[(size_t)(s < s2 ? s : s2) * W + j] = cconv<double>((-t) * acc);
      }
      __syncthreads();                       // prevc read before Gprev is rewritten
      for (int e = threadIdx.x; e < 2 * W; e += DY_THREADS) {
        const int jj = e / W, c = e - jj * W, j = jj ? w - 1 : 0;
        Gprev[e] = (-t) * Cm[c * W + j];
        if (mid) Gmid[e] = (-t) * Cm[j * W + c];
      }
    }
    // g_s + t^2 (g_s A) g_s is complex symmetric: the upper triangle, then the mirror
    for (int e = threadIdx.x; e < n; e += DY_THREADS) {
      int r = e / W, c = e - r * W;
      if (c < r) continue;
      C acc = {0, 0};
      const C* xr = Cm + r * W;
      for (int k = 0; k < W; ++k) acc = cfma(xr[k], Bm[k * W + c], acc);
      A[e] = Bm[e] + t2 * acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n; e += DY_THREADS) {
      int r = e / W, c = e - r * W;
      if (c < r) A[e] = A[c * W + r];
    }
    __syncthreads();
    diag_out(s);
  };

  if constexpr (!two) {
    for (int s = 0; s < Lx; ++s) {          // forward: A holds g_{s-1} on entry
      form(s, s > 0 ? A : nullptr, nullptr);
      invert_store(s);
    }
    diag_out(Lx - 1);                        // backward: A holds G_{s+1,s+1}
    for (int s = Lx - 2; s >= 0; --s) grow_G(s, s + 1, s < Lx - 2 ? Gprev : nullptr, false);
  } else {
    const int m = Lx / 2;
    for (int s = 0; s < m; ++s) {           // left chain
      form(s, s > 0 ? A : nullptr, nullptr);
      invert_store(s);
    }
    for (int s = Lx - 1; s > m; --s) {      // right chain
      form(s, s < Lx - 1 ? A : nullptr, nullptr);
      invert_store(s);
    }
    form(m, m > 0 ? gout + (size_t)(m - 1) * n : nullptr,
         m < Lx - 1 ? gout + (size_t)(m + 1) * n : nullptr);
    invert_store(m);                         // G_mm
    diag_out(m);
    // right side first, so that the left side's first step finds G_{m,m+1}
    for (int s = m + 1; s < Lx; ++s) grow_G(s, s - 1, s > m + 1 ? Gprev : nullptr, s == m + 1);
    for (int e = threadIdx.x; e < n; e += DY_THREADS) A[e] = gout[(size_t)m * n + e];
    __syncthreads();
    for (int s = m - 1; s >= 0; --s)
      grow_G(s, s + 1, s < m - 1 ? Gprev : (m + 1 < Lx ? Gmid : nullptr), false);
  }
  // interface part of diag(B^-1) is zero (blkdiag(B^-1, 0), Eq. 9)
  if (i == g.p - 1) {
    cxd* dI = b.diagB + (size_t)kf * g.Ndd + g.ifc_off;
    size_t m = (size_t)(g.p - 1) * g.A;
    for (size_t e = threadIdx.x; e < m; e += DY_THREADS) dI[e] = cxd{0, 0};
  }
}

// ---------------------------------------------------------------- wide slices
// 64 < W <= 256 (3D slabs): a W x W block no longer fits shared memory.  The
// same recursion runs on global memory, which at these sizes stays in L2: the
// forward g_s is formed and inverted in place in its final slot of b.g (or
// b.g64), and the backward pass keeps G_{s+1,s+1} and the product g_s G_{s+1}
// in two W x W matrices of a per-CTA workspace.  A persistent grid of
// DY_FACTOR_CTAS CTAs walks the (subdomain, frequency) units, so the workspace
// is bounded by the grid, not by K.

// In-place inverse of a complex symmetric global W x W matrix by the
// symmetric sweep operator (see gj_invert): the upper triangle only, then
// negation and mirror.  Step k caches column k (unscaled in prow, scaled by
// the pivot inverse in fcol, -1/a_kk at fcol[k]) on chip.
template <typename R>
__device__ void gj_invert_global(cx<R>* A, int W, cx<R>* prow, cx<R>* fcol) {
  using C = cx<R>;
  const int n = W * W;
  for (int k = 0; k < W; ++k) {
    __syncthreads();                         // step k-1 finished by every thread
    for (int e = threadIdx.x; e < W; e += DY_THREADS) {
      const C piv = cinv(A[(size_t)k * W + k]);
      const C a = (e < k) ? A[(size_t)e * W + k] : A[(size_t)k * W + e];
      prow[e] = a;
      fcol[e] = (e == k) ? -piv : a * piv;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n; e += DY_THREADS) {
      const int r = e / W, c = e - r * W;
      if (c < r) continue;
      if (r == k || c == k) A[e] = fcol[r == k ? c : r];
      else A[e] = cfma(-fcol[r], prow[c], A[e]);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += DY_THREADS) {
    const int r = e / W, c = e - r * W;
    if (c >= r) A[e] = -A[e];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += DY_THREADS) {
    const int r = e / W, c = e - r * W;
    if (c < r) A[e] = A[(size_t)c * W + r];
  }
  __syncthreads();
}

// C = base + scale * X Y for global W x W matrices (base may be null: C = X Y),
// in 32 x 32 output tiles staged through shared memory; W need not be a
// multiple of 32.  C must not alias X or Y.
template <typename R>
__device__ void gmem_matmul(cx<R>* C, const cx<R>* X, const cx<R>* Y, const cx<R>* base, R scale,
                            int W, cx<R> (*tx)[32], cx<R> (*ty)[32]) {
  using CC = cx<R>;
  const int tid = threadIdx.x, lc = tid & 31, lr = tid >> 5;   // 8 row groups x 32 columns
  const int nt = (W + 31) / 32;
  for (int tile = 0; tile < nt * nt; ++tile) {
    const int r0 = (tile / nt) * 32, c0 = (tile % nt) * 32;
    CC acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (int k0 = 0; k0 < W; k0 += 32) {
      __syncthreads();                       // previous tiles fully read
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int r = lr + 8 * m;
        tx[r][lc] = (r0 + r < W && k0 + lc < W) ? X[(size_t)(r0 + r) * W + k0 + lc] : CC{0, 0};
        ty[r][lc] = (k0 + r < W && c0 + lc < W) ? Y[(size_t)(k0 + r) * W + c0 + lc] : CC{0, 0};
      }
      __syncthreads();
#pragma unroll 8
      for (int k = 0; k < 32; ++k) {
        const CC yv = ty[k][lc];
#pragma unroll
        for (int m = 0; m < 4; ++m) acc[m] = cfma(tx[lr + 8 * m][k], yv, acc[m]);
      }
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int r = r0 + lr + 8 * m, c = c0 + lc;
      if (r < W && c < W) {
        const size_t e = (size_t)r * W + c;
        C[e] = base ? base[e] + scale * acc[m] : acc[m];
      }
    }
  }
  __syncthreads();
}

// R: the recursion's arithmetic, binary64 (FP64 form) or double-float (mixed
// form, R12: on the FP32 pipe), stored in b.g (FP64 form) or b.g64 (mixed: the
// double-float factors, beside their complex64 copy in b.g for the sweeps).
template <typename R, typename S>
__global__ void __launch_bounds__(DY_THREADS) k_factor_big(Geo g, Bufs b, int K) {
  using C = cx<R>;
  __shared__ C prow[DY_MAXW], fcol[DY_MAXW];
  __shared__ C tx[32][32], ty[32][32];
  constexpr bool two = sizeof(S) != sizeof(double);
  static_assert(sizeof(C) == sizeof(cxd), "factor storage holds 16 bytes per entry");
  const int W = g.W, Lx = g.Lx, T = g.T;
  const size_t n = (size_t)W * W;
  const R t = (R)g.t, t2 = (R)(g.t * g.t);
  C* Gw = reinterpret_cast<C*>(b.fwork) + (size_t)blockIdx.x * 2 * n;   // G_{s+1,s+1}
  C* Pw = Gw + n;                                                    // g_s G_{s+1,s+1}
  for (int unit = blockIdx.x; unit < g.p * K; unit += gridDim.x) {
    const int i = unit % g.p, kf = unit / g.p, w = T * g.h[i];
    const size_t uoff = ((size_t)kf * g.p + i) * (size_t)Lx * n;
    C* gout = reinterpret_cast<C*>(two ? b.g64 : b.g) + uoff;
    cx<S>* gsw = reinterpret_cast<cx<S>*>(b.g) + uoff;
    cxd* dB = b.diagB + (size_t)kf * g.Ndd + (size_t)i * Lx * W;
    // forward: g_s = (D_s - t^2 g_{s-1})^-1, formed and inverted in place
    for (int s = 0; s < Lx; ++s) {
      C* A = gout + (size_t)s * n;
      const C* Ap = A - n;
      __syncthreads();                       // g_{s-1} complete
      for (int e = threadIdx.x; e < (int)n; e += DY_THREADS) {
        const int r = e / W, c = e - r * W;
        C v = {0, 0};
        if (r < w && c < w) {
          if (s > 0) v = (-t2) * Ap[e];
          if (r == c) {
            v = v + cconv<R>(dyson_diag(g, b, kf, sub_nat(g, i, s, r)));
          } else if (slice_adjacent<R>(r, c, T)) {
            v.x += t;
          }
        } else if (r == c) {
          v = C{1, 0};                       // padding: identity, inverted to itself
        }
        A[e] = v;
      }
      gj_invert_global<R>(A, W, prow, fcol);
      for (int e = threadIdx.x; e < (int)n; e += DY_THREADS) {
        const int r = e / W, c = e - r * W;
        C v = A[e];
        if (r >= w || c >= w) {
          v = C{0, 0};
          A[e] = v;
        }
        if (two) gsw[(size_t)s * n + e] = cconv<S>(v);
      }
    }
    __syncthreads();
    // backward: Gw holds G_{s+1,s+1}
    const C* glast = gout + (size_t)(Lx - 1) * n;
    for (int e = threadIdx.x; e < (int)n; e += DY_THREADS) Gw[e] = glast[e];
    for (int r = threadIdx.x; r < W; r += DY_THREADS)
      dB[(size_t)(Lx - 1) * W + r] = (r < w) ? cconv<double>(glast[(size_t)r * W + r]) : cxd{0, 0};
    for (int s = Lx - 2; s >= 0; --s) {
      const C* gs = gout + (size_t)s * n;
      gmem_matmul<R>(Pw, gs, Gw, nullptr, R(0), W, tx, ty);   // g_s G_{s+1}
      if (b.offB) {                                           // diag of G_{s,s+1} = -t g_s G_{s+1}
        cxd* oB = b.offB + ((size_t)kf * g.p + i) * (size_t)Lx * W + (size_t)s * W;
        for (int r = threadIdx.x; r < W; r += DY_THREADS)
          oB[r] = (r < w) ? cconv<double>((-t) * Pw[(size_t)r * W + r]) : cxd{0, 0};
      }
      gmem_matmul<R>(Gw, Pw, gs, gs, t2, W, tx, ty);          // g_s + t^2 g_s G_{s+1} g_s
      for (int r = threadIdx.x; r < W; r += DY_THREADS)
        dB[(size_t)s * W + r] = (r < w) ? cconv<double>(Gw[(size_t)r * W + r]) : cxd{0, 0};
    }
    if (i == g.p - 1) {
      cxd* dI = b.diagB + (size_t)kf * g.Ndd + g.ifc_off;
      const size_t m = (size_t)(g.p - 1) * g.A;
      for (size_t e = threadIdx.x; e < m; e += DY_THREADS) dI[e] = cxd{0, 0};
    }
    __syncthreads();                         // workspace reads done before the next unit
  }
}

// Banded preconditioner of the interface Schur system.  The Schur complement
// S = C - E^T B^-1 E (Eq. 4) is never formed; its cheap approximation keeps,
// on each x line of interface layer l, the entries of S_ll within two sites
// along x (one in 3D slabs), which need only the diagonal, first and second
// off-diagonal blocks of B^-1 on the rows next to the layer, all from the
// factorization:
//   M[x][x]   = d_C(x) - t^2 (G_{x,x}^{l,top}   + G_{x,x}^{l+1,bot})
//   M[x][x+1] = t      - t^2 (G_{x,x+1}^{l,top} + G_{x,x+1}^{l+1,bot})
//   M[x][x+2] =        - t^2 (G_{x,x+2}^{l,top} + G_{x,x+2}^{l+1,bot})
// (in 3D the in-plane y hopping is dropped).  At the lowest Matsubara frequency
// of the 128^2 workload COCG needs 16 iterations to 1e-5 with the diagonal
// correction alone, 9 with the first off-diagonal and 6 with both.  Factors
// per x line, M = L D L^T without conjugation, computed in FP64 and stored in
// precision R: 1/d_x, l1_x, l2_x.
template <typename R>
__global__ void __launch_bounds__(DY_THREADS) k_precond(Geo g, Bufs b) {
  const int l = blockIdx.x, kf = blockIdx.y;
  const int Lx = g.Lx, T = g.T, A = g.A, W = g.W;
  const cxd* dB = b.diagB + (size_t)kf * g.Ndd;
  const size_t nsub = (size_t)Lx * W;
  const cxd* oB = b.offB + (size_t)kf * g.p * nsub;
  const cxd* o2 = (g.penta && b.off2) ? b.off2 + (size_t)kf * g.p * nsub : nullptr;
  cx<R>* pre = reinterpret_cast<cx<R>*>(b.pre) + ((size_t)kf * nifc(g) + (size_t)l * A) * 3;
  const double t = g.t, t2 = g.t * g.t;
  const cxd zero = {0, 0};
  for (int tr = threadIdx.x; tr < T; tr += DY_THREADS) {
    // row just below the layer: top row of subdomain l; just above: bottom row of l+1
    const size_t jb = (size_t)l * nsub + tr + T * (g.h[l] - 1);
    const size_t ja = (size_t)(l + 1) * nsub + tr;
    auto e1 = [&](int x) {                   // M[x][x+1]
      return (x >= 0 && x + 1 < Lx) ? cxd{t, 0} - t2 * (oB[jb + (size_t)x * W] + oB[ja + (size_t)x * W]) : zero;
    };
    auto e2 = [&](int x) {                   // M[x][x+2]
      return (o2 && x >= 0 && x + 2 < Lx) ? -(t2 * (o2[jb + (size_t)x * W] + o2[ja + (size_t)x * W])) : zero;
    };
    cxd d1 = zero, d2 = zero, l1p = zero;    // d_{x-1}, d_{x-2}, l1_{x-1}
    for (int x = 0; x < Lx; ++x) {
      const int a = x + Lx * tr;
      const cxd mxx = dyson_diag(g, b, kf, a + A * g.ylayer[l]) -
                      t2 * (dB[jb + (size_t)x * W] + dB[ja + (size_t)x * W]);
      const cxd l2 = (x >= 2) ? e2(x - 2) * cinv(d2) : zero;
      const cxd l1 = (x >= 1) ? (e1(x - 1) - l2 * l1p * d2) * cinv(d1) : zero;
      const cxd dx = mxx - l1 * l1 * d1 - l2 * l2 * d2;
      pre[a] = cconv<R>(cinv(dx));
      pre[A + a] = cconv<R>(l1);
      pre[2 * A + a] = cconv<R>(l2);
      d2 = d1;
      d1 = dx;
      l1p = l1;
    }
  }
}

}  // namespace

// H_ii (Eq. 1) of every DD slot, zero on padding: the mixed form's FP64
// residuals read it coalesced instead of gathering V and Sigma in natural order.
__global__ void __launch_bounds__(DY_THREADS) k_hdiag(Geo g, Bufs b) {
  const int kf = blockIdx.y;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < (size_t)g.Ndd;
       k += (size_t)gridDim.x * blockDim.x) {
    const int nat = b.dd2nat[k];
    b.hdiag[(size_t)kf * g.Ndd + k] = nat >= 0 ? dyson_diag(g, b, kf, nat) : cxd{0, 0};
  }
}

template <typename R, typename S>
cudaError_t launch_factor(const Geo& g, const Bufs& b, int K, cudaStream_t st) {
  if (b.hdiag) {
    const size_t blocks = ((size_t)g.Ndd + DY_THREADS - 1) / DY_THREADS;
    k_hdiag<<<dim3((unsigned)(blocks < 1024 ? blocks : 1024), K), DY_THREADS, 0, st>>>(g, b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (g.W > DY_MAXW_SMEM) {
    // wide slices: the recursion in global memory (binary64, or double-float in the
    // mixed form)
    if constexpr (sizeof(cx<R>) == sizeof(cxd)) {
      if (g.W > DY_MAXW || !b.fwork) return cudaErrorInvalidValue;
      int units = g.p * K;
      k_factor_big<R, S><<<units < DY_FACTOR_CTAS ? units : DY_FACTOR_CTAS, DY_THREADS, 0, st>>>(g, b, K);
      return cudaGetLastError();
    } else {
      return cudaErrorInvalidValue;
    }
  }
  size_t smem = (3 * (size_t)g.W * g.W + 6 * (size_t)g.W) * sizeof(cx<R>);
  cudaError_t e = raise_smem_limit((const void*)k_factor<R, S>, smem);
  if (e != cudaSuccess) return e;
  k_factor<R, S><<<dim3(g.p, K), DY_THREADS, smem, st>>>(g, b);
  return cudaGetLastError();
}
template cudaError_t launch_factor<double, double>(const Geo&, const Bufs&, int, cudaStream_t);
template cudaError_t launch_factor<dfl, float>(const Geo&, const Bufs&, int, cudaStream_t);
template cudaError_t launch_factor<float, float>(const Geo&, const Bufs&, int, cudaStream_t);

template <typename R>
cudaError_t launch_precond(const Geo& g, const Bufs& b, int K, cudaStream_t st) {
  if (g.p < 2) return cudaSuccess;
  if (g.lpre) {
    cudaError_t e = launch_surface(g, b, K, st);
    if (e != cudaSuccess) return e;
    return launch_layer_inv<R>(g, b, K, st);
  }
  k_precond<R><<<dim3(g.p - 1, K), DY_THREADS, 0, st>>>(g, b);
  return cudaGetLastError();
}
template cudaError_t launch_precond<double>(const Geo&, const Bufs&, int, cudaStream_t);
template cudaError_t launch_precond<float>(const Geo&, const Bufs&, int, cudaStream_t);

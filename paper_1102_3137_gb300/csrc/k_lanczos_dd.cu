// Lanczos step of the mixed form (Sec. 2.1 recurrence in the bilinear form,
// CGS2 re-orthogonalisation, Eq. 9 assembly) with its dot products and
// basis updates in double-float arithmetic on the FP32 pipe.
//
// The basis Q is stored as double-floats (cdfl: hi + lo binary32 per real
// part, 47 significant bits, 16 bytes per complex entry like binary64), so the
// passes over it read the split form directly; the X-matvec output u, the
// running diagonal and every scalar of T stay in binary64.  What moves off the
// binary64 pipe (GB300 issues binary32 FMAs at ~64x its binary64 rate) is the
// arithmetic of the passes over Q: products accumulated with
// TwoProduct/TwoSum (~2^-47 relative per operation); u is split by integer
// operations where it is read.
//
// Classical Gram-Schmidt twice, with the three-term part folded in and the
// second pass's coefficients taken from the Gram matrix of the stored basis:
//   pass A:  g  = Q_j^T u                     (alpha_j = g_j)
//            h  = g - M g,  M = Q_j^T Q_j     (M kept per frequency, binary64)
//   pass B:  r  = u - Q_j (g + h)             (formed in binary64, stored split)
//            M's next column: Q_j^T r / beta_{j+1}
// In exact arithmetic h = Q_j^T (u - Q_j g) is the second pass's coefficient
// vector, so r is the classical Gram-Schmidt residual orthogonalised twice;
// reading Q_j^T Q_j from M instead of re-projecting u - Q_j g saves a sweep
// over the basis (two reads of Q per step instead of three, three multiply-
// accumulates per basis entry instead of four).  With the unit diagonal of M
// exact, M - I holds the basis's measured loss of orthogonality, which h
// removes to second order (one-reduce CGS2 in the Gram-matrix form); the
// remaining error is the rounding of g, ~2^-47 ||u|| / |beta_{j+1}|.
// Thread layout.  The CTA's part of the DD layout is walked in groups of
// TG = 128 consecutive entries.  The per-site sum over the basis (r) runs two
// threads per site along l (even and odd l), reading each vector's entries
// coalesced across the warp.  Per-vector sums (g and the Gram column) run one
// warp per eight vectors l = w + 8m, the lanes over the
// group's sites, with the group's u (pass A) or r (pass B) staged in shared
// memory; pass B re-reads the group's basis entries right after its per-site
// half, from L2.  Per-vector totals are warp-shuffled, then summed over the
// cluster's CTAs in rank order in binary64, so every CTA of a frequency holds
// bit-identical coefficients.  Rank caps up to 64 (eight vectors per warp);
// larger caps take the binary64 kernel.  The running sums are double-floats
// updated by TwoProduct and TwoSum without renormalising the low word.
#include "solve_device.cuh"

namespace {

constexpr int LPW = 8;                   // basis vectors per warp in the per-vector passes
constexpr int LDD_MAX = DY_WARPS * LPW;  // 64: largest j + 1 this kernel takes
constexpr int TG = 128;                  // sites per group
static_assert(DY_THREADS == 2 * TG, "two threads per site of a group");
// The Lanczos thresholds scaled to double-float arithmetic: the same multiples of the
// unit roundoff as TERM_TOL and BRK_TOL are of binary64's (2^-47 / 2^-53 = 64).
constexpr double TERM_TOL_DD = 64.0 * TERM_TOL;
constexpr double BRK_TOL_DD = 64.0 * BRK_TOL;
// A step re-projects r when ||r|| < REORTH_ETA ||u||: the Gram form's orthogonality is
// ~2^-47 ||u|| / ||r||, held below ~1.5e-13 this way.
constexpr double REORTH_ETA = 0.05;

__device__ __forceinline__ cdfl czero() { return {dfl(0.f, 0.f), dfl(0.f, 0.f)}; }

// acc + a*b for double-floats: the product's hi part and its exact error
// (TwoProduct) plus the cross terms; hi added to acc.hi by TwoSum; every
// error term lands in acc.lo, which is not renormalised (it stays within a
// few ulp of acc.hi, so TwoSum stays exact and acc.lo's own rounding is of
// the order 2^-48 |acc|).
__device__ __forceinline__ void dmac(dfl& acc, dfl a, dfl b) {
  float p, e, s, t;
  dfl_two_prod(a.hi, b.hi, p, e);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  dfl_two_sum(acc.hi, p, s, t);
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(t, e));
}
__device__ __forceinline__ void cmac(cdfl& acc, const cdfl& a, const cdfl& b) {
  dmac(acc.x, a.x, b.x);
  dmac(acc.x, dfl(-a.y.hi, -a.y.lo), b.y);
  dmac(acc.y, a.x, b.y);
  dmac(acc.y, a.y, b.x);
}
// renormalised sum / difference of two double-floats
__device__ __forceinline__ cdfl cadd(const cdfl& a, const cdfl& b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cdfl csub(const cdfl& a, const cdfl& b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ cdfl cnorm(const cdfl& a) { return {dfl_fast(a.x.hi, a.x.lo), dfl_fast(a.y.hi, a.y.lo)}; }

__device__ __forceinline__ cdfl warp_sum_dd(cdfl v) {
  v = cnorm(v);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    v.x = v.x + shfl_xor_any(v.x, off);
    v.y = v.y + shfl_xor_any(v.y, off);
  }
  return v;
}

struct LanDDSmem {
  cxd vpart[2][LDD_MAX];               // this CTA's per-vector partial sums (phase double-buffered)
  cxd vres[LDD_MAX];                   // the cluster totals
  cxd gv[LDD_MAX];                     // g = Q^T u (pass A totals)
  cdfl coef[LDD_MAX];                  // coefficients of the current pass, double-float
  cdfl st[2][TG];                      // staged per-site values of one group (u; r1 halves)
};

// Cluster total of the per-vector partials vpart[phase][0..n): every CTA adds
// the P CTAs' partials in rank order (binary64), so all hold the same bits.
__device__ void cluster_vec_sum(cg::cluster_group& cl, LanDDSmem& sm, int& vphase, int P, int n) {
  __syncthreads();
  cl.sync();
  for (int l = threadIdx.x; l < n; l += DY_THREADS) {
    cxd s = {0, 0};
    for (int r = 0; r < P; ++r) {
      const LanDDSmem* rem = cl.map_shared_rank(&sm, r);
      s = s + rem->vpart[vphase][l];
    }
    sm.vres[l] = s;
  }
  __syncthreads();
  vphase ^= 1;
}

// this warp's accumulated per-vector sums -> vpart (binary64), vectors l = w + 8m <= j
__device__ __forceinline__ void put_partials(LanDDSmem& sm, int vphase, int j, const cdfl (&acc)[LPW]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int m = 0; m < LPW; ++m) {
    const int l = w + DY_WARPS * m;
    if (l <= j) {
      const cdfl s = warp_sum_dd(acc[m]);
      if (lane == 0) sm.vpart[vphase][l] = cwiden(s);
    }
  }
}

// sum over l = l0, l0 + dl, ... <= j of Q_l[k] c_l (double-float): the entries of
// eight vectors are loaded before any is used (eight loads in flight per
// thread), then summed in two interleaved chains
__device__ __forceinline__ cdfl basis_sum(const cdfl* Q, size_t Ndd, size_t k, int j, int l0, int dl,
                                          const cdfl* coef) {
  cdfl s0 = czero(), s1 = czero();
  for (int lb = l0; lb <= j; lb += 8 * dl) {
    cdfl qv[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int l = lb + m * dl;
      qv[m] = l <= j ? Q[(size_t)l * Ndd + k] : czero();
    }
#pragma unroll
    for (int m = 0; m < 8; m += 2) {
      const int l = lb + m * dl;
      if (l <= j) cmac(s0, qv[m], coef[l]);
      if (l + dl <= j) cmac(s1, qv[m + 1], coef[l + dl]);
    }
  }
  return cadd(cnorm(s0), cnorm(s1));
}

template <int SPLIT>
__global__ void __launch_bounds__(DY_THREADS, 2) k_lanczos_dd(Geo g, Bufs b, int j) {
  cg::cluster_group cl = cg::this_cluster();
  __shared__ RedSmem rs;
  __shared__ LanDDSmem sm;
  const int i = blockIdx.x / SPLIT, part = blockIdx.x - i * SPLIT, kf = blockIdx.y, P = g.p * SPLIT;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  int* stt = b.st + (size_t)kf * ST_N;
  if (stt[ST_DONE]) return;
  int phase = 0, vphase = 0;
  const size_t Ndd = g.Ndd;
  const int nsub = g.Lx * g.W, n = own_count(g, i);
  const int ngrp = (n + TG - 1) / TG;
  // the basis is stored as double-floats (Geo::qsplit)
  cdfl* Q = reinterpret_cast<cdfl*>(b.Q + (size_t)kf * (g.k_max + g.nb) * Ndd);
  const cdfl* qj = Q + (size_t)j * Ndd;
  const cdfl* qm = (j > 0) ? Q + (size_t)(j - 1) * Ndd : nullptr;
  cdfl* r = Q + (size_t)(j + 1) * Ndd;
  const cxd* u = b.u + (size_t)kf * Ndd;
  cxd* acc = b.acc + (size_t)kf * Ndd;
  cxd* lan = b.lan + (size_t)kf * (g.k_max + g.nb) * 2;
  const int K1 = g.k_max + 1;
  cxd* gram = b.gram + (size_t)kf * K1 * K1;
  const cxd beta_j = (j > 0) ? lan[2 * j + 1] : cxd{0, 0};
  // read before the first cluster barrier: CTA 0 updates it once all CTAs passed the last one
  const double maxT_prev = b.maxT[kf];

  // ---- pass A: g = Q^T u (warp w: vectors w + 8m; lanes over the group's sites)
  {
    cdfl a[LPW];
#pragma unroll
    for (int m = 0; m < LPW; ++m) a[m] = czero();
    for (int gr = part; gr < ngrp; gr += SPLIT) {
      const int e0 = gr * TG;
      if (tid < TG) {
        const int e = e0 + tid;
        sm.st[0][tid] = e < n ? csplit(u[own_idx(g, i, e, nsub)]) : czero();
      }
      __syncthreads();
      for (int c = lane; c < TG; c += 32) {
        const int e = e0 + c;
        if (e >= n) break;
        const size_t k = own_idx(g, i, e, nsub);
        const cdfl ud = sm.st[0][c];
        cdfl qv[LPW];
#pragma unroll
        for (int m = 0; m < LPW; ++m) {
          const int l = w + DY_WARPS * m;
          qv[m] = l <= j ? Q[(size_t)l * Ndd + k] : czero();
        }
#pragma unroll
        for (int m = 0; m < LPW; ++m)
          if (w + DY_WARPS * m <= j) cmac(a[m], qv[m], ud);
      }
      __syncthreads();
    }
    put_partials(sm, vphase, j, a);
  }
  cluster_vec_sum(cl, sm, vphase, P, j + 1);
  const cxd alpha = sm.vres[j];
  for (int l = tid; l <= j; l += DY_THREADS) sm.gv[l] = sm.vres[l];
  __syncthreads();
  // ---- second Gram-Schmidt coefficients from the Gram matrix M = Q_j^T Q_j of the
  // stored basis: h = Q_j^T (u - Q_j g) = g - M g, so g + h = g - (M - I) g (the unit
  // diagonal of M taken as exact; binary64)
  for (int l = tid; l <= j; l += DY_THREADS) {
    cxd s = {0, 0};
    for (int m = 0; m <= j; ++m) {
      if (m == l) continue;
      const cxd e = l < m ? gram[(size_t)m * K1 + l] : gram[(size_t)l * K1 + m];
      s = cfma(e, sm.gv[m], s);
    }
    sm.coef[l] = csplit(sm.gv[l] - s);
  }
  __syncthreads();

  // ---- pass B: r = u - Q (g + h) per site (two threads per site, even and odd l),
  // finished in binary64 and stored split, with r^T r, ||r||^2 and the Eq. 9
  // three-vector update; then h' = Q^T r (warp w: vectors w + 8m, lanes over the
  // group's sites, r staged in shared memory), the Gram column of the next vector
  cxd v2[3] = {{0, 0}, {0, 0}, {0, 0}};   // r^T r, ||r||^2, ||u||^2
  const cdfl ad = csplit(alpha), bd = csplit(2.0 * beta_j);
  const int c0 = tid & (TG - 1), half = tid / TG;
  {
    cdfl a[LPW];
#pragma unroll
    for (int m = 0; m < LPW; ++m) a[m] = czero();
    for (int gr = part; gr < ngrp; gr += SPLIT) {
      const int e0 = gr * TG;
      {
        const int e = e0 + c0;
        cdfl s = czero();
        if (e < n) s = basis_sum(Q, Ndd, own_idx(g, i, e, nsub), j, half, 2, sm.coef);
        sm.st[half][c0] = s;
      }
      __syncthreads();
      cdfl rd = czero();
      if (half == 0 && e0 + c0 < n) {
        const size_t k = own_idx(g, i, e0 + c0, nsub);
        const cdfl tot = cadd(sm.st[0][c0], sm.st[1][c0]);
        const cxd uv = u[k];
        const cxd rv = {(uv.x - f2d_bits(tot.x.hi)) - f2d_bits(tot.x.lo),
                        (uv.y - f2d_bits(tot.y.hi)) - f2d_bits(tot.y.lo)};
        rd = csplit(rv);
        r[k] = rd;
        v2[0] = cfma(rv, rv, v2[0]);
        v2[1].x += cabs2(rv);
        v2[2].x += cabs2(uv);
        const cdfl qjd = qj[k];
        cdfl sq = czero(), d = czero();
        cmac(sq, qjd, qjd);
        cmac(d, ad, cnorm(sq));
        if (qm) {
          cdfl pr = czero();
          cmac(pr, qm[k], qjd);
          cmac(d, bd, cnorm(pr));
        }
        d = cnorm(d);
        const cxd av = acc[k];
        acc[k] = cxd{(av.x + f2d_bits(d.x.hi)) + f2d_bits(d.x.lo), (av.y + f2d_bits(d.y.hi)) + f2d_bits(d.y.lo)};
      }
      __syncthreads();                     // both halves have read st before it is overwritten
      if (half == 0) sm.st[0][c0] = rd;
      __syncthreads();
      for (int c = lane; c < TG; c += 32) {
        const int e = e0 + c;
        if (e >= n) break;
        const size_t k = own_idx(g, i, e, nsub);
        cdfl qv[LPW];
#pragma unroll
        for (int m = 0; m < LPW; ++m) {
          const int l = w + DY_WARPS * m;
          qv[m] = l <= j ? Q[(size_t)l * Ndd + k] : czero();
        }
        const cdfl rc = sm.st[0][c];
#pragma unroll
        for (int m = 0; m < LPW; ++m)
          if (w + DY_WARPS * m <= j) cmac(a[m], qv[m], rc);
      }
      __syncthreads();
    }
    put_partials(sm, vphase, j, a);
  }
  cluster_vec_sum(cl, sm, vphase, P, j + 1);   // sm.vres[l] = q_l^T r
  cluster_sum<3>(cl, rs, phase, P, v2);
  cxd rr = v2[0];
  double rn2 = v2[1].x;
  // ---- pass C, only when r lost most of u (||r|| < REORTH_ETA ||u||, near an
  // invariant subspace): the Gram form leaves r's rounding error ~2^-47 ||u|| in
  // place, so project r once more onto the complement, r -= Q (Q^T r), as the
  // classical second pass would (the selective test of Daniel, Gragg, Kaufman and
  // Stewart, 1976); the next vector's Gram column is then zero to working accuracy
  const bool reorth = rn2 < REORTH_ETA * REORTH_ETA * v2[2].x;
  if (reorth) {
    for (int l = tid; l <= j; l += DY_THREADS) sm.coef[l] = csplit(sm.vres[l]);
    __syncthreads();
    cxd w2[2] = {{0, 0}, {0, 0}};
    for (int gr = part + half * SPLIT; gr < ngrp; gr += 2 * SPLIT) {
      const int e = gr * TG + c0;
      if (e >= n) continue;
      const size_t k = own_idx(g, i, e, nsub);
      const cdfl tot = basis_sum(Q, Ndd, k, j, 0, 1, sm.coef);
      const cdfl rn = csub(r[k], tot);
      r[k] = rn;
      const cxd rv = cwiden(rn);
      w2[0] = cfma(rv, rv, w2[0]);
      w2[1].x += cabs2(rv);
    }
    cluster_sum<2>(cl, rs, phase, P, w2);
    rr = w2[0];
    rn2 = w2[1].x;
  }
  const cxd beta = csqrt_principal(rr);
  const double maxT = fmax(maxT_prev, sqrt(cabs2(alpha)));
  const double babs = sqrt(cabs2(beta));
  int done = 0, flag = 0;
  if (j == g.k_max - 1) {
    done = 1;
  } else if (sqrt(rn2) <= TERM_TOL_DD * maxT) {         // r vanished: invariant subspace
    done = 1;
    flag = 1;
  } else if (sqrt(cabs2(rr)) <= BRK_TOL_DD * rn2) {     // r != 0, (r, r)_C ~ 0: breakdown
    done = 1;
    flag = 2;
  }
  if (!done) {
    // Gram column of q_{j+1} = r / beta: q_l^T q_{j+1} = (q_l^T r) / beta, l <= j
    if (blockIdx.x == 0) {
      const cxd ibd = cinv(beta);
      for (int l = tid; l <= j; l += DY_THREADS)
        gram[(size_t)(j + 1) * K1 + l] = reorth ? cxd{0, 0} : sm.vres[l] * ibd;
    }
    // q_{j+1} = r / beta in double-float
    const cdfl ib = csplit(cinv(beta));
    for (int gr = part + half * SPLIT; gr < ngrp; gr += 2 * SPLIT) {
      const int e = gr * TG + c0;
      if (e < n) {
        const size_t k = own_idx(g, i, e, nsub);
        cdfl q = czero();
        cmac(q, r[k], ib);
        r[k] = cnorm(q);
      }
    }
  }
  if (blockIdx.x == 0 && tid == 0) {
    lan[2 * j] = alpha;
    stt[ST_STEPS] = j + 1;
    if (done) {
      stt[ST_DONE] = 1;
      stt[ST_STATUS] |= flag;
    } else {
      lan[2 * (j + 1) + 1] = beta;
      b.maxT[kf] = fmax(maxT, babs);
    }
  }
  cl.sync();          // no CTA exits while a peer may still read its shared memory
}

}  // namespace

// The mixed form's Lanczos step (rank caps up to 64; the binary64 kernel otherwise).
cudaError_t launch_lanczos_dd(const Geo& g, const Bufs& b, int K, int j, cudaStream_t st) {
  if (g.k_max > LDD_MAX || g.nb != 1) return cudaErrorInvalidValue;
  if (2 * g.p <= 8) return launch_cluster(k_lanczos_dd<2>, dim3(2 * g.p, K), 2 * g.p, 0, st, g, b, j);
  return launch_cluster(k_lanczos_dd<1>, dim3(g.p, K), g.p, 0, st, g, b, j);
}

// Block complex-symmetric Lanczos on X (block size nb = 2..4).  Not in the
// paper: the block form of the Sec. 2.1 recurrence in the bilinear form, for
// an X whose eigenvalues are degenerate (one start vector reaches only one
// direction of each eigenspace, so the scalar method stops short of range(X)).
//
//   X Q_j = Q_{j-1} B_j^T + Q_j A_j + Q_{j+1} B_{j+1},   A_j = Q_j^T X Q_j,
//   R_j = X Q_j - Q_j A_j - Q_{j-1} B_j^T  (then CGS2 against all blocks) = Q_{j+1} B_{j+1}
//
// with R_j split column by column by Gram-Schmidt (twice) in the bilinear
// form; a column whose 2-norm falls to TERM_TOL max|T| is deflated to zero.
// The diagonal of Q T Q^T gains diag(Q_j A_j Q_j^T) + 2 diag(Q_j B_j Q_{j-1}^T)
// per block step (Eq. 9 per block).  One cluster per frequency, one CTA per
// subdomain, fixed-order cluster reductions as in the scalar step.
#include "solve_device.cuh"

namespace {

// Column c of the block at Qb (columns nb apart by Ndd): remove the earlier
// columns of the block twice, then normalise in the bilinear form.  Bs[d*nb+c]
// accumulates the removed coefficients, Bs[c*nb+c] receives the pivot.
// Returns 0, 1 (deflated: |pivot| <= tol, the column is set to zero) or
// 2 (breakdown: (r, r)_C vanished for a column that is not small).
__device__ int qr_column(cg::cluster_group& cl, RedSmem& rs, int& phase, const Geo& g, int i,
                         cxd* Qb, int c, cxd* Bs, double tol) {
  const int nb = g.nb, n = own_count(g, i), nsub = g.Lx * g.W;
  const size_t Ndd = g.Ndd;
  cxd* rc = Qb + (size_t)c * Ndd;
  for (int pass = 0; pass < 2 && c > 0; ++pass) {
    cxd h[DY_MAXNB] = {};
    for (int e = threadIdx.x; e < n; e += DY_THREADS) {
      const size_t k = own_idx(g, i, e, nsub);
      const cxd rv = rc[k];
#pragma unroll
      for (int d = 0; d < DY_MAXNB; ++d)
        if (d < c) h[d] = cfma(Qb[(size_t)d * Ndd + k], rv, h[d]);
    }
    cluster_sum<DY_MAXNB>(cl, rs, phase, g.p, h);
    for (int e = threadIdx.x; e < n; e += DY_THREADS) {
      const size_t k = own_idx(g, i, e, nsub);
      cxd rv = rc[k];
#pragma unroll
      for (int d = 0; d < DY_MAXNB; ++d)
        if (d < c) rv = cfma(-h[d], Qb[(size_t)d * Ndd + k], rv);
      rc[k] = rv;
    }
    if (threadIdx.x == 0)
      for (int d = 0; d < c; ++d) Bs[d * nb + c] = Bs[d * nb + c] + h[d];
  }
  cxd v2[2] = {{0, 0}, {0, 0}};
  for (int e = threadIdx.x; e < n; e += DY_THREADS) {
    const cxd rv = rc[own_idx(g, i, e, nsub)];
    v2[0] = cfma(rv, rv, v2[0]);
    v2[1].x += cabs2(rv);
  }
  cluster_sum<2>(cl, rs, phase, g.p, v2);
  const cxd beta = csqrt_principal(v2[0]);
  int res = 0;
  cxd scale = {0, 0};
  if (sqrt(v2[1].x) <= tol) {          // the column vanished (2-norm): deflate
    res = 1;
  } else if (sqrt(cabs2(v2[0])) <= BRK_TOL * v2[1].x) {
    return 2;
  } else {
    scale = cinv(beta);
  }
  for (int e = threadIdx.x; e < n; e += DY_THREADS) {
    const size_t k = own_idx(g, i, e, nsub);
    rc[k] = rc[k] * scale;
  }
  if (threadIdx.x == 0) Bs[c * nb + c] = res ? cxd{0, 0} : beta;
  return res;
}

// Sum over this cluster of x_m^T y_m for the pairs m < npairs (x_m, y_m from
// the callback, as DD-layout column pointers), eight pairs per reduction;
// the totals land in out[m] (shared memory, every CTA).
template <typename Pair>
__device__ void pair_dots(cg::cluster_group& cl, RedSmem& rs, int& phase, const Geo& g, int i,
                          int npairs, Pair pair, cxd* out) {
  const int n = own_count(g, i), nsub = g.Lx * g.W;
  for (int m0 = 0; m0 < npairs; m0 += 8) {
    cxd h8[8] = {};
    for (int e = threadIdx.x; e < n; e += DY_THREADS) {
      const size_t k = own_idx(g, i, e, nsub);
#pragma unroll
      for (int mm = 0; mm < 8; ++mm)
        if (m0 + mm < npairs) {
          const cxd* x;
          const cxd* y;
          pair(m0 + mm, x, y);
          h8[mm] = cfma(x[k], y[k], h8[mm]);
        }
    }
    cluster_sum<8>(cl, rs, phase, g.p, h8);
    if (threadIdx.x < 8 && m0 + threadIdx.x < npairs) out[m0 + threadIdx.x] = h8[threadIdx.x];
  }
  __syncthreads();
}

// Gather the nb real start columns into block 0 and split them by the
// bilinear QR (a start block of lower rank is a breakdown).  Clears the
// per-frequency state.
__global__ void __launch_bounds__(DY_THREADS) k_init_block(Geo g, Bufs b) {
  cg::cluster_group cl = cg::this_cluster();
  __shared__ RedSmem rs;
  __shared__ cxd Bs[DY_MAXNB * DY_MAXNB];
  const int i = blockIdx.x, f = blockIdx.y, nb = g.nb;
  int phase = 0;
  const int nsub = g.Lx * g.W, n = own_count(g, i);
  const size_t Ndd = g.Ndd;
  cxd* Q0 = b.Q + (size_t)f * (g.k_max + nb) * Ndd;
  cxd* acc = b.acc + (size_t)f * Ndd;
  if (threadIdx.x < nb * nb) Bs[threadIdx.x] = cxd{0, 0};
  for (int e = threadIdx.x; e < n; e += DY_THREADS) {
    const size_t k = own_idx(g, i, e, nsub);
    const int nat = b.dd2nat[k];
    for (int c = 0; c < nb; ++c) Q0[(size_t)c * Ndd + k] = cxd{nat >= 0 ? b.q1[(size_t)c * g.N + nat] : 0.0, 0};
    acc[k] = cxd{0, 0};
  }
  int bad = 0;
  for (int c = 0; c < nb && !bad; ++c) bad = qr_column(cl, rs, phase, g, i, Q0, c, Bs, 0.0);
  if (threadIdx.x == 0 && b.sweeps)
    for (int c = 0; c < nb; ++c) b.sweeps[((size_t)f * nb + c) * g.p + i] = 0;
  if (i == 0 && threadIdx.x == 0) {
    int* st = b.st + (size_t)f * ST_N;
    for (int k = 0; k < ST_N; ++k) st[k] = 0;
    if (g.p < 2) st[ST_DONE] = 1;        // one subdomain: X = 0, no Lanczos steps
    if (bad) {
      st[ST_DONE] = 1;
      st[ST_STATUS] = 2;
    }
    cxd* lan = b.lan + (size_t)f * (g.k_max + nb) * 2 * nb;
    for (int k = 0; k < 2 * nb * nb; ++k) lan[k] = cxd{0, 0};
    b.maxT[f] = 0.0;
  }
  cl.sync();          // no CTA exits while a peer may still read its shared memory
}

// Block step j: A_j, the Eq. 9 update, R_j with CGS2, and (unless j is the
// last step) its bilinear QR into block j + 1 with the deflation and
// breakdown tests.  U = X Q_j sits in the frequency's nb work slots.
__global__ void __launch_bounds__(DY_THREADS) k_block_lanczos(Geo g, Bufs b, int j) {
  cg::cluster_group cl = cg::this_cluster();
  __shared__ RedSmem rs;
  __shared__ cxd As[DY_MAXNB * DY_MAXNB], Bj[DY_MAXNB * DY_MAXNB], Bn[DY_MAXNB * DY_MAXNB];
  __shared__ cxd hs[DY_BLOCK_H];
  const int i = blockIdx.x, f = blockIdx.y, nb = g.nb;
  int* st = b.st + (size_t)f * ST_N;
  if (st[ST_DONE]) return;
  int phase = 0;
  const size_t Ndd = g.Ndd;
  const int nsub = g.Lx * g.W, n = own_count(g, i);
  cxd* Qf = b.Q + (size_t)f * (g.k_max + nb) * Ndd;
  const cxd* Qj = Qf + (size_t)j * nb * Ndd;
  const cxd* Qm = j > 0 ? Qf + (size_t)(j - 1) * nb * Ndd : nullptr;
  cxd* Rn = Qf + (size_t)(j + 1) * nb * Ndd;
  const cxd* U = b.u + (size_t)f * nb * Ndd;
  cxd* acc = b.acc + (size_t)f * Ndd;
  cxd* lan = b.lan + (size_t)f * (g.k_max + nb) * 2 * nb;
  // read before the first cluster barrier: CTA 0 updates it once all CTAs passed the last one
  const double maxT_prev = b.maxT[f];
  const int nn = nb * nb;
  if (threadIdx.x < nn) {
    Bj[threadIdx.x] = lan[(size_t)(2 * j + 1) * nn + threadIdx.x];   // zero for j = 0
    Bn[threadIdx.x] = cxd{0, 0};
  }
  // A_j[d][c] = q_{j,d}^T u_c
  pair_dots(cl, rs, phase, g, i, nn,
            [&](int m, const cxd*& x, const cxd*& y) {
              x = Qj + (size_t)(m / nb) * Ndd;
              y = U + (size_t)(m % nb) * Ndd;
            },
            As);
  // Eq. 9 per block, and R_j = U - Q_j A_j - Q_{j-1} B_j^T into block j + 1
  for (int e = threadIdx.x; e < n; e += DY_THREADS) {
    const size_t k = own_idx(g, i, e, nsub);
    cxd qv[DY_MAXNB], qm[DY_MAXNB];
#pragma unroll
    for (int d = 0; d < DY_MAXNB; ++d) {
      qv[d] = d < nb ? Qj[(size_t)d * Ndd + k] : cxd{0, 0};
      qm[d] = (d < nb && Qm) ? Qm[(size_t)d * Ndd + k] : cxd{0, 0};
    }
    cxd a = acc[k];
#pragma unroll
    for (int c = 0; c < DY_MAXNB; ++c) {
      if (c >= nb) break;
      cxd ta = {0, 0}, tb = {0, 0};
#pragma unroll
      for (int d = 0; d < DY_MAXNB; ++d)
        if (d < nb) {
          ta = cfma(As[c * nb + d], qv[d], ta);
          tb = cfma(Bj[c * nb + d], qm[d], tb);
        }
      a = cfma(qv[c], ta, a);
      a = cfma(2.0 * qv[c], tb, a);
    }
    acc[k] = a;
#pragma unroll
    for (int c = 0; c < DY_MAXNB; ++c) {
      if (c >= nb) break;
      cxd r = U[(size_t)c * Ndd + k];
#pragma unroll
      for (int d = 0; d < DY_MAXNB; ++d)
        if (d < nb) {
          r = cfma(-As[d * nb + c], qv[d], r);
          r = cfma(-Bj[c * nb + d], qm[d], r);
        }
      Rn[(size_t)c * Ndd + k] = r;
    }
  }
  // CGS2 in the bilinear form against every column of blocks 0..j
  const int ncol = (j + 1) * nb;
  for (int pass = 0; pass < 2; ++pass) {
    pair_dots(cl, rs, phase, g, i, ncol * nb,
              [&](int m, const cxd*& x, const cxd*& y) {
                x = Qf + (size_t)(m / nb) * Ndd;
                y = Rn + (size_t)(m % nb) * Ndd;
              },
              hs);
    for (int e = threadIdx.x; e < n; e += DY_THREADS) {
      const size_t k = own_idx(g, i, e, nsub);
      cxd r[DY_MAXNB];
#pragma unroll
      for (int c = 0; c < DY_MAXNB; ++c) r[c] = c < nb ? Rn[(size_t)c * Ndd + k] : cxd{0, 0};
      for (int col = 0; col < ncol; ++col) {
        const cxd qv = Qf[(size_t)col * Ndd + k];
#pragma unroll
        for (int c = 0; c < DY_MAXNB; ++c)
          if (c < nb) r[c] = cfma(-hs[col * nb + c], qv, r[c]);
      }
#pragma unroll
      for (int c = 0; c < DY_MAXNB; ++c)
        if (c < nb) Rn[(size_t)c * Ndd + k] = r[c];
    }
    __syncthreads();
  }
  double maxT = maxT_prev;
  for (int m = 0; m < nn; ++m) maxT = fmax(maxT, sqrt(cabs2(As[m])));
  int done = 0, flag = 0;
  if (j == g.k_max / nb - 1) {
    done = 1;
  } else {
    int ndefl = 0;
    for (int c = 0; c < nb; ++c) {
      const int r = qr_column(cl, rs, phase, g, i, Rn, c, Bn, TERM_TOL * maxT);
      if (r == 2) {
        done = 1;
        flag = 2;
        break;
      }
      ndefl += r;
    }
    if (!done && ndefl == nb) {
      done = 1;
      flag = 1;
    }
    __syncthreads();
  }
  if (i == 0 && threadIdx.x == 0) {
    for (int m = 0; m < nn; ++m) lan[(size_t)(2 * j) * nn + m] = As[m];
    st[ST_STEPS] = j + 1;
    if (done) {
      st[ST_DONE] = 1;
      st[ST_STATUS] |= flag;
    } else {
      double mt = maxT;
      for (int m = 0; m < nn; ++m) {
        lan[(size_t)(2 * j + 3) * nn + m] = Bn[m];
        mt = fmax(mt, sqrt(cabs2(Bn[m])));
      }
      b.maxT[f] = mt;
    }
  }
  cl.sync();          // no CTA exits while a peer may still read its shared memory
}

}  // namespace

cudaError_t launch_init_block(const Geo& g, const Bufs& b, int K, cudaStream_t st) {
  if (g.nb < 2 || g.nb > DY_MAXNB) return cudaErrorInvalidValue;
  return launch_cluster(k_init_block, dim3(g.p, K), g.p, 0, st, g, b);
}

cudaError_t launch_block_lanczos(const Geo& g, const Bufs& b, int K, int j, cudaStream_t st) {
  if (g.nb < 2 || g.nb > DY_MAXNB || g.k_max % g.nb || g.k_max * g.nb > DY_BLOCK_H)
    return cudaErrorInvalidValue;
  return launch_cluster(k_block_lanczos, dim3(g.p, K), g.p, 0, st, g, b, j);
}

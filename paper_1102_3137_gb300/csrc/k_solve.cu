// Lanczos step, start vector and the small per-frequency kernels (the
// X-matvec and subdomain-solve kernels, which carry the block sweeps, are
// compiled in k_xmatvec_c64.cu and k_xmatvec_c128.cu).
#include "solve_device.cuh"

namespace {

// One step of complex-symmetric Lanczos on X with the bilinear form
// (Sec. 2.1, Freund et al.), full CGS2 re-orthogonalisation in the same form,
// and the three-vector update of diag(Q T Q^T) (Sec. 2.3 after Eq. 9).
// One cluster per frequency; SPLIT CTAs share each subdomain's entries
// (interleaved), so the FP64 work of a frequency spreads over SPLIT * p SMs.
template <int SPLIT>
__global__ void __launch_bounds__(DY_THREADS) k_lanczos(Geo g, Bufs b, int j) {
  cg::cluster_group cl = cg::this_cluster();
  __shared__ RedSmem rs;
  __shared__ cxd hs[KMAX_SMEM];
  const int i = blockIdx.x / SPLIT, part = blockIdx.x - i * SPLIT, kf = blockIdx.y, p = g.p * SPLIT;
  const int e0 = threadIdx.x + part * DY_THREADS;
  constexpr int ES = SPLIT * DY_THREADS;
  int* st = b.st + (size_t)kf * ST_N;
  if (st[ST_DONE]) return;
  int phase = 0;
  const size_t Ndd = g.Ndd;
  const int nsub = g.Lx * g.W, n = own_count(g, i);
  cxd* Q = b.Q + (size_t)kf * (g.k_max + g.nb) * Ndd;
  const cxd* qj = Q + (size_t)j * Ndd;
  const cxd* qm = (j > 0) ? Q + (size_t)(j - 1) * Ndd : nullptr;
  cxd* r = Q + (size_t)(j + 1) * Ndd;
  const cxd* u = b.u + (size_t)kf * Ndd;
  cxd* acc = b.acc + (size_t)kf * Ndd;
  cxd* lan = b.lan + (size_t)kf * (g.k_max + g.nb) * 2;
  const cxd beta_j = (j > 0) ? lan[2 * j + 1] : cxd{0, 0};
  // read before the first cluster barrier: CTA 0 updates it once all CTAs passed the last one
  const double maxT_prev = b.maxT[kf];

  cxd v1[1] = {{0, 0}};
  for (int e = e0; e < n; e += ES) {
    size_t k = own_idx(g, i, e, nsub);
    v1[0] = cfma(qj[k], u[k], v1[0]);
  }
  cluster_sum<1>(cl, rs, phase, p, v1);
  const cxd alpha = v1[0];
  for (int e = e0; e < n; e += ES) {
    size_t k = own_idx(g, i, e, nsub);
    cxd rv = cfma(-alpha, qj[k], u[k]);
    if (qm) rv = cfma(-beta_j, qm[k], rv);
    r[k] = rv;
  }
  for (int pass = 0; pass < 2; ++pass) {
    for (int c0 = 0; c0 <= j; c0 += 8) {
      cxd h8[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) h8[m] = cxd{0, 0};
      for (int e = e0; e < n; e += ES) {
        size_t k = own_idx(g, i, e, nsub);
        cxd rv = r[k];
#pragma unroll
        for (int m = 0; m < 8; ++m)
          if (c0 + m <= j) h8[m] = cfma(Q[(size_t)(c0 + m) * Ndd + k], rv, h8[m]);
      }
      cluster_sum<8>(cl, rs, phase, p, h8);
      if (threadIdx.x < 8 && c0 + threadIdx.x <= j) hs[c0 + threadIdx.x] = h8[threadIdx.x];
    }
    __syncthreads();
    for (int e = e0; e < n; e += ES) {
      size_t k = own_idx(g, i, e, nsub);
      cxd rv = r[k];
      for (int m = 0; m <= j; ++m) rv = cfma(-hs[m], Q[(size_t)m * Ndd + k], rv);   // fused: 4 FP64 ops
      r[k] = rv;
    }
    __syncthreads();
  }
  cxd v2[2] = {{0, 0}, {0, 0}};
  for (int e = e0; e < n; e += ES) {
    size_t k = own_idx(g, i, e, nsub);
    cxd rv = r[k];
    v2[0] = cfma(rv, rv, v2[0]);
    v2[1].x += cabs2(rv);
    cxd a = acc[k] + alpha * (qj[k] * qj[k]);
    if (qm) a = a + (2.0 * beta_j) * (qm[k] * qj[k]);
    acc[k] = a;
  }
  cluster_sum<2>(cl, rs, phase, p, v2);
  const cxd rr = v2[0];
  const cxd beta = csqrt_principal(rr);
  const double maxT = fmax(maxT_prev, sqrt(cabs2(alpha)));
  const double babs = sqrt(cabs2(beta));
  int done = 0, flag = 0;
  if (j == g.k_max - 1) {
    done = 1;
  } else if (sqrt(v2[1].x) <= TERM_TOL * maxT) {      // r vanished: invariant subspace
    done = 1;
    flag = 1;
  } else if (sqrt(cabs2(rr)) <= BRK_TOL * v2[1].x) {   // r != 0, (r, r)_C ~ 0: breakdown
    done = 1;
    flag = 2;
  }
  if (!done) {
    const cxd ib = cinv(beta);
    for (int e = e0; e < n; e += ES) {
      size_t k = own_idx(g, i, e, nsub);
      r[k] = r[k] * ib;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    lan[2 * j] = alpha;
    st[ST_STEPS] = j + 1;
    if (done) {
      st[ST_DONE] = 1;
      st[ST_STATUS] |= flag;
    } else {
      lan[2 * (j + 1) + 1] = beta;
      b.maxT[kf] = fmax(maxT, babs);
    }
  }
  cl.sync();          // no CTA exits while a peer may still read its shared memory
}

// Gather the real start vector into DD layout and normalise it in the
// bilinear form: q_1 = q / sqrt(q^T q).  Clears the per-frequency state.
__global__ void __launch_bounds__(DY_THREADS) k_init(Geo g, Bufs b) {
  cg::cluster_group cl = cg::this_cluster();
  __shared__ RedSmem rs;
  const int i = blockIdx.x, kf = blockIdx.y;
  int phase = 0;
  const int nsub = g.Lx * g.W, n = own_count(g, i);
  cxd* q = b.Q + (size_t)kf * (g.k_max + g.nb) * g.Ndd;
  cxd* acc = b.acc + (size_t)kf * g.Ndd;
  cxd v1[1] = {{0, 0}};
  for (int e = threadIdx.x; e < n; e += DY_THREADS) {
    size_t k = own_idx(g, i, e, nsub);
    int nat = b.dd2nat[k];
    double v = nat >= 0 ? b.q1[nat] : 0.0;
    q[k] = cxd{v, 0};
    acc[k] = cxd{0, 0};
    v1[0].x += v * v;
  }
  cluster_sum<1>(cl, rs, phase, g.p, v1);
  const cxd inv = cinv(csqrt_principal(v1[0]));
  for (int e = threadIdx.x; e < n; e += DY_THREADS) {
    size_t k = own_idx(g, i, e, nsub);
    const cxd v = q[k] * inv;
    if (g.qsplit) reinterpret_cast<cdfl*>(q)[k] = csplit(v);   // basis stored as double-floats
    else q[k] = v;
  }
  if (threadIdx.x == 0 && b.sweeps) b.sweeps[(size_t)kf * g.p + i] = 0;
  if (i == 0 && threadIdx.x == 0) {
    int* st = b.st + (size_t)kf * ST_N;
    for (int k = 0; k < ST_N; ++k) st[k] = 0;
    if (g.p < 2) st[ST_DONE] = 1;        // one subdomain: X = 0, no Lanczos steps
    cxd* lan = b.lan + (size_t)kf * (g.k_max + g.nb) * 2;
    lan[0] = lan[1] = cxd{0, 0};
    b.maxT[kf] = 0.0;
  }
  cl.sync();          // no CTA exits while a peer may still read its shared memory
}

// diag(G) = diag(blkdiag(B^-1, 0)) + diag(Q T Q^T)  (Eq. 9), natural order.
__global__ void k_finalize(Geo g, Bufs b) {
  const int kf = blockIdx.y;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < (size_t)g.Ndd;
       k += (size_t)gridDim.x * blockDim.x) {
    int nat = b.dd2nat[k];
    if (nat < 0) continue;
    size_t o = (size_t)kf * g.Ndd + k;
    b.out[(size_t)kf * g.N + nat] = b.diagB[o] + b.acc[o];
  }
}

__global__ void k_gather(Geo g, const int* dd2nat, const cxd* nat, cxd* dd, size_t ds) {
  const int kf = blockIdx.y;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < (size_t)g.Ndd;
       k += (size_t)gridDim.x * blockDim.x) {
    int n = dd2nat[k];
    dd[(size_t)kf * ds + k] = n >= 0 ? nat[(size_t)kf * g.N + n] : cxd{0, 0};
  }
}

__global__ void k_scatter(Geo g, const int* dd2nat, const cxd* dd, cxd* nat, size_t ds) {
  const int kf = blockIdx.y;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < (size_t)g.Ndd;
       k += (size_t)gridDim.x * blockDim.x) {
    int n = dd2nat[k];
    if (n >= 0) nat[(size_t)kf * g.N + n] = dd[(size_t)kf * ds + k];
  }
}

__global__ void k_status(const int* st, int K, int* status) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x)
    status[k] = st[(size_t)k * ST_N + ST_STATUS];
}

// Failure-detection self-test of the bounded wait every copy ring uses: one
// thread waits on a fresh mbarrier that nothing arrives on (phase 0 never
// completes), so the wait must give up after limit_ns; out[0] receives
// ST_WAIT_TIMEOUT if it did (0 if the phase completed), out[1] the time waited
// in microseconds.  No copy is in flight, so returning early is safe.
__global__ void k_wait_selftest(unsigned long long limit_ns, int* out) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    const unsigned long long t0 = global_ns();
    const bool ok = mbar_wait_for(&bar, 0u, limit_ns);
    const unsigned long long dt = global_ns() - t0;
    out[0] = ok ? 0 : ST_WAIT_TIMEOUT;
    out[1] = (int)(dt / 1000ull > 0x7fffffffull ? 0x7fffffffull : dt / 1000ull);
  }
}

}  // namespace

cudaError_t launch_wait_selftest(unsigned long long limit_ns, int* out, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(limit_ns, out);
  return cudaGetLastError();
}

size_t dyson_internal_sweep_smem(const Geo& g, bool mixed) {
  return mixed ? sweep_smem<float>(g) : sweep_smem<double>(g);
}

void dyson_internal_ring_plan(const Geo& g, bool mixed, int* S, int* CR, int* NT) {
  const RingPlan rp = mixed ? ring_plan<float>(g) : ring_plan<double>(g);
  *S = rp.S;
  *CR = rp.CR;
  *NT = mixed ? xm_threads<float>(g) : xm_threads<double>(g);
}

int dyson_internal_ring_candidates(const Geo& g, bool mixed, int* S, int* CR, int* NT, int max) {
  return mixed ? ring_candidates<float>(g, S, CR, NT, max) : ring_candidates<double>(g, S, CR, NT, max);
}



cudaError_t launch_lanczos(const Geo& g, const Bufs& b, int K, int j, cudaStream_t st) {
  if (g.k_max > KMAX_SMEM) return cudaErrorInvalidValue;
  if (2 * g.p <= 8) return launch_cluster(k_lanczos<2>, dim3(2 * g.p, K), 2 * g.p, 0, st, g, b, j);
  return launch_cluster(k_lanczos<1>, dim3(g.p, K), g.p, 0, st, g, b, j);
}

cudaError_t launch_init(const Geo& g, const Bufs& b, int K, cudaStream_t st) {
  return launch_cluster(k_init, dim3(g.p, K), g.p, 0, st, g, b);
}

static dim3 flat_grid(const Geo& g, int K) {
  int bx = (g.Ndd + DY_THREADS - 1) / DY_THREADS;
  if (bx > 1024) bx = 1024;
  return dim3(bx, K);
}

cudaError_t launch_finalize(const Geo& g, const Bufs& b, int K, cudaStream_t st) {
  k_finalize<<<flat_grid(g, K), DY_THREADS, 0, st>>>(g, b);
  return cudaGetLastError();
}

cudaError_t launch_gather(const Geo& g, const Bufs& b, int K, const cxd* nat, cxd* dd,
                          size_t dd_stride, cudaStream_t st) {
  k_gather<<<flat_grid(g, K), DY_THREADS, 0, st>>>(g, b.dd2nat, nat, dd, dd_stride);
  return cudaGetLastError();
}

cudaError_t launch_scatter(const Geo& g, const Bufs& b, int K, const cxd* dd, cxd* nat,
                           size_t dd_stride, cudaStream_t st) {
  k_scatter<<<flat_grid(g, K), DY_THREADS, 0, st>>>(g, b.dd2nat, dd, nat, dd_stride);
  return cudaGetLastError();
}

// Vector 0 of each frequency's basis, written in binary64 (dyson_xmatvec's
// caller vector), rewritten in place as double-floats when the basis is split.
__global__ void k_qsplit(Geo g, Bufs b) {
  const int kf = blockIdx.y;
  cxd* q = b.Q + (size_t)kf * (g.k_max + g.nb) * g.Ndd;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < (size_t)g.Ndd;
       k += (size_t)gridDim.x * blockDim.x) {
    const cxd v = q[k];
    reinterpret_cast<cdfl*>(q)[k] = csplit(v);
  }
}

cudaError_t launch_qsplit(const Geo& g, const Bufs& b, int K, cudaStream_t st) {
  if (!g.qsplit) return cudaSuccess;
  k_qsplit<<<flat_grid(g, K), DY_THREADS, 0, st>>>(g, b);
  return cudaGetLastError();
}

cudaError_t launch_status(const Geo&, const Bufs& b, int K, int* status, cudaStream_t st) {
  k_status<<<(K + 255) / 256, 256, 0, st>>>(b.st, K, status);
  return cudaGetLastError();
}



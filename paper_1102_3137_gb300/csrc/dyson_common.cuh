// Shared device-side definitions of the GB300 Dyson solver.
//
// Notation follows the low-rank correction method (Sec. 2.2-2.3): H is
// ordered as [B E; E^T C] with p subdomains (strips in 2D, slabs in 3D) cut
// along the slowest axis by p-1 single interface layers.  Inside a subdomain
// the sites are sliced along x; slice s holds the w = T*h sites with that x,
// local index j = tr + T*sl (tr: transverse coordinate, y in 3D, T = 1 in 2D;
// sl: slow coordinate inside the subdomain).  Consecutive slices couple
// through t*I, so every subdomain block B_i is block tridiagonal.
//
// Internal vector layout ("DD layout", per frequency):
//   [subdomain 0: Lx slices x W][subdomain 1] ... [subdomain p-1]
//   [interface layer 0: A = Lx*T sites, index x + Lx*tr] ... [layer p-2]
// W is the slice width padded to the widest subdomain; padded entries are 0.
#pragma once

#include <cstdint>
#include <string>

#include <cuda_runtime.h>
#include "dfl.cuh"

#define DY_MAXP 16          // largest cluster (one CTA per subdomain)
#define DY_THREADS 256      // threads per CTA of every solver kernel
#define DY_WARPS (DY_THREADS / 32)
#define DY_MAXW 320         // widest slice the sweep kernels take (48^3 with p = 8: 288)
#define DY_MAXW_SMEM 64     // widest slice the shared-memory factor kernel takes
#define DY_MAXNB 4          // largest Lanczos block size
#define DY_LPRE_MAXLX 160   // widest interface line of the shared-memory layer preconditioner
#define DY_LPRE_MAXLX_G 1024 // widest interface line of its global-memory form
#define DY_LPRE_MAXW 32     // widest slice it takes
#define DY_FREQ_GROUPS 4    // most frequency groups of a solve by default (parallel graph branches)
#define DY_MAX_GROUPS 8
#define DY_BLOCK_H 1024     // block Lanczos: k_max * nb bound (CGS2 coefficients kept in shared memory)
#define DY_FACTOR_CTAS 304  // persistent grid of the wide-slice factor kernel (2 per SM on 152 SMs)

// per-frequency state words
enum {
  ST_DONE = 0,       // Lanczos finished for this frequency
  ST_STATUS = 1,     // DYSON_ST_* flags
  ST_STEPS = 2,      // Lanczos steps taken
  ST_ITERS = 3,      // interface Krylov iterations, summed over all solves
  ST_SOLVES = 4,     // interface solves performed
  ST_REFINE = 5,     // refinement passes (mixed form)
  ST_N = 8
};

// ---------------------------------------------------------------- complex
template <typename R>
struct alignas(2 * sizeof(R)) cx {
  R x, y;
};
using cxd = cx<double>;
using cxf = cx<float>;

template <typename R>
__host__ __device__ __forceinline__ cx<R> mk(R a, R b) { return cx<R>{a, b}; }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return {a.x + b.x, a.y + b.y}; }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return {a.x - b.x, a.y - b.y}; }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator-(cx<R> a) { return {-a.x, -a.y}; }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return {s * a.x, s * a.y}; }
// acc + a*b with fused multiply-adds
template <typename R>
__host__ __device__ __forceinline__ cx<R> cfma(cx<R> a, cx<R> b, cx<R> acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
template <typename R>
__host__ __device__ __forceinline__ R cabs2(cx<R> a) { return a.x * a.x + a.y * a.y; }
// 1/a = conj(a)/|a|^2
template <typename R>
__host__ __device__ __forceinline__ cx<R> cinv(cx<R> a) {
  R d = a.x * a.x + a.y * a.y;
  return {a.x / d, -a.y / d};
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> cdiv(cx<R> a, cx<R> b) { return a * cinv(b); }
// principal square root: Re >= 0, branch cut on the negative real axis with the
// sign of the imaginary part (+0 or -0) selecting the side.
__host__ __device__ __forceinline__ cxd csqrt_principal(cxd z) {
  double r = sqrt(z.x * z.x + z.y * z.y);
  if (r == 0.0) return {0.0, z.y};
  if (z.x >= 0.0) {
    double s = sqrt(0.5 * (r + z.x));
    return {s, z.y / (2.0 * s)};
  }
  double s = sqrt(0.5 * (r - z.x));
  return {fabs(z.y) / (2.0 * s), copysign(s, z.y)};
}
template <typename R, typename S>
__host__ __device__ __forceinline__ cx<R> cconv(cx<S> a) { return {(R)a.x, (R)a.y}; }

// Precision conversions by integer operations on the IEEE-754 bit patterns.
// The hardware conversions between binary64 and binary32 issue on the FP64
// pipe, which on this part runs at ~1/64 of the FP32 rate (ncu: FP64 pipe 92 %
// busy in the complex64 stencil with hardware conversions).
//   d2f_bits: binary64 -> binary32, round to nearest even; results below the
//             binary32 normal range flush to a signed zero, overflow gives inf,
//             NaN stays NaN.
//   f2d_bits: binary32 -> binary64, exact for normal numbers; binary32
//             subnormals flush to a signed zero.
__device__ __forceinline__ float d2f_bits(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int ed = (int)((hi >> 20) & 0x7ffu);
  const int e = ed - 1023 + 127;
  unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);      // top 23 of the 52 mantissa bits
  const unsigned rest = lo & 0x1fffffffu;                  // the 29 bits dropped
  unsigned out = ((unsigned)e << 23) | m;
  out += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;   // carry may reach inf
  if (e >= 255) out = 0x7f800000u;
  if (e <= 0) out = 0u;
  if (ed == 0x7ff) out = 0x7f800000u | (((hi & 0xfffffu) | lo) ? 0x400000u : 0u);
  return __uint_as_float(sign | out);
}
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u;
  const unsigned ef = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  unsigned hi = sign | ((ef + (1023u - 127u)) << 20) | (m >> 3), lo = m << 29;
  if (ef == 0u) hi = sign, lo = 0u;
  if (ef == 0xffu) hi = sign | 0x7ff00000u | (m >> 3), lo = m << 29;
  return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}
// binary64 -> double-float by integer operations (no binary64 instruction):
// hi takes the leading 24 significant bits (truncated: the exponent rebiased in
// place, then sign, exponent and the top 23 mantissa bits funnel-shifted into
// binary32 position), lo the remaining 29 bits rounded to 23 at the fixed
// exponent of hi's last place (lo = F - B with F, B binary32 numbers of one
// exponent, an exact subtraction); hi + lo holds 47 significant bits, relative
// error at most 2^-47.  Magnitudes below 2^-103 keep only hi (absolute error
// below 2^-126), below 2^-126 give a signed zero; infinities, NaN and
// magnitudes of 2^128 and above are not handled (every input here is a finite
// Lanczos or X-matvec vector entry).
__device__ __forceinline__ dfl d2dfl_bits(double d) {
  const unsigned hw = (unsigned)__double2hiint(d), lw = (unsigned)__double2loint(d);
  const unsigned sign = hw & 0x80000000u;
  const unsigned e11 = (hw >> 20) & 0x7ffu;                       // binary64 biased exponent
  const unsigned hb = (__funnelshift_l(lw, hw - 0x38000000u, 3) & 0x7fffffffu) | sign;
  const unsigned ebits = hb & 0x7f800000u;                        // exponent field of hi
  const unsigned el = ebits - (23u << 23);                        // exponent of hi's last place
  const unsigned m_lo = ((lw & 0x1fffffffu) + 32u) >> 6;          // may reach 2^23: carries into el
  const float lo = __fsub_rn(__uint_as_float((el + m_lo) | sign), __uint_as_float(el | sign));
  return dfl(e11 >= 897u ? __uint_as_float(hb) : 0.f, e11 >= 920u ? lo : 0.f);
}
// double-float -> binary64: both parts widened exactly, one binary64 add
__device__ __forceinline__ double dfl2d_bits(dfl v) { return f2d_bits(v.hi) + f2d_bits(v.lo); }

// A complex number as two double-floats {re.hi, re.lo, im.hi, im.lo}: 16 bytes, the
// size of the binary64 complex it stands for (47 significant bits per part).  The
// mixed form keeps its Lanczos basis in this form, so the Lanczos step's dot
// products and updates read it without splitting.
struct cdfl {
  dfl x, y;
};
__device__ __forceinline__ cdfl csplit(cxd a) { return {d2dfl_bits(a.x), d2dfl_bits(a.y)}; }
__device__ __forceinline__ cxd cwiden(const cdfl& a) { return {dfl2d_bits(a.x), dfl2d_bits(a.y)}; }

__device__ __forceinline__ cxf c2f_bits(cxd a) { return {d2f_bits(a.x), d2f_bits(a.y)}; }
__device__ __forceinline__ cxd c2d_bits(cxf a) { return {f2d_bits(a.x), f2d_bits(a.y)}; }

// ---------------------------------------------------------------- geometry
struct Geo {
  int dim;        // 2 or 3
  int Lx, Ly, Lz; // lattice extents (Lz = 1 in 2D); x fastest
  int N;          // sites
  int p;          // subdomains
  int T;          // transverse count per slice row (1 in 2D, Ly in 3D)
  int A;          // sites per slow layer = Lx*T
  int Ls;         // slow extent (Ly in 2D, Lz in 3D)
  int W;          // padded slice width
  int Ndd;        // DD-layout vector length
  int ifc_off;    // start of the interface part = p*Lx*W
  int k_max;      // Lanczos rank cap
  int krylov_maxit;
  int refine_max; // mixed form: most refinement passes per solve
  double t, mu;
  double krylov_tol;   // relative residual target of an interface solve
  double refine_tol;   // mixed form: relative residual target after refinement
  int h[DY_MAXP];      // subdomain heights along the slow axis
  int s0[DY_MAXP];     // subdomain start along the slow axis
  int ylayer[DY_MAXP]; // slow coordinate of interface layer l
  int penta;           // interface preconditioner keeps the distance-2 coupling (2D strips, W <= 64)
  double eta;          // 0: Matsubara axis; > 0: real axis w + i eta
  int real_axis;       // eta > 0 (an integer test on the device)
  int ring_S;          // copy-ring slots chosen by the autotuner (0: shared-memory heuristic)
  int ring_CR;         // rows per streamed chunk chosen by the autotuner (W > 64; 0: heuristic)
  int nb;              // Lanczos block size (1: the scalar recurrence of Sec. 2.1)
  int lpre;            // interface preconditioner: 1 exact layer blocks of S (2D strips), 0 banded
  int xm_nt;           // threads per X-matvec CTA in the complex64 two-chain form (128: four CTAs
                       // per SM; 0 or 256: two), chosen by the heuristic or the autotuner
  int qsplit;          // the Lanczos basis is stored as double-floats (cdfl; mixed form, nb = 1,
                       // k_max <= 64, where the double-float Lanczos step runs)
};

// Work slots: the X-matvec runs one cluster per (frequency f, block column c),
// slot vs = f * nb + c; factors and per-frequency state are indexed by f.
__host__ __device__ __forceinline__ int slot_freq(const Geo& g, int vs) { return g.nb > 1 ? vs / g.nb : vs; }

// Device buffers of one plan; every per-frequency array is [K_cap][...],
// every per-slot array [K_cap * nb][...].
struct Bufs {
  const double* V;      // [N] trap/local potential, natural order
  const double* omega;  // [K] Matsubara frequencies
  const cxd* sigma;     // [K][N] self-energy, natural order
  const double* q1;     // [nb][N] real Lanczos start vector(s)
  const int* dd2nat;    // [Ndd] natural index of each DD slot, -1 on padding
  void* g;              // [K][p][Lx][W][W] slice factors g_s read by the sweeps (precision of the form)
  cxd* g64;             // [K][p][Lx][W][W] FP64 g_s kept for the mixed form's FP64 recursion
  cxd* diagB;           // [K][Ndd] diag(B^-1), zero on the interface
  cxd* hdiag;           // [K][Ndd] H_ii (Eq. 1) in DD layout, zero on padding (mixed form), or null
  cxd* offB;            // [K][p][Lx][W] diag of G_{s,s+1} (B_i^-1 between slices s, s+1), or null
  cxd* off2;            // [K][p][Lx][W] diag of G_{s,s+2} on the boundary rows (2D strips), or null
  cxd* Q;               // [K][k_max+nb][Ndd] Lanczos vectors (column j*nb + c of block j)
  cxd* acc;             // [K][Ndd] running diag(Q T Q^T)
  cxd* u;               // [K*nb][Ndd] X q, per slot
  cxd* v1;              // [K*nb][Ndd] work vectors of the mixed form, per slot
  cxd* v2;
  cxd* v3;
  void* yscr;           // [K*nb][p][Lx][W] forward-sweep intermediates (precision of the form)
  cxd* bnd;             // [K*nb][p][2][A] sweep values on the subdomain boundary rows
  cxd* ifv;             // [K*nb][IF_N][(p-1)*A] interface Krylov vectors
  cxd* pre;             // [K][p-1][3][A] tridiagonal preconditioner factors
  cxd* lan;             // nb = 1: [K][k_max+1][2] (alpha_j, beta_j), beta_j couples q_{j-1}, q_j;
                        // nb > 1: [K][k_max/nb+1][2][nb][nb] (A_j, B_j), B_j couples blocks j-1, j
  double* maxT;         // [K] running max |T| entry
  int* st;              // [K][ST_N]
  cxd* out;             // [K][N] diag(G), natural order
  unsigned long long* sweeps;  // [K*nb][p] subdomain sweeps performed (work accounting)
  cxd* fwork;           // [DY_FACTOR_CTAS][2][W][W] wide-slice factor workspace (W > 64 only)
  cx<float>* lpt;       // [K][p][2][Lx][Lx] boundary-row surface Green's functions (lpre)
  cx<float>* lpg;       // [K][p][Lx][W][W] complex64 slice factors of that recursion (lpre scratch)
  void* lpm;            // [K][p-1][Lx][Lx] inverse layer blocks of S, precision of the form (lpre)
  cx<float>* lpv;       // [K][p][2][Lx][W] boundary columns of the surface recursion (lpre, Lx > 160)
  cx<float>* lpw;       // [DY_FACTOR_CTAS][2][W][2 Lx T] boundary-column chains of the 3D slab
                        // surface recursion (lpre with T > 1), not per frequency
  cxd* gram;            // [K][k_max+1][k_max+1] Gram matrix q_l^T q_m of the stored basis, entry
                        // (l, m) at m (k_max+1) + l for l < m (double-float Lanczos step), or null
};

// interface Krylov vector slots inside ifv
enum { IF_X = 0, IF_R = 1, IF_Z = 2, IF_P = 3, IF_SP = 4, IF_B = 5, IF_D = 6, IF_N = 7 };

__host__ __device__ __forceinline__ size_t nifc(const Geo& g) { return (size_t)(g.p > 1 ? g.p - 1 : 1) * g.A; }

// H_ii(i w) = i w + mu - V_i - Sigma_i(i w)   (Eq. 1); on the real axis
// (eta > 0) i w -> w + i eta
__device__ __forceinline__ cxd dyson_diag(const Geo& g, const Bufs& b, int kf, int nat) {
  cxd s = b.sigma[(size_t)kf * g.N + nat];
  const double w = b.omega[kf];
  return g.real_axis ? cxd{w + g.mu - b.V[nat] - s.x, g.eta - s.y}
                     : cxd{g.mu - b.V[nat] - s.x, w - s.y};
}

// natural index of row j of slice s in subdomain i
__device__ __forceinline__ int sub_nat(const Geo& g, int i, int s, int j) {
  int tr = j % g.T, sl = j / g.T;
  return s + g.Lx * tr + g.A * (g.s0[i] + sl);
}

// ---------------------------------------------------------------- host helpers
// Raise (never lower) a kernel's dynamic shared-memory limit to at least
// `bytes`.  Plans of different sizes share the kernels, and a graph captured
// for a large plan may be replayed after a small plan ran, so the limit only grows.
cudaError_t raise_smem_limit(const void* func, size_t bytes);

// Record msg as this thread's dyson_last_error() and return code.
int dyson_internal_fail(int code, const std::string& msg);
struct dyson_plan_s;
// dyson_solve without the final wait (all copies and the graph launch enqueued on stream)
int dyson_internal_solve_enqueue(dyson_plan_s* p, int K, const double* omega, const double* V,
                                 const double* sigma, const double* q1, double* diagG, int* status,
                                 int mem_kind, void* stream);
size_t dyson_internal_plan_bytes(dyson_plan_s* p);
// Dynamic shared memory of the sweep-based solver kernels for this geometry in
// the given form; 0 when the slice width and x extent do not fit on chip.
size_t dyson_internal_sweep_smem(const Geo& g, bool mixed);
// Copy-ring configurations the autotuner times for this geometry and form:
// up to max pairs (slots, chunk rows), the shared-memory heuristic's first.
int dyson_internal_ring_candidates(const Geo& g, bool mixed, int* S, int* CR, int* NT, int max);
// The copy-ring configuration the kernels use for this geometry (slots, chunk rows).
void dyson_internal_ring_plan(const Geo& g, bool mixed, int* S, int* CR, int* NT);

// ---------------------------------------------------------------- host launchers
template <typename R, typename S>
cudaError_t launch_factor(const Geo& g, const Bufs& b, int K, cudaStream_t st);
template <typename R>
cudaError_t launch_precond(const Geo& g, const Bufs& b, int K, cudaStream_t st);
cudaError_t launch_init(const Geo& g, const Bufs& b, int K, cudaStream_t st);
template <typename R>
cudaError_t launch_xmatvec(const Geo& g, const Bufs& b, int K, int j, int mixed, int ncols, cudaStream_t st);
cudaError_t launch_lanczos(const Geo& g, const Bufs& b, int K, int j, cudaStream_t st);
cudaError_t launch_block_lanczos(const Geo& g, const Bufs& b, int K, int j, cudaStream_t st);
cudaError_t launch_init_block(const Geo& g, const Bufs& b, int K, cudaStream_t st);
cudaError_t launch_surface(const Geo& g, const Bufs& b, int K, cudaStream_t st);
template <typename R>
cudaError_t launch_layer_inv(const Geo& g, const Bufs& b, int K, cudaStream_t st);
size_t dyson_internal_surface_smem(const Geo& g);
size_t dyson_internal_layer_inv_smem(const Geo& g);
cudaError_t launch_finalize(const Geo& g, const Bufs& b, int K, cudaStream_t st);
template <typename R>
cudaError_t launch_spmv(const Geo& g, const double* V, const double* omega, const cxd* sigma,
                        const cx<R>* x, cx<R>* y, int K, cudaStream_t st);
template <typename R>
cudaError_t launch_bsolve(const Geo& g, const Bufs& b, int K, const cxd* q_dd, cxd* w_dd,
                          cudaStream_t st);
// the X-matvec and subdomain-solve launchers exist for complex64 (k_xmatvec_c64.cu)
// and complex128 (k_xmatvec_c128.cu)
template <>
cudaError_t launch_xmatvec<float>(const Geo& g, const Bufs& b, int K, int j, int mixed, int ncols, cudaStream_t st);
template <>
cudaError_t launch_xmatvec<double>(const Geo& g, const Bufs& b, int K, int j, int mixed, int ncols, cudaStream_t st);
template <>
cudaError_t launch_bsolve<float>(const Geo& g, const Bufs& b, int K, const cxd* q_dd, cxd* w_dd,
                                 cudaStream_t st);
template <>
cudaError_t launch_bsolve<double>(const Geo& g, const Bufs& b, int K, const cxd* q_dd, cxd* w_dd,
                                  cudaStream_t st);
cudaError_t launch_gather(const Geo& g, const Bufs& b, int K, const cxd* nat, cxd* dd,
                          size_t dd_stride, cudaStream_t st);
cudaError_t launch_scatter(const Geo& g, const Bufs& b, int K, const cxd* dd, cxd* nat,
                           size_t dd_stride, cudaStream_t st);
cudaError_t launch_qsplit(const Geo& g, const Bufs& b, int K, cudaStream_t st);
cudaError_t launch_status(const Geo& g, const Bufs& b, int K, int* status, cudaStream_t st);
cudaError_t launch_wait_selftest(unsigned long long limit_ns, int* out, cudaStream_t st);
cudaError_t launch_lanczos_dd(const Geo& g, const Bufs& b, int K, int j, cudaStream_t st);

// Complex64 32 x 32 x 32 block products on the tensor cores, at binary32
// accuracy, for the dense parts of the exact layer preconditioner.
//
// Precision: every binary32 operand x is split into two TF32 numbers,
// x = hi + lo with hi = tf32(x) and lo = tf32(x - hi), and a real product is
// taken as hi*hi + hi*lo + lo*hi with binary32 accumulation (the lo*lo term is
// below binary32 resolution): the 3xTF32 scheme of Ootomo and Yokota,
// "Recovering single precision accuracy from Tensor Cores while surpassing the
// FP32 theoretical peak performance" (2022).  A complex product takes four real
// products (Re = Xr Yr - Xi Yi, Im = Xr Yi + Xi Yr), twelve TF32 MMAs per
// k-step.
//
// Instruction: mma.sync m16n8k8 with TF32 inputs and FP32 accumulators.  Its
// fragments (PTX ISA, matrix fragments of mma.m16n8k8 for .tf32), with
// g = lane / 4 and c = lane % 4:
//   A (16 x 8, row):  a0 (g, c)    a1 (g + 8, c)    a2 (g, c + 4)    a3 (g + 8, c + 4)
//   B (8 x 8, col):   b0 (c, g)    b1 (c + 4, g)                        (row = k, col = n)
//   D (16 x 8):       d0 (g, 2c)   d1 (g, 2c + 1)   d2 (g + 8, 2c)   d3 (g + 8, 2c + 1)
// A 32 x 32 complex output is 2 x 4 tiles of 16 x 8; the 8 warps of a CTA
// take one tile each (warp w: rows 16 (w / 4) .., columns 8 (w % 4) ..).
#pragma once

#include <cstdint>

#include "dyson_common.cuh"

namespace tc {

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// x = hi + lo, both TF32
__device__ __forceinline__ void split(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// d += a b with a = ah + al, b = bh + bl (3xTF32)
__device__ __forceinline__ void mma3(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                     const uint32_t (&bh)[2], const uint32_t (&bl)[2]) {
  mma_tf32(d, al, bh);
  mma_tf32(d, ah, bl);
  mma_tf32(d, ah, bh);
}

// Accumulators of one warp's 16 x 8 complex tile: re[4], im[4] in the D layout.
struct CTile {
  float re[4], im[4];
};

// acc += X(rows m0.., all k) * Y(all k, cols n0..) for 32 x 32 complex64
// matrices in shared memory (row-major, row stride ld, interleaved re/im).
__device__ __forceinline__ void cgemm_tile_3xtf32(CTile& acc, const cx<float>* X, const cx<float>* Y, int ld,
                                                  int m0, int n0) {
  const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
#pragma unroll
  for (int k0 = 0; k0 < 32; k0 += 8) {
    uint32_t arh[4], arl[4], aih[4], ail[4], ainh[4], ainl[4];
    const int ra[4] = {m0 + g, m0 + g + 8, m0 + g, m0 + g + 8};
    const int ka[4] = {k0 + c, k0 + c, k0 + c + 4, k0 + c + 4};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const cx<float> v = X[ra[e] * ld + ka[e]];
      split(v.x, arh[e], arl[e]);
      split(v.y, aih[e], ail[e]);
      split(-v.y, ainh[e], ainl[e]);
    }
    uint32_t brh[2], brl[2], bih[2], bil[2];
    const int kb[2] = {k0 + c, k0 + c + 4};
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const cx<float> v = Y[kb[e] * ld + n0 + g];
      split(v.x, brh[e], brl[e]);
      split(v.y, bih[e], bil[e]);
    }
    mma3(acc.re, arh, arl, brh, brl);     // + Xr Yr
    mma3(acc.re, ainh, ainl, bih, bil);   // - Xi Yi
    mma3(acc.im, arh, arl, bih, bil);     // + Xr Yi
    mma3(acc.im, aih, ail, brh, brl);     // + Xi Yr
  }
}

// Element (row, col) of the tile held in accumulator slot e of this lane.
__device__ __forceinline__ void tile_pos(int e, int m0, int n0, int& row, int& col) {
  const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
  row = m0 + g + ((e & 2) ? 8 : 0);
  col = n0 + 2 * c + (e & 1);
}

}  // namespace tc

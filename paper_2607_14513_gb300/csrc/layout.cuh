// layout.cuh -- where each Gaussian's coefficients sit in a group's 16 blocks (Sec. IV-B).
//
// A group is 16 slots and 16 blocks of 4x4 texels (texel t in raster order) in every layout:
//  D (Fig. SetupD): block k, texel t = coefficient k of slot t;
//  A (Fig. SetupA): block k, texel t = coefficient t of slot k (one Gaussian per block);
//  B (Fig. SetupB): quads of 4 slots and 4 blocks; block b of quad v (k = 4v + b), row i,
//    column j = coefficient 4b + j of slot 4v + i.
// A fixed coding with j BC7 blocks per group makes BC7: D the first j blocks (the rate streams
// keep this rule), A all or none, B the first j / 4 blocks of every quad; a group's bytes are its
// BC7 blocks in block order, then its BC1 blocks in block order.
#pragma once
#include "gsc_internal.cuh"

// slot u, coefficient c -> block k, texel t
__host__ __device__ __forceinline__ void lay_inv(int layout, int u, int c, int& k, int& t) {
  if (layout == GSC_LAYOUT_A) { k = u; t = c; }
  else if (layout == GSC_LAYOUT_B) { k = (u & ~3) | (c >> 2); t = ((u & 3) << 2) | (c & 3); }
  else { k = c; t = u; }
}

__host__ __device__ __forceinline__ bool lay_bc7(int layout, int j, int k) {
  if (layout == GSC_LAYOUT_A) return j == 16;
  if (layout == GSC_LAYOUT_B) return (k & 3) < (j >> 2);
  return k < j;
}

// position of block k among the group's blocks of its own format (BC7 or BC1)
__host__ __device__ __forceinline__ int lay_rank(int layout, int j, int k) {
  if (layout == GSC_LAYOUT_B) {
    const int q = j >> 2, b = k & 3, v = k >> 2;
    return b < q ? v * q + b : v * (4 - q) + (b - q);
  }
  if (layout == GSC_LAYOUT_A) return k;
  return k < j ? k : k - j;
}

__host__ __device__ __forceinline__ bool lay_ok(int layout, int j) {
  if (layout == GSC_LAYOUT_D) return j >= 0 && j <= 16;
  if (layout == GSC_LAYOUT_A) return j == 0 || j == 16;
  if (layout == GSC_LAYOUT_B) return j >= 0 && j <= 16 && (j & 3) == 0;
  return false;
}

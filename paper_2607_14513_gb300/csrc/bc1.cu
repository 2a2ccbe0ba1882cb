// bc1.cu -- BC1 encoder (Sec. III-A with P = 16, Q = 2 on 4x4 blocks; Sec. III-B).
//
// One thread per block: every lane of a warp runs the same deterministic integer
// search on its own block, so control flow stays uniform except for the data-dependent
// early exits. Texels live in registers (packed RGB in a u32).
//
// Search (the codec's own encoder; ties go to the lowest index, candidates in a fixed order):
//  constant block: per channel the code pair whose two-thirds point is nearest (table);
//  otherwise: bounding-box diagonal oriented by covariance signs, inset by range/16,
//  565 quantisation; two least-squares refinements on the current indices; then up to
//  four rounds of the best strictly improving +-1 step on the six endpoint channels.
//  Every candidate is scored with the four-colour palette of the GB300 texture unit.
#include "bc1_dev.cuh"


static int h_ex5(int x) { return (x << 3) | (x >> 2); }
static int h_ex6(int x) { return (x << 2) | (x >> 4); }
static int h_third(int a, int b, int bits) {
  if (bits == 5) return ((2 * a + b) * 11) >> 2;
  int A = h_ex6(a), B = h_ex6(b);
  int num = (B - A) * 321 + 512;
  return A + (num >= 0 ? num / 1024 : -((-num + 1023) / 1024));
}

void bc1_const_tables(uint16_t* t5, uint16_t* t6) {
  for (int v = 0; v < 256; v++) {
    for (int bits = 5; bits <= 6; bits++) {
      int lim = 1 << bits, be = -1, ba = 0, bb = 0;
      for (int a = 0; a < lim; a++)
        for (int b = 0; b < lim; b++) {
          int e = abs(h_third(a, b, bits) - v);
          if (be < 0 || e < be) { be = e; ba = a; bb = b; }
        }
      (bits == 5 ? t5 : t6)[v] = (uint16_t)(ba | (bb << 8));
    }
  }
}

cudaError_t bc1_init_tables() {
  uint16_t t5[256], t6[256];
  bc1_const_tables(t5, t6);
  (void)h_ex5;
  cudaError_t e = cudaMemcpyToSymbol(c_const5, t5, sizeof(t5));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_const6, t6, sizeof(t6));
}

__global__ void __launch_bounds__(STAGE_THREADS) k_bc1_groups(const float* __restrict__ sh,
                                                              const int32_t* __restrict__ perm,
                                                              const float* __restrict__ scales, int64_t n_groups,
                                                              uint2* __restrict__ blocks, uint32_t* __restrict__ sse1,
                                                              uint32_t* __restrict__ sse0) {
  __shared__ uint32_t tex[16][STAGE_STRIDE];
  __shared__ float s_scale[16];
  if (threadIdx.x < 16) s_scale[threadIdx.x] = scales[threadIdx.x];
  __syncthreads();
  for (int64_t g0 = (int64_t)blockIdx.x * STAGE_GROUPS; g0 < n_groups; g0 += (int64_t)gridDim.x * STAGE_GROUPS) {
    stage_groups(sh, perm, s_scale, g0, n_groups, tex, threadIdx.x);
    __syncthreads();
    const int64_t blk = g0 * 16 + threadIdx.x;
    if (blk < n_groups * 16) {
      uint32_t tx[16];
#pragma unroll
      for (int t = 0; t < 16; t++) tx[t] = tex[t][threadIdx.x];
      Bc1Res r = bc1_encode(tx);
      blocks[blk] = bc1_bits(r);
      if (sse1) sse1[blk] = r.sse;
      if (sse0) sse0[blk] = sse_zero(tx);
    }
    __syncthreads();
  }
}

__global__ void k_bc1_blocks(const uint8_t* __restrict__ texin, int64_t nblk, uint2* __restrict__ out,
                             uint64_t* __restrict__ sse) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t* p = texin + b * 48;
    uint32_t tx[16];
#pragma unroll
    for (int t = 0; t < 16; t++) tx[t] = (uint32_t)p[3 * t] | ((uint32_t)p[3 * t + 1] << 8) | ((uint32_t)p[3 * t + 2] << 16);
    Bc1Res r = bc1_encode(tx);
    out[b] = bc1_bits(r);
    if (sse) sse[b] = r.sse;
  }
}

static int grid_for(int64_t work, int per_cta) {
  int64_t g = ceil_div64(work, per_cta);
  if (g > gsc_sm_count() * 64) g = gsc_sm_count() * 64;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_bc1_groups(const float* sh, const int32_t* perm, const float* scales, int64_t n_groups,
                              uint8_t* blocks, uint32_t* sse1, uint32_t* sse0, cudaStream_t st) {
  if (n_groups <= 0) return cudaSuccess;
  gsc_count_launch(); k_bc1_groups<<<grid_for(n_groups, STAGE_GROUPS), STAGE_THREADS, 0, st>>>(sh, perm, scales, n_groups,
                                                                         reinterpret_cast<uint2*>(blocks), sse1, sse0);
  return cudaGetLastError();
}

cudaError_t launch_bc1_blocks(const uint8_t* tex, int64_t nblk, uint8_t* out, uint64_t* sse, cudaStream_t st) {
  if (nblk <= 0) return cudaSuccess;
  gsc_count_launch(); k_bc1_blocks<<<grid_for(nblk, 128), 128, 0, st>>>(tex, nblk, reinterpret_cast<uint2*>(out), sse);
  return cudaGetLastError();
}

// layout.cu -- fixed codings of any block layout (Sec. IV-B, Figs. SetupA / SetupB / SetupD;
// Table I's BC1, BC7 and "BC7 on the first block(s), BC1 on the rest" rows).
//
// Three steps on the caller's stream: one thread per slot quantises its Gaussian (Sec. V-A)
// and scatters the 16 texels to their blocks, BC7 blocks and BC1 blocks into two dense texel
// arrays in output order; the block encoders code each array (the same search as every other
// coding); an interleave writes every group's BC7 blocks then its BC1 blocks. A coding with
// one format writes the encoder's output in place and skips the interleave.
#include "gsc_internal.cuh"
#include "layout.cuh"

namespace {

__global__ void k_stage_layout(const float* __restrict__ sh, const int32_t* __restrict__ perm,
                               const float* __restrict__ scales, int64_t n_groups, int layout, int j,
                               uint8_t* __restrict__ tex7, uint8_t* __restrict__ tex1) {
  __shared__ float s_scale[16];
  if (threadIdx.x < 16) s_scale[threadIdx.x] = scales[threadIdx.x];
  __syncthreads();
  const int64_t ns = n_groups * 16;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = s >> 4;
    const int u = (int)(s & 15);
    // a padding slot repeats the last valid slot before it in its group (none: texel 128)
    int32_t src = __ldg(perm + s);
    for (int v = u - 1; src < 0 && v >= 0; v--) src = __ldg(perm + g * 16 + v);
    float x[48];
    if (src >= 0) {
      const float4* p = reinterpret_cast<const float4*>(sh + (int64_t)src * 48);
#pragma unroll
      for (int i = 0; i < 12; i++) {
        const float4 f = __ldg(p + i);
        x[4 * i] = f.x; x[4 * i + 1] = f.y; x[4 * i + 2] = f.z; x[4 * i + 3] = f.w;
      }
    }
#pragma unroll
    for (int c = 0; c < 16; c++) {
      int k, t;
      lay_inv(layout, u, c, k, t);
      const bool b7 = lay_bc7(layout, j, k);
      const int r = lay_rank(layout, j, k);
      uint8_t* d = b7 ? tex7 + ((g * j + r) * 16 + t) * 3 : tex1 + ((g * (16 - j) + r) * 16 + t) * 3;
      const float sk = s_scale[c];
      d[0] = src >= 0 ? (uint8_t)gsc_quant1(x[3 * c], sk) : 128;
      d[1] = src >= 0 ? (uint8_t)gsc_quant1(x[3 * c + 1], sk) : 128;
      d[2] = src >= 0 ? (uint8_t)gsc_quant1(x[3 * c + 2], sk) : 128;
    }
  }
}

// group g's 16 + j 8-byte words: 2j from its BC7 blocks, then 16 - j from its BC1 blocks
__global__ void k_interleave(const uint2* __restrict__ lin7, const uint2* __restrict__ lin1, int64_t n_groups, int j,
                             uint2* __restrict__ out) {
  const int64_t words = 16 + j, total = n_groups * words;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = w / words;
    const int i = (int)(w - g * words);
    out[w] = i < 2 * j ? __ldg(lin7 + g * 2 * j + i) : __ldg(lin1 + g * (16 - j) + (i - 2 * j));
  }
}

int grid_of(int64_t work) {
  int64_t g = ceil_div64(work, 256);
  if (g > gsc_sm_count() * 16) g = gsc_sm_count() * 16;
  return (int)(g < 1 ? 1 : g);
}

struct LayoutWs {
  uint8_t *tex7, *tex1, *lin7, *lin1;
};

LayoutWs carve_layout(void* ws, size_t cap, int64_t ng, int j, bool* ok) {
  Carve cv{reinterpret_cast<uint8_t*>(ws), 0, cap};
  LayoutWs L;
  L.tex7 = cv.take<uint8_t>(ng * j * 48);
  L.tex1 = cv.take<uint8_t>(ng * (16 - j) * 48);
  const bool mixed = j > 0 && j < 16;
  L.lin7 = mixed ? cv.take<uint8_t>(ng * j * 16) : nullptr;
  L.lin1 = mixed ? cv.take<uint8_t>(ng * (16 - j) * 8) : nullptr;
  *ok = cv.ok();
  return L;
}

}  // namespace

size_t layout_ws_bytes(int64_t n_groups, int j) {
  size_t b = 0;
  auto add = [&](int64_t bytes) { b = align_up(b, 256) + (size_t)(bytes > 0 ? bytes : 1); };
  add(n_groups * j * 48);
  add(n_groups * (16 - j) * 48);
  if (j > 0 && j < 16) {
    add(n_groups * j * 16);
    add(n_groups * (16 - j) * 8);
  }
  return align_up(b, 256);
}

gsc_status layout_encode_run(gsc_ctx* c, const float* sh, int64_t n, const int32_t* perm, const float* scales,
                             int layout, int j, uint8_t* blocks, void* ws, size_t ws_bytes, cudaStream_t st) {
  const int64_t ng = ceil_div64(n, 16);
  if (ng == 0) return GSC_OK;
  bool ok = false;
  const LayoutWs L = carve_layout(ws, ws_bytes, ng, j, &ok);
  if (!ws || !ok) return GSC_ERR_OOM;
  gsc_count_launch();
  k_stage_layout<<<grid_of(ng * 16), 256, 0, st>>>(sh, perm, scales, ng, layout, j, L.tex7, L.tex1);
  GSC_CUDA(cudaGetLastError());
  if (j > 0) {
    GscTimed tm(c, T_BC7, st);
    GSC_CUDA(launch_bc7_blocks(L.tex7, ng * j, j == 16 ? blocks : L.lin7, nullptr, st));
  }
  if (j < 16) {
    GscTimed tm(c, T_BC1, st);
    GSC_CUDA(launch_bc1_blocks(L.tex1, ng * (16 - j), j == 0 ? blocks : L.lin1, nullptr, st));
  }
  if (j > 0 && j < 16) {
    gsc_count_launch();
    k_interleave<<<grid_of(ng * (16 + j)), 256, 0, st>>>(reinterpret_cast<const uint2*>(L.lin7),
                                                          reinterpret_cast<const uint2*>(L.lin1), ng, j,
                                                          reinterpret_cast<uint2*>(blocks));
    GSC_CUDA(cudaGetLastError());
  }
  return GSC_OK;
}

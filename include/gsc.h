/*
 * gsc.h -- C ABI of the GB300 block-texture codec for 3DGS spherical-harmonic colour
 * (Said & Rauwendaal, "Compression of 3D Gaussian Splatting Data Using GPU-friendly
 * Graphics Texture Coding").
 *
 * Problem statement (Sec. II and Sec. V-A): a scene holds n Gaussians with centres
 * p in R^3 and opacity-premultiplied SH colour coefficients H~ = mu H (Eq. premult),
 * 16 RGB coefficients each (k = l*l + l + m, degree 3). The codec quantises H~ to
 * 8-bit texels, reorders the Gaussians by colour inside spatial groups (Sec. III-C),
 * packs coefficient k of 16 Gaussians into one 4x4 block (Sec. IV-B, Fig. SetupD; or one
 * Gaussian per block, Fig. SetupA, or four Gaussians in four blocks, Fig. SetupB),
 * codes every block with BC1 (8 bytes) or BC7 (16 bytes) (Sec. III-B), optionally
 * spreading groups over several fixed-rate streams (Sec. IV-B), and decodes the
 * blocks back, evaluating the view-dependent colour c(f) = H w(f - p) (Sec. II).
 *
 * Conventions for every call:
 *  - Pointers named d_* are device pointers on the context's device; h_* are host
 *    pointers. The caller owns every buffer and the stream; the library owns only the
 *    context. Scratch memory is passed in as d_ws / ws_bytes (size from
 *    gsc_workspace_bytes); the library allocates no device memory on these paths,
 *    except the texture path (gsc_decode_tex, gsc_decode_blocks_tex), which builds CUDA
 *    arrays for texture objects.
 *  - stream is a cudaStream_t (NULL = legacy default stream). Calls are asynchronous
 *    on that stream unless stated otherwise.
 *  - Argument errors are returned synchronously and nothing is launched. Errors the
 *    device detects are recorded in the context and returned by gsc_ctx_sync.
 *  - Arrays are C-contiguous: float positions [n][3]; float SH [n][16][3] with the
 *    RGB triple innermost; texels uint8 [n][16][3]; perm int32 [n_groups * 16].
 *  - There is no CPU fallback: without a usable GB300 every call returns
 *    GSC_ERR_UNSUPPORTED (except the host-only calls: gsc_server_simulate and the
 *    checkpoint file calls on host buffers).
 *  - A context serves one host thread at a time (it holds a pinned staging buffer and the
 *    kernel timers); use one context per thread, as the request loop does per worker. The
 *    request loop's own calls (gsc_server_*) may be made from any thread.
 *  - Beyond the texture path, the batched form, the request loop and the allocation-free plan
 *    allocate what their calls say (graphs, a memory pool, a static array).
 */
#ifndef GSC_H
#define GSC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GSC_OK = 0,
  GSC_ERR_INVALID_ARG = 1, /* bad pointer, size, alignment or parameter */
  GSC_ERR_CUDA = 2,        /* a CUDA runtime call failed */
  GSC_ERR_OOM = 3,         /* workspace too small */
  GSC_ERR_BUDGET = 4,      /* rate target below the cheapest coding of the scene */
  GSC_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  GSC_ERR_UNSUPPORTED = 6, /* no usable sm_103 device, or a feature the device lacks */
  GSC_ERR_DEVICE = 7,      /* an index check inside a kernel failed (record in the context) */
  GSC_ERR_CANCELLED = 8    /* a queued request of the request loop was cancelled */
} gsc_status;

/* GSC_FMT_MIXED: a fixed number of BC7 blocks per group (gsc_encode_params.bc7_blocks), the
 * rest BC1 (Table I's "BC7 on the first block(s), BC1 on the rest" rows). */
typedef enum { GSC_FMT_RATE = 0, GSC_FMT_BC1 = 1, GSC_FMT_MIXED = 2, GSC_FMT_BC7 = 7 } gsc_format;

/* Block layouts (Sec. IV-B). A group is 16 slots (16g..16g+15) and 16 blocks of 4x4 texels
 * (texel t in raster order) in every layout:
 *  D (Fig. SetupD): block k holds coefficient k of the 16 Gaussians, texel t = slot 16g + t.
 *  A (Fig. SetupA): block k holds the 16 coefficients of slot 16g + k, texel t = coefficient t.
 *  B (Fig. SetupB): quads of 4 slots and 4 blocks; block b of quad v (k = 4v + b), row i,
 *    column j holds coefficient 4b + j of slot 16g + 4v + i (block 0 of a quad carries the
 *    first four coefficients of its Gaussians). */
typedef enum { GSC_LAYOUT_D = 0, GSC_LAYOUT_A = 1, GSC_LAYOUT_B = 2 } gsc_layout;

typedef enum {
  GSC_OUT_VIEW_MAJOR = 0,  /* rgb [V][n][3], original Gaussian order (through the inverse permutation) */
  GSC_OUT_SLOT_ORDER = 1,  /* rgb [V][n_groups*16][3], slot order, padding slots written as 0 */
  GSC_OUT_GAUSS_MAJOR = 2, /* rgb [n][V][3], original Gaussian order */
  GSC_OUT_SLOT_ROWS = 3    /* rgb [n_groups*16][V][3], slot order (the order the coded scene keeps its
                              Gaussians in: Sec. III-C reorders them with their coefficients), one
                              row per Gaussian, padding rows written as 0; direct calls and the
                              batched graph only (the request loop takes orders 0-2) */
} gsc_out_order;

typedef struct gsc_ctx gsc_ctx;

/* Reorder and scale parameters (Sec. III-C, Sec. V-A). */
typedef struct {
  int64_t n;                  /* number of Gaussians, 0 <= n < 2^31 - 16 */
  int64_t group_size;         /* spatial chunk G for the colour sort; multiple of 16; 0 = whole scene */
  int32_t sort;               /* 0: keep the original order; 1: colour sort inside spatial chunks */
  uint32_t quantile_permille; /* coverage of [-0.5, 0.5] after scaling, 1..1000 (paper: 995) */
} gsc_plan_params;

/* Coding parameters (Sec. III-B, Sec. IV-B). */
typedef struct {
  int32_t format;         /* gsc_format: BC1 or BC7 in every block, or rate-controlled */
  uint32_t target_bpt_x4; /* rate target in quarter bits per coefficient texel (e.g. 12, 16, 24, 32) */
  /* GSC_FMT_RATE only, optional (NULL = not wanted): the rate control codes every block
   * both ways, and these receive the all-BC1 and all-BC7 layouts of the same planned order
   * ([n_groups][16][8] and [n_groups][16][16] bytes, 16-byte aligned), i.e. exactly what
   * GSC_FMT_BC1 and GSC_FMT_BC7 would write for d_perm. */
  uint8_t* d_bc1_blocks;
  uint8_t* d_bc7_blocks;
  /* Block layout (gsc_layout; 0 = D). Layouts A and B take BC1, BC7 and GSC_FMT_MIXED, not the
   * rate control (its streams drop coefficients, which layout D's blocks make possible). */
  int32_t layout;
  /* GSC_FMT_MIXED only: BC7 blocks per group, j. D: 0..16, the first j blocks; B: 0, 4, 8, 12 or
   * 16, the first j / 4 blocks of every quad (j = 4 is Table I's 10 bytes per Gaussian); A: 0 or 16. */
  int32_t bc7_blocks;
} gsc_encode_params;

/* One fixed-rate stream: every group in it keeps `bands` coefficients, `bc7_blocks` of its
 * blocks coded BC7 (16 B) and the rest BC1 (8 B); coefficients not kept decode to zero
 * (texel 128). Group bytes = 16 * bc7_blocks + 8 * (bands - bc7_blocks): the group's BC7
 * blocks in block order, then its BC1 blocks in block order. Which blocks are BC7 follows the
 * layout (gsc_encode_params.bc7_blocks); layouts A and B keep all 16 coefficients. */
typedef struct {
  int32_t bands, bc7_blocks;
  int64_t first_group, n_groups, byte_offset;
} gsc_stream;

/* Everything a decoder needs besides the blocks and the permutation. */
typedef struct {
  int32_t n_streams, format;
  int64_t n, n_groups, total_bytes;
  uint64_t budget_bits, used_bits, lambda;
  float scales[16];     /* s_k: x' = (q - 128) / 255 * s_k */
  uint32_t weights[16]; /* w_k used by the rate control */
  gsc_stream s[14];
  int32_t layout;       /* gsc_layout of the blocks */
} gsc_stream_table;

/* Context on one device (made current by every call). */
gsc_status gsc_ctx_create(gsc_ctx** out, int device);
/* Waits for the device, then frees the context's own buffers (not the caller's). */
gsc_status gsc_ctx_destroy(gsc_ctx* ctx);
/* Waits for `stream` and returns the first error a kernel recorded since the last
 * sync (then clears it). */
gsc_status gsc_ctx_sync(gsc_ctx* ctx, void* stream);
/* A static description of a status code (never NULL). */
const char* gsc_status_string(gsc_status s);

/* Bytes of scratch that gsc_plan_reorder and gsc_encode need for n Gaussians. */
size_t gsc_workspace_bytes(int64_t n, const gsc_encode_params* ep);

/* Sec. V-A and Sec. III-C. Computes the 16 scales s_k = 2 a_k, a_k the
 * ceil(permille * 3n / 1000)-th smallest |H~[:, k, :]| (exact order statistic; 1 if
 * zero), quantises the DC coefficient, and writes the slot order
 * d_perm[s] = original index of slot s, s < n_groups * 16 (padding slots = -1).
 * Slot order: sort = 1 ranks Gaussians by 30-bit Morton code of the bounding-box
 * grid (10 bits per axis; original index breaks ties), cuts the ranks into chunks
 * of group_size, and orders by (chunk, 24-bit RGB bit interleave of the DC texel,
 * rank). d_pos [n][3] float, d_sh [n][16][3] float, d_scales [16] float. */
gsc_status gsc_plan_reorder(gsc_ctx* ctx, const float* d_pos, const float* d_sh, const gsc_plan_params* pp,
                            int32_t* d_perm, float* d_scales, void* d_ws, size_t ws_bytes, void* stream);

/* Allocation-free form of gsc_plan_reorder (the paper has no counterpart: this is a
 * service for callers that cannot call cudaMalloc, e.g. a host framework that owns all
 * device memory and forbids foreign allocations, or a latency-bound loop that must not
 * pay for cudaMalloc's implicit synchronisation or risk an out-of-memory failure there).
 * Same arguments and results as gsc_plan_reorder without d_ws / ws_bytes: its scratch is
 * a 2 MiB array inside the library that every GPU loading the library keeps until the
 * process exits. Limits: 0 <= n <= GSC_PLAN_STATIC_MAX_N (65536) Gaussians; larger n
 * returns GSC_ERR_INVALID_ARG and launches nothing. It calls no cudaMalloc, cudaFree or
 * allocating library routine. The first call on a device looks up the array's device
 * address (with that device current); make that first call before any stream capture. The
 * address is kept for the life of the process: after a cudaDeviceReset of that device it is
 * stale, so do not call this entry point on a device that was reset. Records its time under
 * "plan" like gsc_plan_reorder when the context's timing is on.
 * All calls share the one array, which keeps the last call's contents (the call clears
 * what it needs): calls that overlap on the GPU, from any stream or context of the
 * process, race on it and must be serialised by the caller. */
#define GSC_PLAN_STATIC_MAX_N 65536
gsc_status gsc_plan_reorder_static(gsc_ctx* ctx, const float* d_pos, const float* d_sh, const gsc_plan_params* pp,
                                   int32_t* d_perm, float* d_scales, void* stream);

/* Sec. V-A: q = clamp(128 + rint(fl(fl(x / s_k) * 255)), 0, 255), round half to even.
 * d_sh [n][16][3] float -> d_q [n][16][3] uint8. */
gsc_status gsc_quantise(gsc_ctx* ctx, const float* d_sh, int64_t n, const float* d_scales, uint8_t* d_q, void* stream);

/* Sec. IV-B (Figs. SetupD, SetupA, SetupB), Sec. III-B, Sec. IV-B rate control. Group g =
 * slots 16g..16g+15; its 16 blocks hold those Gaussians' coefficients as the layout says (a
 * padding slot repeats the group's last valid slot). BC1 / BC7 formats code all 16 blocks
 * of every group; GSC_FMT_MIXED codes ep->bc7_blocks of them BC7 and the rest BC1 (one
 * stream); GSC_FMT_RATE (layout D) picks one of 14 stream modes per group under the budget
 * floor(target_bpt_x4 * 4 * n) bits. Layouts A and B and GSC_FMT_MIXED stage the texels in
 * the workspace and need ws_bytes >= gsc_workspace_bytes(n, ep).
 * d_blocks receives the streams back to back (capacity n_groups * 256 bytes),
 * d_perm_out the final slot order, *h_table the stream table. Synchronises `stream`
 * before returning (the table carries the scales and, in GSC_FMT_RATE, device results);
 * returns GSC_ERR_BUDGET if even the cheapest mode everywhere exceeds the budget. */
gsc_status gsc_encode(gsc_ctx* ctx, const float* d_sh, int64_t n, const int32_t* d_perm, const float* d_scales,
                      const gsc_encode_params* ep, uint8_t* d_blocks, int32_t* d_perm_out, gsc_stream_table* h_table,
                      void* d_ws, size_t ws_bytes, void* stream);

/* Host only. The stream table of the all-BC1 (format GSC_FMT_BC1) or all-BC7 (GSC_FMT_BC7)
 * coding of the scene that `table` describes (same n, scales, weights and layout): one stream of
 * every group with all 16 coefficients, n_groups * 16 * (8 or 16) bytes. It describes exactly the
 * d_bc1_blocks / d_bc7_blocks outputs of a GSC_FMT_RATE gsc_encode, and what GSC_FMT_BC1 /
 * GSC_FMT_BC7 write for the same slot order (budget_bits 0, used_bits = 8 * total_bytes,
 * lambda 0). GSC_ERR_INVALID_ARG if `table` is not a valid stream table or format is another. */
gsc_status gsc_forced_table(const gsc_stream_table* table, int32_t format, gsc_stream_table* out);

/* Sec. I and III-A (random access: block = stream offset + index x block size) and
 * Sec. II. Decodes every stream to texels d_texels [n][16][3] uint8 in original order
 * (through the inverse permutation); coefficients a stream does not keep are 128. */
gsc_status gsc_decode(gsc_ctx* ctx, const gsc_stream_table* table, const uint8_t* d_blocks, const int32_t* d_perm,
                      uint8_t* d_texels, void* stream);

/* Sec. II, c(f) = H w(f - p): fused decode and SH evaluation in FP32.
 * x'_{k} = (q - 128) / 255 * s_k; rgb = sum_k x'_k Y_k(d), with real SH to degree 3
 * (k = l*l + l + m, Condon-Shortley phase), no offset and no clamp. Directions: either
 * d_dirs [V][3] unit vectors shared by all Gaussians, or d_cams [V][3] camera centres
 * with d = (cam - p) / |cam - p| from d_pos [n][3] ((0, 0, 1) if the camera sits on p).
 * Exactly one of d_dirs, d_cams is non-NULL. 1 <= V <= 64. out_order: gsc_out_order.
 * d_rgb must be 16-byte aligned. */
gsc_status gsc_decode_eval_sh(gsc_ctx* ctx, const gsc_stream_table* table, const uint8_t* d_blocks,
                              const int32_t* d_perm, const float* d_dirs, const float* d_pos, const float* d_cams,
                              int32_t V, int32_t out_order, float* d_rgb, void* stream);

/* Sec. II and Sec. III-C: gsc_decode_eval_sh with the Gaussians' centres given in slot order.
 * The reorder moves each Gaussian's position with its colour (Sec. III-C: no side data), so a
 * coded scene can keep d_pos_slot [n_groups * 16][3] float, row s = the centre of the Gaussian in
 * slot s (padding rows are not read); the evaluation then reads it contiguously instead of through
 * the inverse permutation. Same results as gsc_decode_eval_sh with d_pos; d_pos_slot replaces
 * d_pos (required with d_cams, ignored with d_dirs). d_blocks 8-byte and d_pos_slot 4-byte
 * aligned; d_rgb 16-byte aligned. */
gsc_status gsc_decode_eval_sh_slots(gsc_ctx* ctx, const gsc_stream_table* table, const uint8_t* d_blocks,
                                    const int32_t* d_perm, const float* d_dirs, const float* d_pos_slot,
                                    const float* d_cams, int32_t V, int32_t out_order, float* d_rgb, void* stream);

/* Centres in slot order for gsc_decode_eval_sh_slots: d_pos_slot[s] = d_pos[d_perm[s]] for the
 * n_slots = n_groups * 16 slots of a slot order d_perm over n Gaussians (0 for padding slots).
 * d_pos [n][3] and d_pos_slot [n_slots][3] float, 4-byte aligned. Asynchronous on `stream`. */
gsc_status gsc_positions_to_slots(gsc_ctx* ctx, const float* d_pos, int64_t n, const int32_t* d_perm,
                                  int64_t n_slots, float* d_pos_slot, void* stream);

/* Same output as gsc_decode, sampled through CUDA BC1/BC7 texture objects (the GPU's
 * fixed-function block decoders, Sec. I): blocks are gathered into 2-D CUDA arrays
 * (16384 blocks per row) and read with point sampling; texel = rint(255 * f). The
 * arrays and staging buffers live in the context and are rebuilt (with a stream
 * synchronisation) only when the block counts change; otherwise the call is
 * asynchronous. Calls on one context must not overlap on different streams. */
gsc_status gsc_decode_tex(gsc_ctx* ctx, const gsc_stream_table* table, const uint8_t* d_blocks,
                          const int32_t* d_perm, uint8_t* d_texels, void* stream);

/* Sec. I (blocks decoded by the GPU's fixed-function texture unit) and Sec. II. A coded
 * scene kept resident as BC1/BC7 texture objects: gsc_tex_scene_create gathers every
 * stream's blocks into 2-D CUDA arrays (16384 blocks per row) and, when d_perm and d_pos
 * [n][3] are given, keeps the positions in slot order (Sec. III-C: positions move with
 * the Gaussians, so no side data is needed). It allocates the arrays, the positions and a
 * temporary staging buffer, and synchronises `stream`; the scene owns its memory until
 * gsc_tex_scene_destroy. The inputs may be freed or overwritten after create returns. */
typedef struct gsc_tex_scene gsc_tex_scene;
gsc_status gsc_tex_scene_create(gsc_ctx* ctx, const gsc_stream_table* table, const uint8_t* d_blocks,
                                const int32_t* d_perm, const float* d_pos, gsc_tex_scene** out, void* stream);
gsc_status gsc_tex_scene_destroy(gsc_tex_scene* scene);
/* gsc_decode_eval_sh with the texels fetched through the texture unit from a resident
 * scene (same arguments otherwise; d_perm is the scene's slot order; d_pos may be NULL
 * when the scene holds positions). The dequantisation
 * recovers q - 128 exactly from the UNORM8 sample and the SH evaluation is the same code,
 * so the colours equal gsc_decode_eval_sh's bit for bit. */
gsc_status gsc_decode_eval_sh_tex(gsc_ctx* ctx, const gsc_tex_scene* scene, const int32_t* d_perm,
                                  const float* d_dirs, const float* d_pos, const float* d_cams, int32_t V,
                                  int32_t out_order, float* d_rgb, void* stream);

/* Splatting renderer (Sec. II: Eq. sigmoid mu = 1 / (1 + e^-t), Eq. covar Sigma = R(q) D(s) D(s)^T
 * R(q)^T, Eq. opac, Eq. preblend a = sum_i g_i c~_i prod_{j<i} (1 - mu_j g_j) with the premultiplied
 * c~ = H~ w(f - p) of Eq. premult; Fig. GSRend). Pinhole camera: x_cam = R x + t; pixel (x, y)
 * covers [x, x+1) x [y, y+1) and is sampled at its centre; Gaussians at camera depth <= near_z are
 * culled. g is the EWA screen-space splat: the Gaussian projected with the pinhole Jacobian at its
 * centre plus a 0.3 px^2 low-pass, evaluated on the 16 x 16 pixel tiles that its 3-sigma square
 * touches; Gaussians are blended nearest first (camera depth, then index), with no early stop. */
typedef struct {
  float R[9];           /* world -> camera rotation, row-major (rows: image right, image down, view) */
  float t[3];           /* world -> camera translation */
  float fx, fy, cx, cy; /* focal lengths and principal point, pixels */
  int32_t width, height; /* 1..16384 */
  float near_z;         /* > 0 */
} gsc_camera;

/* Workspace bytes of gsc_render for n Gaussians and up to max_pairs (Gaussian, tile) overlaps; 0
 * when n or max_pairs is negative or the camera is missing or invalid. */
size_t gsc_render_workspace_bytes(int64_t n, const gsc_camera* cam, int64_t max_pairs);

/* Renders a coded scene (any layout and coding) for one camera into d_image [height][width][3]
 * float (background 0) and, if d_trans is not NULL, the final transmittance prod (1 - mu g)
 * [height][width]. Per Gaussian, in original order: d_pos [n][3], d_scale [n][3] (axis scales s),
 * d_rot [n][4] (quaternion w, x, y, z; normalised here; 16-byte aligned), d_logit [n] (opacity
 * logit t). The colour of every Gaussian is decoded from the blocks and evaluated for the camera
 * centre f = -R^T t in one fused pass. The call synchronises `stream` once, to size the sort: it
 * writes the number of (Gaussian, tile) overlaps to *h_pairs (if not NULL) and returns
 * GSC_ERR_OOM, with nothing rendered, when ws_bytes is below gsc_render_workspace_bytes(n, cam,
 * that number). */
gsc_status gsc_render(gsc_ctx* ctx, const gsc_stream_table* table, const uint8_t* d_blocks, const int32_t* d_perm,
                      const float* d_pos, const float* d_scale, const float* d_rot, const float* d_logit,
                      const gsc_camera* cam, float* d_image, float* d_trans, int64_t* h_pairs, void* d_ws,
                      size_t ws_bytes, void* stream);

/* Geometry streams and chunk hierarchy (Sec. IV-A: position and shape are coded apart from
 * appearance, each parameter quantised to a fixed number of bits in its own bitstream; a
 * hierarchy lets a view use only the primitives of the part it sees). In slot order (the
 * positions move with the Gaussians, so no index is stored), 17 bytes per slot: position 3 x 16
 * bits over the box of its chunk (chunk_slots consecutive slots, a multiple of 16), scale 3 x
 * bfloat16 (round to nearest even), rotation as the smallest three of the unit quaternion (2-bit
 * index of the largest component, made non-negative; three 10-bit codes of 1022 steps over
 * [-1/sqrt2, 1/sqrt2]), opacity logit 8 bits over [-8, 8]. Per chunk a gsc_chunk: the box of its
 * centres and its largest decoded scale (a chunk of padding only is zero). Decoding: position
 * lo + (code / 65535) (hi - lo), rotation component (code / 1022 - 1/2) sqrt2 and the largest
 * sqrt(1 - sum of the other squares), logit (code / 255) 16 - 8. One buffer holds the streams at
 * 256-byte aligned offsets: qpos u16 [n_slots][3], qscale u16 [n_slots][3], qrot u32 [n_slots],
 * qlogit u8 [n_slots], chunks [n_chunks]. */
typedef struct {
  float lo[3], hi[3];
  float max_scale;
  float pad;
} gsc_chunk;
/* Bytes of the geometry buffer for n_slots slots in chunks of chunk_slots; 0 when n_slots < 0 or
 * chunk_slots is not a positive multiple of 16. */
size_t gsc_geometry_bytes(int64_t n_slots, int64_t chunk_slots);
/* Host only. Byte offsets of the five sections of a geometry buffer (centre codes u16 [n_slots][3],
 * scale codes u16 [n_slots][3], rotation codes u32 [n_slots], opacity codes u8 [n_slots], chunk
 * table gsc_chunk [ceil(n_slots / chunk_slots)], each 256-byte aligned) into offsets[5]; returns
 * the buffer size (gsc_geometry_bytes), or 0 for invalid sizes or a NULL offsets. */
size_t gsc_geometry_layout(int64_t n_slots, int64_t chunk_slots, size_t* offsets);
/* Codes the geometry of a planned scene (d_perm [n_slots], n_slots a multiple of 16; geometry in
 * original order as gsc_render takes it) into d_geom (256-byte aligned, gsc_geometry_bytes). */
gsc_status gsc_geometry_encode(gsc_ctx* ctx, const float* d_pos, const float* d_scale, const float* d_rot,
                               const float* d_logit, const int32_t* d_perm, int64_t n_slots, int64_t chunk_slots,
                               uint8_t* d_geom, void* stream);
/* gsc_render from a fully coded scene: colour from the blocks, geometry from d_geom. Chunks are
 * culled first (kept unless the box of their centres, grown by 6 times their largest scale, lies
 * entirely at camera depth <= near_z / 2, or entirely in front of the camera and more than 64
 * pixels beyond one image side, corners projected in float in a fixed order), and only the kept
 * chunks' groups are decoded and splatted; *h_chunks (if not NULL) receives the kept count. The
 * image equals gsc_render's of the decoded geometry restricted to the kept chunks. */
gsc_status gsc_render_coded(gsc_ctx* ctx, const gsc_stream_table* table, const uint8_t* d_blocks,
                            const int32_t* d_perm, const uint8_t* d_geom, int64_t chunk_slots, const gsc_camera* cam,
                            float* d_image, float* d_trans, int64_t* h_pairs, int64_t* h_chunks, void* d_ws,
                            size_t ws_bytes, void* stream);

/* Batched form: many scenes of uneven sizes (the paper codes one scene at a time; this packages
 * the same steps for throughput). Per scene the results equal the single-scene calls bit for bit:
 * the plan of gsc_plan_reorder (quantile 995), then the blocks, slot order and stream table of
 * gsc_encode with the scene's format. All BC1/BC7 block searches of all scenes run in one
 * persistent launch whose CTAs claim tiles of groups (Sec. IV-B layout D); rate scenes then
 * select their streams one by one. At most 1024 scenes (else GSC_ERR_INVALID_ARG). Scenes are
 * coded in layout D (the layouts of Figs. SetupA / SetupB go through gsc_encode). The caller
 * owns every buffer; the call synchronises `stream`. */
typedef struct {
  const float* d_pos;       /* [n][3] (needed when sort = 1 and for evaluation) */
  const float* d_sh;        /* [n][16][3], 16-byte aligned */
  int64_t n;
  int64_t group_size;       /* as gsc_plan_params */
  int32_t sort;
  int32_t format;           /* GSC_FMT_BC1, GSC_FMT_BC7 or GSC_FMT_RATE */
  uint32_t target_bpt_x4;   /* rate scenes */
  int32_t* d_perm;          /* out: planned slot order [n_groups*16] */
  float* d_scales;          /* out: [16] */
  uint8_t* d_blocks;        /* out: n_groups*256 bytes of capacity, 16-byte aligned */
  int32_t* d_perm_out;      /* out: final slot order [n_groups*16] */
  gsc_stream_table table;   /* out */
} gsc_batch_scene;

/* How the encode launch hands out work: schedule 0 = static round robin over tiles, 1 = atomic
 * work queue, 2 = atomic queue, 3 = one CTA unit per tile; schedules other than 1 list the scenes
 * by decreasing cost. CTAs per SM 1..32 (schedules 0-2; a BC1 CTA is 128 threads, 5 fit per SM; a
 * BC7 CTA is five 128-thread units that claim their own tiles, 1 fits per SM; above what fits the
 * grid is oversubscribed and the hardware block scheduler balances); groups per BC1 tile (multiple
 * of 8; BC7 tiles are 8 groups). The plans of the scenes run on 4 streams at once. */
typedef struct {
  int32_t schedule;
  int32_t ctas_per_sm;
  int32_t bc1_tile_groups;
} gsc_batch_tuning;

/* Workspace bytes of gsc_batch_encode / gsc_batch_autotune for these scenes (0 if invalid). */
size_t gsc_batch_workspace_bytes(const gsc_batch_scene* scenes, int32_t n_scenes);
gsc_status gsc_batch_encode(gsc_ctx* ctx, gsc_batch_scene* scenes, int32_t n_scenes, const gsc_batch_tuning* tune,
                            void* d_ws, size_t ws_bytes, void* stream);
/* Times 9 tunings (work queues on resident grids, oversubscribed round robin, one CTA per
 * tile) on a 1/8-scale proxy of the same batch (each scene's first groups) and returns the
 * fastest. It writes the
 * scenes' plans and partial blocks (gsc_batch_encode overwrites them). */
gsc_status gsc_batch_autotune(gsc_ctx* ctx, gsc_batch_scene* scenes, int32_t n_scenes, gsc_batch_tuning* out,
                              double* proxy_ms, void* d_ws, size_t ws_bytes, void* stream);

/* Decode + SH evaluation (gsc_decode_eval_sh with camera centres) of every scene of an encoded
 * batch, captured once into a CUDA graph on `stream` (a created stream, not the legacy one)
 * and replayed with gsc_graph_launch. d_rgb[i] is scene i's output (16-byte aligned). The
 * graph reads the scenes' buffers at launch time but keeps each scene's stream table as it
 * was at capture: capture again after a re-encode that changes a table. */
typedef struct gsc_graph gsc_graph;
gsc_status gsc_batch_eval_graph(gsc_ctx* ctx, const gsc_batch_scene* scenes, int32_t n_scenes, const float* d_cams,
                                int32_t V, int32_t out_order, float* const* d_rgb, gsc_graph** out, void* stream);
gsc_status gsc_graph_launch(gsc_graph* graph, void* stream);
gsc_status gsc_graph_destroy(gsc_graph* graph);

/* Request loop (serving form; the paper codes scenes offline, this keeps the same calls
 * behind a queue). Encode and evaluation requests are submitted at any time from any host
 * thread; coded scenes stay resident on the device; n_slots worker threads each own a
 * context and two CUDA streams (evaluations on the high-priority one) and take the next
 * admissible request as soon as they are free, so the work of several requests overlaps on
 * the device. A request is admitted when a slot is free and its device memory fits in
 * hbm_budget_bytes (resident scenes + running requests' buffers), evicting idle resident
 * scenes least recently used first when that makes it fit. Requests on one scene keep their
 * submission order around encodes. Queued evaluations of one scene with the same output
 * order and view kind merge into one launch of up to max_views views. Every result equals
 * the single calls' bit for bit: an encode is gsc_plan_reorder (quantile 995) + gsc_encode
 * (layout D; a loaded checkpoint keeps the layout its table names),
 * an evaluation is gsc_decode_eval_sh of the scene's resident coding. */
typedef struct {
  uint64_t hbm_budget_bytes;
  int32_t n_slots;            /* 1..16 */
  int32_t merge;              /* 0 or 1 */
  int32_t max_views;          /* 1..64: views of one evaluation request and of one merged launch */
  int32_t priority;           /* 1: evaluations on high-priority streams */
  int32_t encode_slots;       /* encodes running at once, 1..n_slots (0: n_slots - 1, at least 1), so
                               * that evaluations keep a slot while long encodes run */
  int64_t hold_us;            /* a request older than this that does not fit holds back later ones */
} gsc_server_params;

enum { GSC_REQ_ENCODE = 0, GSC_REQ_EVAL = 1, GSC_REQ_LOAD = 2 };

/* Pointers may be host (pinned or pageable) or device memory and must stay valid until the
 * request completes. Encode: pos [n][3], sh [n][16][3] (16-byte aligned), format, rate target,
 * group_size and sort as in gsc_plan_reorder / gsc_encode. Evaluation: n = the resident scene's
 * Gaussian count (the request fails with GSC_ERR_INVALID_ARG if the scene is not resident or has
 * another size), exactly one of dirs / cams [V][3], out [n][V][3] / [V][n][3] / [V][ns][3] by
 * out_order, 16-byte aligned. */
typedef struct {
  int32_t kind;
  int32_t scene;              /* caller's id, >= 0 */
  const float* pos;
  const float* sh;
  int64_t n;
  int32_t format;
  uint32_t target_bpt_x4;
  int64_t group_size;
  int32_t sort;
  int32_t V;
  const float* dirs;
  const float* cams;
  int32_t out_order;
  float* out;
  const char* path;           /* load: a checkpoint file written with positions (gsc_scene_write); n = its
                               * Gaussian count. The load is ordered and admitted like an encode. */
} gsc_request;

typedef struct {
  int32_t status;             /* gsc_status of the request */
  int32_t kind;
  int32_t scene;
  int32_t merged;             /* requests in its launch */
  int64_t n;
  double t_submit_ms, t_admit_ms, t_done_ms;  /* since gsc_server_create */
} gsc_request_result;

typedef struct {
  uint64_t submitted, done, failed, merged, evictions;
  uint64_t resident_bytes, used_bytes, peak_bytes;
  int32_t queued, resident_versions;
} gsc_server_stats;

typedef struct gsc_server gsc_server;
gsc_status gsc_server_create(gsc_ctx* ctx, const gsc_server_params* p, gsc_server** out);
/* GSC_ERR_BUDGET when the request could never fit; otherwise queued, *ticket identifies it. */
gsc_status gsc_server_submit(gsc_server* srv, const gsc_request* req, uint64_t* ticket);
/* Waits for a ticket (timeout_ms < 0: no limit; GSC_ERR_TIMEOUT when it runs out) and
 * consumes it. The request's own outcome is res->status. */
gsc_status gsc_server_wait(gsc_server* srv, uint64_t ticket, int64_t timeout_ms, gsc_request_result* res);
/* Waits until no request is queued or running (timeout_ms < 0: no limit; GSC_ERR_TIMEOUT). */
gsc_status gsc_server_drain(gsc_server* srv, int64_t timeout_ms);
/* Copies a resident scene's table, blocks and slot order out (host or device buffers). */
gsc_status gsc_server_read_scene(gsc_server* srv, int32_t scene, gsc_stream_table* table, uint8_t* blocks,
                                 size_t blocks_cap, int32_t* perm, size_t perm_bytes_cap);
/* Cancels a queued request: it completes with GSC_ERR_CANCELLED (collect it with
 * gsc_server_wait). A request already admitted or completed cannot be cancelled
 * (GSC_ERR_INVALID_ARG). */
gsc_status gsc_server_cancel(gsc_server* srv, uint64_t ticket);
/* Writes a resident scene (with its positions) to a checkpoint file (gsc_scene_write). */
gsc_status gsc_server_save_scene(gsc_server* srv, int32_t scene, const char* path);
/* Frees a resident scene that no queued or running request uses (else GSC_ERR_INVALID_ARG). */
gsc_status gsc_server_evict(gsc_server* srv, int32_t scene);
/* Counters since creation and the current memory figures. */
gsc_status gsc_server_get_stats(gsc_server* srv, gsc_server_stats* st);
/* Drains, stops the workers and frees every resident scene. */
gsc_status gsc_server_destroy(gsc_server* srv);

/* The admission policy of the request loop run on the host against a trace: arrivals in ms,
 * a service time per request (a merged launch takes the sum of its requests'), n_slots
 * launches at a time. No device work; the memory figures are the server's. */
typedef struct {
  int32_t kind, scene;
  int64_t n;
  int32_t format;
  uint32_t target_bpt_x4;
  int32_t V, out_order, cams, out_device, host_input;
  double t_arrival_ms, service_ms;
} gsc_sim_request;

typedef struct {
  int32_t status;             /* GSC_OK, GSC_ERR_INVALID_ARG (rejected), GSC_ERR_BUDGET (never fits) */
  int32_t merged;
  int32_t evictions;          /* scenes evicted to admit it */
  int32_t pad;
  double t_admit_ms, t_done_ms;
  uint64_t used_bytes_at_admit;
} gsc_sim_result;

gsc_status gsc_server_simulate(const gsc_server_params* p, const gsc_sim_request* reqs, int32_t n,
                               gsc_sim_result* res, uint64_t* peak_bytes);

/* 1 in the checked build (libgsc_checked.so, selected with GSC_CHECKED=1 by the binding): every
 * slot-order entry the decoders read is checked against [-1, n); entries outside are treated as
 * empty slots (never used for an access) and the first one is reported by the next
 * gsc_ctx_sync as GSC_ERR_DEVICE. 0 in the normal build, which trusts the slot order. */
int32_t gsc_build_checked(void);

/* Checkpoint file of a coded scene (the paper stores scenes as these streams; the file format is
 * this codec's own): a versioned header with the stream table, section sizes and an FNV-1a 64
 * checksum, then the blocks (table->total_bytes), the final slot order (n_groups * 16 int32) and
 * optionally the positions (n * 3 float). Buffers may be host or device memory. Reading checks the
 * magic, version, sizes against the table and the checksum (GSC_ERR_INVALID_ARG on any mismatch or
 * a capacity too small); the bytes read back equal the bytes written. */
gsc_status gsc_scene_write(const char* path, const gsc_stream_table* table, const uint8_t* blocks,
                           const int32_t* perm, const float* pos);
/* Reads and checks the header only: the table and whether positions are stored, to size the
 * buffers of gsc_scene_read. */
gsc_status gsc_scene_read_info(const char* path, gsc_stream_table* table, int32_t* has_pos);
gsc_status gsc_scene_read(const char* path, gsc_stream_table* table, uint8_t* blocks, size_t blocks_cap,
                          int32_t* perm, size_t perm_bytes_cap, float* pos, size_t pos_bytes_cap);

/* Block-level codecs (Sec. III-B): nblk independent 4x4 blocks.
 * d_tex [nblk][16][3] uint8 -> d_out [nblk][8 or 16] bytes; d_sse [nblk] (optional)
 * receives each block's squared error. format: GSC_FMT_BC1 or GSC_FMT_BC7. */
gsc_status gsc_encode_blocks(gsc_ctx* ctx, const uint8_t* d_tex, int64_t nblk, int32_t format, uint8_t* d_out,
                             uint64_t* d_sse, void* stream);
/* d_blocks [nblk][8 or 16] -> d_rgba [nblk][16][4] uint8 (software decoder). */
gsc_status gsc_decode_blocks(gsc_ctx* ctx, const uint8_t* d_blocks, int64_t nblk, int32_t format, uint8_t* d_rgba,
                             void* stream);
/* Same through a texture object; synchronises `stream`. */
gsc_status gsc_decode_blocks_tex(gsc_ctx* ctx, const uint8_t* d_blocks, int64_t nblk, int32_t format,
                                 uint8_t* d_rgba, void* stream);

/* ---- One scene split over shards (ranks or streams) ------------------------------------
 * Sec. V-A fixes the 16 scales as order statistics of the whole scene, Sec. III-C reorders
 * chunk by chunk within the spatial order, and Sec. IV-B spends one rate budget on the whole
 * scene. These calls split that work: every shard computes an integer partial, the caller
 * combines the partials of all shards (elementwise minimum / maximum / sum, or a gather) by any
 * means (torch.distributed, NCCL, or in one process), and passes the combined values to the next
 * call. With them every shard takes the decisions of the whole-scene calls, so the scales, the
 * slot order, lambda, the streams and the permutation equal those of gsc_plan_reorder (sort = 1,
 * group_size > 0) followed by gsc_encode (GSC_FMT_RATE), byte for byte. All partials are int64
 * in device memory (`d_part` arguments: written; `d_total`/`d_in`/`d_hist`/`d_bb` as inputs: the
 * combined values). Every call is queued on `stream` and does not synchronise it, except
 * gsc_shard_rate_assemble. Errors: GSC_ERR_INVALID_ARG for a null or misaligned pointer, a size
 * out of range or a pass out of range; GSC_ERR_OOM for a short workspace; GSC_ERR_BUDGET from
 * the assembly when the budget cannot be met.
 *
 * Order of calls (S shards; "combine" is over all S; shard s holds inputs [in_s, in_s + m_s),
 * contiguous and in shard order):
 *  1. gsc_shard_bbox -> combine: min of [0,3), max of [3,6)            (6 values)
 *  2. gsc_shard_morton with the combined box -> gather all keys in input order
 *  3. gsc_shard_order on all keys: the spatial order of the scene (input indices); with
 *     gsc_shard_bounds, shard s owns order[b_s, b_s+1), chunk-aligned; the caller moves those
 *     Gaussians (centres, SH) to shard s, in that order.
 *  4. gsc_shard_select_begin (the whole scene's n); for pass 0..3: gsc_shard_select_hist ->
 *     combine: sum (16 x 256) -> gsc_shard_select_pick; then gsc_shard_select_scales.
 *  5. gsc_shard_plan on the shard's owned Gaussians -> the shard's slot order (local indices).
 *  6. gsc_shard_rate_begin -> combine: sum (1) -> gsc_shard_rate_search_begin; for pass 0..12:
 *     gsc_shard_rate_count -> combine: sum (64) -> gsc_shard_rate_narrow.
 *  7. gsc_shard_rate_fill -> d_part = {sum at lambda*, sum of this shard's fill deltas}; pass to
 *     gsc_shard_rate_apply d_in = {sum over all shards of the first, sum of the second over the
 *     shards before this one} -> d_part (15: groups per mode, bits used) -> gather all shards'.
 *  8. gsc_shard_rate_assemble with the gathered parts [S][15]: writes this shard's groups into
 *     the scene's stream buffer and slot order at the places the whole-scene call writes them
 *     (d_index_map maps the shard's local indices to the scene's input indices), and fills the
 *     whole scene's stream table. */
#define GSC_SHARD_SELECT_PASSES 4
#define GSC_SHARD_RATE_PASSES 13
#define GSC_SHARD_RATE_PART 15
/* Shard s of S gets chunks [floor(C s / S), floor(C (s + 1) / S)) of the C = ceil(n_total /
 * group_size) chunks: bounds[s] = min(n_total, that chunk index x group_size), s = 0..S (host). */
gsc_status gsc_shard_bounds(int64_t n_total, int32_t n_shards, int64_t group_size, int64_t* bounds);
/* d_bb [6] out: order-preserving 32-bit codes of the per-axis minimum (3) and maximum (3) centre
 * coordinate of the shard's n centres d_pos [n][3] (empty shard: 0xFFFFFFFF and 0). */
gsc_status gsc_shard_bbox(gsc_ctx* ctx, const float* d_pos, int64_t n, int64_t* d_bb, void* stream);
/* d_keys [n] out: the 30-bit Morton code of each centre on the 1024^3 grid of the combined box. */
gsc_status gsc_shard_morton(gsc_ctx* ctx, const float* d_pos, int64_t n, const int64_t* d_bb, uint64_t* d_keys,
                            void* stream);
/* d_keys [n_total] (all shards' keys in input order; overwritten) -> d_order [n_total]: input
 * indices stably sorted by key (the whole-scene spatial rank). Workspace: gsc_shard_order_ws_bytes,
 * 256-byte aligned. */
size_t gsc_shard_order_ws_bytes(int64_t n_total);
gsc_status gsc_shard_order(gsc_ctx* ctx, uint64_t* d_keys, int64_t n_total, int32_t* d_order, void* d_ws,
                           size_t ws_bytes, void* stream);
/* Selection state (device, gsc_shard_select_state_bytes, 256-byte aligned, owned by the caller):
 * begin sets the target rank ceil(permille x 3 n_total / 1000) - 1 per scale; pass p examines bits
 * [24 - 8p, 32 - 8p) of |x|: hist writes the shard's d_hist [16][256], pick takes the combined
 * one; scales writes d_scales [16] (s_k = 2 a_k, 1 where a_k = 0). */
size_t gsc_shard_select_state_bytes(void);
gsc_status gsc_shard_select_begin(gsc_ctx* ctx, int64_t n_total, uint32_t permille, void* d_state, void* stream);
gsc_status gsc_shard_select_hist(gsc_ctx* ctx, const float* d_sh, int64_t n, int32_t pass, void* d_state,
                                 int64_t* d_hist, void* stream);
gsc_status gsc_shard_select_pick(gsc_ctx* ctx, void* d_state, const int64_t* d_hist, int32_t pass, void* stream);
gsc_status gsc_shard_select_scales(gsc_ctx* ctx, const void* d_state, float* d_scales, void* stream);
/* The slot order of a shard: d_sh [n][48] holds the shard's Gaussians in spatial-rank order, the
 * first one starting a chunk of group_size (> 0, multiple of 16); d_perm [ceil(n/16)*16] out,
 * local indices, -1 padding. Workspace gsc_shard_plan_ws_bytes(n), 256-byte aligned. */
size_t gsc_shard_plan_ws_bytes(int64_t n);
gsc_status gsc_shard_plan(gsc_ctx* ctx, const float* d_sh, int64_t n, const float* d_scales, int64_t group_size,
                          int32_t* d_perm, void* d_ws, size_t ws_bytes, void* stream);
/* Rate control of a shard of n Gaussians (its own workspace, gsc_shard_rate_ws_bytes(n), kept
 * across the calls 6-8). begin codes the shard's groups (d_perm: its slot order) in BC1 into
 * d_bc1 [ceil(n/16)][16][8] and in BC7 into d_bc7 [ceil(n/16)][16][16] (16-byte aligned; kept by
 * the caller until assemble) and writes d_part [1]: the rate at lambda = 2^62. search_begin takes
 * the combined value, the scene's n_total and target (1..64, in quarter bits per texel). */
size_t gsc_shard_rate_ws_bytes(int64_t n);
gsc_status gsc_shard_rate_begin(gsc_ctx* ctx, const float* d_sh, int64_t n, const int32_t* d_perm,
                                const float* d_scales, uint8_t* d_bc1, uint8_t* d_bc7, void* d_ws, size_t ws_bytes,
                                int64_t* d_part, void* stream);
gsc_status gsc_shard_rate_search_begin(gsc_ctx* ctx, int64_t n, void* d_ws, int64_t n_total, uint32_t target_x4,
                                       const int64_t* d_min_total, void* stream);
gsc_status gsc_shard_rate_count(gsc_ctx* ctx, int64_t n, void* d_ws, int32_t pass, int64_t* d_part, void* stream);
gsc_status gsc_shard_rate_narrow(gsc_ctx* ctx, int64_t n, void* d_ws, int32_t pass, const int64_t* d_total,
                                 void* stream);
gsc_status gsc_shard_rate_fill(gsc_ctx* ctx, int64_t n, void* d_ws, int64_t* d_part, void* stream);
gsc_status gsc_shard_rate_apply(gsc_ctx* ctx, int64_t n, void* d_ws, const int64_t* d_in, int64_t* d_part,
                                void* stream);
/* d_blocks: the scene's stream buffer (16-byte aligned, at least the table's total_bytes);
 * d_perm_out: the scene's slot order [ceil(n_total/16)*16]; d_index_map [n] (optional): the
 * scene's input index of each of the shard's Gaussians; h_table: the whole scene's table, the
 * same on every shard. Synchronises `stream`. */
gsc_status gsc_shard_rate_assemble(gsc_ctx* ctx, int64_t n, void* d_ws, const uint8_t* d_bc1, const uint8_t* d_bc7,
                                   const int32_t* d_perm, const int32_t* d_index_map, const float* d_scales,
                                   const int64_t* d_parts_all, int32_t n_shards, int32_t shard, int64_t n_total,
                                   uint8_t* d_blocks, int32_t* d_perm_out, gsc_stream_table* h_table, void* stream);

/* Measurement helpers (not part of the codec).
 * gsc_launch_count: kernels this library has launched in this process so far.
 * gsc_probe_int_peak: runs an integer microbenchmark (independent IADD3 / LOP3 / IMAD
 * chains, 3 source-level operations per step, full occupancy) on the context's device
 * and stores the achieved 32-bit integer operations per second; synchronises `stream`. */
uint64_t gsc_launch_count(void);
gsc_status gsc_probe_int_peak(gsc_ctx* ctx, double* ops_per_s, void* stream);
/* gsc_probe_op_rate: throughput of one 32-bit integer instruction kind, independent chains at
 * full occupancy: kind 1 three-input add, 2 three-input logic op (lop3), 3 multiply-add,
 * 4 four-way byte dot product (dp4a), 5 the BC7 search's palette evaluation (dp4a of a texel
 * with a palette entry, key - 32 * dot, running minimum: 3 operations per evaluation). Stores
 * operations per second; GSC_ERR_INVALID_ARG for another kind; synchronises `stream`. */
gsc_status gsc_probe_op_rate(gsc_ctx* ctx, int32_t kind, double* ops_per_s, void* stream);
/* gsc_probe_bc7_mode1: the BC7 search restricted to mode 1 (64 two-subset partitions) over d_tex
 * [nblk][16][3] (u8 texels, the layout of gsc_encode_blocks), mapped thread per block
 * (warp_per_block 0, as the encoder) or warp per block (1: two partitions per lane and a shuffle
 * minimum). Writes each block's least error d_sse [nblk] and its partition d_part [nblk] (ties to
 * the lowest), the same for both mappings, and the launch's duration in *ms; synchronises `stream`. */
gsc_status gsc_probe_bc7_mode1(gsc_ctx* ctx, const uint8_t* d_tex, int64_t nblk, int32_t warp_per_block,
                               uint32_t* d_sse, int32_t* d_part, double* ms, void* stream);
/* Kernel timing: when enabled, each call records CUDA events on its own stream around its
 * main kernels. gsc_kernel_time waits for the recorded events and returns the summed
 * milliseconds and launch count of one kernel ("plan", "bc1_encode", "bc7_encode",
 * "rate_select", "decode", "decode_eval", "decode_tex", "decode_eval_tex", "batch_encode",
 * "render" (a whole frame), "render_blend") since timing was last enabled. */
gsc_status gsc_ctx_set_timing(gsc_ctx* ctx, int enable);
gsc_status gsc_kernel_time(gsc_ctx* ctx, const char* name, double* ms, int64_t* launches);

#ifdef __cplusplus
}
#endif
#endif

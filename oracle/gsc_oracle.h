/*
 * gsc_oracle.h -- declarations of the plain CPU oracle (test infrastructure only).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load
 * this library. The product path (the CUDA library under the package) never does.
 * This header is the oracle's own; it shares nothing with include/gsc.h.
 */
#ifndef GSC_ORACLE_H
#define GSC_ORACLE_H
#include <stdint.h>

#define OR_SH 16
#define OR_MODES 14

typedef struct {
  int32_t bands;       /* coefficients kept per Gaussian (1, 4, 9 or 16) */
  int32_t bc7_blocks;  /* leading blocks coded BC7; the rest of the kept blocks are BC1 */
  int64_t first_group; /* first group (in final order) of this stream */
  int64_t n_groups;
  int64_t byte_offset; /* offset of the stream in the block buffer */
} or_stream;

typedef struct {
  int32_t n_streams;
  int32_t format;      /* 1 BC1, 7 BC7, 0 rate-controlled, 2 a fixed BC7 / BC1 mix */
  int64_t n, n_groups, total_bytes;
  uint64_t budget_bits, used_bits, lambda;
  float scales[OR_SH];
  uint32_t weights[OR_SH];
  or_stream s[OR_MODES];
  int32_t layout;      /* OR_LAYOUT_D, _A or _B */
} or_table;

/* Block layouts (Sec. IV-B): a group is 16 slots and 16 blocks in every layout. */
#define OR_LAYOUT_D 0 /* Fig. SetupD: block k holds coefficient k of the 16 Gaussians */
#define OR_LAYOUT_A 1 /* Fig. SetupA: block k holds the 16 coefficients of one Gaussian */
#define OR_LAYOUT_B 2 /* Fig. SetupB: 4 blocks hold the 16 coefficients of 4 Gaussians */

int or_scales(const float* sh, int64_t n, uint32_t permille, float* scales);
uint8_t or_quant1(float x, float s);
void or_quantise(const float* sh, int64_t n, const float* scales, uint8_t* q);
uint32_t or_morton30(uint32_t x, uint32_t y, uint32_t z);
uint32_t or_colour_key(uint32_t r, uint32_t g, uint32_t b);
int or_plan(const float* pos, const uint8_t* q, int64_t n, int64_t group_size, int sort, int32_t* perm);
void or_stage_group(const uint8_t* q, const int32_t* perm, int64_t g, uint8_t* tex /*[16 blocks][16 texels][3]*/);
void or_layout_map(int layout, int k, int t, int* u, int* c);
int or_layout_ok(int layout, int bc7_blocks);
int or_layout_bc7(int layout, int bc7_blocks, int k);
void or_stage_layout(const uint8_t* q, const int32_t* perm, int layout, int64_t g, uint8_t* tex /*[16][16][3]*/);
int or_encode_layout(const uint8_t* q, int64_t n, const int32_t* perm, const float* scales, int layout,
                     int bc7_blocks, uint8_t* blocks, or_table* t);

void or_bc1_palette(uint16_t c0, uint16_t c1, uint8_t* pal /*[4][4] RGBA*/);
void or_bc1_decode(const uint8_t* blk, uint8_t* out /*[16][4]*/);
uint64_t or_bc1_candidate_sse(const uint8_t* tex, uint16_t c0, uint16_t c1);
uint64_t or_bc1_encode(const uint8_t* tex /*[16][3]*/, uint8_t* out /*[8]*/);

int or_bc7_subset(int ns, int part, int t);
int or_bc7_anchor(int ns, int part, int s);
void or_bc7_decode(const uint8_t* blk, uint8_t* out /*[16][4]*/);
int or_bc7_n_candidates(void);
uint64_t or_bc7_candidate(const uint8_t* tex, int cand, uint8_t* out /*[16] or NULL*/);
uint64_t or_bc7_encode(const uint8_t* tex /*[16][3]*/, uint8_t* out /*[16]*/);
void or_encode_blocks(const uint8_t* tex, int64_t nblk, int format, uint8_t* out, uint64_t* sse);

void or_mode_table(int32_t* bands, int32_t* bc7);
void or_weights(const float* scales, uint32_t* w);
int or_rate_choose(const uint64_t* D, int64_t ng, uint64_t lambda, uint8_t* mode);
int or_rate_control(const uint64_t* D, int64_t ng, uint64_t budget, uint8_t* mode, uint64_t* lambda);
/* The rate path in two steps (or_encode with format 0 runs both): both codings of every
 * group with the D table [ng][14], then rate control and stream assembly for one target.
 * or_set_threads splits the coding step over threads (default 1); results are identical. */
void or_set_threads(int threads);
void or_code_groups(const uint8_t* q, int64_t n, const int32_t* perm, const float* scales, uint8_t* b1, uint8_t* b7,
                    uint64_t* D);
int or_rate_assemble(int64_t n, const int32_t* perm, const float* scales, uint32_t target_x4, const uint8_t* b1,
                     const uint8_t* b7, const uint64_t* D, uint8_t* blocks, int32_t* perm_out, or_table* t);
int or_encode(const uint8_t* q, int64_t n, const int32_t* perm, const float* scales, int format,
              uint32_t target_x4, uint8_t* blocks, int32_t* perm_out, or_table* t, uint64_t* dtab);
int or_decode(const or_table* t, const uint8_t* blocks, const int32_t* perm, uint8_t* texels);

/* Splatting renderer (Sec. II, Eqs. sigmoid, covar, opac, preblend; Fig. GSRend). */
typedef struct {
  float R[9];        /* world -> camera rotation, row-major: x_cam = R x + t */
  float t[3];
  float fx, fy, cx, cy; /* pinhole intrinsics in pixels; pixel (x, y) covers [x, x+1) x [y, y+1) */
  int32_t width, height;
  float near_z;      /* Gaussians at camera depth <= near_z are culled */
} or_camera;
typedef struct {
  float u, v, depth;      /* projected centre (pixels), camera depth */
  float a, b, c;          /* 2-D covariance (with the 0.3 px^2 low-pass) */
  int32_t x0, y0, x1, y1; /* tile rectangle [x0, x1) x [y0, y1) of 16 x 16 pixel tiles */
  int32_t visible;
} or_splat;
void or_camera_centre(const or_camera* cam, float* f /*[3]*/);
int or_splat_setup(const float* p, const float* s, const float* q, const or_camera* cam, or_splat* out);
int or_render(int64_t n, const float* pos, const float* scale, const float* rot, const float* logit,
              const double* colour /*[n][3]*/, const or_camera* cam, const int32_t* tiles, int64_t n_tiles,
              double* image /*[H][W][3]*/, double* trans /*[H][W] or NULL*/, double* abs_sum /*or NULL*/);

/* Geometry streams and chunk hierarchy (Sec. IV-A); 17 bytes per slot. */
int64_t or_chunks(int64_t n_slots, int64_t chunk_slots);
void or_chunk_table(const float* pos, const float* scale, const int32_t* perm, int64_t n_slots, int64_t chunk_slots,
                    float* chunk /*[n_chunks][8]*/);
void or_geometry_encode(const float* pos, const float* scale, const float* rot, const float* logit,
                        const int32_t* perm, int64_t n_slots, int64_t chunk_slots, const float* chunk,
                        uint16_t* qpos, uint16_t* qscale, uint32_t* qrot, uint8_t* qlogit);
void or_geometry_decode_slot(const uint16_t* qpos, const uint16_t* qscale, const uint32_t* qrot, const uint8_t* qlogit,
                             int64_t s, int64_t chunk_slots, const float* chunk, float* p, float* sc, float* q,
                             float* t);
void or_geometry_decode_all(const uint16_t* qpos, const uint16_t* qscale, const uint32_t* qrot, const uint8_t* qlogit,
                            int64_t n_slots, int64_t chunk_slots, const float* chunk, float* p, float* sc, float* q,
                            float* t);
int or_chunk_visible(const float* chunk_entry, const or_camera* cam);

void or_sh_basis(double x, double y, double z, double* Y /*[16]*/);
void or_eval_sh(const uint8_t* texels, int64_t n, const float* scales, const float* pos,
                const float* dirs, const float* cams, int V, double* out /*[V][n][3]*/,
                double* abs_sum /*[V][n][3] or NULL*/);
#endif

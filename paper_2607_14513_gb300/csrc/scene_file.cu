// scene_file.cu -- the coded scene as a checkpoint file: a versioned header (stream table,
// section sizes, checksum) followed by the blocks, the final slot order and, optionally, the
// positions. Reading it back gives the same bytes, so a decode or evaluation of the reloaded
// scene equals the original's (Sec. IV-B streams are self-describing given the table).
#include <stdio.h>
#include <string.h>

#include <vector>

#include "gsc_internal.cuh"

namespace {

const char kMagic[8] = {'G', 'S', 'C', 'S', 'C', 'E', 'N', 'E'};
const uint32_t kVersion = 2;  // 2: the stream table carries the block layout

struct FileHeader {
  char magic[8];
  uint32_t version;
  uint32_t header_bytes;
  uint64_t blocks_bytes, perm_bytes, pos_bytes;
  uint64_t checksum;  // FNV-1a 64 over blocks, slot order and positions, in that order
  gsc_stream_table table;
};

uint64_t fnv1a(uint64_t h, const uint8_t* p, size_t n) {
  for (size_t i = 0; i < n; i++) { h ^= p[i]; h *= 0x100000001B3ull; }
  return h;
}

// Host view of a buffer that may live on the device: `host` is either the pointer itself or a
// copy staged in `stage`.
gsc_status to_host(const void* p, size_t bytes, std::vector<uint8_t>* stage, const uint8_t** host) {
  if (bytes == 0) { *host = nullptr; return GSC_OK; }
  cudaPointerAttributes a;
  const bool dev = cudaPointerGetAttributes(&a, p) == cudaSuccess &&
                   (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  if (!dev) { *host = static_cast<const uint8_t*>(p); return GSC_OK; }
  stage->resize(bytes);
  if (cudaMemcpy(stage->data(), p, bytes, cudaMemcpyDefault) != cudaSuccess) { cudaGetLastError(); return GSC_ERR_CUDA; }
  *host = stage->data();
  return GSC_OK;
}

gsc_status from_host(void* dst, const uint8_t* src, size_t bytes) {
  if (bytes == 0) return GSC_OK;
  cudaPointerAttributes a;
  const bool dev = cudaPointerGetAttributes(&a, dst) == cudaSuccess &&
                   (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  if (!dev) { memcpy(dst, src, bytes); return GSC_OK; }
  if (cudaMemcpy(dst, src, bytes, cudaMemcpyDefault) != cudaSuccess) { cudaGetLastError(); return GSC_ERR_CUDA; }
  return GSC_OK;
}

bool table_ok(const gsc_stream_table* t) {
  if (!t || t->n < 0 || t->n >= (int64_t)0x7FFFFFF0 || t->n_groups != (t->n + 15) / 16) return false;
  if (t->n_streams < 1 || t->n_streams > GSC_MODES || t->total_bytes < 0) return false;
  return true;
}

gsc_status read_header(FILE* f, FileHeader* h) {
  if (fread(h, sizeof(*h), 1, f) != 1) return GSC_ERR_INVALID_ARG;
  if (memcmp(h->magic, kMagic, 8) != 0 || h->version != kVersion || h->header_bytes != sizeof(FileHeader))
    return GSC_ERR_INVALID_ARG;
  if (!table_ok(&h->table) || h->blocks_bytes != (uint64_t)h->table.total_bytes ||
      h->perm_bytes != (uint64_t)h->table.n_groups * 16 * 4 || (h->pos_bytes != 0 && h->pos_bytes != (uint64_t)h->table.n * 12))
    return GSC_ERR_INVALID_ARG;
  return GSC_OK;
}

}  // namespace

extern "C" gsc_status gsc_scene_write(const char* path, const gsc_stream_table* table, const uint8_t* blocks,
                                      const int32_t* perm, const float* pos) {
  GscRange gsc_range_("gsc_scene_write");
  if (!path || !table_ok(table) || (table->total_bytes > 0 && !blocks) || (table->n_groups > 0 && !perm))
    return GSC_ERR_INVALID_ARG;
  FileHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, kMagic, 8);
  h.version = kVersion;
  h.header_bytes = sizeof(FileHeader);
  h.blocks_bytes = (uint64_t)table->total_bytes;
  h.perm_bytes = (uint64_t)table->n_groups * 16 * 4;
  h.pos_bytes = pos ? (uint64_t)table->n * 12 : 0;
  h.table = *table;
  std::vector<uint8_t> s1, s2, s3;
  const uint8_t *hb = nullptr, *hp = nullptr, *hq = nullptr;
  gsc_status rc = to_host(blocks, h.blocks_bytes, &s1, &hb);
  if (rc == GSC_OK) rc = to_host(perm, h.perm_bytes, &s2, &hp);
  if (rc == GSC_OK) rc = to_host(pos, h.pos_bytes, &s3, &hq);
  if (rc != GSC_OK) return rc;
  uint64_t c = 0xCBF29CE484222325ull;
  c = fnv1a(c, hb, h.blocks_bytes);
  c = fnv1a(c, hp, h.perm_bytes);
  c = fnv1a(c, hq, h.pos_bytes);
  h.checksum = c;
  FILE* f = fopen(path, "wb");
  if (!f) return GSC_ERR_INVALID_ARG;
  bool ok = fwrite(&h, sizeof(h), 1, f) == 1;
  if (ok && h.blocks_bytes) ok = fwrite(hb, 1, h.blocks_bytes, f) == h.blocks_bytes;
  if (ok && h.perm_bytes) ok = fwrite(hp, 1, h.perm_bytes, f) == h.perm_bytes;
  if (ok && h.pos_bytes) ok = fwrite(hq, 1, h.pos_bytes, f) == h.pos_bytes;
  ok = (fclose(f) == 0) && ok;
  return ok ? GSC_OK : GSC_ERR_INVALID_ARG;
}

extern "C" gsc_status gsc_scene_read_info(const char* path, gsc_stream_table* table, int32_t* has_pos) {
  if (!path || !table) return GSC_ERR_INVALID_ARG;
  FILE* f = fopen(path, "rb");
  if (!f) return GSC_ERR_INVALID_ARG;
  FileHeader h;
  gsc_status rc = read_header(f, &h);
  fclose(f);
  if (rc != GSC_OK) return rc;
  *table = h.table;
  if (has_pos) *has_pos = h.pos_bytes != 0;
  return GSC_OK;
}

extern "C" gsc_status gsc_scene_read(const char* path, gsc_stream_table* table, uint8_t* blocks, size_t blocks_cap,
                                     int32_t* perm, size_t perm_bytes_cap, float* pos, size_t pos_bytes_cap) {
  GscRange gsc_range_("gsc_scene_read");
  if (!path || !table) return GSC_ERR_INVALID_ARG;
  FILE* f = fopen(path, "rb");
  if (!f) return GSC_ERR_INVALID_ARG;
  FileHeader h;
  gsc_status rc = read_header(f, &h);
  std::vector<uint8_t> buf;
  if (rc == GSC_OK) {
    if ((h.blocks_bytes && (!blocks || blocks_cap < h.blocks_bytes)) ||
        (h.perm_bytes && (!perm || perm_bytes_cap < h.perm_bytes)) || (pos && pos_bytes_cap < h.pos_bytes) ||
        (pos && h.pos_bytes == 0))
      rc = GSC_ERR_INVALID_ARG;
  }
  if (rc == GSC_OK) {
    const size_t total = (size_t)(h.blocks_bytes + h.perm_bytes + h.pos_bytes);
    buf.resize(total + 1);
    if (total && fread(buf.data(), 1, total, f) != total) rc = GSC_ERR_INVALID_ARG;
    uint8_t extra;
    if (rc == GSC_OK && fread(&extra, 1, 1, f) != 0) rc = GSC_ERR_INVALID_ARG;  // trailing bytes
    if (rc == GSC_OK) {
      uint64_t c = 0xCBF29CE484222325ull;
      c = fnv1a(c, buf.data(), total);
      if (c != h.checksum) rc = GSC_ERR_INVALID_ARG;
    }
  }
  fclose(f);
  if (rc != GSC_OK) return rc;
  rc = from_host(blocks, buf.data(), h.blocks_bytes);
  if (rc == GSC_OK) rc = from_host(perm, buf.data() + h.blocks_bytes, h.perm_bytes);
  if (rc == GSC_OK && pos) rc = from_host(pos, buf.data() + h.blocks_bytes + h.perm_bytes, h.pos_bytes);
  if (rc == GSC_OK) *table = h.table;
  return rc;
}

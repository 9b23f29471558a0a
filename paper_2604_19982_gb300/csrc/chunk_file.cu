// Out-of-core chunks: a set streamed from chunk files on local storage,
// read ahead by a thread of its own while the join works on earlier chunks.
// The paper streams R from host memory (section 3.2, Algorithm 3) and names
// facets kept on disk as future work; here a chunk file holds exactly what a
// pj_mesh_set_desc describes, and a chunk source is a pj_fill_fn over such
// files for pj_load_set_streamed.  Host code only: nothing here touches the
// GPU.
//
// File layout (little-endian): a 1,024-byte header (magic "PJCHUNK1",
// version, object and LoD counts, per LoD the vertex, face-row and facet
// counts, whether the faces are a shared template, which of hd / ph are
// present, and the byte offset of every array), then the arrays, each at a
// 64-byte aligned offset.
//
// Reading: a source keeps readahead + 2 chunk buffers.  The join holds the
// arrays of chunk c until it asks for chunk c + 2 (the pageable-array
// contract of pj_load_set_streamed), so when chunk c is asked for the
// buffer of chunk c - 2 is free again and the reader thread may load up to
// chunk c + readahead.  A request that does not continue the previous one
// (the next join over the same set starts again at chunk 0) restarts the
// reader at that chunk.
#include <fcntl.h>
#include <sys/stat.h>
#include <unistd.h>

#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/pj.h"

namespace {

constexpr char MAGIC[8] = {'P', 'J', 'C', 'H', 'U', 'N', 'K', '1'};
constexpr uint32_t VERSION = 1;
constexpr size_t HEADER_BYTES = 1024;
constexpr size_t ALIGN = 64;

struct LodHdr {
  int64_t nv;          // vertices
  int64_t face_rows;   // rows of the faces array
  int64_t n_facets;    // facets of the LoD over all objects (length of hd / ph)
  int32_t shared;      // 1: faces is one template shared by every object
  int32_t n_faces_shared;
  int32_t has_hd, has_ph;
  uint64_t off_verts, off_vert_off, off_faces, off_face_off, off_hd, off_ph;
};

struct Header {
  char magic[8];
  uint32_t version;
  int32_t n_objects;
  int32_t n_lods;
  int32_t reserved;
  LodHdr lod[PJ_MAX_LODS];
  uint64_t off_anchor;
  uint64_t file_bytes;
};
static_assert(sizeof(Header) <= HEADER_BYTES, "chunk file header");

size_t up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

bool bad(std::string* why, const char* msg) {
  *why = msg;
  return false;
}

// The header of a desc, with every array's offset laid out; false (and a
// message) when the desc is inconsistent.
bool layout(const pj_mesh_set_desc* d, Header* h, std::string* why) {
  memset(h, 0, sizeof *h);
  memcpy(h->magic, MAGIC, 8);
  h->version = VERSION;
  const int n = d->n_objects, L = d->n_lods;
  if (n < 0 || L < 1 || L > PJ_MAX_LODS) return bad(why, "n_objects < 0 or n_lods outside 1..PJ_MAX_LODS");
  if (n > 0 && !d->anchor) return bad(why, "anchor is NULL");
  h->n_objects = n;
  h->n_lods = L;
  size_t off = HEADER_BYTES;
  for (int l = 0; l < L; ++l) {
    LodHdr& e = h->lod[l];
    if (!d->vert_off[l] || (n > 0 && (!d->verts[l] || !d->faces[l])))
      return bad(why, "verts / vert_off / faces of a LoD is NULL");
    const int64_t* vo = d->vert_off[l];
    if (vo[0] != 0) return bad(why, "vert_off must start at 0");
    for (int o = 0; o < n; ++o)
      if (vo[o + 1] < vo[o]) return bad(why, "vert_off not non-decreasing");
    e.nv = vo[n];
    e.shared = d->face_off[l] == nullptr;
    if (e.shared) {
      e.n_faces_shared = d->n_faces_shared[l];
      if (n > 0 && e.n_faces_shared <= 0) return bad(why, "shared topology needs n_faces_shared > 0");
      e.face_rows = n > 0 ? e.n_faces_shared : 0;
      e.n_facets = (int64_t)n * e.n_faces_shared;
    } else {
      const int64_t* fo = d->face_off[l];
      if (fo[0] != 0) return bad(why, "face_off must start at 0");
      for (int o = 0; o < n; ++o)
        if (fo[o + 1] < fo[o]) return bad(why, "face_off not non-decreasing");
      e.face_rows = fo[n];
      e.n_facets = fo[n];
    }
    e.has_hd = d->hd[l] != nullptr;
    e.has_ph = d->ph[l] != nullptr;
    e.off_verts = off;
    off = up(off + (size_t)e.nv * 12);
    e.off_vert_off = off;
    off = up(off + ((size_t)n + 1) * 8);
    e.off_faces = off;
    off = up(off + (size_t)e.face_rows * 12);
    if (!e.shared) {
      e.off_face_off = off;
      off = up(off + ((size_t)n + 1) * 8);
    }
    if (e.has_hd) {
      e.off_hd = off;
      off = up(off + (size_t)e.n_facets * 4);
    }
    if (e.has_ph) {
      e.off_ph = off;
      off = up(off + (size_t)e.n_facets * 4);
    }
  }
  h->off_anchor = off;
  off = up(off + (size_t)n * 12);
  h->file_bytes = off;
  return true;
}

// Every offset and size of a header read from a file lies inside the file.
bool check_header(const Header& h, uint64_t file_bytes, std::string* why) {
  if (memcmp(h.magic, MAGIC, 8) != 0) return bad(why, "not a chunk file (magic)");
  if (h.version != VERSION) return bad(why, "unsupported chunk file version");
  if (h.n_objects < 0 || h.n_lods < 1 || h.n_lods > PJ_MAX_LODS) return bad(why, "bad object or LoD count");
  if (h.file_bytes != file_bytes) return bad(why, "chunk file size differs from its header");
  const uint64_t n = (uint64_t)h.n_objects;
  auto in = [&](uint64_t off, uint64_t bytes) { return off >= HEADER_BYTES && off <= file_bytes && bytes <= file_bytes - off; };
  for (int l = 0; l < h.n_lods; ++l) {
    const LodHdr& e = h.lod[l];
    if (e.nv < 0 || e.face_rows < 0 || e.n_facets < 0) return bad(why, "negative count");
    if (e.shared ? e.n_facets != (int64_t)n * e.n_faces_shared : e.n_facets != e.face_rows)
      return bad(why, "facet count inconsistent with the faces");
    if (!in(e.off_verts, (uint64_t)e.nv * 12) || !in(e.off_vert_off, (n + 1) * 8) ||
        !in(e.off_faces, (uint64_t)e.face_rows * 12) || (!e.shared && !in(e.off_face_off, (n + 1) * 8)) ||
        (e.has_hd && !in(e.off_hd, (uint64_t)e.n_facets * 4)) || (e.has_ph && !in(e.off_ph, (uint64_t)e.n_facets * 4)))
      return bad(why, "an array lies outside the chunk file");
  }
  if (!in(h.off_anchor, n * 12)) return bad(why, "anchor lies outside the chunk file");
  return true;
}

bool pwrite_all(int fd, const void* p, size_t bytes, uint64_t off) {
  const char* c = static_cast<const char*>(p);
  while (bytes > 0) {
    ssize_t w = pwrite(fd, c, bytes, (off_t)off);
    if (w <= 0) return false;
    c += w;
    bytes -= (size_t)w;
    off += (uint64_t)w;
  }
  return true;
}

bool pread_all(int fd, void* p, size_t bytes, uint64_t off) {
  char* c = static_cast<char*>(p);
  while (bytes > 0) {
    ssize_t r = pread(fd, c, bytes, (off_t)off);
    if (r <= 0) return false;
    c += r;
    bytes -= (size_t)r;
    off += (uint64_t)r;
  }
  return true;
}

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

// A chunk source (see pj_chunk_source_open).
struct pj_chunk_source {
  struct Slot {
    unsigned char* buf = nullptr;
    size_t cap = 0;
    int chunk = -1;         // the chunk the buffer holds (or is being read into)
    uint64_t gen = 0;       // reader generation that filled it
    bool ready = false;
    pj_status st = PJ_OK;
  };
  std::vector<std::string> paths;
  std::vector<Header> hdr;
  int n_chunks = 0;
  int readahead = 2;
  int64_t n_objects = 0;
  std::vector<Slot> slot;
  std::thread reader;
  std::mutex mu;
  std::condition_variable cv;
  uint64_t gen = 0;         // bumped at every restart
  int next_read = 0;        // next chunk the reader loads
  int last = -1;            // the last chunk handed out
  int released = -2;        // chunks up to this one are no longer needed
  bool reading = false;     // the reader is inside a read
  bool stop = false;
  // statistics
  uint64_t bytes_read = 0;
  int64_t chunks_read = 0, restarts = 0;
  double ms_read = 0, ms_wait = 0;
  std::string error;

  // chunk x goes to buffer x % slots, whose previous chunk x - slots must
  // be released
  bool may_load(int x) const { return x < n_chunks && x - (int)slot.size() <= released; }

  void run() {
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      cv.wait(lk, [&] { return stop || may_load(next_read); });
      if (stop) return;
      const int c = next_read++;
      const uint64_t g = gen;
      Slot& sl = slot[(size_t)c % slot.size()];
      sl.chunk = c;
      sl.gen = g;
      sl.ready = false;
      reading = true;
      lk.unlock();
      const double t0 = now_ms();
      pj_status st = load(c, sl);
      const double t1 = now_ms();
      lk.lock();
      reading = false;
      sl.st = st;
      sl.ready = true;
      ms_read += t1 - t0;
      if (st == PJ_OK) {
        bytes_read += hdr[(size_t)c].file_bytes;
        ++chunks_read;
      }
      cv.notify_all();
    }
  }

  // read chunk c into sl (outside the lock: no other thread touches the
  // buffer of a chunk being read)
  pj_status load(int c, Slot& sl) {
    const size_t bytes = hdr[(size_t)c].file_bytes;
    if (sl.cap < bytes) {
      free(sl.buf);
      sl.buf = nullptr;
      sl.cap = 0;
      void* p = nullptr;
      if (posix_memalign(&p, 4096, bytes) != 0) return PJ_ENOMEM;
      sl.buf = static_cast<unsigned char*>(p);
      sl.cap = bytes;
    }
    const int fd = open(paths[(size_t)c].c_str(), O_RDONLY);
    if (fd < 0) return PJ_ESOURCE;
#ifdef POSIX_FADV_SEQUENTIAL
    (void)posix_fadvise(fd, 0, 0, POSIX_FADV_SEQUENTIAL);
#endif
    const bool ok = pread_all(fd, sl.buf, bytes, 0);
    close(fd);
    if (!ok) return PJ_ESOURCE;
    Header h;
    memcpy(&h, sl.buf, sizeof h);
    if (memcmp(&h, &hdr[(size_t)c], sizeof h) != 0) return PJ_ESOURCE;   // changed since it was opened
    return PJ_OK;
  }

  pj_status fill(int c, pj_mesh_set_desc* out) {
    if (c < 0 || c >= n_chunks || !out) return PJ_EINVAL;
    std::unique_lock<std::mutex> lk(mu);
    if (c != last + 1) {
      // a new pass (or a jump): wait for a read in flight, then restart at c
      cv.wait(lk, [&] { return !reading; });
      ++gen;
      ++restarts;
      for (Slot& sl : slot) {
        sl.chunk = -1;
        sl.ready = false;
      }
      next_read = c;
      last = c - 1;
      released = c - 1;   // every buffer is free
      cv.notify_all();
    }
    // asking for chunk c releases chunk c - 2
    if (c - 2 > released) {
      released = c - 2;
      cv.notify_all();
    }
    Slot& sl = slot[(size_t)c % slot.size()];
    const double t0 = now_ms();
    cv.wait(lk, [&] { return sl.chunk == c && sl.gen == gen && sl.ready; });
    ms_wait += now_ms() - t0;
    if (sl.st != PJ_OK) return sl.st;
    last = c;
    const Header& h = hdr[(size_t)c];
    memset(out, 0, sizeof *out);
    out->n_objects = h.n_objects;
    out->n_lods = h.n_lods;
    unsigned char* b = sl.buf;
    for (int l = 0; l < h.n_lods; ++l) {
      const LodHdr& e = h.lod[l];
      out->verts[l] = reinterpret_cast<const float*>(b + e.off_verts);
      out->vert_off[l] = reinterpret_cast<const int64_t*>(b + e.off_vert_off);
      out->faces[l] = reinterpret_cast<const int32_t*>(b + e.off_faces);
      out->face_off[l] = e.shared ? nullptr : reinterpret_cast<const int64_t*>(b + e.off_face_off);
      out->n_faces_shared[l] = e.shared ? e.n_faces_shared : 0;
      out->hd[l] = e.has_hd ? reinterpret_cast<const float*>(b + e.off_hd) : nullptr;
      out->ph[l] = e.has_ph ? reinterpret_cast<const float*>(b + e.off_ph) : nullptr;
    }
    out->anchor = reinterpret_cast<const float*>(b + h.off_anchor);
    return PJ_OK;
  }

  ~pj_chunk_source() {
    {
      std::lock_guard<std::mutex> lk(mu);
      stop = true;
    }
    cv.notify_all();
    if (reader.joinable()) reader.join();
    for (Slot& sl : slot) free(sl.buf);
  }
};

extern "C" {

pj_status pj_chunk_file_write(const char* path, const pj_mesh_set_desc* desc) {
  if (!path || !desc) return PJ_EINVAL;
  Header h;
  std::string why;
  if (!layout(desc, &h, &why)) return PJ_EINVAL;
  const std::string tmp = std::string(path) + ".part";
  const int fd = open(tmp.c_str(), O_WRONLY | O_CREAT | O_TRUNC, 0644);
  if (fd < 0) return PJ_ESOURCE;
  std::vector<unsigned char> head(HEADER_BYTES, 0);
  memcpy(head.data(), &h, sizeof h);
  const int n = desc->n_objects;
  bool ok = pwrite_all(fd, head.data(), head.size(), 0);
  for (int l = 0; ok && l < desc->n_lods; ++l) {
    const LodHdr& e = h.lod[l];
    ok = ok && pwrite_all(fd, desc->verts[l], (size_t)e.nv * 12, e.off_verts);
    ok = ok && pwrite_all(fd, desc->vert_off[l], ((size_t)n + 1) * 8, e.off_vert_off);
    ok = ok && pwrite_all(fd, desc->faces[l], (size_t)e.face_rows * 12, e.off_faces);
    if (!e.shared) ok = ok && pwrite_all(fd, desc->face_off[l], ((size_t)n + 1) * 8, e.off_face_off);
    if (e.has_hd) ok = ok && pwrite_all(fd, desc->hd[l], (size_t)e.n_facets * 4, e.off_hd);
    if (e.has_ph) ok = ok && pwrite_all(fd, desc->ph[l], (size_t)e.n_facets * 4, e.off_ph);
  }
  ok = ok && pwrite_all(fd, desc->anchor, (size_t)n * 12, h.off_anchor);
  ok = ok && ftruncate(fd, (off_t)h.file_bytes) == 0;
  ok = (close(fd) == 0) && ok;
  if (!ok || rename(tmp.c_str(), path) != 0) {
    unlink(tmp.c_str());
    return PJ_ESOURCE;
  }
  return PJ_OK;
}

pj_status pj_chunk_source_open(const char* const* paths, int n_chunks, int readahead, pj_chunk_source** out) {
  if (!out) return PJ_EINVAL;
  *out = nullptr;
  if (!paths || n_chunks < 1 || readahead < 0 || readahead > 16) return PJ_EINVAL;
  pj_chunk_source* s = new (std::nothrow) pj_chunk_source();
  if (!s) return PJ_ENOMEM;
  s->n_chunks = n_chunks;
  s->readahead = readahead;
  int L = -1;
  for (int c = 0; c < n_chunks; ++c) {
    if (!paths[c]) {
      delete s;
      return PJ_EINVAL;
    }
    s->paths.emplace_back(paths[c]);
    const int fd = open(paths[c], O_RDONLY);
    struct stat sb;
    Header h;
    std::string why;
    const bool ok = fd >= 0 && fstat(fd, &sb) == 0 && (uint64_t)sb.st_size >= HEADER_BYTES &&
                    pread_all(fd, &h, sizeof h, 0) && check_header(h, (uint64_t)sb.st_size, &why);
    if (fd >= 0) close(fd);
    if (!ok || (L >= 0 && h.n_lods != L)) {
      delete s;
      return fd < 0 ? PJ_ESOURCE : PJ_EINVAL;
    }
    L = h.n_lods;
    s->hdr.push_back(h);
    s->n_objects += h.n_objects;
  }
  s->slot.resize((size_t)readahead + 2);
  try {
    s->reader = std::thread([s] { s->run(); });
  } catch (...) {
    delete s;
    return PJ_ENOMEM;
  }
  *out = s;
  return PJ_OK;
}

pj_status pj_chunk_source_info(const pj_chunk_source* src, int64_t* n_objects, int* n_chunks, int* n_lods) {
  if (!src) return PJ_EINVAL;
  if (n_objects) *n_objects = src->n_objects;
  if (n_chunks) *n_chunks = src->n_chunks;
  if (n_lods) *n_lods = src->hdr.empty() ? 0 : src->hdr[0].n_lods;
  return PJ_OK;
}

pj_status pj_chunk_source_fill(void* src, int chunk, pj_mesh_set_desc* out) {
  if (!src) return PJ_EINVAL;
  return static_cast<pj_chunk_source*>(src)->fill(chunk, out);
}

pj_status pj_chunk_source_stats(pj_chunk_source* src, char* json_buf, size_t cap) {
  if (!src || !json_buf || cap == 0) return PJ_EINVAL;
  std::lock_guard<std::mutex> lk(src->mu);
  const int w = snprintf(json_buf, cap,
                         "{\"chunks_read\": %lld, \"bytes_read\": %llu, \"ms_read\": %.3f, \"read_gbs\": %.3f, "
                         "\"ms_fill_wait\": %.3f, \"restarts\": %lld, \"buffers\": %d}",
                         (long long)src->chunks_read, (unsigned long long)src->bytes_read, src->ms_read,
                         src->ms_read > 0 ? src->bytes_read / (src->ms_read * 1e6) : 0.0, src->ms_wait,
                         (long long)src->restarts, (int)src->slot.size());
  return (w < 0 || (size_t)w >= cap) ? PJ_EINVAL : PJ_OK;
}

void pj_chunk_source_close(pj_chunk_source* src) { delete src; }

}  // extern "C"

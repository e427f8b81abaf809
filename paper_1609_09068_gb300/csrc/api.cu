// api.cu -- the extern "C" entry points declared in include/prgb.h.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include <map>
#include <mutex>
#include <new>

#include "common.cuh"
#include "global.cuh"
#include "solve.cuh"

namespace prgb {
int last_cuda_error();
void set_wait_limit_us(unsigned int us);
pr_status build_layout(pr_partition_s* P, const int32_t* crep, const int32_t* wave, int32_t max_wave, Arena& tmp,
                       Ctl* ctl);
pr_status graph_digest(const DevGraph& g, Arena& tmp, uint64_t* out);
pr_status partition_digest(int32_t n, const int32_t* comp, const uint8_t* type, const int32_t* level,
                           const int32_t* wave, int32_t n_comp, int32_t n_levels, int32_t max_wave, bool check,
                           Arena& tmp, Ctl* ctl, uint64_t* out);
pr_status smallest_members(int32_t n, int32_t n_comp, const int32_t* comp, int32_t* crep, Arena& tmp);
pr_status check_same_ids(int32_t n, const int32_t* a, const int32_t* b, Ctl* ctl, cudaStream_t s);

// keep freed stream-ordered memory cached in the device's default pool so
// repeated calls do not return it to the CUDA driver
static void tune_pool() {
  static bool done[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  done[dev] = true;
}

// CUDA events between the phases of a partition (PR_PARTITION_TIMING); a
// no-op when off
struct PhaseEvents {
  bool on;
  cudaEvent_t e[7] = {};
  explicit PhaseEvents(bool want) : on(want) {}
  ~PhaseEvents() {
    for (cudaEvent_t x : e)
      if (x) cudaEventDestroy(x);
  }
  pr_status start(cudaStream_t s) {
    if (!on) return PR_OK;
    for (cudaEvent_t& x : e) {
      PRGB_CUDA(cudaEventCreate(&x));
      PRGB_CUDA(cudaEventRecord(x, s));
    }
    return PR_OK;
  }
  pr_status mark(int i, cudaStream_t s) {
    if (on) PRGB_CUDA(cudaEventRecord(e[i], s));
    return PR_OK;
  }
  // after the stream has synchronised: trim, giant, colouring, levels,
  // layout, total
  pr_status read(float* ms) {
    PRGB_CUDA(cudaEventSynchronize(e[6]));
    for (int i = 0; i < 5; i++) PRGB_CUDA(cudaEventElapsedTime(&ms[i], e[i], e[i + 1]));
    PRGB_CUDA(cudaEventElapsedTime(&ms[5], e[0], e[6]));
    return PR_OK;
  }
};

static pr_status copy_waves(int32_t (*dst)[2], const Ctl* ctl) {
  PRGB_CUDA(cudaMemcpy(dst, ctl->waves, 5 * 2 * sizeof(int32_t), cudaMemcpyDeviceToHost));
  return PR_OK;
}

static pr_status finish_sync(cudaStream_t s, Ctl* ctl, int* flags_out) {
  int h[2] = {0, 0};
  PRGB_CUDA(cudaMemcpyAsync(&h[0], &ctl->err, 4, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaMemcpyAsync(&h[1], &ctl->flags[0], 4, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaStreamSynchronize(s));
  if (flags_out) *flags_out = h[1];
  return (pr_status)h[0];
}

// The header of a partition file (pr_partition_save); host byte order,
// which is little endian on every host this library builds for.
struct PartFileHeader {
  char magic[8];
  uint32_t version;
  uint32_t header_bytes;
  int64_t n;
  int64_t m;
  uint64_t graph_digest;
  uint64_t part_digest;
  int32_t n_comp;
  int32_t n_levels;
  int32_t max_wave;
  int32_t zero;
};
static_assert(sizeof(PartFileHeader) == 64, "the partition file header is 64 bytes");
static const char kPartMagic[8] = {'P', 'R', 'G', 'B', 'P', 'A', 'R', 'T'};
constexpr uint32_t kPartVersion = 1;

// the arrays' digest with the header's three counts folded in, so that a
// damaged count is refused like a damaged array entry
static uint64_t counts_digest(uint64_t arrays, int32_t n_comp, int32_t n_levels, int32_t max_wave) {
  const uint64_t counts[3] = {(uint32_t)n_comp, (uint32_t)n_levels, (uint32_t)max_wave};
  uint64_t x = arrays;
  for (uint64_t v : counts) x ^= v + 0x9E3779B97F4A7C15ull + (x << 6) + (x >> 2);
  return x;
}

struct FileCloser {
  FILE* f;
  ~FileCloser() {
    if (f) fclose(f);
  }
};

// a host staging buffer of at most 64 MiB for the copies between a file and
// device arrays of `bytes` bytes
struct IoBuf {
  char* p = nullptr;
  size_t size = 0;
  explicit IoBuf(size_t bytes) {
    size = std::min(bytes, (size_t)64 << 20);
    if (size < 16) size = 16;
    p = new (std::nothrow) char[size];
  }
  ~IoBuf() { delete[] p; }
};

static pr_status write_dev(FILE* f, const void* d, size_t bytes, IoBuf& b, cudaStream_t s) {
  for (size_t o = 0; o < bytes; o += b.size) {
    const size_t k = std::min(b.size, bytes - o);
    PRGB_CUDA(cudaMemcpyAsync(b.p, (const char*)d + o, k, cudaMemcpyDeviceToHost, s));
    PRGB_CUDA(cudaStreamSynchronize(s));
    if (fwrite(b.p, 1, k, f) != k) return PR_EINVAL;
  }
  return PR_OK;
}

static pr_status read_dev(FILE* f, void* d, size_t bytes, IoBuf& b, cudaStream_t s) {
  for (size_t o = 0; o < bytes; o += b.size) {
    const size_t k = std::min(b.size, bytes - o);
    if (fread(b.p, 1, k, f) != k) return PR_EINVAL;
    PRGB_CUDA(cudaMemcpyAsync((char*)d + o, b.p, k, cudaMemcpyHostToDevice, s));
    PRGB_CUDA(cudaStreamSynchronize(s));
  }
  return PR_OK;
}

}  // namespace prgb

using namespace prgb;

extern "C" {

const char* pr_status_str(pr_status s) {
  switch (s) {
    case PR_OK: return "ok";
    case PR_EINVAL: return "invalid argument";
    case PR_ENOMEM: return "out of device memory";
    case PR_ECUDA: return "CUDA runtime error";
    case PR_ENOCONV: return "not converged within max_iter";
    case PR_ETIMEOUT: return "device-side wait timed out";
    case PR_EINTERNAL: return "internal error";
  }
  return "unknown status";
}

int pr_last_cuda_error(void) { return prgb::last_cuda_error(); }

pr_status pr_last_device_error(void) { return prgb::take_last_status(); }

int64_t pr_launch_count(void) { return (int64_t)prgb::launch_count(); }

pr_status pr_set_wait_limit(uint32_t microseconds) {
  prgb::set_wait_limit_us(microseconds);
  return PR_OK;
}

static pr_status pr_graph_create_body(const pr_csr* csr, uint32_t flags, void* stream, pr_graph** out) {
  if (!out) return PR_EINVAL;
  *out = nullptr;
  if (flags & ~(uint32_t)PR_CANONICALIZE) return PR_EINVAL;
  if (!csr || csr->n < 0 || csr->nnz < 0 || csr->nnz >= ((int64_t)1 << 31)) return PR_EINVAL;
  if (csr->n > 0 && (!csr->rowptr || (csr->nnz > 0 && !csr->col))) return PR_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  tune_pool();
  pr_graph_s* G = new (std::nothrow) pr_graph_s;
  if (!G) return PR_ENOMEM;
  G->stream = s;
  G->keep = new (std::nothrow) Arena(s);
  if (!G->keep) {
    delete G;
    return PR_ENOMEM;
  }
  pr_status st;
  {
    Arena tmp(s);
    Ctl* ctl = nullptr;
    st = tmp.alloc(&ctl, 1);
    if (st == PR_OK) {
      st = init_ctl(ctl, s);
      if (st == PR_OK) st = ingest(csr, flags, &G->g, *G->keep, tmp, ctl);
    }
    if (st == PR_OK) {
      int e = 0;
      st = finish_sync(s, ctl, &e);
    }
  }
  if (st != PR_OK) {
    delete G->keep;
    delete G;
    return st;
  }
  *out = G;
  return PR_OK;
}

pr_status pr_graph_create(const pr_csr* csr, void* stream, pr_graph** out) {
  return prgb::note_status(pr_graph_create_body(csr, 0, stream, out));
}

pr_status pr_graph_create_ex(const pr_csr* csr, uint32_t flags, void* stream, pr_graph** out) {
  prgb::NvtxRange nvtx("prgb graph_create");
  return prgb::note_status(pr_graph_create_body(csr, flags, stream, out));
}

void pr_graph_destroy(pr_graph* g) {
  if (!g) return;
  delete g->keep;
  delete g;
}

// The end of creating or loading a partition: the class boundary and grid
// shape an earlier tuning chose, or the partition released on failure.
static pr_status finish_partition(pr_partition_s* P, pr_status st, pr_partition** out) {
  if (st == PR_OK) {
    int32_t tc = kCtaCompMax, tb = 4, tl = 1;
    tuned_defaults(&tc, &tb, &tl);
    if (tc != P->cta_max || tb != P->coop_blocks || tl != P->balance) retune_levels(P, tc, tb, tl);
    else split_fx_ranges(P);
  }
  if (st != PR_OK) {
    delete P->keep;
    delete P;
    return st;
  }
  *out = P;
  return PR_OK;
}

static pr_status pr_partition_create_body(const pr_graph* g, uint32_t flags, void* stream, pr_partition** out) {
  if (!out) return PR_EINVAL;
  *out = nullptr;
  if (!g || (flags & ~PR_PARTITION_TIMING) != 0) return PR_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  tune_pool();
  pr_partition_s* P = new (std::nothrow) pr_partition_s;
  if (!P) return PR_ENOMEM;
  P->stream = s;
  P->keep = new (std::nothrow) Arena(s);
  if (!P->keep) {
    delete P;
    return PR_ENOMEM;
  }
  P->g = g->g;
  const int32_t n = P->g.n;
  pr_status st = PR_OK;
  {
    Arena tmp(s);
    Ctl* ctl = nullptr;
    int32_t *rep = nullptr, *crep = nullptr;
    int32_t max_wave = 0;
    if (st == PR_OK) st = tmp.alloc(&ctl, 1);
    if (st == PR_OK) st = P->keep->alloc(&P->comp_id, (size_t)n);
    if (st == PR_OK) st = P->keep->alloc(&P->type, (size_t)n);
    if (st == PR_OK) st = P->keep->alloc(&P->level, (size_t)n);
    if (st == PR_OK) st = tmp.alloc(&rep, (size_t)n);
    if (st == PR_OK) st = tmp.alloc(&crep, (size_t)n);
    if (st == PR_OK) st = P->keep->alloc(&P->wave, (size_t)n);
    int32_t* wave = P->wave;
    if (st == PR_OK) st = init_ctl(ctl, s);
    if (st == PR_OK && cudaMemsetAsync(ctl->waves, 0, sizeof(ctl->waves), s) != cudaSuccess) st = PR_ECUDA;
    // phase events: 0 start, 1 trim, 2 giant, 3 colouring, 4 levels,
    // 5 layout, 6 end; all recorded at the start, so a phase that does not
    // run reads 0 ms
    PhaseEvents ev(flags & PR_PARTITION_TIMING);
    if (st == PR_OK) st = ev.start(s);
    if (st == PR_OK) {
      NvtxRange r("prgb scc");
      st = scc_detect(P->g, rep, tmp, ctl, ev.on ? ev.e + 1 : nullptr, &P->colour_rounds);
    }
    if (st == PR_OK) st = ev.mark(3, s);
    if (st == PR_OK) {
      NvtxRange r("prgb levels");
      st = levels_and_merge(P->g, rep, crep, P->level, P->type, wave, &max_wave, tmp, ctl);
    }
    if (st == PR_OK) st = ev.mark(4, s);
    P->max_wave = max_wave;
    if (st == PR_OK) {
      NvtxRange r("prgb layout");
      st = build_layout(P, crep, wave, max_wave, tmp, ctl);
    }
    if (st == PR_OK) st = ev.mark(5, s);
    if (st == PR_OK) st = finish_sync(s, ctl, nullptr);
    if (st == PR_OK) st = ev.mark(6, s);
    if (st == PR_OK && ev.on) {
      P->timed = true;
      st = ev.read(P->phase_ms);
      if (st == PR_OK) st = copy_waves(P->waves, ctl);
    }
  }
  return finish_partition(P, st, out);
}

pr_status pr_partition_create(const pr_graph* g, uint32_t flags, void* stream, pr_partition** out) {
  prgb::NvtxRange nvtx("prgb partition");
  return prgb::note_status(pr_partition_create_body(g, flags, stream, out));
}

static pr_status pr_partition_save_body(const pr_partition* part, const char* path, void* stream) {
  if (!part || !path) return PR_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const pr_partition_s* P = part;
  const int32_t n = P->g.n;
  PartFileHeader h = {};
  memcpy(h.magic, kPartMagic, sizeof(h.magic));
  h.version = kPartVersion;
  h.header_bytes = sizeof(h);
  h.n = n;
  h.m = P->g.m;
  h.n_comp = P->n_comp;
  h.n_levels = P->n_levels;
  h.max_wave = P->max_wave;
  {
    Arena tmp(s);
    Ctl* ctl = nullptr;
    PRGB_TRY(tmp.alloc(&ctl, 1));
    PRGB_TRY(init_ctl(ctl, s));
    PRGB_TRY(graph_digest(P->g, tmp, &h.graph_digest));
    uint64_t pd = 0;
    PRGB_TRY(partition_digest(n, P->comp_id, P->type, P->level, P->wave, P->n_comp, P->n_levels, P->max_wave, false,
                              tmp, ctl, &pd));
    h.part_digest = counts_digest(pd, h.n_comp, h.n_levels, h.max_wave);
  }
  IoBuf b((size_t)n * 4);
  if (!b.p) return PR_ENOMEM;
  FILE* f = fopen(path, "wb");
  if (!f) return PR_EINVAL;
  pr_status st = fwrite(&h, sizeof(h), 1, f) == 1 ? PR_OK : PR_EINVAL;
  if (st == PR_OK) st = write_dev(f, P->comp_id, (size_t)n * 4, b, s);
  if (st == PR_OK) st = write_dev(f, P->level, (size_t)n * 4, b, s);
  if (st == PR_OK) st = write_dev(f, P->wave, (size_t)n * 4, b, s);
  if (st == PR_OK) st = write_dev(f, P->type, (size_t)n, b, s);
  if (fclose(f) != 0 && st == PR_OK) st = PR_EINVAL;
  if (st != PR_OK) remove(path);
  return st;
}

pr_status pr_partition_save(const pr_partition* part, const char* path, void* stream) {
  prgb::NvtxRange nvtx("prgb partition_save");
  return prgb::note_status(pr_partition_save_body(part, path, stream));
}

static pr_status pr_partition_load_body(const pr_graph* g, const char* path, uint32_t flags, void* stream,
                                        pr_partition** out) {
  if (!out) return PR_EINVAL;
  *out = nullptr;
  if (!g || !path || flags != 0) return PR_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  tune_pool();
  FileCloser fc{fopen(path, "rb")};
  if (!fc.f) return PR_EINVAL;
  PartFileHeader h;
  if (fread(&h, sizeof(h), 1, fc.f) != 1) return PR_EINVAL;
  const int32_t n = g->g.n;
  if (memcmp(h.magic, kPartMagic, sizeof(h.magic)) != 0 || h.version != kPartVersion ||
      h.header_bytes != sizeof(h) || h.n != n || h.m != g->g.m || h.zero != 0)
    return PR_EINVAL;
  // every vertex lies in one component of one level (none of either when n = 0)
  const int32_t lo = n > 0 ? 1 : 0;
  if (h.n_comp < lo || h.n_comp > n || h.n_levels < lo || h.n_levels > n || h.max_wave < 0) return PR_EINVAL;
  IoBuf b((size_t)n * 4);
  if (!b.p) return PR_ENOMEM;
  pr_partition_s* P = new (std::nothrow) pr_partition_s;
  if (!P) return PR_ENOMEM;
  P->stream = s;
  P->keep = new (std::nothrow) Arena(s);
  if (!P->keep) {
    delete P;
    return PR_ENOMEM;
  }
  P->g = g->g;
  P->max_wave = h.max_wave;
  pr_status st = PR_OK;
  {
    Arena tmp(s);
    Ctl* ctl = nullptr;
    int32_t *saved = nullptr, *crep = nullptr;
    uint64_t gd = 0, pd = 0;
    if (st == PR_OK) st = tmp.alloc(&ctl, 1);
    if (st == PR_OK) st = P->keep->alloc(&P->comp_id, (size_t)n);
    if (st == PR_OK) st = P->keep->alloc(&P->type, (size_t)n);
    if (st == PR_OK) st = P->keep->alloc(&P->level, (size_t)n);
    if (st == PR_OK) st = P->keep->alloc(&P->wave, (size_t)n);
    if (st == PR_OK) st = tmp.alloc(&saved, (size_t)n);
    if (st == PR_OK) st = tmp.alloc(&crep, (size_t)n);
    if (st == PR_OK) st = read_dev(fc.f, saved, (size_t)n * 4, b, s);
    if (st == PR_OK) st = read_dev(fc.f, P->level, (size_t)n * 4, b, s);
    if (st == PR_OK) st = read_dev(fc.f, P->wave, (size_t)n * 4, b, s);
    if (st == PR_OK) st = read_dev(fc.f, P->type, (size_t)n, b, s);
    if (st == PR_OK && fgetc(fc.f) != EOF) st = PR_EINVAL;
    if (st == PR_OK) st = init_ctl(ctl, s);
    if (st == PR_OK) st = graph_digest(P->g, tmp, &gd);
    if (st == PR_OK && gd != h.graph_digest) st = PR_EINVAL;
    if (st == PR_OK)
      st = partition_digest(n, saved, P->type, P->level, P->wave, h.n_comp, h.n_levels, h.max_wave, true, tmp, ctl,
                            &pd);
    // the range checks' result comes before any kernel indexes with the arrays
    if (st == PR_OK) st = finish_sync(s, ctl, nullptr);
    if (st == PR_OK && counts_digest(pd, h.n_comp, h.n_levels, h.max_wave) != h.part_digest) st = PR_EINVAL;
    if (st == PR_OK) st = smallest_members(n, h.n_comp, saved, crep, tmp);
    if (st == PR_OK) {
      NvtxRange r("prgb layout");
      st = build_layout(P, crep, P->wave, h.max_wave, tmp, ctl);
    }
    if (st == PR_OK && (P->n_comp != h.n_comp || P->n_levels != h.n_levels)) st = PR_EINVAL;
    if (st == PR_OK) st = check_same_ids(n, P->comp_id, saved, ctl, s);
    if (st == PR_OK) st = finish_sync(s, ctl, nullptr);
  }
  return finish_partition(P, st, out);
}

pr_status pr_partition_load(const pr_graph* g, const char* path, uint32_t flags, void* stream, pr_partition** out) {
  prgb::NvtxRange nvtx("prgb partition_load");
  return prgb::note_status(pr_partition_load_body(g, path, flags, stream, out));
}

pr_status pr_partition_timing_get(const pr_partition* part, pr_partition_timing* out) {
  if (!part || !out || !part->timed) return PR_EINVAL;
  out->trim_ms = part->phase_ms[0];
  out->giant_ms = part->phase_ms[1];
  out->colour_ms = part->phase_ms[2];
  out->levels_ms = part->phase_ms[3];
  out->layout_ms = part->phase_ms[4];
  out->total_ms = part->phase_ms[5];
  out->colour_rounds = part->colour_rounds;
  for (int k = 0; k < 5; k++)
    for (int j = 0; j < 2; j++) out->waves[k][j] = part->waves[k][j];
  return PR_OK;
}

static pr_status pr_partition_query_body(const pr_partition* part, int32_t* comp_id, uint8_t* type, int32_t* level,
                             int32_t* n_comp, int32_t* n_levels, void* stream) {
  if (!part) return PR_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)part->g.n;
  if (n > 0) {
    if (comp_id) PRGB_CUDA(cudaMemcpyAsync(comp_id, part->comp_id, n * 4, cudaMemcpyDeviceToDevice, s));
    if (type) PRGB_CUDA(cudaMemcpyAsync(type, part->type, n, cudaMemcpyDeviceToDevice, s));
    if (level) PRGB_CUDA(cudaMemcpyAsync(level, part->level, n * 4, cudaMemcpyDeviceToDevice, s));
  }
  if (n_comp) *n_comp = part->n_comp;
  if (n_levels) *n_levels = part->n_levels;
  return PR_OK;
}

pr_status pr_partition_query(const pr_partition* part, int32_t* comp_id, uint8_t* type, int32_t* level,
                             int32_t* n_comp, int32_t* n_levels, void* stream) {
  return prgb::note_status(pr_partition_query_body(part, comp_id, type, level, n_comp, n_levels, stream));
}

static pr_status pr_partition_info_body(const pr_partition* part, int32_t* n, int64_t* m, int32_t* n_comp,
                                        int32_t* n_levels, int32_t* n_scc, int32_t* n_scc_vertices) {
  if (!part) return PR_EINVAL;
  if (n) *n = part->g.n;
  if (m) *m = part->g.m;
  if (n_comp) *n_comp = part->n_comp;
  if (n_levels) *n_levels = part->n_levels;
  if (n_scc) *n_scc = part->n_scc;
  if (n_scc_vertices) *n_scc_vertices = part->n_scc_vertices;
  return PR_OK;
}

pr_status pr_partition_info(const pr_partition* part, int32_t* n, int64_t* m, int32_t* n_comp, int32_t* n_levels,
                            int32_t* n_scc, int32_t* n_scc_vertices) {
  return prgb::note_status(pr_partition_info_body(part, n, m, n_comp, n_levels, n_scc, n_scc_vertices));
}

void pr_partition_destroy(pr_partition* part) {
  if (!part) return;
  delete part->plan;
  delete part->keep;
  delete part;
}

static pr_status check_solve_args(double c, const double* u, double tol, const double* R) {
  if (!(c > 0.0 && c < 1.0) || !(tol > 0.0) || !isfinite(tol)) return PR_EINVAL;
  if (!u || !R) return PR_EINVAL;
  return PR_OK;
}

static pr_status pr_solve_body(const pr_partition* part, double c, const double* u, double tol,
                               const pr_solve_opts* opts, double* R, pr_solve_stats* stats, void* stream) {
  if (!part) return PR_EINVAL;
  const int32_t n = part->g.n;
  if (n > 0) PRGB_TRY(check_solve_args(c, u, tol, R));
  pr_solve_opts o = {PR_NORM_L1, 10000, PR_PREC_FP64, 0, nullptr, nullptr, 0};
  if (opts) o = *opts;
  if (o.max_iter <= 0) o.max_iter = 10000;
  if (fault_hit(kFaultNoconv)) o.max_iter = 1;
  if (o.norm != PR_NORM_L1 && o.norm != PR_NORM_LINF) return PR_EINVAL;
  if (o.precision != PR_PREC_FP64 && o.precision != PR_PREC_MIXED) return PR_EINVAL;
  const bool mixed = o.precision == PR_PREC_MIXED;
  if (mixed && (o.norm != PR_NORM_L1 || o.replay_iters)) return PR_EINVAL;
  if (o.warm_start && o.replay_iters) return PR_EINVAL;
  if (o.lu_threshold < 0 || o.lu_threshold > 129) return PR_EINVAL;
  if (o.replay_iters) {
    for (int32_t k = 0; k < part->n_comp; k++)
      if (o.replay_iters[k] < 0 || o.replay_iters[k] > 1000000) return PR_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int32_t K = part->n_comp;
  const bool timing = stats && stats->timing;
  const bool level_events = timing && stats->timing >= 2;
  Arena tmp(s);
  Ctl* ctl = nullptr;
  int32_t* iters = nullptr;
  int32_t* iters64 = nullptr;
  int64_t launches = 0;
  KernelTiming kt_local;
  kt_local.levels = level_events;
  KernelTiming* kt = &kt_local;
  pr_partition_s* P = const_cast<pr_partition_s*>(part);  // the plan is a cache
  std::unique_lock<std::mutex> lock(P->plan_mu, std::defer_lock);
  if (!o.replay_iters) {
    // the level loop replayed from the partition's cached CUDA graph
    lock.lock();
    SolvePlan* pl = nullptr;
    PRGB_TRY(plan_solve(P, c, u, o.io_on_host != 0, tol, o.norm, o.max_iter, mixed,
                        timing ? (level_events ? 2 : 1) : 0, o.warm_start,
                        o.lu_threshold, R, o.io_on_host != 0, s, &pl, &launches));
    ctl = pl->ctl;
    iters = pl->iters;
    iters64 = mixed ? pl->iters64 : nullptr;
    kt = &pl->kt;
  } else {
    // replayed iteration counts: buffers of its own, launched directly
    int32_t* replay = nullptr;
    const double* du = u;
    double* dR = R;
    PRGB_TRY(tmp.alloc(&ctl, 1));
    PRGB_TRY(init_ctl(ctl, s));
    PRGB_TRY(tmp.alloc(&iters, (size_t)K));
    if (K > 0) PRGB_CUDA(cudaMemsetAsync(iters, 0, (size_t)K * 4, s));
    if (K > 0) {
      PRGB_TRY(tmp.alloc(&replay, (size_t)K));
      PRGB_CUDA(cudaMemcpyAsync(replay, o.replay_iters, (size_t)K * 4, cudaMemcpyHostToDevice, s));
    }
    if (o.io_on_host && n > 0) {
      double *tu = nullptr, *tR = nullptr;
      PRGB_TRY(tmp.alloc(&tu, (size_t)n));
      PRGB_TRY(tmp.alloc(&tR, (size_t)n));
      PRGB_COPY(cudaMemcpyAsync(tu, u, (size_t)n * 8, cudaMemcpyHostToDevice, s));
      du = tu;
      dR = tR;
    }
    PRGB_TRY(run_solve(part, c, du, tol, o.norm, o.max_iter, replay, false, o.lu_threshold, dR, iters, nullptr, tmp,
                       ctl, &launches, timing ? kt : nullptr));
    if (o.io_on_host && n > 0) PRGB_COPY(cudaMemcpyAsync(R, dR, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
  }
  int flags = 0;
  PRGB_TRY(finish_sync(s, ctl, &flags));
  if (stats) {
    stats->n_levels = part->n_levels;
    stats->launches = launches;
    stats->iters_max = 0;
    stats->edge_visits = 0;
    stats->fp64_sweeps_max = 0;
    stats->fp64_edge_visits = 0;
    if (K > 0) {
      // per-component sweep counts: all of them, or (counts_off) only the
      // timed grid-wide components' for the byte count
      const bool counts = !stats->counts_off;
      std::map<int32_t, int32_t> hl;
      int32_t* h = stats->comp_iters;
      std::vector<int32_t> local, h64;
      if (counts) {
        if (!h) {
          local.resize(K);
          h = local.data();
        }
        PRGB_CUDA(cudaMemcpyAsync(h, iters, (size_t)K * 4, cudaMemcpyDeviceToHost, s));
        if (mixed) {
          h64.resize(K);
          PRGB_CUDA(cudaMemcpyAsync(h64.data(), iters64, (size_t)K * 4, cudaMemcpyDeviceToHost, s));
        }
        PRGB_TRY(solve_edge_visits(part, iters, iters64, &stats->edge_visits, &stats->fp64_edge_visits,
                                   tmp));  // synchronises
        for (int32_t k = 0; k < K; k++) stats->iters_max = h[k] > stats->iters_max ? h[k] : stats->iters_max;
        for (int32_t k = 0; k < (int32_t)h64.size(); k++)
          stats->fp64_sweeps_max = h64[k] > stats->fp64_sweeps_max ? h64[k] : stats->fp64_sweeps_max;
      } else if (timing) {
        for (const LargeComp& L : kt->comps)
          PRGB_CUDA(cudaMemcpyAsync(&hl[L.c], iters + L.c, 4, cudaMemcpyDeviceToHost, s));
        PRGB_CUDA(cudaStreamSynchronize(s));
      }
      auto sweeps = [&](int32_t c) -> int64_t { return counts ? h[c] : hl[c]; };
      if (level_events && stats->level_ms && kt->level.size() >= part->levels.size() + 1) {
        for (size_t li = 0; li < part->levels.size(); li++)
          PRGB_CUDA(cudaEventElapsedTime(&stats->level_ms[li], kt->level[li], kt->level[li + 1]));
      }
      if (timing) {
        stats->kernel_ms = 0.0f;
        stats->kernel_bytes = 0;
        stats->kernel_launches = (int64_t)kt->comps.size();
        for (size_t i = 0; i < kt->comps.size(); i++) {
          float ms = 0.0f;
          PRGB_CUDA(cudaEventElapsedTime(&ms, kt->start[i], kt->stop[i]));
          stats->kernel_ms += ms;
          const LargeComp& L = kt->comps[i];
          const int64_t it = sweeps(L.c);
          // the fixed-point series: per sweep 4 B per edge + per row the z
          // gather and write (16 B each, or 8 B when z is gathered as FP64
          // values), R read and write (16 B each) and c/outdeg (8 B); once
          // per launch: the start (W and c/outdeg read, R and z written) and
          // the end (R and 1/outdeg read, R and R/outdeg written)
          const int64_t zb = giant_fits_l2(L) ? 16 : 8;
          stats->kernel_bytes += it * (4 * (int64_t)L.m_int + (2 * zb + 40) * (int64_t)L.size) +
                                 (72 + zb) * (int64_t)L.size;
        }
      }
    }
  }
  return flags ? PR_ENOCONV : PR_OK;
}

pr_status pr_solve(const pr_partition* part, double c, const double* u, double tol, const pr_solve_opts* opts,
                   double* R, pr_solve_stats* stats, void* stream) {
  prgb::NvtxRange nvtx("prgb solve");
  return prgb::note_status(pr_solve_body(part, c, u, tol, opts, R, stats, stream));
}

static pr_status pr_partition_set_shape_body(pr_partition* part, int32_t cta_max, int32_t coop_blocks,
                                             int32_t balance) {
  if (!part || cta_max < kWarpCompMax || cta_max > kCtaCompMax || coop_blocks < 1 || coop_blocks > 8 ||
      (balance != 0 && balance != 1))
    return PR_EINVAL;
  std::lock_guard<std::mutex> lock(part->plan_mu);
  retune_levels(part, cta_max, coop_blocks, balance);
  return PR_OK;
}

pr_status pr_partition_set_shape(pr_partition* part, int32_t cta_max, int32_t coop_blocks, int32_t balance) {
  return prgb::note_status(pr_partition_set_shape_body(part, cta_max, coop_blocks, balance));
}

static pr_status pr_partition_tune_body(pr_partition* part, double c, const double* u, double tol, void* stream,
                            int32_t* cta_max, int32_t* coop_blocks, int32_t* balance, float* best_ms) {
  if (!part) return PR_EINVAL;
  if (part->g.n > 0 && (!u || !(c > 0.0 && c < 1.0) || !(tol > 0.0))) return PR_EINVAL;
  std::lock_guard<std::mutex> lock(part->plan_mu);
  return tune_partition(part, c, u, tol, (cudaStream_t)stream, cta_max, coop_blocks, balance, best_ms);
}

pr_status pr_partition_tune(pr_partition* part, double c, const double* u, double tol, void* stream,
                            int32_t* cta_max, int32_t* coop_blocks, int32_t* balance, float* best_ms) {
  prgb::NvtxRange nvtx("prgb tune");
  return prgb::note_status(pr_partition_tune_body(part, c, u, tol, stream, cta_max, coop_blocks, balance, best_ms));
}

static pr_status pr_global_power_body(const pr_graph* g, double c, const double* u, double tol,
                                      const pr_solve_opts* opts, double* R, pr_solve_stats* stats, void* stream) {
  if (!g) return PR_EINVAL;
  const int32_t n = g->g.n;
  if (n > 0) PRGB_TRY(check_solve_args(c, u, tol, R));
  pr_solve_opts o = {PR_NORM_L1, 10000, PR_PREC_FP64, 0, nullptr, nullptr, 0};
  if (opts) o = *opts;
  if (o.max_iter <= 0) o.max_iter = 10000;
  if (fault_hit(kFaultNoconv)) o.max_iter = 1;
  if (o.norm != PR_NORM_L1 && o.norm != PR_NORM_LINF) return PR_EINVAL;
  if (o.precision != PR_PREC_FP64 || o.warm_start || o.lu_threshold) return PR_EINVAL;
  int fixed = -1;
  if (o.replay_iters) {
    fixed = o.replay_iters[0];
    if (fixed < 0 || fixed > 1000000) return PR_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Arena tmp(s);
  Ctl* ctl = nullptr;
  PRGB_TRY(tmp.alloc(&ctl, 1));
  PRGB_TRY(init_ctl(ctl, s));
  const double* du = u;
  double* dR = R;
  if (o.io_on_host && n > 0) {
    double *tu = nullptr, *tR = nullptr;
    PRGB_TRY(tmp.alloc(&tu, (size_t)n));
    PRGB_TRY(tmp.alloc(&tR, (size_t)n));
    PRGB_COPY(cudaMemcpyAsync(tu, u, (size_t)n * 8, cudaMemcpyHostToDevice, s));
    du = tu;
    dR = tR;
  }
  int iters = 0;
  float kms = 0.0f;
  const bool timing = stats && stats->timing;
  pr_status st = run_global(g->g, c, du, tol, o.norm, o.max_iter, fixed, dR, &iters, tmp, ctl,
                            timing ? &kms : nullptr);
  if (st != PR_OK && st != PR_ENOCONV) return st;
  if (o.io_on_host && n > 0) {
    PRGB_COPY(cudaMemcpyAsync(R, dR, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
    PRGB_CUDA(cudaStreamSynchronize(s));
  }
  if (stats) {
    stats->iters_max = iters;
    stats->n_levels = 1;
    stats->launches = 2;  // c / outdeg, then the series
    stats->edge_visits = (int64_t)iters * g->g.m;
    if (stats->comp_iters) stats->comp_iters[0] = iters;
    if (timing) {
      stats->kernel_ms = kms;
      stats->kernel_launches = 1;
      stats->kernel_bytes = (int64_t)iters * (4 * g->g.m + 40 * (int64_t)g->g.n) + 28 * (int64_t)g->g.n;
    }
  }
  return st;
}

pr_status pr_global_power(const pr_graph* g, double c, const double* u, double tol, const pr_solve_opts* opts,
                          double* R, pr_solve_stats* stats, void* stream) {
  prgb::NvtxRange nvtx("prgb global_power");
  return prgb::note_status(pr_global_power_body(g, c, u, tol, opts, R, stats, stream));
}

static pr_status pr_residual_l1_body(const pr_graph* g, double c, const double* u, const double* R, double* out_host,
                         void* stream) {
  if (!g || !out_host) return PR_EINVAL;
  if (g->g.n > 0 && (!u || !R)) return PR_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  Arena tmp(s);
  double* part = nullptr;
  double* out = nullptr;
  PRGB_TRY(tmp.alloc(&part, (size_t)residual_grid()));
  PRGB_TRY(tmp.alloc(&out, 1));
  PRGB_TRY(run_residual(g->g, c, u, R, part, out, tmp));
  PRGB_CUDA(cudaMemcpyAsync(out_host, out, 8, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaStreamSynchronize(s));
  return PR_OK;
}

pr_status pr_residual_l1(const pr_graph* g, double c, const double* u, const double* R, double* out_host,
                         void* stream) {
  prgb::NvtxRange nvtx("prgb residual_l1");
  return prgb::note_status(pr_residual_l1_body(g, c, u, R, out_host, stream));
}

}  // extern "C"

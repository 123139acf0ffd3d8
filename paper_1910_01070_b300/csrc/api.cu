// api.cu -- host implementation of the C ABI declared in include/hr2.h:
// contexts with a device-memory budget, resident opacity tables, setups,
// per-stream workspaces, and the batch entry points that launch the kernels
// of kern_forward.cu.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "hr2_internal.cuh"

using namespace hr2;

namespace hr2 {
// streamed level-gridded operand (kern_setup.cu)
cudaError_t build_level_stream(const SetupDev* d_setup, int n_lev, int n_rows, int tile_lo, int n_tiles,
                               const unsigned char* mask, int mask_stride, float* ring, cudaStream_t s);
cudaError_t build_cell_mask(const FwdArgs& a, int max_lev, int stride, unsigned char* mask, cudaStream_t s);
cudaError_t build_stream_views(const SetupDev* d_setup, const float* ring, int group_tiles, int n_groups, int ord,
                               int n_setups, SetupDev* views, cudaStream_t s);
}  // namespace hr2

// ------------------------------------------------------------ tracing
// An NVTX range over the host side of an entry point (argument checks,
// workspace, launches), named after it, so that a timeline profiler (or ncu's
// --nvtx filter) shows each call over the kernels it launched.  Without a tool
// attached the push and pop return at once.
namespace {
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace
#define HR2_RANGE(name) const NvtxRange hr2_range_(name)

// ------------------------------------------------------------ errors
static thread_local std::string t_last_error;

static int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_last_error = buf;
  return code;
}

#define HR2_CU(call)                                                                       \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return fail(HR2_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// ------------------------------------------------------------ objects
struct Workspace {
  int n_cap = 0, lev_cap = 0, nu_cap = 0, nu64_cap = 0, io_cap = 0, io_bins_cap = 0;
  LevRec* recs = nullptr;
  SampleDev* samp = nullptr;
  int* perm = nullptr;
  PlanDev* plan = nullptr;
  unsigned int* counter = nullptr;   // [0] work counter, [1] error word
  unsigned int* h_counter = nullptr; // pinned host copy of counter (kept across growth)
  float* highres = nullptr;
  double* highres64 = nullptr;
  double* io_params = nullptr;
  int* io_sos = nullptr;
  double* io_logeps = nullptr;
  double* io_lnl = nullptr;
  float* io_bins = nullptr;
  float* chi = nullptr;       // two-pass direct path: absorption coefficients
  size_t chi_cap = 0;         // floats
  float* ring = nullptr;      // streamed operand: one group of tiles
  size_t ring_cap = 0;        // floats
  SetupDev* views = nullptr;  // streamed operand: one setup view per group
  int views_cap = 0;
  unsigned char* cells = nullptr;   // streamed operand: the batch's (level, T cell) mask
  size_t cells_cap = 0;
};

struct hr2_ctx {
  int device = 0;
  int n_sm = 0;
  size_t budget = 0;
  size_t used = 0;
  hr2_launch_cfg cfg{2, 8, 1, 0, kDefaultSplitMaxBatch};
  int stream_group = 0;                        // tiles per group of the streamed operand (0: by batch)
  long long wait_limit = kDefaultWaitCycles;   // bounded device-side waits, SM clock cycles
  bool wait_fault = false;                     // test hook: first stages wait for bytes that never come
  std::mutex mu;
  std::map<void*, size_t> blocks;  // device allocations and their sizes
  std::map<void*, Workspace*> ws;  // per stream
  std::vector<hr2_tables*> tables;
  std::vector<hr2_setup*> setups;
  bool profiling = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof;
};

struct hr2_tables {
  hr2_ctx* ctx = nullptr;
  TablesDev host{};
  TablesDev* dev = nullptr;
  void* data = nullptr;  // sig16 or sig64
  void* cia = nullptr;
  size_t bytes = 0;
  int n_nu = 0;
};

struct hr2_setup {
  hr2_ctx* ctx = nullptr;
  const hr2_tables* tables = nullptr;
  SetupDev host{};
  SetupDev* dev = nullptr;
  std::vector<void*> mem;
  size_t operand_bytes = 0;
  bool streamed = false;             // HR2_LEVEL_CACHE_STREAM: operand built per call, per group of tiles
  SetupDev* dev_stream = nullptr;    // ... and the descriptor its batches are prepared with (cached records)
  int n_bins = 0;
  bool has_obs = false;
  double* d_obs = nullptr;  // [2][n_bins]: D then sigma
};

// ------------------------------------------------------------ memory
static int dalloc(hr2_ctx* ctx, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (ctx->budget && ctx->used + bytes > ctx->budget)
    return fail(HR2_ENOMEM, "memory budget exceeded: %zu used + %zu requested > %zu", ctx->used, bytes, ctx->budget);
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(HR2_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  }
  ctx->blocks[*p] = bytes;
  ctx->used += bytes;
  return HR2_OK;
}

static void dfree(hr2_ctx* ctx, void* p) {
  if (!p) return;
  auto it = ctx->blocks.find(p);
  if (it != ctx->blocks.end()) {
    ctx->used -= it->second;
    ctx->blocks.erase(it);
  }
  cudaFree(p);
}

template <class T>
static int dalloc_t(hr2_ctx* ctx, T** p, size_t count) {
  void* v = nullptr;
  int rc = dalloc(ctx, &v, count * sizeof(T));
  *p = (T*)v;
  return rc;
}

static void ws_free(hr2_ctx* ctx, Workspace* w) {
  dfree(ctx, w->recs);
  dfree(ctx, w->samp);
  dfree(ctx, w->perm);
  dfree(ctx, w->plan);
  dfree(ctx, w->counter);
  dfree(ctx, w->highres);
  dfree(ctx, w->highres64);
  dfree(ctx, w->io_params);
  dfree(ctx, w->io_sos);
  dfree(ctx, w->io_logeps);
  dfree(ctx, w->io_lnl);
  dfree(ctx, w->io_bins);
  dfree(ctx, w->chi);
  dfree(ctx, w->ring);
  dfree(ctx, w->views);
  dfree(ctx, w->cells);
  unsigned int* keep = w->h_counter;
  *w = Workspace();
  w->h_counter = keep;
}

static bool stream_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return st != cudaStreamCaptureStatusNone;
}

// Grow the workspace of `stream` to hold n samples with up to lev levels,
// an FP32 F+ scratch of nu points (0: none), FP64 F+ scratch of nu64 points,
// and host-I/O staging for io samples with io_bins bins each.
static int ws_ensure(hr2_ctx* ctx, cudaStream_t stream, int n, int lev, int nu, int nu64, int io, int io_bins,
                     Workspace** out) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  Workspace*& w = ctx->ws[(void*)stream];
  if (!w) {
    w = new Workspace();
    // pinned word for reading the error flag with the batch's own copies
    if (cudaHostAlloc((void**)&w->h_counter, 2 * sizeof(unsigned int), cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      w->h_counter = nullptr;
    }
  }
  *out = w;
  bool grow = n > w->n_cap || lev > w->lev_cap || (nu > 0 && (n > w->n_cap || nu > w->nu_cap || !w->highres)) ||
              (nu64 > 0 && (n > w->n_cap || nu64 > w->nu64_cap || !w->highres64)) || io > w->io_cap ||
              (io > 0 && io_bins > w->io_bins_cap) || !w->plan;
  if (!grow) return HR2_OK;
  if (stream_capturing(stream))
    return fail(HR2_EBUSY, "workspace must grow (n=%d) while the stream is capturing; call hr2_reserve first", n);
  HR2_CU(cudaStreamSynchronize(stream));
  Workspace nw;
  nw.h_counter = w->h_counter;
  nw.n_cap = std::max(n, w->n_cap);
  nw.lev_cap = std::max(lev, w->lev_cap);
  nw.nu_cap = std::max(nu, w->nu_cap);
  nw.nu64_cap = std::max(nu64, w->nu64_cap);
  nw.io_cap = std::max(io, w->io_cap);
  nw.io_bins_cap = std::max(io_bins, w->io_bins_cap);
  ws_free(ctx, w);
  int rc;
  const size_t nc = (size_t)std::max(nw.n_cap, 1);
  if ((rc = dalloc_t(ctx, &nw.recs, nc * std::max(nw.lev_cap, 1))) ||
      (rc = dalloc_t(ctx, &nw.samp, nc)) || (rc = dalloc_t(ctx, &nw.perm, nc)) ||
      (rc = dalloc_t(ctx, &nw.plan, 1)) || (rc = dalloc_t(ctx, &nw.counter, 2)))
    goto bad;
  if (nw.nu_cap > 0 && (rc = dalloc_t(ctx, &nw.highres, nc * nw.nu_cap))) goto bad;
  if (nw.nu64_cap > 0 && (rc = dalloc_t(ctx, &nw.highres64, nc * nw.nu64_cap))) goto bad;
  if (nw.io_cap > 0) {
    const size_t ic = (size_t)nw.io_cap;
    if ((rc = dalloc_t(ctx, &nw.io_params, ic * HR2_NPARAM)) || (rc = dalloc_t(ctx, &nw.io_sos, ic)) ||
        (rc = dalloc_t(ctx, &nw.io_logeps, ic)) || (rc = dalloc_t(ctx, &nw.io_lnl, ic)) ||
        (rc = dalloc_t(ctx, &nw.io_bins, ic * std::max(nw.io_bins_cap, 1))))
      goto bad;
  }
  if (cudaMemset(nw.counter, 0, 2 * sizeof(unsigned int)) != cudaSuccess) {
    rc = fail(HR2_ECUDA, "workspace counter initialisation failed");
    goto bad;
  }
  *w = nw;
  return HR2_OK;
bad:
  ws_free(ctx, &nw);
  return rc;
}

// The workspace's absorption-coefficient buffer of the two-pass direct path,
// grown to at least `floats` (outside stream capture).
static int ws_ensure_chi(hr2_ctx* ctx, cudaStream_t stream, Workspace* w, size_t floats) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (w->chi_cap >= floats) return HR2_OK;
  if (stream_capturing(stream))
    return fail(HR2_EBUSY, "the two-pass buffer must grow while the stream is capturing; call the batch once first");
  HR2_CU(cudaStreamSynchronize(stream));
  dfree(ctx, w->chi);
  w->chi = nullptr;
  w->chi_cap = 0;
  int rc = dalloc_t(ctx, &w->chi, floats);
  if (rc) return rc;
  w->chi_cap = floats;
  return HR2_OK;
}

// The workspace's ring, setup views and cell mask of the streamed operand,
// grown to at least `floats`, `views` and `cells` (outside stream capture).
static int ws_ensure_stream(hr2_ctx* ctx, cudaStream_t stream, Workspace* w, size_t floats, int views, size_t cells) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (w->ring_cap >= floats && w->views_cap >= views && w->cells_cap >= cells) return HR2_OK;
  if (stream_capturing(stream))
    return fail(HR2_EBUSY, "the streamed operand's ring must grow while the stream is capturing; call the batch once first");
  HR2_CU(cudaStreamSynchronize(stream));
  int rc;
  if (w->ring_cap < floats) {
    dfree(ctx, w->ring);
    w->ring = nullptr;
    w->ring_cap = 0;
    if ((rc = dalloc_t(ctx, &w->ring, floats))) return rc;
    w->ring_cap = floats;
  }
  if (w->views_cap < views) {
    dfree(ctx, w->views);
    w->views = nullptr;
    w->views_cap = 0;
    if ((rc = dalloc_t(ctx, &w->views, (size_t)views))) return rc;
    w->views_cap = views;
  }
  if (w->cells_cap < cells) {
    dfree(ctx, w->cells);
    w->cells = nullptr;
    w->cells_cap = 0;
    if ((rc = dalloc_t(ctx, &w->cells, cells))) return rc;
    w->cells_cap = cells;
  }
  return HR2_OK;
}

// ------------------------------------------------------------ contexts
extern "C" int hr2_ctx_create(int device, size_t mem_budget_bytes, hr2_ctx** out) {
  if (!out) return fail(HR2_EINVAL, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  HR2_CU(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(HR2_EINVAL, "device %d outside [0, %d)", device, ndev);
  HR2_CU(cudaSetDevice(device));
  cudaDeviceProp prop;
  HR2_CU(cudaGetDeviceProperties(&prop, device));
  if (prop.major != 10 || prop.minor != 3)
    return fail(HR2_EINVAL, "device %d is sm_%d%d; this library is built for sm_103a (B300)", device, prop.major,
                prop.minor);
  hr2_ctx* c = new hr2_ctx();
  c->device = device;
  c->n_sm = prop.multiProcessorCount;
  c->budget = mem_budget_bytes;
  *out = c;
  return HR2_OK;
}

extern "C" int hr2_setup_destroy(hr2_ctx* ctx, hr2_setup* setup);
extern "C" int hr2_tables_destroy(hr2_ctx* ctx, hr2_tables* tables);

extern "C" int hr2_ctx_destroy(hr2_ctx* ctx) {
  if (!ctx) return fail(HR2_EINVAL, "ctx is NULL");
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  while (!ctx->setups.empty()) hr2_setup_destroy(ctx, ctx->setups.back());
  while (!ctx->tables.empty()) hr2_tables_destroy(ctx, ctx->tables.back());
  for (auto& kv : ctx->ws) {
    ws_free(ctx, kv.second);
    if (kv.second->h_counter) cudaFreeHost(kv.second->h_counter);
    delete kv.second;
  }
  ctx->ws.clear();
  for (auto& kv : ctx->blocks) cudaFree(kv.first);
  for (auto& ev : ctx->prof) {
    cudaEventDestroy(ev.first);
    cudaEventDestroy(ev.second);
  }
  delete ctx;
  return HR2_OK;
}

extern "C" const char* hr2_last_error(const hr2_ctx* ctx) {
  (void)ctx;
  return t_last_error.c_str();
}

extern "C" int hr2_ctx_memory(const hr2_ctx* ctx, size_t* used, size_t* budget) {
  if (!ctx) return fail(HR2_EINVAL, "ctx is NULL");
  if (used) *used = ctx->used;
  if (budget) *budget = ctx->budget;
  return HR2_OK;
}

extern "C" int hr2_set_launch_config(hr2_ctx* ctx, const hr2_launch_cfg* cfg) {
  if (!ctx || !cfg) return fail(HR2_EINVAL, "NULL argument");
  if (cfg->warps_per_cta < 1 || cfg->warps_per_cta > kMaxWarps || cfg->ctas_per_sm < 1 || cfg->ctas_per_sm > 32)
    return fail(HR2_EINVAL, "launch config out of range (warps 1..%d, ctas_per_sm 1..32)", kMaxWarps);
  if (cfg->tiles_per_item < 1 || cfg->tiles_per_item > 16)
    return fail(HR2_EINVAL, "tiles_per_item %d outside 1..16", cfg->tiles_per_item);
  if (cfg->stages < 0 || cfg->stages > 2) return fail(HR2_EINVAL, "stages %d is not 0, 1 or 2", cfg->stages);
  if (cfg->split_max_batch < 0 || cfg->split_max_batch > 65535)   // the absorption pass puts the batch on grid z
    return fail(HR2_EINVAL, "split_max_batch %d outside 0..65535", cfg->split_max_batch);
  ctx->cfg = *cfg;
  return HR2_OK;
}

extern "C" int hr2_set_stream_group(hr2_ctx* ctx, int tiles) {
  if (!ctx) return fail(HR2_EINVAL, "ctx is NULL");
  if (tiles < 0) return fail(HR2_EINVAL, "tiles %d < 0", tiles);
  ctx->stream_group = tiles;
  return HR2_OK;
}

extern "C" int hr2_get_launch_config(const hr2_ctx* ctx, hr2_launch_cfg* cfg) {
  if (!ctx || !cfg) return fail(HR2_EINVAL, "NULL argument");
  *cfg = ctx->cfg;
  return HR2_OK;
}

extern "C" int hr2_set_wait_limit(hr2_ctx* ctx, long long cycles) {
  if (!ctx) return fail(HR2_EINVAL, "ctx is NULL");
  if (cycles < 0) return fail(HR2_EINVAL, "wait limit %lld < 0", cycles);
  ctx->wait_limit = cycles;
  return HR2_OK;
}

extern "C" int hr2_set_wait_fault(hr2_ctx* ctx, int on) {
  if (!ctx) return fail(HR2_EINVAL, "ctx is NULL");
  ctx->wait_fault = on != 0;
  return HR2_OK;
}

extern "C" int hr2_get_wait_limit(const hr2_ctx* ctx, long long* cycles) {
  if (!ctx || !cycles) return fail(HR2_EINVAL, "NULL argument");
  *cycles = ctx->wait_limit;
  return HR2_OK;
}

extern "C" int hr2_reserve(hr2_ctx* ctx, void* stream, int n, int n_nu_max) {
  HR2_RANGE("hr2_reserve");
  if (!ctx || n < 0 || n_nu_max < 0) return fail(HR2_EINVAL, "invalid argument");
  HR2_CU(cudaSetDevice(ctx->device));
  Workspace* w;
  return ws_ensure(ctx, (cudaStream_t)stream, n, HR2_MAX_LEVELS, n_nu_max, 0, 0, 0, &w);
}

// ------------------------------------------------------------ tables
static int check_grid(const double* g, int n, bool positive, const char* what) {
  if (!g) return fail(HR2_EINVAL, "%s is NULL", what);
  for (int i = 0; i < n; ++i) {
    if (!std::isfinite(g[i])) return fail(HR2_EINVAL, "%s[%d] is not finite", what, i);
    if (positive && !(g[i] > 0)) return fail(HR2_EINVAL, "%s[%d] must be > 0", what, i);
    if (i && !(g[i] > g[i - 1])) return fail(HR2_EINVAL, "%s is not strictly ascending at %d", what, i);
  }
  return HR2_OK;
}

// off = rint((min+max)/2) over n finite values; -1 if a value is not finite.
static int scan_offset(const double* v, size_t n, double* off) {
  double mn = INFINITY, mx = -INFINITY;
  for (size_t t = 0; t < n; ++t) {
    const double x = v[t];
    if (!std::isfinite(x)) return -1;
    mn = std::min(mn, x);
    mx = std::max(mx, x);
  }
  *off = std::rint(0.5 * (mn + mx));
  return 0;
}

// Copy `rows` rows of n_nu host doubles into device rows of nu_pad entries,
// quantised (FP16 - off) or as FP64, through a bounded staging buffer.
static int upload_rows(hr2_ctx* ctx, const double* host, long long rows, int n_nu, int nu_pad, int storage,
                       double off, void* dst) {
  const size_t stage_elems = std::max<size_t>((size_t)n_nu, (size_t)8 << 20);
  const long long rows_per = std::max<long long>(1, (long long)(stage_elems / (size_t)n_nu));
  double* stage = nullptr;
  HR2_CU(cudaMalloc(&stage, sizeof(double) * (size_t)rows_per * n_nu));
  int rc = HR2_OK;
  for (long long r0 = 0; r0 < rows && rc == HR2_OK; r0 += rows_per) {
    const long long nr = std::min(rows_per, rows - r0);
    cudaError_t e = cudaMemcpy(stage, host + (size_t)r0 * n_nu, sizeof(double) * (size_t)nr * n_nu,
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      if (storage == HR2_STORE_FP16_OFFSET)
        e = quantise_fp16(stage, (__half*)dst + (size_t)r0 * nu_pad, nr, n_nu, nu_pad, off, 0);
      else
        e = copy_pad_fp64(stage, (double*)dst + (size_t)r0 * nu_pad, nr, n_nu, nu_pad, 0);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) rc = fail(HR2_ECUDA, "table upload: %s", cudaGetErrorString(e));
  }
  cudaFree(stage);
  return rc;
}

static int sync_tables_dev(hr2_tables* t) {
  HR2_CU(cudaMemcpy(t->dev, &t->host, sizeof(TablesDev), cudaMemcpyHostToDevice));
  return HR2_OK;
}

extern "C" int hr2_tables_upload_species(hr2_ctx* ctx, hr2_tables* t, int s, const double* v) {
  HR2_RANGE("hr2_tables_upload_species");
  if (!ctx || !t || !v) return fail(HR2_EINVAL, "NULL argument");
  if (s < 0 || s >= t->host.n_species) return fail(HR2_EINVAL, "species %d outside [0, %d)", s, t->host.n_species);
  HR2_CU(cudaSetDevice(ctx->device));
  const TablesDev& h = t->host;
  const long long rows = (long long)h.n_T * h.n_p;
  double off = 0.0;
  if (scan_offset(v, (size_t)rows * h.n_nu, &off)) return fail(HR2_EINVAL, "species %d has a non-finite value", s);
  if (h.storage == HR2_STORE_FP64) off = 0.0;
  const size_t elem = h.storage == HR2_STORE_FP16_OFFSET ? 2 : 8;
  char* dst = (char*)t->data + (size_t)s * rows * h.nu_pad * elem;
  int rc = upload_rows(ctx, v, rows, h.n_nu, h.nu_pad, h.storage, off, dst);
  if (rc) return rc;
  t->host.off[s] = off;
  return sync_tables_dev(t);
}

extern "C" int create_opacity_tables(hr2_ctx* ctx, const hr2_table_desc* d, const double* log10_sigma,
                                     const double* cia_h2h2, const double* cia_h2he, int storage, hr2_tables** out) {
  HR2_RANGE("create_opacity_tables");
  if (!ctx || !d || !out) return fail(HR2_EINVAL, "NULL argument");
  *out = nullptr;
  if (storage != HR2_STORE_FP16_OFFSET && storage != HR2_STORE_FP64)
    return fail(HR2_EINVAL, "unknown storage %d", storage);
  if (d->n_species < 1 || d->n_species > HR2_MAX_SPECIES)
    return fail(HR2_EINVAL, "n_species %d outside [1, %d]", d->n_species, HR2_MAX_SPECIES);
  if (d->n_T < 2 || d->n_T > HR2_MAX_TGRID) return fail(HR2_EINVAL, "n_T %d outside [2, %d]", d->n_T, HR2_MAX_TGRID);
  if (d->n_p < 2 || d->n_p > HR2_MAX_PGRID) return fail(HR2_EINVAL, "n_p %d outside [2, %d]", d->n_p, HR2_MAX_PGRID);
  if (d->n_nu < 1) return fail(HR2_EINVAL, "n_nu must be >= 1");
  if (!(d->nu0 > 0) || !(d->dnu > 0) || !std::isfinite(d->nu0) || !std::isfinite(d->dnu))
    return fail(HR2_EINVAL, "nu0 and dnu must be positive and finite");
  int rc;
  if ((rc = check_grid(d->T_grid, d->n_T, true, "T_grid"))) return rc;
  if ((rc = check_grid(d->log10p_grid, d->n_p, false, "log10p_grid"))) return rc;
  if (!d->species_mass) return fail(HR2_EINVAL, "species_mass is NULL");
  for (int s = 0; s < d->n_species; ++s)
    if (!(d->species_mass[s] > 0)) return fail(HR2_EINVAL, "species_mass[%d] must be > 0", s);
  if ((d->has_cia_h2h2 && !cia_h2h2) || (d->has_cia_h2he && !cia_h2he))
    return fail(HR2_EINVAL, "a CIA table flagged present is NULL");
  const long long nu_pad = ((long long)d->n_nu + kTileNu - 1) / kTileNu * kTileNu;
  if (nu_pad * d->n_T * d->n_p > (1ll << 31) - 1)
    return fail(HR2_EINVAL, "one species table exceeds 2^31 entries");
  HR2_CU(cudaSetDevice(ctx->device));

  hr2_tables* t = new hr2_tables();
  t->ctx = ctx;
  TablesDev& h = t->host;
  h.storage = storage;
  h.n_species = d->n_species;
  h.n_T = d->n_T;
  h.n_p = d->n_p;
  h.n_nu = d->n_nu;
  h.nu_pad = (int)nu_pad;
  h.nu0 = d->nu0;
  h.dnu = d->dnu;
  h.has_cia[0] = d->has_cia_h2h2 ? 1 : 0;
  h.has_cia[1] = d->has_cia_h2he ? 1 : 0;
  for (int a = 0; a < d->n_T; ++a) {
    h.T_grid[a] = (float)d->T_grid[a];
    h.T_grid64[a] = d->T_grid[a];
  }
  for (int b = 0; b < d->n_p; ++b) h.log10p_grid64[b] = d->log10p_grid[b];
  for (int s = 0; s < d->n_species; ++s) h.mass[s] = d->species_mass[s];
  const size_t elem = storage == HR2_STORE_FP16_OFFSET ? 2 : 8;
  const size_t rows = (size_t)d->n_T * d->n_p;
  const size_t sig_bytes = (size_t)d->n_species * rows * nu_pad * elem;
  const size_t cia_bytes = 2 * (size_t)d->n_T * nu_pad * elem;
  if ((rc = dalloc(ctx, &t->data, sig_bytes)) || (rc = dalloc(ctx, &t->cia, cia_bytes)) ||
      (rc = dalloc(ctx, (void**)&t->dev, sizeof(TablesDev)))) {
    dfree(ctx, t->data);
    dfree(ctx, t->cia);
    dfree(ctx, t->dev);
    delete t;
    return rc;
  }
  t->bytes = sig_bytes + cia_bytes + sizeof(TablesDev);
  if (cudaMemset(t->data, 0, sig_bytes) != cudaSuccess || cudaMemset(t->cia, 0, cia_bytes) != cudaSuccess) {
    rc = fail(HR2_ECUDA, "cudaMemset of the tables failed");
  }
  if (storage == HR2_STORE_FP16_OFFSET) {
    h.sig16 = (const __half*)t->data;
    h.cia16 = (const __half*)t->cia;
  } else {
    h.sig64 = (const double*)t->data;
    h.cia64 = (const double*)t->cia;
  }
  ctx->tables.push_back(t);
  if (!rc) rc = sync_tables_dev(t);
  for (int s = 0; s < d->n_species && !rc && log10_sigma; ++s)
    rc = hr2_tables_upload_species(ctx, t, s, log10_sigma + (size_t)s * rows * d->n_nu);
  const double* cia[2] = {cia_h2h2, cia_h2he};
  for (int p = 0; p < 2 && !rc; ++p) {
    if (!h.has_cia[p]) continue;
    double off = 0.0;
    if (scan_offset(cia[p], (size_t)d->n_T * d->n_nu, &off)) {
      rc = fail(HR2_EINVAL, "CIA table %d has a non-finite value", p);
      break;
    }
    if (storage == HR2_STORE_FP64) off = 0.0;
    rc = upload_rows(ctx, cia[p], d->n_T, d->n_nu, (int)nu_pad, storage, off,
                     (char*)t->cia + (size_t)p * d->n_T * nu_pad * elem);
    h.off[kCiaH2H2 + p] = off;
  }
  if (!rc) rc = sync_tables_dev(t);
  if (rc) {
    std::string keep = t_last_error;
    hr2_tables_destroy(ctx, t);
    t_last_error = keep;
    return rc;
  }
  *out = t;
  return HR2_OK;
}

extern "C" int hr2_tables_info(const hr2_tables* t, double* offsets, size_t* bytes) {
  if (!t) return fail(HR2_EINVAL, "tables is NULL");
  if (offsets) {
    for (int s = 0; s < t->host.n_species; ++s) offsets[s] = t->host.off[s];
    offsets[t->host.n_species] = t->host.off[kCiaH2H2];
    offsets[t->host.n_species + 1] = t->host.off[kCiaH2He];
  }
  if (bytes) *bytes = t->bytes;
  return HR2_OK;
}

extern "C" int hr2_tables_destroy(hr2_ctx* ctx, hr2_tables* t) {
  if (!ctx || !t) return fail(HR2_EINVAL, "NULL argument");
  for (hr2_setup* s : ctx->setups)
    if (s->tables == t) return fail(HR2_EBUSY, "a setup still uses these tables");
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  dfree(ctx, t->data);
  dfree(ctx, t->cia);
  dfree(ctx, t->dev);
  ctx->tables.erase(std::remove(ctx->tables.begin(), ctx->tables.end(), t), ctx->tables.end());
  delete t;
  return HR2_OK;
}

// ------------------------------------------------------------ setups
extern "C" int hr2_setup_set_observation(hr2_ctx* ctx, hr2_setup* s, const double* D, const double* sigma) {
  HR2_RANGE("hr2_setup_set_observation");
  if (!ctx || !s || !D || !sigma) return fail(HR2_EINVAL, "NULL argument");
  for (int b = 0; b < s->n_bins; ++b) {
    if (!std::isfinite(D[b])) return fail(HR2_EINVAL, "obs_flux[%d] is not finite", b);
    if (!(sigma[b] > 0) || !std::isfinite(sigma[b])) return fail(HR2_EINVAL, "obs_sigma[%d] must be > 0", b);
  }
  HR2_CU(cudaSetDevice(ctx->device));
  int rc;
  // [D][sigma][1 / (2 sigma^2)][sum of -ln(2 pi sigma^2) / 2]
  if (!s->d_obs) {
    if ((rc = dalloc_t(ctx, &s->d_obs, 3 * (size_t)s->n_bins + 1))) return rc;
    s->mem.push_back(s->d_obs);
  }
  HR2_CU(cudaMemcpy(s->d_obs, D, sizeof(double) * s->n_bins, cudaMemcpyHostToDevice));
  HR2_CU(cudaMemcpy(s->d_obs + s->n_bins, sigma, sizeof(double) * s->n_bins, cudaMemcpyHostToDevice));
  s->host.obs_D = s->d_obs;
  s->host.obs_sigma = s->d_obs + s->n_bins;
  s->host.obs_inv2s2 = s->d_obs + 2 * (size_t)s->n_bins;
  s->host.obs_lnorm = s->d_obs + 3 * (size_t)s->n_bins;
  HR2_CU(launch_obs_terms(s->host.obs_sigma, s->n_bins, const_cast<double*>(s->host.obs_inv2s2),
                          const_cast<double*>(s->host.obs_lnorm), 0));
  HR2_CU(cudaDeviceSynchronize());
  s->has_obs = true;
  HR2_CU(cudaMemcpy(s->dev, &s->host, sizeof(SetupDev), cudaMemcpyHostToDevice));
  return HR2_OK;
}

extern "C" int hr2_setup_create(hr2_ctx* ctx, const hr2_tables* tab, const hr2_setup_desc* d, hr2_setup** out) {
  HR2_RANGE("hr2_setup_create");
  if (!ctx || !tab || !d || !out) return fail(HR2_EINVAL, "NULL argument");
  *out = nullptr;
  const TablesDev& th = tab->host;
  if (d->n_nu < 1 || d->nu_first < 0 || (long long)d->nu_first + d->n_nu > th.n_nu)
    return fail(HR2_EINVAL, "wavenumber range [%d, %d) outside the table's %d columns", d->nu_first,
                d->nu_first + d->n_nu, th.n_nu);
  if (d->n_layers < 1 || d->n_layers + 1 > HR2_MAX_LEVELS)
    return fail(HR2_EINVAL, "n_layers %d outside [1, %d]", d->n_layers, HR2_MAX_LEVELS - 1);
  if (!(d->p_top > 0) || !(d->p_bot > d->p_top) || !std::isfinite(d->p_bot))
    return fail(HR2_EINVAL, "need 0 < p_top < p_bot");
  if (d->n_species < 0 || d->n_species > HR2_MAX_SPECIES || (d->n_species && !d->species))
    return fail(HR2_EINVAL, "n_species %d outside [0, %d]", d->n_species, HR2_MAX_SPECIES);
  for (int s = 0; s < d->n_species; ++s)
    if (d->species[s] < 0 || d->species[s] >= th.n_species)
      return fail(HR2_EINVAL, "species[%d] = %d is not a table species", s, d->species[s]);
  if (d->n_mu < 1 || d->n_mu > HR2_MAX_MU) return fail(HR2_EINVAL, "n_mu %d outside [1, %d]", d->n_mu, HR2_MAX_MU);
  if (d->fe_elements < 1 || d->fe_order < 1 || d->fe_elements * d->fe_order + 1 > HR2_MAX_TNODES)
    return fail(HR2_EINVAL, "finite elements: need K_e >= 1, q >= 1, K_e q + 1 <= %d", HR2_MAX_TNODES);
  if (d->n_bins < 1 || !d->bin_edges) return fail(HR2_EINVAL, "need n_bins >= 1 and bin_edges");
  for (int b = 0; b <= d->n_bins; ++b)
    if (!std::isfinite(d->bin_edges[b]) || (b && !(d->bin_edges[b] > d->bin_edges[b - 1])))
      return fail(HR2_EINVAL, "bin_edges must be finite and strictly ascending");
  if (!(d->r_he >= 0) || !(d->radius_cm > 0)) return fail(HR2_EINVAL, "need r_he >= 0 and radius_cm > 0");
  if ((d->obs_flux == nullptr) != (d->obs_sigma == nullptr))
    return fail(HR2_EINVAL, "obs_flux and obs_sigma must both be given or both be NULL");
  if (d->interp != HR2_INTERP_LOG10 && d->interp != HR2_INTERP_LINEAR)
    return fail(HR2_EINVAL, "interp %d is neither HR2_INTERP_LOG10 nor HR2_INTERP_LINEAR", d->interp);
  if (d->interp == HR2_INTERP_LINEAR && th.storage == HR2_STORE_FP16_OFFSET &&
      (!d->level_cache || d->level_cache == HR2_LEVEL_CACHE_STREAM))
    return fail(HR2_EINVAL, "the linear interpolation option on FP16 tables needs level_cache (not streamed)");
  if (d->level_cache == HR2_LEVEL_CACHE_STREAM && th.storage != HR2_STORE_FP16_OFFSET)
    return fail(HR2_EINVAL, "the streamed operand needs FP16 tables");
  if (d->profile != HR2_PROFILE_FE && d->profile != HR2_PROFILE_MILNE)
    return fail(HR2_EINVAL, "profile %d is neither HR2_PROFILE_FE nor HR2_PROFILE_MILNE", d->profile);
  if (d->sc != HR2_SC_LINEAR && d->sc != HR2_SC_PARABOLIC)
    return fail(HR2_EINVAL, "sc %d is neither HR2_SC_LINEAR nor HR2_SC_PARABOLIC", d->sc);
  HR2_CU(cudaSetDevice(ctx->device));

  hr2_setup* st = new hr2_setup();
  st->ctx = ctx;
  st->tables = tab;
  st->n_bins = d->n_bins;
  SetupDev& h = st->host;
  h.nu_first = d->nu_first;
  h.n_nu = d->n_nu;
  h.tile0 = d->nu_first / kTileNu;
  h.n_tiles = (d->nu_first + d->n_nu - 1) / kTileNu - h.tile0 + 1;
  h.n_lev = d->n_layers + 1;
  h.n_species = d->n_species;
  for (int s = 0; s < d->n_species; ++s) {
    h.species[s] = d->species[s];
    h.mass64[s] = th.mass[d->species[s]];
    h.mass[s] = (float)h.mass64[s];
  }
  h.n_mu = d->n_mu;
  h.fe_elements = d->fe_elements;
  h.fe_order = d->fe_order;
  h.n_tnodes = d->fe_elements * d->fe_order + 1;
  h.r_he = d->r_he;
  h.radius_cm = d->radius_cm;
  h.interp = d->interp;
  h.profile = d->profile;
  h.cloud = d->cloud != 0;
  h.sc = d->sc;
  h.n_bins = d->n_bins;
  h.tables = tab->dev;
  const int n_cia = th.has_cia[0] + th.has_cia[1];
  h.cost = (float)(h.n_lev * (d->n_species + n_cia + 2 + 1.5 * d->n_mu));

  auto track = [&](void* p) { st->mem.push_back(p); };
  int rc = HR2_OK;
  LevelDev* d_lev = nullptr;
  double* d_quad = nullptr;
  double* d_edges = nullptr;
  int *d_lo = nullptr, *d_hi = nullptr, *d_bin = nullptr, *d_rowinfo = nullptr, *d_err = nullptr;
  double* d_invz = nullptr;
  std::vector<int> rowinfo(4 * (size_t)d->n_bins);
  std::vector<long long> rowptr((size_t)d->n_bins + 1);
  std::vector<int> col0((size_t)d->n_bins);
  long long nnz = 0;
  int err = 0;
  std::vector<double> quad(2 * (size_t)d->n_mu + d->fe_order + 1);
  cudaError_t e;

  if ((rc = dalloc_t(ctx, &d_lev, h.n_lev))) goto fail_all;
  track(d_lev);
  h.levels = d_lev;
  if ((rc = dalloc_t(ctx, &d_quad, quad.size()))) goto fail_all;
  if ((e = build_setup_levels(h.n_lev, d->p_top, d->p_bot, tab->dev, d_lev, 0)) != cudaSuccess ||
      (e = build_quadratures(d->n_mu, d->fe_order + 1, d_quad, 0)) != cudaSuccess ||
      (e = cudaMemcpy(quad.data(), d_quad, sizeof(double) * quad.size(), cudaMemcpyDeviceToHost)) != cudaSuccess) {
    rc = fail(HR2_ECUDA, "setup levels/quadrature: %s", cudaGetErrorString(e));
    goto fail_all;
  }
  for (int k = 0; k < d->n_mu; ++k) {
    const double mu = quad[k], w = quad[d->n_mu + k];
    h.mu64[k] = mu;
    h.wmu64[k] = w;
    h.mu[k] = (float)mu;
    h.inv_mu[k] = (float)(1.0 / mu);
    h.mu_nlog2e[k] = (float)(-kLog2e / mu);
    h.wflux[k] = (float)(2.0 * kPi * w * mu);
    h.lwmu[k] = (float)std::log2(2.0 * kPi * w * mu * mu);
  }
  // nodes beyond n_mu (up to the kernel's compile-time count) are padding:
  // mu = 1 with zero weight, so they add nothing to F+
  for (int k = d->n_mu; k < HR2_MAX_MU; ++k) {
    h.mu64[k] = 1.0;
    h.wmu64[k] = 0.0;
    h.mu[k] = 1.f;
    h.inv_mu[k] = 1.f;
    h.mu_nlog2e[k] = (float)(-kLog2e);
    h.wflux[k] = 0.f;
    h.lwmu[k] = -1e4f;
  }
  for (int i = 0; i <= d->fe_order; ++i) h.gll[i] = quad[2 * d->n_mu + i];
  if (d->profile != HR2_PROFILE_MILNE) {
    int* d_fek = nullptr;
    double* d_feb = nullptr;
    if ((rc = dalloc_t(ctx, &d_fek, h.n_lev))) goto fail_all;
    track(d_fek);
    if ((rc = dalloc_t(ctx, &d_feb, (size_t)h.n_lev * (d->fe_order + 1)))) goto fail_all;
    track(d_feb);
    h.fe_k = d_fek;
    h.fe_b = d_feb;
    if ((e = build_fe_basis(h.n_lev, d->fe_elements, d->fe_order, h.gll, d_fek, d_feb, 0)) != cudaSuccess) {
      rc = fail(HR2_ECUDA, "setup profile basis: %s", cudaGetErrorString(e));
      goto fail_all;
    }
  }

  // instrument profile + binning operator
  if ((rc = dalloc_t(ctx, &d_edges, d->n_bins + 1)) || (rc = dalloc_t(ctx, &d_lo, d->n_nu)) ||
      (rc = dalloc_t(ctx, &d_hi, d->n_nu)) || (rc = dalloc_t(ctx, &d_bin, d->n_nu)) ||
      (rc = dalloc_t(ctx, &d_invz, d->n_nu)) || (rc = dalloc_t(ctx, &d_rowinfo, 4 * (size_t)d->n_bins)) ||
      (rc = dalloc_t(ctx, &d_err, 1)))
    goto fail_tmp;
  if ((e = cudaMemcpy(d_edges, d->bin_edges, sizeof(double) * (d->n_bins + 1), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemset(d_err, 0, sizeof(int))) != cudaSuccess ||
      (e = build_w_rows(tab->dev, d->nu_first, d->n_nu, d->resolving_power, d->n_bins, d_edges, d_lo, d_hi, d_invz,
                        d_bin, d_rowinfo, d_err, 0)) != cudaSuccess ||
      (e = cudaMemcpy(rowinfo.data(), d_rowinfo, sizeof(int) * rowinfo.size(), cudaMemcpyDeviceToHost)) !=
          cudaSuccess ||
      (e = cudaMemcpy(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) {
    rc = fail(HR2_ECUDA, "setup operator rows: %s", cudaGetErrorString(e));
    goto fail_tmp;
  }
  if (err) {
    rc = fail(HR2_EINVAL, "a bin contains no wavenumber point of the setup");
    goto fail_tmp;
  }
  for (int b = 0; b < d->n_bins; ++b) {
    rowptr[b] = nnz;
    col0[b] = rowinfo[4 * b + 2];
    nnz += rowinfo[4 * b + 3];
  }
  rowptr[d->n_bins] = nnz;
  h.w_nnz = nnz;
  {
    long long* d_rowptr = nullptr;
    int* d_col0 = nullptr;
    float* d_w32 = nullptr;
    double* d_w64 = nullptr;
    if ((rc = dalloc_t(ctx, &d_rowptr, rowptr.size()))) goto fail_tmp;
    track(d_rowptr);
    if ((rc = dalloc_t(ctx, &d_col0, col0.size()))) goto fail_tmp;
    track(d_col0);
    if ((rc = dalloc_t(ctx, &d_w32, (size_t)nnz))) goto fail_tmp;
    track(d_w32);
    if ((rc = dalloc_t(ctx, &d_w64, (size_t)nnz))) goto fail_tmp;
    track(d_w64);
    h.w_rowptr = d_rowptr;
    h.w_col0 = d_col0;
    h.w32 = d_w32;
    h.w64 = d_w64;
    if ((e = cudaMemcpy(d_rowptr, rowptr.data(), sizeof(long long) * rowptr.size(), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(d_col0, col0.data(), sizeof(int) * col0.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = build_w_values(tab->dev, d->nu_first, d->resolving_power, d->n_bins, d_lo, d_hi, d_invz, d_rowinfo,
                            d_rowptr, d_w32, d_w64, 0)) != cudaSuccess ||
        (e = cudaDeviceSynchronize()) != cudaSuccess) {
      rc = fail(HR2_ECUDA, "setup operator values: %s", cudaGetErrorString(e));
      goto fail_tmp;
    }
  }
  if (d->profile == HR2_PROFILE_MILNE) {
    double* d_hopf = nullptr;
    if ((rc = dalloc_t(ctx, &d_hopf, (size_t)kHopfN))) goto fail_tmp;
    track(d_hopf);
    h.hopf_q = d_hopf;
    if ((e = build_hopf_table(d_hopf, 0)) != cudaSuccess || (e = cudaDeviceSynchronize()) != cudaSuccess) {
      rc = fail(HR2_ECUDA, "setup Hopf function: %s", cudaGetErrorString(e));
      goto fail_tmp;
    }
  }
  {
    float4* d_nu = nullptr;
    float2* d_c1n = nullptr;
    const size_t n_pairs = (size_t)h.n_tiles * (kTileNu / 2);
    if ((rc = dalloc_t(ctx, &d_nu, n_pairs))) goto fail_tmp;
    track(d_nu);
    if ((rc = dalloc_t(ctx, &d_c1n, n_pairs))) goto fail_tmp;
    track(d_c1n);
    h.nu_pair = d_nu;
    h.c1n_pair = d_c1n;
    if ((e = build_nu_pairs(tab->dev, h.tile0, h.n_tiles, d_nu, d_c1n, 0)) != cudaSuccess ||
        (e = cudaDeviceSynchronize()) != cudaSuccess) {
      rc = fail(HR2_ECUDA, "setup wavenumber constants: %s", cudaGetErrorString(e));
      goto fail_tmp;
    }
  }
  {
  // per tile, level, T cell and operand row (absorbers, then the two CIA
  // pairs): 2 kTileNu floats (row and T difference)
  const size_t per_tile = (size_t)h.n_lev * (h.n_species + 2) * (th.n_T - 1) * 2 * kTileNu;
  bool stream_op = d->level_cache == HR2_LEVEL_CACHE_STREAM;
  bool want_operand = d->level_cache != 0 && !stream_op && th.storage == HR2_STORE_FP16_OFFSET;
  if (want_operand && d->level_cache == HR2_LEVEL_CACHE_AUTO) {
    // the operand where it fits the context's budget and half the free memory
    const size_t bytes = per_tile * h.n_tiles * sizeof(float);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      cudaGetLastError();
      free_b = 0;
    }
    const bool fits = bytes <= free_b / 2 && (!ctx->budget || ctx->used + bytes <= ctx->budget);
    if (!fits && d->interp == HR2_INTERP_LINEAR) {
      rc = fail(HR2_ENOMEM, "the linear option needs the level-gridded operand (%zu bytes), which does not fit", bytes);
      goto fail_tmp;
    }
    want_operand = fits;
    stream_op = !fits;   // the operand per call and group of tiles instead
  }
  if (stream_op) {
    h.lvl32_tile_floats = (long long)per_tile;   // the ring's tile stride
    st->streamed = true;
  }
  if (want_operand) {
    float* d_lvl = nullptr;
    if ((rc = dalloc_t(ctx, &d_lvl, per_tile * h.n_tiles))) goto fail_tmp;
    track(d_lvl);
    h.lvl32 = d_lvl;
    h.lvl32_tile_floats = (long long)per_tile;
    h.cached = 1;
    st->operand_bytes = per_tile * h.n_tiles * sizeof(float);
    if ((e = build_level_cache(tab->dev, h, d_lvl, 0)) != cudaSuccess ||
        (e = cudaDeviceSynchronize()) != cudaSuccess) {
      rc = fail(HR2_ECUDA, "setup level-gridded operand: %s", cudaGetErrorString(e));
      goto fail_tmp;
    }
  }
  }
  if ((rc = dalloc_t(ctx, &st->dev, 1))) goto fail_tmp;
  track(st->dev);
  if ((e = cudaMemcpy(st->dev, &h, sizeof(SetupDev), cudaMemcpyHostToDevice)) != cudaSuccess) {
    rc = fail(HR2_ECUDA, "setup descriptor: %s", cudaGetErrorString(e));
    goto fail_tmp;
  }
  if (st->streamed) {
    // the descriptor batches are prepared with on the streamed path: records
    // and weights of the level-gridded sweep (the operand itself comes per
    // group of tiles through the views); st->dev above stays the direct one
    SetupDev hs = h;
    hs.cached = 1;
    if ((rc = dalloc_t(ctx, &st->dev_stream, 1))) goto fail_tmp;
    track(st->dev_stream);
    if ((e = cudaMemcpy(st->dev_stream, &hs, sizeof(SetupDev), cudaMemcpyHostToDevice)) != cudaSuccess) {
      rc = fail(HR2_ECUDA, "setup descriptor: %s", cudaGetErrorString(e));
      goto fail_tmp;
    }
  }
  dfree(ctx, d_quad);
  dfree(ctx, d_edges);
  dfree(ctx, d_lo);
  dfree(ctx, d_hi);
  dfree(ctx, d_bin);
  dfree(ctx, d_invz);
  dfree(ctx, d_rowinfo);
  dfree(ctx, d_err);
  ctx->setups.push_back(st);
  if (d->obs_flux) {
    rc = hr2_setup_set_observation(ctx, st, d->obs_flux, d->obs_sigma);
    if (rc) {
      std::string keep = t_last_error;
      hr2_setup_destroy(ctx, st);
      t_last_error = keep;
      return rc;
    }
  }
  *out = st;
  return HR2_OK;
fail_tmp:
  dfree(ctx, d_edges);
  dfree(ctx, d_lo);
  dfree(ctx, d_hi);
  dfree(ctx, d_bin);
  dfree(ctx, d_invz);
  dfree(ctx, d_rowinfo);
  dfree(ctx, d_err);
fail_all:
  dfree(ctx, d_quad);
  for (void* p : st->mem) dfree(ctx, p);
  delete st;
  return rc;
}

extern "C" int hr2_setup_info(const hr2_setup* s, int* n_bins, int* n_nu, long long* nnz) {
  if (!s) return fail(HR2_EINVAL, "setup is NULL");
  if (n_bins) *n_bins = s->host.n_bins;
  if (n_nu) *n_nu = s->host.n_nu;
  if (nnz) *nnz = s->host.w_nnz;
  return HR2_OK;
}

extern "C" int hr2_setup_memory(const hr2_setup* s, size_t* bytes, size_t* operand_bytes, int* level_gridded) {
  if (!s) return fail(HR2_EINVAL, "setup is NULL");
  size_t total = 0;
  for (void* p : s->mem) {
    auto it = s->ctx->blocks.find(p);
    if (it != s->ctx->blocks.end()) total += it->second;
  }
  if (bytes) *bytes = total;
  if (operand_bytes) *operand_bytes = s->operand_bytes;
  if (level_gridded) *level_gridded = s->host.cached ? 1 : (s->streamed ? HR2_LEVEL_CACHE_STREAM : 0);
  return HR2_OK;
}

extern "C" int hr2_setup_destroy(hr2_ctx* ctx, hr2_setup* s) {
  if (!ctx || !s) return fail(HR2_EINVAL, "NULL argument");
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (void* p : s->mem) dfree(ctx, p);
  ctx->setups.erase(std::remove(ctx->setups.begin(), ctx->setups.end(), s), ctx->setups.end());
  delete s;
  return HR2_OK;
}

// ------------------------------------------------------------ batch calls
struct BatchShape {
  int max_lev = 0, max_nu = 0, max_bins = 0, max_mu = 0, max_k = 0, min_k = 1 << 30, storage = 0, cached = 0;
  int max_tiles = 0;
  int linear = 0, para = 0;
};

static int check_setups(hr2_ctx* ctx, int n_setups, const hr2_setup* const* setups, BatchShape* sh) {
  if (n_setups < 1 || n_setups > HR2_MAX_SETUPS)
    return fail(HR2_EINVAL, "n_setups %d outside [1, %d]", n_setups, HR2_MAX_SETUPS);
  if (!setups) return fail(HR2_EINVAL, "setups is NULL");
  const hr2_tables* t0 = nullptr;
  for (int g = 0; g < n_setups; ++g) {
    const hr2_setup* s = setups[g];
    if (!s || s->ctx != ctx) return fail(HR2_EINVAL, "setups[%d] is not a setup of this context", g);
    if (!t0) t0 = s->tables;
    if (s->tables->host.storage != t0->host.storage)
      return fail(HR2_EINVAL, "setups of one batch must share the table storage type");
    if (s->host.cached != setups[0]->host.cached)
      return fail(HR2_EINVAL, "setups of one batch must all use, or all not use, the level-gridded operand");
    if (s->host.interp != setups[0]->host.interp)
      return fail(HR2_EINVAL, "setups of one batch must share the interpolation option");
    if (s->host.sc != setups[0]->host.sc)
      return fail(HR2_EINVAL, "setups of one batch must share the source interpolation (linear or parabolic)");
    sh->max_lev = std::max(sh->max_lev, s->host.n_lev);
    sh->max_nu = std::max(sh->max_nu, s->host.n_nu);
    sh->max_bins = std::max(sh->max_bins, s->host.n_bins);
    sh->max_mu = std::max(sh->max_mu, s->host.n_mu);
    sh->max_k = std::max(sh->max_k, s->host.n_species);
    sh->min_k = std::min(sh->min_k, s->host.n_species);
    sh->max_tiles = std::max(sh->max_tiles, s->host.n_tiles);
  }
  sh->storage = t0->host.storage;
  sh->cached = setups[0]->host.cached;
  sh->linear = setups[0]->host.interp == HR2_INTERP_LINEAR;
  sh->para = setups[0]->host.sc == HR2_SC_PARABOLIC;
  return HR2_OK;
}

// Launch shape of one batch: the configured samples per work item, reduced
// for batches smaller than that (a work item's warps would idle otherwise)
// and so that the cached path's per-warp pipelines fit the CTA's shared
// memory; the persistent CTAs per SM are raised to keep the configured
// number of warps per SM.
struct LaunchShape {
  int warps, ctas_per_sm, stages;
};
// Compile-time absorber bound of the cached forward kernel: the batch's
// largest absorber count rounded up to even, when no setup of the batch has
// more than 4 absorbers fewer (padded absorbers get weight 0 and read finite
// values of the stage; on the uneven 6-10-absorber batch this is 3 % faster
// than the runtime-count loop, with identical results), else 0 (runtime
// count).
static int absorber_bound(const BatchShape& sh) {
  if (!sh.cached || sh.max_k < 1) return 0;
  const int kt = (sh.max_k + 1) & ~1;
  return (kt - sh.min_k <= 4 && kt <= HR2_MAX_SPECIES) ? kt : 0;
}

// The angle-node constants of each setup as packed pairs of equal floats.
static void fill_node_constants(FwdArgs& a, int n_setups, const hr2_setup* const* setups) {
  auto pair = [](float f) {
    unsigned u;
    memcpy(&u, &f, sizeof(u));
    return ((unsigned long long)u << 32) | u;
  };
  for (int g = 0; g < n_setups; ++g)
    for (int k = 0; k < HR2_MAX_MU; ++k) {
      a.node_im[g][k] = pair(setups[g]->host.inv_mu[k]);
      a.node_lw[g][k] = pair(setups[g]->host.lwmu[k]);
    }
  if (n_setups > 0)
    for (int k = 0; k < HR2_MAX_MU; ++k) {
      a.node_mnl0[k] = pair(setups[0]->host.mu_nlog2e[k]);
      a.node_mu0[k] = pair(setups[0]->host.mu[k]);
    }
}

static LaunchShape shape_for(const hr2_ctx* ctx, const BatchShape& sh, int n) {
  int w = std::min(std::min(ctx->cfg.warps_per_cta, kForwardMaxThreads / 32), std::max(1, n));
  int st = forward32_stages(sh.max_mu, sh.para != 0, absorber_bound(sh), n);
  // a requested pipeline depth where the kernel exists in both depths
  if (ctx->cfg.stages && forward32_has_both_depths(sh.max_mu, sh.para != 0, absorber_bound(sh)))
    st = ctx->cfg.stages;
  if (sh.cached) {
    while (w > 1 && forward32_smem_bytes(w, sh.max_k, st) > kForwardSmemCap) --w;
  }
  const int target = ctx->cfg.warps_per_cta * ctx->cfg.ctas_per_sm;
  const int ctas = std::max(1, std::min(32, (target + w - 1) / w));
  return {w, ctas, st};
}

// The fields of a batch's kernel arguments that come from the context, the
// stream's workspace and the caller's inputs (setups, outputs and the
// two-pass or streamed extras are the caller's).
static void fill_batch_args(FwdArgs& a, const hr2_ctx* ctx, const Workspace* w, const LaunchShape& ls,
                            const int* setup_of_sample, const double* params, int n, int* out_status) {
  a.n = n;
  a.setup_of_sample = setup_of_sample;
  a.params = params;
  a.perm = w->perm;
  a.plan = w->plan;
  a.counter = w->counter;
  a.status = out_status;
  a.recs = w->recs;
  a.rec_ld = w->lev_cap;
  a.samp = w->samp;
  a.warps = ls.warps;
  a.tiles_per_item = ctx->cfg.tiles_per_item;
  a.err = (int*)(w->counter + 1);
  a.wait_limit = ctx->wait_limit;
  a.tx_extra = ctx->wait_fault ? 16u : 0u;
}

// Batches of at least this many samples on a single streamed setup take the
// streamed operand; smaller ones (and mixed batches) read the tables directly.
// On the 290001-point, 12-absorber tables (a prior-drawn batch, about half of
// the (level, T cell) blocks built): 12.4 ms at 32 samples against 13.0 ms
// read directly, 15.1 against 19.4 ms at 48; below 32 the direct path wins.
constexpr int kStreamMinBatch = 32;
// largest ring of the streamed operand chosen automatically (on the
// 290001-point tables at batch 64: 27.1 ms with 1 GiB, 22.4 ms with 4 GiB)
constexpr size_t kStreamRingMaxBytes = (size_t)4 << 30;
// forward_streamed: no ring fits; the caller evaluates the batch directly
constexpr int kStreamFallback = 1;

// One batch on setups created with HR2_LEVEL_CACHE_STREAM (all of the call's
// setups): the samples are prepared once (records of the level-gridded
// sweep), then, per group of consecutive tiles (the same count of each
// setup's own tiles), each setup's operand of the group is built into its
// section of the stream's ring (k_level_stream; only the (level, T cell)
// blocks some sample of the batch sits in, from k_mark_cells), the work of
// the group is planned and the persistent forward kernel sweeps it through
// the group's setup views (a setup whose tiles are all behind has none);
// the binning runs once over the whole range.  Groups are sized so that each
// holds about eight work items per persistent CTA (or ctx->stream_group
// tiles), with the ring at most kStreamRingMaxBytes.
static int forward_streamed(hr2_ctx* ctx, int n_setups, const hr2_setup* const* setups, BatchShape sh,
                            const int* setup_of_sample, const double* params, int n, float* out_bins, int bins_ld,
                            float* out_highres, int highres_ld, int* out_status, cudaStream_t s) {
  sh.cached = 1;   // the sweep reads a level-gridded operand, from the ring
  Workspace* w = nullptr;
  int rc = ws_ensure(ctx, s, n, sh.max_lev, out_highres ? 0 : sh.max_nu, 0, 0, 0, &w);
  if (rc) return rc;
  const LaunchShape ls = shape_for(ctx, sh, n);
  const int grid = ctx->n_sm * ls.ctas_per_sm;
  // floats of one tile of every setup's operand, and its section offsets
  size_t per_tile_all = 0;
  int max_cells = 1;
  for (int g = 0; g < n_setups; ++g) {
    per_tile_all += (size_t)setups[g]->host.lvl32_tile_floats;
    max_cells = std::max(max_cells, setups[g]->tables->host.n_T - 1);
  }
  const int max_tiles = sh.max_tiles;
  int group = ctx->stream_group;
  if (group <= 0) {
    const long long sblocks = (n + ls.warps - 1) / ls.warps;
    const long long tpi = std::max(1, ctx->cfg.tiles_per_item);
    group = (int)std::min<long long>(max_tiles, (8LL * grid * tpi + sblocks - 1) / sblocks);
    group = (int)std::min<size_t>((size_t)group, std::max<size_t>(1, kStreamRingMaxBytes / (per_tile_all * sizeof(float))));
  }
  group = std::max(1, std::min(group, max_tiles));
  const size_t mask_bytes = (size_t)n_setups * sh.max_lev * max_cells;
  {
    // within the context's budget (what the ring already holds counts as free)
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->budget) {
      const size_t held = w->ring_cap * sizeof(float) + (size_t)w->views_cap * sizeof(SetupDev) + w->cells_cap;
      const size_t room = ctx->budget > ctx->used - std::min(ctx->used, held) ? ctx->budget - (ctx->used - std::min(ctx->used, held)) : 0;
      const size_t fixed = (size_t)max_tiles * n_setups * sizeof(SetupDev) + mask_bytes;
      const size_t fit = room > fixed ? (room - fixed) / (per_tile_all * sizeof(float)) : 0;
      group = (int)std::min<size_t>((size_t)group, fit);
    }
  }
  if (group < 1) return kStreamFallback;
  const int n_groups = (max_tiles + group - 1) / group;
  if ((rc = ws_ensure_stream(ctx, s, w, (size_t)group * per_tile_all, n_groups * n_setups, mask_bytes))) {
    if (rc == HR2_ENOMEM) return kStreamFallback;   // the call reads the tables directly
    return rc;
  }
  FwdArgs a{};
  for (int g = 0; g < n_setups; ++g) a.setups[g] = setups[g]->dev_stream;
  a.n_setups = n_setups;
  fill_batch_args(a, ctx, w, ls, setup_of_sample, params, n, out_status);
  a.highres = out_highres ? out_highres : w->highres;
  a.highres_ld = out_highres ? highres_ld : w->nu_cap;
  fill_node_constants(a, n_setups, setups);
  cudaError_t e;
  if ((e = launch_prep(a, s)) != cudaSuccess) return fail(HR2_ECUDA, "prep launch: %s", cudaGetErrorString(e));
  std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
  if (ctx->profiling) {
    HR2_CU(cudaEventCreate(&ev.first));
    if ((e = cudaEventCreate(&ev.second)) != cudaSuccess) {
      cudaEventDestroy(ev.first);
      return fail(HR2_ECUDA, "cudaEventCreate: %s", cudaGetErrorString(e));
    }
  }
  auto launch_failed = [&](const char* what, cudaError_t err) {
    if (ev.first) cudaEventDestroy(ev.first);
    if (ev.second) cudaEventDestroy(ev.second);
    return fail(HR2_ECUDA, "%s launch: %s", what, cudaGetErrorString(err));
  };
  // (the profiling events bracket every group: operand builds, plans and sweeps)
  if (ev.first && (e = cudaEventRecord(ev.first, s)) != cudaSuccess) return launch_failed("event", e);
  std::vector<size_t> off(n_setups);
  size_t acc = 0;
  for (int g = 0; g < n_setups; ++g) {
    off[g] = acc;
    acc += (size_t)group * setups[g]->host.lvl32_tile_floats;
    if ((e = build_stream_views(setups[g]->dev_stream, w->ring + off[g], group, n_groups, g, n_setups, w->views, s)) !=
        cudaSuccess)
      return launch_failed("setup views", e);
  }
  // the (level, T cell) pairs the batch's samples sit in, per setup: the only blocks built
  if ((e = build_cell_mask(a, sh.max_lev, max_cells, w->cells, s)) != cudaSuccess) return launch_failed("cell mask", e);
  for (int q = 0; q < n_groups; ++q) {
    const int lo = q * group;
    FwdArgs ag = a;
    for (int g = 0; g < n_setups; ++g) {
      const SetupDev& h = setups[g]->host;
      const int cnt = std::min(group, h.n_tiles - lo);
      if (cnt > 0 &&
          (e = build_level_stream(setups[g]->dev_stream, h.n_lev, h.n_species + 2, lo, cnt,
                                  w->cells + (size_t)g * sh.max_lev * max_cells, max_cells, w->ring + off[g], s)) !=
              cudaSuccess)
        return launch_failed("streamed operand", e);
      ag.setups[g] = w->views + (size_t)q * n_setups + g;
    }
    FwdArgs ap = ag;
    if (q > 0) ap.err = nullptr;   // the first plan cleared the error word; later groups keep what it holds
    if ((e = launch_plan(ap, w->perm, w->plan, s)) != cudaSuccess) return launch_failed("plan", e);
    if ((e = launch_forward32(ag, sh.max_mu, grid, true, sh.linear != 0, sh.para != 0, sh.max_k, absorber_bound(sh),
                              ls.stages, s)) != cudaSuccess)
      return launch_failed("forward32", e);
  }
  if (ev.second && (e = cudaEventRecord(ev.second, s)) != cudaSuccess) return launch_failed("event", e);
  if (ev.first) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->prof.push_back(ev);
  }
  if ((e = launch_bins(a, out_bins, bins_ld, false, s)) != cudaSuccess)
    return fail(HR2_ECUDA, "bins launch: %s", cudaGetErrorString(e));
  return HR2_OK;
}

extern "C" int forward_model_batch(hr2_ctx* ctx, int n_setups, const hr2_setup* const* setups,
                                   const int* setup_of_sample, const double* params, int n, float* out_bins,
                                   int bins_ld, float* out_highres, int highres_ld, int* out_status, void* stream) {
  HR2_RANGE("forward_model_batch");
  if (!ctx) return fail(HR2_EINVAL, "ctx is NULL");
  if (n < 0) return fail(HR2_EINVAL, "n < 0");
  BatchShape sh;
  int rc = check_setups(ctx, n_setups, setups, &sh);
  if (rc) return rc;
  if (n == 0) return HR2_OK;
  if (!setup_of_sample || !params || !out_bins) return fail(HR2_EINVAL, "setup_of_sample, params, out_bins required");
  if (bins_ld < sh.max_bins) return fail(HR2_EINVAL, "bins_ld %d < largest n_bins %d", bins_ld, sh.max_bins);
  if (out_highres && highres_ld < sh.max_nu)
    return fail(HR2_EINVAL, "highres_ld %d < largest n_nu %d", highres_ld, sh.max_nu);
  const bool fp64 = sh.storage == HR2_STORE_FP64;
  if (fp64 && n > 65535) return fail(HR2_EINVAL, "the FP64 path takes at most 65535 samples per call");
  HR2_CU(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  bool all_streamed = true;
  for (int g = 0; g < n_setups; ++g) all_streamed = all_streamed && setups[g]->streamed;
  if (all_streamed && n >= kStreamMinBatch) {
    rc = forward_streamed(ctx, n_setups, setups, sh, setup_of_sample, params, n, out_bins, bins_ld, out_highres,
                          highres_ld, out_status, s);
    if (rc != kStreamFallback) return rc;
    t_last_error.clear();
  }
  Workspace* w = nullptr;
  rc = ws_ensure(ctx, s, n, sh.max_lev, (!fp64 && !out_highres) ? sh.max_nu : 0, fp64 ? sh.max_nu : 0, 0, 0, &w);
  if (rc) return rc;
  FwdArgs a{};
  for (int g = 0; g < n_setups; ++g) a.setups[g] = setups[g]->dev;
  a.n_setups = n_setups;
  const LaunchShape ls = shape_for(ctx, sh, n);
  fill_batch_args(a, ctx, w, ls, setup_of_sample, params, n, out_status);
  fill_node_constants(a, n_setups, setups);
  // small batches on tables read in place run in two passes: the absorption
  // coefficients of every level first, in parallel, then the sweep; their
  // buffer is sized before anything is launched
  const bool two_pass = !fp64 && !sh.cached && !sh.para && n <= ctx->cfg.split_max_batch;
  if (two_pass) {
    a.chi_ld = (long long)sh.max_tiles * kTileNu;
    if ((rc = ws_ensure_chi(ctx, s, w, (size_t)n * w->lev_cap * a.chi_ld))) return rc;
    a.chi = w->chi;
  }
  cudaError_t e;
  if ((e = launch_prep(a, s)) != cudaSuccess) return fail(HR2_ECUDA, "prep launch: %s", cudaGetErrorString(e));
  std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
  if (ctx->profiling) {
    HR2_CU(cudaEventCreate(&ev.first));
    if ((e = cudaEventCreate(&ev.second)) != cudaSuccess) {
      cudaEventDestroy(ev.first);
      return fail(HR2_ECUDA, "cudaEventCreate: %s", cudaGetErrorString(e));
    }
  }
  // a failed launch after the events exist releases them
  auto launch_failed = [&](const char* what, cudaError_t err) {
    if (ev.first) cudaEventDestroy(ev.first);
    if (ev.second) cudaEventDestroy(ev.second);
    return fail(HR2_ECUDA, "%s launch: %s", what, cudaGetErrorString(err));
  };
  if (fp64) {
    if ((e = cudaMemsetAsync(a.err, 0, sizeof(int), s)) != cudaSuccess)   // the planner clears it on the FP32 path
      return launch_failed("error-word clear", e);
    if (ev.first && (e = cudaEventRecord(ev.first, s)) != cudaSuccess) return launch_failed("event", e);
    a.highres64 = w->highres64;
    a.highres64_ld = w->nu64_cap;
    a.user_highres = out_highres;
    a.highres = out_highres;
    a.highres_ld = highres_ld;
    if ((e = launch_forward64(a, sh.max_mu, sh.max_nu, s)) != cudaSuccess) return launch_failed("forward64", e);
    if (ev.second && (e = cudaEventRecord(ev.second, s)) != cudaSuccess) return launch_failed("event", e);
  } else {
    a.highres = out_highres ? out_highres : w->highres;
    a.highres_ld = out_highres ? highres_ld : w->nu_cap;
    if ((e = launch_plan(a, w->perm, w->plan, s)) != cudaSuccess) return launch_failed("plan", e);
    // (the profiling events bracket both passes of the two-pass path)
    if (ev.first && (e = cudaEventRecord(ev.first, s)) != cudaSuccess) return launch_failed("event", e);
    if (two_pass && (e = launch_chi_direct(a, sh.max_lev, sh.max_tiles, s)) != cudaSuccess)
      return launch_failed("absorption pass", e);
    const int grid = ctx->n_sm * ls.ctas_per_sm;
    if ((e = launch_forward32(a, sh.max_mu, grid, sh.cached != 0, sh.linear != 0, sh.para != 0, sh.max_k, absorber_bound(sh),
                              ls.stages, s)) != cudaSuccess)
      return launch_failed("forward32", e);
    if (ev.second && (e = cudaEventRecord(ev.second, s)) != cudaSuccess) return launch_failed("event", e);
  }
  if (ev.first) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->prof.push_back(ev);
  }
  if ((e = launch_bins(a, out_bins, bins_ld, fp64, s)) != cudaSuccess)
    return fail(HR2_ECUDA, "bins launch: %s", cudaGetErrorString(e));
  return HR2_OK;
}

extern "C" int log_likelihood_batch(hr2_ctx* ctx, int n_setups, const hr2_setup* const* setups,
                                    const int* setup_of_sample, const float* model_bins, int bins_ld,
                                    const double* log_eps, int n, double* out_lnL, void* stream) {
  HR2_RANGE("log_likelihood_batch");
  if (!ctx) return fail(HR2_EINVAL, "ctx is NULL");
  if (n < 0) return fail(HR2_EINVAL, "n < 0");
  BatchShape sh;
  int rc = check_setups(ctx, n_setups, setups, &sh);
  if (rc) return rc;
  for (int g = 0; g < n_setups; ++g)
    if (!setups[g]->has_obs) return fail(HR2_EINVAL, "setups[%d] has no observation", g);
  if (n == 0) return HR2_OK;
  if (!setup_of_sample || !model_bins || !out_lnL) return fail(HR2_EINVAL, "NULL buffer");
  if (bins_ld < sh.max_bins) return fail(HR2_EINVAL, "bins_ld %d < largest n_bins %d", bins_ld, sh.max_bins);
  HR2_CU(cudaSetDevice(ctx->device));
  LnlArgs a{};
  for (int g = 0; g < n_setups; ++g) a.setups[g] = setups[g]->dev;
  a.n_setups = n_setups;
  a.setup_of_sample = setup_of_sample;
  a.bins = model_bins;
  a.bins_ld = bins_ld;
  a.log_eps = log_eps;
  a.n = n;
  a.lnl = out_lnL;
  cudaError_t e = launch_lnl(a, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(HR2_ECUDA, "lnL launch: %s", cudaGetErrorString(e));
  return HR2_OK;
}

// The status a batch's device error word stands for.
static int error_word_status(unsigned word, const char* what) {
  if (word & (unsigned)kErrBounds)
    return fail(HR2_EBOUNDS, "a device-side index check failed during %s (bounds-checked build)", what);
  if (word & (unsigned)kErrWait) return fail(HR2_ETIMEDOUT, "a bounded device-side wait gave up during %s", what);
  return HR2_OK;
}

// Reads the device error word of a workspace (the stream must be idle).
static int check_device_error(const Workspace* w) {
  if (!w || !w->counter) return HR2_OK;
  unsigned int word[2] = {0, 0};
  HR2_CU(cudaMemcpy(word, w->counter, sizeof(word), cudaMemcpyDeviceToHost));
  return error_word_status(word[1], "the last batch");
}

extern "C" int hr2_evaluate_host(hr2_ctx* ctx, int n_setups, const hr2_setup* const* setups,
                                 const int* setup_of_sample, const double* params, const double* log_eps, int n,
                                 double* out_lnL, float* out_bins, int bins_ld, void* stream) {
  HR2_RANGE("hr2_evaluate_host");
  if (!ctx) return fail(HR2_EINVAL, "ctx is NULL");
  if (n < 0) return fail(HR2_EINVAL, "n < 0");
  BatchShape sh;
  int rc = check_setups(ctx, n_setups, setups, &sh);
  if (rc) return rc;
  if (n == 0) return HR2_OK;
  if (!setup_of_sample || !params || !out_lnL) return fail(HR2_EINVAL, "NULL buffer");
  if (out_bins && bins_ld < sh.max_bins) return fail(HR2_EINVAL, "bins_ld %d < largest n_bins", bins_ld);
  const int ld = out_bins ? bins_ld : sh.max_bins;
  HR2_CU(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  Workspace* w = nullptr;
  // size everything the batch needs up front, so that the calls below do not
  // grow (and so move) the buffers the inputs were copied into
  const bool fp64 = sh.storage == HR2_STORE_FP64;
  if ((rc = ws_ensure(ctx, s, n, sh.max_lev, fp64 ? 0 : sh.max_nu, fp64 ? sh.max_nu : 0, n, ld, &w))) return rc;
  HR2_CU(cudaMemcpyAsync(w->io_sos, setup_of_sample, sizeof(int) * n, cudaMemcpyHostToDevice, s));
  HR2_CU(cudaMemcpyAsync(w->io_params, params, sizeof(double) * HR2_NPARAM * (size_t)n, cudaMemcpyHostToDevice, s));
  if (log_eps) HR2_CU(cudaMemcpyAsync(w->io_logeps, log_eps, sizeof(double) * n, cudaMemcpyHostToDevice, s));
  if ((rc = forward_model_batch(ctx, n_setups, setups, w->io_sos, w->io_params, n, w->io_bins, ld, nullptr, 0,
                                nullptr, stream)))
    return rc;
  if ((rc = log_likelihood_batch(ctx, n_setups, setups, w->io_sos, w->io_bins, ld, log_eps ? w->io_logeps : nullptr,
                                 n, w->io_lnl, stream)))
    return rc;
  HR2_CU(cudaMemcpyAsync(out_lnL, w->io_lnl, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  if (out_bins)
    HR2_CU(cudaMemcpyAsync(out_bins, w->io_bins, sizeof(float) * (size_t)n * ld, cudaMemcpyDeviceToHost, s));
  if (w->h_counter) {
    // the error word comes back with the results: no second round trip
    HR2_CU(cudaMemcpyAsync(w->h_counter, w->counter, 2 * sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    HR2_CU(cudaStreamSynchronize(s));
    return error_word_status(w->h_counter[1], "the last batch");
  }
  HR2_CU(cudaStreamSynchronize(s));
  return check_device_error(w);
}

extern "C" int hr2_stream_check(hr2_ctx* ctx, void* stream) {
  HR2_RANGE("hr2_stream_check");
  if (!ctx) return fail(HR2_EINVAL, "ctx is NULL");
  HR2_CU(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  HR2_CU(cudaStreamSynchronize(s));
  Workspace* w = nullptr;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->ws.find((void*)s);
    if (it == ctx->ws.end()) return HR2_OK;
    w = it->second;
  }
  return check_device_error(w);
}

// ------------------------------------------------------------ effective temperature
extern "C" int hr2_effective_temperature(hr2_ctx* ctx, int n_setups, const hr2_setup* const* setups,
                                         const int* setup_of_sample, const float* highres, int highres_ld, int n,
                                         double* out_teff, void* stream) {
  HR2_RANGE("hr2_effective_temperature");
  if (!ctx) return fail(HR2_EINVAL, "ctx is NULL");
  if (n < 0) return fail(HR2_EINVAL, "n < 0");
  BatchShape sh;
  int rc = check_setups(ctx, n_setups, setups, &sh);
  if (rc) return rc;
  if (n == 0) return HR2_OK;
  if (!setup_of_sample || !highres || !out_teff) return fail(HR2_EINVAL, "setup_of_sample, highres, out_teff required");
  if (highres_ld < sh.max_nu) return fail(HR2_EINVAL, "highres_ld %d < largest n_nu %d", highres_ld, sh.max_nu);
  HR2_CU(cudaSetDevice(ctx->device));
  FwdArgs a{};
  for (int g = 0; g < n_setups; ++g) a.setups[g] = setups[g]->dev;
  a.n_setups = n_setups;
  a.n = n;
  a.setup_of_sample = setup_of_sample;
  cudaError_t e = launch_teff(a, highres, highres_ld, out_teff, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(HR2_ECUDA, "effective temperature launch: %s", cudaGetErrorString(e));
  return HR2_OK;
}

// ------------------------------------------------------------ nested sampling
extern "C" int hr2_ns_state_init(hr2_ctx* ctx, hr2_ns_state* state, void* stream) {
  if (!ctx || !state) return fail(HR2_EINVAL, "NULL argument");
  HR2_CU(cudaSetDevice(ctx->device));
  cudaError_t e = launch_ns_init(state, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(HR2_ECUDA, "ns init launch: %s", cudaGetErrorString(e));
  return HR2_OK;
}

extern "C" int hr2_ns_absorb(hr2_ctx* ctx, int n_live, double* live_lnl, double* live_theta, int n_cand,
                             const double* cand_lnl, const double* cand_theta, hr2_ns_state* state, double* dead_lnl,
                             double* dead_logw, double* dead_theta, long long dead_cap, void* stream) {
  HR2_RANGE("hr2_ns_absorb");
  if (!ctx) return fail(HR2_EINVAL, "ctx is NULL");
  if (n_live < 1 || n_cand < 0 || dead_cap < 0) return fail(HR2_EINVAL, "need n_live >= 1, n_cand >= 0, dead_cap >= 0");
  if (!live_lnl || !live_theta || !state || (n_cand && (!cand_lnl || !cand_theta)) ||
      (dead_cap && (!dead_lnl || !dead_logw || !dead_theta)))
    return fail(HR2_EINVAL, "NULL argument");
  HR2_CU(cudaSetDevice(ctx->device));
  cudaError_t e = launch_ns_absorb(n_live, live_lnl, live_theta, n_cand, cand_lnl, cand_theta, state, dead_lnl,
                                   dead_logw, dead_theta, dead_cap, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(HR2_ECUDA, "ns absorb launch: %s", cudaGetErrorString(e));
  return HR2_OK;
}

extern "C" int hr2_ns_propose(hr2_ctx* ctx, int n_live, const double* live_theta, const double* prior_lo,
                              const double* prior_hi, double enlarge, int n, double* box, double* out_theta,
                              unsigned long long seed, unsigned long long counter, void* stream) {
  HR2_RANGE("hr2_ns_propose");
  if (!ctx) return fail(HR2_EINVAL, "ctx is NULL");
  if (n_live < 1 || n < 0 || !(enlarge >= 0.0)) return fail(HR2_EINVAL, "need n_live >= 1, n >= 0, enlarge >= 0");
  if (!live_theta || !prior_lo || !prior_hi || !box || (n && !out_theta)) return fail(HR2_EINVAL, "NULL argument");
  HR2_CU(cudaSetDevice(ctx->device));
  cudaError_t e = launch_ns_propose(n_live, live_theta, prior_lo, prior_hi, enlarge, n, box, out_theta, seed, counter,
                                    (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(HR2_ECUDA, "ns propose launch: %s", cudaGetErrorString(e));
  return HR2_OK;
}

extern "C" int hr2_ns_finalize(hr2_ctx* ctx, int n_live, const double* live_lnl, const hr2_ns_state* state,
                               double* out, void* stream) {
  HR2_RANGE("hr2_ns_finalize");
  if (!ctx) return fail(HR2_EINVAL, "ctx is NULL");
  if (n_live < 1 || !live_lnl || !state || !out) return fail(HR2_EINVAL, "need n_live >= 1 and non-NULL pointers");
  HR2_CU(cudaSetDevice(ctx->device));
  cudaError_t e = launch_ns_finalize(n_live, live_lnl, state, out, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(HR2_ECUDA, "ns finalize launch: %s", cudaGetErrorString(e));
  return HR2_OK;
}

// ------------------------------------------------------------ instrumentation
extern "C" int hr2_profile_enable(hr2_ctx* ctx, int on) {
  if (!ctx) return fail(HR2_EINVAL, "ctx is NULL");
  ctx->profiling = on != 0;
  return HR2_OK;
}

extern "C" int hr2_profile_read(hr2_ctx* ctx, int reset, double* kernel_ms, int* launches) {
  if (!ctx) return fail(HR2_EINVAL, "ctx is NULL");
  std::lock_guard<std::mutex> lk(ctx->mu);
  double total = 0.0;
  for (auto& ev : ctx->prof) {
    HR2_CU(cudaEventSynchronize(ev.second));
    float ms = 0.f;
    HR2_CU(cudaEventElapsedTime(&ms, ev.first, ev.second));
    total += ms;
  }
  if (kernel_ms) *kernel_ms = total;
  if (launches) *launches = (int)ctx->prof.size();
  if (reset) {
    for (auto& ev : ctx->prof) {
      cudaEventDestroy(ev.first);
      cudaEventDestroy(ev.second);
    }
    ctx->prof.clear();
  }
  return HR2_OK;
}

// ------------------------------------------------------------ helpers
extern "C" int hr2_nodes_from_b(int n_nodes, double T1, const double* b, double* nodes) {
  if (n_nodes < 1 || (n_nodes > 1 && !b) || !nodes) return fail(HR2_EINVAL, "invalid argument");
  nodes[0] = T1;
  for (int i = 1; i < n_nodes; ++i) nodes[i] = b[i - 1] * nodes[i - 1];
  return HR2_OK;
}

extern "C" const char* hr2_version(void) { return "hr2-b300 0.1 (sm_103a)"; }

// ------------------------------------------------------------ allocation-free variant
// forward_model_batch_noalloc: the FP32 forward path with its scratch in one
// static device array instead of the context's workspace.  Nothing here calls
// cudaMalloc, cudaFree or an allocating routine.
namespace {
constexpr size_t kNoallocBytes = HR2_NOALLOC_SCRATCH_BYTES;
constexpr int kNoallocMaxDevices = 64;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoallocMaxDevices] = {};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
// the array's layout: plan, then {work counter, error word}, then the batch's
// permutation, per-sample records and per-level records
size_t noalloc_counter_offset() { return align256(sizeof(PlanDev)); }

// Device address of the array on the current device (looked up once per device).
int noalloc_scratch(int device, void** out) {
  if (device < 0 || device >= kNoallocMaxDevices) return fail(HR2_EINVAL, "device %d unsupported", device);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return fail(HR2_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_noalloc_addr[device] = p;
  }
  *out = g_noalloc_addr[device];
  return HR2_OK;
}
}  // namespace

extern "C" int forward_model_batch_noalloc(hr2_ctx* ctx, int n_setups, const hr2_setup* const* setups,
                                           const int* setup_of_sample, const double* params, int n, float* out_bins,
                                           int bins_ld, float* out_highres, int highres_ld, int* out_status,
                                           void* stream) {
  HR2_RANGE("forward_model_batch_noalloc");
  if (!ctx) return fail(HR2_EINVAL, "ctx is NULL");
  if (n < 0) return fail(HR2_EINVAL, "n < 0");
  BatchShape sh;
  int rc = check_setups(ctx, n_setups, setups, &sh);
  if (rc) return rc;
  if (sh.storage != HR2_STORE_FP16_OFFSET)
    return fail(HR2_EINVAL, "the allocation-free variant runs FP16-offset tables only");
  if (n == 0) return HR2_OK;
  if (!setup_of_sample || !params || !out_bins || !out_highres)
    return fail(HR2_EINVAL, "setup_of_sample, params, out_bins and out_highres are required");
  if (bins_ld < sh.max_bins) return fail(HR2_EINVAL, "bins_ld %d < largest n_bins %d", bins_ld, sh.max_bins);
  if (highres_ld < sh.max_nu) return fail(HR2_EINVAL, "highres_ld %d < largest n_nu %d", highres_ld, sh.max_nu);
  const size_t off_counter = noalloc_counter_offset();
  const size_t off_perm = off_counter + 256;
  const size_t off_samp = off_perm + align256(sizeof(int) * (size_t)n);
  const size_t off_recs = off_samp + align256(sizeof(SampleDev) * (size_t)n);
  const size_t need = off_recs + sizeof(LevRec) * (size_t)n * sh.max_lev;
  if (need > kNoallocBytes)
    return fail(HR2_EINVAL, "batch of %d samples with %d levels needs %zu bytes of scratch; the allocation-free "
                "variant holds %zu", n, sh.max_lev, need, kNoallocBytes);
  HR2_CU(cudaSetDevice(ctx->device));
  char* base = nullptr;
  if ((rc = noalloc_scratch(ctx->device, (void**)&base))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  FwdArgs a{};
  for (int g = 0; g < n_setups; ++g) a.setups[g] = setups[g]->dev;
  a.n_setups = n_setups;
  a.n = n;
  a.setup_of_sample = setup_of_sample;
  a.params = params;
  a.plan = (const PlanDev*)base;
  a.counter = (unsigned int*)(base + off_counter);
  a.err = (int*)(base + off_counter + sizeof(unsigned int));
  a.perm = (const int*)(base + off_perm);
  a.samp = (SampleDev*)(base + off_samp);
  a.recs = (LevRec*)(base + off_recs);
  a.rec_ld = sh.max_lev;
  a.status = out_status;
  a.highres = out_highres;
  a.highres_ld = highres_ld;
  const LaunchShape ls = shape_for(ctx, sh, n);
  a.warps = ls.warps;
  a.tiles_per_item = ctx->cfg.tiles_per_item;
  a.wait_limit = ctx->wait_limit;
  a.tx_extra = ctx->wait_fault ? 16u : 0u;
  fill_node_constants(a, n_setups, setups);
  cudaError_t e;
  // the planner resets the work counter to zero on the device before the
  // forward kernel reads it; everything else is overwritten by the kernels
  if ((e = launch_prep(a, s)) != cudaSuccess || (e = launch_plan(a, (int*)a.perm, (PlanDev*)a.plan, s)) != cudaSuccess ||
      (e = launch_forward32(a, sh.max_mu, ctx->n_sm * ls.ctas_per_sm, sh.cached != 0, sh.linear != 0, sh.para != 0,
                        sh.max_k, absorber_bound(sh), ls.stages, s)) != cudaSuccess ||
      (e = launch_bins(a, out_bins, bins_ld, false, s)) != cudaSuccess)
    return fail(HR2_ECUDA, "allocation-free launch: %s", cudaGetErrorString(e));
  return HR2_OK;
}

extern "C" int hr2_noalloc_check(hr2_ctx* ctx, void* stream) {
  HR2_RANGE("hr2_noalloc_check");
  if (!ctx) return fail(HR2_EINVAL, "ctx is NULL");
  HR2_CU(cudaSetDevice(ctx->device));
  HR2_CU(cudaStreamSynchronize((cudaStream_t)stream));
  char* base = nullptr;
  int rc = noalloc_scratch(ctx->device, (void**)&base);
  if (rc) return rc;
  unsigned int word = 0;
  // the error word follows the work counter in the array (see the layout in
  // forward_model_batch_noalloc); a 4-byte copy allocates nothing
  HR2_CU(cudaMemcpy(&word, base + noalloc_counter_offset() + sizeof(unsigned int), sizeof(word),
                    cudaMemcpyDeviceToHost));
  return error_word_status(word, "the last allocation-free batch");
}

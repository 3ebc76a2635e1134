// C ABI (include/ebr.h): context, planning, and the orchestration of the
// classification, level, fill, force and adjoint kernels.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/ebr.h"
#include "ebr_kernels.cuh"

using namespace ebr;

namespace ebr {
int g_pdl = 1;
}

// an NVTX range around every entry point (a no-op unless a profiler is
// attached), so that a timeline shows the library's calls
struct EbrRange {
  explicit EbrRange(const char* name) { nvtxRangePushA(name); }
  ~EbrRange() { nvtxRangePop(); }
};

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct ChainPlan {
  int* d_list = nullptr;
  int n_list = 0;
  size_t smem = 0;
  std::vector<int> fallback;   // geometries served by level launches
};

// Launch shapes a caller may tune: threads per block of the kernels that run
// one thread per item (interface cell, ghost or fluid target), where the
// block size changes scheduling only, never a result.  Names are those of
// the kernels' profiling records (ebr_profile_read).
enum TuneId { TU_IFACE, TU_PLACE, TU_GHOST, TU_DEPS, TU_TABLES, TU_GSRC, TU_FILL_PART, TU_ADJ_SEED,
              TU_ADJ_PART, TU_ADJ_PROBE, TU_ADJ_FLUID, TU_ADJ_BC, TU_N };
static const char* const kTuneNames[TU_N] = {"iface", "place", "ghost_geom", "deps", "tables", "gsrc",
                                             "fill_part", "adj_seed", "adj_part", "adj_probe", "adj_fluid",
                                             "adj_bc"};
constexpr int TUNE_DEFAULT = 128;
constexpr int TUNE_MAX = 256;     // every kernel fits at 256 threads (<= 255 registers each)

static int tune_id(const char* name) {
  if (!name) return -1;
  for (int i = 0; i < TU_N; ++i)
    if (std::strcmp(name, kTuneNames[i]) == 0) return i;
  return -1;
}

struct Ctx {
  int device = 0;
  std::string err;
  long long launches = 0;
  std::vector<DevBuf> bufs;    // allocations of the derived plans, freed at the next plan
  struct Slot {
    void* p = nullptr;
    size_t cap = 0;
  };
  std::map<const void*, Slot> slots;   // grow-only buffers of the context's pointer members
  std::map<long long, Slot> chain_slots;  // grow-only geometry lists of the chain plans, by key
  long long n_alloc = 0;               // device allocations made so far

  // geometry set
  int B = 0, placement = 0, layers = 1;
  // stretched grids: per geometry and axis the host cell centres; device
  // centres + widths (doubles) and float centres of all stretched geometries
  std::vector<std::array<std::vector<double>, 3>> h_cen;
  double* coord_d = nullptr;
  float* coord_f = nullptr;
  unsigned long long* stats_buf = nullptr;   // ebr_stats: extrema and histograms
  bool planned = false, levelled = false;
  std::vector<Geom> hG;
  std::vector<int> h_row_off;
  long long total_cells = 0;
  int total_rows = 0;
  Geom* dG = nullptr;
  int* d_row_off = nullptr;

  // status / stats
  int* d_status = nullptr;
  int* d_stats = nullptr;      // [0] row fallbacks, [1] rmax, [2..] n_levels per geometry follow in d_nlev
  int* d_nlev = nullptr;

  // classification
  int2* runs = nullptr;
  int* row_cnt = nullptr;
  int* row_ptr = nullptr;
  int n_iface = 0;
  int* iface_cell = nullptr;
  int* iface_geo = nullptr;
  int8_t* iface_solid = nullptr;
  uint8_t* iface_meta = nullptr;   // normal sign / zero bytes of the HGC candidates
  int8_t* iface_tag = nullptr;     // final tags of a fused re-run, written by the position kernel
  bool tags_pending = false;       // iface_tag holds tags not yet in the tag array
  int* gflag = nullptr;
  int* gpos = nullptr;
  void* scan_tmp = nullptr;
  int8_t* tags = nullptr;      // last tag array the caller gave
  // single-pass scan states of a re-run (rows, interface cells, ghost
  // targets): counters and tile words in one buffer, zeroed at every plan
  unsigned* lb_mem = nullptr;
  Lookback lb_rows{}, lb_iface{}, lb_gsrc{};

  // ghosts
  int ng = 0;
  int rmax = 1;
  int *gs_cell = nullptr, *gs_geo = nullptr, *dep = nullptr, *level = nullptr, *order_pos = nullptr;
  double *gs_psi = nullptr, *gs_n = nullptr;
  uint32_t* gs_meta = nullptr;
  int *g_cell = nullptr, *g_geo = nullptr, *g_dep = nullptr, *g_level = nullptr;
  double *g_psi = nullptr, *g_n = nullptr;
  uint32_t* g_meta = nullptr;
  int* pos_of_cell = nullptr;
  int* lev_ptr = nullptr;
  size_t levels_smem = 0;      // dynamic shared memory of k_levels (planned)
  std::vector<int> h_lev_ptr;
  double* wtab = nullptr;
  double* ftab = nullptr;
  float* wtab_f = nullptr;     // float copies of the tables (kernels of FP32 fields)
  float* ftab_f = nullptr;
  int *gsrc_cnt = nullptr, *gsrc_ptr = nullptr, *gsrc = nullptr;
  int* gsrc_mem = nullptr;     // ghost position of each stencil member [K][ng] (-1: not a ghost)
  int n_gsrc = 0;
  std::vector<int> h_gsrc_geo;   // sources per geometry
  int *own_flag = nullptr, *own_ptr = nullptr, *ft_cell = nullptr, *ft_geo = nullptr,
      *ft_cnt = nullptr, *ft_ptr = nullptr, *ft_src = nullptr;
  int nft = 0, n_fsrc = 0;
  std::vector<long long> h_nft_geo;

  // forces
  int n_chunks = 0;
  int4* chunks = nullptr;
  int* chunk_ptr = nullptr;
  int* chunk_done = nullptr;   // finished chunks per geometry (zero between launches)
  double* partial = nullptr;

  // adjoint scratch
  double* sv = nullptr;        // force coefficients [F * 8][ng] in the field type (room for doubles)
  void* lam = nullptr;
  void* fpart = nullptr;       // fill partial sums [F <= 8][ng] (field type)
  void* apart = nullptr;       // adjoint start values [F <= 8][ng] (field type)
  int* acq = nullptr;          // adjoint incidence records: consumer [n_gsrc]
  void* acw = nullptr;         //   and weights [2][n_gsrc] (field type)
  // fluid targets of the adjoint at reach 1, per (ghost, member) incidence:
  // source count when it owns its target, target cell, sources [cap]
  int *af_cnt = nullptr, *af_cell = nullptr, *af_src = nullptr;
  int af_cap = 0;

  std::vector<int> order_by_size;            // geometries, largest ghost count first
  int tb[TU_N] = {TUNE_DEFAULT, TUNE_DEFAULT, TUNE_DEFAULT, TUNE_DEFAULT, TUNE_DEFAULT, TUNE_DEFAULT,
                  TUNE_DEFAULT, TUNE_DEFAULT, TUNE_DEFAULT, TUNE_DEFAULT, TUNE_DEFAULT,
                  TUNE_DEFAULT};   // threads per block
  PackedPlan pplan;                          // schedule of the packed kernels
  void* lamP = nullptr;                      // packed adjoint scratch [ng][F]
  size_t lamP_bytes = 0;
  std::map<long long, ChainPlan> chain_plans;

  // tile schedule of the tiled fill (ebr_tiled_plan); its device buffers are
  // its own (freed by the next tiled plan, ebr_plan or ebr_destroy)
  struct Tiled {
    bool built = false;
    int tile[3] = {0, 0, 0};
    TiledPlanDev dev;
    int grid[2] = {0, 0};
    void* xbuf = nullptr;
    unsigned* bar = nullptr;
    std::vector<void*> mem;
    std::vector<int> h_tile_global;       // per ghost (canonical): geometry tile offset + tile id
    std::vector<int> h_slot;              // per ghost: exchange slot or -1
    std::vector<long long> sent_per_level;
    long long total_tiles = 0, pairs = 0, halo = 0;
    int extra_once = 0, spin_once = 0;    // bounded-wait test of the next launch
  } tiled;

  // optional per-kernel timing: events recorded on the launching stream
  struct ProfRec {
    const char* name;
    cudaEvent_t a, b;
  };
  bool prof = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;

  // second stream for independent branches inside one call (fork / join by
  // events, so that a stream capture records them as parallel graph branches)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_lam = nullptr, ev_bc = nullptr;   // adjoint: lambda final / BC gradients done
  // the closest points of a split re-run (ebr_classify_levels), still
  // running on the side stream until the reorder waits for them
  cudaEvent_t ev_geom = nullptr;
  bool geom_pending = false;
};

cudaEvent_t take_event(Ctx* c) {
  if (c->pool_used == c->pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->pool.push_back(e);
  }
  return c->pool[c->pool_used++];
}

// Inside a stream capture the events become event-record nodes of the graph
// (re-recorded at every replay), so a captured step can be timed per kernel
// without the host launch gaps of an eager step.
void prof_record(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &st);
  if (st == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else cudaEventRecord(e, s);
}

void prof_begin(Ctx* c, cudaStream_t s, const char* name) {
  if (!c->prof) return;
  Ctx::ProfRec r{name, take_event(c), nullptr};
  if (r.a) prof_record(r.a, s);
  c->recs.push_back(r);
}

void prof_end(Ctx* c, cudaStream_t s) {
  if (!c->prof || c->recs.empty()) return;
  c->recs.back().b = take_event(c);
  if (c->recs.back().b) prof_record(c->recs.back().b, s);
}

ebr_status fail(Ctx* c, ebr_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(c, EBR_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),       \
                  __FILE__, __LINE__);                                                        \
  } while (0)

#define CKL()                                                                                 \
  do {                                                                                        \
    cudaError_t e_ = cudaGetLastError();                                                      \
    if (e_ != cudaSuccess)                                                                    \
      return fail(c, EBR_ECUDA, "kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_),   \
                  __FILE__, __LINE__);                                                        \
  } while (0)

// Device allocations.  A buffer held by a pointer member of the context is a
// grow-only slot: a later plan of the same context (ebr_move, the next plan
// of a moving body) reuses it when it is large enough and otherwise replaces
// it with one 25 % larger than asked, so that the counts of a body that
// moves a little settle into the capacity after a few steps.  Buffers of the
// derived plans (chain, field-minor, temporaries) are listed in c->bufs and
// released with them.
ebr_status slot_alloc(Ctx* c, Ctx::Slot& sl, void** p, size_t bytes) {
  bytes = std::max<size_t>(bytes, 16);
  if (sl.p && sl.cap >= bytes) { *p = sl.p; return EBR_OK; }
  const size_t want = sl.p ? bytes + bytes / 4 : bytes;
  if (sl.p) { cudaFree(sl.p); sl.p = nullptr; sl.cap = 0; }
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, EBR_ENOMEM, "cudaMalloc of %zu bytes failed: %s", want, cudaGetErrorString(e));
  }
  sl.p = q;
  sl.cap = want;
  ++c->n_alloc;
  *p = q;
  return EBR_OK;
}

ebr_status balloc(Ctx* c, void** p, size_t bytes) {
  bytes = std::max<size_t>(bytes, 16);
  const char* a = reinterpret_cast<const char*>(p);
  const bool member = a >= reinterpret_cast<const char*>(c) && a < reinterpret_cast<const char*>(c + 1);
  if (member) return slot_alloc(c, c->slots[p], p, bytes);
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, EBR_ENOMEM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  c->bufs.push_back({q, bytes});
  ++c->n_alloc;
  *p = q;
  return EBR_OK;
}

template <typename T>
ebr_status dalloc(Ctx* c, T** p, size_t count) {
  return balloc(c, reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T));
}

#define AL(ptr, count)                                           \
  do {                                                           \
    ebr_status s_ = dalloc(c, &(ptr), (size_t)(count));          \
    if (s_ != EBR_OK) return s_;                                 \
  } while (0)

void tiled_free(Ctx* c) {
  for (void* q : c->tiled.mem) cudaFree(q);
  c->tiled = Ctx::Tiled();
}

// the plans derived from the levels (chain, field-minor, tiled) and their buffers
void release_derived(Ctx* c) {
  tiled_free(c);
  for (auto& b : c->bufs) cudaFree(b.p);
  c->bufs.clear();
  c->lamP = nullptr;
  c->lamP_bytes = 0;
  c->pplan = PackedPlan();
  c->chain_plans.clear();
}

void free_all(Ctx* c) {
  release_derived(c);
  for (auto& e : c->pool) cudaEventDestroy(e);
  c->pool.clear();
  c->pool_used = 0;
  c->recs.clear();
  for (auto& kv : c->slots)
    if (kv.second.p) cudaFree(kv.second.p);
  c->slots.clear();
  for (auto& kv : c->chain_slots)
    if (kv.second.p) cudaFree(kv.second.p);
  c->chain_slots.clear();
}

cudaStream_t S(ebr_stream s) { return reinterpret_cast<cudaStream_t>(s); }

ebr_status ensure_side(Ctx* c) {
  if (c->side) return EBR_OK;
  CK(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&c->ev_lam, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&c->ev_bc, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&c->ev_geom, cudaEventDisableTiming));
  return EBR_OK;
}

void destroy_side(Ctx* c) {
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_lam) cudaEventDestroy(c->ev_lam);
  if (c->ev_bc) cudaEventDestroy(c->ev_bc);
  if (c->ev_geom) cudaEventDestroy(c->ev_geom);
  if (c->side) cudaStreamDestroy(c->side);
  c->side = nullptr;
  c->ev_fork = c->ev_join = c->ev_lam = c->ev_bc = c->ev_geom = nullptr;
  c->geom_pending = false;
}

int max_smem_optin() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}


ebr_status upload_geoms(Ctx* c) {
  CK(cudaMemcpy(c->dG, c->hG.data(), sizeof(Geom) * c->B, cudaMemcpyHostToDevice));
  return EBR_OK;
}

// the coefficient tables in a field type (FP32: the float copies)
const void* wtab_of(const Ctx* c, int dtype) {
  return dtype == EBR_F32 ? static_cast<const void*>(c->wtab_f) : static_cast<const void*>(c->wtab);
}
const void* ftab_of(const Ctx* c, int dtype) {
  return dtype == EBR_F32 ? static_cast<const void*>(c->ftab_f) : static_cast<const void*>(c->ftab);
}

// the single-pass scan states of the re-run kernels (sizes of the plan)
constexpr int LB_SPIN_LIMIT = 1 << 20;

ebr_status lookback_alloc(Ctx* c, cudaStream_t s) {
  const size_t t[3] = {(size_t)(c->total_rows + LB_T - 1) / LB_T, (size_t)(c->n_iface + LB_T - 1) / LB_T,
                       (size_t)(c->ng + LB_T - 1) / LB_T};
  // 16 counter words (three used per state), then the tile words (8 bytes)
  const size_t words = 16 + 2 * (t[0] + t[1] + t[2]);
  AL(c->lb_mem, words);
  CK(cudaMemsetAsync(c->lb_mem, 0, words * sizeof(unsigned), s));
  unsigned long long* tiles = reinterpret_cast<unsigned long long*>(c->lb_mem + 16);
  Lookback* L[3] = {&c->lb_rows, &c->lb_iface, &c->lb_gsrc};
  for (int i = 0; i < 3; ++i) {
    L[i]->ctr = c->lb_mem + 4 * i;
    L[i]->tiles = tiles;
    L[i]->spin_limit = LB_SPIN_LIMIT;
    tiles += t[i];
  }
  return EBR_OK;
}

// ---------------------------------------------------------------------------
// classification pipeline (planning == true: synchronise and size buffers)
// ---------------------------------------------------------------------------
// split (re-run of one-layer HGC only): the placement records the signs and
// zeros of the candidates' normals, the compaction completes the meta words
// from them, and the double closest points run on the side stream beside the
// positions, dependencies and levels; run_levels joins them before the
// reorder.
ebr_status run_classify(Ctx* c, int8_t* d_tags, cudaStream_t s, bool planning, bool split) {
  c->tags = d_tags;
  prof_begin(c, s, "rows");
  launch_rows(c->dG, c->d_row_off, c->B, c->total_rows, c->runs, d_tags, c->d_status, c->d_stats, s);
  prof_end(c, s);
  c->launches += 1;
  CKL();
  if (planning) {
    // counts, their scan, the sizes on the host, then the interface cells
    prof_begin(c, s, "iface");
    launch_iface(c->dG, c->d_row_off, c->B, c->total_rows, c->runs, c->row_cnt, nullptr, nullptr,
                 nullptr, nullptr, 0, 0, c->d_status, s, c->tb[TU_IFACE]);
    prof_end(c, s);
    prof_begin(c, s, "scan");
    launch_scan(c->row_cnt, c->row_ptr, c->total_rows, c->scan_tmp, s);
    prof_end(c, s);
    c->launches += 3;
    CKL();
    std::vector<int> hp(c->total_rows + 1);
    CK(cudaMemcpyAsync(hp.data(), c->row_ptr, sizeof(int) * (c->total_rows + 1), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    c->n_iface = hp[c->total_rows];
    for (int b = 0; b < c->B; ++b) {
      c->hG[b].iface_off = hp[c->hG[b].row_off];
      c->hG[b].n_iface = hp[c->hG[b].row_off + c->hG[b].n_rows] - c->hG[b].iface_off;
    }
    int ni = c->n_iface;
    AL(c->iface_cell, ni);
    AL(c->iface_geo, ni);
    AL(c->iface_solid, ni);
    AL(c->iface_meta, ni);
    AL(c->iface_tag, ni);
    AL(c->gflag, ni);
    AL(c->gpos, ni + 1);
    prof_begin(c, s, "iface");
    launch_iface(c->dG, c->d_row_off, c->B, c->total_rows, c->runs, nullptr, c->row_ptr,
                 c->iface_cell, c->iface_geo, c->iface_solid, 1, c->n_iface, c->d_status, s, c->tb[TU_IFACE]);
    prof_end(c, s);
    c->launches += 1;
  } else {
    // a re-run with the plan's sizes: counts, offsets and cells in one launch
    prof_begin(c, s, "iface");
    launch_iface_fused(c->dG, c->d_row_off, c->B, c->total_rows, c->runs, c->row_ptr, c->iface_cell,
                       c->iface_geo, c->iface_solid, c->n_iface, c->lb_rows, c->d_status, s);
    prof_end(c, s);
    c->launches += 1;
  }
  // a re-run of one-layer HGC takes pass B of the reclassification into the
  // compaction launch
  const bool fuse_b = !planning && c->placement == EBR_HGC && c->layers == 1;
  split = split && fuse_b;
  prof_begin(c, s, "place");
  launch_place(c->dG, c->n_iface, c->iface_cell, c->iface_geo, c->iface_solid, c->placement,
               d_tags, split ? c->iface_meta : nullptr, c->d_status, s, c->tb[TU_PLACE]);
  prof_end(c, s);
  c->launches += 1;
  c->tags_pending = false;
  if (c->placement == EBR_HGC) {
    // the fused re-run decides both passes in the compaction (split below)
    if (!split) {
      prof_begin(c, s, "reclassify");
      launch_reclassify(c->dG, c->n_iface, c->iface_cell, c->iface_geo, d_tags, 0, s);
      prof_end(c, s);
      c->launches += 1;
    }
    if (!fuse_b) {
      prof_begin(c, s, "reclassify");
      launch_reclassify(c->dG, c->n_iface, c->iface_cell, c->iface_geo, d_tags, 1, s);
      prof_end(c, s);
      c->launches += 1;
    }
  }
  if (c->layers == 2) {
    prof_begin(c, s, "layer2");
    launch_layer2(c->dG, c->n_iface, c->iface_cell, c->iface_geo, d_tags, c->d_status, s);
    prof_end(c, s);
    c->launches += 1;
  }
  if (!planning) {
    prof_begin(c, s, "ghost_compact");
    launch_ghost_compact(c->dG, c->n_iface, c->iface_cell, c->iface_geo, d_tags, split ? 2 : (fuse_b ? 1 : 0),
                         split ? c->iface_meta : nullptr, c->iface_tag, c->gpos, c->ng, c->gs_cell, c->gs_geo,
                         c->gs_meta, c->lb_iface, c->d_status, s);
    prof_end(c, s);
    // the final tags of the interface cells reach the tag array with the
    // positions (the next launch of run_levels)
    c->tags_pending = split;
    // the offsets against the plan: block 0 of the closest-point kernel
    cudaStream_t sg = s;
    if (split) {
      ebr_status st = ensure_side(c);
      if (st) return st;
      CK(cudaEventRecord(c->ev_fork, s));
      CK(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
      sg = c->side;
    }
    prof_begin(c, sg, "ghost_geom");
    launch_ghost_geom(c->dG, c->placement, c->ng, c->gs_cell, c->gs_geo, c->gs_psi, c->gs_n, c->gs_meta,
                      split ? 1 : 0, c->d_stats + 1, c->d_status, sg, c->tb[TU_GHOST],
                      PlanCheck{c->row_ptr, c->gpos, c->d_nlev, c->B, c->n_iface, c->ng, 0});
    prof_end(c, sg);
    if (split) {
      CK(cudaEventRecord(c->ev_geom, c->side));
      c->geom_pending = true;
    }
    c->launches += 2;
    CKL();
    return EBR_OK;
  }
  prof_begin(c, s, "ghost_flags");
  launch_ghost_flags(c->dG, c->n_iface, c->iface_cell, c->iface_geo, d_tags, c->gflag, s);
  prof_end(c, s);
  prof_begin(c, s, "scan");
  launch_scan(c->gflag, c->gpos, c->n_iface, c->scan_tmp, s);
  prof_end(c, s);
  c->launches += 3;
  CKL();
  {
    std::vector<int> hp(c->n_iface + 1);
    CK(cudaMemcpyAsync(hp.data(), c->gpos, sizeof(int) * (c->n_iface + 1), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    c->ng = hp[c->n_iface];
    for (int b = 0; b < c->B; ++b) {
      Geom& g = c->hG[b];
      g.ghost_off = hp[g.iface_off];
      g.n_ghost = hp[g.iface_off + g.n_iface] - g.ghost_off;
      g.lev_off = g.ghost_off + b;
    }
    int ng = c->ng;
    AL(c->gs_cell, ng);
    AL(c->gs_geo, ng);
    AL(c->gs_psi, ng);
    AL(c->gs_n, 3 * (size_t)ng);
    AL(c->gs_meta, ng);
    CK(cudaMemsetAsync(c->d_stats + 1, 0, sizeof(int), s));
  }
  prof_begin(c, s, "ghost_write");
  launch_ghost_write(c->dG, c->n_iface, c->iface_cell, c->iface_geo, d_tags, c->gpos, c->placement,
                     c->ng, c->gs_cell, c->gs_geo, c->gs_psi,
                     c->gs_n, c->gs_meta, c->d_stats + 1, c->d_status, s, c->tb[TU_GHOST]);
  prof_end(c, s);
  c->launches += 2;
  CKL();
  CK(cudaMemcpyAsync(&c->rmax, c->d_stats + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (c->rmax < 1) c->rmax = 1;
  ebr_status st = upload_geoms(c);
  if (st) return st;
  return lookback_alloc(c, s);
}

// ---------------------------------------------------------------------------
// levels pipeline
// ---------------------------------------------------------------------------
ebr_status run_levels(Ctx* c, cudaStream_t s, bool planning) {
  int ng = c->ng;
  if (planning) {
    AL(c->dep, 8 * (size_t)ng);
    AL(c->level, ng);
    AL(c->order_pos, ng);
    AL(c->g_cell, ng);
    AL(c->g_geo, ng);
    AL(c->g_dep, 8 * (size_t)ng);
    AL(c->g_level, ng);
    AL(c->g_psi, ng);
    AL(c->g_n, 3 * (size_t)ng);
    AL(c->g_meta, ng);
    AL(c->lev_ptr, ng + c->B + 1);
    {
      // the level kernel also holds ~9 KB of static shared memory
      size_t cap = (size_t)max_smem_optin() - 12 * 1024, need = 0;
      for (int b = 0; b < c->B; ++b) {
        size_t q = levels_smem(c->hG[b].dim, c->hG[b].n_ghost);
        if (q <= cap) need = std::max(need, q);
      }
      c->levels_smem = need;
    }
    AL(c->wtab, 16 * (size_t)ng);
    AL(c->ftab, 33 * (size_t)ng);
    AL(c->wtab_f, 16 * (size_t)ng);
    AL(c->ftab_f, 33 * (size_t)ng);
    AL(c->gsrc_cnt, ng);
    AL(c->gsrc_ptr, ng + 1);
    AL(c->gsrc_mem, (size_t)stencil_k(c->hG[0].dim) * ng);
    AL(c->sv, 64 * (size_t)ng);
    {
      ebr_status st = balloc(c, &c->lam, 8 * 8 * (size_t)ng);   // [F <= 8][ng] doubles
      if (st) return st;
      st = balloc(c, &c->fpart, 8 * 8 * (size_t)ng);
      if (st) return st;
      st = balloc(c, &c->apart, 8 * 8 * (size_t)ng);
      if (st) return st;
    }
    {
      const int kmax = stencil_k(c->hG[0].dim);
      c->af_cap = adj_fluid_cap(c->hG[0].dim);
      AL(c->af_cnt, (size_t)ng * kmax);
      AL(c->af_cell, (size_t)ng * kmax);
      AL(c->af_src, (size_t)ng * kmax * c->af_cap);
    }
  }
  prof_begin(c, s, "poscell");
  launch_poscell(c->dG, ng, c->gs_cell, c->gs_geo, nullptr, c->pos_of_cell, c->gsrc_cnt, s, c->n_iface,
                 c->iface_cell, c->iface_geo, c->tags_pending ? c->iface_tag : nullptr, c->tags);
  c->tags_pending = false;
  prof_end(c, s);
  prof_begin(c, s, "deps");
  launch_deps(c->dG, ng, c->gs_cell, c->gs_geo, c->gs_meta, c->tags, c->pos_of_cell,
              c->dep, c->d_status, s, c->tb[TU_DEPS]);
  prof_end(c, s);
  prof_begin(c, s, "levels");
  launch_levels(c->dG, c->B, c->dep, ng, c->level, c->order_pos, c->lev_ptr, c->d_nlev,
                c->levels_smem, c->d_status, s);
  prof_end(c, s);
  c->launches += 3;
  CKL();
  if (planning) {
    std::vector<int> nl(c->B);
    CK(cudaMemcpyAsync(nl.data(), c->d_nlev, sizeof(int) * c->B, cudaMemcpyDeviceToHost, s));
    int hs = 0;
    CK(cudaMemcpyAsync(&hs, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hs != 0) return fail(c, (ebr_status)hs, "device status %d while building levels", hs);
    for (int b = 0; b < c->B; ++b) c->hG[b].n_levels = nl[b];
    c->h_lev_ptr.assign(ng + c->B + 1, 0);
    CK(cudaMemcpy(c->h_lev_ptr.data(), c->lev_ptr, sizeof(int) * (ng + c->B + 1), cudaMemcpyDeviceToHost));
    ebr_status st = upload_geoms(c);
    if (st) return st;
  }
  // the closest points of a split re-run join here: the reorder moves them
  if (c->geom_pending) {
    CK(cudaStreamWaitEvent(s, c->ev_geom, 0));
    c->geom_pending = false;
  }
  prof_begin(c, s, "reorder");
  // a re-run checks the level counts against the plan in block 0 of the reorder
  launch_reorder(c->dG, c->pos_of_cell, ng, c->order_pos, c->gs_cell, c->gs_geo, c->gs_psi, c->gs_n,
                 c->gs_meta, c->dep, c->level, c->g_cell, c->g_geo, c->g_psi, c->g_n, c->g_meta, c->g_dep,
                 c->g_level, s, PlanCheck{c->row_ptr, c->gpos, c->d_nlev, c->B, c->n_iface, c->ng, planning ? -1 : 1},
                 c->d_status);
  prof_end(c, s);
  // The coefficient tables and the ghost-target source lists (adjoint only)
  // are independent: outside planning the source lists run on the second
  // stream, joined before the call returns.
  cudaStream_t sg = s;
  if (!planning) {
    ebr_status st = ensure_side(c);
    if (st) return st;
    CK(cudaEventRecord(c->ev_fork, s));
    CK(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    sg = c->side;
  }
  prof_begin(c, s, "tables");
  launch_tables(c->dG, ng, c->g_cell, c->g_geo, c->g_psi, c->g_n, c->g_meta, c->tags, c->wtab,
                c->ftab, c->wtab_f, c->ftab_f, s, c->tb[TU_TABLES]);
  prof_end(c, s);
  c->launches += 2;   // reorder, tables
  // ghost-target sources by transposition: member positions and counts; when
  // planning the scan, the sizes on the host and the lists; in a re-run the
  // offsets in one single-pass launch, then the lists
  const int kmax = stencil_k(c->hG[0].dim);
  prof_begin(c, sg, "gsrc");
  launch_gsrc_count(c->dG, ng, c->g_cell, c->g_geo, c->g_meta, c->g_dep, c->tags, c->pos_of_cell, kmax,
                    c->gsrc_mem, c->gsrc_cnt, sg, c->tb[TU_GSRC]);
  if (planning) {
    launch_scan(c->gsrc_cnt, c->gsrc_ptr, ng, c->scan_tmp, sg);
    c->launches += 3;
    CKL();
    CK(cudaMemcpyAsync(&c->n_gsrc, c->gsrc_ptr + ng, sizeof(int), cudaMemcpyDeviceToHost, s));
    std::vector<int> hp(ng + 1);
    CK(cudaMemcpyAsync(hp.data(), c->gsrc_ptr, sizeof(int) * (ng + 1), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    c->h_gsrc_geo.assign(c->B, 0);
    for (int b = 0; b < c->B; ++b) {
      const Geom& g = c->hG[b];
      c->h_gsrc_geo[b] = hp[g.ghost_off + g.n_ghost] - hp[g.ghost_off];
    }
    AL(c->gsrc, c->n_gsrc);
    AL(c->acq, c->n_gsrc);
    ebr_status st = balloc(c, &c->acw, 2 * 8 * std::max<size_t>((size_t)c->n_gsrc, 1));
    if (st) return st;
    launch_gsrc_lists(ng, kmax, c->gsrc_mem, c->gsrc_ptr, c->gsrc_cnt, c->gsrc, c->n_gsrc, c->d_status, true, sg,
                      c->tb[TU_GSRC]);
    c->launches += 3;
  } else {
    launch_gsrc_place(ng, c->gsrc_cnt, c->gsrc_ptr, c->gsrc, c->n_gsrc, c->lb_gsrc, c->d_status, sg);
    launch_gsrc_lists(ng, kmax, c->gsrc_mem, c->gsrc_ptr, c->gsrc_cnt, c->gsrc, c->n_gsrc, c->d_status, false,
                      sg, c->tb[TU_GSRC]);
    c->launches += 4;
  }
  prof_end(c, sg);
  if (!planning) {
    CK(cudaEventRecord(c->ev_join, c->side));
    CK(cudaStreamWaitEvent(s, c->ev_join, 0));
  }
  CKL();
  if (planning) {
    // force chunks (<= 256 ghosts, never straddling geometries)
    std::vector<int4> ch;
    std::vector<int> cp(c->B + 1, 0);
    for (int b = 0; b < c->B; ++b) {
      const Geom& g = c->hG[b];
      cp[b] = (int)ch.size();
      for (int p = g.ghost_off; p < g.ghost_off + g.n_ghost; p += 256)
        ch.push_back(make_int4(b, p, std::min(p + 256, g.ghost_off + g.n_ghost), 0));
    }
    cp[c->B] = (int)ch.size();
    c->n_chunks = (int)ch.size();
    AL(c->chunks, c->n_chunks);
    AL(c->chunk_ptr, c->B + 1);
    AL(c->chunk_done, c->B);
    CK(cudaMemset(c->chunk_done, 0, sizeof(int) * c->B));
    AL(c->partial, 8 * (size_t)std::max(c->n_chunks, 1));
    CK(cudaMemcpy(c->chunks, ch.data(), sizeof(int4) * ch.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->chunk_ptr, cp.data(), sizeof(int) * cp.size(), cudaMemcpyHostToDevice));
    c->order_by_size.resize(c->B);
    for (int b = 0; b < c->B; ++b) c->order_by_size[b] = b;
    std::stable_sort(c->order_by_size.begin(), c->order_by_size.end(),
                     [&](int a, int b) { return c->hG[a].n_ghost > c->hG[b].n_ghost; });
  }
  return EBR_OK;
}


// Body of geometry b (kind, centre, radii or semi-axes, rotation, airfoil
// parameters) and the float copies and margins derived from it; the grid
// fields of g (dim, n, lo, h) are set already.
ebr_status set_body(Ctx* c, Geom& g, const ebr_body& bd, int b) {
  if (bd.kind < 0 || bd.kind > 3) return fail(c, EBR_EINVAL, "geometry %d: bad body kind", b);
  const int want_dim = bd.kind == EBR_SPHERE ? 3 : 2;
  if (want_dim != g.dim) return fail(c, EBR_EINVAL, "geometry %d: body kind needs dim %d", b, want_dim);
  if ((bd.kind == EBR_CIRCLE || bd.kind == EBR_SPHERE) && !(bd.radii[0] > 0))
    return fail(c, EBR_EINVAL, "geometry %d: radius must be positive", b);
  if (bd.kind == EBR_ELLIPSE && !(bd.radii[0] > 0 && bd.radii[1] > 0))
    return fail(c, EBR_EINVAL, "geometry %d: semi-axes must be positive", b);
  if (bd.kind == EBR_AIRFOIL4 && !(bd.thickness > 0 && bd.chord > 0 && bd.rot[0] > 0))
    return fail(c, EBR_EINVAL, "geometry %d: airfoil needs t > 0, chord > 0, |angle| < 90 deg", b);
  g.kind = bd.kind;
  for (int a = 0; a < 3; ++a) { g.centre[a] = bd.centre[a]; g.radii[a] = bd.radii[a]; }
  for (int q = 0; q < 9; ++q) g.rot[q] = bd.rot[q];
  g.t = bd.thickness;
  g.c = bd.chord;
  // float copies and the margin of the float HGC decision: it covers the
  // float rounding of cell centres, body-frame coordinates, the float
  // closest point and dn/2 by a wide factor (1e-4 of the finest width plus
  // 4e-6 of the largest coordinate magnitude)
  // (on a stretched grid h holds the smallest widths; the far end of axis a
  // is then the last face, kept in far[a])
  float hmin = 3.4e38f, ext = 1.0f;
  double far[3];
  for (int a = 0; a < 3; ++a)
    far[a] = g.stretched && a < g.dim ? g.lo[a] + g.span[a] : g.lo[a] + g.n[a] * g.h[a];
  for (int a = 0; a < 3; ++a) {
    g.flo[a] = (float)g.lo[a];
    g.fh[a] = (float)g.h[a];
    g.fcentre[a] = (float)g.centre[a];
    g.fradii[a] = (float)g.radii[a];
    if (a < g.dim) {
      hmin = std::min(hmin, (float)g.h[a]);
      ext = std::max(ext, std::max(std::fabs((float)g.lo[a]), std::fabs((float)far[a])));
    }
  }
  for (int q = 0; q < 9; ++q) g.frot[q] = (float)g.rot[q];
  g.ft = (float)g.t;
  g.fc = (float)g.c;
  g.hgc_mrg = 1e-4f * hmin + 4e-6f * ext;
  float extc = 1.0f;
  for (int a = 0; a < g.dim; ++a)
    extc = std::max(extc, std::max(std::fabs((float)(g.lo[a] - g.centre[a])),
                                   std::fabs((float)(far[a] - g.centre[a]))));
  g.fext = extc;
  return EBR_OK;
}

// Chain plan for (kind of pass, dtype, F): geometries whose state fits in one
// CTA's shared memory, largest first; the rest use level launches.
ebr_status chain_plan(Ctx* c, int which, int dtype, int F, ChainPlan** out) {
  long long key = (long long)which * 1000 + dtype * 100 + F;
  auto it = c->chain_plans.find(key);
  if (it != c->chain_plans.end()) { *out = &it->second; return EBR_OK; }
  ChainPlan cp;
  size_t limit = (size_t)max_smem_optin();
  std::vector<int> list;
  for (int b : c->order_by_size) {
    const Geom& g = c->hG[b];
    if (g.n_ghost == 0) continue;
    size_t need = which == 0 ? fill_chain_smem(dtype, g.dim, F, g.n_ghost)
                             : adj_chain_smem(dtype, F, g.n_ghost, c->h_gsrc_geo[b]);
    if (need <= limit) {
      list.push_back(b);
      cp.smem = std::max(cp.smem, need);
    } else {
      cp.fallback.push_back(b);
    }
  }
  cp.n_list = (int)list.size();
  {
    ebr_status st = slot_alloc(c, c->chain_slots[key], reinterpret_cast<void**>(&cp.d_list),
                               sizeof(int) * std::max<size_t>(list.size(), 1));
    if (st) return st;
  }
  if (!list.empty())
    CK(cudaMemcpy(cp.d_list, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice));
  c->chain_plans[key] = cp;
  *out = &c->chain_plans[key];
  return EBR_OK;
}

}  // namespace

extern "C" {

ebr_status ebr_create(void** out) {
  if (!out) return EBR_EINVAL;
  Ctx* c = new Ctx();
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) {
    delete c;
    *out = nullptr;
    return EBR_ECUDA;
  }
  *out = c;
  return EBR_OK;
}

void ebr_destroy(void* ctx) {
  if (!ctx) return;
  Ctx* c = static_cast<Ctx*>(ctx);
  free_all(c);
  destroy_side(c);
  delete c;
}

const char* ebr_last_error(const void* ctx) {
  if (!ctx) return "null context";
  return static_cast<const Ctx*>(ctx)->err.c_str();
}

int64_t ebr_launch_count(const void* ctx) {
  return ctx ? static_cast<const Ctx*>(ctx)->launches : 0;
}

void ebr_set_pdl(int32_t enable) { ebr::g_pdl = enable != 0; }

int32_t ebr_get_pdl(void) { return ebr::g_pdl; }

}  // extern "C"

namespace {

// ebr_plan and ebr_plan_faces (h_faces null: every grid uniform)
ebr_status plan_impl(Ctx* c, int32_t n_geom, const ebr_grid* h_grids, const double* const* h_faces,
                     const ebr_body* h_bodies, int32_t placement, int8_t* d_tags, ebr_stream stream) {
  c->err.clear();
  if (n_geom < 1 || !h_grids || !h_bodies || !d_tags)
    return fail(c, EBR_EINVAL, "ebr_plan: n_geom >= 1 and non-null grids, bodies, tags required");
  const int layers = (placement & EBR_SECOND_LAYER) ? 2 : 1;
  placement &= ~EBR_SECOND_LAYER;
  if (placement < 0 || placement > 2) return fail(c, EBR_EINVAL, "ebr_plan: bad placement %d", placement);
  if (layers == 2 && placement == EBR_CGC)
    return fail(c, EBR_EINVAL, "ebr_plan: the second ghost layer goes with EBR_HGC or EBR_CGC_ES");
  free_all(c);
  c->B = n_geom;
  c->placement = placement;
  c->layers = layers;
  c->planned = c->levelled = false;
  c->hG.assign(n_geom, Geom{});
  c->h_row_off.assign(n_geom + 1, 0);
  c->h_cen.assign(n_geom, {});
  long long cells = 0, n_coord = 0;
  int rows = 0;
  std::vector<std::array<std::vector<double>, 3>> h_wid(n_geom);
  for (int b = 0; b < n_geom; ++b) {
    const ebr_grid& gr = h_grids[b];
    const ebr_body& bd = h_bodies[b];
    Geom& g = c->hG[b];
    if (gr.dim != 2 && gr.dim != 3) return fail(c, EBR_EINVAL, "geometry %d: dim must be 2 or 3", b);
    g.dim = gr.dim;
    const double* faces = h_faces ? h_faces[b] : nullptr;
    g.stretched = faces != nullptr;
    long long n3 = 1;
    const double* fa = faces;
    for (int a = 0; a < 3; ++a) {
      long long na = a < gr.dim ? gr.n[a] : 1;
      if (na < 2 && a < gr.dim) return fail(c, EBR_EINVAL, "geometry %d: n[%d] < 2", b, a);
      g.n[a] = (int)na;
      if (a < gr.dim && faces) {
        // faces of axis a: na + 1 strictly increasing values
        std::vector<double>& cen = c->h_cen[b][a];
        std::vector<double>& wid = h_wid[b][a];
        cen.resize(na);
        wid.resize(na);
        double wmin = 1e300;
        for (long long i = 0; i < na; ++i) {
          if (!(fa[i + 1] > fa[i])) return fail(c, EBR_EINVAL, "geometry %d: faces of axis %d not increasing", b, a);
          cen[i] = 0.5 * (fa[i] + fa[i + 1]);
          wid[i] = fa[i + 1] - fa[i];
          wmin = std::min(wmin, wid[i]);
        }
        g.lo[a] = fa[0];
        g.h[a] = wmin;
        g.span[a] = fa[na] - fa[0];
        fa += na + 1;
        n_coord += na;
      } else {
        if (a < gr.dim && !(gr.hi[a] > gr.lo[a])) return fail(c, EBR_EINVAL, "geometry %d: hi <= lo", b);
        g.lo[a] = a < gr.dim ? gr.lo[a] : 0.0;
        g.h[a] = a < gr.dim ? (gr.hi[a] - gr.lo[a]) / (double)na : 1.0;
        g.span[a] = a < gr.dim ? gr.hi[a] - gr.lo[a] : 1.0;
      }
      n3 *= na;
    }
    if (n3 > (1LL << 31) - 1) return fail(c, EBR_EINVAL, "geometry %d: more than 2^31-1 cells", b);
    g.placement = placement;
    // largest width of each axis (the spacing of a uniform grid)
    double hx[3] = {1.0, 1.0, 1.0};
    g.hmax = 0.0;
    for (int a = 0; a < gr.dim; ++a) {
      hx[a] = g.stretched ? *std::max_element(h_wid[b][a].begin(), h_wid[b][a].end()) : g.h[a];
      g.hmax = std::max(g.hmax, hx[a]);
    }
    // second layer: box reach per axis that holds a fluid cell for every
    // solid cell with psi <= 1.5 dn: ceil((1.5 max h + |h| / 2) / h_a + 1/2);
    // stretched: the largest widths in the distances, the axis' smallest
    // width as the unit, the containing cell's half width included
    g.layers = layers;
    {
      double hm = 0.0, D2 = 0.0;
      for (int a = 0; a < gr.dim; ++a) {
        const double ha = g.stretched ? hx[a] : (gr.hi[a] - gr.lo[a]) / (double)gr.n[a];
        hm = std::max(hm, ha);
        D2 += ha * ha;
      }
      for (int a = 0; a < 3; ++a) {
        if (a >= gr.dim) { g.reach[a] = 0; continue; }
        if (g.stretched) {
          g.reach[a] = (int)std::ceil((1.5 * hm + 0.5 * std::sqrt(D2) + 0.5 * hx[a]) / g.h[a]);
        } else {
          const double ha = (gr.hi[a] - gr.lo[a]) / (double)gr.n[a];
          g.reach[a] = (int)std::ceil((1.5 * hm + 0.5 * std::sqrt(D2)) / ha + 0.5);
        }
      }
    }
    {
      ebr_status st = set_body(c, g, bd, b);
      if (st) return st;
    }
    g.cell_off = cells;
    g.row_off = rows;
    g.n_rows = g.n[1] * g.n[2];
    c->h_row_off[b] = rows;
    cells += n3;
    rows += g.n_rows;
  }
  c->h_row_off[n_geom] = rows;
  c->total_cells = cells;
  c->total_rows = rows;
  if (n_coord > 0) {
    // device centres, widths and float centres of the stretched grids
    AL(c->coord_d, 2 * (size_t)n_coord);
    AL(c->coord_f, (size_t)n_coord);
    std::vector<double> hd(2 * (size_t)n_coord);
    std::vector<float> hf((size_t)n_coord);
    size_t o = 0;
    for (int b = 0; b < n_geom; ++b) {
      Geom& g = c->hG[b];
      if (!g.stretched) continue;
      for (int a = 0; a < g.dim; ++a) {
        const size_t na = (size_t)g.n[a];
        for (size_t i = 0; i < na; ++i) {
          hd[o + i] = c->h_cen[b][a][i];
          hd[(size_t)n_coord + o + i] = h_wid[b][a][i];
          hf[o + i] = (float)c->h_cen[b][a][i];
        }
        g.cen[a] = c->coord_d + o;
        g.wid[a] = c->coord_d + n_coord + o;
        g.fcen[a] = c->coord_f + o;
        o += na;
      }
    }
    CK(cudaMemcpy(c->coord_d, hd.data(), sizeof(double) * hd.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->coord_f, hf.data(), sizeof(float) * hf.size(), cudaMemcpyHostToDevice));
  }
  AL(c->dG, n_geom);
  AL(c->d_row_off, n_geom + 1);
  AL(c->d_status, 1);
  AL(c->d_stats, 4);
  AL(c->d_nlev, n_geom);
  AL(c->runs, rows);
  AL(c->row_cnt, rows);
  AL(c->row_ptr, rows + 1);
  AL(c->pos_of_cell, cells);
  {
    size_t tb = scan_temp_bytes(std::max(rows, 1 << 26));
    ebr_status st = balloc(c, &c->scan_tmp, tb);
    if (st) return st;
  }
  ebr_status st = upload_geoms(c);
  if (st) return st;
  CK(cudaMemcpy(c->d_row_off, c->h_row_off.data(), sizeof(int) * (n_geom + 1), cudaMemcpyHostToDevice));
  CK(cudaMemset(c->d_status, 0, sizeof(int)));
  CK(cudaMemset(c->d_stats, 0, 4 * sizeof(int)));
  cudaStream_t s = S(stream);
  st = run_classify(c, d_tags, s, true, false);
  if (st) return st;
  int hs = 0;
  CK(cudaMemcpyAsync(&hs, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (hs != 0) {
    CK(cudaMemset(c->d_status, 0, sizeof(int)));
    return fail(c, (ebr_status)hs, "device status %d during classification", hs);
  }
  c->planned = true;
  return EBR_OK;
}

}  // namespace

extern "C" {

ebr_status ebr_plan(void* ctx, int32_t n_geom, const ebr_grid* h_grids, const ebr_body* h_bodies,
                    int32_t placement, int8_t* d_tags, ebr_stream stream) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c) return EBR_EINVAL;
  EbrRange range_("ebr_plan");
  return plan_impl(c, n_geom, h_grids, nullptr, h_bodies, placement, d_tags, stream);
}

ebr_status ebr_plan_faces(void* ctx, int32_t n_geom, const ebr_grid* h_grids, const double* const* h_faces,
                          const ebr_body* h_bodies, int32_t placement, int8_t* d_tags, ebr_stream stream) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c) return EBR_EINVAL;
  EbrRange range_("ebr_plan_faces");
  if (!h_faces) return fail(c, EBR_EINVAL, "ebr_plan_faces: null face array");
  return plan_impl(c, n_geom, h_grids, h_faces, h_bodies, placement, d_tags, stream);
}

ebr_status ebr_classify(void* ctx, int8_t* d_tags, ebr_stream stream) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c) return EBR_EINVAL;
  EbrRange range_("ebr_classify");
  c->err.clear();
  if (!c->planned) return fail(c, EBR_EINVAL, "ebr_classify: call ebr_plan first");
  if (!d_tags) return fail(c, EBR_EINVAL, "ebr_classify: null tags");
  return run_classify(c, d_tags, S(stream), false, false);
}

ebr_status ebr_classify_levels(void* ctx, int8_t* d_tags, ebr_stream stream) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c) return EBR_EINVAL;
  EbrRange range_("ebr_classify_levels");
  c->err.clear();
  if (!c->planned || !c->levelled)
    return fail(c, EBR_EINVAL, "ebr_classify_levels: call ebr_plan and ebr_build_levels first");
  if (!d_tags) return fail(c, EBR_EINVAL, "ebr_classify_levels: null tags");
  cudaStream_t s = S(stream);
  ebr_status st = run_classify(c, d_tags, s, false, true);
  if (st == EBR_OK) st = run_levels(c, s, false);
  if (c->geom_pending) {
    cudaStreamWaitEvent(s, c->ev_geom, 0);
    c->geom_pending = false;
  }
  return st;
}

ebr_status ebr_move(void* ctx, const ebr_body* h_bodies, int8_t* d_tags, ebr_stream stream) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c) return EBR_EINVAL;
  EbrRange range_("ebr_move");
  c->err.clear();
  if (c->B == 0 || c->hG.empty()) return fail(c, EBR_EINVAL, "ebr_move: call ebr_plan first");
  if (!h_bodies || !d_tags) return fail(c, EBR_EINVAL, "ebr_move: null bodies or tags");
  cudaStream_t s = S(stream);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone)
    return fail(c, EBR_EINVAL, "ebr_move: re-plans on the host; call it outside stream capture");
  // every body first: on an error nothing changes
  std::vector<Geom> hg = c->hG;
  for (int b = 0; b < c->B; ++b) {
    ebr_status st = set_body(c, hg[b], h_bodies[b], b);
    if (st) return st;
  }
  CK(cudaStreamSynchronize(s));
  if (c->side) CK(cudaStreamSynchronize(c->side));
  release_derived(c);
  c->hG = hg;
  c->planned = c->levelled = false;
  ebr_status st = upload_geoms(c);
  if (st) return st;
  CK(cudaMemsetAsync(c->d_status, 0, sizeof(int), s));
  CK(cudaMemsetAsync(c->d_stats, 0, 4 * sizeof(int), s));
  st = run_classify(c, d_tags, s, true, false);
  if (st) return st;
  int hs = 0;
  CK(cudaMemcpyAsync(&hs, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (hs != 0) {
    CK(cudaMemset(c->d_status, 0, sizeof(int)));
    return fail(c, (ebr_status)hs, "device status %d during classification", hs);
  }
  c->planned = true;
  return EBR_OK;
}

ebr_status ebr_layout(const void* ctx, int64_t* h_cell_offset) {
  const Ctx* c = static_cast<const Ctx*>(ctx);
  if (!c || !h_cell_offset || !c->planned) return EBR_EINVAL;
  for (int b = 0; b < c->B; ++b) h_cell_offset[b] = c->hG[b].cell_off;
  h_cell_offset[c->B] = c->total_cells;
  return EBR_OK;
}

ebr_status ebr_counts(const void* ctx, ebr_geom_counts* h_counts) {
  const Ctx* c = static_cast<const Ctx*>(ctx);
  if (!c || !h_counts || !c->planned) return EBR_EINVAL;
  for (int b = 0; b < c->B; ++b) {
    const Geom& g = c->hG[b];
    h_counts[b].n_cells = (int64_t)g.n[0] * g.n[1] * g.n[2];
    h_counts[b].n_interface = g.n_iface;
    h_counts[b].n_ghosts = g.n_ghost;
    h_counts[b].n_levels = c->levelled ? g.n_levels : 0;
    h_counts[b].reserved = 0;
  }
  return EBR_OK;
}

ebr_status ebr_build_levels(void* ctx, ebr_stream stream) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c) return EBR_EINVAL;
  EbrRange range_("ebr_build_levels");
  c->err.clear();
  if (!c->planned) return fail(c, EBR_EINVAL, "ebr_build_levels: call ebr_plan first");
  bool planning = !c->levelled;
  ebr_status st = run_levels(c, S(stream), planning);
  if (st) return st;
  c->levelled = true;
  return EBR_OK;
}

ebr_status ebr_ghost_info(void* ctx, int32_t* h_geom, int64_t* h_cell, int32_t* h_level,
                          int8_t* h_tag, double* h_psi, double* h_normal, double* h_S,
                          int32_t* h_r, ebr_stream stream) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c) return EBR_EINVAL;
  EbrRange range_("ebr_ghost_info");
  c->err.clear();
  if (!c->levelled) return fail(c, EBR_EINVAL, "ebr_ghost_info: build the levels first");
  cudaStream_t s = S(stream);
  int ng = c->ng;
  std::vector<int> geo(ng), cell(ng), lev(ng);
  std::vector<uint32_t> meta(ng);
  std::vector<double> psi(ng), n(3 * (size_t)ng);
  CK(cudaMemcpyAsync(geo.data(), c->g_geo, sizeof(int) * ng, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(cell.data(), c->g_cell, sizeof(int) * ng, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(lev.data(), c->g_level, sizeof(int) * ng, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(meta.data(), c->g_meta, sizeof(uint32_t) * ng, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(psi.data(), c->g_psi, sizeof(double) * ng, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(n.data(), c->g_n, sizeof(double) * 3 * ng, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int p = 0; p < ng; ++p) {
    const Geom& g = c->hG[geo[p]];
    if (h_geom) h_geom[p] = geo[p];
    if (h_cell) h_cell[p] = cell[p];
    if (h_level) h_level[p] = lev[p];
    if (h_tag) h_tag[p] = meta_fluid(meta[p]) ? -2 : 2;
    if (h_psi) h_psi[p] = psi[p];
    int ijk[3] = {cell[p] % g.n[0], (cell[p] / g.n[0]) % g.n[1], cell[p] / (g.n[0] * g.n[1])};
    for (int a = 0; a < 3; ++a) {
      double na = n[(size_t)a * ng + p];
      if (h_normal) h_normal[3 * (size_t)p + a] = na;
      if (h_S) {
        double x = a >= g.dim ? 0.0
                   : g.stretched ? c->h_cen[geo[p]][a][ijk[a]] : g.lo[a] + ((double)ijk[a] + 0.5) * g.h[a];
        h_S[3 * (size_t)p + a] = a < g.dim ? x + psi[p] * na : 0.0;
      }
      if (h_r) h_r[3 * (size_t)p + a] = a < g.dim ? meta_r(meta[p], a) : 0;
    }
  }
  return EBR_OK;
}

ebr_status ebr_reconstruct(void* ctx, int32_t n_fields, void* const* d_fields,
                           const int32_t* h_bc_kind, const void* const* d_bc, int32_t dtype,
                           int32_t mode, ebr_stream stream) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c) return EBR_EINVAL;
  EbrRange range_("ebr_reconstruct");
  c->err.clear();
  if (!c->levelled) return fail(c, EBR_EINVAL, "ebr_reconstruct: build the levels first");
  if (n_fields < 1 || n_fields > 8 || !d_fields || !h_bc_kind || !d_bc)
    return fail(c, EBR_EINVAL, "ebr_reconstruct: 1..8 fields with kinds and boundary data required");
  if (dtype != EBR_F32 && dtype != EBR_F64) return fail(c, EBR_EINVAL, "ebr_reconstruct: bad dtype");
  for (int f = 0; f < n_fields; ++f) {
    if (!d_fields[f] || (!d_bc[f] && c->ng > 0))
      return fail(c, EBR_EINVAL, "ebr_reconstruct: null field %d", f);
    if (h_bc_kind[f] != 0 && h_bc_kind[f] != 1) return fail(c, EBR_EINVAL, "ebr_reconstruct: bad bc kind");
  }
  cudaStream_t s = S(stream);
  int kinds[8];
  for (int f = 0; f < n_fields; ++f) kinds[f] = h_bc_kind[f];
  std::vector<int> level_geoms;
  if (mode == EBR_MODE_PERSISTENT) {
    ChainPlan* cp = nullptr;
    ebr_status st = chain_plan(c, 0, dtype, n_fields, &cp);
    if (st) return st;
    if (cp->n_list > 0) {
      prof_begin(c, s, "fill_part");
      launch_fill_partial(dtype, n_fields, d_fields, kinds, d_bc, c->dG, c->g_geo, c->g_cell, c->g_meta,
                          wtab_of(c, dtype), c->ng, c->fpart, s, c->tb[TU_FILL_PART]);
      prof_end(c, s);
      prof_begin(c, s, "fill_chain");
      launch_fill_chain(dtype, 0, n_fields, d_fields, kinds, d_bc, c->dG, cp->d_list, cp->n_list,
                        c->g_cell, c->g_meta, c->g_dep, c->lev_ptr, wtab_of(c, dtype), c->ng, cp->smem,
                        c->fpart, c->d_status, s);
      prof_end(c, s);
      c->launches += 2;
      CKL();
    }
    level_geoms = cp->fallback;
  } else if (mode == EBR_MODE_LEVEL_LAUNCH) {
    for (int b = 0; b < c->B; ++b) level_geoms.push_back(b);
  } else {
    return fail(c, EBR_EINVAL, "ebr_reconstruct: bad mode %d", mode);
  }
  for (int b : level_geoms) {
    const Geom& g = c->hG[b];
    for (int lv = 1; lv <= g.n_levels; ++lv) {
      int p0 = c->h_lev_ptr[g.lev_off + lv - 1], p1 = c->h_lev_ptr[g.lev_off + lv];
      prof_begin(c, s, "fill_level");
      launch_fill_level(dtype, g.dim, n_fields, d_fields, kinds, d_bc, g.cell_off, p0, p1, c->g_cell,
                        c->g_meta, wtab_of(c, dtype), c->ng, g.n[0], g.n[1], c->d_status, s);
      prof_end(c, s);
      c->launches += 1;
    }
  }
  CKL();
  return EBR_OK;
}

ebr_status ebr_boundary_forces(void* ctx, const void* const* d_vel, const void* d_p, int32_t dtype,
                               double mu, const double* h_dirs, double* d_out, ebr_stream stream) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c) return EBR_EINVAL;
  EbrRange range_("ebr_boundary_forces");
  c->err.clear();
  if (!c->levelled) return fail(c, EBR_EINVAL, "ebr_boundary_forces: build the levels first");
  if (!d_vel || !d_p || !h_dirs || !d_out) return fail(c, EBR_EINVAL, "ebr_boundary_forces: null argument");
  if (dtype != EBR_F32 && dtype != EBR_F64) return fail(c, EBR_EINVAL, "ebr_boundary_forces: bad dtype");
  int dim = c->hG[0].dim;
  for (int b = 1; b < c->B; ++b)
    if (c->hG[b].dim != dim) return fail(c, EBR_EINVAL, "ebr_boundary_forces: mixed dimensions");
  cudaStream_t s = S(stream);
  prof_begin(c, s, "forces");
  launch_forces(dtype, dim, d_vel, d_p, mu, h_dirs, c->dG, c->n_chunks, c->chunks, c->g_cell,
                c->g_geo, c->g_n, c->g_meta, ftab_of(c, dtype), c->ng, c->partial, c->chunk_done, c->B, d_out,
                c->chunk_ptr, s);
  prof_end(c, s);
  c->launches += 1;
  CKL();
  return EBR_OK;
}

ebr_status ebr_reconstruct_adjoint(void* ctx, int32_t n_fields, const int32_t* h_bc_kind,
                                   const int32_t* h_vel_index, int32_t p_index, double mu,
                                   const double* h_dirs, const double* d_seed,
                                   void* const* d_grad_fields, void* const* d_grad_bc, int32_t dtype,
                                   int32_t accumulate, int32_t mode, ebr_stream stream) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c) return EBR_EINVAL;
  EbrRange range_("ebr_reconstruct_adjoint");
  c->err.clear();
  if (!c->levelled) return fail(c, EBR_EINVAL, "ebr_reconstruct_adjoint: build the levels first");
  if (n_fields < 1 || n_fields > 8 || !h_bc_kind || !h_vel_index || !h_dirs || !d_seed ||
      !d_grad_fields || !d_grad_bc)
    return fail(c, EBR_EINVAL, "ebr_reconstruct_adjoint: bad arguments");
  if (dtype != EBR_F32 && dtype != EBR_F64) return fail(c, EBR_EINVAL, "ebr_reconstruct_adjoint: bad dtype");
  int dim = c->hG[0].dim;
  for (int b = 1; b < c->B; ++b)
    if (c->hG[b].dim != dim) return fail(c, EBR_EINVAL, "ebr_reconstruct_adjoint: mixed dimensions");
  int role[4] = {-1, -1, -1, p_index};
  for (int a = 0; a < dim; ++a) role[a] = h_vel_index[a];
  for (int f = 0; f < n_fields; ++f) {
    if (!d_grad_fields[f] || (!d_grad_bc[f] && c->ng > 0))
      return fail(c, EBR_EINVAL, "ebr_reconstruct_adjoint: null gradient %d", f);
    if (h_bc_kind[f] != 0 && h_bc_kind[f] != 1) return fail(c, EBR_EINVAL, "ebr_reconstruct_adjoint: bad bc kind");
  }
  if (mode != EBR_MODE_PERSISTENT && mode != EBR_MODE_LEVEL_LAUNCH)
    return fail(c, EBR_EINVAL, "ebr_reconstruct_adjoint: bad mode %d", mode);
  cudaStream_t s = S(stream);
  int kinds[8];
  for (int f = 0; f < n_fields; ++f) kinds[f] = h_bc_kind[f];
  // everything that can fail runs before the fork below, so that an error
  // return never leaves the side stream unjoined (a stream capture would be
  // invalidated by the dangling branch)
  ChainPlan* cp = nullptr;
  if (mode == EBR_MODE_PERSISTENT) {
    ebr_status st = chain_plan(c, 1, dtype, n_fields, &cp);
    if (st) return st;
  }
  // at reach 1 the fluid targets' probe (which needs no lambda) runs on the
  // second stream beside the seed and chain kernels; the pull joins it
  const int kmax = stencil_k(dim);
  const bool split = c->rmax == 1 && c->ng > 0 && c->total_cells < (1LL << 31) && c->ng < (1 << 27) &&
                     c->af_cap > 0;
  if (split) {
    ebr_status st = ensure_side(c);
    if (st) return st;
    CK(cudaEventRecord(c->ev_fork, s));
    CK(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    prof_begin(c, c->side, "adj_probe");
    launch_adj_fprobe(c->ng, c->dG, c->g_geo, c->g_cell, c->g_meta, c->tags, c->pos_of_cell, kmax, c->af_cap,
                      c->af_cnt, c->af_cell, c->af_src, c->d_status, c->side, c->tb[TU_ADJ_PROBE]);
    prof_end(c, c->side);
    CK(cudaEventRecord(c->ev_join, c->side));
    c->launches += 1;
  }
  prof_begin(c, s, "adj_seed");
  launch_adj_seed(dtype, dim, n_fields, role, mu, h_dirs, d_seed, c->ng, c->g_geo, c->g_n, ftab_of(c, dtype), c->sv, s,
                  c->tb[TU_ADJ_SEED]);
  prof_end(c, s);
  c->launches += 1;
  std::vector<int> level_geoms;
  if (mode == EBR_MODE_PERSISTENT) {
    if (cp->n_list > 0) {
      prof_begin(c, s, "adj_part");
      launch_adj_part(dtype, n_fields, c->ng, c->gsrc_ptr, c->gsrc, c->g_meta, wtab_of(c, dtype), c->sv, c->apart,
                      c->acq, c->acw, c->n_gsrc, s, c->tb[TU_ADJ_PART]);
      prof_end(c, s);
      prof_begin(c, s, "adj_chain");
      launch_adj_chain(dtype, dim, n_fields, kinds, c->dG, cp->d_list, cp->n_list, c->lev_ptr,
                       c->gsrc_ptr, c->apart, c->acq, c->acw, c->n_gsrc, c->ng, c->lam, cp->smem, s);
      prof_end(c, s);
      c->launches += 2;
    }
    level_geoms = cp->fallback;
  } else {
    for (int b = 0; b < c->B; ++b) level_geoms.push_back(b);
  }
  for (int b : level_geoms) {
    const Geom& g = c->hG[b];
    for (int lv = g.n_levels; lv >= 1; --lv) {
      int p0 = c->h_lev_ptr[g.lev_off + lv - 1], p1 = c->h_lev_ptr[g.lev_off + lv];
      prof_begin(c, s, "adj_level");
      launch_adj_level(dtype, dim, n_fields, kinds, p0, p1, c->gsrc_ptr, c->gsrc, c->g_meta, wtab_of(c, dtype),
                       c->sv, c->ng, c->lam, s);
      prof_end(c, s);
      c->launches += 1;
    }
  }
  if (split) {
    // lambda is final: the BC gradients (and the zeros of the ghost cells'
    // gradient entries) on the second stream beside the fluid targets' pull
    // (disjoint outputs: ghost cells and boundary data there, fluid cells here)
    CK(cudaEventRecord(c->ev_lam, s));
    CK(cudaStreamWaitEvent(c->side, c->ev_lam, 0));
    prof_begin(c, c->side, "adj_bc");
    launch_adj_bc(dtype, n_fields, kinds, c->ng, c->dG, c->g_geo, c->g_cell, wtab_of(c, dtype), c->lam, d_grad_bc,
                  d_grad_fields, accumulate, c->side, c->tb[TU_ADJ_BC]);
    prof_end(c, c->side);
    CK(cudaEventRecord(c->ev_bc, c->side));
    c->launches += 1;
    CK(cudaStreamWaitEvent(s, c->ev_join, 0));
    prof_begin(c, s, "adj_fluid");
    launch_adj_fpull(dtype, n_fields, kinds, c->ng, kmax, c->af_cap, c->af_cnt, c->af_cell, c->af_src, wtab_of(c, dtype),
                     c->sv, c->lam, d_grad_fields, accumulate, s, c->tb[TU_ADJ_FLUID]);
    prof_end(c, s);
    c->launches += 1;
    CK(cudaStreamWaitEvent(s, c->ev_bc, 0));
    CKL();
    return EBR_OK;
  } else {
    prof_begin(c, s, "adj_fluid");
    launch_adj_fluid(dtype, n_fields, kinds, c->ng, c->dG, c->g_geo, c->g_cell, c->g_meta, c->tags,
                     c->pos_of_cell, c->rmax, wtab_of(c, dtype), c->sv, c->lam, d_grad_fields, accumulate, kmax, s,
                     c->tb[TU_ADJ_FLUID]);
    prof_end(c, s);
  }
  c->launches += 1;
  prof_begin(c, s, "adj_bc");
  launch_adj_bc(dtype, n_fields, kinds, c->ng, c->dG, c->g_geo, c->g_cell, wtab_of(c, dtype), c->lam, d_grad_bc,
                d_grad_fields, accumulate, s, c->tb[TU_ADJ_BC]);
  prof_end(c, s);
  c->launches += 1;
  CKL();
  return EBR_OK;
}

// ---------------------------------------------------------------------------
// many fields, field-minor layout
// ---------------------------------------------------------------------------
// Packed schedule: L0 = the last level in which some geometry has more than
// PACKED_TAIL_MAX ghosts; levels 1..L0 become grid-wide ghost lists, the
// geometries with more levels form the tail (deepest first).
static ebr_status packed_plan(Ctx* c, cudaStream_t s, const char* who) {
  if (c->pplan.built) return EBR_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone)
    return fail(c, EBR_EINVAL, "%s: the first packed call must precede stream capture (it plans the schedule)", who);
  PackedPlan pp;
  int maxlev = 0;
  for (int b = 0; b < c->B; ++b) maxlev = std::max(maxlev, c->hG[b].n_levels);
  std::vector<int> mx(maxlev + 2, 0);
  for (int b = 0; b < c->B; ++b) {
    const Geom& g = c->hG[b];
    for (int lv = 1; lv <= g.n_levels; ++lv)
      mx[lv] = std::max(mx[lv], c->h_lev_ptr[g.lev_off + lv] - c->h_lev_ptr[g.lev_off + lv - 1]);
  }
  pp.L0 = 1;
  pp.L0a = 1;
  for (int lv = 2; lv <= maxlev; ++lv) {
    if (mx[lv] > PACKED_TAIL_MAX) pp.L0 = lv;
    if (mx[lv] > PACKED_TAIL_MAX_ADJ) pp.L0a = lv;
  }
  const int Lmax = std::max(pp.L0, pp.L0a);
  std::vector<int> lst;
  pp.h_lvl_off.assign(Lmax + 1, 0);
  for (int lv = 1; lv <= Lmax; ++lv) {
    for (int b = 0; b < c->B; ++b) {
      const Geom& g = c->hG[b];
      if (lv > g.n_levels) continue;
      for (int q = c->h_lev_ptr[g.lev_off + lv - 1]; q < c->h_lev_ptr[g.lev_off + lv]; ++q) lst.push_back(q);
    }
    pp.h_lvl_off[lv] = (int)lst.size();
  }
  std::vector<int> tail, tail_a;
  for (int b = 0; b < c->B; ++b) {
    if (c->hG[b].n_levels > pp.L0) tail.push_back(b);
    if (c->hG[b].n_levels > pp.L0a) tail_a.push_back(b);
  }
  auto deeper = [&](int a, int b) { return c->hG[a].n_levels > c->hG[b].n_levels; };
  std::stable_sort(tail.begin(), tail.end(), deeper);
  std::stable_sort(tail_a.begin(), tail_a.end(), deeper);
  pp.n_tail = (int)tail.size();
  pp.n_tail_a = (int)tail_a.size();
  AL(pp.d_tail_a, std::max<size_t>(tail_a.size(), 1));
  if (!tail_a.empty())
    CK(cudaMemcpy(pp.d_tail_a, tail_a.data(), sizeof(int) * tail_a.size(), cudaMemcpyHostToDevice));
  AL(pp.d_lvl, std::max<size_t>(lst.size(), 1));
  AL(pp.d_tail, std::max<size_t>(tail.size(), 1));
  if (!lst.empty()) CK(cudaMemcpy(pp.d_lvl, lst.data(), sizeof(int) * lst.size(), cudaMemcpyHostToDevice));
  if (!tail.empty()) CK(cudaMemcpy(pp.d_tail, tail.data(), sizeof(int) * tail.size(), cudaMemcpyHostToDevice));
  const int ng = c->ng;
  const int kmax = stencil_k(c->hG[0].dim);
  // consumer lists of the ghosts
  AL(pp.cons_ptr, ng + 1);
  int* tmp_cnt = nullptr;
  AL(tmp_cnt, std::max<long long>((long long)ng * kmax, 1) + 1);
  launch_packed_plan_cons(ng, c->gsrc_ptr, c->gsrc, c->g_meta, nullptr, tmp_cnt, s);
  launch_scan(tmp_cnt, pp.cons_ptr, ng, c->scan_tmp, s);
  CKL();
  int n_cons = 0;
  CK(cudaMemcpyAsync(&n_cons, pp.cons_ptr + ng, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  AL(pp.cons, std::max(n_cons, 1));
  launch_packed_plan_cons(ng, c->gsrc_ptr, c->gsrc, c->g_meta, pp.cons_ptr, pp.cons, s);
  // fluid targets: owner flags and source counts per incidence, two scans
  const long long ninc = (long long)ng * kmax;
  if (ninc >= (1LL << 26)) return fail(c, EBR_EINVAL, "%s: too many ghost incidences for the packed plan", who);
  int *flag = nullptr, *tpos = nullptr, *epos = nullptr;
  AL(flag, ninc + 1);
  AL(tpos, ninc + 1);
  AL(epos, ninc + 1);
  launch_packed_plan_ftgt(ng, kmax, c->dG, c->g_geo, c->g_cell, c->g_meta, c->tags, c->pos_of_cell,
                          c->rmax, flag, tmp_cnt, nullptr, nullptr, nullptr, nullptr, nullptr, s);
  launch_scan(flag, tpos, (int)ninc, c->scan_tmp, s);
  launch_scan(tmp_cnt, epos, (int)ninc, c->scan_tmp, s);
  CKL();
  int tot[2] = {0, 0};
  CK(cudaMemcpyAsync(&tot[0], tpos + ninc, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&tot[1], epos + ninc, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  pp.n_ft = tot[0];
  AL(pp.ft_cell, std::max(tot[0], 1));
  AL(pp.ft_ptr, tot[0] + 1);
  AL(pp.ft_src, std::max(tot[1], 1));
  launch_packed_plan_ftgt(ng, kmax, c->dG, c->g_geo, c->g_cell, c->g_meta, c->tags, c->pos_of_cell,
                          c->rmax, nullptr, nullptr, tpos, epos, pp.ft_cell, pp.ft_ptr, pp.ft_src, s);
  CKL();
  CK(cudaMemcpyAsync(pp.ft_ptr + tot[0], &tot[1], sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  pp.built = true;
  c->pplan = pp;
  return EBR_OK;
}

// item records of the packed kernels for one field type (once per plan)
static ebr_status packed_records(Ctx* c, cudaStream_t s, int dtype, const char* who) {
  PackedPlan& pp = c->pplan;
  if (pp.rec_built[dtype]) return EBR_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone)
    return fail(c, EBR_EINVAL, "%s: the first packed call of a field type must precede stream capture", who);
  const int dim = c->hG[0].dim, ng = c->ng;
  AL(pp.rec_fwd[dtype], std::max<size_t>((size_t)ng * packed_rec_words(dtype, dim, 0), 1));
  AL(pp.rec_adj[dtype], std::max<size_t>((size_t)ng * packed_rec_words(dtype, dim, 1), 1));
  AL(pp.rec_fl[dtype], std::max<size_t>((size_t)pp.n_ft * packed_rec_words(dtype, dim, 1), 1));
  launch_packed_records(dtype, dim, c->dG, ng, c->g_geo, c->g_cell, c->g_meta, c->g_dep, c->wtab, pp,
                        pp.rec_fwd[dtype], pp.rec_adj[dtype], pp.rec_fl[dtype], s);
  int max_nt = 0, max_nta = 0;
  for (int b = 0; b < c->B; ++b) {
    const Geom& g = c->hG[b];
    const int end = c->h_lev_ptr[g.lev_off + g.n_levels];
    if (g.n_levels > pp.L0) max_nt = std::max(max_nt, end - c->h_lev_ptr[g.lev_off + pp.L0]);
    if (g.n_levels > pp.L0a) max_nta = std::max(max_nta, end - c->h_lev_ptr[g.lev_off + pp.L0a]);
  }
  pp.tail_max = max_nt;
  pp.tail_max_a = max_nta;
  pp.tail_smem[0][dtype] = packed_tail_smem(dtype, dim, 0, max_nt, max_smem_optin());
  pp.tail_smem[1][dtype] = packed_tail_smem(dtype, dim, 1, max_nta, max_smem_optin());
  CKL();
  CK(cudaStreamSynchronize(s));
  pp.rec_built[dtype] = true;
  return EBR_OK;
}

static ebr_status packed_args(Ctx* c, const char* who, int32_t n_fields, const int32_t* h_bc_kind,
                              int32_t dtype, KindBits* kb) {
  if (!c->levelled) return fail(c, EBR_EINVAL, "%s: build the levels first", who);
  if (n_fields < 1 || n_fields > PACKED_MAX_FIELDS || !h_bc_kind)
    return fail(c, EBR_EINVAL, "%s: 1..%d fields with kinds required", who, PACKED_MAX_FIELDS);
  if (dtype != EBR_F32 && dtype != EBR_F64) return fail(c, EBR_EINVAL, "%s: bad dtype", who);
  for (int b = 1; b < c->B; ++b)
    if (c->hG[b].dim != c->hG[0].dim) return fail(c, EBR_EINVAL, "%s: mixed dimensions", who);
  if (c->total_cells >= (1LL << 31)) return fail(c, EBR_EINVAL, "%s: more than 2^31 cells", who);
  std::memset(kb, 0, sizeof(KindBits));
  for (int f = 0; f < n_fields; ++f) {
    if (h_bc_kind[f] != 0 && h_bc_kind[f] != 1) return fail(c, EBR_EINVAL, "%s: bad bc kind", who);
    if (h_bc_kind[f]) kb->w[f >> 5] |= 1u << (f & 31);
  }
  return EBR_OK;
}

ebr_status ebr_reconstruct_packed(void* ctx, int32_t n_fields, void* d_fields,
                                  const int32_t* h_bc_kind, const void* d_bc, int32_t dtype,
                                  ebr_stream stream) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c) return EBR_EINVAL;
  EbrRange range_("ebr_reconstruct_packed");
  c->err.clear();
  KindBits kb;
  ebr_status st = packed_args(c, "ebr_reconstruct_packed", n_fields, h_bc_kind, dtype, &kb);
  if (st) return st;
  if (!d_fields || !d_bc) return fail(c, EBR_EINVAL, "ebr_reconstruct_packed: null field or boundary data");
  cudaStream_t s = S(stream);
  st = packed_plan(c, s, "ebr_reconstruct_packed");
  if (st) return st;
  st = packed_records(c, s, dtype, "ebr_reconstruct_packed");
  if (st) return st;
  static const char* names[3] = {"pfill_part", "pfill_lvl", "pfill_tail"};
  for (int ph = 0; ph < 3; ++ph) {
    prof_begin(c, s, names[ph]);
    launch_pfill(dtype, c->hG[0].dim, n_fields, d_fields, d_bc, kb, c->dG, c->lev_ptr, c->ng, c->pplan,
                 c->pplan.rec_fwd[dtype], c->d_status, s, ph);
    prof_end(c, s);
  }
  c->launches += pfill_launches(c->pplan, c->ng);
  CKL();
  return EBR_OK;
}

ebr_status ebr_reconstruct_packed_adjoint(void* ctx, int32_t n_fields, const int32_t* h_bc_kind,
                                          void* d_cot, void* d_grad_bc, int32_t dtype,
                                          ebr_stream stream) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c) return EBR_EINVAL;
  EbrRange range_("ebr_reconstruct_packed_adjoint");
  c->err.clear();
  KindBits kb;
  ebr_status st = packed_args(c, "ebr_reconstruct_packed_adjoint", n_fields, h_bc_kind, dtype, &kb);
  if (st) return st;
  if (!d_cot || !d_grad_bc) return fail(c, EBR_EINVAL, "ebr_reconstruct_packed_adjoint: null cotangent or gradient");
  cudaStream_t s = S(stream);
  st = packed_plan(c, s, "ebr_reconstruct_packed_adjoint");
  if (st) return st;
  st = packed_records(c, s, dtype, "ebr_reconstruct_packed_adjoint");
  if (st) return st;
  size_t need = (size_t)std::max(c->ng, 1) * n_fields * (dtype == EBR_F32 ? 4 : 8);
  if (need > c->lamP_bytes) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone)
      return fail(c, EBR_EINVAL, "ebr_reconstruct_packed_adjoint: first call with %d fields must precede stream capture (it sizes scratch)", n_fields);
    void* q = nullptr;
    st = balloc(c, &q, need);
    if (st) return st;
    c->lamP = q;
    c->lamP_bytes = need;
  }
  const int dim = c->hG[0].dim;
  for (int b = 1; b < c->B; ++b)
    if (c->hG[b].dim != dim) return fail(c, EBR_EINVAL, "ebr_reconstruct_packed_adjoint: mixed dimensions");
  static const char* names[3] = {"padj_tail", "padj_lvl", "padj_fluid"};
  for (int ph = 0; ph < 3; ++ph) {
    prof_begin(c, s, names[ph]);
    launch_padj(dtype, n_fields, d_cot, c->lamP, d_grad_bc, kb, c->dG, c->ng, c->lev_ptr, c->wtab,
                c->pplan, c->pplan.rec_adj[dtype], c->pplan.rec_fl[dtype], c->d_status, s, ph);
    prof_end(c, s);
  }
  c->launches += padj_launches(c->pplan, c->ng);
  CKL();
  return EBR_OK;
}

// ---------------------------------------------------------------------------
// tiled fill with per-level exchange (Sec. 3.2, distributed memory)
// ---------------------------------------------------------------------------
static ebr_status tiled_alloc(Ctx* c, void** p, size_t bytes) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, EBR_ENOMEM, "ebr_tiled_plan: cudaMalloc of %zu bytes failed", bytes);
  }
  c->tiled.mem.push_back(q);
  *p = q;
  return EBR_OK;
}

ebr_status ebr_tiled_plan(void* ctx, const int32_t* h_tile, ebr_stream stream) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c) return EBR_EINVAL;
  EbrRange range_("ebr_tiled_plan");
  c->err.clear();
  if (!c->levelled) return fail(c, EBR_EINVAL, "ebr_tiled_plan: build the levels first");
  if (!h_tile) return fail(c, EBR_EINVAL, "ebr_tiled_plan: null tile sizes");
  const int dim = c->hG[0].dim;
  int T[3] = {1, 1, 1};
  for (int a = 0; a < dim; ++a) {
    if (h_tile[a] < 1) return fail(c, EBR_EINVAL, "ebr_tiled_plan: tile size %d along axis %d", h_tile[a], a);
    T[a] = h_tile[a];
  }
  cudaStream_t s = S(stream);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone)
    return fail(c, EBR_EINVAL, "ebr_tiled_plan: plans on the host; call it outside stream capture");
  tiled_free(c);
  Ctx::Tiled& tp = c->tiled;
  const int ng = c->ng;
  std::vector<int> geo(ng), cell(ng), lev(ng), dep((size_t)MAXK * ng);
  if (ng > 0) {
    CK(cudaMemcpyAsync(geo.data(), c->g_geo, sizeof(int) * ng, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(cell.data(), c->g_cell, sizeof(int) * ng, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(lev.data(), c->g_level, sizeof(int) * ng, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(dep.data(), c->g_dep, sizeof(int) * MAXK * (size_t)ng, cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
  // tiles of every geometry, numbered after those of the geometries before it
  std::vector<long long> toff(c->B + 1, 0);
  std::vector<std::array<int, 3>> ntile(c->B);
  for (int b = 0; b < c->B; ++b) {
    long long nt = 1;
    for (int a = 0; a < 3; ++a) {
      ntile[b][a] = a < dim ? (c->hG[b].n[a] + T[a] - 1) / T[a] : 1;
      nt *= ntile[b][a];
    }
    toff[b + 1] = toff[b] + nt;
  }
  if (toff[c->B] >= (1LL << 31)) return fail(c, EBR_EINVAL, "ebr_tiled_plan: more than 2^31 tiles");
  tp.total_tiles = toff[c->B];
  tp.h_tile_global.assign(ng, 0);
  for (int p = 0; p < ng; ++p) {
    const Geom& g = c->hG[geo[p]];
    const int i = cell[p] % g.n[0], j = (cell[p] / g.n[0]) % g.n[1], k = cell[p] / (g.n[0] * g.n[1]);
    const long long t = i / T[0] + (long long)ntile[geo[p]][0] * (j / T[1] + (long long)ntile[geo[p]][1] * (k / T[2]));
    tp.h_tile_global[p] = (int)(toff[geo[p]] + t);
  }
  // active tiles (those owning a ghost), in tile order
  std::vector<int> act(tp.h_tile_global);
  std::sort(act.begin(), act.end());
  act.erase(std::unique(act.begin(), act.end()), act.end());
  const int NT = (int)act.size();
  std::vector<int> tile_of(ng);
  for (int p = 0; p < ng; ++p)
    tile_of[p] = (int)(std::lower_bound(act.begin(), act.end(), tp.h_tile_global[p]) - act.begin());
  int Lmax = 0;
  for (int b = 0; b < c->B; ++b) Lmax = std::max(Lmax, c->hG[b].n_levels);
  const int W = Lmax + 1;
  // ghosts of each (tile, level), in canonical order: level L (1-based) of
  // active tile i is bucket i W + L - 1, [t_ptr[i W + L - 1], t_ptr[i W + L])
  std::vector<int> t_ptr((size_t)NT * W + 1, 0), t_list(ng);
  for (int p = 0; p < ng; ++p) {
    if (lev[p] < 1 || lev[p] > Lmax) return fail(c, EBR_EINVAL, "ebr_tiled_plan: ghost %d without a level", p);
    ++t_ptr[(size_t)tile_of[p] * W + lev[p] - 1];
  }
  {
    int run = 0;
    for (size_t q = 0; q < t_ptr.size(); ++q) {
      const int v = t_ptr[q];
      t_ptr[q] = run;
      run += v;
    }
  }
  {
    std::vector<int> cur(t_ptr.begin(), t_ptr.end() - 1);
    for (int p = 0; p < ng; ++p) t_list[cur[(size_t)tile_of[p] * W + lev[p] - 1]++] = p;
  }
  // sent ghosts: a dependency of a ghost of another tile; (ghost, receiving
  // tile) pairs for the statistics
  std::vector<char> sent(ng, 0);
  std::vector<long long> pairs;
  for (int p = 0; p < ng; ++p)
    for (int k = 0; k < MAXK; ++k) {
      const int d = dep[(size_t)k * ng + p];
      if (d >= 0 && tile_of[d] != tile_of[p]) {
        sent[d] = 1;
        pairs.push_back((long long)d * (long long)(NT + 1) + tile_of[p]);
      }
    }
  std::sort(pairs.begin(), pairs.end());
  tp.pairs = (long long)(std::unique(pairs.begin(), pairs.end()) - pairs.begin());
  tp.h_slot.assign(ng, -1);
  tp.sent_per_level.assign(Lmax, 0);
  int n_slots = 0;
  for (int p = 0; p < ng; ++p)
    if (sent[p]) {
      tp.h_slot[p] = n_slots++;
      ++tp.sent_per_level[lev[p] - 1];
    }
  // conventional comparison: every sweep exchanges the ghosts within the
  // stencil reach of a tile face (to the tile across it); n_levels sweeps
  tp.halo = 0;
  {
    const int R = std::max(c->rmax, 1);
    std::vector<long long> per(c->B, 0);
    for (int p = 0; p < ng; ++p) {
      const Geom& g = c->hG[geo[p]];
      const int ijk[3] = {cell[p] % g.n[0], (cell[p] / g.n[0]) % g.n[1], cell[p] / (g.n[0] * g.n[1])};
      for (int a = 0; a < dim; ++a) {
        const int r = ijk[a] % T[a], base = ijk[a] - r;
        if (r < R && base > 0) ++per[geo[p]];
        if (T[a] - 1 - r < R && base + T[a] < g.n[a]) ++per[geo[p]];
      }
    }
    for (int b = 0; b < c->B; ++b) tp.halo += per[b] * c->hG[b].n_levels;
  }
  // upload
  int *d_ptr = nullptr, *d_list = nullptr, *d_tile = nullptr, *d_slot = nullptr;
  ebr_status st;
  if ((st = tiled_alloc(c, (void**)&d_ptr, sizeof(int) * t_ptr.size()))) return st;
  if ((st = tiled_alloc(c, (void**)&d_list, sizeof(int) * std::max(ng, 1)))) return st;
  if ((st = tiled_alloc(c, (void**)&d_tile, sizeof(int) * std::max(ng, 1)))) return st;
  if ((st = tiled_alloc(c, (void**)&d_slot, sizeof(int) * std::max(ng, 1)))) return st;
  if ((st = tiled_alloc(c, &tp.xbuf, (size_t)8 * 8 * std::max(n_slots, 1)))) return st;   // [F <= 8][slots] doubles
  if ((st = tiled_alloc(c, (void**)&tp.bar, 2 * sizeof(unsigned)))) return st;
  CK(cudaMemcpy(d_ptr, t_ptr.data(), sizeof(int) * t_ptr.size(), cudaMemcpyHostToDevice));
  if (ng > 0) {
    CK(cudaMemcpy(d_list, t_list.data(), sizeof(int) * ng, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_tile, tile_of.data(), sizeof(int) * ng, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_slot, tp.h_slot.data(), sizeof(int) * ng, cudaMemcpyHostToDevice));
  }
  tp.dev.n_tiles = NT;
  tp.dev.Lmax = Lmax;
  tp.dev.n_slots = std::max(n_slots, 1);
  tp.dev.spin_limit = 1 << 21;
  tp.dev.t_ptr = d_ptr;
  tp.dev.t_list = d_list;
  tp.dev.tile_of = d_tile;
  tp.dev.slot_of = d_slot;
  for (int a = 0; a < 3; ++a) tp.tile[a] = T[a];
  for (int dt = 0; dt < 2; ++dt) tp.grid[dt] = tiled_grid(dt, NT);
  CKL();
  tp.built = true;
  return EBR_OK;
}

ebr_status ebr_reconstruct_tiled(void* ctx, int32_t n_fields, void* const* d_fields,
                                 const int32_t* h_bc_kind, const void* const* d_bc, int32_t dtype,
                                 ebr_stream stream) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c) return EBR_EINVAL;
  EbrRange range_("ebr_reconstruct_tiled");
  c->err.clear();
  if (!c->tiled.built) return fail(c, EBR_EINVAL, "ebr_reconstruct_tiled: call ebr_tiled_plan first");
  if (n_fields < 1 || n_fields > 8 || !d_fields || !h_bc_kind || !d_bc)
    return fail(c, EBR_EINVAL, "ebr_reconstruct_tiled: 1..8 fields with kinds and boundary data required");
  if (dtype != EBR_F32 && dtype != EBR_F64) return fail(c, EBR_EINVAL, "ebr_reconstruct_tiled: bad dtype");
  for (int f = 0; f < n_fields; ++f) {
    if (!d_fields[f] || (!d_bc[f] && c->ng > 0))
      return fail(c, EBR_EINVAL, "ebr_reconstruct_tiled: null field %d", f);
    if (h_bc_kind[f] != 0 && h_bc_kind[f] != 1) return fail(c, EBR_EINVAL, "ebr_reconstruct_tiled: bad bc kind");
  }
  for (int b = 1; b < c->B; ++b)
    if (c->hG[b].dim != c->hG[0].dim) return fail(c, EBR_EINVAL, "ebr_reconstruct_tiled: mixed dimensions");
  Ctx::Tiled& tp = c->tiled;
  if (tp.dev.n_tiles == 0 || tp.dev.Lmax == 0) return EBR_OK;
  cudaStream_t s = S(stream);
  TiledPlanDev A = tp.dev;
  const int extra = tp.extra_once;
  if (tp.spin_once > 0) A.spin_limit = tp.spin_once;
  tp.extra_once = tp.spin_once = 0;
  prof_begin(c, s, "tiled_fill");
  cudaError_t e = launch_tiled_fill(dtype, c->hG[0].dim, n_fields, d_fields, h_bc_kind, d_bc, c->dG, A, tp.grid[dtype],
                                    c->g_geo, c->g_cell, c->g_meta, c->g_dep, wtab_of(c, dtype), c->ng, tp.xbuf, tp.bar,
                                    extra, c->d_status, s);
  prof_end(c, s);
  c->launches += 1;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, EBR_ECUDA, "ebr_reconstruct_tiled: launch failed: %s", cudaGetErrorString(e));
  }
  return EBR_OK;
}

ebr_status ebr_tiled_info(void* ctx, int64_t* h_out, int32_t n) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || !h_out || n < 1) return EBR_EINVAL;
  if (!c->tiled.built) return fail(c, EBR_EINVAL, "ebr_tiled_info: call ebr_tiled_plan first");
  const Ctx::Tiled& tp = c->tiled;
  long long nsent = 0;
  for (long long q : tp.sent_per_level) nsent += q;
  const long long v[8] = {tp.dev.n_tiles, tp.total_tiles, nsent, tp.pairs, tp.halo, tp.dev.Lmax,
                          tp.grid[0], tp.grid[1]};
  for (int k = 0; k < n; ++k)
    h_out[k] = k < 8 ? v[k] : (k - 8 < (int)tp.sent_per_level.size() ? tp.sent_per_level[k - 8] : 0);
  return EBR_OK;
}

ebr_status ebr_tiled_lists(void* ctx, int32_t* h_tile, int32_t* h_slot) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c) return EBR_EINVAL;
  if (!c->tiled.built) return fail(c, EBR_EINVAL, "ebr_tiled_lists: call ebr_tiled_plan first");
  for (int p = 0; p < c->ng; ++p) {
    if (h_tile) h_tile[p] = c->tiled.h_tile_global[p];
    if (h_slot) h_slot[p] = c->tiled.h_slot[p];
  }
  return EBR_OK;
}

ebr_status ebr_tiled_wait_test(void* ctx, int32_t spins) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c) return EBR_EINVAL;
  if (!c->tiled.built) return fail(c, EBR_EINVAL, "ebr_tiled_wait_test: call ebr_tiled_plan first");
  if (spins < 1 || spins > (1 << 24)) return fail(c, EBR_EINVAL, "ebr_tiled_wait_test: spins in 1..2^24");
  c->tiled.extra_once = 1;
  c->tiled.spin_once = spins;
  return EBR_OK;
}

ebr_status ebr_stats(void* ctx, double* h_alpha, int64_t* h_alpha_hist, int32_t n_bins, int64_t* h_level_hist,
                     int32_t n_levels, int64_t* h_r_hist, ebr_stream stream) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c) return EBR_EINVAL;
  EbrRange range_("ebr_stats");
  c->err.clear();
  if (!c->levelled) return fail(c, EBR_EINVAL, "ebr_stats: build the levels first");
  if (n_bins < 1 || n_bins > 4096 || n_levels < 0)
    return fail(c, EBR_EINVAL, "ebr_stats: 1..4096 bins, n_levels >= 0");
  cudaStream_t s = S(stream);
  const size_t n_ext = 6 * (size_t)c->B, n_a = 3 * (size_t)n_bins, n_r = 48;
  unsigned long long* buf = nullptr;
  {
    ebr_status st = dalloc(c, &c->stats_buf, n_ext + n_a + n_r);
    if (st) return st;
    buf = c->stats_buf;
  }
  // extrema start at the smallest ordered value, counts at zero
  CK(cudaMemsetAsync(buf, 0, sizeof(unsigned long long) * (n_ext + n_a + n_r), s));
  launch_stats(c->dG, c->ng, c->g_geo, c->g_cell, c->g_psi, c->g_n, c->g_meta, n_bins, buf, buf + n_ext,
               buf + n_ext + n_a, s);
  c->launches += c->ng > 0 ? 1 : 0;
  CKL();
  std::vector<unsigned long long> h(n_ext + n_a + n_r);
  CK(cudaMemcpyAsync(h.data(), buf, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  auto unbits = [](unsigned long long u) {
    const unsigned long long b = (u >> 63) ? (u & ~(1ull << 63)) : ~u;
    double v;
    std::memcpy(&v, &b, sizeof v);
    return v;
  };
  for (int b = 0; b < c->B; ++b) {
    const Geom& g = c->hG[b];
    for (int a = 0; a < 3; ++a) {
      const bool any = g.n_ghost > 0 && a < g.dim;
      if (h_alpha) {
        h_alpha[(size_t)b * 6 + a] = any ? unbits(h[(size_t)b * 6 + a]) : 0.0;
        h_alpha[(size_t)b * 6 + 3 + a] = any ? -unbits(h[(size_t)b * 6 + 3 + a]) : 0.0;
      }
    }
  }
  if (h_alpha_hist)
    for (size_t q = 0; q < n_a; ++q) h_alpha_hist[q] = (int64_t)h[n_ext + q];
  if (h_r_hist)
    for (size_t q = 0; q < n_r; ++q) h_r_hist[q] = (int64_t)h[n_ext + n_a + q];
  if (h_level_hist) {
    for (int k = 0; k < n_levels; ++k) h_level_hist[k] = 0;
    for (int b = 0; b < c->B; ++b) {
      const Geom& g = c->hG[b];
      for (int lv = 1; lv <= g.n_levels && lv <= n_levels; ++lv)
        h_level_hist[lv - 1] += c->h_lev_ptr[g.lev_off + lv] - c->h_lev_ptr[g.lev_off + lv - 1];
    }
  }
  return EBR_OK;
}

int32_t ebr_tunable_kernels(char* h_names, int32_t max_entries) {
  for (int i = 0; i < TU_N && i < max_entries; ++i) {
    if (!h_names) break;
    std::strncpy(h_names + 32 * i, kTuneNames[i], 31);
    h_names[32 * i + 31] = 0;
  }
  return TU_N;
}

ebr_status ebr_set_block_size(void* ctx, const char* kernel, int32_t threads) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c) return EBR_EINVAL;
  c->err.clear();
  const int id = tune_id(kernel);
  if (id < 0) return fail(c, EBR_EINVAL, "ebr_set_block_size: no tunable kernel named '%s'", kernel ? kernel : "(null)");
  if (threads < 32 || threads > TUNE_MAX || threads % 32 != 0)
    return fail(c, EBR_EINVAL, "ebr_set_block_size: %d threads (a multiple of 32 in 32..%d)", threads, TUNE_MAX);
  c->tb[id] = threads;
  return EBR_OK;
}

int32_t ebr_get_block_size(const void* ctx, const char* kernel) {
  const Ctx* c = static_cast<const Ctx*>(ctx);
  if (!c) return EBR_EINVAL;
  const int id = tune_id(kernel);
  return id < 0 ? EBR_EINVAL : c->tb[id];
}

ebr_status ebr_profile(void* ctx, int32_t enable) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c) return EBR_EINVAL;
  c->prof = enable != 0;
  if (c->prof) {
    c->recs.clear();
    c->pool_used = 0;
  }
  return EBR_OK;
}

int32_t ebr_profile_read(void* ctx, int32_t max_entries, char* h_names, double* h_ms,
                         int64_t* h_count, int32_t keep) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c) return EBR_EINVAL;
  std::vector<std::string> names;
  std::vector<double> ms;
  std::vector<long long> cnt;
  for (auto& r : c->recs) {
    if (!r.a || !r.b) continue;
    if (cudaEventSynchronize(r.b) != cudaSuccess) return fail(c, EBR_ECUDA, "event synchronise failed");
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return fail(c, EBR_ECUDA, "event timing failed");
    size_t k = 0;
    while (k < names.size() && names[k] != r.name) ++k;
    if (k == names.size()) { names.push_back(r.name); ms.push_back(0.0); cnt.push_back(0); }
    ms[k] += t;
    cnt[k] += 1;
  }
  int n = (int)names.size();
  for (int k = 0; k < n && k < max_entries; ++k) {
    if (h_names) {
      std::strncpy(h_names + 32 * k, names[k].c_str(), 31);
      h_names[32 * k + 31] = 0;
    }
    if (h_ms) h_ms[k] = ms[k];
    if (h_count) h_count[k] = cnt[k];
  }
  if (!keep) {
    c->recs.clear();
    c->pool_used = 0;
  }
  return n;
}

int32_t ebr_profile_timeline(void* ctx, int32_t max_entries, char* h_names, double* h_start_ms,
                             double* h_end_ms) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c) return EBR_EINVAL;
  const Ctx::ProfRec* first = nullptr;
  for (auto& r : c->recs)
    if (r.a && r.b) { first = &r; break; }
  if (!first) return 0;
  int n = 0;
  for (auto& r : c->recs) {
    if (!r.a || !r.b) continue;
    if (cudaEventSynchronize(r.b) != cudaSuccess) return fail(c, EBR_ECUDA, "event synchronise failed");
    if (n < max_entries) {
      float t0 = 0.0f, t1 = 0.0f;
      // a record that began before the first one reads as a negative start
      if (cudaEventElapsedTime(&t0, first->a, r.a) != cudaSuccess ||
          cudaEventElapsedTime(&t1, first->a, r.b) != cudaSuccess)
        return fail(c, EBR_ECUDA, "event timing failed");
      if (h_names) {
        std::strncpy(h_names + 32 * n, r.name, 31);
        h_names[32 * n + 31] = 0;
      }
      if (h_start_ms) h_start_ms[n] = t0;
      if (h_end_ms) h_end_ms[n] = t1;
    }
    ++n;
  }
  return n;
}

ebr_status ebr_diagnostics(void* ctx, int64_t* h_out, int32_t n, ebr_stream stream) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || !h_out || n < 1) return EBR_EINVAL;
  if (!c->planned) return fail(c, EBR_EINVAL, "ebr_diagnostics: call ebr_plan first");
  int st[2] = {0, 0};
  cudaStream_t s = S(stream);
  CK(cudaMemcpyAsync(st, c->d_stats, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (n > 0) h_out[0] = st[0];
  if (n > 1) h_out[1] = c->rmax;
  if (n > 2) h_out[2] = c->launches;
  if (n > 3) h_out[3] = c->n_gsrc;
  // packed schedule (zeros before the first packed call)
  const PackedPlan& pp = c->pplan;
  const long long pk[7] = {pp.L0, pp.L0a, pp.n_tail, pp.n_tail_a, pp.tail_max, pp.tail_max_a, pp.n_ft};
  for (int k = 0; k < 7 && 4 + k < n; ++k) h_out[4 + k] = pp.built ? pk[k] : 0;
  if (n > 11) h_out[11] = c->n_alloc;
  return EBR_OK;
}

ebr_status ebr_sync_status(void* ctx, ebr_stream stream) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c) return EBR_EINVAL;
  EbrRange range_("ebr_sync_status");
  if (!c->d_status) return EBR_OK;
  int hs = 0;
  cudaStream_t s = S(stream);
  CK(cudaMemcpyAsync(&hs, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (hs != 0) {
    CK(cudaMemset(c->d_status, 0, sizeof(int)));
    return fail(c, (ebr_status)hs, "device status %d", hs);
  }
  return EBR_OK;
}

}  // extern "C"

// Kernel declarations shared by the host-side orchestration (api.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "ebr_device.cuh"
#include "lookback.cuh"

namespace ebr {

// flat-row -> geometry by binary search over offsets [B + 1]
__device__ inline int find_seg(const int* off, int B, int x) {
  int lo = 0, hi = B - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Programmatic dependent launch.  A kernel launched through launch() may be
// launched before the kernel ahead of it in the stream has completed: once
// every block of that kernel has exited, not after its completion has been
// signalled.  Every such kernel therefore begins with pdl_enter():
// griddepcontrol.wait returns once the preceding grids have completed and
// their writes are visible, and no memory is touched before it.  No kernel
// triggers its dependents early (griddepcontrol.launch_dependents): blocks of
// the next kernel parked on the SMs took slots from the kernels of the other
// stream of a step and made the step slower.  A no-op for a plain launch.
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Item of this thread when the warps of the grid take 32-item chunks
// interleaved across blocks (warp w of block b: chunk w * gridDim.x + b)
// instead of consecutively: consecutive chunks land in different blocks, so
// that a stretch of expensive items (one geometry's airfoil cells, say) is
// spread over all SMs instead of loading a few.  A bijection onto
// [0, gridDim.x * blockDim.x) for a block size that is a multiple of 32;
// every warp still reads 32 consecutive items.
__device__ __forceinline__ int interleaved_item() {
  return ((threadIdx.x >> 5) * gridDim.x + blockIdx.x) * 32 + (threadIdx.x & 31);
}

// process-wide switch (ebr_set_pdl), on by default
extern int g_pdl;

// Launch of a library kernel on stream s (errors surface through
// cudaGetLastError like a <<< >>> launch).
template <typename... P, typename... A>
inline void launch(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = g_pdl ? at : nullptr;
  cfg.numAttrs = g_pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}

// Raise (never lower) the dynamic shared-memory opt-in of kernel K on the
// current device to `bytes`: the opt-in is per function and per device, and a
// graph captured earlier may still hold a launch with a larger size.
template <auto K>
inline void smem_raise(size_t bytes) {
  static size_t seen[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && bytes <= seen[dev]) return;
  cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (dev >= 0 && dev < 64) seen[dev] = bytes;
}

// Check of a re-run against the plan, done by block 0 of the next kernel:
// stage 0 the interface offsets of the rows and the ghost offsets of the
// interface list at the geometry boundaries, stage 1 the level count of every
// geometry; stage -1 (planning) nothing.  A difference is EBR_ESHAPE.
struct PlanCheck {
  const int* row_ptr;
  const int* gpos;
  const int* nlev;
  int B, n_iface, ng, stage;
};

__device__ inline void plan_check(const Geom* G, const PlanCheck& C, int* status) {
  if (C.stage < 0 || blockIdx.x != 0) return;
  for (int b = threadIdx.x; b < C.B; b += blockDim.x) {
    const Geom& g = G[b];
    if (C.stage == 0) {
      if (C.row_ptr[g.row_off] != g.iface_off) set_status(status, S_ESHAPE);
      if (b == C.B - 1 && C.row_ptr[g.row_off + g.n_rows] != C.n_iface) set_status(status, S_ESHAPE);
      if (C.gpos[g.iface_off] != g.ghost_off) set_status(status, S_ESHAPE);
      if (b == C.B - 1 && C.gpos[C.n_iface] != C.ng) set_status(status, S_ESHAPE);
    } else if (C.nlev[b] != g.n_levels) {
      set_status(status, S_ESHAPE);
    }
  }
}

// kind (0 Dirichlet, 1 Neumann) of field f of a packed field array: bit f
struct KindBits {
  uint32_t w[32];
};
constexpr int PACKED_MAX_FIELDS = 1024;

// ---- classify.cu
void launch_rows(const Geom* G, const int* row_off, int B, int total_rows, int2* runs,
                 int8_t* tags, int* status, int* stats, cudaStream_t s);
void launch_iface(const Geom* G, const int* row_off, int B, int total_rows, const int2* runs,
                  int* row_cnt, const int* row_ptr, int* iface_cell, int* iface_geo,
                  int8_t* iface_solid, int write, int iface_cap, int* status, cudaStream_t s, int T = 128);
// iface_meta (may be null): normal sign / zero bytes of the HGC candidates
void launch_place(const Geom* G, int n_iface, const int* iface_cell, const int* iface_geo,
                  const int8_t* iface_solid, int placement, int8_t* tags, uint8_t* iface_meta,
                  int* status, cudaStream_t s, int T = 128);
void launch_reclassify(const Geom* G, int n_iface, const int* iface_cell, const int* iface_geo,
                       int8_t* tags, int pass, cudaStream_t s);
// single-pass variants for a classification re-run (sizes known from the
// plan): interface cells with their row offsets in one launch; ghost flags,
// offsets and records in one launch (pass 1: HGC reclassification pass B of
// each cell first, in place; pass 2: passes A and B both from the placement's
// tags, the final tags to iface_tag; iface_meta: complete meta words from the
// placement's normal bytes); the per-ghost geometry after either (split: it
// leaves the compaction's meta words alone and checks them)
void launch_iface_fused(const Geom* G, const int* row_off, int B, int total_rows, const int2* runs,
                        int* row_ptr, int* iface_cell, int* iface_geo, int8_t* iface_solid, int iface_cap,
                        const Lookback& L, int* status, cudaStream_t s);
void launch_ghost_compact(const Geom* G, int n_iface, const int* iface_cell, const int* iface_geo,
                          int8_t* tags, int pass, const uint8_t* iface_meta, int8_t* iface_tag, int* gpos,
                          int ng_cap, int* gs_cell, int* gs_geo, uint32_t* gs_meta, const Lookback& L,
                          int* status, cudaStream_t s);
void launch_ghost_geom(const Geom* G, int placement, int ng_cap, int* gs_cell, int* gs_geo, double* gs_psi,
                       double* gs_n, uint32_t* gs_meta, int split, int* rmax, int* status, cudaStream_t s,
                       int T = 128, const PlanCheck& chk = PlanCheck{nullptr, nullptr, nullptr, 0, 0, 0, -1});
// second ghost layer (geometries with layers == 2), after the reclassification
void launch_layer2(const Geom* G, int n_iface, const int* iface_cell, const int* iface_geo, int8_t* tags,
                   int* status, cudaStream_t s);
void launch_ghost_flags(const Geom* G, int n_iface, const int* iface_cell, const int* iface_geo,
                        const int8_t* tags, int* flags, cudaStream_t s);
void launch_ghost_write(const Geom* G, int n_iface, const int* iface_cell, const int* iface_geo,
                        const int8_t* tags, const int* gpos, int placement, int ng_cap, int* gs_cell,
                        int* gs_geo, double* gs_psi, double* gs_n, uint32_t* gs_meta, int* rmax,
                        int* status, cudaStream_t s, int T = 128);

// ---- scan.cu : exclusive scan of n int32 values into out[0..n]; out[n] = total
size_t scan_temp_bytes(int n);
void launch_scan(const int* in, int* out, int n, void* temp, cudaStream_t s);

// ---- levels.cu
// (iface_tag non-null: also the final tags of the n_iface interface cells,
// decided by a compaction with pass 2, written to tags)
void launch_poscell(const Geom* G, int ng, const int* cell, const int* geo, const int* pos_of,
                    int* pos_of_cell, int* src_cnt, cudaStream_t s, int n_iface = 0,
                    const int* iface_cell = nullptr, const int* iface_geo = nullptr,
                    const int8_t* iface_tag = nullptr, int8_t* tags = nullptr);
void launch_deps(const Geom* G, int ng, const int* gs_cell, const int* gs_geo, uint32_t* gs_meta,
                 const int8_t* tags, const int* pos_of_cell, int* dep, int* status, cudaStream_t s,
                 int T = 128);
size_t levels_smem(int dim, int n_ghost);
void launch_levels(const Geom* G, int B, const int* dep, int ng_total, int* level, int* order_pos,
                   int* lev_ptr, int* n_levels, size_t smem, int* status, cudaStream_t s);
// canonical reorder of the ghost records; writes pos_of_cell (canonical
// position of each ghost cell) as well
void launch_reorder(const Geom* G, int* pos_of_cell, int ng, const int* order_pos, const int* gs_cell,
                    const int* gs_geo,
                    const double* gs_psi, const double* gs_n, const uint32_t* gs_meta,
                    const int* dep, const int* level, int* g_cell, int* g_geo, double* g_psi,
                    double* g_n, uint32_t* g_meta, int* g_dep, int* g_level, cudaStream_t s,
                    const PlanCheck& chk = PlanCheck{nullptr, nullptr, nullptr, 0, 0, 0, -1},
                    int* status = nullptr);
// weight table wtab [2][8][ng], force table ftab [33][ng] (double) and
// their float copies
void launch_tables(const Geom* G, int ng, const int* g_cell, const int* g_geo, const double* g_psi,
                   const double* g_n, const uint32_t* g_meta, const int8_t* tags, double* wtab,
                   double* ftab, float* wtab_f, float* ftab_f, cudaStream_t s, int T = 128);
// ghost targets' source lists by transposition: member ghost positions
// mem [MAXK][ng] and source counts (cnt preset to 1); offsets by a scan, then
// the own entries (self, planning), the scattered sources and the sort; or
// offsets + own entries in one single-pass launch (a re-run)
void launch_gsrc_count(const Geom* G, int ng, const int* g_cell, const int* g_geo, const uint32_t* g_meta,
                       const int* g_dep, const int8_t* tags, const int* pos_of_cell, int kmax, int* mem, int* cnt,
                       cudaStream_t s, int T = 128);
void launch_gsrc_lists(int ng, int kmax, const int* mem, const int* ptr, int* cursor, int* src, int cap,
                       int* status, bool self, cudaStream_t s, int T = 128);
void launch_gsrc_place(int ng, int* cnt_cursor, int* ptr, int* src, int cap, const Lookback& L, int* status,
                       cudaStream_t s);


// ---- fill.cu
void launch_fill_level(int dtype, int dim, int F, void* const* fields, const int* bc_kind,
                       const void* const* bc, long long cell_off, int p0, int p1, const int* g_cell,
                       const uint32_t* g_meta, const void* wtab, int ng_total, int nx, int ny,
                       int* status, cudaStream_t s);
size_t fill_chain_smem(int dtype, int dim, int F, int n_ghost);
void launch_fill_chain(int dtype, int dim, int F, void* const* fields, const int* bc_kind,
                       const void* const* bc, const Geom* G, const int* geo_list, int n_list,
                       const int* g_cell, const uint32_t* g_meta, const int* g_dep,
                       const int* lev_ptr, const void* wtab, int ng_total, size_t smem,
                       const void* part, int* status, cudaStream_t s);
// partial sums [F][ng] (boundary term + fluid members) of every ghost, read
// by the chain kernel
void launch_fill_partial(int dtype, int F, void* const* fields, const int* bc_kind, const void* const* bc,
                         const Geom* G, const int* g_geo, const int* g_cell, const uint32_t* g_meta,
                         const void* wtab, int ng, void* part, cudaStream_t s, int T = 128);

// ---- forces.cu
void launch_forces(int dtype, int dim, const void* const* vel, const void* p, double mu,
                   const double* dirs, const Geom* G, int n_chunks, const int4* chunks,
                   const int* g_cell, const int* g_geo, const double* g_n, const uint32_t* g_meta,
                   const void* ftab, int ng_total, double* partial, int* done, int B, double* out,
                   const int* chunk_ptr, cudaStream_t s);

// ---- adjoint.cu
// the force coefficients sv [F * 8][ng] in the field type (dtype)
void launch_adj_seed(int dtype, int dim, int F, const int* role, double mu, const double* dirs,
                     const double* seed, int ng, const int* g_geo, const double* g_n,
                     const void* ftab, void* sv, cudaStream_t s, int T = 128);
void launch_adj_level(int dtype, int dim, int F, const int* bc_kind, int p0, int p1,
                      const int* gsrc_ptr, const int* gsrc, const uint32_t* g_meta,
                      const void* wtab, const void* sv, int ng_total, void* lam, cudaStream_t s);
size_t adj_chain_smem(int dtype, int F, int n_ghost, int n_src);
// lambda's start values [F][ng] and the incidence records of the source
// lists (consumer position or -1, weights [2][n_src]) for the chain kernel
void launch_adj_part(int dtype, int F, int ng, const int* gsrc_ptr, const int* gsrc, const uint32_t* g_meta,
                     const void* wtab, const void* sv, void* lpart, int* cq_g, void* cw_g, int n_src,
                     cudaStream_t s, int T = 128);
void launch_adj_chain(int dtype, int dim, int F, const int* bc_kind, const Geom* G,
                      const int* geo_list, int n_list, const int* lev_ptr, const int* gsrc_ptr,
                      const void* lpart, const int* cq_g, const void* cw_g, int n_src,
                      int ng_total, void* lam, size_t smem, cudaStream_t s);
// fluid targets in two passes at reach 1: probe (no lambda needed) and pull
int adj_fluid_cap(int dim);
void launch_adj_fprobe(int ng, const Geom* G, const int* g_geo, const int* g_cell, const uint32_t* g_meta,
                       const int8_t* tags, const int* pos_of_cell, int kmax, int cap, int* fcnt, int* fcell,
                       int* fsrc, int* status, cudaStream_t s, int T = 128);
void launch_adj_fpull(int dtype, int F, const int* bc_kind, int ng, int kmax, int cap, const int* fcnt,
                      const int* fcell, const int* fsrc, const void* wtab, const void* sv, const void* lam,
                      void* const* grad, int accumulate, cudaStream_t s, int T = 128);
void launch_adj_fluid(int dtype, int F, const int* bc_kind, int ng, const Geom* G, const int* g_geo,
                      const int* g_cell, const uint32_t* g_meta, const int8_t* tags,
                      const int* pos_of_cell, int rmax, const void* wtab, const void* sv,
                      const void* lam, void* const* grad, int accumulate, int kmax, cudaStream_t s, int T = 128);
void launch_adj_bc(int dtype, int F, const int* bc_kind, int ng, const Geom* G, const int* g_geo,
                   const int* g_cell, const void* wtab, const void* lam, void* const* grad_bc,
                   void* const* grad, int accumulate, cudaStream_t s, int T = 128);

// ---- stats.cu (Sec. 7, Eq. stability_alpha_max): ext [B][6] ordered bits of
// max alpha_x,y,z and max -alpha_x,y,z; ahist [3][n_bins] over [-0.5, 1);
// rhist [3][16] multipliers
void launch_stats(const Geom* G, int ng, const int* g_geo, const int* g_cell, const double* g_psi,
                  const double* g_n, const uint32_t* g_meta, int n_bins, unsigned long long* ext,
                  unsigned long long* ahist, unsigned long long* rhist, cudaStream_t s);

// ---- tiled.cu (Sec. 3.2, distributed memory: tiles with a per-level exchange)
// Device view of a tile schedule: the ghosts of active tile i in level L are
// t_list[t_ptr[i (Lmax + 1) + L - 1] .. t_ptr[i (Lmax + 1) + L]) (canonical
// positions); tile_of[p] is the active tile of ghost p, slot_of[p] its slot in
// the exchange buffer ([F][n_slots]) when another tile's stencil reads it, else -1.
struct TiledPlanDev {
  int n_tiles = 0;
  int Lmax = 0;
  int n_slots = 0;
  int spin_limit = 0;
  const int* t_ptr = nullptr;
  const int* t_list = nullptr;
  const int* tile_of = nullptr;
  const int* slot_of = nullptr;
};
// CTAs of the cooperative tiled fill: all tiles, at most the resident CTAs
int tiled_grid(int dtype, int n_tiles);
// zeroes the barrier words and launches the cooperative fill; extra_arrivals
// > 0 makes the first barrier wait for arrivals that never come (the bounded
// wait then reports EBR_ETIMEOUT)
cudaError_t launch_tiled_fill(int dtype, int dim, int F, void* const* fields, const int* bc_kind, const void* const* bc,
                              const Geom* G, const TiledPlanDev& A, int grid, const int* g_geo,
                              const int* g_cell, const uint32_t* g_meta, const int* g_dep, const void* wtab,
                              int ng, void* xbuf, unsigned* bar, int extra_arrivals, int* status,
                              cudaStream_t s);

// ---- packed.cu (field-minor layout [cells][F])
// Schedule of the packed kernels, planned once per levelled geometry set:
// forward levels 1..L0 (adjoint 1..L0a) run grid-wide from the ghost lists
// d_lvl[h_lvl_off[l - 1] .. h_lvl_off[l]); the levels above (at most
// PACKED_TAIL_MAX, resp. PACKED_TAIL_MAX_ADJ, ghosts per geometry and level)
// run in one CTA per geometry of d_tail (d_tail_a).
// (measured on the 256-geometry batch with 192 fields, with 256-thread tail
// CTAs: forward 64 / transpose 16 against 128 / 128 with 512-thread CTAs
// took the overlapped step from 0.285 to 0.246 ms -- more levels as
// grid-wide launches, shorter shared-memory tails, more tail CTAs per SM)
#ifndef EBR_PACKED_TAIL_MAX
#define EBR_PACKED_TAIL_MAX 64
#endif
#ifndef EBR_PACKED_TAIL_MAX_ADJ
#define EBR_PACKED_TAIL_MAX_ADJ 16
#endif
constexpr int PACKED_TAIL_MAX = EBR_PACKED_TAIL_MAX;           // forward tail (shared memory)
constexpr int PACKED_TAIL_MAX_ADJ = EBR_PACKED_TAIL_MAX_ADJ;   // adjoint tail (shared memory; else global memory)
constexpr int PACKED_MAX_SOURCES = 64;   // sources of one item (consumers / fluid sources)
struct PackedPlan {
  bool built = false;
  int L0 = 1;
  int* d_lvl = nullptr;
  std::vector<int> h_lvl_off;
  int* d_tail = nullptr;
  int n_tail = 0;
  int L0a = 1;
  int* d_tail_a = nullptr;
  int n_tail_a = 0;
  int* cons_ptr = nullptr;     // [ng + 1] active consumers of each ghost (q << 3 | slot)
  int* cons = nullptr;
  int n_ft = 0;                // fluid targets
  int* ft_cell = nullptr;      // [n_ft] global cell
  int* ft_ptr = nullptr;       // [n_ft + 1]
  int* ft_src = nullptr;       // sources (q << 3 | slot), fixed probe order
  // per field type (0 FP32, 1 FP64): item records (forward, adjoint, fluid)
  bool rec_built[2] = {false, false};
  uint32_t* rec_fwd[2] = {nullptr, nullptr};
  uint32_t* rec_adj[2] = {nullptr, nullptr};
  uint32_t* rec_fl[2] = {nullptr, nullptr};
  // dynamic shared memory of the tail kernels [forward, adjoint][type];
  // 0 = the largest tail does not fit, the global-memory tail kernels run
  size_t tail_smem[2][2] = {{0, 0}, {0, 0}};
  int tail_max = 0;            // largest forward tail (ghosts of levels > L0 in one geometry)
  int tail_max_a = 0;          // largest adjoint tail (levels > L0a)
};
size_t packed_tail_smem(int dtype, int dim, int which, int max_nt, int limit);
// words per record: which = 0 forward, 1 adjoint / fluid
size_t packed_rec_words(int dtype, int dim, int which);
void launch_packed_records(int dtype, int dim, const Geom* G, int ng, const int* g_geo,
                           const int* g_cell, const uint32_t* g_meta, const int* g_dep,
                           const double* wtab, const PackedPlan& pp, uint32_t* fwd, uint32_t* adj,
                           uint32_t* fl, cudaStream_t s);
// forward phases: 0 partial sums of every ghost, 1 levels 2..L0 grid-wide,
// 2 the tail CTAs.  Adjoint phases (lambda in reverse level order, with the
// boundary-data gradients and the ghost cotangents cleared): 0 the tail CTAs,
// 1 levels L0..1 grid-wide; 2 the fluid targets.
void launch_pfill(int dtype, int dim, int F, void* fld, const void* bc, const KindBits& kb,
                  const Geom* G, const int* lev_ptr, int ng, const PackedPlan& pp,
                  const uint32_t* rec, int* status, cudaStream_t s, int phase);
int pfill_launches(const PackedPlan& pp, int ng);
void launch_padj(int dtype, int F, void* cot, void* lamP, void* gbc, const KindBits& kb,
                 const Geom* G, int ng, const int* lev_ptr, const double* wtab,
                 const PackedPlan& pp, const uint32_t* rec_adj, const uint32_t* rec_fl,
                 int* status, cudaStream_t s, int phase);
int padj_launches(const PackedPlan& pp, int ng);
// plan kernels: ptr == null counts (out = counts), else writes the lists
void launch_packed_plan_cons(int ng, const int* gsrc_ptr, const int* gsrc, const uint32_t* g_meta,
                             const int* ptr, int* out, cudaStream_t s);
// tpos == null: flag / count per (ghost, member) incidence; else writes the
// target cells, offsets and sources
void launch_packed_plan_ftgt(int ng, int kmax, const Geom* G, const int* g_geo, const int* g_cell,
                             const uint32_t* g_meta, const int8_t* tags, const int* pos_of_cell,
                             int R, int* flag, int* cnt, const int* tpos, const int* epos,
                             int* ft_cell, int* ft_ptr, int* ft_src, cudaStream_t s);

}  // namespace ebr

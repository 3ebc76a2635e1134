/*
 * ebr.h -- C ABI of the B300 (sm_103a) direct ghost-cell reconstruction library.
 *
 * Method: "Stable, Compact, and Direct Ghost-Cell Reconstruction: A
 * Non-Iterative Approach for Embedded-Boundary Methods".  The library
 *   1. classifies the cells of Cartesian grids against analytic convex bodies
 *      and places ghost cells (HGC, CGC, CGC_ES; Sec. 3.1, Sec. 7),
 *   2. builds the ghost dependency DAG and its topological levels (Sec. 3.2),
 *   3. fills the ghost values level by level from the closed-form Dirichlet /
 *      Neumann relations (Secs. 4-5, Eqs. phi_G_Dir_2d, phi_G_Neu_2d,
 *      phi_G_Dir_3d, phi_G_Neu_3d),
 *   4. evaluates boundary values, gradients, pressure and viscous forces,
 *      drag and lift from the same relations (Sec. 6),
 *   5. and runs the adjoint of 3-4 (reverse level walk) for d(drag, lift).
 *
 * Conventions (all entry points):
 *   - Every call returns an ebr_status; 0 is success, negative is an error.
 *     No C++ exception crosses the ABI.  ebr_last_error() returns a message
 *     for the last failing call on that context (valid until the next call).
 *   - "d_" pointers are device pointers, "h_" pointers host pointers.  All
 *     caller-owned buffers stay caller-owned; the library never frees them.
 *     Library-owned device memory lives in the context and is released by
 *     ebr_destroy().
 *   - A call that takes a cudaStream_t enqueues its kernels on that stream
 *     and returns without synchronising, except where stated.  Faults found
 *     on the device (stencil outside the grid, cycle, non-finite input, a
 *     mismatch with the planned sizes, a barrier timeout) set a status word in
 *     the context; ebr_sync_status() synchronises the stream and returns it.
 *   - A context handles one "geometry set": B >= 1 independent geometries,
 *     each a grid and a body.  Cells of geometry b occupy the flat index range
 *     [cell_offset[b], cell_offset[b+1]) of every per-cell array (tags,
 *     fields, gradients), with offsets from ebr_layout() (geometries are
 *     concatenated in order, without padding).  Inside a geometry the linear
 *     index of cell (i, j, k) is i + n_x (j + n_y k).
 *   - Ghosts of all geometries are numbered in the canonical order
 *     (geometry, level, linear index).  Boundary data (d_bc) and boundary
 *     gradients (d_grad_bc) use this order; ebr_ghost_info() returns the
 *     ghost cells, their boundary points S and normals in the same order.
 *   - One context must not be used from two host threads at once.
 */
#ifndef EBR_H
#define EBR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* ebr_stream;   /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
  EBR_OK = 0,
  EBR_EINVAL = -1,          /* bad argument (null pointer, size, enum, order of calls)     */
  EBR_ENOMEM = -2,          /* device allocation failed                                    */
  EBR_ECUDA = -3,           /* a CUDA runtime call failed                                  */
  EBR_ECYCLE = -4,          /* the dependency graph has a cycle (Sec. 3.2 requires a DAG) */
  EBR_ESTENCIL_OOB = -5,    /* a stencil member lies outside its grid                      */
  EBR_ESTENCIL_SOLID = -6,  /* a stencil member is a solid (tag 1) cell: value undefined  */
  EBR_ETIMEOUT = -7,        /* a bounded device-side wait gave up                          */
  EBR_ENONFINITE = -8,      /* non-finite value met where the path needs a finite one     */
  EBR_ESHAPE = -9           /* the geometry differs from the plan (counts of a re-run, or
                               ghost tags in the tag buffer that the plan does not hold)  */
} ebr_status;

typedef enum { EBR_HGC = 0, EBR_CGC = 1, EBR_CGC_ES = 2 } ebr_placement;
/* OR'ed into the placement of ebr_plan: a second ghost layer (Sec. 7,
 * "Additional ghost-cell layers"), with EBR_HGC or EBR_CGC_ES. */
#define EBR_SECOND_LAYER 16
typedef enum { EBR_F32 = 0, EBR_F64 = 1 } ebr_dtype;
typedef enum { EBR_DIRICHLET = 0, EBR_NEUMANN = 1 } ebr_bc;
typedef enum { EBR_CIRCLE = 0, EBR_SPHERE = 1, EBR_ELLIPSE = 2, EBR_AIRFOIL4 = 3 } ebr_body_kind;

/* Uniform cell-centred grid.  dim = 2 or 3; n[2] = 1, lo[2] = 0, hi[2] = 1 in 2D.
 * Cell widths h_a = (hi_a - lo_a) / n_a; cell centres lo_a + (i_a + 1/2) h_a. */
typedef struct {
  int32_t dim;
  int32_t reserved;
  int64_t n[3];
  double lo[3];
  double hi[3];
} ebr_grid;

/* Analytic convex body.  rot (row-major 3x3) maps body-frame vectors to the
 * world frame: x_world = rot * x_body + centre.
 *   EBR_CIRCLE   (2D): centre, radii[0] = r.
 *   EBR_SPHERE   (3D): centre, radii[0] = r.
 *   EBR_ELLIPSE  (2D): centre, semi-axes radii[0], radii[1] along the body x, y axes, rot.
 *   EBR_AIRFOIL4 (2D): symmetric 4-digit thickness-formula section with an
 *       open trailing edge closed by the base x = chord:
 *       y_t(x) = 5 t c [0.2969 sqrt(x/c) - 0.1260 (x/c) - 0.3516 (x/c)^2
 *                       + 0.2843 (x/c)^3 - 0.1015 (x/c)^4],
 *       body frame with the leading edge at the origin and the chord along +x;
 *       centre = leading edge in the world, thickness = t, chord = c, rot. */
typedef struct {
  int32_t kind;
  int32_t reserved;
  double centre[3];
  double radii[3];
  double rot[9];
  double thickness;
  double chord;
} ebr_body;

/* Per-geometry counts after planning (host copy). */
typedef struct {
  int64_t n_cells;
  int64_t n_interface;   /* cells with a face neighbour on the other side of the boundary */
  int64_t n_ghosts;
  int32_t n_levels;
  int32_t reserved;
} ebr_geom_counts;

/* ---------------------------------------------------------------------------
 * Context
 * ------------------------------------------------------------------------- */

/* Create a context on the current CUDA device.  *out receives the handle. */
ebr_status ebr_create(void** out);
/* Release all library-owned device memory of the context; NULL is ignored. */
void ebr_destroy(void* ctx);
/* Message of the last failing call on ctx ("" if none).  Never NULL. */
const char* ebr_last_error(const void* ctx);

/* ---------------------------------------------------------------------------
 * Step 1: classification and ghost placement (Sec. 3.1, Sec. 7)
 * ------------------------------------------------------------------------- */

/* Plan a geometry set and classify it.
 * n_geom >= 1 geometries; h_grids / h_bodies: host arrays [n_geom] (copied).
 * Cell classification (Sec. 3.1, Eq. signed_distance): a cell is solid
 * (tag 1) when its centre lies in the closed body, else fluid (tag 0).
 * Placement: EBR_CGC -- solid cells with a fluid face neighbour become ghosts
 * (+2); EBR_HGC -- Eqs. delta_n and HGC_criterion give candidates +2 / -2, then
 * a -2 cell without a tag-1 face neighbour becomes 0 and (afterwards) a +2
 * cell without a tag-0 face neighbour becomes 1; EBR_CGC_ES -- the CGC set with
 * the stencil multipliers of Eq. stencil_anisotropic.
 * placement | EBR_SECOND_LAYER (EBR_HGC or EBR_CGC_ES): after the first
 * layer is placed and reclassified, every remaining solid cell with
 * psi <= 1.5 dn (Eq. delta_n, its own normal and widths) becomes a ghost
 * (+2) too, and every ghost takes the multipliers of Eq. stencil_anisotropic
 * (HGC's first layer keeps r = 1).  The interface list then also holds the
 * solid cells within a box reach of a fluid cell (the candidates), and
 * ebr_counts' n_interface counts them.
 * d_tags: caller-owned int8 [total cells] receiving 0, 1, +2, -2.
 * This call synchronises the stream (it sizes the context's buffers) and
 * must come first; later calls reuse the plan until the next ebr_plan. */
ebr_status ebr_plan(void* ctx, int32_t n_geom, const ebr_grid* h_grids,
                    const ebr_body* h_bodies, int32_t placement, int8_t* d_tags,
                    ebr_stream stream);

/* ebr_plan on stretched grids (Sec. 7: the local mesh spacing; the meshes of
 * Secs. 8.1 and 8.2 are stretched away from the body).  h_faces: host array
 * [n_geom] of host pointers; h_faces[b] holds the cell faces of geometry b,
 * n_x + 1 strictly increasing x-faces, then n_y + 1 y-faces (then n_z + 1
 * z-faces), copied; NULL makes that grid uniform (its lo, hi).  For a
 * stretched grid lo and hi are taken from the first and last faces.  Cell
 * centres are the face midpoints, widths the face differences; Eq. delta_n
 * and Eq. stencil_anisotropic use the ghost cell's own widths, the closed
 * forms the stencil's actual x_2 - x_1 (the centre of the cell r_i e_i cells
 * away minus the ghost's), the surface weights the ghost cell's face areas.
 * Everything else as ebr_plan. */
ebr_status ebr_plan_faces(void* ctx, int32_t n_geom, const ebr_grid* h_grids, const double* const* h_faces,
                          const ebr_body* h_bodies, int32_t placement, int8_t* d_tags, ebr_stream stream);

/* Re-run the classification of the planned geometry set without host
 * synchronisation (capturable in a CUDA graph).  Writes d_tags and the
 * context's ghost records; a count that differs from the plan sets EBR_ESHAPE
 * in the device status.  The stream compactions (interface cells of the
 * rows, ghosts of the interface list) count, scan and write in one launch
 * each: a single-pass scan whose blocks wait, bounded (EBR_ETIMEOUT), on the
 * prefixes of blocks already running; its state lives in the context, so two
 * re-runs of one context must not overlap (one stream at a time). */
ebr_status ebr_classify(void* ctx, int8_t* d_tags, ebr_stream stream);

/* Move the bodies of the planned geometry set (Sec. 7: a moving body is
 * classified anew every step): h_bodies [n_geom] (host, copied) replace the
 * bodies of ebr_plan, same kinds and grids; the geometry set is re-planned
 * and classified into d_tags as by ebr_plan, and must be levelled again
 * (ebr_build_levels) before the next fill.  Device buffers are reused: every
 * buffer sized by the counts is grow-only (a buffer that is too small is
 * replaced by one 25 % larger than needed), so a body that moves a little
 * settles into the capacity after a few steps and its steps then allocate
 * nothing (ebr_diagnostics h_out[11] counts allocations).  Synchronises the
 * stream; not inside a stream capture; graphs captured before refer to the
 * old plan and must be captured again.  On an invalid body nothing changes. */
ebr_status ebr_move(void* ctx, const ebr_body* h_bodies, int8_t* d_tags, ebr_stream stream);

/* Flat layout: h_cell_offset [n_geom + 1] (host) receives the cell offsets. */
ebr_status ebr_layout(const void* ctx, int64_t* h_cell_offset);
/* Planned counts: h_counts [n_geom] (host). */
ebr_status ebr_counts(const void* ctx, ebr_geom_counts* h_counts);

/* ---------------------------------------------------------------------------
 * Step 2: dependency DAG and levels (Sec. 3.2)
 * ------------------------------------------------------------------------- */

/* Build the dependency levels of the classified ghosts: ghost G depends on
 * each stencil member P_k that is a ghost with a structurally non-zero weight
 * (n_i != 0 on every axis along which P_k is offset); level(G) = 1 + max level
 * of its dependencies, 1 without any.  Ghosts are then stored in the canonical
 * order (geometry, level, linear index).  Also validates every stencil member
 * (EBR_ESTENCIL_OOB / EBR_ESTENCIL_SOLID) and detects cycles (EBR_ECYCLE),
 * and builds the transposed incidence lists used by the adjoint.  The tags
 * are read from the buffer last given to ebr_plan / ebr_classify; a member
 * tagged +-2 there that is not a ghost of the plan (the buffer was edited)
 * adds no dependency and sets EBR_ESHAPE -- every position the kernels look
 * up through a ghost tag is checked against the plan's ghost records.
 * Device-side failures are reported through the status word.  After the first
 * call the incidence lists are built on a second, library-owned stream that
 * forks from and joins back into `stream` by events inside this call, so the
 * call stays ordered on `stream` (and a stream capture records the two
 * branches as parallel graph nodes). */
ebr_status ebr_build_levels(void* ctx, ebr_stream stream);

/* ebr_classify followed by ebr_build_levels on a planned and levelled
 * context, in one call (the per-step work of a body re-classified every
 * step; capturable).  Same results, bitwise, as the two calls.  For a
 * one-layer EBR_HGC plan the two overlap: the placement kernel (Eqs.
 * delta_n, HGC_criterion) also records the sign and zero pattern of each
 * candidate's normal -- from its float closest point where that is well
 * conditioned (no component within 1e-3 of zero, no near tie of the closest
 * point's branches, no foot point near the evolute), else from the double
 * closest point -- so the ghost records carry their stencil orientation
 * (Sec. 3.1: e_i from the sign of n_i; r_i = 1) before the double closest
 * points (psi, S, n; Eq. signed_distance) are evaluated; those then run on
 * the library's second stream beside the dependency levels and join before
 * the canonical reorder, and check the recorded signs (a difference sets
 * EBR_EINVAL in the device status).  Both reclassification passes are then
 * decided by the ghost compaction from the placement's tags (pass A of a
 * neighbour evaluated where pass B needs it), and the final tags of the
 * interface cells reach d_tags with the ghost positions, inside this call.
 * Other placements run the two steps one after the other.  The call is
 * ordered on `stream` like the two calls. */
ebr_status ebr_classify_levels(void* ctx, int8_t* d_tags, ebr_stream stream);

/* Ghost records in canonical order, copied to host arrays sized by the total
 * ghost count (sum of n_ghosts); any pointer may be NULL to skip it.
 *   h_geom  [Ng] int32 geometry of each ghost,
 *   h_cell  [Ng] int64 linear cell index inside its geometry,
 *   h_level [Ng] int32 dependency level (1-based),
 *   h_tag   [Ng] int8  +2 (centre in the solid) or -2 (centre in the fluid),
 *   h_psi   [Ng] double signed normal distance (Eq. signed_distance),
 *   h_normal[Ng][3] double unit normal at S into the fluid,
 *   h_S     [Ng][3] double boundary point S = centre + psi * normal,
 *   h_r     [Ng][3] int32 stencil multipliers r_i (Eq. stencil_anisotropic).
 * Synchronises the stream. */
ebr_status ebr_ghost_info(void* ctx, int32_t* h_geom, int64_t* h_cell, int32_t* h_level,
                          int8_t* h_tag, double* h_psi, double* h_normal, double* h_S,
                          int32_t* h_r, ebr_stream stream);

/* ---------------------------------------------------------------------------
 * Step 3: level-by-level reconstruction (Secs. 3.2, 4, 5)
 * ------------------------------------------------------------------------- */

typedef enum {
  EBR_MODE_LEVEL_LAUNCH = 0,  /* one grid-wide launch per level per geometry            */
  EBR_MODE_PERSISTENT = 1     /* one launch; one CTA per geometry walks its levels with
                                 block barriers (geometries larger than the CTA's shared
                                 memory fall back to level launches)                    */
} ebr_mode;

/* Fill the ghost entries of n_fields fields in place.
 * d_fields: host array [n_fields] of device pointers, each [total cells] of
 *   dtype (float or double); only ghost entries are written, only stencil
 *   members are read.
 * h_bc_kind: host [n_fields] of ebr_bc.
 * d_bc: host array [n_fields] of device pointers, each [total ghosts] of dtype
 *   in canonical order: phi at S (Dirichlet) or dphi/dn at S (Neumann).
 *   A pointer may be null when the geometry set has no ghost cell.
 * Weights are evaluated in double (Eqs. phi_G_*), once per ghost; FP32 fields
 * are combined in float with the weights rounded to float. */
ebr_status ebr_reconstruct(void* ctx, int32_t n_fields, void* const* d_fields,
                           const int32_t* h_bc_kind, const void* const* d_bc,
                           int32_t dtype, int32_t mode, ebr_stream stream);

/* ---------------------------------------------------------------------------
 * Step 4: boundary quantities and forces (Sec. 6)
 * ------------------------------------------------------------------------- */

/* Per geometry b, d_out[b * (2 dim + 2) + ...] = [Fp (dim), Fv (dim), drag, lift]:
 *   Fp = sum_G w_G (-p_s n),  Fv = sum_G w_G mu (grad u + grad u^T)|_S n,
 *   drag = (Fp + Fv) . h_dirs[0..dim), lift = (Fp + Fv) . h_dirs[dim..2 dim).
 * p_s is the Dirichlet relation solved for phi_s on the filled pressure
 * field; grad u at S from Eq. derivative_bilinear (2D) or
 * Eqs. derivative_trilinear_x/y/z (3D).  w_G = sum over the faces of G shared
 * with a tag-0 cell of (face area) |n_face . n| (the paper gives no quadrature;
 * this local surface-element weight is the reading taken).
 * d_vel: host array [dim] of device pointers to the filled velocity fields
 *   (an entry may be NULL: that component is identically zero); d_p: filled
 *   pressure field; d_out: device double [n_geom * (2 dim + 2)], written.
 * Per ghost the terms are evaluated in the field type (FP32 fields: the
 * coefficients rounded to float, as in the fill); sums over ghosts in double,
 * deterministic (a fixed tree per chunk of 256 ghosts, the chunks of a
 * geometry in order).  The chunk partials and counters are context scratch:
 * two force calls of one context must not overlap (one stream at a time). */
ebr_status ebr_boundary_forces(void* ctx, const void* const* d_vel, const void* d_p,
                               int32_t dtype, double mu, const double* h_dirs,
                               double* d_out, ebr_stream stream);

/* ---------------------------------------------------------------------------
 * Step 5: adjoint (reverse level walk of steps 3-4)
 * ------------------------------------------------------------------------- */

/* Gradient of J = sum_b seed[b][0] drag_b + seed[b][1] lift_b with respect to
 * the fluid field values and the boundary data.  Same field roles as
 * ebr_boundary_forces: fields d_fields[0..n_fields) with kinds h_bc_kind, of
 * which vel_index[0..dim) (-1: component absent) are the velocity components
 * and p_index the pressure.
 * d_seed: device double [n_geom][2].
 * d_grad_fields: host array [n_fields] of device pointers [total cells] of
 *   dtype; entries at stencil cells are written (accumulate = 0: overwritten,
 *   1: added); ghost cells receive 0 (their input value is overwritten by the
 *   fill); all other entries are left untouched.
 * d_grad_bc: host array [n_fields] of device pointers [total ghosts] of dtype
 *   (canonical order), written (or added when accumulate = 1).
 *   A pointer may be null when the geometry set has no ghost cell.
 * The pull form over transposed incidence lists makes the result bitwise
 * deterministic.  The geometry must have been planned and levelled.  The
 * field values themselves are not needed (the map is linear).  When every
 * stencil reaches one cell (HGC, CGC), the search for the fluid targets'
 * sources runs on the context's second stream, forked from and joined back
 * into `stream` by events inside this call (a stream capture records it as
 * a parallel branch); the call's work is complete in `stream` order. */
ebr_status ebr_reconstruct_adjoint(void* ctx, int32_t n_fields, const int32_t* h_bc_kind,
                                   const int32_t* h_vel_index, int32_t p_index, double mu,
                                   const double* h_dirs, const double* d_seed,
                                   void* const* d_grad_fields, void* const* d_grad_bc,
                                   int32_t dtype, int32_t accumulate, int32_t mode,
                                   ebr_stream stream);

/* ---------------------------------------------------------------------------
 * Many fields in the field-minor layout (Sec. 3.2 fill and its transpose)
 *
 * One device array holds all n_fields values of a cell contiguously:
 * element (cell c, field f) at index c * n_fields + f, c the flat cell index of
 * ebr_layout().  This is the layout for a solver that carries many fields per
 * cell (several velocity sets, species, ensemble members): the stencil gather
 * of one ghost then reads n_fields consecutive values per member.
 * 1 <= n_fields <= 1024; h_bc_kind: host int32 [n_fields], EBR_DIRICHLET or
 * EBR_NEUMANN per field.  Same ghost set, levels and weights as
 * ebr_reconstruct (closed forms of Secs. 4-5, one pass per ghost in level
 * order); FP32 fields combine with the weights rounded to float.
 * ------------------------------------------------------------------------- */

/* Fill the ghost entries of d_fields (device, dtype, [total cells][n_fields])
 * in place from the fluid entries and d_bc (device, dtype,
 * [total ghosts][n_fields], canonical ghost order).  Other entries are not
 * written.  A non-finite result sets EBR_ENONFINITE in the status word. */
ebr_status ebr_reconstruct_packed(void* ctx, int32_t n_fields, void* d_fields,
                                  const int32_t* h_bc_kind, const void* d_bc, int32_t dtype,
                                  ebr_stream stream);

/* Transpose of ebr_reconstruct_packed (vector-Jacobian product).
 * d_cot (device, dtype, [total cells][n_fields], in/out): on entry dJ/dy for
 * the filled field y; on exit dJ/dx for the field x before the fill: ghost
 * entries set to 0 (the fill overwrites them), each fluid entry read by a
 * ghost stencil incremented by sum_G w lambda_G, other entries unchanged.
 * d_grad_bc (device, dtype, [total ghosts][n_fields]): written with dJ/d(bc).
 * lambda (dJ/d ghost value, reverse level order) lives in library scratch of
 * total ghosts * n_fields elements, allocated by the first call with a
 * larger n_fields; that call must not be inside a stream capture (it returns
 * EBR_EINVAL there).  Every output element is written by one thread in a
 * fixed summation order: bitwise deterministic, no atomics. */
ebr_status ebr_reconstruct_packed_adjoint(void* ctx, int32_t n_fields, const int32_t* h_bc_kind,
                                          void* d_cot, void* d_grad_bc, int32_t dtype,
                                          ebr_stream stream);

/* ---------------------------------------------------------------------------
 * Tiled fill with a per-level exchange (Sec. 3.2, distributed memory)
 *
 * The grids are cut into rectangular tiles (subdomains) and a ghost belongs
 * to the tile of its cell.  The fill runs as one persistent cooperative
 * launch: each CTA owns tiles; for every level L_k it fills the ghosts of
 * its tiles in L_k, reading fluid values and its own tiles' ghosts from the
 * fields and other tiles' ghosts only from an exchange buffer, writes to that
 * buffer the ghosts of L_k that other tiles' stencils read (only those: the
 * level-wise exchange of Sec. 3.2), and meets all CTAs at a device-wide
 * barrier before L_{k+1}.  Same closed forms and summation order as
 * EBR_MODE_LEVEL_LAUNCH: the results are the same bits.
 * ------------------------------------------------------------------------- */

/* Plan the tiles of the levelled geometry set: h_tile [dim] cells per tile
 * along x, y (, z), each >= 1.  Tile t of cell (i, j, k) of geometry b is
 * tile_offset[b] + i / T_x + n_tx (j / T_y + n_ty (k / T_z)), n_ta = ceil(n_a /
 * T_a), tile offsets accumulated over the geometries in order.  Plans on the
 * host (synchronises the stream; not inside a stream capture) and allocates
 * the schedule and the exchange buffer (released by the next tiled plan,
 * ebr_plan or ebr_destroy).  Plan again after ebr_build_levels re-plans. */
ebr_status ebr_tiled_plan(void* ctx, const int32_t* h_tile, ebr_stream stream);

/* Fill the ghost entries in place, tiled (same arguments and layouts as
 * ebr_reconstruct, 1..8 fields).  Every wait at the device-wide barrier is
 * bounded: a wait that gives up sets EBR_ETIMEOUT in the status word and the
 * launch ends (ghosts of the levels not reached are left unwritten). */
ebr_status ebr_reconstruct_tiled(void* ctx, int32_t n_fields, void* const* d_fields,
                                 const int32_t* h_bc_kind, const void* const* d_bc, int32_t dtype,
                                 ebr_stream stream);

/* Schedule statistics, h_out[0 .. n): [0] tiles owning a ghost, [1] tiles in
 * all, [2] sent ghosts (ghosts read by another tile's stencil), [3] values
 * exchanged ((sent ghost, receiving tile) pairs, all levels), [4] values a
 * conventional halo exchange would send (every sweep, the ghosts within the
 * stencil reach of a face of their tile, one sweep per level), [5] levels,
 * [6] / [7] CTAs of the FP32 / FP64 launch, [8 + k - 1] sent ghosts of level
 * k.  Host values; no synchronisation. */
ebr_status ebr_tiled_info(void* ctx, int64_t* h_out, int32_t n);

/* Per ghost (canonical order), host arrays [total ghosts]: h_tile receives
 * its tile (numbering of ebr_tiled_plan), h_slot its slot in the exchange
 * buffer or -1 when no other tile reads it.  Either pointer may be NULL. */
ebr_status ebr_tiled_lists(void* ctx, int32_t* h_tile, int32_t* h_slot);

/* Failure test of the bounded barrier (the paper has no counterpart): the
 * next ebr_reconstruct_tiled waits at its first barrier for one arrival more
 * than its CTAs provide and gives up after `spins` polls (1 .. 2^24): it
 * reports EBR_ETIMEOUT through ebr_sync_status, and the context stays usable.
 * No GPU fault is involved: the wait is a bounded loop. */
ebr_status ebr_tiled_wait_test(void* ctx, int32_t spins);

/* ---------------------------------------------------------------------------
 * Stability diagnostics (Sec. 7, Eq. stability_alpha_max)
 * ------------------------------------------------------------------------- */

/* For every ghost and axis the normalized distance
 *   alpha_i = (x_s,i - x_1,i) / (x_2,i - x_1,i)
 * (x_1 the ghost centre, x_s its boundary point, x_2 the stencil point r_i e_i
 * cells away; alpha_i < 0 for a ghost centre in the fluid).  Host outputs,
 * any may be NULL:
 *   h_alpha      [n_geom][6]: max alpha_x, y, z, then min alpha_x, y, z of the
 *                geometry's ghosts (0 for absent axes and empty geometries);
 *   h_alpha_hist [3][n_bins]: alpha_i of all ghosts in n_bins bins of equal
 *                width over [-0.5, 1.0) (values outside go to the end bins);
 *   h_level_hist [n_levels]: ghosts in level k at index k - 1 (all geometries);
 *   h_r_hist     [3][16]: count of each stencil multiplier r_i.
 * 1 <= n_bins <= 4096.  The geometry set must be levelled.  Synchronises the
 * stream; counts and extrema do not depend on the schedule. */
ebr_status ebr_stats(void* ctx, double* h_alpha, int64_t* h_alpha_hist, int32_t n_bins, int64_t* h_level_hist,
                     int32_t n_levels, int64_t* h_r_hist, ebr_stream stream);

/* ---------------------------------------------------------------------------
 * Status
 * ------------------------------------------------------------------------- */

/* Synchronise the stream, read and clear the device status word. */
ebr_status ebr_sync_status(void* ctx, ebr_stream stream);

/* Diagnostics (synchronises the stream): h_out[0] = x-rows whose solid run
 * the 4-cell windows could not confirm, so that the whole row was swept with
 * the exact predicate, accumulated since ebr_plan; h_out[1] = largest stencil
 * multiplier r_i; h_out[2] = kernel launches so far; h_out[3] = entries of
 * the ghost-target source lists of the adjoint (after ebr_build_levels);
 * h_out[4..10] = schedule of the field-minor kernels (0 before their first
 * call): last grid-wide level of the fill and of its transpose, geometries
 * with a level tail in each, largest tail of each (ghosts), fluid targets;
 * h_out[11] = device allocations the context has made so far.
 * n = entries wanted. */
ebr_status ebr_diagnostics(void* ctx, int64_t* h_out, int32_t n, ebr_stream stream);

/* Number of kernel launches this context has issued since creation. */
int64_t ebr_launch_count(const void* ctx);

/* Programmatic dependent launch (process-wide; on by default).  enable != 0:
 * kernels of the library are launched with the programmatic stream
 * serialization attribute, so that a kernel's blocks may be scheduled while
 * the kernel before it in the stream is still running; each of them waits
 * (griddepcontrol.wait) for the preceding kernels to complete before it
 * touches memory, so results and stream order are unchanged.  Inside a stream
 * capture such launches become programmatic edges of the graph.  enable = 0:
 * plain launches.  A launch reads the switch when it is issued, so a graph
 * captured earlier keeps the mode it was captured with.  Not synchronised
 * with launches issued concurrently from other host threads. */
void ebr_set_pdl(int32_t enable);
/* Current switch: 1 on, 0 off. */
int32_t ebr_get_pdl(void);

/* ---------------------------------------------------------------------------
 * Launch shapes (tuning; the paper has no counterpart)
 *
 * Threads per block of the kernels that run one thread per item (interface
 * cell, ghost, fluid target): "iface", "place", "ghost_geom" (the per-ghost
 * closest-point kernel), "deps", "tables", "gsrc", "fill_part"
 * (the partial sums of the persistent fill), "adj_seed", "adj_part" (the
 * start values and incidence records of the persistent adjoint chain),
 * "adj_probe" (the fluid targets' sources at reach 1, found beside the
 * chain), "adj_fluid", "adj_bc" -- the names under which ebr_profile_read
 * reports them.  The block size changes scheduling only: every result is bitwise the
 * same for every allowed value.  A launch reads the context's value when it
 * is issued, so a graph captured earlier keeps the shapes it was captured
 * with.  "iface" and "gsrc" shape the planning pass (ebr_plan,
 * ebr_build_levels after a plan); a re-run (ebr_classify, ebr_build_levels on
 * a levelled context) counts, scans and writes in one launch of 256 threads
 * per block.  The Python autotuner (paper_2609_10165_b300/autotune.py) times
 * the candidates with ebr_profile and sets the fastest.
 * ------------------------------------------------------------------------- */

/* Number of tunable kernels; writes up to max_entries names into h_names
 * [max_entries][32] (NUL-terminated) when h_names is not NULL. */
int32_t ebr_tunable_kernels(char* h_names, int32_t max_entries);
/* Set the threads per block of one tunable kernel of this context: a
 * multiple of 32 in 32..256 (default 128).  EBR_EINVAL for an unknown name
 * or value (the old value stays). */
ebr_status ebr_set_block_size(void* ctx, const char* kernel, int32_t threads);
/* Current threads per block of a tunable kernel, or EBR_EINVAL (negative)
 * for an unknown name. */
int32_t ebr_get_block_size(const void* ctx, const char* kernel);

/* ---------------------------------------------------------------------------
 * Timing (diagnostics; the paper has no counterpart)
 * ------------------------------------------------------------------------- */

/* enable != 0: from now on every kernel launch of the context is bracketed by
 * two CUDA events recorded on the launching stream (adds a small gap between
 * kernels).  Inside a stream capture the events become event-record nodes of
 * the graph and are re-recorded at every replay.  Clears earlier records.
 * enable = 0 stops adding records (existing ones stay readable). */
ebr_status ebr_profile(void* ctx, int32_t enable);
/* Synchronise the recorded events and aggregate them by kernel name:
 * h_names [max_entries][32] (NUL-terminated), h_ms [max_entries] total
 * milliseconds, h_count [max_entries] launches.  Returns the number of
 * distinct names (may exceed max_entries) or a negative ebr_status.  keep = 0
 * clears the records; keep != 0 keeps them (to read a replayed graph again).
 * Any output pointer may be NULL. */
int32_t ebr_profile_read(void* ctx, int32_t max_entries, char* h_names, double* h_ms,
                         int64_t* h_count, int32_t keep);
/* The records one by one, in the order they were issued (launches on
 * several streams interleave): name, start and end in milliseconds after the
 * start of the first record (a launch on another stream may start earlier:
 * negative).  Synchronises the events; keeps the records.  Returns the
 * number of records (may exceed max_entries) or a negative ebr_status. */
int32_t ebr_profile_timeline(void* ctx, int32_t max_entries, char* h_names, double* h_start_ms,
                             double* h_end_ms);

/* ---------------------------------------------------------------------------
 * Allocation-free classification of one grid (the paper has no counterpart)
 * ------------------------------------------------------------------------- */

/* Largest n_y * n_z (number of x-rows) ebr_classify_cells_static accepts. */
#define EBR_STATIC_MAX_ROWS (1 << 18)

/* Fluid / solid tags of ONE grid against ONE body, for callers that cannot let
 * the library allocate device memory: programs that own every device byte
 * through their own pool or a fixed memory budget, and code that must not
 * call cudaMalloc while other work runs, because cudaMalloc may synchronise
 * the device.  Nothing is allocated and no context is needed.
 *   d_tags         caller-owned int8 [n_x n_y n_z], receives 0 (fluid) / 1
 *                  (solid, centre in the closed body) -- the tags before
 *                  ghost placement; same layout as the other calls.
 *   d_n_interface  caller-owned device int64, receives the number of cells
 *                  with a face neighbour on the other side of the boundary,
 *                  or, when the device recorded a failure (a row whose solid
 *                  run the row kernel could not determine, left all fluid),
 *                  that negative ebr_status instead of the count.  The host
 *                  checks on the body make that failure unreachable for the
 *                  bodies of this header; the value is the only channel by
 *                  which a device-side failure of this call is reported.
 * The per-row solid runs needed between the two kernels live in a fixed
 * device array inside the library (EBR_STATIC_MAX_ROWS rows, 2 MiB, held by
 * every device that loads the library until the process exits).  Grids with
 * more rows are rejected with EBR_EINVAL before any GPU work, as are invalid
 * grids or bodies (no message: there is no context).  Every call looks the
 * array's device address up in the current context (cudaGetSymbolAddress);
 * the first call in a context may load the library's device code, so make
 * it before any stream capture.  All calls share the array and it keeps the
 * last call's contents: the call clears what must start at zero itself, and
 * calls that overlap on the GPU (other streams, other threads) race on it.
 * Asynchronous on the stream. */
ebr_status ebr_classify_cells_static(const ebr_grid* h_grid, const ebr_body* h_body,
                                     int8_t* d_tags, int64_t* d_n_interface, ebr_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* EBR_H */

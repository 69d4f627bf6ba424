/*
 * gs103.h -- C ABI of the GB300 (sm_103a) 3D Gaussian Splatting training hot path.
 *
 * Method: BalanceGS (arXiv 2510.14564).  Sec. II-A of the paper defines what is
 * computed: a Gaussian's influence G(x) = exp(-1/2 (x-mu)^T Sigma^-1 (x-mu)),
 * its screen covariance Sigma' = J W Sigma W^T J^T, and front-to-back
 * blending C = sum_i c_i alpha_i prod_{j<i} (1 - alpha_j) over the Gaussians
 * of a pixel sorted by depth, rendered in 16x16 pixel blocks (Sec. IV-C1).
 * Readings the paper leaves to the 3DGS renderer it builds on: Sigma' gets a
 * +0.3 I dilation; a Gaussian covers the tiles of its 3-sigma square
 * (radius ceil(3 sqrt(lambda_max))); alpha = min(0.99, o G); alpha < 1/255 is
 * skipped; a pixel stops before the Gaussian that would take its
 * transmittance below 1e-4; colour = max(0, 0.5 + sum_lm Y_lm(d) k_lm) with
 * real degree-3 SH and d the unit vector from the camera centre to mu.
 *
 * Conventions shared by every call:
 *   - Pointers named d_* (and every array argument unless stated) are DEVICE
 *     pointers owned by the caller; the library never allocates or frees.
 *     Host arrays are marked "host".
 *   - Every call is asynchronous on the given CUDA stream (0 = legacy default
 *     stream) and returns a gs_status for host-side argument checks and launch
 *     errors.  Errors found by kernels are OR-ed as GS_EW_* bits into the
 *     caller's device word *err_word (read it after the stream synchronises).
 *   - A batch holds n_views cameras (host array); Gaussians are per view,
 *     view-major: record v*N + i belongs to view v, Gaussian i.
 *   - Tiles are 16x16 pixels; view v has TX_v = ceil(W/16) x TY_v = ceil(H/16)
 *     tiles, numbered row-major, and the batch numbers its tiles globally as
 *     tile_base_v + ty*TX_v + tx (tile_base = running sum over earlier views).
 *   - Pixels: view v's image occupies [3, H_v, W_v] floats (planar RGB) at float
 *     offset 3*pix_base_v, pix_base_v = running sum of W*H over earlier views;
 *     per-pixel maps (T_final, n_proc) use offset pix_base_v.
 *   - Parameters of N Gaussians sit in one grouped FP32 buffer of 59 N floats:
 *     [means 3N | log_scales 3N | quats 4N (w,x,y,z) | opacity_logits N |
 *      sh 48N ([N,16,3], coefficient-major, RGB innermost)].  Gradients and
 *     Adam moments use the same layout.
 */
#ifndef GS103_H
#define GS103_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *gs_stream_t; /* = cudaStream_t */

#define GS_TILE 16
#define GS_MAX_VIEWS 64
#define GS_PARAM_FLOATS 59

typedef enum {
    GS_OK = 0,
    GS_ERR_ARG = 1,       /* null / misaligned pointer, bad size or dtype */
    GS_ERR_CAPACITY = 2,  /* an output buffer is too small; see the call */
    GS_ERR_CUDA = 3,      /* a CUDA launch or copy failed */
    GS_ERR_TIMEOUT = 4,   /* a persistent kernel ran out of its time budget */
    GS_ERR_NONFINITE = 5  /* non-finite input (host-detected) */
} gs_status;

/* Bits OR-ed into *err_word by kernels. */
#define GS_EW_NONFINITE 0x1u /* a Gaussian had a non-finite parameter; it was culled */
#define GS_EW_CAPACITY 0x2u  /* instance count exceeded the capacity given */
#define GS_EW_TIMEOUT 0x4u   /* a persistent render kernel exceeded its budget */
#define GS_EW_BOUNDS 0x8u    /* an index check failed; the access was skipped */

typedef enum { GS_F32 = 0, GS_BF16 = 1, GS_F16 = 2 } gs_dtype;

/* Pinhole camera.  world -> camera: p_cam = R p + t (R row-major); the camera
 * looks along +z_cam; pixel (px, py) has its centre at (px + 0.5, py + 0.5);
 * u = fx x/z + cx, v = fy y/z + cy.  Gaussians with z <= znear are culled.
 * campos = -R^T t (the SH view direction origin); bg is added as T_final*bg. */
typedef struct {
    int W, H;
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
    float campos[3];
    float znear;
    float bg[3];
} gs_camera;

/* Screen-space splat record written by gs_project and read by the renderer.
 * Geometry is FP32; the conic and opacity are stored pre-scaled for exp2:
 *   e = lo + Ap dx^2 + Bp dx dy + Cp dy^2,  alpha = min(0.99, 2^e)
 * with Ap = -A/2 log2(e), Bp = -B log2(e), Cp = -C/2 log2(e), lo = log2(o),
 * (A, B; B, C) = Sigma'^-1, d = pixel centre - (u, v).
 * GS_F32 colour: record of 48 bytes  {u, v, Ap, Bp}, {Cp, lo, r, g}, {b, 0, 0, 0}.
 * GS_BF16 / GS_F16 colour: 32 bytes  {u, v, Ap, Bp}, {Cp, lo, rg, b0} where rg
 * packs r (low half) and g (high half), b0 packs b (low half). */
#define GS_SPLAT_BYTES_F32 48
#define GS_SPLAT_BYTES_HALF 32

/* ------------------------------------------------------------------------ */

/* Library version, and a human-readable message for a gs_status. */
int gs_version(void);
const char *gs_strerror(int status);

/* Number of CUDA kernels this library has launched in the process so far
 * (a host-side counter; thread-safe). */
long long gs_launch_count(void);

/* Zero n_bytes at d_ptr on the stream (a memset, not a kernel launch): the
 * accumulating outputs (gs_render_bwd's d_grad2d, gs_render_fwd's
 * d_flag_count, gs_rank_judge's d_out, gs_grad2d_norm's d_out) start from
 * zero.  d_ptr NULL with n_bytes > 0: GS_ERR_ARG. */
int gs_zero(void *d_ptr, size_t n_bytes, gs_stream_t stream);

/* Bounded device waits (no paper counterpart: a property of this library).
 * The depth sort inside gs_bin_sort, gs_bin_sort_noalloc and
 * gs_bin_sort_prefix is a onesweep radix sort: each 4096-key tile of a digit
 * pass reads the digit counts of earlier tiles from status words those tiles
 * publish (decoupled look-back).  A tile makes at most `reads` rounds of
 * status-word reads (each round reads the words of four earlier tiles at
 * once) per digit; past that it gives up, sets GS_EW_TIMEOUT in *err_word
 * and goes on with the counts it has.  The call then completes with an
 * unspecified instance order, but every buffer it leaves still holds record
 * indices in [0, V*N) (the sort's last pass rewrites its outputs as an
 * identity when any look-back gave up), and the counts the lists are placed
 * by are taken from that same order, so no later kernel reads or writes out
 * of bounds.  A healthy look-back makes a few hundred rounds at most; 0
 * makes every tile but the first give up at once (how the tests reach this
 * path without a stuck GPU).  The limit is process-wide and applies to calls
 * made after gs_set_wait_limit returns; reads < 0 returns GS_ERR_ARG.
 * gs_get_wait_limit returns the limit in force. */
#define GS_WAIT_LIMIT_DEFAULT (1LL << 20)
int gs_set_wait_limit(long long reads);
long long gs_get_wait_limit(void);

/* a1. Projection and SH colour (Sec. II-A projection equation).
 * In:  N Gaussians' parameters (grouped layout above; d_sh may instead be a
 *      separate [N,16,3] array of dtype sh_dtype = GS_F32, GS_BF16 or GS_F16).
 * Out, per (view, Gaussian), V*N entries each:
 *   d_splats  records of colour dtype rgb_dtype (size above, 16-B aligned)
 *   d_depth   camera-space z (FP32), the sort key
 *   d_rect    int16 [V*N, 4] tile rectangle (xmin, ymin, xmax, ymax), local to the view
 *   d_touched int32 tiles covered = (xmax-xmin)(ymax-ymin); 0 = culled
 *   d_radius  int32 radius in pixels (may be NULL)
 * Depth, radius, rectangle and culling are computed in FP32 with IEEE-rounded
 * + - * / sqrt in a fixed order (no FMA contraction), so they are reproducible
 * bit for bit by any IEEE implementation of the same order.
 * d_quats, d_sh and d_splats must be 16-byte aligned and d_rect 8-byte
 * aligned (in the grouped layout: N a multiple of 4), else GS_ERR_ARG.
 * d_sh may be NULL: no SH is read and every record's colour is zero, to be
 * filled in by gs_colour_records for the records the tile lists reference.
 * Non-finite parameters cull the Gaussian and set GS_EW_NONFINITE. */
int gs_project(const gs_camera *cams, int n_views, int N, const float *d_means,
               const float *d_log_scales, const float *d_quats, const float *d_opacity_logits,
               const void *d_sh, int sh_dtype, void *d_splats, int rgb_dtype, float *d_depth,
               int16_t *d_rect, int32_t *d_touched, int32_t *d_radius, int *d_err_word,
               gs_stream_t stream);

/* a1, deferred colour: only the records the tile lists reference are ever
 * read by the blend loops, so after gs_project with d_sh NULL their colours
 * alone are computed, as gs_project computes them (the same code, the same
 * bits), and written into their splat records (the other fields untouched).
 * gs_colour_records colours each record d_list[0, *d_count) (device uint32
 * count; record indices v*N+i, those at or above V*N ignored): the list
 * gs_bin_sort_prefix leaves (d_colour_list, the records its kept lists
 * reference, each once, marked colour_epoch in d_colour_mark).
 * gs_colour_repaired colours, after a repair, the records of the lists of
 * the *d_n_tiles tiles d_tiles[] (as gs_render_fwd lists the tiles to
 * repair; ranges from d_tile_ranges, entries clamped to capacity) whose mark
 * in d_mark (V*N uint32) is not yet epoch, marking them epoch (one atomic
 * exchange each: each is coloured once); with no tile it returns at once.
 * d_sh / d_splats not 16-byte or d_tile_ranges not 8-byte aligned, or a
 * NULL pointer: GS_ERR_ARG. */
int gs_colour_records(const gs_camera *cams, int n_views, int N, const float *d_means,
                      const void *d_sh, int sh_dtype, const uint32_t *d_list, const uint32_t *d_count,
                      void *d_splats, int rgb_dtype, gs_stream_t stream);
int gs_colour_repaired(const gs_camera *cams, int n_views, int N, const float *d_means,
                       const void *d_sh, int sh_dtype, const uint32_t *d_vals, long long capacity,
                       const int32_t *d_tiles, const int32_t *d_n_tiles, const uint32_t *d_tile_ranges,
                       uint32_t *d_mark, uint32_t epoch, void *d_splats, int rgb_dtype,
                       gs_stream_t stream);

/* a2. Tile binning and the (tile, depth) sort.
 * gs_bin_sort_workspace gives the scratch bytes gs_bin_sort needs for V*N
 * Gaussians, an instance capacity and T total tiles.
 * gs_bin_sort emits one instance per (Gaussian, covered tile) and sorts them
 * by the 64-bit key (global tile id << 32 | FP32 depth bits), ties by
 * record index (v*N + i); the order is exactly that of a stable sort of that
 * key over index-ordered input.
 * In: d_depth, d_rect, d_touched as gs_project writes them: a record with
 * d_touched > 0 covers its rectangle's (xmax-xmin)(ymax-ymin) tiles, a
 * culled record (d_touched <= 0) has an empty rectangle.
 * Out: d_vals [capacity] u32 record index per sorted instance;
 *      d_tile_ranges [T, 2] u32 [start, end) into d_vals per global tile
 *                    (an empty tile reads [0, 0));
 *      d_keys [capacity] u64 (optional, NULL = not written) the sorted keys;
 *      d_n_instances (device, 1 x int64) the instance count.
 * If the count exceeds capacity, nothing past the capacity is written,
 * GS_EW_CAPACITY is set and *d_n_instances still holds the count needed.
 * d_workspace must be 256-byte aligned. */
int gs_bin_sort_workspace(int n_views, int N, long long capacity, const gs_camera *cams,
                          size_t *bytes);
int gs_bin_sort(const gs_camera *cams, int n_views, int N, const float *d_depth,
                const int16_t *d_rect, const int32_t *d_touched, long long capacity,
                uint32_t *d_vals, uint32_t *d_tile_ranges, uint64_t *d_keys,
                long long *d_n_instances, void *d_workspace, size_t workspace_bytes,
                int *d_err_word, gs_stream_t stream);

/* a2 for rendering: the same stable (tile, depth) lists, each cut to an exact
 * prefix that blending never runs past.  A splat whose opacity at every
 * pixel of a tile is at least a = min(0.99, 0.99 o / e) (over the tiles of a
 * core rectangle inside its ellipse Q <= 2) is blended by each pixel that has
 * not stopped and multiplies its transmittance by at most 1 - a.  A tile
 * keeps its list up to the depth-ordered chunk where the sum of -ln(1 - a)
 * over its entries first exceeds 10 > ln(1e4) (fixed point, rounded down):
 * past that point every pixel of the tile has stopped, so rendering with the
 * prefix gives the images, T_final, processed counts and gradients of the
 * full list.  Tiles that never reach the bound keep their whole list.
 * Inputs as gs_bin_sort plus the splat records of gs_project (d_splats,
 * rgb_dtype).  Out: d_vals and d_tile_ranges of the prefixes (an empty tile
 * reads [0, 0)); d_tile_count [T] u32 the full list lengths (optional);
 * d_keys the prefix keys (optional); *d_n_instances the entries kept.
 * d_tile_limit (optional, [T] int32, e.g. the d_tile_nproc of the previous
 * step) replaces the bound: a tile with limit > 0 keeps the chunks up to the
 * one holding entry 2 limit + 64 (a tile with limit <= 0 keeps its whole
 * list).  Such a cut is not guaranteed, so gs_render_fwd checks it
 * (d_tile_count) and gs_bin_sort_prefix_repair rebuilds the tiles it lists.
 * d_colour_list (optional, V*N uint32): the records the lists reference,
 * each once, in no fixed order, *d_colour_count (uint32, zeroed by the call)
 * of them, each marked colour_epoch in d_colour_mark (V*N uint32; both
 * needed with the list) -- the input of gs_colour_records; refused
 * (GS_ERR_ARG) for views that get the full lists.
 * Overflow and workspace rules as gs_bin_sort.  Views of more than 16384
 * tiles get the full lists. */
int gs_bin_sort_prefix_workspace(int n_views, int N, long long capacity, const gs_camera *cams,
                                 size_t *bytes);
int gs_bin_sort_prefix(const gs_camera *cams, int n_views, int N, const float *d_depth,
                       const int16_t *d_rect, const int32_t *d_touched, const void *d_splats,
                       int rgb_dtype, const int32_t *d_tile_limit, long long capacity,
                       uint32_t *d_vals, uint32_t *d_tile_ranges, uint32_t *d_tile_count,
                       uint64_t *d_keys, long long *d_n_instances, uint32_t *d_colour_list,
                       uint32_t *d_colour_count, uint32_t *d_colour_mark, uint32_t colour_epoch,
                       void *d_workspace, size_t workspace_bytes, int *d_err_word, gs_stream_t stream);

/* Rebuild the full lists of the *d_flag_count tiles in d_flag_tiles (as
 * listed by gs_render_fwd) after the kept entries (*d_n_instances of them),
 * within the capacity, and point their ranges there; the workspace is the
 * one the preceding gs_bin_sort_prefix call used.  Tiles that do not fit set
 * GS_EW_CAPACITY and keep their prefix.  Does nothing when the count is 0. */
int gs_bin_sort_prefix_repair(const gs_camera *cams, int n_views, int N, const int16_t *d_rect,
                              const int32_t *d_touched, const int32_t *d_flag_tiles,
                              const int32_t *d_flag_count, long long capacity, uint32_t *d_vals,
                              uint32_t *d_tile_ranges, const long long *d_n_instances,
                              void *d_workspace, size_t workspace_bytes, int *d_err_word,
                              gs_stream_t stream);

/* gs_bin_sort without a workspace argument: no counterpart in the paper.
 * For callers that cannot allocate device memory themselves (a runtime that
 * owns all device memory through its own pool, a steady-state loop that must
 * not call cudaMalloc/cudaFree because they can synchronise the device, an
 * embedding handed only its inputs and outputs).  The call allocates nothing:
 * its scratch is a file-scope device array of GS_NOALLOC_SCRATCH_BYTES that
 * every GPU loading this library holds until the process exits.  The caller
 * still passes every input and output, with the meaning gs_bin_sort gives
 * them.  A problem whose gs_bin_sort_workspace exceeds that size is rejected
 * with GS_ERR_CAPACITY before any work is queued.  The first call on a device
 * looks up the array's device address on the current device (once per
 * device); make that first call before any stream capture.  All calls share
 * the one array, which keeps the previous call's contents (the call clears
 * what it needs zeroed), so calls that overlap on the GPU (other streams,
 * other host threads) race on it and must be serialised by the caller. */
#define GS_NOALLOC_SCRATCH_BYTES (32u << 20)
#define GS_NOALLOC_MAX_DEVICES 64
int gs_bin_sort_noalloc(const gs_camera *cams, int n_views, int N, const float *d_depth,
                        const int16_t *d_rect, const int32_t *d_touched, long long capacity,
                        uint32_t *d_vals, uint32_t *d_tile_ranges, uint64_t *d_keys,
                        long long *d_n_instances, int *d_err_word, gs_stream_t stream);

/* Work schedule for the render kernels (a8).  mode GS_SCHED_RASTER: one CTA
 * per tile in tile order.  GS_SCHED_ORDER: persistent CTAs take tiles from
 * d_order (a permutation of the T global tiles) through an atomic queue
 * (d_queue: one device int, zeroed by the call); the image does not depend
 * on the order.  budget_ns > 0 bounds a CTA's time: a CTA past it takes no
 * new tile and sets GS_EW_TIMEOUT (unrendered tiles are then left as they
 * were). */
#define GS_SCHED_RASTER 0
#define GS_SCHED_ORDER 1
typedef struct {
    int mode;
    const int32_t *d_order;
    int *d_queue;
    long long budget_ns;
    const int32_t *d_n_order;  /* device count of tiles in d_order; NULL = all T tiles */
    int32_t *d_split;          /* gs_render_bwd only: one device int of scratch; non-NULL lets the
                                  heaviest head-of-order tiles be taken in four strips (images and
                                  gradients are unchanged up to the order of additions) */
    uint64_t *d_tile_ns;       /* gs_render_bwd only: [T] u64; each tile's nanoseconds are ADDED
                                  (the strips of a split tile add up; the caller zeroes it);
                                  NULL = not measured.  gs_render_fwd takes its own d_tile_ns. */
    const float *d_split_cost; /* gs_render_bwd with d_split only: [T] predicted log costs (e.g. the
                                  cost MLP's); the heavy tiles counted for splitting are then those
                                  whose exp(cost) exceeds a CTA's mean share of the total, instead of
                                  those whose processed count does.  NULL = processed counts */
} gs_schedule;

/* a3. Forward blending (Sec. II-A blending equation), one CTA per 16x16 tile.
 * Out: d_img [3, H, W] per view; d_T_final per pixel (transmittance left);
 *      d_n_proc per pixel: entries of the tile list processed up to and
 *      including the last Gaussian blended (0 if none);
 *      d_tile_nproc [T] the maximum of d_n_proc over the tile;
 *      d_tile_ns [T] u64 nanoseconds the tile took (NULL = not measured).
 * With d_tile_count (the full list lengths of gs_bin_sort_prefix), a tile
 * whose kept prefix ended while a pixel was still blending is appended to
 * d_flag_tiles and counted in *d_flag_count (zeroed by the caller); its
 * outputs are then incomplete until gs_bin_sort_prefix_repair and a render
 * of the listed tiles (GS_SCHED_ORDER over d_flag_tiles, d_n_order =
 * d_flag_count).  NULL = no check.  sched may be NULL (raster). */
int gs_render_fwd(const gs_camera *cams, int n_views, const uint32_t *d_tile_ranges,
                  const uint32_t *d_vals, const void *d_splats, int rgb_dtype,
                  const gs_schedule *sched, float *d_img, float *d_T_final, int32_t *d_n_proc,
                  int32_t *d_tile_nproc, uint64_t *d_tile_ns, const uint32_t *d_tile_count,
                  int32_t *d_flag_tiles, int32_t *d_flag_count, int *d_err_word,
                  gs_stream_t stream);

/* a3, colour-layout ablation (Sec. V: batch loading, reordering into
 * per-Gaussian RGB, coalesced access).  Not on the training path: it
 * measures what the layout of the colour costs the forward pass.
 *
 * gs_colour_arrays copies the colour of VN FP32 splat records (GS_F32
 * records from gs_project) into d_planar [3, VN] (all R, then all G, then
 * all B) and/or d_interleaved [VN, 3] (R G B per Gaussian); either may be
 * NULL.
 *
 * gs_render_fwd_colour is gs_render_fwd with FP32 records and one CTA per
 * tile in raster order, except that the colour of each list entry is read
 * from d_colour (laid out as the layout says) instead of from the record:
 *   GS_COLOUR_PLANAR_GLOBAL       planar, read in the blend loop by every
 *                                 pixel that blends the Gaussian;
 *   GS_COLOUR_INTERLEAVED_GLOBAL  interleaved, read the same way;
 *   GS_COLOUR_PLANAR_STAGED       planar, loaded into shared memory with the
 *                                 batch's geometry;
 *   GS_COLOUR_INTERLEAVED_STAGED  interleaved, loaded the same way.
 * Writes d_img, d_T_final and d_n_proc as gs_render_fwd does, equal bit for
 * bit for every layout (and to gs_render_fwd on the same records).  Full
 * lists, or kept prefixes none of whose pixels ran out (the ablation does
 * not flag tiles). */
#define GS_COLOUR_PLANAR_GLOBAL 0
#define GS_COLOUR_INTERLEAVED_GLOBAL 1
#define GS_COLOUR_PLANAR_STAGED 2
#define GS_COLOUR_INTERLEAVED_STAGED 3
int gs_colour_arrays(long long VN, const void *d_splats_f32, float *d_planar, float *d_interleaved,
                     gs_stream_t stream);
int gs_render_fwd_colour(const gs_camera *cams, int n_views, int N, const uint32_t *d_tile_ranges,
                         const uint32_t *d_vals, const void *d_splats_f32, int layout,
                         const float *d_colour, float *d_img, float *d_T_final, int32_t *d_n_proc,
                         gs_stream_t stream);

/* a4. L1 loss over n floats: *d_loss (device float, overwritten)
 * = mean |img - tgt|; d_dimg = sign(img - tgt)/n with sign(0) = 0. */
int gs_l1_loss(long long n, const float *d_img, const float *d_tgt, float *d_loss,
               float *d_dimg, gs_stream_t stream);

/* a5. Reverse mode of the blending.  Walks each pixel's list back to front
 * from d_n_proc, recovering the transmittance in front of each Gaussian as
 * T <- T / (1 - alpha) from T_final (nothing per Gaussian is stored).
 * Accumulates (adds) into d_grad2d [V*N, 12] FP32 per record: dL/d(u, v, A,
 * B, C, opacity, r, g, b) in entries 0..8 (A, B, C the conic entries, power =
 * -1/2 (A dx^2 + C dy^2) - B dx dy); entries 9..11 are padding.  The caller
 * zeroes d_grad2d before the first accumulation. */
int gs_render_bwd(const gs_camera *cams, int n_views, const uint32_t *d_tile_ranges,
                  const uint32_t *d_vals, const void *d_splats, int rgb_dtype,
                  const gs_schedule *sched, const float *d_dimg, const float *d_T_final,
                  const int32_t *d_n_proc, const int32_t *d_tile_nproc, float *d_grad2d,
                  int *d_err_word, gs_stream_t stream);

/* a6. Chain d_grad2d through the projection to the 59 parameters of each
 * Gaussian, summed over views, WRITTEN (not added) into d_dparams (grouped
 * layout, 16-byte aligned; N must be a multiple of 4 so that every group
 * stays 16-byte aligned).  Same parameter inputs as gs_project. */
int gs_project_bwd(const gs_camera *cams, int n_views, int N, const float *d_means,
                   const float *d_log_scales, const float *d_quats,
                   const float *d_opacity_logits, const void *d_sh, int sh_dtype,
                   const int32_t *d_touched, const float *d_grad2d, float *d_dparams,
                   gs_stream_t stream);

/* a6 + a7 fused: the projection backward of gs_project_bwd followed, for
 * each Gaussian, by the Adam step of gs_adam_step on its 59 entries, without
 * writing the gradients (unless d_dparams != NULL).  d_params is the grouped
 * FP32 buffer (read for the backward, then updated); d_sh is the SH the
 * forward read (e.g. the BF16 shadow; NULL = the SH group of d_params, FP32);
 * the updated SH is also written to d_sh_shadow if given.  N must be a
 * multiple of 4.  d_sh and d_sh_shadow may be the same buffer (the shadow
 * refreshed in place): each Gaussian's coefficients are read before its
 * update is written.  Gradients and updates equal those of the two calls (up
 * to the last bit of the SH basis, evaluated by two code paths).  With one
 * view d_grad2d is consumed and left all zero: a nonzero record serves as
 * scratch (its entries 0..5 hold the factors of its SH gradient) and is
 * zeroed after use, a zero record is neither used nor written, so a caller
 * that zeroed the records before gs_render_bwd need not zero them again for
 * the next step; with several views d_grad2d is only read. */
int gs_project_bwd_adam(const gs_camera *cams, int n_views, int N, float *d_params,
                        const void *d_sh, int sh_dtype, const int32_t *d_touched,
                        float *d_grad2d, float *d_m, float *d_v, const float *lr, float b1,
                        float b2, float eps, int t, void *d_sh_shadow, int shadow_dtype,
                        float *d_dparams, gs_stream_t stream);

/* a7. One bias-corrected Adam step (Kingma & Ba) over the grouped buffers of
 * N Gaussians (59 N floats each, 16-B aligned), step t >= 1:
 *   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 *   p -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)
 * lr (host, 6 floats) per group: means, log_scales, quats, logits, SH DC
 * (coefficient 0), SH rest.  If d_sh_shadow != NULL, the updated SH group is
 * also written there as [N,16,3] in shadow_dtype (GS_BF16 or GS_F16). */
int gs_adam_step(int N, float *d_params, const float *d_grads, float *d_m, float *d_v,
                 const float *lr, float b1, float b2, float eps, int t, void *d_sh_shadow,
                 int shadow_dtype, gs_stream_t stream);

/* Plain Adam over n floats with one learning rate (used for the MLP). */
int gs_adam_flat(long long n, float *d_p, const float *d_g, float *d_m, float *d_v, float lr,
                 float b1, float b2, float eps, int t, gs_stream_t stream);

/* a9. Dynamic training: one clone-and-prune step between training steps, the
 * plain form of the adaptive density control of 3DGS training (Sec. II-A:
 * Gaussians are cloned where reconstruction is poor and pruned where they
 * contribute nothing).
 *
 * gs_grad2d_norm ADDS to d_out[i] (N floats, zeroed by the caller before the
 * first step it covers) the screen-space gradient norm of Gaussian i summed
 * over views, sum_v |(dL/du, dL/dv)|, read from entries 0 and 1 of the
 * records of d_grad2d [V*N, 12] (view v, Gaussian i at record v*N + i) as
 * gs_render_bwd leaves them.  Call it before gs_project_bwd_adam, which
 * consumes d_grad2d for one view.
 *
 * gs_densify: from N Gaussians (grouped layout, 59 N floats; Adam moments
 * d_m, d_v the same) and a per-Gaussian gradient statistic d_grad_norm:
 *   - Gaussian i is kept iff its opacity logit >= logit_threshold (the logit
 *     of the minimum opacity, compared in FP32);
 *   - the kept ones are ranked by d_grad_norm descending, ties by index
 *     (values <= 0 and NaN rank as 0), and the first c = min(n_clone, kept)
 *     are cloned;
 *   - the new count n2 is a multiple of 4 (every group stays 16-byte
 *     aligned): the last (kept + c) mod 4 clones are dropped when there are
 *     that many, else copies of the first kept Gaussian with logit -30
 *     (opacity ~1e-13, invisible) pad the count;
 *   - output, in the grouped layout of n2 (59 n2 floats) in d_params_out,
 *     d_m_out, d_v_out: the kept Gaussians in index order, the clones in rank
 *     order, the pads; clones and pads start with zero moments.  With
 *     d_sh_shadow_out, the SH group is also written there as [n2,16,3] in
 *     shadow_dtype (GS_BF16 or GS_F16, rounded to nearest).
 * n2 is written to *d_n_out on the device (0 when nothing is kept); the host
 * reads it when it needs the new count.  capacity (Gaussians) bounds n2; the
 * output buffers hold 59 * capacity floats (N + n_clone + 3 always
 * suffices).  If n2 would exceed it, GS_EW_CAPACITY is set in *d_err_word,
 * *d_n_out is 0 and nothing is written.  Output buffers must not alias the
 * inputs.  d_workspace: gs_densify_workspace(N) bytes. */
int gs_grad2d_norm(int n_views, int N, const float *d_grad2d, float *d_out, gs_stream_t stream);
int gs_densify_workspace(int N, size_t *bytes);
int gs_densify(int N, const float *d_params, const float *d_m, const float *d_v,
               const float *d_grad_norm, float logit_threshold, int n_clone, long long capacity,
               float *d_params_out, float *d_m_out, float *d_v_out, void *d_sh_shadow_out,
               int shadow_dtype, int32_t *d_n_out, void *d_workspace, size_t workspace_bytes,
               int *d_err_word, gs_stream_t stream);

/* Colour hashing of the Gaussians listed per tile (Sec. IV-C1).  For every
 * entry of every tile's list [d_tile_ranges[t].x, .y) (the lists of
 * gs_bin_sort or gs_bin_sort_prefix) the colour of its splat record
 * (rgb_dtype as gs_render_fwd; 16-bit colours widened) goes to 8 bits per
 * channel as floor(fl32(fl32(c * 255) + 0.5)) clamped to [0, 255], is
 * quantised to c_q = c8 >> 4 (= floor(c8 / 256 * 16)) and hashed to
 * R_q * 256 + G_q * 16 + B_q in [0, 4095].  Per bucket, ADDED to d_count
 * [4096] and d_sums [4, 4096] (sums of R, G, B and of the opacity
 * 2^lo of the record; the caller zeroes both): the number of entries and the
 * sums, accumulated per tile in shared memory and then across tiles (FP32
 * per tile, FP64 across, in no fixed order).  d_tile_distinct [n_tiles]
 * receives the number of distinct buckets among each tile's entries. */
int gs_colour_buckets(int n_tiles, const uint32_t *d_tile_ranges, const uint32_t *d_vals,
                      const void *d_splats, int rgb_dtype, unsigned long long *d_count, double *d_sums,
                      int32_t *d_tile_distinct, gs_stream_t stream);

/* Similarity-based sampling and merging of the tile lists (Sec. IV-C1), an
 * opt-in lossy render mode.  Per tile, the entries of its list (as
 * gs_colour_buckets reads them) are grouped by the same colour bucket; the
 * paper merges a bucket by averaging the colour and accumulating the
 * opacity.  Reading taken: the bucket's first entry in list (depth) order
 * represents it, keeping its record's position, conic and place in the list,
 * with colour = the mean of the members' record colours and opacity
 * min(1, sum of the members' opacities 2^lo); the other entries are dropped.
 * Out: d_out_ranges [n_tiles, 2] the merged lists (each within its input
 * range, from its start; an empty tile reads [0, 0)); d_out_splats FP32 splat
 * records (GS_SPLAT_BYTES_F32 each) and d_out_vals (u32, = position) at the
 * positions of the merged lists, so gs_render_fwd(d_out_ranges, d_out_vals,
 * d_out_splats, GS_F32, ...) renders them; optional d_out_src (the record
 * index of each representative) and d_out_members (its member count).  The
 * output arrays are indexed like d_vals (its length suffices).  Sums are FP32
 * in shared memory, in no fixed order (last-bit differences between runs).
 * Forward only: no reverse pass is defined for merged lists. */
int gs_colour_merge(int n_tiles, const uint32_t *d_tile_ranges, const uint32_t *d_vals,
                    const void *d_splats, int rgb_dtype, uint32_t *d_out_ranges, uint32_t *d_out_vals,
                    void *d_out_splats, uint32_t *d_out_src, uint32_t *d_out_members,
                    gs_stream_t stream);

/* Workload-sensitive density control (Sec. III-C), one round.  Positions are
 * the first 3N floats of the grouped layout ([N, 3], finite).  Squared
 * distances are (dx^2 + dy^2) + dz^2 in FP32 with every operation rounded.
 *
 * gs_density_stats: per point, the local density rho (other points with
 * squared distance <= fl(r * r), Sec. III-C1), the mean distance d_bar to the
 * k nearest other points (1 <= k <= 8; the k smallest distances added in
 * ascending order, then divided by k; fewer when fewer points exist, 0 with
 * none, Sec. III-C2), the nearest other point (ties to the lower index; -1
 * with none) and its distance.  With d_thresholds (device, 3 doubles) and
 * thr_params (host, 3 floats: alpha, beta, gamma >= 0) it also writes, in
 * FP64, rho_low = mu - alpha sigma and rho_high = mu + beta sigma (mu, sigma
 * the mean and population standard deviation of rho, from exact integer
 * sums) and d_merge = mu_d + gamma sigma_d over the nearest-neighbour
 * distances (Sec. III-C3; summed in FP64 in no fixed order).
 *
 * gs_density_control: from N Gaussians (grouped layout; moments d_m, d_v the
 * same; draws d_z ~ N(0,1) and d_u ~ U[0,1), [N, 3] each):
 *   - a point with rho < rho_low spawns one point at
 *     p + (alpha_d d_bar) z + delta (2u - 1), every other parameter copied;
 *   - a point with rho > rho_high whose nearest neighbour is also above
 *     rho_high, has it as its own nearest neighbour and lies within d_merge
 *     merges with it: position = opacity-weighted centroid (weights
 *     sigmoid(logit)), log-scale = log(mean of the two scales) per axis, the
 *     rest from the larger logit (ties to the lower index);
 *   - output, grouped layout of the new count n2 in d_params_out, d_m_out,
 *     d_v_out (and the SH group in d_sh_shadow_out as [n2,16,3] of
 *     shadow_dtype, if given): untouched points in index order, merged points
 *     in the order of their lower index, spawned points in the order of their
 *     parents, then copies of output point 0 with logit -30 up to a multiple
 *     of 4; merged, spawned and padding points have zero moments.
 * n2 goes to *d_n_out (device); rho_low, rho_high, d_merge to d_thresholds if
 * given.  capacity (Gaussians) bounds n2 (2N + 3 always suffices); beyond it
 * GS_EW_CAPACITY is set, *d_n_out = 0 and nothing is written.  Outputs must
 * not alias inputs.  d_workspace: gs_density_workspace(N) bytes (it holds a
 * cell table of 2^24 + 1 entries; the grid's cells are at least 1.0001 r and
 * grow until at most 2^24 cover the points' bounding box). */
int gs_density_workspace(int N, size_t *bytes);
int gs_density_stats(int N, const float *d_means, float r, int k, int32_t *d_rho, float *d_dbar,
                     int32_t *d_nn, float *d_dnn, const float *thr_params, double *d_thresholds,
                     void *d_workspace, size_t workspace_bytes, gs_stream_t stream);
int gs_density_control(int N, const float *d_params, const float *d_m, const float *d_v,
                       const float *d_z, const float *d_u, float r, int k, float alpha, float beta,
                       float alpha_d, float delta, float gamma, long long capacity,
                       float *d_params_out, float *d_m_out, float *d_v_out, void *d_sh_shadow_out,
                       int shadow_dtype, int32_t *d_n_out, double *d_thresholds, void *d_workspace,
                       size_t workspace_bytes, int *d_err_word, gs_stream_t stream);

/* a8. Learned tile-cost scheduler.  The paper balances rendering work by a
 * region density rho = active Gaussians / pixels (Sec. IV-C2); here a small
 * MLP predicts each tile's render cost from eight tile statistics and the
 * renderer takes tiles longest-predicted first (GS_SCHED_ORDER).
 *
 * gs_tile_features: eight FP32 features per global tile into d_feats [T, 8],
 * from the first min(count, cap) entries of the tile's list:
 *   f0 log1p(count), f1 mean opacity, f2 max opacity,
 *   f3 mean coverage cov = min(1, pi sqrt(det Sigma') / 256),
 *   f4 log1p(sum o cov),
 *   f5 log1p(sum of Th_j over entries with Th_j >= 1e-4), where Th_0 = 1 and
 *      Th_{j+1} = Th_j (1 - min(0.99, o_j cov_j)) (expected transmittance),
 *   f6 fraction of the tile's pixels inside the image, f7 log1p(W H) / 16.
 * With d_w16 (FP16 MLP weights, as gs_mlp_predict) and d_pred, the
 * prediction of each tile is also written (both NULL: features only). */
int gs_tile_features(const gs_camera *cams, int n_views, const uint32_t *d_tile_ranges,
                     const uint32_t *d_vals, const void *d_splats, int rgb_dtype, int cap,
                     float *d_feats, const void *d_w16, float *d_pred, gs_stream_t stream);

/* a8, the reverse pass's cost features: eight per tile from what the
 * forward pass of the same step left, [T, 8] FP32 into d_feats:
 *   b0 log1p(d_tile_nproc, the tile's largest processed count),
 *   b1 log1p(mean of d_n_proc over the tile's in-image pixels),
 *   b2 log1p(the forward's d_tile_ns of the tile; 0 if NULL),
 *   b3 log1p(the tile's kept list length, from d_tile_ranges),
 *   b4 log1p(mean over the tile's upper and lower 16x8 halves of their
 *      largest d_n_proc),
 *   b5 the fraction of in-image pixels with d_n_proc > 0,
 *   b6 the in-image pixel fraction, b7 log1p(W H) / 16.
 * With d_w16 and d_pred the MLP's prediction is written as in
 * gs_tile_features. */
int gs_bwd_tile_features(const gs_camera *cams, int n_views, const uint32_t *d_tile_ranges,
                         const int32_t *d_tile_nproc, const int32_t *d_n_proc,
                         const uint64_t *d_tile_ns, float *d_feats, const void *d_w16, float *d_pred,
                         gs_stream_t stream);

/* MLP 8 -> 32 (ReLU) -> 1.  Weights are 321 values in the order W1 [32, 8]
 * (row-major), b1 [32], W2 [32], b2 [1].  gs_mlp_predict reads FP16 weights
 * (d_w16, 321 halves) and accumulates in FP32: d_pred[i] = W2 relu(W1 f_i +
 * b1) + b2 for n rows of d_feats [n, 8]. */
int gs_mlp_predict(const void *d_w16, const float *d_feats, int n, float *d_pred,
                   gs_stream_t stream);

/* Mean squared error of the FP32-weight MLP (d_w32) against targets and its
 * gradient: target_i = d_target[i] if d_target != NULL, else
 * log(max(d_tile_ns[i], 1)).  Writes d_grad [321] and *d_loss (device). */
int gs_mlp_grad(const float *d_w32, const float *d_feats, const uint64_t *d_tile_ns,
                const float *d_target, int n, float *d_grad, float *d_loss, gs_stream_t stream);

/* gs_mlp_grad, then one Adam step (b1 0.9, b2 0.999, eps 1e-8, step t) on the
 * FP32 weights with moments d_m, d_v [321], then the FP16 copy d_w16. */
int gs_mlp_train_step(float *d_w32, void *d_w16, float *d_m, float *d_v, int t, float lr,
                      const float *d_feats, const uint64_t *d_tile_ns, const float *d_target, int n,
                      float *d_grad, float *d_loss, gs_stream_t stream);

/* a8, the count order as judge of the learned one (Sec. IV: tile cost drives
 * the balanced partition).  Over n_pairs seeded pairs of tiles (i, j), drawn
 * by a counter-based 32-bit mix of seed and the pair index, skipping pairs
 * where a tile time is 0 (empty tile) or both times are equal, d_out[0]
 * gains 2 when d_a orders the pair as d_tile_ns does, 1 when d_a ties, 0
 * otherwise; d_out[1] the same for d_b[i * b_stride] (e.g. the instance-
 * count feature in the [T, 8] feature array, b_stride 8).  d_out is
 * 2 x uint64 on the device, ADDED to (zero it first).  Integer results:
 * exact. */
int gs_rank_judge(const float *d_a, const float *d_b, int b_stride, const uint64_t *d_tile_ns, int n,
                  int n_pairs, uint32_t seed, unsigned long long *d_out, gs_stream_t stream);

/* d_cost[i] = (float) d_counts[i] for n entries. */
int gs_int_cost(const int32_t *d_counts, int n, float *d_cost, gs_stream_t stream);

/* d_cost[t] = entries in tile t's list (from d_tile_ranges [T, 2]). */
int gs_range_cost(const uint32_t *d_tile_ranges, int T, float *d_cost, gs_stream_t stream);

/* A work order: d_order = the n indices sorted by d_cost descending (ties by
 * index).  d_workspace (256-byte aligned) of gs_sched_order_workspace bytes. */
int gs_sched_order_workspace(int n, size_t *bytes);
int gs_sched_order(const float *d_cost, int n, int32_t *d_order, void *d_workspace,
                   size_t workspace_bytes, gs_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* GS103_H */

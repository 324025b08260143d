/*
 * star_nt.h -- C ABI of the STAR-NT per-frame hot path on one B300 (sm_103a).
 *
 * STAR-NT (arXiv 2606.16747) renders order-independent transparency with
 * three geometry passes (nearest fragment, second-nearest fragment, tail
 * statistics), a small MLP that predicts the colour of the fragments behind
 * the two nearest ones, and the decoupled composite of Eq. 4.  Passes 2 and 3
 * run at reduced resolution chosen by an adaptive quadtree over the previous
 * frame (Sec. 3.1, 3.2, Eq. 2); interpolated frames reuse the last real frame
 * through depth-based reprojection (Sec. 3.3, last paragraph).
 *
 * Conventions common to every call
 *  - All buffers are caller-owned device memory given as plain pointers.  The
 *    library never allocates, frees or synchronises, and enqueues all work on
 *    the stream it is given (a cudaStream_t passed as void*).
 *  - Pointers must be 16-byte aligned; workspaces 256-byte aligned.
 *  - Every call returns a star_nt_status.  Bad host arguments are rejected
 *    before anything is enqueued (STAR_NT_ERR_ARG).  A failed launch returns
 *    STAR_NT_ERR_CUDA.  Conditions found on the device (capacity overflow, an
 *    expired wait) are written to a caller-provided device int32 status word
 *    (first error wins) that the caller reads after its own synchronisation;
 *    later calls that depend on a failed one do no work.  Nothing traps.
 *  - Sizes that change from frame to frame (the reduced pass resolutions) are
 *    read on the device, so one captured CUDA graph replays every frame.
 *  - Images are row-major, pixel p = y * width + x, y pointing down.
 *  - Colours are straight RGBA8 packed in a uint32 (R bits 0-7, G 8-15,
 *    B 16-23, A 24-31); c = c8 / 255, alpha = a8 / 255.
 */
#ifndef STAR_NT_H
#define STAR_NT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define STAR_NT_VERSION 1

typedef int32_t star_nt_status;
#define STAR_NT_OK 0
#define STAR_NT_ERR_ARG 1
#define STAR_NT_ERR_CAPACITY 2
#define STAR_NT_ERR_CUDA 3
#define STAR_NT_ERR_TIMEOUT 4
#define STAR_NT_ERR_UNSUPPORTED 5

/* element types of the network input */
#define STAR_NT_F32 0  /* [P][8] float32: x0..x4, tail flag, 0, 0 */
#define STAR_NT_BF16 1 /* [P][8] bfloat16: x0..x4, tail flag, 0, 0 */

/* Quadtree tiles: base tile side (pixels) and levels (Sec. 3.1). */
#define STAR_NT_QT_LEVELS 4

int32_t star_nt_version(void);
const char *star_nt_status_string(int32_t status);

/* ------------------------------------------------------------------------ */
/* Inputs                                                                    */

/* A soup of flat-coloured transparent triangles (device memory).
 * verts: [n_tris][3][4] float32 world-space (x, y, z, w); rgba8: [n_tris].
 * The primitive id of a triangle is its index. */
typedef struct {
    const float *verts;
    const uint32_t *rgba8;
    int32_t n_tris;
} star_nt_scene;

/* Render target of one geometry pass.
 * view_proj: device, 16 float32, row-major, clip = M (x, y, z, w)^T; the
 *   projection maps the visible depth range to NDC z in [0, 1].
 * size: device, {W_p, H_p}, the pass's resolution (read on the device).
 * max_w, max_h: host upper bounds of size[]; they size the launches.
 * merge_at: optional device {W, H} of pass 1 (NULL: never merged).  The
 *   pass is merged when W_p >= merge_scale * W and H_p >= merge_scale * H
 *   (merge_scale <= 0 is read as 1: only a pass at the full size merges):
 *   it is then left to pass 1 (star_nt_geometry_pass_merged /
 *   star_nt_geometry_passes), which produces its planes at the full size W x H,
 *   and the bins are marked merged, record the full size and hold no
 *   triangles.  A merge below full size is a cost choice: pass 1 keeping two
 *   layers costs less than a second traversal at nearly full size, and the
 *   planes are then exact rather than upscaled.
 * merge_scale: see merge_at. */
typedef struct {
    const float *view_proj;
    const int32_t *size;
    int32_t max_w, max_h;
    const int32_t *merge_at;
    float merge_scale;
} star_nt_target;

/* Parameters of the method.  Defaults (star_nt_default_params):
 * bg = (1, 1, 1), kappa_n = 1/64, tau_split = 24, tau_merge = 12,
 * delta2 = 2.2, delta3 = 3.0 (Eq. 2), base_tile = 16, relax_iters = 2. */
typedef struct {
    float bg[3];       /* background colour C_b of Eq. 4 */
    float kappa_n;     /* feature x0 = kappa_n * N */
    double tau_split;  /* split a leaf when D_i > tau_split (8-bit units) */
    double tau_merge;  /* merge a node when D_i < tau_merge, tau_merge < tau_split */
    double delta2;     /* Eq. 2 offset of pass 2 */
    double delta3;     /* Eq. 2 offset of pass 3 */
    int32_t base_tile; /* quadtree base tile side: 16 or 64 pixels */
    int32_t relax_iters;
} star_nt_params;

void star_nt_default_params(star_nt_params *p);

/* star_nt_preload: load every kernel of the library onto the current device.
 * Optional; call once per device before the first frame.  CUDA loads modules
 * lazily on first use; a first use inside a stream capture, or beside work
 * on other streams, can stall the calling thread while the module loads.
 * Returns STAR_NT_ERR_CUDA if a kernel cannot be loaded (no device, or a
 * device of another architecture). */
star_nt_status star_nt_preload(void);

/* star_nt_set_wait_limit: bound, in nanoseconds, of every wait of the
 * tensor-core kernels (star_nt_infer in BF16, the resolves, the pass launch
 * that produces the frame) for an MMA or a TMA copy.  Default 1e9 (one
 * second), at most STAR_NT_MAX_WAIT_LIMIT_NS, else STAR_NT_ERR_ARG.  A wait
 * that runs out raises STAR_NT_ERR_TIMEOUT in the call's status word; the
 * kernel then stops its work, lets the MMA or copy it has in flight complete
 * (under a second, fixed one-second bound), frees its tensor memory and
 * returns, so the device stays usable.  0 makes every such wait run out at
 * once (to exercise that path).  Process-wide; read when a call enqueues its
 * launch, so a captured CUDA graph keeps the value in force at capture.
 * The paper has no counterpart: this is the library's failure detection.
 * star_nt_wait_limit returns the value in force. */
#define STAR_NT_MAX_WAIT_LIMIT_NS 60000000000ull
star_nt_status star_nt_set_wait_limit(uint64_t ns);
uint64_t star_nt_wait_limit(void);

/* ------------------------------------------------------------------------ */
/* star_nt_raster -- geometry front end of one pass (Sec. 3, Fig. 1).         */
/*                                                                           */
/* Transforms and snaps every triangle to the pass's render target (1/256    */
/* pixel fixed point), drops triangles with a vertex outside the depth range */
/* or behind the camera and degenerate ones (no back-face culling), and bins */
/* the rest to 16 x 16-pixel tiles.  Optionally materialises every fragment  */
/* (per-pixel lists in CSR form).  Coverage is exact: a pixel centre is      */
/* covered when all three edge functions are positive, or zero on an edge    */
/* with dy > 0 or (dy == 0 and dx < 0).  Depth is the NDC z interpolated in  */
/* screen space with fixed float32 operations.                               */

/* Workspace of binned triangles for one pass: caller allocates
 * star_nt_bins_bytes(...) bytes of device memory (256-byte aligned) and
 * zero-fills it once before its first use.  Every call leaves the per-tile
 * counters and the work counters in it at zero again, so no call has to clear
 * them (one fewer graph node per pass). */
typedef struct {
    void *mem;
    size_t bytes;
    int32_t max_w, max_h;   /* largest render target this workspace serves */
    int32_t max_tris;       /* largest scene */
    int64_t pair_capacity;  /* (triangle, tile) pairs it can hold */
} star_nt_bins;

star_nt_status star_nt_bins_bytes(int32_t max_w, int32_t max_h, int32_t max_tris,
                                  int64_t pair_capacity, size_t *bytes);

/* Materialised fragments of a pass (optional output of star_nt_raster).
 * count [max_w * max_h], offset [max_w * max_h + 1] (exclusive prefix sum of
 * count over the pass's W_p * H_p pixels), z / prim [capacity], total: device
 * uint32 receiving the fragment count (also when it exceeds capacity, in
 * which case STAR_NT_ERR_CAPACITY is raised and no fragment is written).
 * The order of a pixel's fragments is unspecified. */
typedef struct {
    uint32_t *count;
    uint32_t *offset;
    float *z;
    int32_t *prim;
    int64_t capacity;
    uint32_t *total;
} star_nt_frags;

star_nt_status star_nt_raster(const star_nt_scene *scene, const star_nt_target *target,
                              const star_nt_bins *bins, const star_nt_frags *frags_or_null,
                              int32_t *d_status, void *stream);

/* The front end of up to STAR_NT_MAX_RASTER_PASSES passes at once (targets[i]
 * into bins[i], distinct workspaces), in the same three launches: the frame's
 * passes share each launch instead of running one after another.  No
 * fragment lists. */
#define STAR_NT_MAX_RASTER_PASSES 9
star_nt_status star_nt_raster_passes(const star_nt_scene *scene, int32_t n_passes,
                                     const star_nt_target *targets, const star_nt_bins *bins,
                                     int32_t *d_status, void *stream);

/* ------------------------------------------------------------------------ */
/* star_nt_build_inputs -- the three geometry passes and the network input    */
/* (Sec. 3.2, Sec. 3.3, Eq. 4).                                              */
/*                                                                           */
/* Per pixel of each pass (at its own resolution), fragments are ordered by   */
/* (z, primitive id).  Pass 1 keeps the nearest (id1, z1); pass 2 the second  */
/* nearest (id2); pass 3 the fragment count N and, over the tail (all but the */
/* two nearest), sum a8, sum a8 c8 per channel and the tail transmittance    */
/* t_tail = prod (1 - alpha_i).  The planes of passes 2 and 3 are upscaled   */
/* bilinearly to W x H (half-pixel centres, clamp to edge), then             */
/*   x     = [kappa_n N, t_tail, sum a8 c8 / (255 sum a8)]  (zero colour when */
/*           the tail has no alpha) plus a tail flag (upscaled N > 2);       */
/*   front = (C_exact,2 + T_2 t_tail C_b, T_2), C_exact,2 = a1 c1 + (1-a1) a2 c2, */
/*           T_2 = (1 - a1)(1 - a2).                                         */
/* When the three bins are the same object every pass runs at full           */
/* resolution in one fused kernel (the plain neural OIT pipeline).           */
/* The tail sums are exact integers (uint32 per channel) for up to 66,052    */
/* fragments per pixel, where sum a8 c8 reaches 2^32; beyond that they wrap. */

/* Per-pass planes at the pass's resolution; members may be NULL when not
 * wanted.  tail is [P][4] uint32: sum a8, sum a8 r8, sum a8 g8, sum a8 b8. */
typedef struct {
    int32_t *id1;
    float *z1;
    int32_t *id2;
    uint32_t *n;
    uint32_t *tail;
    float *t_tail;
} star_nt_layers;

/* Full-resolution network input and front terms. */
typedef struct {
    void *x;         /* [W*H][8] float32 or [W*H][8] bfloat16 (x_dtype) */
    int32_t x_dtype; /* STAR_NT_F32 or STAR_NT_BF16 */
    float *front;    /* [W*H][4] */
} star_nt_features;

/* bins1/2/3: the binned passes (written by star_nt_raster); layers1/2/3: the
 * per-pass planes (layers1 needs id1 and z1 unless fused; layers2 needs id2;
 * layers3 needs n, tail, t_tail).  W, H: full resolution. */
star_nt_status star_nt_build_inputs(const star_nt_scene *scene, const star_nt_bins *bins1,
                                    const star_nt_bins *bins2, const star_nt_bins *bins3,
                                    const star_nt_layers *layers1, const star_nt_layers *layers2,
                                    const star_nt_layers *layers3, int32_t W, int32_t H,
                                    const star_nt_params *params, const star_nt_features *out,
                                    int32_t *d_status, void *stream);

/* The two halves of star_nt_build_inputs, callable on their own (for example
 * to schedule or time the passes separately).
 * star_nt_geometry_pass: one pass over one bins object at its resolution;
 *   mode 1 writes id1/z1 (nearest fragment), mode 2 id2 (second nearest),
 *   mode 3 n, tail and t_tail (tail statistics).  Members of layers that the
 *   mode does not write may be NULL.
 * star_nt_upscale_features: bilinear upscale of passes 2 and 3 (resolutions read
 *   from their bins) and the full-resolution network input and front terms. */
star_nt_status star_nt_geometry_pass(const star_nt_scene *scene, const star_nt_bins *bins,
                                     int32_t mode, const star_nt_layers *layers,
                                     int32_t *d_status, void *stream);
/* star_nt_geometry_pass_merged: pass 1 (nearest fragment, full resolution)
 * that also performs pass 2 and/or pass 3 at full resolution when their bins
 * are marked merged (see star_nt_target.merge_at): it then writes id2 into
 * layers2 and n, tail, t_tail into layers3 at full resolution, and the
 * merged bins record the full size, so star_nt_upscale_features and
 * star_nt_resolve read them as usual (an identity upscale). */
star_nt_status star_nt_geometry_pass_merged(const star_nt_scene *scene, const star_nt_bins *bins1,
                                            const star_nt_bins *bins2, const star_nt_bins *bins3,
                                            const star_nt_layers *layers1,
                                            const star_nt_layers *layers2,
                                            const star_nt_layers *layers3, int32_t *d_status,
                                            void *stream);
/* Tile shape and launch size of the persistent geometry-pass launches
 * (star_nt_geometry_passes, star_nt_geometry_passes_resolve and
 * star_nt_geometry_passes_leaf; NULL: the defaults).
 * block_w: width of the pixel block a warp owns inside a 16 x 16 tile (4, 8
 *   or 16); default 8.
 * pixels_per_thread: 1: CTAs of 256 threads, one pixel each, the warp's block
 *   block_w x 32/block_w; 2: CTAs of 128 threads, two pixels each (rows r and
 *   r + 32/block_w of a block_w x 64/block_w block), which share the
 *   triangle loads and the loop; 0: 2.
 * ctas_per_sm: one pixel per thread: 0 or 8: full occupancy with an 8-CTA
 *   register budget (32 per thread); 1..7: a 6-CTA budget (40 per thread)
 *   and the grid capped at that many CTAs per SM.  Two pixels per thread:
 *   0 or 8: full occupancy with an 8-CTA budget (64 registers); 10: a
 *   10-CTA budget (48 registers); 1..7 and 9: the 8-CTA budget and the grid
 *   capped at that many.
 *   The launch that also resolves the frame runs at most 6 (one pixel) or 8
 *   (two pixels: 8 x 64 columns, all of tensor memory) CTAs per SM.
 *   Default 0.
 * Results do not depend on the tuning. */
typedef struct {
    int32_t block_w;
    int32_t ctas_per_sm;
    int32_t pixels_per_thread;
} star_nt_tuning;

/* star_nt_geometry_passes: the three geometry passes of a real frame in one
 * persistent launch (the same results as star_nt_geometry_pass_merged, then
 * modes 2 and 3): CTAs take tiles of pass 1, then pass 2, then pass 3 from
 * a work counter kept in bins1's workspace, so uneven tiles and passes of
 * different sizes share the launch.  bins1..3 must be distinct.  Returns
 * without work on the device when bins2 is marked resolved (see
 * star_nt_geometry_passes_resolve). */
star_nt_status star_nt_geometry_passes(const star_nt_scene *scene, const star_nt_bins *bins1,
                                       const star_nt_bins *bins2, const star_nt_bins *bins3,
                                       const star_nt_layers *layers1,
                                       const star_nt_layers *layers2,
                                       const star_nt_layers *layers3,
                                       const star_nt_tuning *tuning, int32_t *d_status,
                                       void *stream);
star_nt_status star_nt_upscale_features(const star_nt_scene *scene, const star_nt_bins *bins2,
                                const star_nt_bins *bins3, const star_nt_layers *layers1,
                                const star_nt_layers *layers2, const star_nt_layers *layers3,
                                int32_t W, int32_t H, const star_nt_params *params,
                                const star_nt_features *out, void *stream);

/* ------------------------------------------------------------------------ */
/* star_nt_infer -- tail-colour MLP 5 -> 32 -> 16 -> 3, ReLU on every layer   */
/* (Sec. 3.3).  f = 0 where the tail flag of x is zero.                      */

/* float32 weights, row-major [out][in], device memory. */
typedef struct {
    const float *w1, *b1; /* [32][5], [32] */
    const float *w2, *b2; /* [16][32], [16] */
    const float *w3, *b3; /* [3][16], [3] */
} star_nt_mlp;

/* x: [P] rows in x_dtype layout; f: [P][4] float32 (rgb, 0).
 * STAR_NT_F32 evaluates in float32 on the CUDA cores; STAR_NT_BF16 runs the
 * three layers on the tcgen05 tensor cores (bf16 operands, fp32 accumulation
 * in tensor memory); x must then be 256-byte aligned. */
star_nt_status star_nt_infer(const star_nt_mlp *w, int32_t x_dtype, const void *x, float *f,
                             int64_t P, int32_t *d_status, void *stream);

/* ------------------------------------------------------------------------ */
/* star_nt_resolve -- the full-resolution end of a real frame fused in one    */
/* kernel: the bilinear upscale and network input of star_nt_upscale_features,*/
/* the tail MLP of star_nt_infer on the tcgen05 tensor cores (bf16 operands,   */
/* fp32 accumulation) and the composite of Eq. 4.  The network input, f(x) and */
/* the front terms stay on chip.  Arguments as star_nt_upscale_features, plus  */
/* the float32 weights w and the frame outputs (rgba32f [P][4], rgba8 [P];     */
/* either may be NULL).                                                       */
star_nt_status star_nt_resolve(const star_nt_scene *scene, const star_nt_bins *bins2,
                               const star_nt_bins *bins3, const star_nt_layers *layers1,
                               const star_nt_layers *layers2, const star_nt_layers *layers3,
                               int32_t W, int32_t H, const star_nt_params *params,
                               const star_nt_mlp *w, float *rgba32f, uint32_t *rgba8,
                               int32_t *d_status, void *stream);

/* star_nt_resolve_fp8 -- star_nt_resolve with the MLP in FP8: e4m3 operands  */
/* on the tcgen05 tensor cores (fp32 accumulation), one power-of-two scale per */
/* weight tensor and per operand row (pixel), biases, rescale and ReLU in     */
/* fp32.  Same arguments and errors as star_nt_resolve.  e4m3 keeps 3 mantissa */
/* bits, so f(x) is coarser than with bf16; the parity test states the bound. */
star_nt_status star_nt_resolve_fp8(const star_nt_scene *scene, const star_nt_bins *bins2,
                                   const star_nt_bins *bins3, const star_nt_layers *layers1,
                                   const star_nt_layers *layers2, const star_nt_layers *layers3,
                                   int32_t W, int32_t H, const star_nt_params *params,
                                   const star_nt_mlp *w, float *rgba32f, uint32_t *rgba8,
                                   int32_t *d_status, void *stream);

/* star_nt_resolve_fp8x2 -- star_nt_resolve_fp8 with compensated operands:    */
/* every weight and activation as a pair of e4m3 values hi + lo (hi = e4m3 of */
/* the scaled value, lo = e4m3 of the remainder) under one power-of-two row   */
/* scale, and the four products hi.hi + lo.hi + hi.lo + lo.lo accumulated in  */
/* fp32 on the tensor cores (kind::f8f6f4).  Each operand keeps about 2^-8    */
/* relative rounding, as a bf16 operand does, for four times the e4m3 MMA     */
/* work.  Same arguments and errors as star_nt_resolve.                       */
star_nt_status star_nt_resolve_fp8x2(const star_nt_scene *scene, const star_nt_bins *bins2,
                                     const star_nt_bins *bins3, const star_nt_layers *layers1,
                                     const star_nt_layers *layers2, const star_nt_layers *layers3,
                                     int32_t W, int32_t H, const star_nt_params *params,
                                     const star_nt_mlp *w, float *rgba32f, uint32_t *rgba8,
                                     int32_t *d_status, void *stream);

/* star_nt_resolve_mlp -- star_nt_resolve with the MLP operand type chosen by  */
/* mlp_type: STAR_NT_BF16 (star_nt_resolve), STAR_NT_E4M3 (star_nt_resolve_fp8: */
/* per-row scales), STAR_NT_E4M3X2 (star_nt_resolve_fp8x2), or the per-tensor  */
/* scaled FP8 variants STAR_NT_E4M3_TENSOR and STAR_NT_E4M3X2_TENSOR: one       */
/* power-of-two scale per weight tensor (its largest |w| at most 448, the e4m3 */
/* maximum) and one per activation tensor, fixed for the launch by interval    */
/* bounds through the network from the input box (x0 = kappa_n N with N <=    */
/* 448 fragments, the other features <= 1), so no activation saturates; each  */
/* accumulator is rescaled by one exact factor per tensor.  Other arguments   */
/* and errors as star_nt_resolve; STAR_NT_ERR_ARG for another mlp_type.       */
star_nt_status star_nt_resolve_mlp(const star_nt_scene *scene, const star_nt_bins *bins2,
                                   const star_nt_bins *bins3, const star_nt_layers *layers1,
                                   const star_nt_layers *layers2, const star_nt_layers *layers3,
                                   int32_t W, int32_t H, const star_nt_params *params,
                                   const star_nt_mlp *w, int32_t mlp_type, float *rgba32f,
                                   uint32_t *rgba8, int32_t *d_status, void *stream);

/* star_nt_geometry_passes_resolve: star_nt_geometry_passes that, when both
 * reduced passes are merged into pass 1 (their bins marked merged: every pass
 * at the full resolution), also produces the frame: pass 1's tiles run the
 * network input, the tail MLP on the tcgen05 tensor cores (bf16 operands,
 * fp32 accumulation) and the composite of Eq. 4 for their pixels, and write
 * rgba32f / rgba8 as star_nt_resolve would, bit for bit.  layers1's id1 and z1
 * are written; the merged passes' planes are not.  bins2's header is then
 * marked resolved, and a following star_nt_resolve or star_nt_resolve_fp8 on
 * the same bins returns without work (use star_nt_resolve, not
 * star_nt_upscale_features, after this call).  With a reduced pass not merged
 * the call is star_nt_geometry_passes and the frame is left to
 * star_nt_resolve.  Two launches: the fused one (which returns at once unless
 * every pass is merged), then star_nt_geometry_passes' (which returns at once
 * when the first resolved the frame).  params (bg, kappa_n), w and the frame
 * outputs as star_nt_resolve; other arguments as star_nt_geometry_passes. */
star_nt_status star_nt_geometry_passes_resolve(const star_nt_scene *scene,
                                               const star_nt_bins *bins1,
                                               const star_nt_bins *bins2,
                                               const star_nt_bins *bins3,
                                               const star_nt_layers *layers1,
                                               const star_nt_layers *layers2,
                                               const star_nt_layers *layers3,
                                               const star_nt_params *params,
                                               const star_nt_mlp *w, float *rgba32f,
                                               uint32_t *rgba8, const star_nt_tuning *tuning,
                                               int32_t *d_status, void *stream);

/* ------------------------------------------------------------------------ */
/* star_nt_composite -- Eq. 4: C = C_exact,2 + T_2 f(x) + T_all C_b.          */
/* front: [P][4] (from star_nt_build_inputs), f: [P][4].  Writes rgba32f      */
/* [P][4] (alpha = 1) and rgba8 [P] (round half to even of clamp(c,0,1)*255). */
star_nt_status star_nt_composite(const float *front, const float *f, int64_t P, float *rgba32f,
                                 uint32_t *rgba8, void *stream);

/* ------------------------------------------------------------------------ */
/* star_nt_quadtree -- adaptive screen-space tiles and tile-guided            */
/* resolution (Sec. 3.1, Sec. 3.2, Eq. 2).                                   */
/*                                                                           */
/* Each base tile keeps a 21-bit mask of "split" bits (root; 4 level-1 nodes; */
/* 16 level-2 nodes, children numbered 2 * y_half + x_half); level-3 nodes    */
/* are leaves.  From mask_prev and the 8-bit composited frame: a leaf splits  */
/* when D > tau_split; a node whose children are leaves, none of them        */
/* splitting, merges when D < tau_merge (every decision on mask_prev, so a   */
/* pixel's level changes by at most one).  D is the mean of the six pairwise */
/* Euclidean RGB distances of the node's four corner pixels.  Then          */
/* relax_iters Jacobi iterations split any leaf with an edge-neighbour leaf  */
/* two or more levels deeper.  Finally N_l counts leaves at level l holding  */
/* a pixel with id1 >= 0, wbar = sum l N_l / sum N_l and                     */
/* s_p = clamp(2^(wbar - delta_p), 0.25, 1), W_p = ceil(s_p W).              */

/* Device-resident resolution state read by the next frame's passes. */
typedef struct {
    int32_t W, H;     /* full resolution */
    int32_t W2, H2;   /* pass 2 resolution */
    int32_t W3, H3;   /* pass 3 resolution */
    float s2, s3;
    double wbar;
    uint32_t hist[4];
} star_nt_pass_state;

star_nt_status star_nt_quadtree_ws_bytes(int32_t W, int32_t H, int32_t base_tile,
                                         size_t *bytes);

/* rgba8, id1: [W*H]; mask_prev, mask_out: [ceil(W/B) * ceil(H/B)] (may be
 * the same buffer: the masks are updated in place); state: device
 * star_nt_pass_state, fully rewritten; ws: workspace of
 * star_nt_quadtree_ws_bytes bytes. */
star_nt_status star_nt_quadtree(const uint32_t *rgba8, const int32_t *id1, int32_t W, int32_t H,
                                const star_nt_params *params, const uint32_t *mask_prev,
                                uint32_t *mask_out, star_nt_pass_state *state, void *ws,
                                size_t ws_bytes, void *stream);

/* star_nt_quadtree_static -- star_nt_quadtree for callers that cannot
 * allocate device memory (a plug-in handed only its inputs and outputs by a
 * host application, or an engine that fixes its GPU memory budget at start-up
 * and allows no allocation on the frame path).  The paper has no counterpart.
 * The workspace is a fixed array inside this library (STAR_NT_QT_STATIC_BYTES
 * bytes, held on every GPU that loads the library until the process exits),
 * enough for STAR_NT_QT_STATIC_MAX_TILES base tiles; larger frames return
 * STAR_NT_ERR_CAPACITY.  Arguments and results are those of star_nt_quadtree
 * minus ws / ws_bytes; nothing is allocated.  The array's device address
 * belongs to a CUDA context: the first call made in a context (the device's
 * primary context, or a context the host application created and made
 * current) looks the address up with that context current and caches it
 * under the context's id, so make that first call before any stream capture
 * in that context.  All calls share the one array on a device's context and
 * it keeps the last call's contents (the parts that must start at zero are
 * cleared by each call), so calls that overlap on the GPU race: serialise
 * them, for instance on one stream. */
#define STAR_NT_QT_STATIC_MAX_TILES 65536
#define STAR_NT_QT_STATIC_BYTES (256 + 2 * 4 * STAR_NT_QT_STATIC_MAX_TILES)
star_nt_status star_nt_quadtree_static(const uint32_t *rgba8, const int32_t *id1, int32_t W,
                                       int32_t H, const star_nt_params *params,
                                       const uint32_t *mask_prev, uint32_t *mask_out,
                                       star_nt_pass_state *state, void *stream);

/* ------------------------------------------------------------------------ */
/* Per-leaf pass resolution: the per-tile variant of Sec. 3.2 / Eq. 2.       */
/*                                                                           */
/* Eq. 2 with the scene index wbar replaced by the level l of the quadtree   */
/* leaf holding the pixel: s_p(l) = clamp(2^(l - delta_p), 1/4, 1) for the   */
/* passes p = 2, 3.  A pixel takes pass 2 and pass 3 from the render target  */
/* of its own leaf's scale (W_p = ceil(s W), H_p = ceil(s H), as for the     */
/* global scale), upscaled bilinearly to W x H exactly as in               */
/* star_nt_resolve; pass 1 stays at W x H.  The scales depend only on l and  */
/* delta_p, so the set of targets is fixed for a frame size: a plan lists    */
/* the distinct sizes (target 0 is W x H itself, shared with pass 1) and     */
/* maps every (pass, level) to one of them.  A 16 x 16 tile of a target runs */
/* only the passes that some pixel needs from it: a pixel needs the samples  */
/* of nonzero bilinear weight of its pass-2 and pass-3 targets.  Leaf levels */
/* are read from the quadtree masks (star_nt_quadtree's mask_out of the      */
/* previous frame).                                                          */

#define STAR_NT_E4M3 2   /* MLP operand type of star_nt_resolve_leaf: FP8 e4m3 */
#define STAR_NT_E4M3X2 3 /* ... compensated FP8: e4m3 pairs (star_nt_resolve_fp8x2) */
#define STAR_NT_E4M3_TENSOR 4   /* ... e4m3 with per-tensor scales (star_nt_resolve_mlp) */
#define STAR_NT_E4M3X2_TENSOR 5 /* ... compensated e4m3 with per-tensor scales */
#define STAR_NT_LEAF_MAX_TARGETS 9

typedef struct {
    int32_t W, H;                                 /* full resolution */
    int32_t base_tile;                            /* quadtree base tile side: 16 or 64 */
    int32_t n_targets;                            /* 1 .. STAR_NT_LEAF_MAX_TARGETS */
    int32_t size[STAR_NT_LEAF_MAX_TARGETS][2];    /* target sizes; size[0] = {W, H} */
    int32_t target_of[2][4];                      /* [pass 2, pass 3][level] -> target index */
} star_nt_leaf_plan;

/* Host only: the plan of frame size W x H under params (delta2, delta3,
 * base_tile); sizes in float64 as in star_nt_quadtree.  Targets are listed
 * as first met over pass 2 then pass 3, levels 0..3, after target 0. */
star_nt_status star_nt_leaf_plan_make(int32_t W, int32_t H, const star_nt_params *params,
                                      star_nt_leaf_plan *plan);

/* Workspace of star_nt_geometry_passes_leaf (one mode byte per target tile). */
star_nt_status star_nt_leaf_ws_bytes(const star_nt_leaf_plan *plan, size_t *bytes);

/* star_nt_geometry_passes_leaf: pass 1 and the per-leaf passes 2 and 3 of a
 * real frame.  Two launches: the pass modes of every target tile from the
 * masks, then one persistent launch over the tiles of all targets (work
 * counter in bins[0]'s workspace, as star_nt_geometry_passes).
 * bins[k]: target k binned by star_nt_raster_passes at size[k] (no merge),
 *   n_targets distinct workspaces.  A bins header whose size differs from the
 *   plan raises STAR_NT_ERR_ARG in d_status and its tiles are skipped.
 * layers[k]: planes at target k's size.  layers[0] needs id1 and z1; every
 *   target that some level maps pass 2 to needs id2; every target that some
 *   level maps pass 3 to needs n, tail and t_tail (others may be NULL).
 *   Planes of tiles no pixel needs are left as they were.
 * masks: [ceil(W/B) * ceil(H/B)] quadtree split masks; ws: star_nt_leaf_ws_bytes
 *   bytes (256-byte aligned); tuning: as star_nt_geometry_passes. */
star_nt_status star_nt_geometry_passes_leaf(const star_nt_scene *scene,
                                            const star_nt_leaf_plan *plan,
                                            const star_nt_bins *bins,
                                            const star_nt_layers *layers, const uint32_t *masks,
                                            void *ws, size_t ws_bytes,
                                            const star_nt_tuning *tuning, int32_t *d_status,
                                            void *stream);

/* star_nt_resolve_leaf: star_nt_resolve with each pixel's pass-2 and pass-3
 * planes taken from the targets of its leaf level (layers and masks as in
 * star_nt_geometry_passes_leaf).  mlp_type: as star_nt_resolve_mlp.  Primitive ids read from the
 * planes are bounds-checked against scene->n_tris. */
star_nt_status star_nt_resolve_leaf(const star_nt_scene *scene, const star_nt_leaf_plan *plan,
                                    const star_nt_layers *layers, const uint32_t *masks,
                                    const star_nt_params *params, const star_nt_mlp *w,
                                    int32_t mlp_type, float *rgba32f, uint32_t *rgba8,
                                    int32_t *d_status, void *stream);

/* ------------------------------------------------------------------------ */
/* star_nt_reproject -- interpolated frame by depth-based reprojection        */
/* (Sec. 3.3, last paragraph; Fig. 1).                                       */
/*                                                                           */
/* For pixel (x, y): d = prev_z1 (first-fragment NDC depth of the last real   */
/* frame, 1.0 where empty); the point (ndc(x, y), d) is unprojected with the */
/* current camera and projected with the previous one; the previous frame is */
/* sampled there bilinearly with clamp to edge.  A point behind the previous */
/* camera keeps its own previous colour.                                    */
/* prev_rgba, out_rgba: [W*H][4] float32 (distinct); out_rgba8: [W*H] 8-bit  */
/* frame (as star_nt_composite); either output may be NULL, not both (a      */
/* display needs only the 8-bit frame); prev_z1: [W*H];                      */
/* vp_prev, vp_cur: device, 16 float64 row-major view-projections; ws: device */
/* scratch of STAR_NT_REPROJECT_WS_BYTES bytes (16-byte aligned) that holds  */
/* the call's offset coefficients (two launches: the coefficients from       */
/* VP_prev inv(VP_cur) in float64, then the per-pixel pass, whose sample      */
/* offsets are float-float, accurate to about 1e-9 pixel).  W, H <= 32768.   */
#define STAR_NT_REPROJECT_WS_BYTES 128
star_nt_status star_nt_reproject(const float *prev_rgba, const float *prev_z1,
                                 const double *vp_prev, const double *vp_cur, int32_t W,
                                 int32_t H, float *out_rgba, uint32_t *out_rgba8, void *ws,
                                 void *stream);

/* ------------------------------------------------------------------------ */
/* Comparison renderers of the evaluation (Sec. 4); not on the STAR-NT path. */

/* star_nt_unsorted_over -- a renderer without OIT: each pixel's materialised
 * fragments (star_nt_raster) composited with "over" in submission order
 * (increasing primitive id) over bg.  Its error against the A-buffer is the
 * E_random of the paper's Q measure.  rgb: [P][4] (colour, transmittance),
 * 16-byte aligned.  float32 arithmetic. */
star_nt_status star_nt_unsorted_over(const star_nt_frags *frags, const uint32_t *rgba8, int32_t W,
                                     int32_t H, const float *bg, float *rgb, void *stream);

/* star_nt_wboit -- weighted blended OIT (McGuire and Bavoil 2013), the
 * paper's baseline OIT method, in one pass over a full-resolution binned
 * target (bins from star_nt_raster, no fragment lists):
 * C = (sum (a c) w / max(sum a w, 1e-5)) (1 - T) + T C_b, T = prod (1 - a),
 * w = a clamp(10 / (1e-5 + (d/5)^2 + (d/200)^6), 1e-2, 3e3), d the view
 * depth recovered from NDC z with the projection's znear, zfar
 * (0 < znear < zfar).  rgba32f [P][4] (colour, T) and/or rgba8 [P]. */
star_nt_status star_nt_wboit(const star_nt_bins *bins, float znear, float zfar, const float *bg,
                             float *rgba32f, uint32_t *rgba8, void *stream);

/* ------------------------------------------------------------------------ */
/* Exact resolve and training of the tail network.                          */

/* star_nt_abuffer -- exact order-independent transparency, the ground truth
 * of the evaluation (Sec. 4): each pixel's materialised fragments (frags of a
 * W x H pass, from star_nt_raster) sorted by (z, primitive id) and
 * composited front to back over bg.  rgb: [P][4] (colour, total
 * transmittance) or NULL; tail: [P][4] the exact tail colour (fragments 3..N
 * composited among themselves, the quantity f(x) predicts in Eq. 4) and the
 * tail transmittance, or NULL.  float32 arithmetic. */
star_nt_status star_nt_abuffer(const star_nt_frags *frags, const uint32_t *rgba8, int32_t W,
                               int32_t H, const float *bg, float *rgb, float *tail, void *stream);

/* Training of the tail MLP with MSE and Adam (Sec. 3.3).  All buffers device
 * memory; ws: scratch of star_nt_train_ws_bytes(B) bytes (256-byte aligned).
 * star_nt_mse_grad: f, y [B][4] (rgb used) -> dy [B][4] = dL/df and the loss
 *   L = mean over B x 3 of (f - y)^2 (one float).
 * star_nt_mlp_backward: gradient of L with respect to the 771 parameters
 *   (w1, b1, w2, b2, w3, b3 order) for inputs x [B][8] float32 (STAR_NT_F32
 *   layout) and dy; the forward pass and the per-layer gradients are
 *   recomputed in float32 with w, and the weight and bias gradients, sums
 *   over the batch of products of a layer's input and its gradient, are one
 *   contraction on the tcgen05 tensor cores (bf16 operands split three ways,
 *   hi + mid + lo, fp32 accumulation: float32 accuracy); deterministic (fixed
 *   summation order).  d_status (device int32, may be NULL) receives
 *   STAR_NT_ERR_TIMEOUT if a tensor-core wait runs out; grad is then NaN.
 * star_nt_adam: bias-corrected Adam step `step` (from 1) on the float32
 *   master parameters; bf16_rounded (may be NULL) receives them rounded to
 *   bfloat16 precision, stored as float32 (the weights of the next forward). */
size_t star_nt_train_ws_bytes(int64_t B);  /* serves both networks' backward passes */
star_nt_status star_nt_mse_grad(const float *f, const float *y, int64_t B, float *dy, float *loss,
                                void *ws, size_t ws_bytes, void *stream);
/* star_nt_wmse_grad: star_nt_mse_grad with a weight per sample, w [B] float32:
 *   L = sum_i w_i |f_i - y_i|^2 / (3B), dy_i = 2 w_i (f_i - y_i) / (3B).  With
 *   w_i = T_2^2 of the pixel, L is the error of the composited frame (Eq. 4
 *   adds T_2 f), so the network is fitted where its output is visible. */
star_nt_status star_nt_wmse_grad(const float *f, const float *y, const float *w, int64_t B, float *dy,
                                 float *loss, void *ws, size_t ws_bytes, void *stream);
star_nt_status star_nt_mlp_backward(const star_nt_mlp *w, const float *x, const float *dy,
                                    int64_t B, float *grad, void *ws, size_t ws_bytes,
                                    int32_t *d_status, void *stream);
star_nt_status star_nt_adam(float *params, const float *grad, float *m, float *v, int64_t n,
                            int64_t step, float lr, float beta1, float beta2, float eps,
                            float *bf16_rounded, void *stream);
/* star_nt_gather_rows: the minibatch rows of a training step (Sec. 3.3 trains
 * on randomly drawn samples): dst[i] = src[idx[i]] for i < n, rows of
 * row_bytes bytes (a multiple of 4); src [n_src] rows, idx [n] int64, all
 * device memory (src, dst 4-byte aligned, idx 8-byte aligned).  An index
 * outside [0, n_src) writes a zero row and STAR_NT_ERR_ARG to d_status (device
 * int32, may be NULL). */
star_nt_status star_nt_gather_rows(const void *src, int64_t n_src, int32_t row_bytes, const int64_t *idx,
                                   int64_t n, void *dst, int32_t *d_status, void *stream);

/* ------------------------------------------------------------------------ */
/* The DFAOIT comparison network (Sec. 3.3; Table 2's "Inf. DFAOIT" column):  */
/* the original method predicts the whole transparency colour C_t from the    */
/* features the paper lists for it, with ReLU hidden layers of 32 and 16      */
/* units and a sigmoid output, and composites C = C_t + C_b prod(1 - a_i).    */
/* The list (the exact blend of the two front fragments, the average colour  */
/* and average opacity of the remaining n - 2 fragments, their accumulated    */
/* premultiplied colour, the fragment count) has eleven scalars although the */
/* text counts ten; all eleven are inputs here:                              */
/*   x[0..2]  a1 c1 + (1 - a1) a2 c2                                          */
/*   x[3..5]  sum_tail c_i / (n - 2)      x[6]  sum_tail a_i / (n - 2)        */
/*   x[7..9]  sum_tail a_i c_i            x[10] kappa_n n                     */
/*   x[11]    1 when the pixel has a fragment (else f = 0), x[12..15] = 0     */
/* with the fragments in (z, primitive id) order and the tail means 0 when   */
/* n <= 2.                                                                    */

/* star_nt_build_inputs_dfaoit: one full-resolution pass over bins (binned by
 * star_nt_raster at W x H) writing x ([W*H][16] float32, or bfloat16 256-byte
 * aligned: out->x_dtype) and front = (T_all C_b, 1) per pixel (out->front,
 * [W*H][4]), so that star_nt_composite(front, f) gives C_t + T_all C_b.
 * layers1 (optional) receives id1 and z1. */
star_nt_status star_nt_build_inputs_dfaoit(const star_nt_scene *scene, const star_nt_bins *bins,
                                           const star_nt_layers *layers1, int32_t W, int32_t H,
                                           const star_nt_params *params,
                                           const star_nt_features *out, int32_t *d_status,
                                           void *stream);

/* star_nt_infer_dfaoit: the network on P rows of x ([P][16] float32, or
 * bfloat16 on the tcgen05 tensor cores: two TMA boxes per 128-row tile, the
 * bias inside a second K = 16 MMA) into f ([P][4] float32, rgb and 0); w
 * holds w1 [32][11], b1 [32], w2 [16][32], b2 [16], w3 [3][16], b3 [3]. */
star_nt_status star_nt_infer_dfaoit(const star_nt_mlp *w, int32_t x_dtype, const void *x, float *f,
                                    int64_t P, int32_t *d_status, void *stream);

/* star_nt_dfaoit_backward: star_nt_mlp_backward for this network: gradient of
 * L with respect to its 963 parameters (w1, b1, w2, b2, w3, b3 order) for x
 * [B][16] float32 and dy [B][4]; the sigmoid's derivative f (1 - f);
 * ws of star_nt_train_ws_bytes(B) bytes; the same tensor-core contraction
 * and d_status. */
star_nt_status star_nt_dfaoit_backward(const star_nt_mlp *w, const float *x, const float *dy,
                                       int64_t B, float *grad, void *ws, size_t ws_bytes,
                                       int32_t *d_status, void *stream);

/* ------------------------------------------------------------------------ */
/* Context: the whole STAR-NT step of Fig. 1 through one call.               */
/*                                                                           */
/* A context belongs to one device.  It holds the method's parameters, the   */
/* frame options below, the launch tuning of the persistent pass launches    */
/* (star_nt_tuning; star_nt_tune chooses it on the caller's own workload),   */
/* and a second stream with two events of its own.  The caller allocates one */
/* device workspace of star_nt_workspace_size bytes for a frame size and a   */
/* largest scene and binds it; it then holds every buffer the frame path     */
/* keeps between frames (the three pass workspaces, the pass planes, the     */
/* quadtree masks and state, the reprojection scratch), so a step needs no   */
/* other buffer than its inputs and outputs and one captured CUDA graph      */
/* replays every frame.  The library allocates no device memory; the context */
/* itself is host memory plus a stream and two events, created by            */
/* star_nt_create on the device and released by star_nt_destroy.  A context  */
/* is not thread-safe: one thread at a time, one workspace, one frame size.  */

typedef struct star_nt_ctx star_nt_ctx;

/* Options of the frame path.  Defaults (star_nt_default_frame_options):
 * mlp_type STAR_NT_BF16, merge scales 1 (a reduced pass is merged into pass
 * 1 only at full size, as Eq. 2 sizes it), fuse_passes 1. */
typedef struct {
    int32_t mlp_type;     /* the resolve's MLP operand type, as star_nt_resolve_mlp */
    float merge_scale2;   /* star_nt_target.merge_scale of pass 2, in (0, 1] */
    float merge_scale3;   /* ... of pass 3 */
    int32_t fuse_passes;  /* BF16: with every pass at full size the pass launch
                             produces the frame (star_nt_geometry_passes_resolve) */
} star_nt_frame_options;
void star_nt_default_frame_options(star_nt_frame_options *o);

/* star_nt_create: a context on `device` with params (NULL: the defaults) and
 * options (NULL: the defaults).  STAR_NT_ERR_ARG for an invalid device,
 * parameters or options; STAR_NT_ERR_CUDA when no CUDA device is usable.
 * star_nt_destroy waits for the context's side stream and releases it. */
star_nt_status star_nt_create(int32_t device, const star_nt_params *params,
                              const star_nt_frame_options *options, star_nt_ctx **out);
star_nt_status star_nt_destroy(star_nt_ctx *ctx);

/* Bytes of the device workspace of frames of W x H pixels with up to T
 * triangles (W, H <= 16384).  Each pass workspace holds max(2^20, 96 T)
 * (triangle, tile) pairs; a scene that needs more raises
 * STAR_NT_ERR_CAPACITY in the frame's status word. */
star_nt_status star_nt_workspace_size(const star_nt_ctx *ctx, int32_t W, int32_t H, int32_t T,
                                      size_t *bytes);

/* Binds a workspace (256-byte aligned, at least star_nt_workspace_size
 * bytes) to the context for frames of W x H and up to T triangles, and
 * enqueues its initialisation on `stream`: the first frame runs every pass
 * at full size, every quadtree leaf at level 0.  Binding again starts a new
 * sequence. */
star_nt_status star_nt_bind_workspace(star_nt_ctx *ctx, int32_t W, int32_t H, int32_t T, void *ws,
                                      size_t ws_bytes, void *stream);

/* Cameras of one step (device memory).  vp: float32[16] view-projection of
 * the real frame (as star_nt_target.view_proj); vp64: the same camera in
 * float64 (the reprojection's source camera); vp64_interp: float64[16]
 * camera of the interpolated frame, or NULL for a step without one. */
typedef struct {
    const float *vp;
    const double *vp64;
    const double *vp64_interp;
} star_nt_cameras;

/* Outputs of one step: the real frame (both required: the reprojection and
 * the quadtree read them) and the interpolated frame (either or both when
 * vp64_interp is given), layouts as star_nt_resolve and star_nt_reproject. */
typedef struct {
    float *rgba32f;
    uint32_t *rgba8;
    float *interp_rgba32f;
    uint32_t *interp_rgba8;
} star_nt_frame_out;

/* star_nt_frame: one STAR-NT step (Fig. 1) on `stream`: the real frame
 * (star_nt_raster_passes of pass 1 at W x H and of passes 2 and 3 at the
 * sizes the quadtree chose on the previous frame; the pass launch; the
 * resolve: upscale, network, composite), then the interpolated frame
 * reprojected from it (star_nt_reproject, on the context's side stream,
 * forked from and joined back to `stream`) beside the quadtree update of
 * Sec. 3.1-3.2 that sets the next frame's pass sizes.  The call enqueues
 * only; the step is complete when `stream` reaches its end.  It can be
 * captured into a CUDA graph on `stream` (fixed addresses, the fork and join
 * through the context's events).  Device-side conditions go to d_status. */
star_nt_status star_nt_frame(star_nt_ctx *ctx, const star_nt_scene *scene, const star_nt_mlp *w,
                             const star_nt_cameras *cams, const star_nt_frame_out *out,
                             int32_t *d_status, void *stream);

/* star_nt_tune: chooses the context's launch tuning on its current frame
 * state (call it after a few frames, so that the quadtree's pass sizes are
 * representative): every candidate tile shape and residency of the
 * persistent pass launch is timed with CUDA events over ten pass launches,
 * the fastest kept; then, with BF16 and fuse_passes, the raster, pass launch
 * and resolve are timed with the pass launch producing the frame and with
 * the separate resolve, and the faster kept when the current frame has both
 * reduced passes merged (otherwise the pass launch returns at once either
 * way, the timings do not compare the two, and the pass launch keeps
 * producing the frames that merge).  Synchronises `stream` (not
 * allowed inside a capture: STAR_NT_ERR_ARG); writes the outputs of frames
 * it renders; leaves the quadtree state unchanged.  report may be NULL. */
#define STAR_NT_TUNE_CANDIDATES 9
typedef struct {
    star_nt_tuning candidates[STAR_NT_TUNE_CANDIDATES];
    float passes_ms[STAR_NT_TUNE_CANDIDATES];  /* mean ms of one pass launch */
    float frame_ms[2];                         /* raster + passes + resolve: [0] separate resolve,
                                                  [1] the pass launch produces the frame */
    star_nt_tuning chosen;
    int32_t fuse_passes;
    int32_t frame_merged;                      /* 1: both reduced passes merged in the timed frame */
} star_nt_tune_report;
star_nt_status star_nt_tune(star_nt_ctx *ctx, const star_nt_scene *scene, const star_nt_mlp *w,
                            const star_nt_cameras *cams, const star_nt_frame_out *out,
                            int32_t *d_status, void *stream, star_nt_tune_report *report);

/* The context's tuning (either pointer may be NULL), and setting it by hand
 * (STAR_NT_ERR_ARG for a tuning star_nt_geometry_passes rejects). */
star_nt_status star_nt_ctx_tuning(const star_nt_ctx *ctx, star_nt_tuning *tuning,
                                  int32_t *fuse_passes);
star_nt_status star_nt_ctx_set_tuning(star_nt_ctx *ctx, const star_nt_tuning *tuning,
                                      int32_t fuse_passes);

/* Device addresses, inside the bound workspace, of the pass state the
 * quadtree leaves for the next frame, the quadtree masks, and the real
 * frame's nearest-layer ids and depths (any pointer may be NULL). */
star_nt_status star_nt_ctx_pass_state(const star_nt_ctx *ctx, star_nt_pass_state **state,
                                      uint32_t **masks, int32_t **id1, float **z1);

#ifdef __cplusplus
}
#endif
#endif /* STAR_NT_H */

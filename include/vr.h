/*
 * vr.h -- C ABI of the GB300 (sm_103a) ray-casting volume renderer for
 * spectral data cubes.
 *
 * The method is the ray-casting renderer of Hassan, Fluke & Barnes,
 * "Distributed GPU Volume Rendering of ASKAP Spectral Data Cubes":
 *   - Abstract and Sec. 1: real-time ray casting of HI spectral cubes larger
 *     than one machine's memory, by decomposing the cube;
 *   - Sec. 3: a static render of the current orientation at a user-defined
 *     output size, e.g. the 5 x 5 wall of 1920 x 1080 panels (9600 x 5400).
 * The paper prints no formulas.  The operations below are the standard
 * front-to-back emission-absorption ray caster; each entry point states the
 * exact discretisation it computes.
 *
 * Conventions for every entry point:
 *   - The caller owns every pointer it passes.  The library copies the cube,
 *     the transfer function and the cameras, and keeps no caller pointer after
 *     an entry point returns.
 *   - "stream" is a cudaStream_t (NULL = the legacy default stream).  Device
 *     outputs are written in stream order and are valid once the caller has
 *     synchronised that stream.
 *   - No C++ exception crosses this boundary.  Every failure is a status code;
 *     vr_last_error() returns a human-readable message for the last failing
 *     call on a context.  An asynchronous CUDA error surfaces as VR_ERR_CUDA
 *     on a later call.
 *   - A context is bound to one device.  Entry points make that device current
 *     for their duration and restore the caller's current device on return.
 *   - Calls on one context are not thread-safe; use one context per thread.
 */
#ifndef VR_H
#define VR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VR_ABI_VERSION 1

typedef enum {
    VR_OK = 0,
    VR_ERR_INVALID_ARG = 1, /* a pointer, size or enum is out of range      */
    VR_ERR_STATE = 2,       /* e.g. render before a cube/camera/TF is set  */
    VR_ERR_OOM = 3,         /* device or pinned-host allocation failed     */
    VR_ERR_CUDA = 4,        /* a CUDA runtime call failed                  */
    VR_ERR_TIMEOUT = 5,     /* a bounded host wait expired                 */
    VR_ERR_IO = 6,          /* a caller-supplied data source failed        */
    VR_ERR_INTERNAL = 7,    /* a device-side check recorded an error       */
    VR_ERR_UNSUPPORTED = 8  /* a valid request the chosen path cannot serve */
} vr_status;

/* Storage type of the bricked cube.  Sampling and compositing are FP32. */
typedef enum { VR_F32 = 0, VR_F16 = 1, VR_BF16 = 2 } vr_dtype;

/* VR_COMPOSITE: front-to-back "over" with early termination, premultiplied
 * RGBA output.  VR_MIP: maximum-intensity projection, output TF(max) as
 * straight RGBA. */
typedef enum { VR_COMPOSITE = 0, VR_MIP = 1 } vr_mode;

/* Which kernel family renders.
 * VR_PATH_RAY: image order -- one thread per ray marches brick by brick
 *   (all modes; early termination).
 * VR_PATH_BRICK: object order -- the cube is streamed once through shared
 *   memory in 32^3 cells (TMA-staged) and every ray segment crossing a cell is
 *   marched there; partial results are folded per pixel.  VR_MIP only; needs
 *   bricks of at least 32 voxels.
 * VR_PATH_SORTLAST: the paper's decomposition into parts rendered apart and
 *   combined.  Composite: every brick renders a partial image (C, T) of the
 *   samples it owns, starting from T = 1, on its screen footprint, and the
 *   partial images are folded per pixel front to back in visibility order
 *   (ascending sum |b - e| over axes, e the eye's brick; sign-weighted brick
 *   sum for orthographic views).  Early termination does not apply: the result
 *   is the composite with ert disabled.  A brick's partial image is built from
 *   its cells staged in shared memory, one pass per visibility key of the cells
 *   within the brick (tables of more than 256 entries: whole-brick marches from
 *   global memory, the same image up to rounding).  VR_MIP: as VR_PATH_BRICK.
 * VR_PATH_LAYERED: composite by bricks, one visibility layer per launch, each
 *   pixel's running (C, T) carried from layer to layer with per-sample early
 *   termination (the same image as VR_PATH_RAY); bricks of terminated pixels
 *   are skipped.  VR_MIP: as VR_PATH_BRICK.
 * Both read back per-view layer sizes (a host synchronisation), so graph mode
 * does not apply to them.
 * VR_PATH_AUTO (default): VR_PATH_BRICK for VR_MIP when available, else
 *   VR_PATH_RAY.  Every path computes the same discretisation. */
typedef enum {
    VR_PATH_AUTO = 0,
    VR_PATH_RAY = 1,
    VR_PATH_BRICK = 2,
    VR_PATH_SORTLAST = 3,
    VR_PATH_LAYERED = 4
} vr_path;

/*
 * Camera.  Pixel (px, py), py = 0 the top row, has window coordinates
 *     u = win[0] + (px + 1/2) (win[1] - win[0]) / width
 *     v = win[3] - (py + 1/2) (win[3] - win[2]) / height
 * type 0 (orthographic): origin eye + u right + v up, direction fwd.
 * type 1 (perspective):  origin eye, direction fwd + u right + v up
 *     (win is a tangent-space window: an off-axis sub-window of a larger
 *     view, such as one panel of a tiled wall, is just a smaller win).
 * Directions are normalised; samples lie at t = k * step along the unit
 * direction from the origin, k integer (Sec. 3's "same orientation, other
 * output size" is the same camera with another width/height).
 * All cameras passed together must have the same width and height.
 * Every component of eye, right, up, fwd and win must be finite and at most
 * 1e9 in magnitude, and right, up, fwd must span space (VR_ERR_INVALID_ARG
 * otherwise).  Rays are set up in
 * float-float arithmetic (about 44 bits): a sample up to 1e6 voxels from the
 * ray origin lies within ~1e-7 voxel of its exact position.
 */
typedef struct {
    int32_t type;
    int32_t pad_;
    double eye[3], right[3], up[3], fwd[3];
    double win[4]; /* l, r, b, t */
    int32_t width, height;
} vr_camera;

typedef struct {
    int32_t brick;  /* interior brick edge in voxels, power of two in [8, 256];
                       default 128.  Bricks carry a 1-voxel ghost layer.    */
    int32_t flags;  /* VR_OPT_* bits; default 0                            */
    double step;    /* sample spacing along the ray in voxels, > 0; default 0.5 */
    double ert;     /* early termination once accumulated alpha >= ert after a
                       sample; default 0.99; a value > 1 disables it          */
} vr_options;

/* vr_options.flags: keep one brick store only.  By default vr_load_cube also
 * keeps, for FP16 and BF16 stores, a copy of the store shifted by one element
 * along x when it fits in half of the free device memory, so that the
 * image-order marcher's composite reads each pair of x-neighbours of a
 * trilinear fetch with one aligned 32-bit load. */
#define VR_OPT_SINGLE_STORE 1

typedef struct vr_ctx vr_ctx;

/* Layout facts of the loaded cube (for byte accounting by callers). */
typedef struct {
    int64_t nx, ny, nz;      /* voxels                                    */
    int32_t nbx, nby, nbz;   /* bricks per axis                           */
    int32_t brick;           /* interior edge                             */
    int32_t pitch;           /* x pitch of a stored brick row, elements   */
    int32_t dtype;           /* vr_dtype                                  */
    int64_t brick_bytes;     /* bytes of one stored brick slot            */
    int64_t store_bytes;     /* bytes of the whole brick store, with its
                                x-shifted copy when one is kept           */
} vr_cube_info;

/* Fill *opt with the defaults (brick 128, step 0.5, ert 0.99). */
void vr_default_options(vr_options* opt);

/* Human-readable name of a status code (static storage). */
const char* vr_status_string(vr_status s);

/* Create a context on CUDA device `device`.  opt may be NULL (defaults).
 * Allocates the scheduler's small device scratch.  *out is set to NULL on
 * failure. */
vr_status vr_create(vr_ctx** out, int device, const vr_options* opt);

/* Free a context and everything it owns.  NULL is accepted.  The caller must
 * have synchronised every stream on which it used the context. */
vr_status vr_destroy(vr_ctx* ctx);

/*
 * Load a cube of nx*ny*nz float32 values, x fastest (RA x Dec x channel),
 * from host memory (src_on_device = 0) or device memory of the context's
 * device (src_on_device = 1), into a device brick store of `storage` type:
 * bricks of brick^3 interior voxels plus a 1-voxel ghost layer (edge values
 * replicated at the cube faces), row pitch padded to 16 bytes, converted
 * with round-to-nearest-even.  Replaces any earlier cube.  Host sources are
 * copied in slabs of brick + 2 planes; the call returns after the copy has
 * been issued on `stream` and a host source may be freed once it returns.
 * Errors: VR_ERR_INVALID_ARG (NULL src, any n <= 0, bad storage),
 * VR_ERR_OOM, VR_ERR_CUDA.
 */
vr_status vr_load_cube(vr_ctx* ctx, const float* src, int src_on_device, int64_t nx,
                       int64_t ny, int64_t nz, vr_dtype storage, void* stream);

/*
 * Set the transfer function: n (2 <= n <= 1024) straight RGBA float32 entries
 * in HOST memory, node-centred over [vmin, vmax] (entry 0 at vmin, entry n-1
 * at vmax), linearly interpolated, clamped outside the range.  vmax > vmin.
 */
vr_status vr_set_transfer_function(vr_ctx* ctx, const float* rgba, int n, float vmin,
                                   float vmax);

/* Set ncams (1..4096) cameras from HOST memory, all of one width x height
 * (width, height <= 65536, width * height <= 2^30, ncams * width * height
 * <= 2^40; VR_ERR_INVALID_ARG otherwise). */
vr_status vr_set_camera(vr_ctx* ctx, const vr_camera* cams, int ncams);

/*
 * Render every camera into out_rgba (DEVICE, ncams x height x width x 4
 * float32, camera-major, rows top-down).  Per pixel:
 *   samples p_k = o + k step d for k in [ceil(t_near/step), ceil(t_far/step)),
 *   (t_near, t_far) the slab interval of the box [0,nx]x[0,ny]x[0,nz] with
 *   t >= 0; trilinear interpolation of voxels centred at integer + 1/2,
 *   clamped to the edge; transfer function as set.
 *   VR_COMPOSITE: C += T a rgb, T *= (1 - a), stop after the sample at which
 *     1 - T >= ert; output (C, 1 - T).  The image-order path skips a brick
 *     whose stored maximum maps to table nodes of opacity 0 (the image is
 *     unchanged; its samples are not counted as executed).
 *   VR_MIP: m = max_k v(p_k); output TF(m) (straight), or 0 with no samples.
 * out_max (DEVICE, ncams x height x width float32, may be NULL) receives m
 * in VR_MIP mode (-inf with no samples); it is ignored in VR_COMPOSITE mode.
 * out_rgba must be 16-byte aligned and out_max 4-byte aligned.  The brick
 * path uses out_max (when given) as its per-pixel accumulator.
 * Errors: VR_ERR_STATE if no cube, TF or camera is set; VR_ERR_INVALID_ARG
 * for a NULL or misaligned output or bad mode; VR_ERR_INTERNAL if a device-side
 * wait of an earlier call gave up (reported once, then cleared).
 */
vr_status vr_render(vr_ctx* ctx, vr_mode mode, float* out_rgba, float* out_max, void* stream);

/*
 * Adjoint (reverse-mode derivative) of vr_render for the current cube, table
 * and cameras.  dL_dimg (DEVICE, ncams x height x width x 4 float32, the
 * layout vr_render writes) holds dL/dI of a scalar loss L with respect to the
 * image of `mode`.  Outputs (DEVICE, overwritten, not accumulated):
 *   dL_dtf  (n x 4 float32): dL/d(table entry, channel), through the
 *           node-centred interpolation (zero slope where the lookup clamps);
 *   dL_dvol (nx*ny*nz float32, x fastest, may be NULL): dL/d(stored voxel
 *           value), through the trilinear weights (clamped corners included).
 * Composite: C = sum_k T_k a_k c_k and A = 1 - T_n over the executed samples
 * (termination is not differentiated); the forward is recomputed segment by
 * segment from per-segment checkpoints of T and swept back to front.  MIP:
 * the gradient reaches the first sample that attains the maximum.
 * Table partials are FP32 per block and summed in FP64.
 * Errors as vr_render; VR_ERR_UNSUPPORTED (reported by the next call) if a
 * ray needs more than 320 checkpoint segments (about 10 000 samples).
 */
vr_status vr_render_backward(vr_ctx* ctx, vr_mode mode, const float* dL_dimg, float* dL_dtf,
                             float* dL_dvol, void* stream);

/* Launch shape of the kernels (chosen by vr_autotune or set directly).
 *   tile_w x tile_h: pixels of one warp work item of the image-order path
 *                    (tile_w * tile_h = 32: one ray per lane);
 *   block:           threads per CTA of the image-order path (64, 128, 256);
 *   group:           lanes per ray segment in the brick path (4, 8, 16), i.e.
 *                    32 / group rays per warp.
 * Defaults 8 x 4, 256, 8.  Results do not depend on the tuning. */
typedef struct {
    int32_t tile_w, tile_h;
    int32_t block;
    int32_t group;
} vr_tuning;

vr_status vr_get_tuning(const vr_ctx* ctx, vr_tuning* out);
vr_status vr_set_tuning(vr_ctx* ctx, const vr_tuning* tuning);

/* Autotuner: renders `mode` for the current cube and cameras with every
 * candidate launch shape of the path that serves it (5 tile shapes x 3 block
 * sizes for the image-order path, 3 group sizes for the brick path), reps
 * timed renders each after one warm-up (CUDA events on `stream`), keeps the
 * fastest in the context and returns it (best, best_ms may be NULL).
 * scratch_rgba: DEVICE output of ncams x height x width x 4 float32.  Blocks
 * until the timings are in. */
vr_status vr_autotune(vr_ctx* ctx, vr_mode mode, float* scratch_rgba, int reps, vr_tuning* best,
                      double* best_ms, void* stream);

/* Graph mode (enable != 0): each vr_render records its launches into a CUDA
 * graph on a private stream, updates the context's cached executable graph
 * with it (new cameras, table and output pointers reach the graph this way)
 * and launches that graph on the caller's stream: one launch per render
 * however many kernels it takes (the 25 panels of a wall, for instance).
 * Profiling events (vr_set_kernel_events) are not recorded in graph mode. */
vr_status vr_set_graph(vr_ctx* ctx, int enable);

/* Select the kernel family used by later vr_render calls (see vr_path).
 * A path that cannot serve a request makes vr_render return
 * VR_ERR_UNSUPPORTED. */
vr_status vr_set_path(vr_ctx* ctx, vr_path path);

/* Optional DEVICE counter (uint64) to which vr_render adds the number of
 * samples it executed (VR_PATH_RAY only); NULL switches counting off. */
vr_status vr_set_sample_counter(vr_ctx* ctx, unsigned long long* device_counter);

/* Failure-detection self-test.  Runs, on `stream`, one thread that waits with
 * the brick pass's bounded mbarrier wait (its 2 s bound shortened to 1 ms) on a barrier
 * phase that no copy will complete, so that the wait gives up and records the
 * device status word exactly as an expired wait of a render would; then
 * synchronises the stream.  Returns VR_OK once the status word is set (the
 * next vr_render or vr_render_mip_noalloc reports VR_ERR_INTERNAL once and
 * clears it; the context stays usable), VR_ERR_INTERNAL if the wait did not
 * expire, VR_ERR_CUDA on a launch error. */
vr_status vr_selftest_wait_timeout(vr_ctx* ctx, void* stream);

/* Profiling hook: when both are non-NULL, vr_render records the CUDA events
 * `start` and `stop` (cudaEvent_t, created by the caller) on its stream just
 * before the first and just after the last launch of its dominant kernel (the
 * ray marcher on VR_PATH_RAY, the staged brick pass on VR_PATH_BRICK), so that
 * cudaEventElapsedTime gives that kernel's device time.  NULL, NULL turns it
 * off. */
vr_status vr_set_kernel_events(vr_ctx* ctx, void* start, void* stop);

/*
 * Allocation-free MIP render.  The paper has no counterpart: this is a
 * service to callers of this library that cannot allocate device memory while
 * they render -- real-time loops that must not meet the device-wide
 * synchronisation cudaMalloc can imply, and programs whose device memory is
 * owned by another allocator or held to a fixed budget, so that a library
 * allocating behind their back would break it.  vr_render's brick path
 * allocates its per-pixel scratch on first use of a larger image; this call
 * instead takes its scratch (per-pixel sample ranges, per-pixel running
 * maxima, the work counter) from one fixed array compiled into the library,
 * VR_NOALLOC_MAX_PIXELS * 12 bytes + 256 (24 MiB), present on every device
 * that loads the library until the process exits; the per-view cell list it
 * also needs belongs to the context and is allocated once by vr_load_cube.
 * It calls no cudaMalloc, cudaFree or other allocating routine.
 * Result: the same as vr_render(ctx, VR_MIP, out_rgba, out_max, stream) on
 * VR_PATH_BRICK (same outputs, layouts and alignment rules).
 * Limits: every camera must have at most VR_NOALLOC_MAX_PIXELS pixels
 * (width * height), else VR_ERR_INVALID_ARG; bricks of at least 32 voxels,
 * else VR_ERR_UNSUPPORTED.
 * Set-up: the first call on each device looks up the device address of the
 * scratch array (with that device current) and keeps it for the life of the
 * process; make that first call before any stream capture.  A device reset
 * (cudaDeviceReset) after that first call is not supported: the kept address
 * would then be stale.
 * Sharing: every call on a device uses the same scratch array, which keeps the
 * last call's contents; each call rewrites what it reads before reading it.
 * Calls whose GPU work overlaps (on different streams, or from several
 * threads, without ordering between them) race on the array and produce wrong
 * images: order them on one stream or synchronise between them.
 */
#define VR_NOALLOC_MAX_PIXELS (1 << 21)
vr_status vr_render_mip_noalloc(vr_ctx* ctx, float* out_rgba, float* out_max, void* stream);

/*
 * Out-of-core cubes (Abstract, Sec. 1: cubes larger than one machine's memory).
 * The cube is never held whole: bricks are produced on demand by a caller
 * callback, copied through page-locked staging (double-buffered) on a side
 * stream into a fixed HBM brick cache of `cache_bytes`, evicted least recently
 * used, and the render waits on CUDA events for the bricks it needs.
 *   VR_MIP renders the visible bricks in cache-sized batches (maxima folded
 *     across batches);
 *   VR_COMPOSITE renders layer by layer in visibility order with each pixel's
 *     running (C, T) carried and per-sample early termination; a brick whose
 *     every footprint pixel has terminated is neither fetched nor rendered.
 * The callback fills dst (float32, x fastest) with the cube values of the
 * region [x0, x0+sx) x [y0, y0+sy) x [z0, z0+sz) and returns 0, or nonzero
 * on failure (the render then returns VR_ERR_IO).  It is called from the
 * thread that calls vr_render, one region at a time.  The library keeps fn and
 * user (the one exception to keeping no caller pointer): both must stay valid
 * until another cube is loaded or the context is destroyed.
 * Host waits (events, callbacks) are bounded by a deadline (default 120 s,
 * vr_set_stream_timeout); on expiry the call returns VR_ERR_TIMEOUT and the
 * context stays usable.  vr_render_backward and graph mode do not apply.
 */
typedef int (*vr_region_fn)(void* user, int64_t x0, int64_t y0, int64_t z0, int64_t sx,
                            int64_t sy, int64_t sz, float* dst);

typedef struct {
    uint64_t bricks_fetched;  /* bricks produced and uploaded            */
    uint64_t bricks_culled;   /* bricks skipped behind terminated rays    */
    uint64_t bytes_h2d;       /* bytes copied host -> device              */
    uint64_t batches;         /* render batches (cache fills)             */
    double generate_s;        /* host time inside the callback            */
    double wait_s;            /* host time waiting on device events       */
} vr_stream_stats;

vr_status vr_load_cube_streamed(vr_ctx* ctx, vr_region_fn fn, void* user, int64_t nx, int64_t ny,
                                int64_t nz, vr_dtype storage, uint64_t cache_bytes);
vr_status vr_get_stream_stats(const vr_ctx* ctx, vr_stream_stats* out);
vr_status vr_set_stream_timeout(vr_ctx* ctx, double seconds);

/*
 * Image pyramid of a render, for viewers that show a high-resolution static
 * render (Sec. 3) at several zoom levels, cut into tiles.  rgba (DEVICE,
 * height x width x 4 float32, premultiplied RGBA such as an image of
 * vr_render, 16-byte aligned) is level 0.  Level l+1 is ceil(W_l/2) x
 * ceil(H_l/2) and its pixel (x, y) is the mean of the pixels (2x+i, 2y+j),
 * i, j in {0, 1}, of level l that lie inside level l (one, two or four).
 * out (DEVICE, 16-byte aligned) receives levels 1 .. L-1 one after the other,
 * down to 1 x 1, 4 floats a pixel; each level row-major (tile = 0) or as
 * ceil(W/tile) x ceil(H/tile) tiles of tile x tile pixels (tile a power of two
 * in [8, 4096]), tiles row-major and pixels row-major inside a tile, with
 * zeros where an edge tile passes the level.  Stream-ordered on `stream`.
 * vr_pyramid_layout returns L (levels counting level 0) and the number of
 * floats out must hold (0 for a 1 x 1 image); either pointer may be NULL.
 * Errors: VR_ERR_INVALID_ARG for sizes outside [1, 2^20], a bad tile, NULL
 * or misaligned images.  The paper's file formats are not written here.
 */
vr_status vr_pyramid_layout(int32_t width, int32_t height, int32_t tile, int32_t* levels, int64_t* floats);
vr_status vr_image_pyramid(vr_ctx* ctx, const float* rgba, int32_t width, int32_t height, int32_t tile,
                           float* out, void* stream);

/*
 * Catalogue overlay (Sec. 2: a source finder's detections, given as bounding
 * cubes, are superimposed as wireframe boxes on the volume rendering, one
 * colour per catalogue).  Draws the 12 edges of every box over the images
 * rgba (DEVICE, ncams x height x width x 4 float32, premultiplied, 16-byte
 * aligned; modified in place) of the cameras cams (HOST, ncams cameras of one
 * size, the ones the images were rendered with).  boxes (HOST, nbox x 6
 * double): x0, y0, z0, x1, y1, z1 in voxel units (the cube spans [0, n]);
 * colours (HOST, nbox x 4 float): straight RGBA of each box.
 * An edge is projected through the camera (the inverse of the mapping in
 * vr_camera; for a perspective camera the part closer than 1e-3 along fwd is
 * clipped away), to continuous pixel coordinates with pixel centres at
 * integers, clipped to the image grown by one pixel, and walked with n + 1
 * evenly spaced points, n = max(1, ceil(max(|dx|, |dy|))), each marking the
 * pixel it rounds to.  A marked pixel takes the colour (c, a) of the highest
 * box index that marks it: C = a c + (1 - a) C, A = a + (1 - a) A.  Show or
 * hide groups of boxes by what is passed.  Stream-ordered on `stream`; the
 * host arrays may be reused when the call returns.
 * Errors: VR_ERR_INVALID_ARG for NULL or misaligned arrays, cameras of
 * different sizes, a bad camera type, an empty window, a non-finite camera
 * or box value, or more than 2^30 pixels per image.
 */
vr_status vr_overlay_boxes(vr_ctx* ctx, const vr_camera* cams, int32_t ncams, const double* boxes, int64_t nbox,
                           const float* colours, float* rgba, void* stream);

/*
 * Object-space sort-last across ranks (Abstract and Sec. 1: a cube larger than one
 * node's memory is split into parts that are rendered separately, and the parts'
 * images are combined).  A rank renders the partial images of the bricks it holds
 * (vr_sortlast_partials); the partials are exchanged so that the owner of a band
 * of image rows holds every partial that covers it, whoever rendered it; the owner
 * folds them in visibility order (vr_sortlast_fold).  The exchange itself is the
 * caller's (the Python package's dist module moves them with torch.distributed);
 * these calls only produce and consume partial images.  Both act on camera 0 and
 * require exactly one camera, an in-core cube and a transfer function
 * (VR_ERR_STATE otherwise).
 *
 * A partial image covers the brick's footprint (the conservative pixel rectangle of
 * its box), float4 per pixel, row-major over the rectangle:
 *   VR_COMPOSITE: (C0, C1, C2, T): the brick's samples of the pixel's ray
 *     composited front to back from T = 1, no termination (premultiplied colour,
 *     transmittance);
 *   VR_MIP: (m, 0, 0, 0): the largest sample value, -inf without samples.
 */
typedef struct {
    int32_t brick;          /* linear brick id, (bz * nby + by) * nbx + bx              */
    int32_t key;            /* visibility key: ascending is front to back (reading R9)  */
    int32_t x0, y0, x1, y1; /* pixel rectangle, inclusive; empty when x1 < x0          */
    int64_t offset;         /* float4 index of the rectangle's first pixel in the buffer */
} vr_footprint;

/* Footprints and partial images of the listed bricks (host array of n distinct
 * linear ids; n = 0, a rank that holds no brick, renders nothing).  foot (host, n entries) receives the footprint of bricks[i]
 * at index i, offsets packed from 0 in list order; *needed the float4 count of
 * all of them.  partial (device, 16-byte aligned, capacity float4) receives the
 * images; NULL only sizes the call (foot and *needed are still filled).
 * Errors: VR_ERR_INVALID_ARG for a bad or repeated id, a NULL foot or needed, or
 * a capacity below *needed; VR_ERR_STATE as above. */
vr_status vr_sortlast_partials(vr_ctx* ctx, vr_mode mode, const int32_t* bricks, int32_t n,
                               vr_footprint* foot, float* partial, int64_t capacity, int64_t* needed,
                               void* stream);

/* Fold n partial images (device buffer partial of capacity float4; host
 * footprints foot, distinct brick ids, any order) over the image rows [y0, y1) of
 * camera 0: per pixel, the partials covering it in ascending (key, brick):
 * VR_COMPOSITE: C += T C_b, T *= T_b from (0, 1), out = (C, 1 - T) premultiplied;
 * VR_MIP: m = max of the maxima, out = TF(m) straight, (0,0,0,0) for -inf.
 * out_rgba (device, 16-byte aligned): width * (y1 - y0) float4, row-major.
 * n = 0 folds nothing (transparent band).  Errors: VR_ERR_INVALID_ARG for bad
 * rows, a footprint outside the image or beyond capacity, repeated ids. */
vr_status vr_sortlast_fold(vr_ctx* ctx, vr_mode mode, const float* partial, int64_t capacity,
                           const vr_footprint* foot, int32_t n, int32_t y0, int32_t y1, float* out_rgba,
                           void* stream);

/* Layout of the loaded cube; VR_ERR_STATE if none is loaded. */
vr_status vr_get_cube_info(const vr_ctx* ctx, vr_cube_info* info);

/* Message of the last failing call on ctx ("" if none); static if ctx is NULL. */
const char* vr_last_error(const vr_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* VR_H */

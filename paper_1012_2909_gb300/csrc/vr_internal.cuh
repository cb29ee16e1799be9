// Internal declarations shared by the renderer's CUDA translation units.
// Nothing here is part of the C ABI (include/vr.h is).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "vr.h"

namespace vr {

constexpr int kMaxLaunchCams = 32;   // cameras carried by value in one launch
constexpr int kMaxTF = 1024;         // transfer-function entries
constexpr int kTileW = 8, kTileH = 4; // pixels of one warp work item

// One camera as the host keeps it (double precision; Sec. 3's off-axis
// sub-windows are just other (l, t, du, dv)); kernels get it as a CamFF.
struct CamDev {
    double eye[3], right[3], up[3], fwd[3];
    double l, t, du, dv;  // u = l + (px + 1/2) du, v = t - (py + 1/2) dv
    int type, width, height, pad;
};

// The bricked cube: slot s holds brick (bx, by, bz) with a 1-voxel ghost,
// element (z, y, x) of the slot at (z * rows + y) * pitch + x, x in [0, rows).
struct VolDev {
    const void* pool;
    const void* pool1; // the store shifted by one element (pool1[e] = pool[e + 1]), or null
    const int* table;  // linear brick id -> slot (-1 = not resident)
    int nx, ny, nz;
    int nbx, nby, nbz;
    int B, log2B;
    int pitch, rows;   // rows = B + 2
    long long slot_elems;
    const unsigned int* range_max;  // per brick: ordered-int maximum of its stored values
                                    // (ghost included), or null when unknown
};

struct TFDev {
    float4 tab[kMaxTF];
    int n;
    float vmin, inv_range;
    int zero_top;  // alpha is 0 at every node 0..zero_top (-1: node 0 is not transparent)
};

// Float-float camera constants, split on the host from a CamDev.  With sx = px + 1/2,
// sy = py + 1/2:  V = base + sx bx + sy by.  Perspective: origin org, direction
// V / |V|.  Orthographic: origin V, direction dir (constant).  minv is the
// inverse of the column matrix [right up fwd], used to project cell corners.
struct CamFF {
    float base_hi[3], base_lo[3], bx_hi[3], bx_lo[3], by_hi[3], by_lo[3];
    float org_hi[3], org_lo[3];  // perspective eye
    float dir_hi[3], dir_lo[3];  // orthographic unit direction
    float minv[9];               // row-major inverse of [right up fwd]
    float eye[3];
    float l, t, du, dv;          // window mapping (FP32 copy, footprints only)
    int type, width, height, pad;
};

struct MarchParams {
    VolDev vol;
    TFDev tf;
    CamFF cams[kMaxLaunchCams];
    int ncams, width, height, mode;
    int tiles_x, tiles_y;
    int tile_w, tile_h;          // pixels of one warp work item (tile_w * tile_h == 32)
    float step_hi, step_lo;      // the sample spacing as a float-float pair
    float ert;
    int pad2;
    float4* out_rgba;            // pixels of camera 0 of this launch
    float* out_max;              // may be null
    unsigned long long* samples; // may be null
    int* work;                   // zeroed work counter of this launch
};



struct BrickFoot;

// Launch parameters of the brick (object-order) pass for up to kMaxLaunchCams
// cameras of one size; per-pixel arrays are camera-major (cam * W * H + pixel).
struct BrickParams {
    VolDev vol;
    CamFF cams[kMaxLaunchCams];
    int ncams, width, height;
    float step, step_lo;     // the sample spacing as a float-float pair
    int ncells_x, ncells_y, ncells_z;  // cells per brick along each axis
    int nbricks, pad_b;
    const int2* krange;      // per pixel [k0, k1) from the pixel set-up
    const float4* pixdir;    // optional, perspective cameras: per pixel the step
                             // vector e in float-float, 2 x float4 (hi.xyz, lo.x),
                             // (lo.y, lo.z, -, -), written by the pixel set-up
    unsigned int* out_enc;   // per pixel ordered-int encoding of the running maximum
    const int* brick_list;   // optional: only the cells of these bricks (out-of-core batches)
    int nlist, pad_l;
    int* work;               // brick counter (zeroed)
    int* status;             // device status word (0 = ok)
    // Sort-last partial images by staged cells (launch_cell_partials), camera 0 only.
    // The cells of one brick are visited in passes of equal local visibility key:
    // perspective key sum_a |c_a - eye_cell_a| minus its least value over the
    // brick's cells; orthographic key sum_a of the cell index counted along the
    // view direction's sign on that axis.  No ray crosses two cells of one brick
    // with the same key, so the cells of a pass fold into disjoint pixels.
    const BrickFoot* foot;   // per brick: rectangle and offset of its partial image
    float4* partial;         // partial images: (C, T), or the maximum in .x (MIP)
    int key_pass;            // k_cell_list keeps the cells of local key key_pass - 1 only (0: all cells)
    int key_persp;           // 1: perspective key, 0: orthographic key
    int eye_cell[3];         // perspective: floor(eye / cell edge) per axis, clamped
    int key_sign[3];         // orthographic: sign of the view direction per axis
};

// Launch parameters of the adjoint (one batch of at most kMaxLaunchCams cameras).
struct AdjParams {
    VolDev vol;
    TFDev tf;
    CamFF cams[kMaxLaunchCams];
    int ncams, width, height, mode;
    int tiles_x, tiles_y;
    float step_hi, step_lo;  // the sample spacing as a float-float pair
    float ert;
    int pad2;
    const float4* dimg;   // dL/dI of camera 0 of this launch
    float* dvol;          // dL/dvoxel, linear x-fastest (may be null)
    float* tf_partials;   // per-block table partials of this launch (grid x ntf x 4)
    int* work;            // zeroed work counter of this launch
    int* status;          // device status word
};

// Screen footprint of one brick for the sort-last paths.
struct BrickFoot {
    int4 rect;          // pixel rectangle (empty: x > z)
    int key;            // visibility layer
    int pad;
    long long offset;   // first pixel of its partial image
};

// Launch parameters of the sort-last / layered paths (one camera).
struct SortParams {
    VolDev vol;
    TFDev tf;
    CamFF cam;
    float step, step_lo;              // the sample spacing as a float-float pair
    float ert;
    int max_layers;
    int eye_brick[3], all_bricks;     // floor(eye / B); all_bricks: ignore residency (out of core)
    const int2* krange;
    BrickFoot* foot;                  // per brick
    int* order;                       // visible bricks grouped by layer
    int* layer_count;                 // max_layers
    int* layer_start;                 // max_layers + 1
    int* layer_fill;                  // max_layers
    int* tile_start;                  // nbricks + 1
    unsigned long long* partial_used; // pixels handed out to partial images
    float4* partial;                  // partial images (C, T)
    float4* state;                    // running (C, T) per pixel (layered path)
    float4* out_rgba;
    int* work;                        // zeroed work counter of a launch
    const int* sub_order;             // optional explicit brick subset (out-of-core batches)
    const int* sub_tile;              // its tile prefix (sub_n + 1)
    int sub_n, mode;                  // mode: VR_COMPOSITE partials (C, T) or VR_MIP maxima
    int fold_y0, fold_rows;           // fold only rows [fold_y0, fold_y0 + fold_rows) into a
                                      // band image (fold_rows = 0: the whole image)
};

// Per-pixel set-up and finalisation around the brick pass.
struct PixelParams {
    VolDev vol;
    TFDev tf;
    CamFF cam;
    float step_hi, step_lo;
    int width, height;
    int2* krange;
    float4* pixdir;  // optional: per-pixel float-float step vector (see BrickParams)
    unsigned int* enc;
    float4* out_rgba;
    float* out_max;
};

// Host-side launchers (defined in the kernel translation units).
cudaError_t launch_repack(const float* src, long long src_z0, long long src_planes, int bz,
                          const VolDev& v, vr_dtype dt, void* pool, unsigned int* minmax,
                          cudaStream_t s);
// The marcher reads x-neighbour pairs with one load when p.vol.pool1 is set.
cudaError_t launch_march(const MarchParams& p, vr_dtype dt, int grid, int block, cudaStream_t s);
int march_blocks_per_sm(vr_dtype dt, int mode, bool paired, int block);
cudaError_t launch_pixel_setup(const PixelParams& p, cudaStream_t s);
cudaError_t launch_mip_finalize(const PixelParams& p, cudaStream_t s);
// `cells` is per-context scratch of brick_cells_bytes(units) bytes (a counter and the
// per-view list of cells with work); the brick kernel's work counter is p.work.
cudaError_t launch_brick_mip(const void* tmap, const BrickParams& p, vr_dtype dt, int grid, void* cells,
                             cudaStream_t s, int group = 8);
size_t brick_cells_bytes(long long nunits);
// Sort-last partial images (the per-brick (C, T), or maxima for VR_MIP) of the
// bricks p.brick_list (or every brick) for camera 0, through staged cells: the
// partial slots [0, npartial) are first set to the empty image, then `npass`
// visibility passes fold every cell segment into its brick's slot.  tmap is the
// store's tensor map with the box brick_part_box_dims; tf must have at most
// kMaxPartTF entries; every slot index must fit an int.
constexpr int kMaxPartTF = 256;
cudaError_t launch_cell_partials(const void* tmap, const BrickParams& p, const TFDev& tf, vr_dtype dt, int mode,
                                 long long npartial, int npass, int grid, void* cells, cudaStream_t s,
                                 int group = 8);
// Number of visibility passes launch_cell_partials needs for a brick edge.
int cell_partial_passes(vr_dtype dt, int brick);
// TMA box of one cell for launch_cell_partials (no spare row), in elements.
void brick_part_box_dims(vr_dtype dt, int* bx, int* by, int* bz);
// Cell (staging unit) edge lengths for a storage type; the brick edge must be a
// multiple of each.
void brick_cell_dims(vr_dtype dt, int* cx, int* cy, int* cz);
// TMA box of one cell (cell + 2 ghost, x padded to 16 bytes, one spare row for
// 16-bit stores), in elements.
void brick_box_dims(vr_dtype dt, int* bx, int* by, int* bz);
// Footprints, keys and the visibility order of the bricks (p.order, p.layer_*).
cudaError_t launch_brick_footprints(const SortParams& p, cudaStream_t s);
// Prefix of the 8 x 4 pixel tiles of the ordered bricks (p.tile_start), for
// launch_brick_partial over p.order.
cudaError_t launch_tile_scan(const SortParams& p, cudaStream_t s);
cudaError_t launch_brick_partial(const SortParams& p, vr_dtype dt, bool carried, int l0, int l1, int grid,
                                 cudaStream_t s);
cudaError_t launch_sortlast_fold(const SortParams& p, cudaStream_t s);
cudaError_t launch_state_init(const SortParams& p, cudaStream_t s);
cudaError_t launch_state_finish(const SortParams& p, cudaStream_t s);
cudaError_t launch_repack_region(const float* src, int rx0, int ry0, int rz0, int rsx, int rsy, int rsz, int bx,
                                 int by, int bz, const VolDev& v, vr_dtype dt, void* slot, cudaStream_t s);
cudaError_t launch_bricks_open(const BrickFoot* foot, const int* list, int n, const float4* state, int width,
                               float ert, int* flags, cudaStream_t s);
// Camera of the catalogue overlay: the caller's vr_camera fields, unchanged.
struct OverlayCam {
    double eye[3], right[3], up[3], fwd[3];
    double l, r, b, t;
    int type, width, height, pad;
};
cudaError_t launch_overlay(const OverlayCam* cams_dev, int ncams, const double* boxes, long long nbox,
                           const float* colours, int* key, float* rgba, int width, int height, cudaStream_t s);

// Image pyramid (vr_pyramid.cu): level sizes/offsets (float4 units) and the passes.
long long pyramid_levels(int w, int h, int tlog2, std::vector<int>& ws, std::vector<int>& hs,
                         std::vector<long long>& offs);
cudaError_t launch_pyramid(const float4* in, int w, int h, int tlog2, float4* out, cudaStream_t s);
// Bounded-wait self-test (vr_selftest.cu): one waiter that gives up after `polls`.
cudaError_t launch_wait_probe(int* status, unsigned long long limit_ns, cudaStream_t s);
int adjoint_threads();
int adjoint_blocks_per_sm(vr_dtype dt, int mode, int ntf);
cudaError_t launch_adjoint(const AdjParams& p, vr_dtype dt, int grid, cudaStream_t s);
cudaError_t launch_tfgrad_reduce(const float* partials, int nblocks, int nval, float* out, cudaStream_t s);
// Brick-path MIP pieces used by the allocation-free entry point (vr_api.cu).
vr_status brick_mip_precheck(vr_ctx* ctx, float* out_rgba, float* out_max, int* device,
                             long long* pixels);
vr_status brick_mip_with_scratch(vr_ctx* ctx, float* out_rgba, float* out_max, cudaStream_t s,
                                 int2* krange, unsigned int* enc, int* work);
vr_status set_error(vr_ctx* ctx, vr_status s, const char* msg);

inline int ilog2(int v) {
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

}  // namespace vr

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

// One camera as the kernels see it (double precision; Sec. 3's off-axis
// sub-windows are just other (l, t, du, dv)).
struct CamDev {
    double eye[3], right[3], up[3], fwd[3];
    double l, t, du, dv;  // u = l + (px + 1/2) du, v = t - (py + 1/2) dv
    int type, width, height, pad;
};

// The bricked cube: slot s holds brick (bx, by, bz) with a 1-voxel ghost,
// element (z, y, x) of the slot at (z * rows + y) * pitch + x, x in [0, rows).
struct VolDev {
    const void* pool;
    const int* table;  // linear brick id -> slot (-1 = not resident)
    int nx, ny, nz;
    int nbx, nby, nbz;
    int B, log2B;
    int pitch, rows;   // rows = B + 2
    long long slot_elems;
};

struct TFDev {
    float4 tab[kMaxTF];
    int n;
    float vmin, inv_range, pad;
};

struct MarchParams {
    VolDev vol;
    TFDev tf;
    CamDev cams[kMaxLaunchCams];
    int ncams, width, height, mode;
    int tiles_x, tiles_y;
    int pad0, pad1;
    double step;
    float ert;
    int pad2;
    float4* out_rgba;            // pixels of camera 0 of this launch
    float* out_max;              // may be null
    unsigned long long* samples; // may be null
    int* work;                   // zeroed work counter of this launch
};

// Host-side launchers (defined in the kernel translation units).
cudaError_t launch_repack(const float* src, long long src_z0, long long src_planes, int bz,
                          const VolDev& v, vr_dtype dt, void* pool, unsigned int* minmax,
                          cudaStream_t s);
cudaError_t launch_march(const MarchParams& p, vr_dtype dt, int grid, cudaStream_t s);
int march_blocks_per_sm(vr_dtype dt, int mode);
constexpr int kMarchThreads = 128;

inline int ilog2(int v) {
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

}  // namespace vr

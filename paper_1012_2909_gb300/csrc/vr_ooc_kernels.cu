// Device side of out-of-core streaming: repack of one generated brick region
// into a cache slot, and the per-brick "any pixel still open" test that lets a
// layered composite skip (and never fetch) bricks behind terminated rays.
#include <algorithm>

#include "vr_internal.cuh"

namespace vr {

namespace {

template <typename T> __device__ __forceinline__ T to_store(float f);
template <> __device__ __forceinline__ float to_store<float>(float f) { return f; }
template <> __device__ __forceinline__ __half to_store<__half>(float f) { return __float2half_rn(f); }
template <> __device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(float f) {
    return __float2bfloat16_rn(f);
}

// src: region [rx0, rx0+rsx) x [ry0, ...) x [rz0, ...) of the cube, x fastest,
// the clamped ghosted extent of brick (bx, by, bz).  Slot element (z, y, x)
// holds cube voxel clamp(b*B + (z|y|x) - 1); padding columns get 0.
template <typename T>
__global__ void k_repack_region(const float* __restrict__ src, int rx0, int ry0, int rz0, int rsx, int rsy,
                                int rsz, int bx, int by, int bz, VolDev v, T* __restrict__ slot) {
    const int rows = v.rows, pitch = v.pitch;
    const long long n = (long long)rows * rows * pitch;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int lx = (int)(i % pitch);
        const long long r = i / pitch;
        const int ly = (int)(r % rows), lz = (int)(r / rows);
        T out = to_store<T>(0.f);
        if (lx < rows) {
            const int gx = min(max(bx * v.B + lx - 1, 0), v.nx - 1);
            const int gy = min(max(by * v.B + ly - 1, 0), v.ny - 1);
            const int gz = min(max(bz * v.B + lz - 1, 0), v.nz - 1);
            const int sx = min(max(gx - rx0, 0), rsx - 1), sy = min(max(gy - ry0, 0), rsy - 1),
                      sz = min(max(gz - rz0, 0), rsz - 1);
            out = to_store<T>(src[((long long)sz * rsy + sy) * rsx + sx]);
        }
        slot[i] = out;
    }
}

// flags[i] = 1 if some pixel of brick list[i]'s rectangle is still open
// (1 - T < ert), one block per brick.
__global__ void k_bricks_open(const BrickFoot* __restrict__ foot, const int* __restrict__ list, int n,
                              const float4* __restrict__ state, int width, float ert, int* __restrict__ flags) {
    __shared__ int s_open;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        if (threadIdx.x == 0) s_open = 0;
        __syncthreads();
        const int4 r = foot[list[i]].rect;
        const int rw = r.z - r.x + 1, npx = rw * (r.w - r.y + 1);
        for (int p = threadIdx.x; p < npx && !s_open; p += blockDim.x) {
            const int px = r.x + p % rw, py = r.y + p / rw;
            if (1.f - state[(long long)py * width + px].w < ert) s_open = 1;
        }
        __syncthreads();
        if (threadIdx.x == 0) flags[i] = s_open;
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_repack_region(const float* src, int rx0, int ry0, int rz0, int rsx, int rsy, int rsz, int bx,
                                 int by, int bz, const VolDev& v, vr_dtype dt, void* slot, cudaStream_t s) {
    const int grid = 304;
    if (dt == VR_F32)
        k_repack_region<float><<<grid, 256, 0, s>>>(src, rx0, ry0, rz0, rsx, rsy, rsz, bx, by, bz, v,
                                                    static_cast<float*>(slot));
    else if (dt == VR_F16)
        k_repack_region<__half><<<grid, 256, 0, s>>>(src, rx0, ry0, rz0, rsx, rsy, rsz, bx, by, bz, v,
                                                     static_cast<__half*>(slot));
    else
        k_repack_region<__nv_bfloat16><<<grid, 256, 0, s>>>(src, rx0, ry0, rz0, rsx, rsy, rsz, bx, by, bz, v,
                                                            static_cast<__nv_bfloat16*>(slot));
    return cudaGetLastError();
}

cudaError_t launch_bricks_open(const BrickFoot* foot, const int* list, int n, const float4* state, int width,
                               float ert, int* flags, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_bricks_open<<<std::min(n, 4096), 256, 0, s>>>(foot, list, n, state, width, ert, flags);
    return cudaGetLastError();
}

}  // namespace vr

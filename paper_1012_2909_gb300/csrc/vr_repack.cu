// Repack of a linear float32 cube (x fastest) into the ghosted brick store:
// one slab of bricks (fixed bz) per launch, with conversion to the storage type
// (round to nearest even) and the per-brick minimum / maximum of the stored
// values (ghost layer included), which bound every trilinear sample taken
// inside the brick.
#include "vr_internal.cuh"

namespace vr {

namespace {

__device__ __forceinline__ unsigned int ord_enc(float f) {
    const unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

template <typename T> __device__ __forceinline__ T to_store(float f);
template <> __device__ __forceinline__ float to_store<float>(float f) { return f; }
template <> __device__ __forceinline__ __half to_store<__half>(float f) { return __float2half_rn(f); }
template <> __device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(float f) {
    return __float2bfloat16_rn(f);
}
template <typename T> __device__ __forceinline__ float widen(T v);
template <> __device__ __forceinline__ float widen<float>(float v) { return v; }
template <> __device__ __forceinline__ float widen<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float widen<__nv_bfloat16>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}

// grid: (nbx * nby, rows); block: 256.  Block (b, lz) writes plane lz of the
// slot of brick (b % nbx, b / nbx, bz).
template <typename T>
__global__ void __launch_bounds__(256)
k_repack(const float* __restrict__ src, long long src_z0, int bz, VolDev v, T* __restrict__ pool,
         unsigned int* __restrict__ minmax, int nbricks) {
    const int b2 = blockIdx.x;
    const int bx = b2 % v.nbx, by = b2 / v.nbx;
    const int lz = blockIdx.y;
    const int bid = (bz * v.nby + by) * v.nbx + bx;
    const int slot = v.table[bid];
    T* dst = pool + (long long)slot * v.slot_elems + (long long)lz * v.rows * v.pitch;
    const int gz = min(max(bz * v.B + lz - 1, 0), v.nz - 1);
    const float* plane = src + (long long)(gz - src_z0) * v.ny * v.nx;
    float mn = INFINITY, mx = -INFINITY;
    const int n = v.rows * v.pitch;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int ly = i / v.pitch, lx = i - ly * v.pitch;
        T out = to_store<T>(0.f);
        if (lx < v.rows) {
            const int gy = min(max(by * v.B + ly - 1, 0), v.ny - 1);
            const int gx = min(max(bx * v.B + lx - 1, 0), v.nx - 1);
            out = to_store<T>(plane[(long long)gy * v.nx + gx]);
            const float w = widen<T>(out);
            mn = fminf(mn, w);
            mx = fmaxf(mx, w);
        }
        dst[i] = out;
    }
    for (int off = 16; off > 0; off >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, off));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&minmax[bid], ord_enc(mn));
        atomicMax(&minmax[nbricks + bid], ord_enc(mx));
    }
}

}  // namespace

cudaError_t launch_repack(const float* src, long long src_z0, long long /*src_planes*/, int bz,
                          const VolDev& v, vr_dtype dt, void* pool, unsigned int* minmax,
                          cudaStream_t s) {
    const dim3 grid(v.nbx * v.nby, v.rows);
    const int nbricks = v.nbx * v.nby * v.nbz;
    if (dt == VR_F32)
        k_repack<float><<<grid, 256, 0, s>>>(src, src_z0, bz, v, static_cast<float*>(pool), minmax, nbricks);
    else if (dt == VR_F16)
        k_repack<__half><<<grid, 256, 0, s>>>(src, src_z0, bz, v, static_cast<__half*>(pool), minmax, nbricks);
    else
        k_repack<__nv_bfloat16><<<grid, 256, 0, s>>>(src, src_z0, bz, v, static_cast<__nv_bfloat16*>(pool), minmax, nbricks);
    return cudaGetLastError();
}

}  // namespace vr

// Adjoint of the ray caster: dL/d(table entries) and dL/d(voxel values) from
// dL/d(image), for front-to-back "over" with early termination and for MIP.
//
// Composite, per ray (samples k = 0..n-1 executed, T_k the transmittance
// before sample k, a_k and c_k the sample's alpha and colour):
//     C = sum_k T_k a_k c_k,   A = 1 - prod_k (1 - a_k)
//     dC/dc_k = T_k a_k,  dC/da_k = T_k (c_k - R_k),  dA/da_k = T_k P_k
// with R_k the colour composited behind sample k starting from transmittance 1
// and P_k the transmittance behind it, both accumulated back to front
// (R <- a c + (1 - a) R, P <- (1 - a) P), so nothing divides by 1 - a.
// The forward march is recomputed segment by segment instead of storing
// samples: the first pass keeps (first sample, T) of every segment (<= 32
// samples inside one brick); the reverse pass re-runs each segment forward from
// its checkpoint, keeps its values and transmittances, then sweeps it back to
// front.  Table gradients go to per-warp FP32 copies in shared memory, then to
// per-block partials that a final kernel sums in FP64; voxel gradients are
// scattered through the trilinear weights with FP32 atomics.
// MIP: the image is TF(max v); the gradient reaches the first maximal sample.
#include <algorithm>

#include "vr_device.cuh"
#include "vr_tma.cuh"

namespace vr {

namespace {

constexpr int kAdjThreads = 128;
constexpr int kAdjSeg = 32;       // samples per checkpoint segment (at most)
constexpr int kAdjMaxSegs = 320;  // checkpoints per ray
constexpr int kDevTooManySegments = 2;

struct TFGrad {
    int i;
    float w;
    float4 rgba, slope;
};

__device__ __forceinline__ TFGrad tf_eval(const float4* __restrict__ tab, int n, float vmin,
                                          float inv_range, float val) {
    TFGrad r;
    const float u0 = (val - vmin) * inv_range;
    const bool inside = u0 > 0.f && u0 < 1.f;
    const float u = fminf(fmaxf(u0, 0.f), 1.f);
    const float x = u * (float)(n - 1);
    r.i = min((int)x, n - 2);
    r.w = x - (float)r.i;
    const float4 a = tab[r.i], b = tab[r.i + 1];
    r.rgba = make_float4(fmaf(r.w, b.x - a.x, a.x), fmaf(r.w, b.y - a.y, a.y), fmaf(r.w, b.z - a.z, a.z),
                         fmaf(r.w, b.w - a.w, a.w));
    const float s = inside ? (float)(n - 1) * inv_range : 0.f;
    r.slope = make_float4((b.x - a.x) * s, (b.y - a.y) * s, (b.z - a.z) * s, (b.w - a.w) * s);
    return r;
}

// Scatter dv to the 8 voxels of the sample at slot coordinate g of brick b.
__device__ __forceinline__ void scatter_voxels(float* __restrict__ dvol, const VolDev& v, int bx, int by,
                                               int bz, float gx, float gy, float gz, float dv) {
    if (dv == 0.f) return;
    const float fx0 = floorf(gx), fy0 = floorf(gy), fz0 = floorf(gz);
    const float fx = gx - fx0, fy = gy - fy0, fz = gz - fz0;
    // slot index s <-> cube index b*B + s - 1, clamped to the cube like the ghost layer
    const int x0 = bx * v.B + (int)fx0 - 1, y0 = by * v.B + (int)fy0 - 1, z0 = bz * v.B + (int)fz0 - 1;
    const int xs[2] = {min(max(x0, 0), v.nx - 1), min(max(x0 + 1, 0), v.nx - 1)};
    const int ys[2] = {min(max(y0, 0), v.ny - 1), min(max(y0 + 1, 0), v.ny - 1)};
    const int zs[2] = {min(max(z0, 0), v.nz - 1), min(max(z0 + 1, 0), v.nz - 1)};
    const float wx[2] = {1.f - fx, fx}, wy[2] = {1.f - fy, fy}, wz[2] = {1.f - fz, fz};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
        const float w = wx[dx] * wy[dy] * wz[dz];
        const long long idx = ((long long)zs[dz] * v.ny + ys[dy]) * v.nx + xs[dx];
        atomicAdd(dvol + idx, w * dv);
    }
}

__device__ __forceinline__ void add_tf(float* __restrict__ g, const TFGrad& t, float4 gc) {
    const float w1 = t.w, w0 = 1.f - t.w;
    float* a = g + 4 * t.i;
    atomicAdd(a + 0, w0 * gc.x);
    atomicAdd(a + 1, w0 * gc.y);
    atomicAdd(a + 2, w0 * gc.z);
    atomicAdd(a + 3, w0 * gc.w);
    atomicAdd(a + 4, w1 * gc.x);
    atomicAdd(a + 5, w1 * gc.y);
    atomicAdd(a + 6, w1 * gc.z);
    atomicAdd(a + 7, w1 * gc.w);
}

__device__ __forceinline__ void brick_of(const Ray& r, int k, const VolDev& v, int& bx, int& by, int& bz) {
    const double px = fma((double)k, r.e[0], r.o[0]);
    const double py = fma((double)k, r.e[1], r.o[1]);
    const double pz = fma((double)k, r.e[2], r.o[2]);
    bx = min(max(((int)floor(px)) >> v.log2B, 0), v.nbx - 1);
    by = min(max(((int)floor(py)) >> v.log2B, 0), v.nby - 1);
    bz = min(max(((int)floor(pz)) >> v.log2B, 0), v.nbz - 1);
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kAdjThreads)
k_adjoint(const __grid_constant__ AdjParams P) {
    extern __shared__ float s_grad[];  // (warps per block) x ntf x 4
    __shared__ float4 s_tf[kMaxTF];
    const int ntf = P.tf.n;
    for (int i = threadIdx.x; i < ntf; i += blockDim.x) s_tf[i] = P.tf.tab[i];
    const int nw = blockDim.x / 32;
    for (int i = threadIdx.x; i < nw * ntf * 4; i += blockDim.x) s_grad[i] = 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* g_tf = s_grad + warp * ntf * 4;
    const int tiles_per_cam = P.tiles_x * P.tiles_y;
    const int total = tiles_per_cam * P.ncams;
    const T* __restrict__ pool = static_cast<const T*>(P.vol.pool);
    const float ert = P.ert;
    int seg_k[kAdjMaxSegs];
    float seg_T[kAdjMaxSegs];

    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(P.work, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= total) break;
        const int cam = item / tiles_per_cam;
        const int tile = item - cam * tiles_per_cam;
        const int ty = tile / P.tiles_x, tx = tile - ty * P.tiles_x;
        const int px = tx * kTileW + (lane % kTileW);
        const int py = ty * kTileH + (lane / kTileW);
        if (px >= P.width || py >= P.height) continue;  // ragged edge tile
        const long long pix = ((long long)cam * P.height + py) * P.width + px;
        const float4 gI = P.dimg[pix];
        if (gI.x == 0.f && gI.y == 0.f && gI.z == 0.f && gI.w == 0.f) continue;
        Ray r;
        if (!make_ray(P.cams[cam], px, py, P.vol, P.step, r)) continue;
        const float3 e32 = make_float3((float)r.e[0], (float)r.e[1], (float)r.e[2]);

        if (MODE == VR_MIP) {
            // forward: first maximal sample
            float m = -INFINITY;
            int kmax = -1;
            for (int k = r.k0; k < r.k1;) {
                Seg s;
                seg_begin(r, k, P.vol, e32, 128, s);
                const T* slot = pool + s.base;
                for (int j = 0; j < s.n; ++j) {
                    const float fj = (float)j;
                    const float v = fetch_trilinear<T>(slot, P.vol, fmaf(fj, e32.x, s.gx), fmaf(fj, e32.y, s.gy),
                                                       fmaf(fj, e32.z, s.gz));
                    if (v > m) {
                        m = v;
                        kmax = k + j;
                    }
                }
                k += s.n;
            }
            if (kmax < 0) continue;
            const TFGrad t = tf_eval(s_tf, ntf, P.tf.vmin, P.tf.inv_range, m);
            add_tf(g_tf, t, gI);
            if (P.dvol) {
                Seg s;
                seg_begin(r, kmax, P.vol, e32, 1, s);
                int bx, by, bz;
                brick_of(r, kmax, P.vol, bx, by, bz);
                const float dv = gI.x * t.slope.x + gI.y * t.slope.y + gI.z * t.slope.z + gI.w * t.slope.w;
                scatter_voxels(P.dvol, P.vol, bx, by, bz, s.gx, s.gy, s.gz, dv);
            }
            continue;
        }

        // ---- composite: forward with checkpoints
        int nseg = 0, last_n = 0;
        bool overflow = false;
        {
            float Tr = 1.f;
            bool done = false;
            for (int k = r.k0; k < r.k1 && !done;) {
                Seg s;
                seg_begin(r, k, P.vol, e32, kAdjSeg, s);
                if (nseg == kAdjMaxSegs) {
                    overflow = true;
                    break;
                }
                seg_k[nseg] = k;
                seg_T[nseg] = Tr;
                ++nseg;
                const T* slot = pool + s.base;
                int j = 0;
                for (; j < s.n; ++j) {
                    const float fj = (float)j;
                    const float v = fetch_trilinear<T>(slot, P.vol, fmaf(fj, e32.x, s.gx), fmaf(fj, e32.y, s.gy),
                                                       fmaf(fj, e32.z, s.gz));
                    const float4 c = tf_lookup(s_tf, ntf, P.tf.vmin, P.tf.inv_range, v);
                    Tr = Tr * (1.f - c.w);
                    if (1.f - Tr >= ert) {
                        done = true;
                        ++j;
                        break;
                    }
                }
                last_n = j;
                k += s.n;
            }
        }
        if (overflow) {
            atomicExch(P.status, kDevTooManySegments);
            continue;
        }
        // ---- reverse sweep, segment by segment
        float R0 = 0.f, R1 = 0.f, R2 = 0.f, Pt = 1.f;
        for (int sg = nseg - 1; sg >= 0; --sg) {
            Seg s;
            seg_begin(r, seg_k[sg], P.vol, e32, kAdjSeg, s);
            const int n = (sg == nseg - 1) ? last_n : s.n;
            int bx, by, bz;
            brick_of(r, seg_k[sg], P.vol, bx, by, bz);
            const T* slot = pool + s.base;
            float vb[kAdjSeg], Tb[kAdjSeg];
            float Tr = seg_T[sg];
#pragma unroll 1
            for (int j = 0; j < n; ++j) {
                const float fj = (float)j;
                const float v = fetch_trilinear<T>(slot, P.vol, fmaf(fj, e32.x, s.gx), fmaf(fj, e32.y, s.gy),
                                                   fmaf(fj, e32.z, s.gz));
                vb[j] = v;
                Tb[j] = Tr;
                Tr = Tr * (1.f - tf_lookup(s_tf, ntf, P.tf.vmin, P.tf.inv_range, v).w);
            }
#pragma unroll 1
            for (int j = n - 1; j >= 0; --j) {
                const TFGrad t = tf_eval(s_tf, ntf, P.tf.vmin, P.tf.inv_range, vb[j]);
                const float a = t.rgba.w, Tk = Tb[j];
                float4 gc;
                gc.x = gI.x * Tk * a;
                gc.y = gI.y * Tk * a;
                gc.z = gI.z * Tk * a;
                gc.w = gI.w * Tk * Pt + gI.x * Tk * (t.rgba.x - R0) + gI.y * Tk * (t.rgba.y - R1) +
                       gI.z * Tk * (t.rgba.z - R2);
                R0 = fmaf(a, t.rgba.x, (1.f - a) * R0);
                R1 = fmaf(a, t.rgba.y, (1.f - a) * R1);
                R2 = fmaf(a, t.rgba.z, (1.f - a) * R2);
                Pt *= (1.f - a);
                add_tf(g_tf, t, gc);
                if (P.dvol) {
                    const float dv = gc.x * t.slope.x + gc.y * t.slope.y + gc.z * t.slope.z + gc.w * t.slope.w;
                    const float fj = (float)j;
                    scatter_voxels(P.dvol, P.vol, bx, by, bz, fmaf(fj, e32.x, s.gx), fmaf(fj, e32.y, s.gy),
                                   fmaf(fj, e32.z, s.gz), dv);
                }
            }
        }
    }
    __syncthreads();
    // block partial: sum of the per-warp copies
    float* out = P.tf_partials + (size_t)blockIdx.x * ntf * 4;
    for (int i = threadIdx.x; i < ntf * 4; i += blockDim.x) {
        float acc = 0.f;
        for (int w = 0; w < nw; ++w) acc += s_grad[w * ntf * 4 + i];
        out[i] = acc;
    }
}

// Final reduction of the per-block table partials, in FP64 (the only FP64
// arithmetic on the gradient path).
__global__ void k_tfgrad_reduce(const float* __restrict__ partials, int nblocks, int nval,
                                float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nval) return;
    double acc = 0.0;
    for (int b = 0; b < nblocks; ++b) acc += (double)partials[(size_t)b * nval + i];
    out[i] = (float)acc;
}

template <typename T, int MODE>
void* adj_ptr() {
    return reinterpret_cast<void*>(&k_adjoint<T, MODE>);
}

void* adj_pick(vr_dtype dt, int mode) {
    if (dt == VR_F32) return mode == VR_MIP ? adj_ptr<float, VR_MIP>() : adj_ptr<float, VR_COMPOSITE>();
    if (dt == VR_F16) return mode == VR_MIP ? adj_ptr<__half, VR_MIP>() : adj_ptr<__half, VR_COMPOSITE>();
    return mode == VR_MIP ? adj_ptr<__nv_bfloat16, VR_MIP>() : adj_ptr<__nv_bfloat16, VR_COMPOSITE>();
}

}  // namespace

int adjoint_threads() { return kAdjThreads; }

int adjoint_blocks_per_sm(vr_dtype dt, int mode, int ntf) {
    const size_t smem = (size_t)(kAdjThreads / 32) * ntf * 4 * sizeof(float);
    void* f = adj_pick(dt, mode);
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 1;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, kAdjThreads, smem) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

cudaError_t launch_adjoint(const AdjParams& p, vr_dtype dt, int grid, cudaStream_t s) {
    const size_t smem = (size_t)(kAdjThreads / 32) * p.tf.n * 4 * sizeof(float);
    void* f = adj_pick(dt, p.mode);
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void* args[] = {const_cast<AdjParams*>(&p)};
    return cudaLaunchKernel(f, dim3(grid), dim3(kAdjThreads), args, smem, s);
}

cudaError_t launch_tfgrad_reduce(const float* partials, int nblocks, int nval, float* out, cudaStream_t s) {
    k_tfgrad_reduce<<<(nval + 255) / 256, 256, 0, s>>>(partials, nblocks, nval, out);
    return cudaGetLastError();
}

}  // namespace vr

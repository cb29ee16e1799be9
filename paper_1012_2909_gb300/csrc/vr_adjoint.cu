// Adjoint of the ray caster: dL/d(table entries) and dL/d(voxel values) from
// dL/d(image), for front-to-back "over" with early termination and for MIP.
//
// Composite, per ray (samples k = 0..n-1 executed, T_k the transmittance
// before sample k, a_k and c_k the sample's alpha and colour):
//     C = sum_k T_k a_k c_k,   A = 1 - prod_k (1 - a_k)
//     dC/dc_k = T_k a_k,  dC/da_k = T_k (c_k - R_k),  dA/da_k = T_k P_k
// with R_k the colour composited behind sample k starting from transmittance 1
// and P_k the transmittance behind it: (R_k, P_k) is the "over" composite of
// the samples after k, an associative product, so nothing divides by 1 - a.
// The forward march is recomputed chunk by chunk instead of storing samples:
// the first pass keeps the transmittance at the start of every 32-sample chunk;
// the reverse pass recomputes each chunk from its checkpoint, one sample per
// lane, and gets (R_k, P_k) from a warp suffix scan carried from the chunks
// behind.  Table gradients go to per-warp FP32 copies in shared memory, then to
// per-block partials that a final kernel sums in FP64; voxel gradients are
// scattered through the trilinear weights with FP32 atomics.
// MIP: the image is TF(max v); the gradient reaches the first maximal sample.
#include <algorithm>

#include "vr_device.cuh"
#include "vr_ff.cuh"
#include "vr_tma.cuh"

namespace vr {

namespace {

constexpr int kAdjThreads = 128;
constexpr int kAdjWarps = kAdjThreads / 32;
constexpr int kAdjMaxChunks = 320;  // 32-sample transmittance checkpoints per ray
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

// g: one warp's table gradient, channel-major (g[c * n + i]), so that the lanes
// of one atomic instruction fall on banks by table entry, not by entry mod 8.
__device__ __forceinline__ void add_tf(float* __restrict__ g, int n, const TFGrad& t, float4 gc) {
    const float w1 = t.w, w0 = 1.f - t.w;
    float* a = g + t.i;
    atomicAdd(a, w0 * gc.x);
    atomicAdd(a + n, w0 * gc.y);
    atomicAdd(a + 2 * n, w0 * gc.z);
    atomicAdd(a + 3 * n, w0 * gc.w);
    atomicAdd(a + 1, w1 * gc.x);
    atomicAdd(a + n + 1, w1 * gc.y);
    atomicAdd(a + 2 * n + 1, w1 * gc.z);
    atomicAdd(a + 3 * n + 1, w1 * gc.w);
}

// One warp per ray, its lanes on 32 consecutive samples (a chunk).  A warp
// claims a tile of 32 pixels, sets up their rays once (one lane each, float-float)
// into shared memory and then walks them.  Composite: the forward pass keeps
// the transmittance at the start of every chunk (one float) and finds the
// termination sample by a ballot on a warp prefix product of (1 - a); the
// reverse pass recomputes each chunk from its checkpoint and gets the colour
// and transmittance behind every sample from a warp suffix scan of "over",
// carried from chunk to chunk.  MIP: a warp maximum per chunk keeps the first
// maximal sample.  Sample positions: the float-float ray from the set-up, one
// float-float anchor per chunk, lane offsets in FP32, each lane
// reading the brick that holds its sample (the ghost layer makes any brick
// within half a voxel give the same value).
struct RaySetup {
    float o_hi[3], o_lo[3], e_hi[3], e_lo[3];
    int k0, k1;
    float4 g;  // dL/dI of the pixel
};

__device__ __forceinline__ unsigned int ord_enc_f(float f) {
    const unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Brick (bx, by, bz) and slot coordinate g of sample k + lane of the ray.
struct LaneSample {
    int bx, by, bz;
    float gx, gy, gz;
    long long base;
};

// brick index along one axis of the float-float position p (clamped to the grid)
// and the slot coordinate of p in it
__device__ __forceinline__ int anchor_axis(ff p, const VolDev& v, int nb, float& g) {
    const int b = min(max(((int)floorf(p.hi)) >> v.log2B, 0), nb - 1);
    g = __fadd_rn(__fsub_rn(p.hi, (float)(b << v.log2B)), p.lo) + 0.5f;
    return b;
}

__device__ __forceinline__ void lane_sample(const RaySetup& r, int k, int lane, float3 e32, const VolDev& v,
                                            LaneSample& s) {
    const ff fk = ff_of_int(k);  // exact for any sample index
    float gx, gy, gz;
    const int bx0 = anchor_axis(ff_add(ff{r.o_hi[0], r.o_lo[0]}, ff_mul(ff{r.e_hi[0], r.e_lo[0]}, fk)), v, v.nbx, gx);
    const int by0 = anchor_axis(ff_add(ff{r.o_hi[1], r.o_lo[1]}, ff_mul(ff{r.e_hi[1], r.e_lo[1]}, fk)), v, v.nby, gy);
    const int bz0 = anchor_axis(ff_add(ff{r.o_hi[2], r.o_lo[2]}, ff_mul(ff{r.e_hi[2], r.e_lo[2]}, fk)), v, v.nbz, gz);
    const float fl = (float)lane;
    gx = fmaf(fl, e32.x, gx);
    gy = fmaf(fl, e32.y, gy);
    gz = fmaf(fl, e32.z, gz);
    const float B = (float)v.B, invB = 1.0f / B;
    const int bx = min(max(bx0 + (int)floorf((gx - 0.5f) * invB), 0), v.nbx - 1);
    const int by = min(max(by0 + (int)floorf((gy - 0.5f) * invB), 0), v.nby - 1);
    const int bz = min(max(bz0 + (int)floorf((gz - 0.5f) * invB), 0), v.nbz - 1);
    s.gx = gx - (float)((bx - bx0) << v.log2B);
    s.gy = gy - (float)((by - by0) << v.log2B);
    s.gz = gz - (float)((bz - bz0) << v.log2B);
    s.bx = bx;
    s.by = by;
    s.bz = bz;
    s.base = (long long)v.table[(bz * v.nby + by) * v.nbx + bx] * v.slot_elems;
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kAdjThreads)
k_adjoint(const __grid_constant__ AdjParams P) {
    constexpr unsigned int FULL = 0xffffffffu;
    // dynamic: (warps per block) x 4 channels x ntf table-gradient floats, then the
    // ntf table entries (sized by the table, not kMaxTF, so more CTAs fit an SM)
    extern __shared__ __align__(16) float s_grad[];
    float4* s_tf = reinterpret_cast<float4*>(s_grad + kAdjWarps * 4 * P.tf.n);
    __shared__ RaySetup s_ray[kAdjWarps][32];
    __shared__ float s_ckT[kAdjWarps][kAdjMaxChunks];
    const int ntf = P.tf.n;
    for (int i = threadIdx.x; i < ntf; i += blockDim.x) s_tf[i] = P.tf.tab[i];
    for (int i = threadIdx.x; i < kAdjWarps * ntf * 4; i += blockDim.x) s_grad[i] = 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* g_tf = s_grad + warp * ntf * 4;
    float* ckT = s_ckT[warp];
    const int tiles_per_cam = P.tiles_x * P.tiles_y;
    const int total = tiles_per_cam * P.ncams;
    const T* __restrict__ pool = static_cast<const T*>(P.vol.pool);
    const float ert = P.ert;

    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(P.work, 1);
        item = __shfl_sync(FULL, item, 0);
        if (item >= total) break;
        const int cam = item / tiles_per_cam;
        const int tile = item - cam * tiles_per_cam;
        const int ty = tile / P.tiles_x, tx = tile - ty * P.tiles_x;
        {  // this lane's ray of the tile
            const int px = tx * kTileW + (lane % kTileW);
            const int py = ty * kTileH + (lane / kTileW);
            bool ok = px < P.width && py < P.height;
            Ray r;
            float4 gI = make_float4(0.f, 0.f, 0.f, 0.f);
            if (ok) {
                gI = P.dimg[((long long)cam * P.height + py) * P.width + px];
                ok = (gI.x != 0.f || gI.y != 0.f || gI.z != 0.f || gI.w != 0.f) &&
                     make_ray(P.cams[cam], px, py, P.vol, ff{P.step_hi, P.step_lo}, r);
            }
            RaySetup& rs = s_ray[warp][lane];
            if (ok) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    rs.o_hi[a] = r.o[a].hi;
                    rs.o_lo[a] = r.o[a].lo;
                    rs.e_hi[a] = r.e[a].hi;
                    rs.e_lo[a] = r.e[a].lo;
                }
                rs.g = gI;
            }
            rs.k0 = ok ? r.k0 : 0;
            rs.k1 = ok ? r.k1 : 0;
        }
        __syncwarp();
        unsigned int pending = __ballot_sync(FULL, s_ray[warp][lane].k1 > s_ray[warp][lane].k0);
        while (pending) {
            const int who = __ffs(pending) - 1;
            pending &= pending - 1;
            const RaySetup r = s_ray[warp][who];
            const float3 e32 = make_float3(r.e_hi[0], r.e_hi[1], r.e_hi[2]);
            const float4 gI = r.g;

            if (MODE == VR_MIP) {
                unsigned int best = ord_enc_f(-INFINITY);
                float m = -INFINITY;
                int kmax = -1;
                for (int k = r.k0; k < r.k1; k += 32) {
                    const bool act = k + lane < r.k1;
                    float v = -INFINITY;
                    if (act) {
                        LaneSample ls;
                        lane_sample(r, k, lane, e32, P.vol, ls);
                        v = fetch_trilinear<T>(pool + ls.base, P.vol, ls.gx, ls.gy, ls.gz);
                    }
                    const unsigned int e = act ? ord_enc_f(v) : 0u;
                    const unsigned int cmax = __reduce_max_sync(FULL, e);
                    if (cmax > best) {  // strictly greater: the first maximal sample is kept
                        best = cmax;
                        const int src = __ffs(__ballot_sync(FULL, act && e == cmax)) - 1;
                        m = __shfl_sync(FULL, v, src);
                        kmax = k + src;
                    }
                }
                if (kmax < 0) continue;
                if (lane == 0) {
                    const TFGrad t = tf_eval(s_tf, ntf, P.tf.vmin, P.tf.inv_range, m);
                    add_tf(g_tf, ntf, t, gI);
                    if (P.dvol) {
                        LaneSample ls;
                        lane_sample(r, kmax, 0, e32, P.vol, ls);
                        const float dv = gI.x * t.slope.x + gI.y * t.slope.y + gI.z * t.slope.z + gI.w * t.slope.w;
                        scatter_voxels(P.dvol, P.vol, ls.bx, ls.by, ls.bz, ls.gx, ls.gy, ls.gz, dv);
                    }
                }
                continue;
            }

            // ---- composite, forward: transmittance checkpoints per chunk, termination by ballot
            int nch = 0, n_last = 0;
            {
                float Tr = 1.f;
                bool overflow = false;
                for (int k = r.k0; k < r.k1; k += 32) {
                    if (nch == kAdjMaxChunks) {
                        overflow = true;
                        break;
                    }
                    if (lane == 0) ckT[nch] = Tr;
                    ++nch;
                    const int n = min(32, r.k1 - k);
                    const bool act = lane < n;
                    float q = 1.f;
                    if (act) {
                        LaneSample ls;
                        lane_sample(r, k, lane, e32, P.vol, ls);
                        const float v = fetch_trilinear<T>(pool + ls.base, P.vol, ls.gx, ls.gy, ls.gz);
                        q = 1.f - tf_lookup(s_tf, ntf, P.tf.vmin, P.tf.inv_range, v).w;
                    }
                    float incl = q;
#pragma unroll
                    for (int off = 1; off < 32; off <<= 1) {
                        const float t = __shfl_up_sync(FULL, incl, off);
                        if (lane >= off) incl *= t;
                    }
                    const float Tout = Tr * incl;
                    const unsigned int done = __ballot_sync(FULL, act && 1.f - Tout >= ert);
                    if (done) {
                        n_last = __ffs(done);
                        break;
                    }
                    n_last = n;
                    Tr = __shfl_sync(FULL, Tout, n - 1);
                }
                if (overflow) {
                    if (lane == 0) atomicExch(P.status, kDevTooManySegments);
                    continue;
                }
            }
            __syncwarp();
            // ---- reverse: chunks back to front, suffix "over" scan within a chunk
            float Rc0 = 0.f, Rc1 = 0.f, Rc2 = 0.f, Pc = 1.f;
            for (int c = nch - 1; c >= 0; --c) {
                const int k = r.k0 + 32 * c;
                const int n = c == nch - 1 ? n_last : 32;
                const bool act = lane < n;
                TFGrad t;
                LaneSample ls;
                float a = 0.f;
                if (act) {
                    lane_sample(r, k, lane, e32, P.vol, ls);
                    const float v = fetch_trilinear<T>(pool + ls.base, P.vol, ls.gx, ls.gy, ls.gz);
                    t = tf_eval(s_tf, ntf, P.tf.vmin, P.tf.inv_range, v);
                    a = t.rgba.w;
                }
                const float q = 1.f - a;
                float incl = q;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const float u = __shfl_up_sync(FULL, incl, off);
                    if (lane >= off) incl *= u;
                }
                float excl = __shfl_up_sync(FULL, incl, 1);
                if (lane == 0) excl = 1.f;
                const float Tin = ckT[c] * excl;
                // inclusive suffix of (A, B) = (a rgb, 1 - a) under (A1, B1) o (A2, B2) = (A1 + B1 A2, B1 B2)
                float A0 = act ? a * t.rgba.x : 0.f, A1 = act ? a * t.rgba.y : 0.f, A2 = act ? a * t.rgba.z : 0.f;
                float Bq = q;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const float o0 = __shfl_down_sync(FULL, A0, off), o1 = __shfl_down_sync(FULL, A1, off);
                    const float o2 = __shfl_down_sync(FULL, A2, off), ob = __shfl_down_sync(FULL, Bq, off);
                    if (lane + off < 32) {
                        A0 = fmaf(Bq, o0, A0);
                        A1 = fmaf(Bq, o1, A1);
                        A2 = fmaf(Bq, o2, A2);
                        Bq *= ob;
                    }
                }
                // behind sample `lane`: the suffix after it, then the chunks behind this one
                float x0 = __shfl_down_sync(FULL, A0, 1), x1 = __shfl_down_sync(FULL, A1, 1);
                float x2 = __shfl_down_sync(FULL, A2, 1), xb = __shfl_down_sync(FULL, Bq, 1);
                if (lane == 31) {
                    x0 = x1 = x2 = 0.f;
                    xb = 1.f;
                }
                const float R0 = fmaf(xb, Rc0, x0), R1 = fmaf(xb, Rc1, x1), R2 = fmaf(xb, Rc2, x2);
                const float Pt = xb * Pc;
                // carry for the chunk in front: this whole chunk over the carry
                const float h0 = __shfl_sync(FULL, A0, 0), h1 = __shfl_sync(FULL, A1, 0);
                const float h2 = __shfl_sync(FULL, A2, 0), hb = __shfl_sync(FULL, Bq, 0);
                Rc0 = fmaf(hb, Rc0, h0);
                Rc1 = fmaf(hb, Rc1, h1);
                Rc2 = fmaf(hb, Rc2, h2);
                Pc *= hb;
                if (act) {
                    float4 gc;
                    gc.x = gI.x * Tin * a;
                    gc.y = gI.y * Tin * a;
                    gc.z = gI.z * Tin * a;
                    gc.w = gI.w * Tin * Pt + gI.x * Tin * (t.rgba.x - R0) + gI.y * Tin * (t.rgba.y - R1) +
                           gI.z * Tin * (t.rgba.z - R2);
                    add_tf(g_tf, ntf, t, gc);
                    if (P.dvol) {
                        const float dv = gc.x * t.slope.x + gc.y * t.slope.y + gc.z * t.slope.z + gc.w * t.slope.w;
                        scatter_voxels(P.dvol, P.vol, ls.bx, ls.by, ls.bz, ls.gx, ls.gy, ls.gz, dv);
                    }
                }
            }
            __syncwarp();
        }
        __syncwarp();  // the tile's ray set-ups are read before the next tile overwrites them
    }
    __syncthreads();
    // block partial: sum of the per-warp copies
    float* out = P.tf_partials + (size_t)blockIdx.x * ntf * 4;
    for (int i = threadIdx.x; i < ntf * 4; i += blockDim.x) {
        float acc = 0.f;
        const int e = i >> 2, c = i & 3;  // output is entry-major (ntf x 4)
        for (int w = 0; w < kAdjWarps; ++w) acc += s_grad[w * ntf * 4 + c * ntf + e];
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
    const size_t smem = (size_t)(kAdjThreads / 32) * ntf * 4 * sizeof(float) + (size_t)ntf * sizeof(float4);
    void* f = adj_pick(dt, mode);
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 1;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, kAdjThreads, smem) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

cudaError_t launch_adjoint(const AdjParams& p, vr_dtype dt, int grid, cudaStream_t s) {
    const size_t smem = (size_t)(kAdjThreads / 32) * p.tf.n * 4 * sizeof(float) + (size_t)p.tf.n * sizeof(float4);
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

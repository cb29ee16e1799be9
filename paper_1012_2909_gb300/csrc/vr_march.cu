// Image-order ray marcher: one thread per ray, one warp per 8 x 4 pixel tile,
// tiles handed out by a persistent scheduler (one atomic counter per launch).
//
// Per ray (the discretisation of include/vr.h, vr_render): float-float ray
// set-up and box interval; brick-by-brick traversal; inside a brick the samples
// are re-anchored in float-float every kAnchorSpan samples and stepped in FP32
// relative to the anchor's voxel, so each position is within 13 u (u = 2^-24)
// voxels of exact at the 0.5-voxel step; trilinear fetch from the ghosted brick
// (x-neighbour pairs with one load each when the store's shifted copy is kept);
// transfer-function lookup from shared memory; front-to-back "over" with early
// termination, or maximum-intensity projection.
#include "vr_device.cuh"

namespace vr {

namespace {

constexpr int kSegCap = 1 << 20;  // a brick segment is cut only where the ray leaves the brick
// Samples fetched together per step.  The marcher waits on its gathers, so more
// loads in flight beat more resident warps: with the register count left free
// (launch bound 256 x 2: at most 128 registers, two CTAs per SM), 4 measured fastest for single loads (3: +2 %, 6: +2 %,
// 2: +9 %; capping registers at 64 for more warps cost 30 %), and 6 with the
// paired loads, which need fewer registers per sample (4: +7 %, 3: +13 %,
// 8: +15 %; survey composite over the orbit).
constexpr int kMarchUnroll = 4;
constexpr int kMarchUnrollPaired = 6;

template <typename T, int MODE, bool PAIRED>
__global__ void __launch_bounds__(256, 2)
k_march(const __grid_constant__ MarchParams P) {
    constexpr int U = PAIRED ? kMarchUnrollPaired : kMarchUnroll;
    __shared__ float4 s_tf[kMaxTF];
    for (int i = threadIdx.x; i < P.tf.n; i += blockDim.x) s_tf[i] = P.tf.tab[i];
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int tiles_per_cam = P.tiles_x * P.tiles_y;
    const int total = tiles_per_cam * P.ncams;
    const T* __restrict__ pool = static_cast<const T*>(P.vol.pool);
    const T* __restrict__ pool1 = static_cast<const T*>(P.vol.pool1);
    const float ert = P.ert;
    unsigned long long my_samples = 0;

    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(P.work, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= total) break;
        const int cam = item / tiles_per_cam;
        const int tile = item - cam * tiles_per_cam;
        const int ty = tile / P.tiles_x, tx = tile - ty * P.tiles_x;
        const int px = tx * P.tile_w + (lane % P.tile_w);
        const int py = ty * P.tile_h + (lane / P.tile_w);
        if (px >= P.width || py >= P.height) continue;  // ragged edge tile; the lane
                                                        // rejoins at the next shuffle
        Ray r;
        const bool hit = make_ray(P.cams[cam], px, py, P.vol, ff{P.step_hi, P.step_lo}, r);
        float c0 = 0.f, c1 = 0.f, c2 = 0.f, Tr = 1.f, m_ = -INFINITY;
        if (hit) {
            const float3 e32 = make_float3(r.e[0].hi, r.e[1].hi, r.e[2].hi);
            int k = r.k0;
            bool done = false;
            while (k < r.k1 && !done) {
                Seg s;
                seg_begin(r, k, P.vol, e32, kSegCap, s);
                if (MODE == VR_COMPOSITE && brick_transparent(P.vol, P.tf, s.brick)) {
                    k += s.n;  // opacity 0 throughout: (C, T) would not change
                    continue;
                }
                const T* slot = pool + s.base;
                const T* slot1 = PAIRED ? pool1 + s.base : nullptr;
                int j = 0;  // samples of this segment done
                while (j < s.n && !done) {
                    // sub-anchor at sample k + j; U samples fetched together (more loads
                    // in flight), then composited in order; a fetch past the span
                    // repeats its last sample
                    const Anchor A = anchor_at(r, k + j, P.vol, s);
                    const int m = min(kAnchorSpan, s.n - j);
                    for (int i = 0; i < m && !done; i += U) {
                        float v[U];
#pragma unroll
                        for (int q = 0; q < U; ++q) {
                            const float fi = (float)min(i + q, m - 1);
                            const float qx = fmaf(fi, e32.x, A.qx), qy = fmaf(fi, e32.y, A.qy),
                                        qz = fmaf(fi, e32.z, A.qz);
                            v[q] = PAIRED ? fetch_near_pair<T>(slot, slot1, P.vol, A, qx, qy, qz)
                                          : fetch_near<T>(slot, P.vol, A, qx, qy, qz);
                        }
#pragma unroll
                        for (int q = 0; q < U; ++q) {
                            if (i + q >= m) break;
                            if (MODE == VR_MIP) {
                                m_ = fmaxf(m_, v[q]);
                            } else {
                                const float4 c = tf_lookup(s_tf, P.tf.n, P.tf.vmin, P.tf.inv_range, v[q]);
                                const float w = Tr * c.w;
                                c0 = fmaf(w, c.x, c0);
                                c1 = fmaf(w, c.y, c1);
                                c2 = fmaf(w, c.z, c2);
                                Tr = Tr * (1.f - c.w);
                                if (1.f - Tr >= ert) {
                                    my_samples += (unsigned long long)(j + i + q + 1);
                                    done = true;
                                    break;
                                }
                            }
                        }
                    }
                    j += m;
                }
                if (!done) my_samples += (unsigned long long)s.n;
                k += s.n;
            }
        }
        const long long pix = ((long long)cam * P.height + py) * P.width + px;
        if (MODE == VR_MIP) {
            float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
            if (m_ > -INFINITY) o = tf_lookup(s_tf, P.tf.n, P.tf.vmin, P.tf.inv_range, m_);
            P.out_rgba[pix] = o;
            if (P.out_max) P.out_max[pix] = m_;
        } else {
            P.out_rgba[pix] = make_float4(c0, c1, c2, 1.f - Tr);
        }
    }
    if (P.samples) {
        unsigned long long s = my_samples;
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (lane == 0 && s) atomicAdd(P.samples, s);
    }
}

template <typename T, int MODE>
void* kernel_ptr(bool paired) {
    return paired ? reinterpret_cast<void*>(&k_march<T, MODE, true>)
                  : reinterpret_cast<void*>(&k_march<T, MODE, false>);
}

// Paired loads only for the composite: its rays stop in a front shell that stays in
// the caches, where halving the gathers pays (survey frame -11 %).  MIP rays cross the
// whole cube, and reading both copies there measured 34 % slower.
template <typename T>
void* pick_mode(int mode, bool paired) {
    return mode == VR_MIP ? reinterpret_cast<void*>(&k_march<T, VR_MIP, false>)
                          : kernel_ptr<T, VR_COMPOSITE>(paired);
}

void* pick(vr_dtype dt, int mode, bool paired) {
    if (dt == VR_F32) return mode == VR_MIP ? reinterpret_cast<void*>(&k_march<float, VR_MIP, false>)
                                            : reinterpret_cast<void*>(&k_march<float, VR_COMPOSITE, false>);
    if (dt == VR_F16) return pick_mode<__half>(mode, paired);
    return pick_mode<__nv_bfloat16>(mode, paired);
}

}  // namespace

int march_blocks_per_sm(vr_dtype dt, int mode, bool paired, int block) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pick(dt, mode, paired), block, 0) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

cudaError_t launch_march(const MarchParams& p, vr_dtype dt, int grid, int block, cudaStream_t s) {
    void* args[] = {const_cast<MarchParams*>(&p)};
    return cudaLaunchKernel(pick(dt, p.mode, p.vol.pool1 != nullptr), dim3(grid), dim3(block), args, 0, s);
}

}  // namespace vr

// Object-order compositing by bricks, in visibility order.
//
// The paper renders a cube larger than one node's memory by giving each node a
// part of it and combining the nodes' images (Abstract, Sec. 1).  Here the
// parts are the bricks of the store:
//
//   * k_brick_footprints: per brick, its screen rectangle (projection of its
//     box), its visibility key and a slice of a partial-image buffer;
//   * the brick's partial image: per pixel of its rectangle, the "over"
//     composite of the ray's samples owned by the brick, from T = 1, stored as
//     (C, T).  It is computed through staged cells (launch_cell_partials in
//     vr_brick.cu: the brick's cells in visibility passes, each cell segment
//     folded into the brick's slot), or, for tables beyond that path's 256
//     entries, by k_brick_partial<INDEPENDENT> marching whole bricks from
//     global memory;
//   * k_sortlast_fold: per pixel, the partial images folded front to back in
//     visibility order (C += T C_b, T *= T_b);
//   * with P.mode == VR_MIP the partial image of a brick is the maximum of its
//     samples per pixel (-inf without samples) and the fold takes the maximum,
//     then the transfer function;
//   * k_brick_partial<CARRIED>: the same march continuing each pixel's running
//     (C, T) with per-sample early termination, one visibility layer of bricks
//     per launch (no two bricks of a layer own samples of the same ray), and
//     bricks of terminated pixels skipped.
//
// Visibility: the brick index along a ray moves monotonically away from the
// eye's brick index e on every axis, so the key sum_a |b_a - e_a|
// (perspective) or sum_a sign(d_a) b_a (orthographic) strictly increases along
// every ray.  Sample ownership per brick uses the same FP32 face-crossing
// partition as the cell pass, clipped to the ray's sample range from the
// pixel set-up.
#include <algorithm>

#include "vr_device.cuh"
#include "vr_ff.cuh"

namespace vr {

namespace {

// brick box -> pixel rectangle (conservative; same projection as the cell pass)
__device__ bool box_rect(const CamFF& c, float3 lo, float3 hi, int4& r) {
    float umin = 3e38f, umax = -3e38f, vmin = 3e38f, vmax = -3e38f;
    bool behind = false;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float wx = ((k & 1) ? hi.x : lo.x) - c.eye[0];
        const float wy = ((k & 2) ? hi.y : lo.y) - c.eye[1];
        const float wz = ((k & 4) ? hi.z : lo.z) - c.eye[2];
        const float a = c.minv[0] * wx + c.minv[1] * wy + c.minv[2] * wz;
        const float b = c.minv[3] * wx + c.minv[4] * wy + c.minv[5] * wz;
        float u = a, v = b;
        if (c.type == 1) {
            const float z = c.minv[6] * wx + c.minv[7] * wy + c.minv[8] * wz;
            if (!(z > 1e-3f)) {
                behind = true;
                continue;
            }
            u = a / z;
            v = b / z;
        }
        umin = fminf(umin, u);
        umax = fmaxf(umax, u);
        vmin = fminf(vmin, v);
        vmax = fmaxf(vmax, v);
    }
    int px0, px1, py0, py1;
    if (behind) {
        px0 = 0;
        py0 = 0;
        px1 = c.width - 1;
        py1 = c.height - 1;
    } else {
        const float xa = (umin - c.l) / c.du - 0.5f, xb = (umax - c.l) / c.du - 0.5f;
        const float ya = (c.t - vmin) / c.dv - 0.5f, yb = (c.t - vmax) / c.dv - 0.5f;
        const float fx0 = fminf(xa, xb) - 1.f, fx1 = fmaxf(xa, xb) + 1.f;
        const float fy0 = fminf(ya, yb) - 1.f, fy1 = fmaxf(ya, yb) + 1.f;
        if (fx1 < 0.f || fy1 < 0.f || fx0 > (float)c.width || fy0 > (float)c.height) return false;
        px0 = max(0, (int)floorf(fmaxf(fx0, -1.f)));
        py0 = max(0, (int)floorf(fmaxf(fy0, -1.f)));
        px1 = min(c.width - 1, (int)ceilf(fminf(fx1, (float)c.width)));
        py1 = min(c.height - 1, (int)ceilf(fminf(fy1, (float)c.height)));
    }
    r = make_int4(px0, py0, px1, py1);
    return px0 <= px1 && py0 <= py1;
}

__global__ void k_brick_footprints(const __grid_constant__ SortParams P) {
    const int nb = P.vol.nbx * P.vol.nby * P.vol.nbz;
    const CamFF& c = P.cam;
    // eye brick (perspective, from the host in double precision) / direction signs (orthographic)
    const int B = P.vol.B;
    const int ex = P.eye_brick[0], ey = P.eye_brick[1], ez = P.eye_brick[2];
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        const int bx = b % P.vol.nbx, by = (b / P.vol.nbx) % P.vol.nby, bz = b / (P.vol.nbx * P.vol.nby);
        const float3 lo = make_float3((float)(bx * B), (float)(by * B), (float)(bz * B));
        const float3 hi = make_float3((float)min((bx + 1) * B, P.vol.nx), (float)min((by + 1) * B, P.vol.ny),
                                      (float)min((bz + 1) * B, P.vol.nz));
        int4 r = make_int4(0, 0, -1, -1);
        const bool vis = (P.all_bricks || P.vol.table[b] >= 0) && box_rect(c, lo, hi, r);
        int key;
        if (c.type == 1) {
            key = abs(bx - ex) + abs(by - ey) + abs(bz - ez);
        } else {
            // orthographic: sum of sign(d) * b, shifted to be non-negative
            const float* d = c.dir_hi;
            key = (d[0] > 0.f ? bx : (d[0] < 0.f ? P.vol.nbx - 1 - bx : 0)) +
                  (d[1] > 0.f ? by : (d[1] < 0.f ? P.vol.nby - 1 - by : 0)) +
                  (d[2] > 0.f ? bz : (d[2] < 0.f ? P.vol.nbz - 1 - bz : 0));
        }
        BrickFoot f;
        f.rect = vis ? r : make_int4(0, 0, -1, -1);
        f.key = min(key, P.max_layers - 1);
        f.offset = 0;
        if (vis) {
            const long long area = (long long)(r.z - r.x + 1) * (r.w - r.y + 1);
            f.offset = atomicAdd(P.partial_used, (unsigned long long)area);
            atomicAdd(&P.layer_count[f.key], 1);
        }
        P.foot[b] = f;
    }
}

// exclusive scan of the per-layer counts (one block) -> layer starts
__global__ void k_layer_scan(const __grid_constant__ SortParams P) {
    if (threadIdx.x != 0) return;
    int acc = 0;
    for (int l = 0; l < P.max_layers; ++l) {
        P.layer_start[l] = acc;
        acc += P.layer_count[l];
        P.layer_fill[l] = 0;
    }
    P.layer_start[P.max_layers] = acc;
}

__global__ void k_layer_scatter(const __grid_constant__ SortParams P) {
    const int nb = P.vol.nbx * P.vol.nby * P.vol.nbz;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        const BrickFoot f = P.foot[b];
        if (f.rect.z < f.rect.x) continue;
        const int pos = P.layer_start[f.key] + atomicAdd(&P.layer_fill[f.key], 1);
        P.order[pos] = b;
    }
}

// Samples of pixel (px, py) owned by brick (bx,by,bz): [ka, kb) and the
// float-float anchored slot coordinate of sample ka; false if none.
__device__ __forceinline__ bool brick_segment(const SortParams& P, int px, int py, int2 kr, int bx, int by,
                                              int bz, float g[3], float e32[3], int& ka, int& kb) {
    const CamFF& c = P.cam;
    const float sx = (float)px + 0.5f, sy = (float)py + 0.5f;
    float o[3], e[3];
    {
        float V[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) V[a] = fmaf(sy, c.by_hi[a], fmaf(sx, c.bx_hi[a], c.base_hi[a]));
        if (c.type == 1) {
            const float inv = rsqrtf(V[0] * V[0] + V[1] * V[1] + V[2] * V[2]) * P.step;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                o[a] = c.org_hi[a];
                e[a] = V[a] * inv;
            }
        } else {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                o[a] = V[a];
                e[a] = c.dir_hi[a] * P.step;
            }
        }
    }
    const int B = P.vol.B;
    const int bi[3] = {bx, by, bz};
    const int nb[3] = {P.vol.nbx, P.vol.nby, P.vol.nbz};
    float klo = -1e9f, khi = 1e9f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const bool first = bi[a] == 0;
        const bool last = bi[a] == nb[a] - 1;
        const float xl = (float)(bi[a] * B), xh = (float)((bi[a] + 1) * B);
        if (e[a] != 0.f) {
            const float inv = __fdividef(1.0f, e[a]);
            const float kl = __fmul_rn(__fsub_rn(xl, o[a]), inv);
            const float kh = __fmul_rn(__fsub_rn(xh, o[a]), inv);
            float a0, a1;
            if (e[a] > 0.f) {
                a0 = first ? -1e9f : kl;
                a1 = last ? 1e9f : kh;
            } else {
                a0 = last ? -1e9f : kh;
                a1 = first ? 1e9f : kl;
            }
            klo = fmaxf(klo, a0);
            khi = fminf(khi, a1);
        } else if (!((first || xl <= o[a]) && (last || o[a] < xh))) {
            return false;
        }
    }
    klo = fminf(fmaxf(klo, -1e9f), 1e9f);
    khi = fminf(fmaxf(khi, -1e9f), 1e9f);
    ka = max((int)ceilf(klo), kr.x);
    kb = min((int)ceilf(khi), kr.y);
    if (ka >= kb) return false;
    ff E[3], O[3];
    if (c.type == 1) {
        ff V[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            V[a] = ff_add(ff_add(ff{c.base_hi[a], c.base_lo[a]}, ff_mul_f(ff{c.bx_hi[a], c.bx_lo[a]}, sx)),
                          ff_mul_f(ff{c.by_hi[a], c.by_lo[a]}, sy));
            O[a] = ff{c.org_hi[a], c.org_lo[a]};
        }
        const ff n2 = ff_add(ff_add(ff_mul(V[0], V[0]), ff_mul(V[1], V[1])), ff_mul(V[2], V[2]));
        const ff r = ff_rsqrt(n2);
#pragma unroll
        for (int a = 0; a < 3; ++a) E[a] = ff_mul(ff_mul(V[a], r), ff{P.step, P.step_lo});
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            O[a] = ff_add(ff_add(ff{c.base_hi[a], c.base_lo[a]}, ff_mul_f(ff{c.bx_hi[a], c.bx_lo[a]}, sx)),
                          ff_mul_f(ff{c.by_hi[a], c.by_lo[a]}, sy));
            E[a] = ff_mul(ff{c.dir_hi[a], c.dir_lo[a]}, ff{P.step, P.step_lo});
        }
    }
    const ff fk = ff_of_int(ka);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const ff p = ff_add(O[a], ff_mul(E[a], fk));
        g[a] = __fadd_rn(__fsub_rn(p.hi, (float)(bi[a] * B)), p.lo) + 0.5f;  // slot coordinate
        e32[a] = E[a].hi;
    }
    return true;
}

// prefix sum of the 8 x 4 tiles of the ordered bricks (one thread; a few
// thousand bricks at most per view)
__global__ void k_tile_scan(const __grid_constant__ SortParams P) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int nvis = P.layer_start[P.max_layers];
    int acc = 0;
    for (int i = 0; i < nvis; ++i) {
        P.tile_start[i] = acc;
        const int4 r = P.foot[P.order[i]].rect;
        acc += ((r.z - r.x + 1 + 7) / 8) * ((r.w - r.y + 1 + 3) / 4);
    }
    P.tile_start[nvis] = acc;
}

// One warp per (brick, 8 x 4 tile of its rectangle); one thread per pixel.
// Bricks of the ordered positions [start of layer l0, start of layer l1).
// PAIRED (16-bit stores with the shifted copy, layered path): each x-neighbour
// pair of a trilinear fetch is one 32-bit load (fetch_trilinear_pair, the same
// values bit for bit), halving the gathers (survey layered composite 3.03 ->
// 2.71 ms).  The independent partials march whole bricks without termination,
// like MIP rays, and reading both copies there measured no faster (9.6-10.1 ->
// 10.2 ms): they read the store alone.
template <typename T, bool CARRIED, bool PAIRED>
__global__ void __launch_bounds__(128)
k_brick_partial(const __grid_constant__ SortParams P, int layer_begin, int layer_end) {
    __shared__ float4 s_tf[kMaxTF];
    for (int i = threadIdx.x; i < P.tf.n; i += blockDim.x) s_tf[i] = P.tf.tab[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    // the bricks of layers [layer_begin, layer_end) of the ordered list, or an explicit subset
    const int* order = P.sub_order ? P.sub_order : P.order;
    const int* tile_start = P.sub_order ? P.sub_tile : P.tile_start;
    const int first = P.sub_order ? 0 : P.layer_start[layer_begin];
    const int end = P.sub_order ? P.sub_n : P.layer_start[layer_end];
    const int t0 = tile_start[first], t1 = tile_start[end];
    const T* __restrict__ pool = static_cast<const T*>(P.vol.pool);
    const T* __restrict__ pool1 = static_cast<const T*>(P.vol.pool1);
    const float ert = P.ert;
    auto fetch = [&](const T* slot, const T* slot1, float gx, float gy, float gz) {
        if constexpr (PAIRED) return fetch_trilinear_pair<T>(slot, slot1, P.vol, gx, gy, gz);
        else return fetch_trilinear<T>(slot, P.vol, gx, gy, gz);
    };
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(P.work, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        const int gt = t0 + item;
        if (gt >= t1) break;
        // ordered position whose tiles hold gt: tile_start[idx] <= gt < tile_start[idx + 1]
        int lo = first, hi = end - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tile_start[mid] <= gt) lo = mid; else hi = mid - 1;
        }
        const int b = order[lo];
        const BrickFoot f = P.foot[b];
        const int4 rect = f.rect;
        const int tx_n = (rect.z - rect.x + 1 + 7) / 8;
        const int rem = gt - tile_start[lo];
        const int ty = rem / tx_n, tx = rem - ty * tx_n;
        const int px = rect.x + tx * 8 + (lane & 7), py = rect.y + ty * 4 + (lane >> 3);
        if (px > rect.z || py > rect.w) continue;  // ragged tile; the lane rejoins at the shuffle
        const long long pix = (long long)py * P.cam.width + px;
        const int bx = b % P.vol.nbx, by = (b / P.vol.nbx) % P.vol.nby, bz = b / (P.vol.nbx * P.vol.nby);
        float C0 = 0.f, C1 = 0.f, C2 = 0.f, Tr = 1.f;
        if (CARRIED) {
            const float4 st = P.state[pix];
            C0 = st.x;
            C1 = st.y;
            C2 = st.z;
            Tr = st.w;
            if (1.f - Tr >= ert) continue;  // terminated: nothing to add
        }
        float g[3], e[3];
        int ka, kb;
        const int2 kr = P.krange[pix];
        const bool any = kr.x < kr.y && brick_segment(P, px, py, kr, bx, by, bz, g, e, ka, kb);
        if (!CARRIED && P.mode == VR_MIP) {  // the brick's maximum (object-space MIP)
            float m = -INFINITY;
            if (any) {
                const long long base = (long long)P.vol.table[b] * P.vol.slot_elems;
                const T* slot = pool + base;
                const T* slot1 = PAIRED ? pool1 + base : nullptr;
                for (int j = 0; j < kb - ka; ++j) {
                    const float fj = (float)j;
                    m = fmaxf(m, fetch(slot, slot1, fmaf(fj, e[0], g[0]), fmaf(fj, e[1], g[1]), fmaf(fj, e[2], g[2])));
                }
            }
            const int rw = rect.z - rect.x + 1;
            P.partial[f.offset + (long long)(py - rect.y) * rw + (px - rect.x)] = make_float4(m, 0.f, 0.f, 0.f);
            continue;
        }
        if (any) {
            const long long base = (long long)P.vol.table[b] * P.vol.slot_elems;
            const T* slot = pool + base;
            const T* slot1 = PAIRED ? pool1 + base : nullptr;
            // at most ~4 B samples per brick: FP32 stepping from the float-float anchor
            // stays within 2e-5 voxel
            for (int j = 0; j < kb - ka; ++j) {
                const float fj = (float)j;
                const float v = fetch(slot, slot1, fmaf(fj, e[0], g[0]), fmaf(fj, e[1], g[1]), fmaf(fj, e[2], g[2]));
                const float4 c = tf_lookup(s_tf, P.tf.n, P.tf.vmin, P.tf.inv_range, v);
                const float w = Tr * c.w;
                C0 = fmaf(w, c.x, C0);
                C1 = fmaf(w, c.y, C1);
                C2 = fmaf(w, c.z, C2);
                Tr = Tr * (1.f - c.w);
                if (CARRIED && 1.f - Tr >= ert) break;
            }
        }
        if (CARRIED) {
            if (any) P.state[pix] = make_float4(C0, C1, C2, Tr);
        } else {
            const int rw = rect.z - rect.x + 1;
            P.partial[f.offset + (long long)(py - rect.y) * rw + (px - rect.x)] = make_float4(C0, C1, C2, Tr);
        }
    }
}

// Fold the partial images per pixel in visibility order.  Block = 16 x 16
// pixels; the block first lists (in order) the bricks whose rectangle meets it.
__global__ void __launch_bounds__(256) k_sortlast_fold(const __grid_constant__ SortParams P) {
    __shared__ int s_list[2048];
    __shared__ int s_n, s_chunk_n;
    __shared__ int s_warp_cnt[8];
    const int tid = threadIdx.x;
    const int ylim = P.fold_rows > 0 ? P.fold_y0 + P.fold_rows : P.cam.height;  // rows folded: [.., ylim)
    const int x0 = blockIdx.x * 16, y0 = P.fold_y0 + blockIdx.y * 16;
    const int px = x0 + (tid & 15), py = y0 + (tid >> 4);
    const int nvis = P.layer_start[P.max_layers];
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, Tr = 1.f, M = -INFINITY;
    for (int base = 0; base < nvis; base += 2048) {
        if (tid == 0) s_n = 0;
        __syncthreads();
        // ordered compaction of the bricks meeting this block, 256 at a time
        for (int c = base; c < min(nvis, base + 2048); c += 256) {
            const int i = c + tid;
            bool hit = false;
            int b = -1;
            if (i < nvis) {
                b = P.order[i];
                const int4 r = P.foot[b].rect;
                hit = r.x <= x0 + 15 && r.z >= x0 && r.y <= y0 + 15 && r.w >= y0;
            }
            const unsigned int m = __ballot_sync(0xffffffffu, hit);
            const int warp = tid >> 5, lane = tid & 31;
            if (lane == 0) s_warp_cnt[warp] = __popc(m);
            __syncthreads();
            int before = 0;
            for (int w = 0; w < warp; ++w) before += s_warp_cnt[w];
            if (hit) s_list[s_n + before + __popc(m & ((1u << lane) - 1u))] = b;
            __syncthreads();
            if (tid == 0) {
                int t = 0;
                for (int w = 0; w < 8; ++w) t += s_warp_cnt[w];
                s_chunk_n = t;
            }
            __syncthreads();
            if (tid == 0) s_n += s_chunk_n;
            __syncthreads();
        }
        const int n = s_n;
        if (px < P.cam.width && py < ylim) {
            for (int q = 0; q < n; ++q) {
                const BrickFoot f = P.foot[s_list[q]];
                if (px < f.rect.x || px > f.rect.z || py < f.rect.y || py > f.rect.w) continue;
                const int rw = f.rect.z - f.rect.x + 1;
                const float4 p = P.partial[f.offset + (long long)(py - f.rect.y) * rw + (px - f.rect.x)];
                if (P.mode == VR_MIP) {
                    M = fmaxf(M, p.x);
                } else {
                    C0 = fmaf(Tr, p.x, C0);
                    C1 = fmaf(Tr, p.y, C1);
                    C2 = fmaf(Tr, p.z, C2);
                    Tr *= p.w;
                }
            }
        }
        __syncthreads();
    }
    if (px < P.cam.width && py < ylim) {
        const long long o = (long long)(py - P.fold_y0) * P.cam.width + px;
        if (P.mode == VR_MIP)
            P.out_rgba[o] = M > -INFINITY ? tf_lookup(P.tf.tab, P.tf.n, P.tf.vmin, P.tf.inv_range, M)
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
        else
            P.out_rgba[o] = make_float4(C0, C1, C2, 1.f - Tr);
    }
}

__global__ void k_state_init(const __grid_constant__ SortParams P) {
    const long long n = (long long)P.cam.width * P.cam.height;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        P.state[i] = make_float4(0.f, 0.f, 0.f, 1.f);
}

__global__ void k_state_finish(const __grid_constant__ SortParams P) {
    const long long n = (long long)P.cam.width * P.cam.height;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float4 s = P.state[i];
        P.out_rgba[i] = make_float4(s.x, s.y, s.z, 1.f - s.w);
    }
}

template <typename T, bool CARRIED>
cudaError_t partial_t(const SortParams& p, int l0, int l1, int grid, cudaStream_t s) {
    if constexpr (sizeof(T) == 2 && CARRIED) {
        if (p.vol.pool1) {
            k_brick_partial<T, CARRIED, true><<<grid, 128, 0, s>>>(p, l0, l1);
            return cudaGetLastError();
        }
    }
    k_brick_partial<T, CARRIED, false><<<grid, 128, 0, s>>>(p, l0, l1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_brick_footprints(const SortParams& p, cudaStream_t s) {
    const int nb = p.vol.nbx * p.vol.nby * p.vol.nbz;
    k_brick_footprints<<<std::min((nb + 255) / 256, 1024), 256, 0, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_layer_scan<<<1, 32, 0, s>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_layer_scatter<<<std::min((nb + 255) / 256, 1024), 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_tile_scan(const SortParams& p, cudaStream_t s) {
    k_tile_scan<<<1, 32, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_brick_partial(const SortParams& p, vr_dtype dt, bool carried, int l0, int l1, int grid,
                                 cudaStream_t s) {
    if (dt == VR_F32) return carried ? partial_t<float, true>(p, l0, l1, grid, s) : partial_t<float, false>(p, l0, l1, grid, s);
    if (dt == VR_F16) return carried ? partial_t<__half, true>(p, l0, l1, grid, s) : partial_t<__half, false>(p, l0, l1, grid, s);
    return carried ? partial_t<__nv_bfloat16, true>(p, l0, l1, grid, s)
                   : partial_t<__nv_bfloat16, false>(p, l0, l1, grid, s);
}

cudaError_t launch_sortlast_fold(const SortParams& p, cudaStream_t s) {
    const int rows = p.fold_rows > 0 ? p.fold_rows : p.cam.height;
    dim3 grid((p.cam.width + 15) / 16, (rows + 15) / 16);
    k_sortlast_fold<<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_state_init(const SortParams& p, cudaStream_t s) {
    k_state_init<<<1024, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_state_finish(const SortParams& p, cudaStream_t s) {
    k_state_finish<<<1024, 256, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace vr

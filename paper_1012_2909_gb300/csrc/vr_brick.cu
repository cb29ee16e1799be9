// Object-order brick pass for maximum-intensity projection.
//
// The paper decomposes a cube larger than one node's memory into pieces that
// are rendered separately and combined (Abstract, Sec. 1).  On one GPU the
// same decomposition streams the cube through shared memory exactly once: CTAs
// claim cells (32^3 interior voxels of a brick + a 1-voxel ghost layer), stage
// each with one TMA copy, and march every ray segment that crosses the staged
// cell, G lanes per segment on interleaved samples.  Partial maxima are folded
// with an atomic maximum, which is exact and order-free, so the result equals
// the per-ray maximum.
//
// Sample ownership: along each axis the cell faces are planes X; the sample
// index where a ray crosses X is kappa(X) = (X - o)/e in FP32, the same number
// in both cells that share the face, and monotone in X.  The intervals
// [ceil(kappa(X_i)), ceil(kappa(X_i+1))) therefore partition the ray's samples
// among the cells (the outermost faces are pushed to infinity), clipped to the
// ray's [k0, k1) from the pixel set-up.  Positions are anchored in
// float-float at the first sample of each segment and stepped in FP32.
#include <algorithm>

#include "vr_device.cuh"
#include "vr_ff.cuh"
#include "vr_tma.cuh"

namespace vr {

namespace {

// Two CTAs of 512 threads per SM: 32 warps at the 64-register limit (the march
// is latency-bound; 256-thread CTAs were 9-11 % slower).
constexpr int kBrickThreads = 512;
constexpr int kSegCap = 512;  // segment records per chunk
static_assert(kSegCap % kBrickThreads == 0, "segment chunk must be a multiple of the CTA size");
constexpr int kUnroll = 1;  // samples per lane per step (2 measured no faster)

// Staged cell: CX x CY x CZ interior voxels, TMA box BX x BY x BZ (ghost
// included, x padded to 16 bytes).  The 16-bit box has one spare row (BY = 35,
// never read back): the slab stride becomes 700 words, 28 banks apart instead
// of 8, which spreads the gathers of neighbouring z-slabs over the banks
// (1 % faster over the survey orbit; the largest box that keeps two CTAs per SM).
template <typename T> struct Cell;
template <> struct Cell<float> {
    static constexpr int CX = 32, CY = 32, CZ = 16, BX = 36, BY = 34, BZ = 18;
};
template <> struct Cell<__half> {
    static constexpr int CX = 32, CY = 32, CZ = 32, BX = 40, BY = 35, BZ = 34;
};
template <> struct Cell<__nv_bfloat16> {
    static constexpr int CX = 32, CY = 32, CZ = 32, BX = 40, BY = 35, BZ = 34;
};

template <typename T> struct TileGeom {
    static constexpr int BYTES = Cell<T>::BX * Cell<T>::BY * Cell<T>::BZ * (int)sizeof(T);
    static constexpr int STRIDE = (BYTES + 127) / 128 * 128;
    static constexpr int SMEM = STRIDE + kSegCap * 32;
};

struct SegRec {
    int pix, n;
    float gx, gy, gz, ex, ey, ez;
};

__device__ __forceinline__ unsigned int ord_enc(float f) {
    const unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord_dec(unsigned int e) {
    return __uint_as_float((e & 0x80000000u) ? (e & 0x7fffffffu) : ~e);
}

template <typename T> __device__ __forceinline__ float cvt(T v);
template <> __device__ __forceinline__ float cvt<float>(float v) { return v; }
template <> __device__ __forceinline__ float cvt<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float cvt<__nv_bfloat16>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}

// (float)a - b with one rounding.  For 16-bit a this is the mixed-precision
// form of sub (the operand is widened exactly), one instruction instead of a
// conversion and an FP32 subtraction, with the same result.
template <typename T> __device__ __forceinline__ float sub_wide(T a, float b);
template <> __device__ __forceinline__ float sub_wide<float>(float a, float b) { return a - b; }
template <> __device__ __forceinline__ float sub_wide<__half>(__half a, float b) {
    float d;
    asm("sub.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(__half_as_ushort(a)), "f"(b));
    return d;
}
template <> __device__ __forceinline__ float sub_wide<__nv_bfloat16>(__nv_bfloat16 a, float b) {
    float d;
    asm("sub.rn.f32.bf16 %0, %1, %2;" : "=f"(d) : "h"(__bfloat16_as_ushort(a)), "f"(b));
    return d;
}

// Two-wide FP32 operations (each lane rounds like its scalar form).  Used for
// the pair of y-lerps of a fetch (measured: packing the x-lerps gained nothing,
// packing position and fraction was slower).
__device__ __forceinline__ unsigned long long pk(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 upk(unsigned long long v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Trilinear fetch from a staged cell; g in tile coordinates (lower corner
// floor(g), 0 = ghost).  CLAMP keeps every access inside the tile; without it
// the caller guarantees 0 <= g < extent + 1 on every axis.  BY: rows of a slab
// of the staged box.
template <typename T, bool CLAMP, int BY = Cell<T>::BY>
__device__ __forceinline__ float tile_fetch(const T* __restrict__ t, float gx, float gy, float gz) {
    using C = Cell<T>;
    if (CLAMP) {
        gx = fminf(fmaxf(gx, 0.f), (float)C::CX + 0.999f);
        gy = fminf(fmaxf(gy, 0.f), (float)C::CY + 0.999f);
        gz = fminf(fmaxf(gz, 0.f), (float)C::CZ + 0.999f);
    }
    const float x0 = floorf(gx), y0 = floorf(gy), z0 = floorf(gz);
    const float fx = gx - x0, fy = gy - y0, fz = gz - z0;
    const int i = (int)fmaf(fmaf(z0, (float)BY, y0), (float)C::BX, x0);
    constexpr int SY = C::BX, SZ = C::BX * BY;
    const float c000 = cvt<T>(t[i]), c010 = cvt<T>(t[i + SY]);
    const float c001 = cvt<T>(t[i + SZ]), c011 = cvt<T>(t[i + SZ + SY]);
    const float a0 = fmaf(fx, sub_wide<T>(t[i + 1], c000), c000);
    const float a1 = fmaf(fx, sub_wide<T>(t[i + SY + 1], c010), c010);
    const float a2 = fmaf(fx, sub_wide<T>(t[i + SZ + 1], c001), c001);
    const float a3 = fmaf(fx, sub_wide<T>(t[i + SZ + SY + 1], c011), c011);
    // y-lerps as one two-wide subtract and FMA: (b0, b1) = (a0, a2) + fy ((a1, a3) - (a0, a2))
    const unsigned long long a02 = pk(a0, a2);
    const float2 b = upk(fma2(pk(fy, fy), sub2(pk(a1, a3), a02), a02));
    return fmaf(fz, b.y - b.x, b.x);
}


// Conservative pixel rectangle of the rays that can cross the box [lo, hi].
__device__ bool cell_rect(const CamFF& c, float3 lo, float3 hi, int4& r) {
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

// Geometry of work unit u = brick * ncells + cell: lower corner and TMA
// coordinates; false if the cell lies outside the cube or its brick is absent.
template <typename T>
__device__ bool unit_cell(const BrickParams& P, int u, float3& lo, int4& coord) {
    using C = Cell<T>;
    const VolDev& v = P.vol;
    const int ncells = P.ncells_x * P.ncells_y * P.ncells_z;
    const int brick = u / ncells, cell = u - brick * ncells;
    const int bx = brick % v.nbx, by = (brick / v.nbx) % v.nby, bz = brick / (v.nbx * v.nby);
    const int cx = cell % P.ncells_x, cy = (cell / P.ncells_x) % P.ncells_y,
              cz = cell / (P.ncells_x * P.ncells_y);
    const int ox = bx * v.B + cx * C::CX, oy = by * v.B + cy * C::CY, oz = bz * v.B + cz * C::CZ;
    if (ox >= v.nx || oy >= v.ny || oz >= v.nz) return false;
    lo = make_float3((float)ox, (float)oy, (float)oz);
    coord = make_int4(cx * C::CX, cy * C::CY, cz * C::CZ, v.table[brick]);
    return coord.w >= 0;
}

// Local visibility key of the cell of unit u (TMA coordinates coord) within its
// brick, as BrickParams describes: it grows along every ray, and no ray crosses
// two cells of one brick with the same key.
template <typename T>
__device__ int cell_key(const BrickParams& P, int u, int4 coord) {
    using C = Cell<T>;
    const VolDev& v = P.vol;
    const int brick = u / (P.ncells_x * P.ncells_y * P.ncells_z);
    const int b3[3] = {brick % v.nbx, (brick / v.nbx) % v.nby, brick / (v.nbx * v.nby)};
    const int nc[3] = {P.ncells_x, P.ncells_y, P.ncells_z};
    const int c3[3] = {coord.x / C::CX, coord.y / C::CY, coord.z / C::CZ};
    int key = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (P.key_persp) {
            const int lo = b3[a] * nc[a], hi = lo + nc[a] - 1, e = P.eye_cell[a];
            key += abs(lo + c3[a] - e) - max(0, max(lo - e, e - hi));
        } else {
            key += P.key_sign[a] > 0 ? c3[a] : (P.key_sign[a] < 0 ? nc[a] - 1 - c3[a] : 0);
        }
    }
    return key;
}

template <typename T>
__device__ __forceinline__ bool cam_cell_rect(const CamFF& c, float3 lo, int4& rect) {
    using C = Cell<T>;
    const float3 hi = make_float3(lo.x + (float)C::CX, lo.y + (float)C::CY, lo.z + (float)C::CZ);
    return cell_rect(c, lo, hi, rect);
}

// Segment of pixel (px, py) inside the cell whose lower corner is lo; false if
// the ray owns no sample there.
template <typename T>
__device__ __forceinline__ bool make_segment(const BrickParams& P, const CamFF& c, int px, int py,
                                             int2 kr, float3 lo, const float4* pd, SegRec& s) {
    using C = Cell<T>;
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
    const float lo3[3] = {lo.x, lo.y, lo.z};
    const int ext[3] = {C::CX, C::CY, C::CZ};
    const int n3[3] = {P.vol.nx, P.vol.ny, P.vol.nz};
    float klo = -1e9f, khi = 1e9f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const bool first = lo3[a] <= 0.f;
        const bool last = (int)lo3[a] + ext[a] >= n3[a];
        const float xl = lo3[a], xh = lo3[a] + (float)ext[a];
        if (e[a] != 0.f) {
            const float inv = __fdividef(1.0f, e[a]);  // any fixed reciprocal keeps kappa
                                                       // deterministic and monotone in X
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
    const int ka = max((int)ceilf(klo), kr.x);
    const int kb = min((int)ceilf(khi), kr.y);
    if (ka >= kb) return false;
    // float-float anchor of sample ka
    ff E[3], O[3];
    if (c.type == 1 && pd) {  // step vector from the pixel set-up
        const float4 d0 = pd[0], d1 = pd[1];
        E[0] = ff{d0.x, d0.w};
        E[1] = ff{d0.y, d1.x};
        E[2] = ff{d0.z, d1.y};
#pragma unroll
        for (int a = 0; a < 3; ++a) O[a] = ff{c.org_hi[a], c.org_lo[a]};
    } else if (c.type == 1) {
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
    float g[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const ff p = ff_add(O[a], ff_mul(E[a], fk));
        g[a] = __fadd_rn(__fsub_rn(p.hi, lo3[a]), p.lo) + 0.5f;
    }
    // Samples lie on the segment between the first and the last one, so if both
    // are inside [eps, extent + 1 - eps) every sample is; otherwise flag the
    // segment for the clamped fetch (bit 31 of n).
    bool inside = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float ea = a == 0 ? E[0].hi : (a == 1 ? E[1].hi : E[2].hi);
        const float gend = fmaf((float)(kb - ka - 1), ea, g[a]);
        const float top = (float)ext[a] + 1.0f - 1e-3f;
        inside = inside && g[a] >= 1e-3f && g[a] < top && gend >= 1e-3f && gend < top;
    }
    s.pix = py * c.width + px;  // the caller adds the camera's image offset
    s.n = (kb - ka) | (inside ? 0 : (int)0x80000000u);
    s.gx = g[0];
    s.gy = g[1];
    s.gz = g[2];
    s.ex = E[0].hi;
    s.ey = E[1].hi;
    s.ez = E[2].hi;
    return true;
}

struct CellDesc {
    float4 lo;    // lower corner (world voxels); w: the brick id (int bits)
    int4 coord;   // TMA coordinates x, y, z (slot elements), slot
    int4 rect0;   // pixel rectangle of camera 0 (empty: x > z)
};

// Compacted list of the cells that some pixel of some camera can reach, in
// roughly linear cell order (warp-aggregated appends), so that neighbouring
// cells -- which share ghost voxels through L2 -- run close in time.
template <typename T>
__global__ void k_cell_list(const __grid_constant__ BrickParams P, CellDesc* __restrict__ list,
                            int* __restrict__ count) {
    // units: every cell of every brick, or of the bricks of an explicit list
    const int ncells = P.ncells_x * P.ncells_y * P.ncells_z;
    const int nunits = (P.brick_list ? P.nlist : P.nbricks) * ncells;
    const int lane = threadIdx.x & 31;
    for (int u0 = blockIdx.x * blockDim.x; u0 < nunits; u0 += gridDim.x * blockDim.x) {
        int u = u0 + threadIdx.x;
        if (P.brick_list && u < nunits) u = P.brick_list[u / ncells] * ncells + u % ncells;
        float3 lo;
        int4 coord;
        bool ok = u0 + threadIdx.x < nunits && unit_cell<T>(P, u, lo, coord);
        if (ok && P.key_pass > 0) ok = cell_key<T>(P, u, coord) == P.key_pass - 1;
        int4 rect0 = make_int4(0, 0, -1, -1);
        if (ok) {
            bool any = cam_cell_rect<T>(P.cams[0], lo, rect0);
            if (!any) rect0 = make_int4(0, 0, -1, -1);
            for (int c = 1; c < P.ncams && !any; ++c) {
                int4 rect;
                any = cam_cell_rect<T>(P.cams[c], lo, rect);
            }
            ok = any;
        }
        const unsigned int m = __ballot_sync(0xffffffffu, ok);
        int base = 0;
        if (lane == 0 && m) base = atomicAdd(count, __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (ok) {
            CellDesc d;
            d.lo = make_float4(lo.x, lo.y, lo.z, __int_as_float(u / ncells));
            d.coord = coord;
            d.rect0 = rect0;
            list[base + __popc(m & ((1u << lane) - 1u))] = d;
        }
    }
}

// One chunk of camera cam's pixel rectangle of a cell -> segment records (phase 1).
// Records of at most kShortRounds group rounds ("short") fill the chunk's buffer
// from the back, the others from the front, so that the groups of a warp see
// segments of similar length without a sorting pass.
constexpr int kShortRounds = 3;

template <typename T, bool ONE, int G>
__device__ __forceinline__ void build_segments(const BrickParams& P, const CamFF& c, int cam_, int4 rect,
                                               float3 lo, int c0, SegRec* segs, int* cnt, int tid) {
    const int cam = ONE ? 0 : cam_;
    const long long img = (long long)P.width * P.height;
    const int2* kr_img = P.krange + (long long)cam * img;
    const float4* pd_img = P.pixdir ? P.pixdir + 2 * (long long)cam * img : nullptr;
    const int rw = rect.z - rect.x + 1;
    const int npx = rw * (rect.w - rect.y + 1);
    const int c1 = min(npx, c0 + kSegCap);
    const float inv_rw = 1.0f / (float)rw;
    constexpr int PER = kSegCap / kBrickThreads;
    int2 kr[PER];
    int pxv[PER], pyv[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int i = c0 + tid + q * kBrickThreads;
        // row i / rw from a float reciprocal (off by at most one), then corrected
        int row = (int)(((float)i + 0.5f) * inv_rw), col = i - row * rw;
        if (col < 0) {
            --row;
            col += rw;
        } else if (col >= rw) {
            ++row;
            col -= rw;
        }
        kr[q] = make_int2(0, 0);
        pyv[q] = rect.y + row;
        pxv[q] = rect.x + col;
        if (i < c1) kr[q] = kr_img[pyv[q] * P.width + pxv[q]];
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        if (kr[q].x >= kr[q].y) continue;
        SegRec s;
        const float4* pd = pd_img ? pd_img + 2 * ((long long)pyv[q] * P.width + pxv[q]) : nullptr;
        if (make_segment<T>(P, c, pxv[q], pyv[q], kr[q], lo, pd, s)) {
            s.pix += (int)(cam * img);
            if ((s.n & 0x7fffffff) > kShortRounds * G * kUnroll)
                segs[atomicAdd(&cnt[0], 1)] = s;
            else
                segs[kSegCap - 1 - atomicAdd(&cnt[1], 1)] = s;
        }
    }
}

// Phase 2: groups of G lanes per segment record (32/G records per warp at a
// time, consecutive records -- neighbouring pixels, similar lengths), lane r of
// a group on samples j = r, r + G, ...; U samples per lane per step so that
// their dependency chains overlap.  Lanes past the end of their segment
// re-sample its last sample: a maximum is unchanged by repeats, and the step
// stays free of divergent branches.  The maximum of a group is folded with
// redux.sync on its ordered-int encoding.
template <typename T, int G, int U, bool CLAMP>
__device__ __forceinline__ float group_max(const T* __restrict__ tile, const SegRec& s, int n, int r,
                                           int iters) {
    float m = -INFINITY;
    const float last = (float)(n - 1);
    float fr = (float)r;  // sample index of this lane (integers < 2^24 are exact)
    for (int it = 0; it < iters; ++it, fr += (float)(U * G)) {
        float v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const float f = fminf(fr + (float)(u * G), last);
            v[u] = tile_fetch<T, CLAMP>(tile, fmaf(f, s.ex, s.gx), fmaf(f, s.ey, s.gy), fmaf(f, s.ez, s.gz));
        }
#pragma unroll
        for (int u = 0; u < U; ++u) m = fmaxf(m, v[u]);
    }
    return m;
}

// Warps claim batches of 32/G records from a shared counter, so that the
// barrier at the end of a chunk waits for at most one batch per warp.
template <typename T, int G, int U>
__device__ __forceinline__ void march_segments(const BrickParams& P, const T* tile, const SegRec* segs,
                                               int nlong, int nshort, int* claim, int lane) {
    constexpr int PER_WARP = 32 / G;
    const int q = lane / G, r = lane % G;
    // batches never mix the lists: the long list is padded to whole batches
    const int nlong_pad = (nlong + PER_WARP - 1) / PER_WARP * PER_WARP;
    for (;;) {
        int s0 = 0;
        if (lane == 0) s0 = atomicAdd(claim, PER_WARP);
        s0 = __shfl_sync(0xffffffffu, s0, 0);
        if (s0 >= nlong_pad + nshort) break;
        // groups past the end of a list repeat its last record (no atomics)
        const bool in_long = s0 < nlong_pad;
        const int j0 = in_long ? s0 : s0 - nlong_pad, nseg = in_long ? nlong : nshort;
        const int j = min(j0 + q, nseg - 1);
        const SegRec s = segs[in_long ? j : kSegCap - 1 - j];
        const int n = s.n & 0x7fffffff;
        const int iters = (int)__reduce_max_sync(0xffffffffu, (unsigned int)((n + U * G - 1) / (U * G)));
        float m;
        if (!__any_sync(0xffffffffu, s.n < 0))
            m = group_max<T, G, U, false>(tile, s, n, r, iters);
        else
            m = group_max<T, G, U, true>(tile, s, n, r, iters);
        // maximum over the group's G lanes: xor shuffles stay inside aligned groups
        unsigned int e = ord_enc(m);
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
        if (r == 0 && j0 + q < nseg) atomicMax(&P.out_enc[s.pix], e);
    }
}

// The brick pass.  Two CTAs per SM, each with one staged cell: while a CTA
// waits for the TMA load of its next cell it already turns that cell's pixel
// rectangles into segment records, and the other CTA of the SM marches.  A
// staged cell serves every camera of the launch (the 25 panels of a wall are
// rendered from one pass over the cube).
template <typename T, bool ONE, int GROUP>
__global__ void __launch_bounds__(kBrickThreads, 2)
k_brick_mip(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ BrickParams P,
            const CellDesc* __restrict__ list, const int* __restrict__ count) {
    using G = TileGeom<T>;
    extern __shared__ __align__(128) unsigned char smem[];
    T* tile = reinterpret_cast<T*>(smem);
    SegRec* segs = reinterpret_cast<SegRec*>(smem + G::STRIDE);
    __shared__ __align__(8) uint64_t bar;
    // three descriptor slots: the unit in progress, the one being loaded, and the
    // one being claimed -- a slot is refilled two units after its last reader
    __shared__ CellDesc s_desc[3];
    __shared__ int4 s_rect[3][kMaxLaunchCams];
    __shared__ int s_u[3];
    __shared__ int s_cnt[2][2];  // per chunk parity: long, short records
    __shared__ int s_claim[2];
    // the camera of the chunk being built: one camera reads its parameters at
    // constant offsets; with several, the chunk's camera is copied here so that
    // the segment build does not index the parameter space dynamically
    __shared__ __align__(16) CamFF s_cam;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nvalid = *count;
    auto stage_cam = [&](int cam) {
        if (ONE) return;
        const int* src = reinterpret_cast<const int*>(&P.cams[cam]);
        int* dst = reinterpret_cast<int*>(&s_cam);
        for (int i = tid; i < (int)(sizeof(CamFF) / sizeof(int)); i += kBrickThreads) dst[i] = src[i];
        __syncthreads();
    };
    const CamFF& cam_ref = ONE ? P.cams[0] : s_cam;
    const int ncams = ONE ? 1 : P.ncams;
    // warp 0: claim the next unit into descriptor slot `slot`, with its pixel
    // rectangle for every camera (camera 0 from the list, the others one lane each)
    auto claim = [&](int slot) {
        int u = 0;
        if (lane == 0) u = atomicAdd(P.work, 1);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (lane == 0) s_u[slot] = u;
        if (u < nvalid) {
            const CellDesc d = list[u];
            if (lane == 0) {
                s_desc[slot] = d;
                s_rect[slot][0] = d.rect0;
            }
            if (lane > 0 && lane < ncams) {
                int4 r;
                if (!cam_cell_rect<T>(P.cams[lane], make_float3(d.lo.x, d.lo.y, d.lo.z), r))
                    r = make_int4(0, 0, -1, -1);
                s_rect[slot][lane] = r;
            }
        }
    };
    auto load = [&](const CellDesc& d) {  // thread 0: stage a cell
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bar, (uint32_t)G::BYTES);
        tma_load_4d(tile, &tmap, &bar, d.coord.x, d.coord.y, d.coord.z, d.coord.w);
    };
    // next (camera, first pixel) of the current unit after (cam, c0), or cam = ncams
    auto next_chunk = [&](int slot, int& cam, int& c0) {
        for (;;) {
            if (cam < ncams) {
                const int4 r = s_rect[slot][cam];
                const int npx = (r.z - r.x + 1) * (r.w - r.y + 1);
                if (r.z >= r.x && r.w >= r.y && c0 < npx) return;
            }
            if (cam >= ncams) return;
            ++cam;
            c0 = 0;
        }
    };

    if (warp == 0) {
        if (lane == 0) {
            mbar_init(&bar, 1);
            fence_mbar_init();
            s_cnt[0][0] = s_cnt[0][1] = 0;
            s_cnt[1][0] = s_cnt[1][1] = 0;
            s_claim[0] = 0;
        }
        claim(0);
        if (s_u[0] < nvalid) {
            if (lane == 0) load(s_desc[0]);
            claim(1);
        }
    }
    __syncthreads();
    if (s_u[0] >= nvalid) return;

    int cur = 0, chunk = 0, cam = 0, c0 = 0;
    uint32_t phase = 0;
    next_chunk(cur, cam, c0);
    float3 lo = make_float3(s_desc[cur].lo.x, s_desc[cur].lo.y, s_desc[cur].lo.z);
    if (cam < ncams) {
        stage_cam(cam);
        build_segments<T, ONE, GROUP>(P, cam_ref, cam, s_rect[cur][cam], lo, c0, segs, s_cnt[0], tid);
    }
    bool ok = mbar_wait(&bar, phase, P.status);
    phase ^= 1u;
    // A failed wait (2 s without the copy completing) means a stalled copy: the CTA
    // stops here and the next call reports the status.  That recovery assumes the
    // copy never lands; one that completed later would write into the shared memory
    // of a CTA that has exited.
    if (!__syncthreads_and(ok)) return;
    for (;;) {
        const int nlong = s_cnt[chunk & 1][0], nshort = s_cnt[chunk & 1][1];
        if (tid == 0) {
            s_cnt[(chunk + 1) & 1][0] = 0;
            s_cnt[(chunk + 1) & 1][1] = 0;
            s_claim[(chunk + 1) & 1] = 0;
        }
        march_segments<T, GROUP, kUnroll>(P, tile, segs, nlong, nshort, &s_claim[chunk & 1], lane);
        __syncthreads();
        ++chunk;
        c0 += kSegCap;
        next_chunk(cur, cam, c0);
        if (cam < ncams) {  // more pixels of the same cell
            stage_cam(cam);
            build_segments<T, ONE, GROUP>(P, cam_ref, cam, s_rect[cur][cam], lo, c0, segs, s_cnt[chunk & 1], tid);
            __syncthreads();
            continue;
        }
        const int nxt = cur == 2 ? 0 : cur + 1;
        if (s_u[nxt] >= nvalid) break;
        if (tid == 0) load(s_desc[nxt]);
        cur = nxt;
        cam = 0;
        c0 = 0;
        next_chunk(cur, cam, c0);
        lo = make_float3(s_desc[cur].lo.x, s_desc[cur].lo.y, s_desc[cur].lo.z);
        if (cam < ncams) {
            stage_cam(cam);
            build_segments<T, ONE, GROUP>(P, cam_ref, cam, s_rect[cur][cam], lo, c0, segs, s_cnt[chunk & 1], tid);
        }
        // the slot after `cur` was last read two units ago: refill it now
        if (warp == 0) claim(cur == 2 ? 0 : cur + 1);
        ok = mbar_wait(&bar, phase, P.status);
        phase ^= 1u;
        if (!__syncthreads_and(ok)) return;
    }
}

// ---------------------------------------------------------------------------
// Sort-last partial images through staged cells: the images of the separately
// rendered parts of a cube, combined afterwards (Abstract, Sec. 1), with the
// bricks as the parts.
//
// The partial image of a brick holds, per pixel, the "over" composite from T = 1
// of the ray's samples that the brick owns (the maximum of their values for
// MIP).  The brick's cells split those samples by the same face-crossing rule,
// so the partial is the front-to-back fold of the pixel's cell segments.  Each
// visibility pass stages the cells of one local key (k_cell_list), marches each
// segment with G lanes on contiguous runs of samples, joins the runs in ray
// order, and folds the segment into the brick's slot: C += T C_seg, T *= T_seg
// (or the maximum).  Slots start as the empty image (0, 0, 0, 1), or -inf.

// Staged box without the spare row (the partial pass also holds the table).
template <typename T> struct PartGeom {
    static constexpr int BY = Cell<T>::CY + 2;
    static constexpr int BYTES = Cell<T>::BX * BY * Cell<T>::BZ * (int)sizeof(T);
    static constexpr int STRIDE = (BYTES + 127) / 128 * 128;
    static constexpr int SMEM = STRIDE + kSegCap * (int)sizeof(SegRec) + kMaxPartTF * (int)sizeof(float4);
};

// Segment records of one chunk of a cell's pixel rectangle, each pointing at its
// slot in the partial image of the cell's brick (foot).  Records of at most
// kShortRounds group rounds fill the buffer from the back, as in the MIP pass.
template <typename T, int G>
__device__ __forceinline__ void build_part_segments(const BrickParams& P, int4 rect, const BrickFoot& f, float3 lo,
                                                    int c0, SegRec* segs, int* cnt, int tid) {
    const CamFF& c = P.cams[0];
    const int rw = rect.z - rect.x + 1;
    const int npx = rw * (rect.w - rect.y + 1);
    const int c1 = min(npx, c0 + kSegCap);
    const float inv_rw = 1.0f / (float)rw;
    const int frw = f.rect.z - f.rect.x + 1;
    constexpr int PER = kSegCap / kBrickThreads;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int i = c0 + tid + q * kBrickThreads;
        if (i >= c1) continue;
        int row = (int)(((float)i + 0.5f) * inv_rw), col = i - row * rw;
        if (col < 0) {
            --row;
            col += rw;
        } else if (col >= rw) {
            ++row;
            col -= rw;
        }
        const int py = rect.y + row, px = rect.x + col;
        // a pixel with a sample in the cell lies in its brick's rectangle
        if (px < f.rect.x || px > f.rect.z || py < f.rect.y || py > f.rect.w) continue;
        const long long pix = (long long)py * P.width + px;
        const int2 kr = P.krange[pix];
        if (kr.x >= kr.y) continue;
        const float4* pd = P.pixdir ? P.pixdir + 2 * pix : nullptr;
        SegRec s;
        if (make_segment<T>(P, c, px, py, kr, lo, pd, s)) {
            s.pix = (int)(f.offset + (long long)(py - f.rect.y) * frw + (px - f.rect.x));
            if ((s.n & 0x7fffffff) > kShortRounds * G)
                segs[atomicAdd(&cnt[0], 1)] = s;
            else
                segs[kSegCap - 1 - atomicAdd(&cnt[1], 1)] = s;
        }
    }
}

// One lane's contiguous run of a segment, samples [k0, k0 + L) clipped to n,
// composited from T = 1 (the warp's lanes all take `iters` steps; steps past the
// run add nothing: alpha 0 leaves C and T exactly as they are).
template <typename T, bool CLAMP>
__device__ __forceinline__ void run_over(const T* __restrict__ tile, const float4* __restrict__ s_tf, const TFDev& tf,
                                         const SegRec& s, int n, int k0, int L, int iters, float& C0, float& C1,
                                         float& C2, float& Tr) {
    C0 = C1 = C2 = 0.f;
    Tr = 1.f;
    const float last = (float)(n - 1);
    for (int j = 0; j < iters; ++j) {
        const int k = k0 + j;
        const float f = fminf((float)k, last);
        const float v = tile_fetch<T, CLAMP, PartGeom<T>::BY>(tile, fmaf(f, s.ex, s.gx), fmaf(f, s.ey, s.gy),
                                                              fmaf(f, s.ez, s.gz));
        const float4 c = tf_lookup(s_tf, tf.n, tf.vmin, tf.inv_range, v);
        const float a = (j < L && k < n) ? c.w : 0.f;
        const float w = Tr * a;
        C0 = fmaf(w, c.x, C0);
        C1 = fmaf(w, c.y, C1);
        C2 = fmaf(w, c.z, C2);
        Tr = Tr * (1.f - a);
    }
}

// Maximum over a segment, lane r on samples r, r + G, ... (repeats of the last
// sample change nothing).
template <typename T, int G, bool CLAMP>
__device__ __forceinline__ float run_max(const T* __restrict__ tile, const SegRec& s, int n, int r, int iters) {
    float m = -INFINITY;
    const float last = (float)(n - 1);
    float fr = (float)r;
    for (int it = 0; it < iters; ++it, fr += (float)G) {
        const float f = fminf(fr, last);
        m = fmaxf(m, tile_fetch<T, CLAMP, PartGeom<T>::BY>(tile, fmaf(f, s.ex, s.gx), fmaf(f, s.ey, s.gy),
                                                            fmaf(f, s.ez, s.gz)));
    }
    return m;
}

// Warps claim batches of 32 / G records (as in march_segments); each group of G
// lanes marches one record and its lane 0 folds the result into the record's
// slot.  A pass never holds two records of one slot.
template <typename T, int MODE, int G>
__device__ __forceinline__ void march_part(const BrickParams& P, const T* tile, const float4* s_tf, const TFDev& tf,
                                           const SegRec* segs, int nlong, int nshort, int* claim, int lane) {
    constexpr int PER_WARP = 32 / G;
    const int q = lane / G, r = lane % G;
    const int nlong_pad = (nlong + PER_WARP - 1) / PER_WARP * PER_WARP;
    for (;;) {
        int s0 = 0;
        if (lane == 0) s0 = atomicAdd(claim, PER_WARP);
        s0 = __shfl_sync(0xffffffffu, s0, 0);
        if (s0 >= nlong_pad + nshort) break;
        const bool in_long = s0 < nlong_pad;
        const int j0 = in_long ? s0 : s0 - nlong_pad, nseg = in_long ? nlong : nshort;
        const int j = min(j0 + q, nseg - 1);
        const SegRec s = segs[in_long ? j : kSegCap - 1 - j];
        const int n = s.n & 0x7fffffff;
        const bool writer = r == 0 && j0 + q < nseg;  // groups past the list's end repeat its last record
        const bool clamp = __any_sync(0xffffffffu, s.n < 0);
        if (MODE == VR_MIP) {
            const int iters = (int)__reduce_max_sync(0xffffffffu, (unsigned int)((n + G - 1) / G));
            float m = clamp ? run_max<T, G, true>(tile, s, n, r, iters) : run_max<T, G, false>(tile, s, n, r, iters);
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (writer) {
                float4* d = P.partial + s.pix;
                d->x = fmaxf(d->x, m);
            }
        } else {
            const int L = (n + G - 1) / G;  // samples per lane: lane r takes [r L, r L + L)
            const int iters = (int)__reduce_max_sync(0xffffffffu, (unsigned int)L);
            // the slot's state, read before the march (no other record of this pass
            // writes it), so that its latency hides behind the samples
            float4 p = make_float4(0.f, 0.f, 0.f, 1.f);
            if (writer) p = __ldcg(P.partial + s.pix);
            float C0, C1, C2, Tr;
            if (clamp)
                run_over<T, true>(tile, s_tf, tf, s, n, r * L, L, iters, C0, C1, C2, Tr);
            else
                run_over<T, false>(tile, s_tf, tf, s, n, r * L, L, iters, C0, C1, C2, Tr);
            // join the runs in ray order: (C, T) of lanes r and r + d, then r and r + 2d, ...
#pragma unroll
            for (int d = 1; d < G; d <<= 1) {
                const float p0 = __shfl_down_sync(0xffffffffu, C0, d, G);
                const float p1 = __shfl_down_sync(0xffffffffu, C1, d, G);
                const float p2 = __shfl_down_sync(0xffffffffu, C2, d, G);
                const float pT = __shfl_down_sync(0xffffffffu, Tr, d, G);
                if ((r & (2 * d - 1)) == 0) {
                    C0 = fmaf(Tr, p0, C0);
                    C1 = fmaf(Tr, p1, C1);
                    C2 = fmaf(Tr, p2, C2);
                    Tr *= pT;
                }
            }
            if (writer) {
                p.x = fmaf(p.w, C0, p.x);
                p.y = fmaf(p.w, C1, p.y);
                p.z = fmaf(p.w, C2, p.z);
                p.w *= Tr;
                P.partial[s.pix] = p;
            }
        }
    }
}

// One pass of the sort-last partials: two CTAs per SM, one staged cell each
// (the same claim / stage / build pipeline as k_brick_mip, one camera).
template <typename T, int MODE, int GROUP>
__global__ void __launch_bounds__(kBrickThreads, 2)
k_cell_partial(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ BrickParams P,
               const __grid_constant__ TFDev tf, const CellDesc* __restrict__ list, const int* __restrict__ count) {
    using PG = PartGeom<T>;
    extern __shared__ __align__(128) unsigned char smem[];
    T* tile = reinterpret_cast<T*>(smem);
    SegRec* segs = reinterpret_cast<SegRec*>(smem + PG::STRIDE);
    float4* s_tf = reinterpret_cast<float4*>(smem + PG::STRIDE + kSegCap * sizeof(SegRec));
    __shared__ __align__(8) uint64_t bar;
    __shared__ CellDesc s_desc[3];
    __shared__ BrickFoot s_foot[3];
    __shared__ int s_u[3];
    __shared__ int s_cnt[2][2];
    __shared__ int s_claim[2];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nvalid = *count;
    if (MODE == VR_COMPOSITE)
        for (int i = tid; i < tf.n; i += kBrickThreads) s_tf[i] = tf.tab[i];
    // warp 0: claim the next unit into descriptor slot `slot` (returns the unit)
    auto claim = [&](int slot) {
        int u = 0;
        if (lane == 0) u = atomicAdd(P.work, 1);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (lane == 0) {
            s_u[slot] = u;
            if (u < nvalid) {
                const CellDesc d = list[u];
                s_desc[slot] = d;
                s_foot[slot] = P.foot[__float_as_int(d.lo.w)];
            }
        }
        return u;
    };
    auto load = [&](const CellDesc& d) {  // thread 0: stage a cell
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bar, (uint32_t)PG::BYTES);
        tma_load_4d(tile, &tmap, &bar, d.coord.x, d.coord.y, d.coord.z, d.coord.w);
    };
    auto npx_of = [&](int slot) {
        const int4 r = s_desc[slot].rect0;
        return (r.z - r.x + 1) * (r.w - r.y + 1);  // listed cells have a non-empty rectangle
    };

    if (warp == 0) {
        if (lane == 0) {
            mbar_init(&bar, 1);
            fence_mbar_init();
            s_cnt[0][0] = s_cnt[0][1] = 0;
            s_cnt[1][0] = s_cnt[1][1] = 0;
            s_claim[0] = 0;
        }
        if (claim(0) < nvalid) {
            __syncwarp();
            if (lane == 0) load(s_desc[0]);
            claim(1);
        }
    }
    __syncthreads();
    if (s_u[0] >= nvalid) return;

    int cur = 0, chunk = 0, c0 = 0;
    uint32_t phase = 0;
    float3 lo = make_float3(s_desc[cur].lo.x, s_desc[cur].lo.y, s_desc[cur].lo.z);
    build_part_segments<T, GROUP>(P, s_desc[cur].rect0, s_foot[cur], lo, c0, segs, s_cnt[0], tid);
    bool ok = mbar_wait(&bar, phase, P.status);
    phase ^= 1u;
    // a failed wait (2 s without the copy completing) stops the CTA; the next call
    // reports the status (the recovery assumes that the stalled copy never lands)
    if (!__syncthreads_and(ok)) return;
    for (;;) {
        const int nlong = s_cnt[chunk & 1][0], nshort = s_cnt[chunk & 1][1];
        if (tid == 0) {
            s_cnt[(chunk + 1) & 1][0] = 0;
            s_cnt[(chunk + 1) & 1][1] = 0;
            s_claim[(chunk + 1) & 1] = 0;
        }
        march_part<T, MODE, GROUP>(P, tile, s_tf, tf, segs, nlong, nshort, &s_claim[chunk & 1], lane);
        __syncthreads();
        ++chunk;
        c0 += kSegCap;
        if (c0 < npx_of(cur)) {  // more pixels of the same cell
            build_part_segments<T, GROUP>(P, s_desc[cur].rect0, s_foot[cur], lo, c0, segs, s_cnt[chunk & 1], tid);
            __syncthreads();
            continue;
        }
        const int nxt = cur == 2 ? 0 : cur + 1;
        if (s_u[nxt] >= nvalid) break;
        if (tid == 0) load(s_desc[nxt]);
        cur = nxt;
        c0 = 0;
        lo = make_float3(s_desc[cur].lo.x, s_desc[cur].lo.y, s_desc[cur].lo.z);
        build_part_segments<T, GROUP>(P, s_desc[cur].rect0, s_foot[cur], lo, c0, segs, s_cnt[chunk & 1], tid);
        // the slot after `cur` was last read two units ago: refill it now
        if (warp == 0) claim(cur == 2 ? 0 : cur + 1);
        ok = mbar_wait(&bar, phase, P.status);
        phase ^= 1u;
        if (!__syncthreads_and(ok)) return;
    }
}

__global__ void k_fill_partial(float4* __restrict__ p, long long n, float4 v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

template <typename T, int MODE, int GROUP>
cudaError_t launch_part(const void* tmap, const BrickParams& p, const TFDev& tf, int grid, const CellDesc* list,
                        const int* count, cudaStream_t s) {
    constexpr int SMEM = PartGeom<T>::SMEM;
    cudaError_t e = cudaFuncSetAttribute(k_cell_partial<T, MODE, GROUP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         SMEM);
    if (e != cudaSuccess) return e;
    k_cell_partial<T, MODE, GROUP><<<grid, kBrickThreads, SMEM, s>>>(*static_cast<const CUtensorMap*>(tmap), p, tf,
                                                                      list, count);
    return cudaGetLastError();
}

template <typename T>
cudaError_t cell_partials_t(const void* tmap, const BrickParams& p0, const TFDev& tf, int mode, long long npartial,
                            int npass, int grid, void* cells, cudaStream_t s, int group) {
    CellDesc* list = reinterpret_cast<CellDesc*>(static_cast<char*>(cells) + 256);
    int* count = static_cast<int*>(cells);
    const float4 empty = mode == VR_MIP ? make_float4(-INFINITY, 0.f, 0.f, 0.f) : make_float4(0.f, 0.f, 0.f, 1.f);
    if (npartial > 0) {
        k_fill_partial<<<(int)std::min<long long>((npartial + 255) / 256, 152 * 16), 256, 0, s>>>(p0.partial,
                                                                                                  npartial, empty);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    BrickParams p = p0;
    const int nunits = (p.brick_list ? p.nlist : p.nbricks) * p.ncells_x * p.ncells_y * p.ncells_z;
    for (int pass = 0; pass < npass; ++pass) {
        p.key_pass = pass + 1;
        cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(p.work, 0, sizeof(int), s);
        if (e != cudaSuccess) return e;
        k_cell_list<T><<<std::min((nunits + 255) / 256, 4096), 256, 0, s>>>(p, list, count);
        if (mode == VR_MIP)
            e = group == 4    ? launch_part<T, VR_MIP, 4>(tmap, p, tf, grid, list, count, s)
                : group == 16 ? launch_part<T, VR_MIP, 16>(tmap, p, tf, grid, list, count, s)
                              : launch_part<T, VR_MIP, 8>(tmap, p, tf, grid, list, count, s);
        else
            e = group == 4    ? launch_part<T, VR_COMPOSITE, 4>(tmap, p, tf, grid, list, count, s)
                : group == 16 ? launch_part<T, VR_COMPOSITE, 16>(tmap, p, tf, grid, list, count, s)
                              : launch_part<T, VR_COMPOSITE, 8>(tmap, p, tf, grid, list, count, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

__global__ void k_pixel_setup(const __grid_constant__ PixelParams P) {
    const int n = P.width * P.height;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        Ray r;
        const bool hit = make_ray(P.cam, i % P.width, i / P.width, P.vol, ff{P.step_hi, P.step_lo}, r);
        P.krange[i] = make_int2(r.k0, r.k1);
        P.enc[i] = ord_enc(-INFINITY);
        if (hit && P.pixdir && P.cam.type == 1) {  // read only for pixels with samples
            P.pixdir[2 * (long long)i] = make_float4(r.e[0].hi, r.e[1].hi, r.e[2].hi, r.e[0].lo);
            P.pixdir[2 * (long long)i + 1] = make_float4(r.e[1].lo, r.e[2].lo, 0.f, 0.f);
        }
    }
}

__global__ void k_mip_finalize(const __grid_constant__ PixelParams P) {
    __shared__ float4 s_tf[kMaxTF];
    for (int i = threadIdx.x; i < P.tf.n; i += blockDim.x) s_tf[i] = P.tf.tab[i];
    __syncthreads();
    const int n = P.width * P.height;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float m = ord_dec(P.enc[i]);
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
        if (m > -INFINITY) o = tf_lookup(s_tf, P.tf.n, P.tf.vmin, P.tf.inv_range, m);
        P.out_rgba[i] = o;
        if (P.out_max) P.out_max[i] = m;
    }
}

template <typename T, bool ONE, int GROUP>
cudaError_t launch_brick(const void* tmap, const BrickParams& p, int grid, const CellDesc* list, const int* count,
                         cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_brick_mip<T, ONE, GROUP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TileGeom<T>::SMEM);
    if (e != cudaSuccess) return e;
    k_brick_mip<T, ONE, GROUP><<<grid, kBrickThreads, TileGeom<T>::SMEM, s>>>(
        *static_cast<const CUtensorMap*>(tmap), p, list, count);
    return cudaGetLastError();
}

template <typename T, int GROUP>
cudaError_t launch_brick_g(const void* tmap, const BrickParams& p, int grid, const CellDesc* list,
                           const int* count, cudaStream_t s) {
    return p.ncams == 1 ? launch_brick<T, true, GROUP>(tmap, p, grid, list, count, s)
                        : launch_brick<T, false, GROUP>(tmap, p, grid, list, count, s);
}

template <typename T>
cudaError_t launch_t(const void* tmap, const BrickParams& p, int grid, void* cells, cudaStream_t s, int group) {
    CellDesc* list = reinterpret_cast<CellDesc*>(static_cast<char*>(cells) + 256);
    int* count = static_cast<int*>(cells);
    const int nunits = (p.brick_list ? p.nlist : p.nbricks) * p.ncells_x * p.ncells_y * p.ncells_z;
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_cell_list<T><<<std::min((nunits + 255) / 256, 4096), 256, 0, s>>>(p, list, count);
    if (group == 4) return launch_brick_g<T, 4>(tmap, p, grid, list, count, s);
    if (group == 16) return launch_brick_g<T, 16>(tmap, p, grid, list, count, s);
    return launch_brick_g<T, 8>(tmap, p, grid, list, count, s);
}

}  // namespace

void brick_cell_dims(vr_dtype dt, int* cx, int* cy, int* cz) {
    if (dt == VR_F32) {
        *cx = Cell<float>::CX;
        *cy = Cell<float>::CY;
        *cz = Cell<float>::CZ;
    } else {
        *cx = Cell<__half>::CX;
        *cy = Cell<__half>::CY;
        *cz = Cell<__half>::CZ;
    }
}

void brick_box_dims(vr_dtype dt, int* bx, int* by, int* bz) {
    if (dt == VR_F32) {
        *bx = Cell<float>::BX;
        *by = Cell<float>::BY;
        *bz = Cell<float>::BZ;
    } else {
        *bx = Cell<__half>::BX;
        *by = Cell<__half>::BY;
        *bz = Cell<__half>::BZ;
    }
}

void brick_part_box_dims(vr_dtype dt, int* bx, int* by, int* bz) {
    if (dt == VR_F32) {
        *bx = Cell<float>::BX;
        *by = PartGeom<float>::BY;
        *bz = Cell<float>::BZ;
    } else {
        *bx = Cell<__half>::BX;
        *by = PartGeom<__half>::BY;
        *bz = Cell<__half>::BZ;
    }
}

int cell_partial_passes(vr_dtype dt, int brick) {
    int cx, cy, cz;
    brick_cell_dims(dt, &cx, &cy, &cz);
    return brick / cx + brick / cy + brick / cz - 2;  // local keys 0 .. sum of (cells per axis - 1)
}

cudaError_t launch_cell_partials(const void* tmap, const BrickParams& p, const TFDev& tf, vr_dtype dt, int mode,
                                 long long npartial, int npass, int grid, void* cells, cudaStream_t s, int group) {
    if (tf.n > kMaxPartTF || !p.partial || !p.foot || !p.work) return cudaErrorInvalidValue;
    if (dt == VR_F32) return cell_partials_t<float>(tmap, p, tf, mode, npartial, npass, grid, cells, s, group);
    if (dt == VR_F16) return cell_partials_t<__half>(tmap, p, tf, mode, npartial, npass, grid, cells, s, group);
    return cell_partials_t<__nv_bfloat16>(tmap, p, tf, mode, npartial, npass, grid, cells, s, group);
}

cudaError_t launch_pixel_setup(const PixelParams& p, cudaStream_t s) {
    const int n = p.width * p.height;
    const int grid = std::min((n + 255) / 256, 152 * 8);
    k_pixel_setup<<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_mip_finalize(const PixelParams& p, cudaStream_t s) {
    const int n = p.width * p.height;
    const int grid = std::min((n + 255) / 256, 152 * 8);
    k_mip_finalize<<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}

size_t brick_cells_bytes(long long nunits) { return 256 + (size_t)nunits * sizeof(CellDesc); }

cudaError_t launch_brick_mip(const void* tmap, const BrickParams& p, vr_dtype dt, int grid, void* cells,
                             cudaStream_t s, int group) {
    if (dt == VR_F32) return launch_t<float>(tmap, p, grid, cells, s, group);
    if (dt == VR_F16) return launch_t<__half>(tmap, p, grid, cells, s, group);
    return launch_t<__nv_bfloat16>(tmap, p, grid, cells, s, group);
}

}  // namespace vr

// Device building blocks of the ray caster: camera ray, box interval,
// brick-local trilinear fetch, transfer-function lookup.
#pragma once

#include "vr_ff.cuh"
#include "vr_internal.cuh"

namespace vr {

// Conversion of a stored voxel to FP32 (exact for all three storage types).
template <typename T> __device__ __forceinline__ float ld_voxel(const T* p);
template <> __device__ __forceinline__ float ld_voxel<float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ float ld_voxel<__half>(const __half* p) {
    return __half2float(__ldg(p));
}
template <> __device__ __forceinline__ float ld_voxel<__nv_bfloat16>(const __nv_bfloat16* p) {
    return __bfloat162float(__ldg(p));
}

// A camera ray in float-float: samples are o + k e, e = step * unit direction,
// for k in [k0, k1).  The sample range is the half-open slab interval of the
// box [0,nx]x[0,ny]x[0,nz] with t >= 0 (Sec. 3 renders the same orientation at
// any output size, so everything is per pixel centre).  The few operations
// here keep about 44 bits, so a sample up to 1e6 voxels from the origin lands
// within 1e-7 voxel of its exact position with no double-precision arithmetic.
struct Ray {
    ff o[3], e[3];
    int k0, k1;
};

// 2^-e for the binade [2^e, 2^(e+1)) holding m > 0 (2^127 for subnormal m).
__device__ __forceinline__ float pow2_recip(float m) {
    const int E = min((__float_as_int(m) >> 23) & 0xff, 253);
    return __int_as_float((254 - E) << 23);
}

// Slab parameter x / d; a quotient beyond 1e30 in magnitude (a direction all
// but parallel to the faces) is kept as +-1e30, which the axis with the
// largest direction component never reaches, so the interval is unchanged.
__device__ __forceinline__ ff slab_t(ff x, ff d) {
    const float q = __fdiv_rn(x.hi, d.hi);
    if (!(fabsf(q) < 1e30f)) return ff{copysignf(1e30f, q), 0.f};
    return ff_div(x, d);
}

// Ray of pixel (px, py) and its sample range [k0, k1); false when the ray has no
// sample in the box (then k0 = k1 = 0).
__device__ __forceinline__ bool make_ray(const CamFF& c, int px, int py, const VolDev& v, ff step, Ray& r) {
    const float sx = (float)px + 0.5f, sy = (float)py + 0.5f;
    const bool persp = c.type == 1;
    const ff nx[3] = {ff_of_int(v.nx), ff_of_int(v.ny), ff_of_int(v.nz)};  // exact box extents
    ff V[3];  // perspective: direction (unnormalised); orthographic: origin
#pragma unroll
    for (int a = 0; a < 3; ++a)
        V[a] = ff_add(ff_add(ff{c.base_hi[a], c.base_lo[a]}, ff_mul_f(ff{c.bx_hi[a], c.bx_lo[a]}, sx)),
                      ff_mul_f(ff{c.by_hi[a], c.by_lo[a]}, sy));
    r.k0 = r.k1 = 0;
    const float nf[3] = {(float)v.nx, (float)v.ny, (float)v.nz};
    {
        // FP32 slab test against the box grown by one voxel: a ray that misses the
        // grown box misses the box whatever the rounding, so it skips the rest.
        float lo32 = 0.f, hi32 = 3e38f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float o = persp ? c.org_hi[a] : V[a].hi, d = persp ? V[a].hi : c.dir_hi[a];
            if (d == 0.f) {
                if (o < -1.f || o > nf[a] + 1.f) return false;
            } else {
                const float t1 = (-1.f - o) / d, t2 = (nf[a] + 1.f - o) / d;
                lo32 = fmaxf(lo32, fminf(t1, t2));
                hi32 = fminf(hi32, fmaxf(t1, t2));
            }
        }
        if (!(lo32 <= hi32 * 1.0001f + 1e-3f)) return false;
    }
    ff dn[3];  // unit direction
    if (persp) {
        // V / |V|, V first scaled by a power of two (exactly) so that |V|^2 can
        // neither overflow nor underflow
        const float m = fmaxf(fmaxf(fabsf(V[0].hi), fabsf(V[1].hi)), fabsf(V[2].hi));
        if (!(m > 0.f)) return false;
        const float sc = pow2_recip(m);
        ff W[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) W[a] = ff{V[a].hi * sc, V[a].lo * sc};
        const ff rn = ff_rsqrt(ff_add(ff_add(ff_mul(W[0], W[0]), ff_mul(W[1], W[1])), ff_mul(W[2], W[2])));
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            r.o[a] = ff{c.org_hi[a], c.org_lo[a]};
            dn[a] = ff_mul(W[a], rn);
        }
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            r.o[a] = V[a];
            dn[a] = ff{c.dir_hi[a], c.dir_lo[a]};
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) r.e[a] = ff_mul(dn[a], step);
    {
        // The sample range from an FP32 slab test, kept only where rounding cannot
        // change it.  With o and d rounded once from their float-float values and
        // correctly rounded FP32 operations, each plane crossing t~ is within
        // |t| 3 u + |o| u / |d| (u = 2^-24) of the exact one; m_a doubles that.
        // t_near then lies in [tnL, tnU] = [max(0, lo_a - m_a), max(0, lo_a + m_a)]
        // and t_far in [tfL, tfU] = [min(hi_a - m_a), min(hi_a + m_a)]; an axis
        // nearly parallel to the faces (huge t, huge m) only widens these if it can
        // be the maximum or minimum.  The range is kept when the interval of
        // t_near / step (and of t_far / step) holds no integer but its ceiling,
        // else the float-float path decides.
        constexpr float u = 5.9604645e-8f;
        const float fstep = step.hi;
        float tnL = 0.f, tnU = 0.f, tfL = 3.0e38f, tfU = 3.0e38f;
        bool clear = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float o = r.o[a].hi, d = dn[a].hi;
            if (d == 0.f) {  // exactly parallel (hi == 0 means the pair is 0)
                if (o < 0.f || ff_lt(nx[a], r.o[a])) return false;
                continue;
            }
            const float t1 = (0.f - o) / d, t2 = (nf[a] - o) / d;
            const float lo_a = fminf(t1, t2), hi_a = fmaxf(t1, t2);
            const float m = (fmaxf(fabsf(t1), fabsf(t2)) * 6.f + fabsf(o) * 2.f / fabsf(d)) * u;
            if (!(fabsf(hi_a) + m <= 3.0e38f) || !(fabsf(lo_a) + m <= 3.0e38f)) {  // overflow: not screened
                clear = false;
                continue;
            }
            tnL = fmaxf(tnL, lo_a - m);
            tnU = fmaxf(tnU, lo_a + m);
            tfL = fminf(tfL, hi_a - m);
            tfU = fminf(tfU, hi_a + m);
        }
        if (clear && tfU < tnL) return false;  // misses the box whatever the rounding
        if (clear && tfL > tnU && tfU < 1e9f) {
            int k0 = 0, k1 = 0;
            bool ok0 = tnU == 0.f;  // every face plane behind the origin: t_near = 0
            if (!ok0 && tnL > 0.f) {
                const float qL = tnL / fstep * (1.f - 4.f * u), qU = tnU / fstep * (1.f + 4.f * u);
                k0 = (int)ceilf(qU);
                ok0 = qL > (float)(k0 - 1);
            }
            const float qL = tfL / fstep * (1.f - 4.f * u), qU = tfU / fstep * (1.f + 4.f * u);
            k1 = (int)ceilf(qU);
            if (ok0 && qL > (float)(k1 - 1)) {
                r.k0 = max(k0, 0);
                r.k1 = k1;
                return r.k1 > r.k0;
            }
        }
    }
    // float-float slab test: t = (plane - o) / d per axis, then ceil(t / step)
    ff lo = {0.f, 0.f}, hi = {1e30f, 0.f};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (dn[a].hi == 0.f) continue;  // inside its slab (checked above)
        const ff t1 = slab_t(ff_neg(r.o[a]), dn[a]);
        const ff t2 = slab_t(ff_add(nx[a], ff_neg(r.o[a])), dn[a]);
        const bool sw = ff_lt(t2, t1);
        const ff tl = sw ? t2 : t1, th = sw ? t1 : t2;
        if (ff_lt(lo, tl)) lo = tl;
        if (ff_lt(th, hi)) hi = th;
    }
    if (!ff_lt(lo, hi)) return false;
    const ff qa = ff_div(lo, step), qb = ff_div(hi, step);
    const long long kmax = 2000000000LL;
    r.k0 = (int)(qa.hi < 2e9f ? max(ff_ceil(qa), 0LL) : kmax);
    r.k1 = (int)(qb.hi < 2e9f ? min(ff_ceil(qb), kmax) : kmax);
    return r.k1 > r.k0;
}

// Brick-local segment state: stored coordinate g = p - brick origin + 1/2,
// so the lower trilinear corner is floor(g) in slot coordinates (0 = ghost).
struct Seg {
    float gx, gy, gz;
    int n;          // samples in this segment
    long long base; // element offset of the slot
    int brick;      // linear brick id
    float ox, oy, oz;  // brick origin (voxels)
};

// Start a segment at sample k: pick the brick holding p_k (any brick whose
// interior plus a half-voxel margin holds every sample of the segment gives
// the same values, thanks to the ghost layer), and count the samples that
// stay inside its interior (at least 1, at most cap).
__device__ __forceinline__ bool seg_begin(const Ray& r, int k, const VolDev& v, float3 e32,
                                          int cap, Seg& s) {
    const ff kk = ff_of_int(k);
    const int nb[3] = {v.nbx, v.nby, v.nbz};
    int b[3];
    float g[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const ff p = ff_add(r.o[a], ff_mul(r.e[a], kk));
        const int bi = min(max((int)ff_floor(p) >> v.log2B, 0), nb[a] - 1);
        b[a] = bi;
        // p.hi minus the brick origin is exact (both are multiples of ulp(p.hi)
        // and the difference is no larger than p.hi or one voxel)
        g[a] = __fadd_rn(__fsub_rn(p.hi, (float)(bi << v.log2B)), p.lo) + 0.5f;
    }
    const int bx = b[0], by = b[1], bz = b[2];
    s.gx = g[0];
    s.gy = g[1];
    s.gz = g[2];
    const float hiB = (float)v.B + 0.5f;
    float m = (float)cap;
    if (e32.x > 0.f) m = fminf(m, (hiB - s.gx) / e32.x); else if (e32.x < 0.f) m = fminf(m, (0.5f - s.gx) / e32.x);
    if (e32.y > 0.f) m = fminf(m, (hiB - s.gy) / e32.y); else if (e32.y < 0.f) m = fminf(m, (0.5f - s.gy) / e32.y);
    if (e32.z > 0.f) m = fminf(m, (hiB - s.gz) / e32.z); else if (e32.z < 0.f) m = fminf(m, (0.5f - s.gz) / e32.z);
    int n = (int)floorf(m) + 1;
    n = max(n, 1);
    n = min(n, min(cap, r.k1 - k));
    s.n = n;
    s.brick = (bz * v.nby + by) * v.nbx + bx;
    s.ox = (float)(bx << v.log2B);
    s.oy = (float)(by << v.log2B);
    s.oz = (float)(bz << v.log2B);
    const int slot = v.table[s.brick];
    s.base = (long long)slot * v.slot_elems;
    return slot >= 0;
}

// Trilinear sample at slot coordinate g (clamped to the slot for safety).
template <typename T>
__device__ __forceinline__ float fetch_trilinear(const T* __restrict__ slot, const VolDev& v,
                                                 float gx, float gy, float gz) {
    const float B = (float)v.B;
    gx = fminf(fmaxf(gx, 0.f), B + 0.999f);
    gy = fminf(fmaxf(gy, 0.f), B + 0.999f);
    gz = fminf(fmaxf(gz, 0.f), B + 0.999f);
    const float fx0 = floorf(gx), fy0 = floorf(gy), fz0 = floorf(gz);
    const float fx = gx - fx0, fy = gy - fy0, fz = gz - fz0;
    const int ix = (int)fx0, iy = (int)fy0, iz = (int)fz0;
    const int slab = v.rows * v.pitch;
    const T* p = slot + (iz * v.rows + iy) * v.pitch + ix;
    const float c000 = ld_voxel(p), c100 = ld_voxel(p + 1);
    const float c010 = ld_voxel(p + v.pitch), c110 = ld_voxel(p + v.pitch + 1);
    const float c001 = ld_voxel(p + slab), c101 = ld_voxel(p + slab + 1);
    const float c011 = ld_voxel(p + slab + v.pitch), c111 = ld_voxel(p + slab + v.pitch + 1);
    const float a0 = fmaf(fx, c100 - c000, c000), a1 = fmaf(fx, c110 - c010, c010);
    const float a2 = fmaf(fx, c101 - c001, c001), a3 = fmaf(fx, c111 - c011, c011);
    const float b0 = fmaf(fy, a1 - a0, a0), b1 = fmaf(fy, a3 - a2, a2);
    return fmaf(fz, b1 - b0, b0);
}

// Word w of a slot read as a pair of adjacent voxels (x, x + 1), widened to FP32.
template <typename T> __device__ __forceinline__ float2 ld_pair(const T* p, int w);
template <> __device__ __forceinline__ float2 ld_pair<__half>(const __half* p, int w) {
    return __half22float2(__ldg(reinterpret_cast<const __half2*>(p) + w));
}
template <> __device__ __forceinline__ float2 ld_pair<__nv_bfloat16>(const __nv_bfloat16* p, int w) {
    return __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(p) + w));
}

// fetch_trilinear with the four x-neighbour pairs read by one aligned load each:
// element i of the slot starts word i / 2 of the store when i is even and word
// i / 2 of the copy shifted by one element (slot1) when i is odd.  The row pitch
// is even, so the parity of i is that of x.  Same operations on the same values
// as fetch_trilinear, so the same result bit for bit.
template <typename T>
__device__ __forceinline__ float fetch_trilinear_pair(const T* __restrict__ slot, const T* __restrict__ slot1,
                                                      const VolDev& v, float gx, float gy, float gz) {
    const float B = (float)v.B;
    gx = fminf(fmaxf(gx, 0.f), B + 0.999f);
    gy = fminf(fmaxf(gy, 0.f), B + 0.999f);
    gz = fminf(fmaxf(gz, 0.f), B + 0.999f);
    const float fx0 = floorf(gx), fy0 = floorf(gy), fz0 = floorf(gz);
    const float fx = gx - fx0, fy = gy - fy0, fz = gz - fz0;
    const int ix = (int)fx0, iy = (int)fy0, iz = (int)fz0;
    const int w = ((iz * v.rows + iy) * v.pitch + ix) >> 1;
    const int hp = v.pitch >> 1, hs = (v.rows * v.pitch) >> 1;  // a row and a slab in words
    const T* p = (ix & 1) ? slot1 : slot;
    const float2 c00 = ld_pair<T>(p, w), c10 = ld_pair<T>(p, w + hp);
    const float2 c01 = ld_pair<T>(p, w + hs), c11 = ld_pair<T>(p, w + hs + hp);
    const float a0 = fmaf(fx, c00.y - c00.x, c00.x), a1 = fmaf(fx, c10.y - c10.x, c10.x);
    const float a2 = fmaf(fx, c01.y - c01.x, c01.x), a3 = fmaf(fx, c11.y - c11.x, c11.x);
    const float b0 = fmaf(fy, a1 - a0, a0), b1 = fmaf(fy, a3 - a2, a2);
    return fmaf(fz, b1 - b0, b0);
}

// Sub-anchor of a ray inside a segment: the sample k's slot coordinate g = G + q0
// split into an integer corner G (as the element offset `base` of voxel G in the
// slot) and a remainder q0 in [0, 1] rounded once from float-float.  The samples
// k + j that follow sit at G + q0 + j e, so for j < kAnchorSpan the FP32
// coordinate q = q0 + j e stays below 1 + kAnchorSpan |e| in magnitude: the
// position keeps about 2^-24 of that magnitude, not of the brick edge.
struct Anchor {
    float qx, qy, qz;     // remainder at the anchor sample
    float lox, loy, loz;  // clamp of q to the slot: [-G, B + 0.999 - G]
    float hix, hiy, hiz;
    int base;             // element offset of voxel G in the slot
};

constexpr int kAnchorSpan = 12;  // samples per sub-anchor

__device__ __forceinline__ Anchor anchor_at(const Ray& r, int k, const VolDev& v, const Seg& s) {
    const ff kk = ff_of_int(k);
    const float org[3] = {s.ox, s.oy, s.oz};
    float q[3], lo[3], hi[3];
    int G[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const ff p = ff_add(r.o[a], ff_mul(r.e[a], kk));
        // p.hi - origin + 1/2 is exact (multiples of ulp(p.hi), at most B + 2 apart)
        const float gh = __fadd_rn(__fsub_rn(p.hi, org[a]), 0.5f);
        const float g0 = floorf(gh);
        q[a] = __fadd_rn(__fsub_rn(gh, g0), p.lo);
        G[a] = (int)g0;
        lo[a] = -g0;
        hi[a] = __fadd_rn((float)v.B - g0, 0.999f);
    }
    Anchor A;
    A.qx = q[0];
    A.qy = q[1];
    A.qz = q[2];
    A.lox = lo[0];
    A.loy = lo[1];
    A.loz = lo[2];
    A.hix = hi[0];
    A.hiy = hi[1];
    A.hiz = hi[2];
    A.base = (G[2] * v.rows + G[1]) * v.pitch + G[0];
    return A;
}

// fetch_trilinear at slot coordinate G + q for the anchor's G: the same lerps on the
// same voxels, with the corner index split as base(G) + index(floor q).
template <typename T>
__device__ __forceinline__ float fetch_near(const T* __restrict__ slot, const VolDev& v, const Anchor& A,
                                            float qx, float qy, float qz) {
    qx = fminf(fmaxf(qx, A.lox), A.hix);
    qy = fminf(fmaxf(qy, A.loy), A.hiy);
    qz = fminf(fmaxf(qz, A.loz), A.hiz);
    const float fx0 = floorf(qx), fy0 = floorf(qy), fz0 = floorf(qz);
    const float fx = qx - fx0, fy = qy - fy0, fz = qz - fz0;
    const int slab = v.rows * v.pitch;
    const T* p = slot + A.base + ((int)fz0 * v.rows + (int)fy0) * v.pitch + (int)fx0;
    const float c000 = ld_voxel(p), c100 = ld_voxel(p + 1);
    const float c010 = ld_voxel(p + v.pitch), c110 = ld_voxel(p + v.pitch + 1);
    const float c001 = ld_voxel(p + slab), c101 = ld_voxel(p + slab + 1);
    const float c011 = ld_voxel(p + slab + v.pitch), c111 = ld_voxel(p + slab + v.pitch + 1);
    const float a0 = fmaf(fx, c100 - c000, c000), a1 = fmaf(fx, c110 - c010, c010);
    const float a2 = fmaf(fx, c101 - c001, c001), a3 = fmaf(fx, c111 - c011, c011);
    const float b0 = fmaf(fy, a1 - a0, a0), b1 = fmaf(fy, a3 - a2, a2);
    return fmaf(fz, b1 - b0, b0);
}

// fetch_trilinear_pair at slot coordinate G + q for the anchor's G (see fetch_near).
template <typename T>
__device__ __forceinline__ float fetch_near_pair(const T* __restrict__ slot, const T* __restrict__ slot1,
                                                 const VolDev& v, const Anchor& A, float qx, float qy, float qz) {
    qx = fminf(fmaxf(qx, A.lox), A.hix);
    qy = fminf(fmaxf(qy, A.loy), A.hiy);
    qz = fminf(fmaxf(qz, A.loz), A.hiz);
    const float fx0 = floorf(qx), fy0 = floorf(qy), fz0 = floorf(qz);
    const float fx = qx - fx0, fy = qy - fy0, fz = qz - fz0;
    const int i = A.base + ((int)fz0 * v.rows + (int)fy0) * v.pitch + (int)fx0;
    const int w = i >> 1;
    const int hp = v.pitch >> 1, hs = (v.rows * v.pitch) >> 1;  // a row and a slab in words
    const T* p = (i & 1) ? slot1 : slot;
    const float2 c00 = ld_pair<T>(p, w), c10 = ld_pair<T>(p, w + hp);
    const float2 c01 = ld_pair<T>(p, w + hs), c11 = ld_pair<T>(p, w + hs + hp);
    const float a0 = fmaf(fx, c00.y - c00.x, c00.x), a1 = fmaf(fx, c10.y - c10.x, c10.x);
    const float a2 = fmaf(fx, c01.y - c01.x, c01.x), a3 = fmaf(fx, c11.y - c11.x, c11.x);
    const float b0 = fmaf(fy, a1 - a0, a0), b1 = fmaf(fy, a3 - a2, a2);
    return fmaf(fz, b1 - b0, b0);
}

// True when every sample of brick b is certain to have opacity exactly 0: its
// stored maximum bounds every trilinear sample in it up to the FP32 rounding of
// the lerps (a sample can exceed it by a few ulps, which can carry it past one
// node boundary but not two), so the skip asks that the segment above the
// maximum's segment be transparent too: the maximum's lower node plus 2 is at
// most zero_top.  Values below the maximum, and NaN, map to lower nodes, and a
// lookup between two zero-alpha nodes returns 0, so such a segment leaves
// (C, T) unchanged and can be skipped.
__device__ __forceinline__ int tf_node(int n, float vmin, float inv_range, float val, float& x);
__device__ __forceinline__ bool brick_transparent(const VolDev& v, const TFDev& tf, int b) {
    if (!v.range_max || tf.zero_top < 1) return false;
    const unsigned int e = v.range_max[b];
    const float mx = __uint_as_float((e & 0x80000000u) ? (e & 0x7fffffffu) : ~e);
    float x;
    return tf_node(tf.n, tf.vmin, tf.inv_range, mx, x) + 2 <= tf.zero_top;
}

// Table position x of a value and its lower node i (node-centred, clamped):
// monotone in the value.  A NaN value maps to node 0 with weight 0.
__device__ __forceinline__ int tf_node(int n, float vmin, float inv_range, float val, float& x) {
    float u = (val - vmin) * inv_range;
    u = fminf(fmaxf(u, 0.f), 1.f);
    x = u * (float)(n - 1);
    return min((int)x, n - 2);
}

// Node-centred linear lookup of the table in shared memory, clamped.
__device__ __forceinline__ float4 tf_lookup(const float4* __restrict__ tab, int n, float vmin,
                                            float inv_range, float val) {
    float x;
    const int i = tf_node(n, vmin, inv_range, val, x);
    const float w = x - (float)i;
    const float4 a = tab[i], b = tab[i + 1];
    return make_float4(fmaf(w, b.x - a.x, a.x), fmaf(w, b.y - a.y, a.y),
                       fmaf(w, b.z - a.z, a.z), fmaf(w, b.w - a.w, a.w));
}

}  // namespace vr

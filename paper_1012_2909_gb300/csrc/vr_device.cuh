// Device building blocks of the ray caster: camera ray, box interval,
// brick-local trilinear fetch, transfer-function lookup.
#pragma once

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

// A camera ray in double precision: samples are o + k e, e = step * unit
// direction, for k in [k0, k1).  The sample range is the half-open slab
// interval of the box [0,nx]x[0,ny]x[0,nz] with t >= 0 (Sec. 3 renders the
// same orientation at any output size, so everything is per pixel centre).
struct Ray {
    double o[3], e[3];
    int k0, k1;
};

__device__ __forceinline__ bool make_ray(const CamDev& c, int px, int py, const VolDev& v,
                                         double step, Ray& r) {
    const double u = c.l + ((double)px + 0.5) * c.du;
    const double w = c.t - ((double)py + 0.5) * c.dv;
    double dd[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (c.type == 0) {
            r.o[a] = c.eye[a] + u * c.right[a] + w * c.up[a];
            dd[a] = c.fwd[a];
        } else {
            r.o[a] = c.eye[a];
            dd[a] = c.fwd[a] + u * c.right[a] + w * c.up[a];
        }
    }
    r.k0 = r.k1 = 0;
    {
        // FP32 slab test against the box grown by one voxel: a ray that misses the
        // grown box misses the box whatever the rounding, so it skips the FP64 work.
        float lo32 = 0.f, hi32 = 3e38f;
        const float nf[3] = {(float)v.nx, (float)v.ny, (float)v.nz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float o = (float)r.o[a], d = (float)dd[a];
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
    // Reciprocals instead of divisions (double-precision division is slow on this
    // part): t_near and t_far move by a few ulps, far inside the tolerance at which
    // a sample range is treated as ambiguous.
    const double inv_len = 1.0 / sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
    const double n[3] = {(double)v.nx, (double)v.ny, (double)v.nz};
    double dn[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        dn[a] = dd[a] * inv_len;
        r.e[a] = dn[a] * step;
    }
    {
        // The sample range from an FP32 slab test, kept only where rounding cannot
        // change it.  With o and d rounded once from double and correctly rounded
        // FP32 operations, each plane crossing t~ is within |t| 3 u + |o| u / |d|
        // (u = 2^-24) of the exact one; m_a doubles that.  t_near then lies in
        // [tnL, tnU] = [max(0, lo_a - m_a), max(0, lo_a + m_a)] and t_far in
        // [tfL, tfU] = [min(hi_a - m_a), min(hi_a + m_a)]; an axis nearly parallel
        // to the faces (huge t, huge m) only widens these if it can be the maximum
        // or minimum.  The range is kept when the interval of t_near / step (and of
        // t_far / step) holds no integer but its ceiling, else the double-precision
        // path decides.
        constexpr float u = 5.9604645e-8f;
        const float fstep = (float)step;
        float tnL = 0.f, tnU = 0.f, tfL = 3.0e38f, tfU = 3.0e38f;
        bool clear = true, miss = false;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (dn[a] == 0.0) {
                if (r.o[a] < 0.0 || r.o[a] > n[a]) miss = true;
                continue;
            }
            const float o = (float)r.o[a], d = (float)dn[a];
            if (d == 0.f) {
                clear = false;
                continue;
            }
            const float t1 = (0.f - o) / d, t2 = ((float)n[a] - o) / d;
            const float lo_a = fminf(t1, t2), hi_a = fmaxf(t1, t2);
            const float m = (fmaxf(fabsf(t1), fabsf(t2)) * 6.f + fabsf(o) * 2.f / fabsf(d)) * u;
            if (!(fabsf(hi_a) + m <= 3.0e38f) || !(fabsf(lo_a) + m <= 3.0e38f)) {  // overflow: leave it to FP64
                clear = false;
                continue;
            }
            tnL = fmaxf(tnL, lo_a - m);
            tnU = fmaxf(tnU, lo_a + m);
            tfL = fminf(tfL, hi_a - m);
            tfU = fminf(tfU, hi_a + m);
        }
        if (miss) return false;
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
    double lo = 0.0, hi = 1e300;
    bool hit = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double d = dn[a];
        if (d == 0.0) {
            if (r.o[a] < 0.0 || r.o[a] > n[a]) hit = false;
        } else {
            const double inv_d = 1.0 / d;
            const double t1 = (0.0 - r.o[a]) * inv_d, t2 = (n[a] - r.o[a]) * inv_d;
            lo = fmax(lo, fmin(t1, t2));
            hi = fmin(hi, fmax(t1, t2));
        }
    }
    if (!hit || !(lo < hi)) return false;
    const double a = ceil(lo / step), b = ceil(hi / step);
    r.k0 = (int)fmax(a, 0.0);
    r.k1 = (int)fmin(b, 2.0e9);
    return r.k1 > r.k0;
}

// Brick-local segment state: stored coordinate g = p - brick origin + 1/2,
// so the lower trilinear corner is floor(g) in slot coordinates (0 = ghost).
struct Seg {
    float gx, gy, gz;
    int n;          // samples in this segment
    long long base; // element offset of the slot
};

// Start a segment at sample k: pick the brick holding p_k (any brick whose
// interior plus a half-voxel margin holds every sample of the segment gives
// the same values, thanks to the ghost layer), and count the samples that
// stay inside its interior (at least 1, at most cap).
__device__ __forceinline__ bool seg_begin(const Ray& r, int k, const VolDev& v, float3 e32,
                                          int cap, Seg& s) {
    const double px = fma((double)k, r.e[0], r.o[0]);
    const double py = fma((double)k, r.e[1], r.o[1]);
    const double pz = fma((double)k, r.e[2], r.o[2]);
    int bx = ((int)floor(px)) >> v.log2B, by = ((int)floor(py)) >> v.log2B,
        bz = ((int)floor(pz)) >> v.log2B;
    bx = min(max(bx, 0), v.nbx - 1);
    by = min(max(by, 0), v.nby - 1);
    bz = min(max(bz, 0), v.nbz - 1);
    s.gx = (float)(px - (double)(bx << v.log2B)) + 0.5f;
    s.gy = (float)(py - (double)(by << v.log2B)) + 0.5f;
    s.gz = (float)(pz - (double)(bz << v.log2B)) + 0.5f;
    const float hiB = (float)v.B + 0.5f;
    float m = (float)cap;
    if (e32.x > 0.f) m = fminf(m, (hiB - s.gx) / e32.x); else if (e32.x < 0.f) m = fminf(m, (0.5f - s.gx) / e32.x);
    if (e32.y > 0.f) m = fminf(m, (hiB - s.gy) / e32.y); else if (e32.y < 0.f) m = fminf(m, (0.5f - s.gy) / e32.y);
    if (e32.z > 0.f) m = fminf(m, (hiB - s.gz) / e32.z); else if (e32.z < 0.f) m = fminf(m, (0.5f - s.gz) / e32.z);
    int n = (int)floorf(m) + 1;
    n = max(n, 1);
    n = min(n, min(cap, r.k1 - k));
    s.n = n;
    const int slot = v.table[(bz * v.nby + by) * v.nbx + bx];
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

// Node-centred linear lookup of the table in shared memory, clamped.
__device__ __forceinline__ float4 tf_lookup(const float4* __restrict__ tab, int n, float vmin,
                                            float inv_range, float val) {
    float u = (val - vmin) * inv_range;
    u = fminf(fmaxf(u, 0.f), 1.f);
    const float x = u * (float)(n - 1);
    const int i = min((int)x, n - 2);
    const float w = x - (float)i;
    const float4 a = tab[i], b = tab[i + 1];
    return make_float4(fmaf(w, b.x - a.x, a.x), fmaf(w, b.y - a.y, a.y),
                       fmaf(w, b.z - a.z, a.z), fmaf(w, b.w - a.w, a.w));
}

}  // namespace vr

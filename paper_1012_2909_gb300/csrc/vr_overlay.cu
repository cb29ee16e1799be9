// Catalogue overlay: a source finder's detections, given as bounding cubes,
// drawn as wireframe boxes over the volume render (Sec. 2), one colour per box
// (per catalogue in the paper's use).
//
// Pass 1, one thread per (camera, box, edge): the edge is projected through
// the camera's inverse mapping, clipped (near plane for perspective views, then
// the image rectangle grown by one pixel) and walked with n + 1 evenly spaced
// points, n = max(1, ceil(max(|dX|, |dY|))); every point marks its pixel with
// atomicMax(box index + 1), so a pixel of several boxes keeps the highest
// index whatever the thread order.  Pass 2 blends that box's straight colour
// over the premultiplied image.  Projection and walk are double precision
// with one rounding per operation in a fixed order (explicit intrinsics, no
// contraction), so the drawn pixels do not depend on the compiler.
#include <algorithm>

#include "vr_internal.cuh"

namespace vr {

namespace {

__device__ __forceinline__ double dm(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double da(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double ds(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dd(double a, double b) { return __ddiv_rn(a, b); }

// Inverse of M = [right | up | fwd] (columns) by adjugate / determinant.
__device__ void basis_inverse(const OverlayCam& c, double inv[9]) {
    const double m00 = c.right[0], m01 = c.up[0], m02 = c.fwd[0];
    const double m10 = c.right[1], m11 = c.up[1], m12 = c.fwd[1];
    const double m20 = c.right[2], m21 = c.up[2], m22 = c.fwd[2];
    const double c0 = ds(dm(m11, m22), dm(m12, m21));
    const double c1 = ds(dm(m12, m20), dm(m10, m22));
    const double c2 = ds(dm(m10, m21), dm(m11, m20));
    const double det = da(da(dm(m00, c0), dm(m01, c1)), dm(m02, c2));
    inv[0] = dd(c0, det);
    inv[1] = dd(ds(dm(m02, m21), dm(m01, m22)), det);
    inv[2] = dd(ds(dm(m01, m12), dm(m02, m11)), det);
    inv[3] = dd(c1, det);
    inv[4] = dd(ds(dm(m00, m22), dm(m02, m20)), det);
    inv[5] = dd(ds(dm(m02, m10), dm(m00, m12)), det);
    inv[6] = dd(c2, det);
    inv[7] = dd(ds(dm(m01, m20), dm(m00, m21)), det);
    inv[8] = dd(ds(dm(m00, m11), dm(m01, m10)), det);
}

__device__ __forceinline__ void cam_coords(const double inv[9], const double eye[3], const double p[3], double o[3]) {
    const double q0 = ds(p[0], eye[0]), q1 = ds(p[1], eye[1]), q2 = ds(p[2], eye[2]);
    o[0] = da(da(dm(inv[0], q0), dm(inv[1], q1)), dm(inv[2], q2));
    o[1] = da(da(dm(inv[3], q0), dm(inv[4], q1)), dm(inv[5], q2));
    o[2] = da(da(dm(inv[6], q0), dm(inv[7], q1)), dm(inv[8], q2));
}

// Liang-Barsky: clip s of x0 + s dx to lo <= x <= hi; false if empty.
__device__ __forceinline__ bool clip_axis(double x0, double dx, double lo, double hi, double& s0, double& s1) {
    if (dx == 0.0) return x0 >= lo && x0 <= hi;
    double a = dd(ds(lo, x0), dx), b = dd(ds(hi, x0), dx);
    if (a > b) {
        const double t = a;
        a = b;
        b = t;
    }
    if (a > s0) s0 = a;
    if (b < s1) s1 = b;
    return s0 <= s1;
}

__global__ void k_overlay_edges(const OverlayCam* __restrict__ cams, int ncams, const double* __restrict__ boxes,
                                long long nbox, int* __restrict__ key) {
    const long long total = (long long)ncams * nbox * 12;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total;
         it += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(it % 12);
        const long long bi = (it / 12) % nbox;
        const int ci = (int)(it / (12 * nbox));
        const OverlayCam& c = cams[ci];
        const int W = c.width, H = c.height;
        double inv[9];
        basis_inverse(c, inv);
        const double sx = dd((double)W, ds(c.r, c.l)), sy = dd((double)H, ds(c.t, c.b));
        const double* bx = boxes + 6 * bi;
        const int axis = e / 4, rest = e % 4;
        double p0[3], p1[3];
        int o = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (a == axis) {
                p0[a] = bx[a];
                p1[a] = bx[3 + a];
            } else {
                const int bit = (rest >> o) & 1;
                ++o;
                p0[a] = p1[a] = bit ? bx[3 + a] : bx[a];
            }
        }
        double c0[3], c1[3];
        cam_coords(inv, c.eye, p0, c0);
        cam_coords(inv, c.eye, p1, c1);
        double u0, v0, u1, v1;
        if (c.type == 1) {
            const double nearc = 1e-3;
            if (c0[2] < nearc && c1[2] < nearc) continue;
            if (c0[2] < nearc || c1[2] < nearc) {
                const double s = dd(ds(nearc, c0[2]), ds(c1[2], c0[2]));
                const double m0 = da(c0[0], dm(s, ds(c1[0], c0[0])));
                const double m1 = da(c0[1], dm(s, ds(c1[1], c0[1])));
                double* lo = c0[2] < nearc ? c0 : c1;
                lo[0] = m0;
                lo[1] = m1;
                lo[2] = nearc;
            }
            u0 = dd(c0[0], c0[2]);
            v0 = dd(c0[1], c0[2]);
            u1 = dd(c1[0], c1[2]);
            v1 = dd(c1[1], c1[2]);
        } else {
            u0 = c0[0];
            v0 = c0[1];
            u1 = c1[0];
            v1 = c1[1];
        }
        const double X0 = ds(dm(ds(u0, c.l), sx), 0.5), Y0 = ds(dm(ds(c.t, v0), sy), 0.5);
        const double X1 = ds(dm(ds(u1, c.l), sx), 0.5), Y1 = ds(dm(ds(c.t, v1), sy), 0.5);
        const double dX = ds(X1, X0), dY = ds(Y1, Y0);
        double s0 = 0.0, s1 = 1.0;
        if (!clip_axis(X0, dX, -1.0, (double)W, s0, s1)) continue;
        if (!clip_axis(Y0, dY, -1.0, (double)H, s0, s1)) continue;
        const double A0 = da(X0, dm(s0, dX)), B0 = da(Y0, dm(s0, dY));
        const double A1 = da(X0, dm(s1, dX)), B1 = da(Y0, dm(s1, dY));
        const double dA = ds(A1, A0), dB = ds(B1, B0);
        const double len = fabs(dA) > fabs(dB) ? fabs(dA) : fabs(dB);
        long long n = (long long)ceil(len);
        if (n < 1) n = 1;
        int* img_key = key + (long long)ci * W * H;
        const int k = (int)(bi + 1);
        for (long long i = 0; i <= n; ++i) {
            const double f = dd((double)i, (double)n);
            const long long px = (long long)floor(da(da(A0, dm(dA, f)), 0.5));
            const long long py = (long long)floor(da(da(B0, dm(dB, f)), 0.5));
            if (px < 0 || px >= W || py < 0 || py >= H) continue;
            atomicMax(img_key + py * W + px, k);
        }
    }
}

__global__ void k_overlay_blend(const int* __restrict__ key, long long npix, const float4* __restrict__ colours,
                                float4* __restrict__ rgba) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npix;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = key[i];
        if (!k) continue;
        const float4 c = colours[k - 1];
        float4 p = rgba[i];
        const float t = 1.f - c.w;
        p.x = fmaf(t, p.x, c.w * c.x);
        p.y = fmaf(t, p.y, c.w * c.y);
        p.z = fmaf(t, p.z, c.w * c.z);
        p.w = fmaf(t, p.w, c.w);
        rgba[i] = p;
    }
}

}  // namespace

cudaError_t launch_overlay(const OverlayCam* cams_dev, int ncams, const double* boxes, long long nbox,
                           const float* colours, int* key, float* rgba, int width, int height, cudaStream_t s) {
    const long long npix = (long long)ncams * width * height;
    cudaError_t e = cudaMemsetAsync(key, 0, sizeof(int) * (size_t)npix, s);
    if (e != cudaSuccess) return e;
    if (nbox > 0) {
        const long long total = (long long)ncams * nbox * 12;
        const int grid = (int)std::min<long long>((total + 127) / 128, 152 * 16);
        k_overlay_edges<<<grid, 128, 0, s>>>(cams_dev, ncams, boxes, nbox, key);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int grid2 = (int)std::min<long long>((npix + 255) / 256, 152 * 16);
    k_overlay_blend<<<grid2, 256, 0, s>>>(key, npix, reinterpret_cast<const float4*>(colours),
                                          reinterpret_cast<float4*>(rgba));
    return cudaGetLastError();
}

}  // namespace vr

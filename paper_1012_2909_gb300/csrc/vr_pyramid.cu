// Image pyramid of a render: the paper's high-resolution static renders are cut
// into tiles and shown at several zoom levels (Sec. 3); this is the render half
// of that path.  Level l+1 halves level l (rounding up) and its pixel is the
// mean of the in-level pixels of its 2 x 2 block (premultiplied RGBA).
//
// One CTA owns a 32 x 32 tile of its input level: it reads the tile once into
// shared memory and derives up to five levels from it there (tiles are aligned
// to 32 input pixels, so the children of every pixel of a level stay inside the
// CTA), writing every level once.  The host repeats the pass on the last level
// written until 1 x 1 is reached; each pass reads 1/1024 of the previous input.
#include <algorithm>

#include "vr_internal.cuh"

namespace vr {

namespace {

constexpr int kPyrTile = 32;
constexpr int kPyrPassLevels = 5;  // 32 -> 16 -> 8 -> 4 -> 2 -> 1
constexpr int kPyrThreads = 256;

struct PyrLevel {
    int w, h;
    long long off;  // float4 offset of the level in the output
};

struct PyrParams {
    const float4* in;
    int in_w, in_h, in_tlog2;  // input level; tile log2, -1 = row-major
    float4* out;
    int tlog2;                 // output layout, -1 = row-major
    int nlev;                  // levels written by this pass
    PyrLevel lev[kPyrPassLevels];
};

__device__ __forceinline__ long long pix_index(int x, int y, int w, int tlog2) {
    if (tlog2 < 0) return (long long)y * w + x;
    const int m = (1 << tlog2) - 1;
    const int tx = (w + m) >> tlog2;
    return (((long long)(y >> tlog2) * tx + (x >> tlog2)) << (2 * tlog2)) + ((y & m) << tlog2) + (x & m);
}

__global__ void __launch_bounds__(kPyrThreads) k_pyramid(const __grid_constant__ PyrParams P) {
    __shared__ float4 buf_a[kPyrTile * kPyrTile];
    __shared__ float4 buf_b[(kPyrTile / 2) * (kPyrTile / 2)];
    const int bx = blockIdx.x, by = blockIdx.y;
    // the input tile (pixels outside the level are never read back)
    for (int i = threadIdx.x; i < kPyrTile * kPyrTile; i += kPyrThreads) {
        const int x = bx * kPyrTile + (i % kPyrTile), y = by * kPyrTile + (i / kPyrTile);
        if (x < P.in_w && y < P.in_h) buf_a[i] = P.in[pix_index(x, y, P.in_w, P.in_tlog2)];
    }
    __syncthreads();
    int pw = P.in_w, ph = P.in_h, side = kPyrTile;
    float4* src = buf_a;
    float4* dst = buf_b;
    for (int k = 0; k < P.nlev; ++k) {
        const int half = side >> 1;
        const PyrLevel L = P.lev[k];
        for (int i = threadIdx.x; i < half * half; i += kPyrThreads) {
            const int x = i % half, y = i / half;
            const int gx = bx * half + x, gy = by * half + y;
            if (gx >= L.w || gy >= L.h) continue;
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            int n = 0;
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    if (2 * gx + q >= pw || 2 * gy + j >= ph) continue;
                    const float4 v = src[(2 * y + j) * side + 2 * x + q];
                    acc.x += v.x;
                    acc.y += v.y;
                    acc.z += v.z;
                    acc.w += v.w;
                    ++n;
                }
            const float inv = n == 4 ? 0.25f : (n == 2 ? 0.5f : 1.f);
            const float4 r = make_float4(acc.x * inv, acc.y * inv, acc.z * inv, acc.w * inv);
            dst[y * half + x] = r;
            P.out[L.off + pix_index(gx, gy, L.w, P.tlog2)] = r;
        }
        __syncthreads();
        float4* t = src;
        src = dst;
        dst = t;
        pw = L.w;
        ph = L.h;
        side = half;
    }
}

}  // namespace

// Level sizes and float4 offsets of levels 1.. for the layout (tlog2 < 0:
// row-major); returns the total float4 count.
long long pyramid_levels(int w, int h, int tlog2, std::vector<int>& ws, std::vector<int>& hs,
                         std::vector<long long>& offs) {
    ws.clear();
    hs.clear();
    offs.clear();
    long long total = 0;
    while (w > 1 || h > 1) {
        w = (w + 1) / 2;
        h = (h + 1) / 2;
        ws.push_back(w);
        hs.push_back(h);
        offs.push_back(total);
        if (tlog2 < 0) {
            total += (long long)w * h;
        } else {
            const long long t = 1LL << tlog2;
            total += ((w + t - 1) / t) * ((h + t - 1) / t) * t * t;
        }
    }
    return total;
}

cudaError_t launch_pyramid(const float4* in, int w, int h, int tlog2, float4* out, cudaStream_t s) {
    std::vector<int> ws, hs;
    std::vector<long long> offs;
    const long long total = pyramid_levels(w, h, tlog2, ws, hs, offs);
    if (ws.empty()) return cudaSuccess;
    if (tlog2 >= 0) {  // padding of edge tiles
        cudaError_t e = cudaMemsetAsync(out, 0, (size_t)total * sizeof(float4), s);
        if (e != cudaSuccess) return e;
    }
    PyrParams P;
    P.in = in;
    P.in_w = w;
    P.in_h = h;
    P.in_tlog2 = -1;
    P.out = out;
    P.tlog2 = tlog2;
    size_t done = 0;
    while (done < ws.size()) {
        P.nlev = (int)std::min<size_t>(kPyrPassLevels, ws.size() - done);
        for (int k = 0; k < P.nlev; ++k) P.lev[k] = PyrLevel{ws[done + k], hs[done + k], offs[done + k]};
        const dim3 grid((unsigned)((P.in_w + kPyrTile - 1) / kPyrTile), (unsigned)((P.in_h + kPyrTile - 1) / kPyrTile));
        k_pyramid<<<grid, kPyrThreads, 0, s>>>(P);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        done += (size_t)P.nlev;
        const size_t last = done - 1;
        P.in = out + offs[last];
        P.in_w = ws[last];
        P.in_h = hs[last];
        P.in_tlog2 = tlog2;
    }
    return cudaSuccess;
}

}  // namespace vr

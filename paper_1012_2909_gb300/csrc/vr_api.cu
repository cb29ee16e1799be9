// C ABI of the renderer (include/vr.h): context, validation, cube loading,
// transfer function, cameras and render dispatch.  No exception crosses the
// boundary; every failure becomes a vr_status with a message on the context.
#include <algorithm>
#include <climits>
#include <chrono>
#include <thread>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "vr_internal.cuh"
#include "vr_tma.cuh"

using namespace vr;

struct vr_ctx {
    int device = 0;
    vr_options opt{};
    std::string err;
    int num_sms = 0;
    // cube
    bool has_cube = false;
    vr_dtype dtype = VR_F32;
    long long nx = 0, ny = 0, nz = 0;
    int nbx = 0, nby = 0, nbz = 0, B = 0, log2B = 0, rows = 0, pitch = 0;
    long long slot_elems = 0;
    size_t elem = 4;
    void* pool = nullptr;
    void* pool1 = nullptr;         // the store shifted by one element, when kept
    int* table = nullptr;
    unsigned int* minmax = nullptr;
    void* cells = nullptr;   // brick-pass cell list of the current view
    long long pool_slots = 0; // slots of the brick store (all bricks in core, the cache out of core)
    // out-of-core streaming
    bool ooc = false;
    vr_region_fn ooc_fn = nullptr;
    void* ooc_user = nullptr;
    std::vector<int> slot_brick, table_host;
    std::vector<long long> slot_use;
    long long ooc_tick = 0;
    float* ooc_pin[2] = {nullptr, nullptr};
    float* ooc_dev[2] = {nullptr, nullptr};
    int* ooc_pin_table = nullptr;
    int* ooc_pin_list = nullptr;
    int* ooc_dev_list = nullptr;
    cudaEvent_t ooc_ev[2] = {nullptr, nullptr};
    cudaEvent_t ooc_ev_table = nullptr, ooc_ev_render = nullptr;
    cudaStream_t ooc_side = nullptr;
    int ooc_next_buf = 0;
    double ooc_timeout_s = 120.0;
    vr_stream_stats ooc_stats{};
    // transfer function
    bool has_tf = false;
    std::vector<float4> tf;
    float vmin = 0.f, vmax = 1.f;
    // cameras
    std::vector<CamDev> cams;
    // brick pass: TMA descriptor of the brick store
    CUtensorMap tmap;
    bool has_tmap = false;
    // the sort-last partial pass: the same store with the box of brick_part_box_dims
    CUtensorMap tmap_part;
    bool has_tmap_part = false;
    vr_path path = VR_PATH_AUTO;
    vr_tuning tune{8, 4, 256, 8};  // tile_w, tile_h, block, group
    bool graph_mode = false;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    // scratch
    int* work = nullptr;
    int work_slots = 0;
    int2* krange = nullptr;        // per-pixel sample range of the brick pass
    float4* pixdir = nullptr;      // per-pixel float-float step vector (2 x float4)
    // catalogue overlay scratch (grown on demand)
    int* ov_key = nullptr;
    long long ov_key_n = 0;
    void* ov_in = nullptr;         // cameras, boxes and colours, copied from the host
    size_t ov_in_bytes = 0;
    unsigned int* enc = nullptr;   // per-pixel running maximum when out_max is NULL
    long long scratch_pix = 0;
    // sort-last / layered scratch
    BrickFoot* foot = nullptr;
    int* order = nullptr;
    int* tile_start = nullptr;
    long long sort_bricks = 0;
    int* layer_buf = nullptr;      // count | start | fill
    int layer_cap = 0;
    unsigned long long* partial_used = nullptr;
    float4* partial = nullptr;
    long long partial_cap = 0;
    float4* state = nullptr;
    long long state_cap = 0;
    int* host_rb = nullptr;        // page-locked read-back buffer
    int host_rb_cap = 0;
    float* tf_partials = nullptr;  // adjoint: per-block table-gradient partials
    size_t tf_partials_n = 0;
    int* status_host = nullptr;    // mapped, page-locked device status word
    int* status_dev = nullptr;
    // distributed sort-last (vr_sortlast_partials / vr_sortlast_fold)
    int* dist_ids = nullptr;       // brick subset | tile prefix | fold order | count
    long long dist_cap = 0;        // bricks the buffer holds
    BrickFoot* dist_foot = nullptr;
    unsigned long long* sample_counter = nullptr;  // caller-owned
    cudaEvent_t ev_start = nullptr, ev_stop = nullptr;  // caller-owned profiling events
};

namespace {

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int d) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != d) cudaSetDevice(d);
    }
    ~DevGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

vr_status fail(vr_ctx* c, vr_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

vr_status cuda_fail(vr_ctx* c, cudaError_t e, const char* what) {
    cudaGetLastError();  // clear a sticky non-fatal error state
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(c, e == cudaErrorMemoryAllocation ? VR_ERR_OOM : VR_ERR_CUDA, m);
}

#define VR_CK(call, what)                                   \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

void free_ooc(vr_ctx* c) {
    if (c->ooc_side) cudaStreamSynchronize(c->ooc_side);
    for (int i = 0; i < 2; ++i) {
        if (c->ooc_pin[i]) cudaFreeHost(c->ooc_pin[i]);
        if (c->ooc_dev[i]) cudaFree(c->ooc_dev[i]);
        if (c->ooc_ev[i]) cudaEventDestroy(c->ooc_ev[i]);
        c->ooc_pin[i] = nullptr;
        c->ooc_dev[i] = nullptr;
        c->ooc_ev[i] = nullptr;
    }
    if (c->ooc_pin_table) cudaFreeHost(c->ooc_pin_table);
    if (c->ooc_pin_list) cudaFreeHost(c->ooc_pin_list);
    if (c->ooc_dev_list) cudaFree(c->ooc_dev_list);
    if (c->ooc_ev_table) cudaEventDestroy(c->ooc_ev_table);
    if (c->ooc_ev_render) cudaEventDestroy(c->ooc_ev_render);
    if (c->ooc_side) cudaStreamDestroy(c->ooc_side);
    c->ooc_pin_table = nullptr;
    c->ooc_pin_list = nullptr;
    c->ooc_dev_list = nullptr;
    c->ooc_ev_table = c->ooc_ev_render = nullptr;
    c->ooc_side = nullptr;
    c->slot_brick.clear();
    c->table_host.clear();
    c->slot_use.clear();
    c->ooc = false;
}

void free_cube(vr_ctx* c) {
    free_ooc(c);
    if (c->pool) cudaFree(c->pool);
    if (c->pool1) cudaFree(c->pool1);
    if (c->table) cudaFree(c->table);
    if (c->minmax) cudaFree(c->minmax);
    if (c->cells) cudaFree(c->cells);
    c->pool = nullptr;
    c->pool1 = nullptr;
    c->table = nullptr;
    c->minmax = nullptr;
    c->cells = nullptr;
    c->has_cube = false;
}

VolDev vol_dev(const vr_ctx* c) {
    VolDev v{};
    v.pool = c->pool;
    v.pool1 = c->pool1;
    v.table = c->table;
    v.nx = (int)c->nx;
    v.ny = (int)c->ny;
    v.nz = (int)c->nz;
    v.nbx = c->nbx;
    v.nby = c->nby;
    v.nbz = c->nbz;
    v.B = c->B;
    v.log2B = c->log2B;
    v.pitch = c->pitch;
    v.rows = c->rows;
    v.slot_elems = c->slot_elems;
    // brick value ranges exist for in-core cubes (the streamed cache has none)
    v.range_max = (c->minmax && !c->ooc) ? c->minmax + (long long)c->nbx * c->nby * c->nbz : nullptr;
    return v;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// TMA descriptor of the brick store viewed as a 4-D tensor (x, y, z, slot), with
// the box of one staged cell.  Only bricks of at least 32 voxels have cells.
bool make_tensor_map(vr_ctx* c) {
    c->has_tmap = false;
    int cx, cy, cz, bx, by, bz;
    brick_cell_dims(c->dtype, &cx, &cy, &cz);
    brick_box_dims(c->dtype, &bx, &by, &bz);
    if (c->B < cx || c->B < cy || c->B < cz || bx > c->pitch) return false;
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t e = c->elem;
    cuuint64_t dims[4] = {(cuuint64_t)c->pitch, (cuuint64_t)c->rows, (cuuint64_t)c->rows,
                          (cuuint64_t)c->pool_slots};
    cuuint64_t strides[3] = {c->pitch * e, (cuuint64_t)c->rows * c->pitch * e, (cuuint64_t)c->slot_elems * e};
    cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUtensorMapDataType dt = c->dtype == VR_F32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                             : c->dtype == VR_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                  : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUresult r = enc(&c->tmap, dt, 4, c->pool, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    c->has_tmap = (r == CUDA_SUCCESS);
    c->has_tmap_part = false;
    if (c->has_tmap) {
        brick_part_box_dims(c->dtype, &bx, &by, &bz);
        cuuint32_t pbox[4] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz, 1};
        // no L2 promotion: a visibility pass stages cells whose x-neighbours belong to
        // other passes, so the rest of a promoted 256-byte line is evicted before
        // its use (survey frame: 16.4 GB of DRAM reads with promotion, 14.7 GB
        // without; the store is 4.7 GB)
        r = enc(&c->tmap_part, dt, 4, c->pool, dims, strides, pbox, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        c->has_tmap_part = (r == CUDA_SUCCESS);
    }
    return c->has_tmap;
}

void split(double x, float& hi, float& lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

// Float-float camera constants (see CamFF) from a double-precision camera; false
// (minv left 0, everything else filled) if the basis is singular.
bool cam_ff(const CamDev& d, CamFF& f) {
    std::memset(&f, 0, sizeof(f));
    const double* R = d.right;
    const double* U = d.up;
    const double* F = d.fwd;
    double fl = std::sqrt(F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
    for (int a = 0; a < 3; ++a) {
        double base = (d.type == 1 ? F[a] : d.eye[a]) + d.l * R[a] + d.t * U[a];
        split(base, f.base_hi[a], f.base_lo[a]);
        split(d.du * R[a], f.bx_hi[a], f.bx_lo[a]);
        split(-d.dv * U[a], f.by_hi[a], f.by_lo[a]);
        split(d.eye[a], f.org_hi[a], f.org_lo[a]);
        split(F[a] / fl, f.dir_hi[a], f.dir_lo[a]);
        f.eye[a] = (float)d.eye[a];
    }
    f.l = (float)d.l;
    f.t = (float)d.t;
    f.du = (float)d.du;
    f.dv = (float)d.dv;
    f.type = d.type;
    f.width = d.width;
    f.height = d.height;
    // inverse of the column matrix M = [R U F]
    const double m[9] = {R[0], U[0], F[0], R[1], U[1], F[1], R[2], U[2], F[2]};
    const double det = m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) +
                       m[2] * (m[3] * m[7] - m[4] * m[6]);
    const double scale = std::sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]) *
                         std::sqrt(U[0] * U[0] + U[1] * U[1] + U[2] * U[2]) * fl;
    if (!(std::fabs(det) > 1e-12 * scale)) return false;
    const double inv[9] = {(m[4] * m[8] - m[5] * m[7]) / det, (m[2] * m[7] - m[1] * m[8]) / det,
                           (m[1] * m[5] - m[2] * m[4]) / det, (m[5] * m[6] - m[3] * m[8]) / det,
                           (m[0] * m[8] - m[2] * m[6]) / det, (m[2] * m[3] - m[0] * m[5]) / det,
                           (m[3] * m[7] - m[4] * m[6]) / det, (m[1] * m[6] - m[0] * m[7]) / det,
                           (m[0] * m[4] - m[1] * m[3]) / det};
    for (int i = 0; i < 9; ++i) f.minv[i] = (float)inv[i];
    return true;
}

// The ray constants of a camera for the paths that project nothing (image-order
// marcher, pixel set-up, adjoint): a singular basis is fine there, minv stays 0.
CamFF ray_cam(const CamDev& d) {
    CamFF f;
    cam_ff(d, f);
    return f;
}

bool beyond(const double* v, int n, double lim) {
    for (int i = 0; i < n; ++i)
        if (std::fabs(v[i]) > lim) return true;
    return false;
}

bool finite3(const double* v) {
    return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]);
}

}  // namespace

extern "C" {

void vr_default_options(vr_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->brick = 128;
    opt->step = 0.5;
    opt->ert = 0.99;
}

const char* vr_status_string(vr_status s) {
    switch (s) {
        case VR_OK: return "VR_OK";
        case VR_ERR_INVALID_ARG: return "VR_ERR_INVALID_ARG";
        case VR_ERR_STATE: return "VR_ERR_STATE";
        case VR_ERR_OOM: return "VR_ERR_OOM";
        case VR_ERR_CUDA: return "VR_ERR_CUDA";
        case VR_ERR_TIMEOUT: return "VR_ERR_TIMEOUT";
        case VR_ERR_IO: return "VR_ERR_IO";
        case VR_ERR_INTERNAL: return "VR_ERR_INTERNAL";
        case VR_ERR_UNSUPPORTED: return "VR_ERR_UNSUPPORTED";
    }
    return "VR_ERR_UNKNOWN";
}

vr_status vr_create(vr_ctx** out, int device, const vr_options* opt) {
    if (!out) return VR_ERR_INVALID_ARG;
    *out = nullptr;
    vr_options o;
    vr_default_options(&o);
    if (opt) o = *opt;
    if (o.brick < 8 || o.brick > 256 || (o.brick & (o.brick - 1)) || !(o.step > 0.0) ||
        !std::isfinite(o.step) || !(o.ert > 0.0) || !std::isfinite(o.ert) || (o.flags & ~VR_OPT_SINGLE_STORE))
        return VR_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return VR_ERR_CUDA;
    }
    if (device < 0 || device >= ndev) return VR_ERR_INVALID_ARG;
    vr_ctx* ctx = new (std::nothrow) vr_ctx();
    if (!ctx) return VR_ERR_OOM;
    ctx->device = device;
    ctx->opt = o;
    DevGuard g(device);
    cudaError_t e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) {
        ctx->work_slots = 4096 / kMaxLaunchCams + 4096 + 1;
        e = cudaMalloc(&ctx->work, sizeof(int) * ctx->work_slots);
    }
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&ctx->status_host), sizeof(int), cudaHostAllocMapped);
    if (e == cudaSuccess) {
        *ctx->status_host = 0;
        e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&ctx->status_dev), ctx->status_host, 0);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (ctx->work) cudaFree(ctx->work);
        if (ctx->status_host) cudaFreeHost(ctx->status_host);
        delete ctx;
        return e == cudaErrorMemoryAllocation ? VR_ERR_OOM : VR_ERR_CUDA;
    }
    *out = ctx;
    return VR_OK;
}

vr_status vr_destroy(vr_ctx* ctx) {
    if (!ctx) return VR_OK;
    {
        DevGuard g(ctx->device);
        free_cube(ctx);
        if (ctx->work) cudaFree(ctx->work);
        if (ctx->krange) cudaFree(ctx->krange);
        if (ctx->pixdir) cudaFree(ctx->pixdir);
        if (ctx->ov_key) cudaFree(ctx->ov_key);
        if (ctx->ov_in) cudaFree(ctx->ov_in);
        if (ctx->enc) cudaFree(ctx->enc);
        if (ctx->tf_partials) cudaFree(ctx->tf_partials);
        for (void* p : {(void*)ctx->foot, (void*)ctx->order, (void*)ctx->tile_start, (void*)ctx->layer_buf,
                        (void*)ctx->partial_used, (void*)ctx->partial, (void*)ctx->state,
                        (void*)ctx->dist_ids, (void*)ctx->dist_foot})
            if (p) cudaFree(p);
        if (ctx->host_rb) cudaFreeHost(ctx->host_rb);
        if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
        if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
        if (ctx->status_host) cudaFreeHost(ctx->status_host);
    }
    delete ctx;
    return VR_OK;
}

vr_status vr_load_cube(vr_ctx* ctx, const float* src, int src_on_device, int64_t nx,
                       int64_t ny, int64_t nz, vr_dtype storage, void* stream) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    if (!src) return fail(ctx, VR_ERR_INVALID_ARG, "vr_load_cube: src is NULL");
    if (nx <= 0 || ny <= 0 || nz <= 0 || nx >= (1LL << 30) || ny >= (1LL << 30) || nz >= (1LL << 30))
        return fail(ctx, VR_ERR_INVALID_ARG, "vr_load_cube: dimensions must be in [1, 2^30)");
    if (storage != VR_F32 && storage != VR_F16 && storage != VR_BF16)
        return fail(ctx, VR_ERR_INVALID_ARG, "vr_load_cube: unknown storage type");
    DevGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    VR_CK(cudaGetLastError(), "vr_load_cube: pending CUDA error");
    free_cube(ctx);
    const int B = ctx->opt.brick;
    ctx->B = B;
    ctx->log2B = ilog2(B);
    ctx->nx = nx;
    ctx->ny = ny;
    ctx->nz = nz;
    ctx->nbx = (int)((nx + B - 1) / B);
    ctx->nby = (int)((ny + B - 1) / B);
    ctx->nbz = (int)((nz + B - 1) / B);
    ctx->dtype = storage;
    ctx->elem = storage == VR_F32 ? 4 : 2;
    ctx->rows = B + 2;
    const int vec = (int)(16 / ctx->elem);
    ctx->pitch = (ctx->rows + vec - 1) / vec * vec;
    long long se = (long long)ctx->rows * ctx->rows * ctx->pitch;
    const long long align = 256 / (long long)ctx->elem;
    ctx->slot_elems = (se + align - 1) / align * align;
    const long long nbricks = (long long)ctx->nbx * ctx->nby * ctx->nbz;
    if (nbricks > (1LL << 30)) return fail(ctx, VR_ERR_INVALID_ARG, "vr_load_cube: too many bricks");
    const size_t pool_bytes = (size_t)nbricks * (size_t)ctx->slot_elems * ctx->elem;
    ctx->pool_slots = nbricks;
    VR_CK(cudaMalloc(&ctx->pool, pool_bytes), "vr_load_cube: brick store allocation");
    VR_CK(cudaMalloc(&ctx->table, sizeof(int) * nbricks), "vr_load_cube: brick table allocation");
    VR_CK(cudaMalloc(&ctx->minmax, sizeof(unsigned int) * 2 * nbricks), "vr_load_cube: range allocation");
    {
        std::vector<int> ident((size_t)nbricks);
        for (long long i = 0; i < nbricks; ++i) ident[(size_t)i] = (int)i;
        VR_CK(cudaMemcpyAsync(ctx->table, ident.data(), sizeof(int) * nbricks, cudaMemcpyHostToDevice, s),
              "vr_load_cube: brick table upload");
        VR_CK(cudaStreamSynchronize(s), "vr_load_cube: brick table upload");
    }
    VR_CK(cudaMemsetAsync(ctx->minmax, 0xff, sizeof(unsigned int) * nbricks, s), "vr_load_cube: memset");
    VR_CK(cudaMemsetAsync(ctx->minmax + nbricks, 0, sizeof(unsigned int) * nbricks, s), "vr_load_cube: memset");
    VolDev v = vol_dev(ctx);
    if (src_on_device) {
        for (int bz = 0; bz < ctx->nbz; ++bz)
            VR_CK(launch_repack(src, 0, nz, bz, v, storage, ctx->pool, ctx->minmax, s), "vr_load_cube: repack");
    } else {
        const size_t plane = (size_t)nx * (size_t)ny;
        const long long maxp = std::min<long long>(ctx->rows, nz);
        float* stage = nullptr;
        VR_CK(cudaMallocAsync(reinterpret_cast<void**>(&stage), plane * maxp * sizeof(float), s),
              "vr_load_cube: staging allocation");
        for (int bz = 0; bz < ctx->nbz; ++bz) {
            const long long z0 = std::max<long long>((long long)bz * B - 1, 0);
            const long long z1 = std::min<long long>((long long)bz * B + B + 1, nz);
            cudaError_t e = cudaMemcpyAsync(stage, src + (size_t)z0 * plane, plane * (z1 - z0) * sizeof(float),
                                            cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = launch_repack(stage, z0, z1 - z0, bz, v, storage, ctx->pool, ctx->minmax, s);
            if (e != cudaSuccess) {
                cudaFreeAsync(stage, s);
                cudaStreamSynchronize(s);
                free_cube(ctx);
                return cuda_fail(ctx, e, "vr_load_cube: slab upload/repack");
            }
        }
        VR_CK(cudaFreeAsync(stage, s), "vr_load_cube: staging free");
    }
    VR_CK(cudaStreamSynchronize(s), "vr_load_cube: repack");
    if (storage != VR_F32 && !(ctx->opt.flags & VR_OPT_SINGLE_STORE)) {
        // the copy shifted by one element (16-bit stores: an x-pair is one 32-bit load;
        // FP32 pairs as 64-bit loads measured no faster), kept only when it fits in half
        // of what is free
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && pool_bytes <= fr / 2) {
            if (cudaMalloc(&ctx->pool1, pool_bytes) == cudaSuccess) {
                const size_t e = (size_t)ctx->elem;
                VR_CK(cudaMemcpyAsync(ctx->pool1, static_cast<char*>(ctx->pool) + e, pool_bytes - e,
                                      cudaMemcpyDeviceToDevice, s), "vr_load_cube: shifted copy");
                VR_CK(cudaMemsetAsync(static_cast<char*>(ctx->pool1) + pool_bytes - e, 0, e, s),
                      "vr_load_cube: shifted copy");
                VR_CK(cudaStreamSynchronize(s), "vr_load_cube: shifted copy");
            } else {
                cudaGetLastError();  // not kept: the single-store path serves every render
                ctx->pool1 = nullptr;
            }
        }
    }
    if (make_tensor_map(ctx)) {
        int cx, cy, cz;
        brick_cell_dims(ctx->dtype, &cx, &cy, &cz);
        const long long units = nbricks * (long long)(B / cx) * (B / cy) * (B / cz);
        VR_CK(cudaMalloc(&ctx->cells, brick_cells_bytes(units)), "vr_load_cube: cell list allocation");
    }
    ctx->has_cube = true;
    return VR_OK;
}

vr_status vr_load_cube_streamed(vr_ctx* ctx, vr_region_fn fn, void* user, int64_t nx, int64_t ny, int64_t nz,
                                vr_dtype storage, uint64_t cache_bytes) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    if (!fn) return fail(ctx, VR_ERR_INVALID_ARG, "vr_load_cube_streamed: fn is NULL");
    if (nx <= 0 || ny <= 0 || nz <= 0 || nx >= (1LL << 30) || ny >= (1LL << 30) || nz >= (1LL << 30))
        return fail(ctx, VR_ERR_INVALID_ARG, "vr_load_cube_streamed: dimensions must be in [1, 2^30)");
    if (storage != VR_F32 && storage != VR_F16 && storage != VR_BF16)
        return fail(ctx, VR_ERR_INVALID_ARG, "vr_load_cube_streamed: unknown storage type");
    DevGuard g(ctx->device);
    VR_CK(cudaGetLastError(), "vr_load_cube_streamed: pending CUDA error");
    VR_CK(cudaDeviceSynchronize(), "vr_load_cube_streamed: drain");
    free_cube(ctx);
    const int B = ctx->opt.brick;
    ctx->B = B;
    ctx->log2B = ilog2(B);
    ctx->nx = nx;
    ctx->ny = ny;
    ctx->nz = nz;
    ctx->nbx = (int)((nx + B - 1) / B);
    ctx->nby = (int)((ny + B - 1) / B);
    ctx->nbz = (int)((nz + B - 1) / B);
    ctx->dtype = storage;
    ctx->elem = storage == VR_F32 ? 4 : 2;
    ctx->rows = B + 2;
    const int vec = (int)(16 / ctx->elem);
    ctx->pitch = (ctx->rows + vec - 1) / vec * vec;
    const long long se = (long long)ctx->rows * ctx->rows * ctx->pitch;
    const long long align = 256 / (long long)ctx->elem;
    ctx->slot_elems = (se + align - 1) / align * align;
    const long long nbricks = (long long)ctx->nbx * ctx->nby * ctx->nbz;
    if (nbricks > (1LL << 30)) return fail(ctx, VR_ERR_INVALID_ARG, "vr_load_cube_streamed: too many bricks");
    const long long slot_bytes = ctx->slot_elems * (long long)ctx->elem;
    const long long nslots = std::min<long long>(nbricks, (long long)(cache_bytes / (uint64_t)slot_bytes));
    if (nslots < 1) return fail(ctx, VR_ERR_INVALID_ARG, "vr_load_cube_streamed: cache smaller than one brick");
    ctx->pool_slots = nslots;
    VR_CK(cudaMalloc(&ctx->pool, (size_t)nslots * (size_t)slot_bytes), "vr_load_cube_streamed: brick cache");
    VR_CK(cudaMalloc(&ctx->table, sizeof(int) * (size_t)nbricks), "vr_load_cube_streamed: brick table");
    VR_CK(cudaMemset(ctx->table, 0xff, sizeof(int) * (size_t)nbricks), "vr_load_cube_streamed: brick table");
    ctx->slot_brick.assign((size_t)nslots, -1);
    ctx->slot_use.assign((size_t)nslots, 0);
    ctx->table_host.assign((size_t)nbricks, -1);
    ctx->ooc_tick = 0;
    ctx->ooc_stats = vr_stream_stats{};
    const size_t region = sizeof(float) * (size_t)ctx->rows * ctx->rows * ctx->rows;
    VR_CK(cudaStreamCreateWithFlags(&ctx->ooc_side, cudaStreamNonBlocking), "vr_load_cube_streamed: side stream");
    for (int i = 0; i < 2; ++i) {
        VR_CK(cudaHostAlloc(&ctx->ooc_pin[i], region, cudaHostAllocDefault), "vr_load_cube_streamed: staging");
        VR_CK(cudaMalloc(&ctx->ooc_dev[i], region), "vr_load_cube_streamed: staging");
        VR_CK(cudaEventCreateWithFlags(&ctx->ooc_ev[i], cudaEventDisableTiming), "vr_load_cube_streamed: events");
        VR_CK(cudaEventRecord(ctx->ooc_ev[i], ctx->ooc_side), "vr_load_cube_streamed: events");
    }
    VR_CK(cudaEventCreateWithFlags(&ctx->ooc_ev_table, cudaEventDisableTiming), "vr_load_cube_streamed: events");
    VR_CK(cudaEventRecord(ctx->ooc_ev_table, ctx->ooc_side), "vr_load_cube_streamed: events");
    VR_CK(cudaEventCreateWithFlags(&ctx->ooc_ev_render, cudaEventDisableTiming), "vr_load_cube_streamed: events");
    VR_CK(cudaHostAlloc(&ctx->ooc_pin_table, sizeof(int) * (size_t)nbricks, cudaHostAllocDefault),
          "vr_load_cube_streamed: table staging");
    VR_CK(cudaHostAlloc(&ctx->ooc_pin_list, sizeof(int) * (size_t)(2 * (nslots + 1)), cudaHostAllocDefault),
          "vr_load_cube_streamed: list staging");
    VR_CK(cudaMalloc(&ctx->ooc_dev_list, sizeof(int) * (size_t)(3 * (nslots + 1))), "vr_load_cube_streamed: lists");
    ctx->ooc_fn = fn;
    ctx->ooc_user = user;
    ctx->ooc = true;
    if (make_tensor_map(ctx)) {
        int cx, cy, cz;
        brick_cell_dims(ctx->dtype, &cx, &cy, &cz);
        const long long units = nslots * (long long)(B / cx) * (B / cy) * (B / cz);
        VR_CK(cudaMalloc(&ctx->cells, brick_cells_bytes(units)), "vr_load_cube_streamed: cell list");
    } else {
        free_cube(ctx);
        return fail(ctx, VR_ERR_UNSUPPORTED, "vr_load_cube_streamed: needs bricks of at least 32 voxels");
    }
    VR_CK(cudaStreamSynchronize(ctx->ooc_side), "vr_load_cube_streamed: set-up");
    ctx->has_cube = true;
    return VR_OK;
}

vr_status vr_get_stream_stats(const vr_ctx* ctx, vr_stream_stats* out) {
    if (!ctx || !out) return VR_ERR_INVALID_ARG;
    if (!ctx->ooc) return VR_ERR_STATE;
    *out = ctx->ooc_stats;
    return VR_OK;
}

vr_status vr_set_stream_timeout(vr_ctx* ctx, double seconds) {
    if (!ctx || !(seconds > 0.0) || !std::isfinite(seconds)) return VR_ERR_INVALID_ARG;
    ctx->ooc_timeout_s = seconds;
    return VR_OK;
}

vr_status vr_set_transfer_function(vr_ctx* ctx, const float* rgba, int n, float vmin, float vmax) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    if (!rgba || n < 2 || n > kMaxTF)
        return fail(ctx, VR_ERR_INVALID_ARG, "vr_set_transfer_function: need 2 <= n <= 1024 entries");
    if (!std::isfinite(vmin) || !std::isfinite(vmax) || !(vmax > vmin))
        return fail(ctx, VR_ERR_INVALID_ARG, "vr_set_transfer_function: need finite vmin < vmax");
    std::vector<float4> t((size_t)n);
    for (int i = 0; i < n; ++i) {
        t[(size_t)i] = make_float4(rgba[4 * i], rgba[4 * i + 1], rgba[4 * i + 2], rgba[4 * i + 3]);
        for (int c = 0; c < 4; ++c)
            if (!std::isfinite(rgba[4 * i + c]))
                return fail(ctx, VR_ERR_INVALID_ARG, "vr_set_transfer_function: non-finite entry");
    }
    ctx->tf.swap(t);
    ctx->vmin = vmin;
    ctx->vmax = vmax;
    ctx->has_tf = true;
    return VR_OK;
}

vr_status vr_set_camera(vr_ctx* ctx, const vr_camera* cams, int ncams) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    if (!cams || ncams < 1 || ncams > 4096)
        return fail(ctx, VR_ERR_INVALID_ARG, "vr_set_camera: need 1 <= ncams <= 4096");
    std::vector<CamDev> out((size_t)ncams);
    for (int i = 0; i < ncams; ++i) {
        const vr_camera& c = cams[i];
        if ((c.type != 0 && c.type != 1) || c.width <= 0 || c.height <= 0 ||
            c.width > 65536 || c.height > 65536 || c.width != cams[0].width ||
            c.height != cams[0].height)
            return fail(ctx, VR_ERR_INVALID_ARG, "vr_set_camera: bad type or size (all cameras must share one size)");
        if (!finite3(c.eye) || !finite3(c.right) || !finite3(c.up) || !finite3(c.fwd) ||
            !std::isfinite(c.win[0]) || !std::isfinite(c.win[1]) || !std::isfinite(c.win[2]) ||
            !std::isfinite(c.win[3]))
            return fail(ctx, VR_ERR_INVALID_ARG, "vr_set_camera: non-finite camera");
        if (beyond(c.eye, 3, 1e9) || beyond(c.right, 3, 1e9) || beyond(c.up, 3, 1e9) || beyond(c.fwd, 3, 1e9) ||
            beyond(c.win, 4, 1e9))
            return fail(ctx, VR_ERR_INVALID_ARG, "vr_set_camera: a camera value is beyond 1e9 in magnitude");
        {
            // right, up and fwd must span space: otherwise every ray of a perspective view lies
            // in one plane and a pixel direction can vanish (orthographic: no direction at all)
            const double* R = c.right;
            const double* U = c.up;
            const double* F = c.fwd;
            const double det = R[0] * (U[1] * F[2] - U[2] * F[1]) - U[0] * (R[1] * F[2] - R[2] * F[1]) +
                               F[0] * (R[1] * U[2] - R[2] * U[1]);
            const double scale = std::sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]) *
                                 std::sqrt(U[0] * U[0] + U[1] * U[1] + U[2] * U[2]) *
                                 std::sqrt(F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
            if (!(std::fabs(det) > 1e-12 * scale))
                return fail(ctx, VR_ERR_INVALID_ARG, "vr_set_camera: right, up and fwd do not span space");
        }
        if (c.win[1] == c.win[0] || c.win[3] == c.win[2])
            return fail(ctx, VR_ERR_INVALID_ARG, "vr_set_camera: empty window");
        CamDev& d = out[(size_t)i];
        for (int a = 0; a < 3; ++a) {
            d.eye[a] = c.eye[a];
            d.right[a] = c.right[a];
            d.up[a] = c.up[a];
            d.fwd[a] = c.fwd[a];
        }
        d.l = c.win[0];
        d.t = c.win[3];
        d.du = (c.win[1] - c.win[0]) / (double)c.width;
        d.dv = (c.win[3] - c.win[2]) / (double)c.height;
        d.type = c.type;
        d.width = c.width;
        d.height = c.height;
        d.pad = 0;
    }
    if ((long long)cams[0].width * cams[0].height > (1LL << 30) ||
        (long long)ncams * cams[0].width * cams[0].height > (1LL << 40))
        return fail(ctx, VR_ERR_INVALID_ARG, "vr_set_camera: too many pixels");
    ctx->cams.swap(out);
    return VR_OK;
}

vr_status vr_selftest_wait_timeout(vr_ctx* ctx, void* stream) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    DevGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    VR_CK(cudaGetLastError(), "vr_selftest_wait_timeout: pending CUDA error");
    VR_CK(launch_wait_probe(ctx->status_dev, 1000000ull, s), "vr_selftest_wait_timeout: launch");  // 1 ms
    VR_CK(cudaStreamSynchronize(s), "vr_selftest_wait_timeout: wait");
    if (*ctx->status_host != (int)kDevWaitTimeout)
        return fail(ctx, VR_ERR_INTERNAL, "vr_selftest_wait_timeout: the bounded wait did not expire");
    return VR_OK;
}

vr_status vr_set_sample_counter(vr_ctx* ctx, unsigned long long* device_counter) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    ctx->sample_counter = device_counter;
    return VR_OK;
}

vr_status vr_set_kernel_events(vr_ctx* ctx, void* start, void* stop) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    if ((start == nullptr) != (stop == nullptr))
        return fail(ctx, VR_ERR_INVALID_ARG, "vr_set_kernel_events: give both events or neither");
    ctx->ev_start = static_cast<cudaEvent_t>(start);
    ctx->ev_stop = static_cast<cudaEvent_t>(stop);
    return VR_OK;
}

vr_status vr_get_cube_info(const vr_ctx* ctx, vr_cube_info* info) {
    if (!ctx || !info) return VR_ERR_INVALID_ARG;
    if (!ctx->has_cube) return VR_ERR_STATE;
    info->nx = ctx->nx;
    info->ny = ctx->ny;
    info->nz = ctx->nz;
    info->nbx = ctx->nbx;
    info->nby = ctx->nby;
    info->nbz = ctx->nbz;
    info->brick = ctx->B;
    info->pitch = ctx->pitch;
    info->dtype = ctx->dtype;
    info->brick_bytes = ctx->slot_elems * (long long)ctx->elem;
    info->store_bytes = info->brick_bytes * (long long)ctx->nbx * ctx->nby * ctx->nbz * (ctx->pool1 ? 2 : 1);
    return VR_OK;
}

}  // extern "C"

namespace {

TFDev tf_dev(const vr_ctx* ctx) {
    TFDev t;
    std::memset(&t, 0, sizeof(t));
    t.n = (int)ctx->tf.size();
    for (int i = 0; i < t.n; ++i) t.tab[i] = ctx->tf[(size_t)i];
    t.vmin = ctx->vmin;
    t.inv_range = 1.0f / (ctx->vmax - ctx->vmin);
    t.zero_top = -1;
    while (t.zero_top + 1 < t.n && t.tab[t.zero_top + 1].w == 0.f) ++t.zero_top;
    return t;
}

vr_status render_ray(vr_ctx* ctx, vr_mode mode, float* out_rgba, float* out_max, cudaStream_t s) {
    const int ncams = (int)ctx->cams.size();
    const int nbatch = (ncams + kMaxLaunchCams - 1) / kMaxLaunchCams;
    VR_CK(cudaMemsetAsync(ctx->work, 0, sizeof(int) * nbatch, s), "vr_render: scheduler reset");
    MarchParams P;
    std::memset(&P, 0, sizeof(P));
    P.vol = vol_dev(ctx);
    P.tf = tf_dev(ctx);
    P.width = ctx->cams[0].width;
    P.height = ctx->cams[0].height;
    P.mode = mode;
    P.tile_w = ctx->tune.tile_w;
    P.tile_h = ctx->tune.tile_h;
    P.tiles_x = (P.width + P.tile_w - 1) / P.tile_w;
    P.tiles_y = (P.height + P.tile_h - 1) / P.tile_h;
    split(ctx->opt.step, P.step_hi, P.step_lo);
    P.ert = (float)ctx->opt.ert;
    P.samples = ctx->sample_counter;
    const int block = ctx->tune.block;
    const int grid = ctx->num_sms * march_blocks_per_sm(ctx->dtype, mode, P.vol.pool1 != nullptr, block) * block / 32;
    const long long img = (long long)P.width * P.height;
    if (ctx->ev_start) VR_CK(cudaEventRecord(ctx->ev_start, s), "vr_render: profiling event");
    for (int b = 0; b < nbatch; ++b) {
        const int c0 = b * kMaxLaunchCams;
        P.ncams = std::min(kMaxLaunchCams, ncams - c0);
        for (int i = 0; i < P.ncams; ++i) P.cams[i] = ray_cam(ctx->cams[(size_t)(c0 + i)]);
        P.out_rgba = reinterpret_cast<float4*>(out_rgba) + (long long)c0 * img;
        P.out_max = (mode == VR_MIP && out_max) ? out_max + (long long)c0 * img : nullptr;
        P.work = ctx->work + b;
        const int tiles = P.tiles_x * P.tiles_y * P.ncams;  // one warp per tile
        const int blocks = std::max(1, std::min(grid / (block / 32), (tiles + block / 32 - 1) / (block / 32)));
        VR_CK(launch_march(P, ctx->dtype, blocks, block, s), "vr_render: march launch");
    }
    if (ctx->ev_stop) VR_CK(cudaEventRecord(ctx->ev_stop, s), "vr_render: profiling event");
    return VR_OK;
}

vr_status ensure_pixel_scratch(vr_ctx* ctx, long long npix) {
    if (npix <= ctx->scratch_pix) return VR_OK;
    if (ctx->krange) cudaFree(ctx->krange);
    if (ctx->pixdir) cudaFree(ctx->pixdir);
    if (ctx->enc) cudaFree(ctx->enc);
    ctx->krange = nullptr;
    ctx->pixdir = nullptr;
    ctx->enc = nullptr;
    ctx->scratch_pix = 0;
    VR_CK(cudaMalloc(&ctx->krange, sizeof(int2) * npix), "vr_render: pixel scratch");
    VR_CK(cudaMalloc(&ctx->pixdir, 2 * sizeof(float4) * npix), "vr_render: pixel scratch");
    VR_CK(cudaMalloc(&ctx->enc, sizeof(unsigned int) * npix), "vr_render: pixel scratch");
    ctx->scratch_pix = npix;
    return VR_OK;
}

// MIP through the brick pass, up to kMaxLaunchCams cameras per pass over the
// cube: pixel set-up per camera (sample ranges, running maxima), one staged
// brick pass for the batch, transfer-function finalisation per camera.
vr_status render_brick_mip(vr_ctx* ctx, float* out_rgba, float* out_max, cudaStream_t s) {
    const int W = ctx->cams[0].width, H = ctx->cams[0].height;
    const long long img = (long long)W * H;
    const int ncams = (int)ctx->cams.size();
    // cameras per pass: at most kMaxLaunchCams, and few enough that a pixel index of the
    // pass (camera * W * H + pixel) fits an int
    const int per = (int)std::min<long long>(std::min(ncams, kMaxLaunchCams), std::max(1LL, INT_MAX / img));
    vr_status st = ensure_pixel_scratch(ctx, img * per);
    if (st != VR_OK) return st;
    PixelParams pp;
    std::memset(&pp, 0, sizeof(pp));
    pp.vol = vol_dev(ctx);
    pp.tf = tf_dev(ctx);
    split(ctx->opt.step, pp.step_hi, pp.step_lo);
    pp.width = W;
    pp.height = H;
    BrickParams bp;
    std::memset(&bp, 0, sizeof(bp));
    bp.vol = pp.vol;
    split(ctx->opt.step, bp.step, bp.step_lo);
    bp.width = W;
    bp.height = H;
    int cx, cy, cz;
    brick_cell_dims(ctx->dtype, &cx, &cy, &cz);
    bp.ncells_x = ctx->B / cx;
    bp.ncells_y = ctx->B / cy;
    bp.ncells_z = ctx->B / cz;
    bp.nbricks = ctx->nbx * ctx->nby * ctx->nbz;
    bp.krange = ctx->krange;
    bp.pixdir = ctx->pixdir;
    bp.status = ctx->status_dev;
    const int grid = 2 * ctx->num_sms;
    for (int c0 = 0; c0 < ncams; c0 += per) {
        const int nb = std::min(per, ncams - c0);
        bp.ncams = nb;
        unsigned int* enc = out_max ? reinterpret_cast<unsigned int*>(out_max + (long long)c0 * img) : ctx->enc;
        for (int i = 0; i < nb; ++i) {
            if (!cam_ff(ctx->cams[(size_t)(c0 + i)], bp.cams[i]))
                return fail(ctx, VR_ERR_INVALID_ARG, "vr_render: camera basis is singular");
            pp.cam = ray_cam(ctx->cams[(size_t)(c0 + i)]);
            pp.krange = ctx->krange + (long long)i * img;
            pp.pixdir = ctx->pixdir + 2 * (long long)i * img;
            pp.enc = enc + (long long)i * img;
            VR_CK(launch_pixel_setup(pp, s), "vr_render: pixel set-up");
        }
        bp.out_enc = enc;
        bp.work = ctx->work + kMaxLaunchCams + (c0 / per) % 4096;
        VR_CK(cudaMemsetAsync(bp.work, 0, sizeof(int), s), "vr_render: scheduler reset");
        if (c0 == 0 && ctx->ev_start) VR_CK(cudaEventRecord(ctx->ev_start, s), "vr_render: profiling event");
        VR_CK(launch_brick_mip(&ctx->tmap, bp, ctx->dtype, grid, ctx->cells, s, ctx->tune.group),
              "vr_render: brick pass");
        if (c0 + nb >= ncams && ctx->ev_stop) VR_CK(cudaEventRecord(ctx->ev_stop, s), "vr_render: profiling event");
        for (int i = 0; i < nb; ++i) {
            pp.cam = ray_cam(ctx->cams[(size_t)(c0 + i)]);
            pp.enc = enc + (long long)i * img;
            pp.out_rgba = reinterpret_cast<float4*>(out_rgba) + (long long)(c0 + i) * img;
            pp.out_max = out_max ? out_max + (long long)(c0 + i) * img : nullptr;
            VR_CK(launch_mip_finalize(pp, s), "vr_render: finalise");
        }
    }
    return VR_OK;
}

// grow a device buffer to at least n elements (contents not kept)
template <typename P>
vr_status grow(vr_ctx* ctx, P*& ptr, long long& cap, long long n, const char* what) {
    if (n <= cap) return VR_OK;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    cap = 0;
    VR_CK(cudaMalloc(&ptr, sizeof(P) * (size_t)n), what);
    cap = n;
    return VR_OK;
}

// Upper bound of the visibility key of any brick for this camera, plus one.
int layer_bound(const vr_ctx* ctx, const CamDev& c) {
    const int nb[3] = {ctx->nbx, ctx->nby, ctx->nbz};
    int m = 0;
    for (int a = 0; a < 3; ++a) {
        if (c.type == 1) {
            const long long e = (long long)std::floor(c.eye[a] / (double)ctx->B);
            m += (int)std::min<long long>(1 << 20, std::max(std::llabs(e), std::llabs((long long)nb[a] - 1 - e)));
        } else {
            m += nb[a] - 1;
        }
    }
    return m + 1;
}

// Sort-last partial images of camera cd through staged cells (launch_cell_partials:
// the bricks of brick_list, or every brick), into sp.partial [0, npartial) with
// the footprints sp.foot.  *done = false, with nothing launched, when this form
// does not apply (no cells, a table beyond kMaxPartTF entries, slot indices
// beyond an int): the caller then marches whole bricks (launch_brick_partial).
vr_status staged_partials(vr_ctx* ctx, const CamDev& cd, const SortParams& sp, int mode, const int* brick_list,
                          int nlist, long long npartial, cudaStream_t s, bool* done) {
    *done = false;
    if (!ctx->has_tmap_part || !ctx->cells || (int)ctx->tf.size() > kMaxPartTF || npartial >= (long long)INT_MAX)
        return VR_OK;
    BrickParams bp;
    std::memset(&bp, 0, sizeof(bp));
    bp.vol = sp.vol;
    bp.cams[0] = sp.cam;
    bp.ncams = 1;
    bp.width = cd.width;
    bp.height = cd.height;
    split(ctx->opt.step, bp.step, bp.step_lo);
    int c3[3];
    brick_cell_dims(ctx->dtype, &c3[0], &c3[1], &c3[2]);
    bp.ncells_x = ctx->B / c3[0];
    bp.ncells_y = ctx->B / c3[1];
    bp.ncells_z = ctx->B / c3[2];
    bp.nbricks = ctx->nbx * ctx->nby * ctx->nbz;
    bp.krange = ctx->krange;
    bp.pixdir = ctx->pixdir;  // written by the pixel set-up of this view
    bp.status = ctx->status_dev;
    bp.work = ctx->work;
    bp.brick_list = brick_list;
    bp.nlist = nlist;
    bp.foot = sp.foot;
    bp.partial = sp.partial;
    bp.key_persp = cd.type == 1;
    for (int a = 0; a < 3; ++a) {
        bp.eye_cell[a] = (int)std::max<double>(-(1 << 20), std::min<double>(1 << 20, std::floor(cd.eye[a] / c3[a])));
        bp.key_sign[a] = sp.cam.dir_hi[a] > 0.f ? 1 : (sp.cam.dir_hi[a] < 0.f ? -1 : 0);
    }
    VR_CK(launch_cell_partials(&ctx->tmap_part, bp, sp.tf, ctx->dtype, mode, npartial,
                               cell_partial_passes(ctx->dtype, ctx->B), 2 * ctx->num_sms, ctx->cells, s,
                               ctx->tune.group),
          "sort-last partial images");
    *done = true;
    return VR_OK;
}

// Composite in object order.  carried = false: per-brick partial images from
// T = 1 folded in visibility order (no early termination).  carried = true:
// one visibility layer of bricks per launch, each pixel's running (C, T)
// carried through with per-sample early termination.
vr_status render_bricks_composite(vr_ctx* ctx, float* out_rgba, cudaStream_t s, bool carried) {
    const int W = ctx->cams[0].width, H = ctx->cams[0].height;
    const long long img = (long long)W * H;
    const long long nbricks = (long long)ctx->nbx * ctx->nby * ctx->nbz;
    vr_status st = ensure_pixel_scratch(ctx, img);
    if (st != VR_OK) return st;
    long long cap = ctx->sort_bricks;
    if (nbricks + 1 > cap) {
        if (ctx->foot) cudaFree(ctx->foot);
        if (ctx->order) cudaFree(ctx->order);
        if (ctx->tile_start) cudaFree(ctx->tile_start);
        ctx->foot = nullptr;
        ctx->order = nullptr;
        ctx->tile_start = nullptr;
        ctx->sort_bricks = 0;
        VR_CK(cudaMalloc(&ctx->foot, sizeof(BrickFoot) * (size_t)nbricks), "sort-last scratch");
        VR_CK(cudaMalloc(&ctx->order, sizeof(int) * (size_t)nbricks), "sort-last scratch");
        VR_CK(cudaMalloc(&ctx->tile_start, sizeof(int) * (size_t)(nbricks + 1)), "sort-last scratch");
        ctx->sort_bricks = nbricks + 1;
    }
    if (!ctx->partial_used) VR_CK(cudaMalloc(&ctx->partial_used, sizeof(unsigned long long)), "sort-last scratch");
    if (carried) {
        st = grow(ctx, ctx->state, ctx->state_cap, img, "layered state");
        if (st != VR_OK) return st;
    }
    SortParams sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.vol = vol_dev(ctx);
    sp.tf = tf_dev(ctx);
    split(ctx->opt.step, sp.step, sp.step_lo);
    sp.ert = carried ? (float)ctx->opt.ert : 2.0f;
    sp.krange = ctx->krange;
    sp.foot = ctx->foot;
    sp.order = ctx->order;
    sp.tile_start = ctx->tile_start;
    sp.partial_used = ctx->partial_used;
    sp.state = ctx->state;
    PixelParams pp;
    std::memset(&pp, 0, sizeof(pp));
    pp.vol = sp.vol;
    pp.tf = sp.tf;
    split(ctx->opt.step, pp.step_hi, pp.step_lo);
    pp.width = W;
    pp.height = H;
    pp.krange = ctx->krange;
    pp.pixdir = ctx->pixdir;
    pp.enc = ctx->enc;
    const int grid = ctx->num_sms * 8;
    for (size_t ci = 0; ci < ctx->cams.size(); ++ci) {
        const CamDev& cd = ctx->cams[ci];
        if (!cam_ff(cd, sp.cam)) return fail(ctx, VR_ERR_INVALID_ARG, "vr_render: camera basis is singular");
        const int L = layer_bound(ctx, cd);
        for (int ax = 0; ax < 3; ++ax)
            sp.eye_brick[ax] = (int)std::max<double>(-(1 << 20), std::min<double>(1 << 20, std::floor(cd.eye[ax] / (double)ctx->B)));
        if (L + 1 > ctx->layer_cap) {
            if (ctx->layer_buf) cudaFree(ctx->layer_buf);
            ctx->layer_buf = nullptr;
            ctx->layer_cap = 0;
            VR_CK(cudaMalloc(&ctx->layer_buf, sizeof(int) * 3 * (size_t)(L + 1)), "sort-last scratch");
            ctx->layer_cap = L + 1;
        }
        if (L + 2 > ctx->host_rb_cap) {
            if (ctx->host_rb) cudaFreeHost(ctx->host_rb);
            ctx->host_rb = nullptr;
            ctx->host_rb_cap = 0;
            VR_CK(cudaHostAlloc(&ctx->host_rb, sizeof(int) * (size_t)(L + 4), cudaHostAllocDefault), "read-back");
            ctx->host_rb_cap = L + 4;
        }
        sp.max_layers = L;
        sp.layer_count = ctx->layer_buf;
        sp.layer_start = ctx->layer_buf + (L + 1);
        sp.layer_fill = ctx->layer_buf + 2 * (L + 1);
        sp.out_rgba = reinterpret_cast<float4*>(out_rgba) + (long long)ci * img;
        pp.cam = ray_cam(cd);
        VR_CK(launch_pixel_setup(pp, s), "vr_render: pixel set-up");
        VR_CK(cudaMemsetAsync(sp.layer_count, 0, sizeof(int) * (size_t)L, s), "vr_render: reset");
        VR_CK(cudaMemsetAsync(sp.partial_used, 0, sizeof(unsigned long long), s), "vr_render: reset");
        VR_CK(launch_brick_footprints(sp, s), "vr_render: brick footprints");
        // read back the layer starts and the partial-image size (host decides the launches)
        VR_CK(cudaMemcpyAsync(ctx->host_rb, sp.layer_start, sizeof(int) * (size_t)(L + 1), cudaMemcpyDeviceToHost, s),
              "vr_render: read-back");
        unsigned long long used = 0;
        VR_CK(cudaMemcpyAsync(&used, sp.partial_used, sizeof(used), cudaMemcpyDeviceToHost, s), "vr_render: read-back");
        VR_CK(cudaStreamSynchronize(s), "vr_render: read-back");
        if (!carried) {
            vr_status g = grow(ctx, ctx->partial, ctx->partial_cap, (long long)std::max<unsigned long long>(used, 1),
                               "partial images");
            if (g != VR_OK) return g;
            sp.partial = ctx->partial;
            sp.work = ctx->work;
            if (ctx->ev_start && ci == 0) VR_CK(cudaEventRecord(ctx->ev_start, s), "vr_render: profiling event");
            bool staged = false;
            st = staged_partials(ctx, cd, sp, VR_COMPOSITE, nullptr, 0, (long long)used, s, &staged);
            if (st != VR_OK) return st;
            if (!staged) {
                VR_CK(launch_tile_scan(sp, s), "vr_render: tile prefix");
                VR_CK(cudaMemsetAsync(sp.work, 0, sizeof(int), s), "vr_render: scheduler reset");
                VR_CK(launch_brick_partial(sp, ctx->dtype, false, 0, L, grid, s), "vr_render: partial images");
            }
            if (ctx->ev_stop && ci + 1 == ctx->cams.size())
                VR_CK(cudaEventRecord(ctx->ev_stop, s), "vr_render: profiling event");
            VR_CK(launch_sortlast_fold(sp, s), "vr_render: sort-last fold");
        } else {
            VR_CK(launch_tile_scan(sp, s), "vr_render: tile prefix");
            VR_CK(launch_state_init(sp, s), "vr_render: state init");
            int slot = 0;
            if (ctx->ev_start && ci == 0) VR_CK(cudaEventRecord(ctx->ev_start, s), "vr_render: profiling event");
            for (int l = 0; l < L; ++l) {
                if (ctx->host_rb[l + 1] == ctx->host_rb[l]) continue;  // empty layer
                sp.work = ctx->work + (slot++ % ctx->work_slots);
                VR_CK(cudaMemsetAsync(sp.work, 0, sizeof(int), s), "vr_render: scheduler reset");
                VR_CK(launch_brick_partial(sp, ctx->dtype, true, l, l + 1, grid, s), "vr_render: layer");
            }
            if (ctx->ev_stop && ci + 1 == ctx->cams.size())
                VR_CK(cudaEventRecord(ctx->ev_stop, s), "vr_render: profiling event");
            VR_CK(launch_state_finish(sp, s), "vr_render: state finish");
        }
    }
    return VR_OK;
}

// ------------------------------------------------------------------ out of core
double seconds_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// Host wait for a device event, bounded by the context's deadline.
vr_status wait_event(vr_ctx* ctx, cudaEvent_t e, const char* what) {
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t q = cudaEventQuery(e);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) return cuda_fail(ctx, q, what);
        if (seconds_since(t0) > ctx->ooc_timeout_s) {
            ctx->ooc_stats.wait_s += seconds_since(t0);
            return fail(ctx, VR_ERR_TIMEOUT, std::string(what) + ": device wait exceeded the deadline");
        }
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    ctx->ooc_stats.wait_s += seconds_since(t0);
    return VR_OK;
}

// Make the bricks of `list` resident (render stream s waits for them).  Slots
// in use by this batch are never evicted; the batch must fit the cache.
vr_status ensure_resident(vr_ctx* ctx, const int* list, int n, cudaStream_t s) {
    const long long tick = ++ctx->ooc_tick;
    const int nslots = (int)ctx->pool_slots;
    if (n > nslots) return fail(ctx, VR_ERR_INTERNAL, "out-of-core batch larger than the brick cache");
    for (int i = 0; i < n; ++i) {
        const int sl = ctx->table_host[(size_t)list[i]];
        if (sl >= 0) ctx->slot_use[(size_t)sl] = tick;
    }
    // the side stream must not overwrite a slot that earlier render work still reads
    VR_CK(cudaEventRecord(ctx->ooc_ev_render, s), "out of core: render event");
    VR_CK(cudaStreamWaitEvent(ctx->ooc_side, ctx->ooc_ev_render, 0), "out of core: stream order");
    const int B = ctx->B;
    const VolDev v = vol_dev(ctx);
    bool changed = false;
    for (int i = 0; i < n; ++i) {
        const int b = list[i];
        if (ctx->table_host[(size_t)b] >= 0) continue;
        // a free slot, else the least recently used one not needed by this batch
        int slot = -1;
        long long best = tick;
        for (int sl = 0; sl < nslots; ++sl) {
            if (ctx->slot_brick[(size_t)sl] < 0) {
                slot = sl;
                break;
            }
            if (ctx->slot_use[(size_t)sl] < best) {
                best = ctx->slot_use[(size_t)sl];
                slot = sl;
            }
        }
        if (slot < 0) return fail(ctx, VR_ERR_INTERNAL, "out of core: no evictable slot");
        if (ctx->slot_brick[(size_t)slot] >= 0) ctx->table_host[(size_t)ctx->slot_brick[(size_t)slot]] = -1;
        ctx->slot_brick[(size_t)slot] = -1;
        const int bx = b % ctx->nbx, by = (b / ctx->nbx) % ctx->nby, bz = b / (ctx->nbx * ctx->nby);
        const long long x0 = std::max<long long>((long long)bx * B - 1, 0), x1 = std::min<long long>((long long)bx * B + B + 1, ctx->nx);
        const long long y0 = std::max<long long>((long long)by * B - 1, 0), y1 = std::min<long long>((long long)by * B + B + 1, ctx->ny);
        const long long z0 = std::max<long long>((long long)bz * B - 1, 0), z1 = std::min<long long>((long long)bz * B + B + 1, ctx->nz);
        const int buf = ctx->ooc_next_buf;
        ctx->ooc_next_buf ^= 1;
        vr_status st = wait_event(ctx, ctx->ooc_ev[buf], "out of core: staging buffer");  // its last upload
        if (st != VR_OK) return st;
        const auto t0 = std::chrono::steady_clock::now();
        const int rc = ctx->ooc_fn(ctx->ooc_user, x0, y0, z0, x1 - x0, y1 - y0, z1 - z0, ctx->ooc_pin[buf]);
        const double dt = seconds_since(t0);
        ctx->ooc_stats.generate_s += dt;
        if (rc != 0) return fail(ctx, VR_ERR_IO, "out of core: the region callback failed (" + std::to_string(rc) + ")");
        if (dt > ctx->ooc_timeout_s) return fail(ctx, VR_ERR_TIMEOUT, "out of core: the region callback exceeded the deadline");
        const size_t bytes = sizeof(float) * (size_t)((x1 - x0) * (y1 - y0) * (z1 - z0));
        VR_CK(cudaMemcpyAsync(ctx->ooc_dev[buf], ctx->ooc_pin[buf], bytes, cudaMemcpyHostToDevice, ctx->ooc_side),
              "out of core: upload");
        void* slotp = static_cast<char*>(ctx->pool) + (size_t)slot * ctx->slot_elems * ctx->elem;
        VR_CK(launch_repack_region(ctx->ooc_dev[buf], (int)x0, (int)y0, (int)z0, (int)(x1 - x0), (int)(y1 - y0),
                                   (int)(z1 - z0), bx, by, bz, v, ctx->dtype, slotp, ctx->ooc_side),
              "out of core: repack");
        VR_CK(cudaEventRecord(ctx->ooc_ev[buf], ctx->ooc_side), "out of core: upload event");
        ctx->slot_brick[(size_t)slot] = b;
        ctx->table_host[(size_t)b] = slot;
        ctx->slot_use[(size_t)slot] = tick;
        ctx->ooc_stats.bricks_fetched++;
        ctx->ooc_stats.bytes_h2d += bytes;
        changed = true;
    }
    if (changed) {
        // publish the brick table (the previous upload of the staging copy must be done)
        vr_status st = wait_event(ctx, ctx->ooc_ev_table, "out of core: table upload");
        if (st != VR_OK) return st;
        const size_t nb = (size_t)ctx->nbx * ctx->nby * ctx->nbz;
        std::memcpy(ctx->ooc_pin_table, ctx->table_host.data(), sizeof(int) * nb);
        VR_CK(cudaMemcpyAsync(ctx->table, ctx->ooc_pin_table, sizeof(int) * nb, cudaMemcpyHostToDevice, ctx->ooc_side),
              "out of core: table upload");
        VR_CK(cudaEventRecord(ctx->ooc_ev_table, ctx->ooc_side), "out of core: table event");
    }
    VR_CK(cudaEventRecord(ctx->ooc_ev_render, ctx->ooc_side), "out of core: ready event");
    VR_CK(cudaStreamWaitEvent(s, ctx->ooc_ev_render, 0), "out of core: stream order");
    ctx->ooc_stats.batches++;
    return VR_OK;
}

// Footprints and visibility order of one camera (read back to the host).
// Footprints, keys and visibility layers of every brick for camera cd, read back to the
// host (the out-of-core batches and the distributed partials are planned from them).
vr_status ooc_footprints(vr_ctx* ctx, const CamDev& cd, SortParams& sp, std::vector<int>& order,
                         std::vector<int>& layer_start, std::vector<BrickFoot>& foot, cudaStream_t s) {
    const long long nbricks = (long long)ctx->nbx * ctx->nby * ctx->nbz;
    if (nbricks + 1 > ctx->sort_bricks) {
        if (ctx->foot) cudaFree(ctx->foot);
        if (ctx->order) cudaFree(ctx->order);
        if (ctx->tile_start) cudaFree(ctx->tile_start);
        ctx->foot = nullptr;
        ctx->order = nullptr;
        ctx->tile_start = nullptr;
        ctx->sort_bricks = 0;
        VR_CK(cudaMalloc(&ctx->foot, sizeof(BrickFoot) * (size_t)nbricks), "footprints: scratch");
        VR_CK(cudaMalloc(&ctx->order, sizeof(int) * (size_t)nbricks), "footprints: scratch");
        VR_CK(cudaMalloc(&ctx->tile_start, sizeof(int) * (size_t)(nbricks + 1)), "footprints: scratch");
        ctx->sort_bricks = nbricks + 1;
    }
    if (!ctx->partial_used) VR_CK(cudaMalloc(&ctx->partial_used, sizeof(unsigned long long)), "footprints: scratch");
    const int L = layer_bound(ctx, cd);
    if (L + 1 > ctx->layer_cap) {
        if (ctx->layer_buf) cudaFree(ctx->layer_buf);
        ctx->layer_buf = nullptr;
        ctx->layer_cap = 0;
        VR_CK(cudaMalloc(&ctx->layer_buf, sizeof(int) * 3 * (size_t)(L + 1)), "footprints: scratch");
        ctx->layer_cap = L + 1;
    }
    if (!cam_ff(cd, sp.cam)) return fail(ctx, VR_ERR_INVALID_ARG, "vr_render: camera basis is singular");
    for (int ax = 0; ax < 3; ++ax)
        sp.eye_brick[ax] = (int)std::max<double>(-(1 << 20), std::min<double>(1 << 20, std::floor(cd.eye[ax] / (double)ctx->B)));
    sp.all_bricks = 1;
    sp.max_layers = L;
    sp.foot = ctx->foot;
    sp.order = ctx->order;
    sp.tile_start = ctx->tile_start;
    sp.partial_used = ctx->partial_used;
    sp.layer_count = ctx->layer_buf;
    sp.layer_start = ctx->layer_buf + (L + 1);
    sp.layer_fill = ctx->layer_buf + 2 * (L + 1);
    VR_CK(cudaMemsetAsync(sp.layer_count, 0, sizeof(int) * (size_t)L, s), "footprints: reset");
    VR_CK(cudaMemsetAsync(sp.partial_used, 0, sizeof(unsigned long long), s), "footprints: reset");
    VR_CK(launch_brick_footprints(sp, s), "footprints: launch");
    layer_start.resize((size_t)L + 1);
    VR_CK(cudaMemcpyAsync(layer_start.data(), sp.layer_start, sizeof(int) * (size_t)(L + 1), cudaMemcpyDeviceToHost, s),
          "footprints: read-back");
    VR_CK(cudaStreamSynchronize(s), "footprints: read-back");
    const int nvis = layer_start[(size_t)L];
    order.resize((size_t)nvis);
    foot.resize((size_t)nbricks);
    if (nvis > 0) {
        VR_CK(cudaMemcpy(order.data(), sp.order, sizeof(int) * (size_t)nvis, cudaMemcpyDeviceToHost), "footprints: read-back");
        VR_CK(cudaMemcpy(foot.data(), sp.foot, sizeof(BrickFoot) * (size_t)nbricks, cudaMemcpyDeviceToHost),
              "footprints: read-back");
    }
    return VR_OK;
}

vr_status render_ooc(vr_ctx* ctx, vr_mode mode, float* out_rgba, float* out_max, cudaStream_t s) {
    const int W = ctx->cams[0].width, H = ctx->cams[0].height;
    const long long img = (long long)W * H;
    vr_status st = ensure_pixel_scratch(ctx, img);
    if (st != VR_OK) return st;
    if (mode == VR_COMPOSITE) {
        st = grow(ctx, ctx->state, ctx->state_cap, img, "layered state");
        if (st != VR_OK) return st;
    }
    const int nslots = (int)ctx->pool_slots;
    SortParams sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.vol = vol_dev(ctx);
    sp.tf = tf_dev(ctx);
    split(ctx->opt.step, sp.step, sp.step_lo);
    sp.ert = (float)ctx->opt.ert;
    sp.krange = ctx->krange;
    sp.state = ctx->state;
    PixelParams pp;
    std::memset(&pp, 0, sizeof(pp));
    pp.vol = sp.vol;
    pp.tf = sp.tf;
    split(ctx->opt.step, pp.step_hi, pp.step_lo);
    pp.width = W;
    pp.height = H;
    pp.krange = ctx->krange;
    pp.pixdir = ctx->pixdir;
    BrickParams bp;
    std::memset(&bp, 0, sizeof(bp));
    bp.vol = sp.vol;
    split(ctx->opt.step, bp.step, bp.step_lo);
    bp.width = W;
    bp.height = H;
    bp.ncams = 1;
    int cx, cy, cz;
    brick_cell_dims(ctx->dtype, &cx, &cy, &cz);
    bp.ncells_x = ctx->B / cx;
    bp.ncells_y = ctx->B / cy;
    bp.ncells_z = ctx->B / cz;
    bp.nbricks = ctx->nbx * ctx->nby * ctx->nbz;
    bp.krange = ctx->krange;
    bp.pixdir = ctx->pixdir;
    bp.status = ctx->status_dev;
    std::vector<int> order, layer_start, list;
    std::vector<BrickFoot> foot;
    for (size_t ci = 0; ci < ctx->cams.size(); ++ci) {
        const CamDev& cd = ctx->cams[ci];
        st = ooc_footprints(ctx, cd, sp, order, layer_start, foot, s);
        if (st != VR_OK) return st;
        pp.cam = ray_cam(cd);
        pp.out_rgba = reinterpret_cast<float4*>(out_rgba) + (long long)ci * img;
        pp.out_max = out_max ? out_max + (long long)ci * img : nullptr;
        pp.enc = (mode == VR_MIP && out_max) ? reinterpret_cast<unsigned int*>(pp.out_max) : ctx->enc;
        VR_CK(launch_pixel_setup(pp, s), "out of core: pixel set-up");
        if (mode == VR_MIP) {
            if (!cam_ff(cd, bp.cams[0])) return fail(ctx, VR_ERR_INVALID_ARG, "vr_render: camera basis is singular");
            bp.out_enc = pp.enc;
            // batches of visible bricks in visibility order, as many as the cache holds
            for (size_t b0 = 0; b0 < order.size(); b0 += (size_t)nslots) {
                const int n = (int)std::min<size_t>((size_t)nslots, order.size() - b0);
                st = ensure_resident(ctx, order.data() + b0, n, s);
                if (st != VR_OK) return st;
                bp.brick_list = sp.order + b0;  // the same list, still on the device
                bp.nlist = n;
                bp.work = ctx->work;
                VR_CK(cudaMemsetAsync(bp.work, 0, sizeof(int), s), "out of core: scheduler reset");
                VR_CK(launch_brick_mip(&ctx->tmap, bp, ctx->dtype, 2 * ctx->num_sms, ctx->cells, s, ctx->tune.group),
                      "out of core: brick pass");
            }
            VR_CK(launch_mip_finalize(pp, s), "out of core: finalise");
            continue;
        }
        // composite: layer by layer, skipping bricks behind terminated pixels
        sp.out_rgba = pp.out_rgba;
        VR_CK(launch_state_init(sp, s), "out of core: state init");
        const int L = sp.max_layers;
        for (int l = 0; l < L; ++l) {
            const int l0 = layer_start[(size_t)l], l1 = layer_start[(size_t)l + 1];
            if (l1 == l0) continue;
            const int n = l1 - l0;
            int* flags = ctx->ooc_dev_list + 2 * (nslots + 1);  // scratch after the two lists
            // flags for this layer's bricks, computed in chunks of up to nslots
            list.clear();
            for (int c0 = 0; c0 < n; c0 += nslots) {
                const int m = std::min(nslots, n - c0);
                VR_CK(launch_bricks_open(sp.foot, sp.order + l0 + c0, m, ctx->state, W, sp.ert, flags, s),
                      "out of core: open test");
                VR_CK(cudaMemcpyAsync(ctx->ooc_pin_list, flags, sizeof(int) * (size_t)m, cudaMemcpyDeviceToHost, s),
                      "out of core: read-back");
                VR_CK(cudaStreamSynchronize(s), "out of core: read-back");
                for (int i = 0; i < m; ++i) {
                    if (ctx->ooc_pin_list[i]) list.push_back(order[(size_t)(l0 + c0 + i)]);
                    else ctx->ooc_stats.bricks_culled++;
                }
            }
            for (size_t b0 = 0; b0 < list.size(); b0 += (size_t)nslots) {
                const int m = (int)std::min<size_t>((size_t)nslots, list.size() - b0);
                st = ensure_resident(ctx, list.data() + b0, m, s);
                if (st != VR_OK) return st;
                // the batch and its 8 x 4 tile prefix, to the device
                int* pin = ctx->ooc_pin_list;
                int acc = 0;
                for (int i = 0; i < m; ++i) {
                    const int4 r = foot[(size_t)list[b0 + (size_t)i]].rect;
                    pin[i] = list[b0 + (size_t)i];
                    pin[nslots + 1 + i] = acc;
                    acc += ((r.z - r.x + 1 + 7) / 8) * ((r.w - r.y + 1 + 3) / 4);
                }
                pin[nslots + 1 + m] = acc;
                VR_CK(cudaMemcpyAsync(ctx->ooc_dev_list, pin, sizeof(int) * (size_t)(2 * (nslots + 1)),
                                      cudaMemcpyHostToDevice, s),
                      "out of core: batch upload");
                sp.sub_order = ctx->ooc_dev_list;
                sp.sub_tile = ctx->ooc_dev_list + nslots + 1;
                sp.sub_n = m;
                sp.work = ctx->work;
                VR_CK(cudaMemsetAsync(sp.work, 0, sizeof(int), s), "out of core: scheduler reset");
                VR_CK(launch_brick_partial(sp, ctx->dtype, true, 0, 0, ctx->num_sms * 8, s), "out of core: layer");
                // the pinned batch buffer is reused by the next batch: wait for this upload
                VR_CK(cudaStreamSynchronize(s), "out of core: batch");
            }
        }
        sp.sub_order = nullptr;
        VR_CK(launch_state_finish(sp, s), "out of core: state finish");
    }
    return VR_OK;
}

}  // namespace

namespace vr {

// Checks shared by allocation-free callers of the brick-path MIP: context
// state, output alignment, a usable brick store.  On success returns the
// context's device and the pixel count of one camera.
vr_status brick_mip_precheck(vr_ctx* ctx, float* out_rgba, float* out_max, int* device,
                             long long* pixels) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    if (!out_rgba) return fail(ctx, VR_ERR_INVALID_ARG, "out_rgba is NULL");
    if (reinterpret_cast<uintptr_t>(out_rgba) % 16 || reinterpret_cast<uintptr_t>(out_max) % 4)
        return fail(ctx, VR_ERR_INVALID_ARG, "out_rgba must be 16-byte aligned, out_max 4-byte");
    if (!ctx->has_cube) return fail(ctx, VR_ERR_STATE, "no cube loaded");
    if (!ctx->has_tf) return fail(ctx, VR_ERR_STATE, "no transfer function set");
    if (ctx->cams.empty()) return fail(ctx, VR_ERR_STATE, "no camera set");
    if (!ctx->has_tmap)
        return fail(ctx, VR_ERR_UNSUPPORTED, "the brick pass needs bricks of at least 32 voxels");
    if (ctx->ooc) return fail(ctx, VR_ERR_UNSUPPORTED, "not for out-of-core cubes");
    if (*ctx->status_host != 0) {
        const int code = *ctx->status_host;
        *ctx->status_host = 0;
        return fail(ctx, VR_ERR_INTERNAL,
                    "an earlier brick pass stopped: a shared-memory load wait exceeded its bound (status " +
                        std::to_string(code) + ")");
    }
    *device = ctx->device;
    *pixels = (long long)ctx->cams[0].width * ctx->cams[0].height;
    return VR_OK;
}

vr_status set_error(vr_ctx* ctx, vr_status s, const char* msg) { return fail(ctx, s, msg); }

// Brick-path MIP of every camera with caller-provided scratch: krange and enc
// hold one camera's pixels, work one int.  Allocates nothing.
vr_status brick_mip_with_scratch(vr_ctx* ctx, float* out_rgba, float* out_max, cudaStream_t s,
                                 int2* krange, unsigned int* enc, int* work) {
    const int W = ctx->cams[0].width, H = ctx->cams[0].height;
    const long long img = (long long)W * H;
    VR_CK(cudaGetLastError(), "pending CUDA error");
    PixelParams pp;
    std::memset(&pp, 0, sizeof(pp));
    pp.vol = vol_dev(ctx);
    pp.tf = tf_dev(ctx);
    split(ctx->opt.step, pp.step_hi, pp.step_lo);
    pp.width = W;
    pp.height = H;
    pp.krange = krange;
    BrickParams bp;
    std::memset(&bp, 0, sizeof(bp));
    bp.vol = pp.vol;
    split(ctx->opt.step, bp.step, bp.step_lo);
    int cx, cy, cz;
    brick_cell_dims(ctx->dtype, &cx, &cy, &cz);
    bp.ncells_x = ctx->B / cx;
    bp.ncells_y = ctx->B / cy;
    bp.ncells_z = ctx->B / cz;
    bp.nbricks = ctx->nbx * ctx->nby * ctx->nbz;
    bp.krange = krange;
    bp.status = ctx->status_dev;
    bp.work = work;
    bp.width = W;
    bp.height = H;
    bp.ncams = 1;
    const int ncams = (int)ctx->cams.size();
    for (int i = 0; i < ncams; ++i) {
        if (!cam_ff(ctx->cams[(size_t)i], bp.cams[0]))
            return fail(ctx, VR_ERR_INVALID_ARG, "camera basis is singular");
        pp.cam = ray_cam(ctx->cams[(size_t)i]);
        pp.out_rgba = reinterpret_cast<float4*>(out_rgba) + (long long)i * img;
        pp.out_max = out_max ? out_max + (long long)i * img : nullptr;
        pp.enc = enc;
        bp.out_enc = enc;
        VR_CK(cudaMemsetAsync(work, 0, sizeof(int), s), "scheduler reset");
        VR_CK(launch_pixel_setup(pp, s), "pixel set-up");
        VR_CK(launch_brick_mip(&ctx->tmap, bp, ctx->dtype, 2 * ctx->num_sms, ctx->cells, s, ctx->tune.group),
              "brick pass");
        VR_CK(launch_mip_finalize(pp, s), "finalise");
    }
    return VR_OK;
}

}  // namespace vr

extern "C" {

vr_status vr_set_path(vr_ctx* ctx, vr_path path) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    if (path != VR_PATH_AUTO && path != VR_PATH_RAY && path != VR_PATH_BRICK && path != VR_PATH_SORTLAST &&
        path != VR_PATH_LAYERED)
        return fail(ctx, VR_ERR_INVALID_ARG, "vr_set_path: unknown path");
    ctx->path = path;
    return VR_OK;
}

}  // extern "C"

namespace {

vr_path resolve_path(const vr_ctx* ctx, vr_mode mode) {
    vr_path path = ctx->path;
    if (path == VR_PATH_AUTO) path = (mode == VR_MIP && ctx->has_tmap) ? VR_PATH_BRICK : VR_PATH_RAY;
    return path;
}

// The launches of one render on stream s (no allocation: scratch is sized first).
vr_status render_dispatch(vr_ctx* ctx, vr_mode mode, float* out_rgba, float* out_max, cudaStream_t s) {
    if (ctx->ooc) return render_ooc(ctx, mode, out_rgba, out_max, s);
    vr_path path = resolve_path(ctx, mode);
    if ((path == VR_PATH_SORTLAST || path == VR_PATH_LAYERED) && mode == VR_COMPOSITE)
        return render_bricks_composite(ctx, out_rgba, s, path == VR_PATH_LAYERED);
    if (path == VR_PATH_SORTLAST || path == VR_PATH_LAYERED) path = VR_PATH_BRICK;  // MIP: order-free
    if (path == VR_PATH_BRICK) {
        if (mode != VR_MIP)
            return fail(ctx, VR_ERR_UNSUPPORTED, "vr_render: the brick path renders VR_MIP only");
        if (!ctx->has_tmap)
            return fail(ctx, VR_ERR_UNSUPPORTED, "vr_render: the brick path needs bricks of at least 32 voxels");
        return render_brick_mip(ctx, out_rgba, out_max, s);
    }
    return render_ray(ctx, mode, out_rgba, out_max, s);
}

vr_status render_checks(vr_ctx* ctx, vr_mode mode, float* out_rgba, float* out_max) {
    if (mode != VR_COMPOSITE && mode != VR_MIP) return fail(ctx, VR_ERR_INVALID_ARG, "vr_render: bad mode");
    if (!out_rgba) return fail(ctx, VR_ERR_INVALID_ARG, "vr_render: out_rgba is NULL");
    if (reinterpret_cast<uintptr_t>(out_rgba) % 16 || reinterpret_cast<uintptr_t>(out_max) % 4)
        return fail(ctx, VR_ERR_INVALID_ARG, "vr_render: out_rgba must be 16-byte aligned, out_max 4-byte");
    if (!ctx->has_cube) return fail(ctx, VR_ERR_STATE, "vr_render: no cube loaded");
    if (!ctx->has_tf) return fail(ctx, VR_ERR_STATE, "vr_render: no transfer function set");
    if (ctx->cams.empty()) return fail(ctx, VR_ERR_STATE, "vr_render: no camera set");
    if (*ctx->status_host != 0) {
        const int code = *ctx->status_host;
        *ctx->status_host = 0;
        return fail(ctx, VR_ERR_INTERNAL,
                    "an earlier device pass stopped: a bounded wait expired or a limit was hit (status " +
                        std::to_string(code) + ")");
    }
    return VR_OK;
}

// Graph mode: capture the render's launches on a private stream, update (or
// instantiate) the cached executable graph, launch it on the caller's stream.
// Camera, table and output changes reach the graph through the update.
vr_status render_graphed(vr_ctx* ctx, vr_mode mode, float* out_rgba, float* out_max, cudaStream_t s) {
    if (resolve_path(ctx, mode) == VR_PATH_BRICK) {
        const long long img = (long long)ctx->cams[0].width * ctx->cams[0].height;
        vr_status st = ensure_pixel_scratch(ctx, img * std::min((int)ctx->cams.size(), kMaxLaunchCams));
        if (st != VR_OK) return st;
    }
    if (!ctx->cap_stream)
        VR_CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking), "vr_render: capture stream");
    // the capture stream must see the caller's earlier work before the graph runs;
    // the graph itself is launched on s, so only the capture is on cap_stream
    cudaEvent_t saved_start = ctx->ev_start, saved_stop = ctx->ev_stop;
    ctx->ev_start = ctx->ev_stop = nullptr;  // profiling events are not recorded in graph mode
    VR_CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal), "vr_render: begin capture");
    vr_status st = render_dispatch(ctx, mode, out_rgba, out_max, ctx->cap_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &graph);
    ctx->ev_start = saved_start;
    ctx->ev_stop = saved_stop;
    if (st != VR_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "vr_render: end capture");
    if (ctx->graph_exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(ctx->graph_exec, graph, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(ctx->graph_exec);
            ctx->graph_exec = nullptr;
        }
    }
    if (!ctx->graph_exec) {
        e = cudaGraphInstantiate(&ctx->graph_exec, graph, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(graph);
            ctx->graph_exec = nullptr;
            return cuda_fail(ctx, e, "vr_render: graph instantiate");
        }
    }
    cudaGraphDestroy(graph);
    VR_CK(cudaGraphLaunch(ctx->graph_exec, s), "vr_render: graph launch");
    return VR_OK;
}

bool tuning_ok(const vr_tuning& t) {
    const bool tile = t.tile_w > 0 && t.tile_h > 0 && t.tile_w * t.tile_h == 32;
    const bool block = t.block == 64 || t.block == 128 || t.block == 256;
    const bool group = t.group == 4 || t.group == 8 || t.group == 16;
    return tile && block && group;
}

}  // namespace

extern "C" {

vr_status vr_render(vr_ctx* ctx, vr_mode mode, float* out_rgba, float* out_max, void* stream) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    vr_status st = render_checks(ctx, mode, out_rgba, out_max);
    if (st != VR_OK) return st;
    DevGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    VR_CK(cudaGetLastError(), "vr_render: pending CUDA error");
    const vr_path path = resolve_path(ctx, mode);
    const bool host_steered = ((path == VR_PATH_SORTLAST || path == VR_PATH_LAYERED) && mode == VR_COMPOSITE) ||
                              ctx->ooc;
    if (ctx->graph_mode && !host_steered) return render_graphed(ctx, mode, out_rgba, out_max, s);
    return render_dispatch(ctx, mode, out_rgba, out_max, s);
}

vr_status vr_set_graph(vr_ctx* ctx, int enable) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    ctx->graph_mode = enable != 0;
    return VR_OK;
}

vr_status vr_get_tuning(const vr_ctx* ctx, vr_tuning* out) {
    if (!ctx || !out) return VR_ERR_INVALID_ARG;
    *out = ctx->tune;
    return VR_OK;
}

vr_status vr_set_tuning(vr_ctx* ctx, const vr_tuning* t) {
    if (!ctx || !t) return VR_ERR_INVALID_ARG;
    if (!tuning_ok(*t))
        return fail(ctx, VR_ERR_INVALID_ARG,
                    "vr_set_tuning: need tile_w * tile_h == 32, block in {64,128,256}, group in {4,8,16}");
    ctx->tune = *t;
    return VR_OK;
}

vr_status vr_autotune(vr_ctx* ctx, vr_mode mode, float* scratch_rgba, int reps, vr_tuning* best,
                      double* best_ms, void* stream) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    if (reps < 1 || reps > 1000) return fail(ctx, VR_ERR_INVALID_ARG, "vr_autotune: reps in [1, 1000]");
    vr_status st = render_checks(ctx, mode, scratch_rgba, nullptr);
    if (st != VR_OK) return st;
    if (ctx->ooc) return fail(ctx, VR_ERR_UNSUPPORTED, "vr_autotune: not for out-of-core cubes");
    DevGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<vr_tuning> cands;
    const vr_tuning base = ctx->tune;
    if (resolve_path(ctx, mode) == VR_PATH_BRICK) {
        for (int grp : {4, 8, 16}) cands.push_back(vr_tuning{base.tile_w, base.tile_h, base.block, grp});
    } else {
        const int tiles[5][2] = {{8, 4}, {4, 8}, {16, 2}, {2, 16}, {32, 1}};
        for (auto& t : tiles)
            for (int blk : {64, 128, 256}) cands.push_back(vr_tuning{t[0], t[1], blk, base.group});
    }
    cudaEvent_t e0, e1;
    VR_CK(cudaEventCreate(&e0), "vr_autotune: event");
    VR_CK(cudaEventCreate(&e1), "vr_autotune: event");
    const bool saved_graph = ctx->graph_mode;
    ctx->graph_mode = false;
    double best_t = 1e300;
    vr_tuning best_c = base;
    for (const vr_tuning& c : cands) {
        ctx->tune = c;
        st = render_dispatch(ctx, mode, scratch_rgba, nullptr, s);  // warm-up
        if (st != VR_OK) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && st == VR_OK; ++r) st = render_dispatch(ctx, mode, scratch_rgba, nullptr, s);
        cudaEventRecord(e1, s);
        if (st != VR_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = cuda_fail(ctx, cudaGetLastError(), "vr_autotune: timing");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms / reps < best_t) {
            best_t = ms / reps;
            best_c = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->graph_mode = saved_graph;
    ctx->tune = (st == VR_OK) ? best_c : base;
    if (st != VR_OK) return st;
    if (best) *best = best_c;
    if (best_ms) *best_ms = best_t;
    return VR_OK;
}

vr_status vr_render_backward(vr_ctx* ctx, vr_mode mode, const float* dL_dimg, float* dL_dtf, float* dL_dvol,
                             void* stream) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    if (mode != VR_COMPOSITE && mode != VR_MIP)
        return fail(ctx, VR_ERR_INVALID_ARG, "vr_render_backward: bad mode");
    if (!dL_dimg || !dL_dtf)
        return fail(ctx, VR_ERR_INVALID_ARG, "vr_render_backward: dL_dimg and dL_dtf are required");
    if (reinterpret_cast<uintptr_t>(dL_dimg) % 16 || reinterpret_cast<uintptr_t>(dL_dtf) % 4 ||
        reinterpret_cast<uintptr_t>(dL_dvol) % 4)
        return fail(ctx, VR_ERR_INVALID_ARG, "vr_render_backward: dL_dimg must be 16-byte aligned");
    if (!ctx->has_cube) return fail(ctx, VR_ERR_STATE, "vr_render_backward: no cube loaded");
    if (ctx->ooc) return fail(ctx, VR_ERR_UNSUPPORTED, "vr_render_backward: not for out-of-core cubes");
    if (!ctx->has_tf) return fail(ctx, VR_ERR_STATE, "vr_render_backward: no transfer function set");
    if (ctx->cams.empty()) return fail(ctx, VR_ERR_STATE, "vr_render_backward: no camera set");
    if (*ctx->status_host != 0) {
        const int code = *ctx->status_host;
        *ctx->status_host = 0;
        return fail(ctx, code == 2 ? VR_ERR_UNSUPPORTED : VR_ERR_INTERNAL,
                    code == 2 ? "an earlier backward pass met a ray with more checkpoint segments than it keeps"
                              : "an earlier device pass stopped on a bounded wait");
    }
    DevGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    VR_CK(cudaGetLastError(), "vr_render_backward: pending CUDA error");
    const int ncams = (int)ctx->cams.size();
    const int nbatch = (ncams + kMaxLaunchCams - 1) / kMaxLaunchCams;
    const int ntf = (int)ctx->tf.size();
    const int grid = ctx->num_sms * adjoint_blocks_per_sm(ctx->dtype, mode, ntf);
    const size_t need = (size_t)nbatch * grid * ntf * 4;
    if (need > ctx->tf_partials_n) {
        if (ctx->tf_partials) cudaFree(ctx->tf_partials);
        ctx->tf_partials = nullptr;
        ctx->tf_partials_n = 0;
        VR_CK(cudaMalloc(&ctx->tf_partials, need * sizeof(float)), "vr_render_backward: partials");
        ctx->tf_partials_n = need;
    }
    if (dL_dvol)
        VR_CK(cudaMemsetAsync(dL_dvol, 0, sizeof(float) * (size_t)ctx->nx * ctx->ny * ctx->nz, s),
              "vr_render_backward: clear dL_dvol");
    VR_CK(cudaMemsetAsync(ctx->work, 0, sizeof(int) * nbatch, s), "vr_render_backward: scheduler reset");
    AdjParams P;
    std::memset(&P, 0, sizeof(P));
    P.vol = vol_dev(ctx);
    P.tf = tf_dev(ctx);
    P.width = ctx->cams[0].width;
    P.height = ctx->cams[0].height;
    P.mode = mode;
    P.tiles_x = (P.width + kTileW - 1) / kTileW;
    P.tiles_y = (P.height + kTileH - 1) / kTileH;
    split(ctx->opt.step, P.step_hi, P.step_lo);
    P.ert = (float)ctx->opt.ert;
    P.dvol = dL_dvol;
    P.status = ctx->status_dev;
    const long long img = (long long)P.width * P.height;
    for (int b = 0; b < nbatch; ++b) {
        const int c0 = b * kMaxLaunchCams;
        P.ncams = std::min(kMaxLaunchCams, ncams - c0);
        for (int i = 0; i < P.ncams; ++i) P.cams[i] = ray_cam(ctx->cams[(size_t)(c0 + i)]);
        P.dimg = reinterpret_cast<const float4*>(dL_dimg) + (long long)c0 * img;
        P.tf_partials = ctx->tf_partials + (size_t)b * grid * ntf * 4;
        P.work = ctx->work + b;
        VR_CK(launch_adjoint(P, ctx->dtype, grid, s), "vr_render_backward: adjoint launch");
    }
    VR_CK(launch_tfgrad_reduce(ctx->tf_partials, nbatch * grid, ntf * 4, dL_dtf, s),
          "vr_render_backward: table reduction");
    return VR_OK;
}

namespace {
int tile_log2(int32_t tile) {
    if (tile == 0) return -1;
    if (tile < 8 || tile > 4096 || (tile & (tile - 1))) return -2;
    int l = 0;
    while ((1 << l) < tile) ++l;
    return l;
}
}  // namespace

vr_status vr_pyramid_layout(int32_t width, int32_t height, int32_t tile, int32_t* levels, int64_t* floats) {
    const int tl = tile_log2(tile);
    if (width <= 0 || height <= 0 || width > (1 << 20) || height > (1 << 20) || tl == -2) return VR_ERR_INVALID_ARG;
    std::vector<int> ws, hs;
    std::vector<long long> offs;
    const long long n = pyramid_levels(width, height, tl, ws, hs, offs);
    if (levels) *levels = (int32_t)ws.size() + 1;
    if (floats) *floats = 4 * n;
    return VR_OK;
}

vr_status vr_image_pyramid(vr_ctx* ctx, const float* rgba, int32_t width, int32_t height, int32_t tile,
                           float* out, void* stream) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    const int tl = tile_log2(tile);
    if (!rgba || !out || width <= 0 || height <= 0 || width > (1 << 20) || height > (1 << 20) || tl == -2)
        return fail(ctx, VR_ERR_INVALID_ARG, "vr_image_pyramid: need images, sizes in [1, 2^20] and tile 0 or a "
                                             "power of two in [8, 4096]");
    if ((reinterpret_cast<uintptr_t>(rgba) | reinterpret_cast<uintptr_t>(out)) & 15)
        return fail(ctx, VR_ERR_INVALID_ARG, "vr_image_pyramid: images must be 16-byte aligned");
    DevGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    VR_CK(launch_pyramid(reinterpret_cast<const float4*>(rgba), width, height, tl, reinterpret_cast<float4*>(out), s),
          "vr_image_pyramid: launch");
    return VR_OK;
}

vr_status vr_overlay_boxes(vr_ctx* ctx, const vr_camera* cams, int32_t ncams, const double* boxes, int64_t nbox,
                           const float* colours, float* rgba, void* stream) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    if (!cams || ncams <= 0 || nbox < 0 || (nbox > 0 && (!boxes || !colours)) || !rgba)
        return fail(ctx, VR_ERR_INVALID_ARG, "vr_overlay_boxes: need cameras, boxes, colours and an image");
    if (nbox > (1LL << 30) || ncams > 4096)
        return fail(ctx, VR_ERR_INVALID_ARG, "vr_overlay_boxes: too many boxes or cameras");
    if (reinterpret_cast<uintptr_t>(rgba) & 15)
        return fail(ctx, VR_ERR_INVALID_ARG, "vr_overlay_boxes: the image must be 16-byte aligned");
    const int W = cams[0].width, H = cams[0].height;
    std::vector<OverlayCam> oc((size_t)ncams);
    for (int i = 0; i < ncams; ++i) {
        const vr_camera& c = cams[i];
        if (c.width != W || c.height != H || W <= 0 || H <= 0 || (c.type != 0 && c.type != 1) ||
            !(c.win[1] != c.win[0]) || !(c.win[3] != c.win[2]))
            return fail(ctx, VR_ERR_INVALID_ARG, "vr_overlay_boxes: cameras need one positive size, a type "
                                                 "and a window of positive extent");
        if (!finite3(c.eye) || !finite3(c.right) || !finite3(c.up) || !finite3(c.fwd) || !finite3(c.win) ||
            !std::isfinite(c.win[3]) || (long long)W * H > (1LL << 30))
            return fail(ctx, VR_ERR_INVALID_ARG, "vr_overlay_boxes: non-finite camera or more than 2^30 pixels");
        OverlayCam& o = oc[(size_t)i];
        std::memset(&o, 0, sizeof(o));
        for (int a = 0; a < 3; ++a) {
            o.eye[a] = c.eye[a];
            o.right[a] = c.right[a];
            o.up[a] = c.up[a];
            o.fwd[a] = c.fwd[a];
        }
        o.l = c.win[0];
        o.r = c.win[1];
        o.b = c.win[2];
        o.t = c.win[3];
        o.type = c.type;
        o.width = W;
        o.height = H;
    }
    for (long long i = 0; i < 6 * nbox; ++i)
        if (!std::isfinite(boxes[i])) return fail(ctx, VR_ERR_INVALID_ARG, "vr_overlay_boxes: non-finite box");
    DevGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long npix = (long long)ncams * W * H;
    if (npix > ctx->ov_key_n) {
        if (ctx->ov_key) cudaFree(ctx->ov_key);
        ctx->ov_key = nullptr;
        ctx->ov_key_n = 0;
        VR_CK(cudaMalloc(&ctx->ov_key, sizeof(int) * (size_t)npix), "vr_overlay_boxes: scratch");
        ctx->ov_key_n = npix;
    }
    // cameras, boxes and colours in one device buffer (each part 256-byte aligned)
    auto up256 = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t cam_b = up256(sizeof(OverlayCam) * (size_t)ncams), box_b = up256(sizeof(double) * 6 * (size_t)nbox);
    const size_t col_b = up256(sizeof(float) * 4 * (size_t)nbox);
    const size_t need = cam_b + box_b + col_b;
    if (need > ctx->ov_in_bytes) {
        if (ctx->ov_in) cudaFree(ctx->ov_in);
        ctx->ov_in = nullptr;
        ctx->ov_in_bytes = 0;
        VR_CK(cudaMalloc(&ctx->ov_in, need), "vr_overlay_boxes: scratch");
        ctx->ov_in_bytes = need;
    }
    char* base = static_cast<char*>(ctx->ov_in);
    VR_CK(cudaMemcpyAsync(base, oc.data(), sizeof(OverlayCam) * (size_t)ncams, cudaMemcpyHostToDevice, s),
          "vr_overlay_boxes: copy cameras");
    if (nbox > 0) {
        VR_CK(cudaMemcpyAsync(base + cam_b, boxes, sizeof(double) * 6 * (size_t)nbox, cudaMemcpyHostToDevice, s),
              "vr_overlay_boxes: copy boxes");
        VR_CK(cudaMemcpyAsync(base + cam_b + box_b, colours, sizeof(float) * 4 * (size_t)nbox, cudaMemcpyHostToDevice,
                              s),
              "vr_overlay_boxes: copy colours");
    }
    VR_CK(launch_overlay(reinterpret_cast<const OverlayCam*>(base), ncams, reinterpret_cast<const double*>(base + cam_b),
                         nbox, reinterpret_cast<const float*>(base + cam_b + box_b), ctx->ov_key, rgba, W, H, s),
          "vr_overlay_boxes: launch");
    return VR_OK;
}

}  // extern "C"

namespace {

// Checks shared by the two distributed sort-last calls.
vr_status dist_checks(vr_ctx* ctx, vr_mode mode, const char* what) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    if (mode != VR_COMPOSITE && mode != VR_MIP) return fail(ctx, VR_ERR_INVALID_ARG, std::string(what) + ": bad mode");
    if (!ctx->has_cube || ctx->ooc) return fail(ctx, VR_ERR_STATE, std::string(what) + ": no in-core cube loaded");
    if (!ctx->has_tf) return fail(ctx, VR_ERR_STATE, std::string(what) + ": no transfer function set");
    if (ctx->cams.size() != 1) return fail(ctx, VR_ERR_STATE, std::string(what) + ": exactly one camera is required");
    return VR_OK;
}

vr_status dist_scratch(vr_ctx* ctx, long long nbricks) {
    if (ctx->dist_ids && nbricks <= ctx->dist_cap) return VR_OK;
    if (ctx->dist_ids) cudaFree(ctx->dist_ids);
    if (ctx->dist_foot) cudaFree(ctx->dist_foot);
    ctx->dist_ids = nullptr;
    ctx->dist_foot = nullptr;
    ctx->dist_cap = 0;
    VR_CK(cudaMalloc(&ctx->dist_ids, sizeof(int) * (size_t)(3 * nbricks + 2)), "sort-last exchange: scratch");
    VR_CK(cudaMalloc(&ctx->dist_foot, sizeof(BrickFoot) * (size_t)nbricks), "sort-last exchange: scratch");
    ctx->dist_cap = nbricks;
    return VR_OK;
}

}  // namespace

extern "C" {

vr_status vr_sortlast_partials(vr_ctx* ctx, vr_mode mode, const int32_t* bricks, int32_t n, vr_footprint* foot,
                               float* partial, int64_t capacity, int64_t* needed, void* stream) {
    vr_status st = dist_checks(ctx, mode, "vr_sortlast_partials");
    if (st != VR_OK) return st;
    DevGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long nbricks = (long long)ctx->nbx * ctx->nby * ctx->nbz;
    if (!needed || n < 0 || n > nbricks || (n > 0 && (!bricks || !foot)))
        return fail(ctx, VR_ERR_INVALID_ARG, "vr_sortlast_partials: bad brick list, foot or needed");
    *needed = 0;
    if (n == 0) return VR_OK;  // a rank that holds no brick renders nothing
    if (reinterpret_cast<uintptr_t>(partial) % 16)
        return fail(ctx, VR_ERR_INVALID_ARG, "vr_sortlast_partials: partial must be 16-byte aligned");
    std::vector<char> seen((size_t)nbricks, 0);
    for (int i = 0; i < n; ++i) {
        if (bricks[i] < 0 || bricks[i] >= nbricks || seen[(size_t)bricks[i]])
            return fail(ctx, VR_ERR_INVALID_ARG, "vr_sortlast_partials: brick id out of range or repeated");
        seen[(size_t)bricks[i]] = 1;
    }
    const CamDev& cd = ctx->cams[0];
    const int W = cd.width, H = cd.height;
    const long long img = (long long)W * H;
    st = ensure_pixel_scratch(ctx, img);
    if (st != VR_OK) return st;
    st = dist_scratch(ctx, nbricks);
    if (st != VR_OK) return st;
    // footprints and keys of every brick (the producer of render_ooc's batches)
    SortParams sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.vol = vol_dev(ctx);
    sp.tf = tf_dev(ctx);
    split(ctx->opt.step, sp.step, sp.step_lo);
    sp.ert = 2.0f;
    sp.mode = mode;
    sp.krange = ctx->krange;
    PixelParams pp;
    std::memset(&pp, 0, sizeof(pp));
    pp.vol = sp.vol;
    pp.tf = sp.tf;
    split(ctx->opt.step, pp.step_hi, pp.step_lo);
    pp.width = W;
    pp.height = H;
    pp.krange = ctx->krange;
    pp.pixdir = ctx->pixdir;
    pp.enc = ctx->enc;
    pp.cam = ray_cam(cd);
    VR_CK(launch_pixel_setup(pp, s), "vr_sortlast_partials: pixel set-up");
    std::vector<int> order, layer_start;
    std::vector<BrickFoot> all;
    st = ooc_footprints(ctx, cd, sp, order, layer_start, all, s);
    if (st != VR_OK) return st;
    if (layer_start.empty() || layer_start.back() == 0)  // no brick visible: nothing was read back
        all.assign((size_t)nbricks, BrickFoot{make_int4(0, 0, -1, -1), 0, 0, 0});
    // packed offsets in list order; the visible listed bricks and their tile prefix
    std::vector<int> sub, tiles(1, 0);
    long long off = 0;
    for (int i = 0; i < n; ++i) {
        BrickFoot& f = all[(size_t)bricks[i]];
        const bool vis = f.rect.z >= f.rect.x && f.rect.w >= f.rect.y;
        vr_footprint& o = foot[i];
        o.brick = bricks[i];
        o.key = f.key;
        o.x0 = vis ? f.rect.x : 0;
        o.y0 = vis ? f.rect.y : 0;
        o.x1 = vis ? f.rect.z : -1;
        o.y1 = vis ? f.rect.w : -1;
        o.offset = off;
        f.offset = off;
        if (vis) {
            off += (long long)(f.rect.z - f.rect.x + 1) * (f.rect.w - f.rect.y + 1);
            sub.push_back(bricks[i]);
            tiles.push_back(tiles.back() + ((f.rect.z - f.rect.x + 1 + 7) / 8) * ((f.rect.w - f.rect.y + 1 + 3) / 4));
        } else {
            f.rect = make_int4(0, 0, -1, -1);
        }
    }
    *needed = off;
    if (!partial) return VR_OK;
    if (capacity < off) return fail(ctx, VR_ERR_INVALID_ARG, "vr_sortlast_partials: capacity below the images' size");
    if (sub.empty()) return VR_OK;
    int* d_sub = ctx->dist_ids;
    int* d_tile = ctx->dist_ids + nbricks;
    VR_CK(cudaMemcpyAsync(sp.foot, all.data(), sizeof(BrickFoot) * (size_t)nbricks, cudaMemcpyHostToDevice, s),
          "vr_sortlast_partials: upload");
    VR_CK(cudaMemcpyAsync(d_sub, sub.data(), sizeof(int) * sub.size(), cudaMemcpyHostToDevice, s),
          "vr_sortlast_partials: upload");
    VR_CK(cudaMemcpyAsync(d_tile, tiles.data(), sizeof(int) * tiles.size(), cudaMemcpyHostToDevice, s),
          "vr_sortlast_partials: upload");
    sp.sub_order = d_sub;
    sp.sub_tile = d_tile;
    sp.sub_n = (int)sub.size();
    sp.partial = reinterpret_cast<float4*>(partial);
    sp.work = ctx->work;
    bool staged = false;
    st = staged_partials(ctx, cd, sp, mode, d_sub, (int)sub.size(), off, s, &staged);
    if (st != VR_OK) return st;
    if (!staged) {
        VR_CK(cudaMemsetAsync(sp.work, 0, sizeof(int), s), "vr_sortlast_partials: scheduler reset");
        VR_CK(launch_brick_partial(sp, ctx->dtype, false, 0, 0, ctx->num_sms * 8, s),
              "vr_sortlast_partials: partials");
    }
    // the host vectors are read by the copies above before the call returns
    VR_CK(cudaStreamSynchronize(s), "vr_sortlast_partials: upload");
    return VR_OK;
}

vr_status vr_sortlast_fold(vr_ctx* ctx, vr_mode mode, const float* partial, int64_t capacity,
                           const vr_footprint* foot, int32_t n, int32_t y0, int32_t y1, float* out_rgba,
                           void* stream) {
    vr_status st = dist_checks(ctx, mode, "vr_sortlast_fold");
    if (st != VR_OK) return st;
    DevGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const CamDev& cd = ctx->cams[0];
    const int W = cd.width, H = cd.height;
    const long long nbricks = (long long)ctx->nbx * ctx->nby * ctx->nbz;
    if (!out_rgba || reinterpret_cast<uintptr_t>(out_rgba) % 16 || reinterpret_cast<uintptr_t>(partial) % 16)
        return fail(ctx, VR_ERR_INVALID_ARG, "vr_sortlast_fold: out_rgba must be given, 16-byte aligned");
    if (y0 < 0 || y1 > H || y0 >= y1) return fail(ctx, VR_ERR_INVALID_ARG, "vr_sortlast_fold: bad rows");
    if (n < 0 || n > nbricks || (n > 0 && (!foot || !partial)))
        return fail(ctx, VR_ERR_INVALID_ARG, "vr_sortlast_fold: bad footprint list");
    st = dist_scratch(ctx, nbricks);
    if (st != VR_OK) return st;
    std::vector<BrickFoot> all((size_t)nbricks, BrickFoot{make_int4(0, 0, -1, -1), 0, 0, 0});
    std::vector<char> seen((size_t)nbricks, 0);
    std::vector<int> order;
    for (int i = 0; i < n; ++i) {
        const vr_footprint& f = foot[i];
        if (f.brick < 0 || f.brick >= nbricks || seen[(size_t)f.brick])
            return fail(ctx, VR_ERR_INVALID_ARG, "vr_sortlast_fold: brick id out of range or repeated");
        seen[(size_t)f.brick] = 1;
        if (f.x1 < f.x0 || f.y1 < f.y0) continue;  // empty: covers no pixel
        if (f.x0 < 0 || f.y0 < 0 || f.x1 >= W || f.y1 >= H || f.offset < 0 ||
            f.offset + (long long)(f.x1 - f.x0 + 1) * (f.y1 - f.y0 + 1) > capacity)
            return fail(ctx, VR_ERR_INVALID_ARG, "vr_sortlast_fold: footprint outside the image or the buffer");
        BrickFoot& b = all[(size_t)f.brick];
        b.rect = make_int4(f.x0, f.y0, f.x1, f.y1);
        b.key = f.key;
        b.offset = f.offset;
        order.push_back(f.brick);
    }
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        return all[(size_t)a].key != all[(size_t)b].key ? all[(size_t)a].key < all[(size_t)b].key : a < b;
    });
    int* d_order = ctx->dist_ids + 2 * nbricks;
    int* d_count = ctx->dist_ids + 3 * nbricks + 1;
    const int cnt = (int)order.size();
    VR_CK(cudaMemcpyAsync(ctx->dist_foot, all.data(), sizeof(BrickFoot) * (size_t)nbricks, cudaMemcpyHostToDevice, s),
          "vr_sortlast_fold: upload");
    if (cnt > 0)
        VR_CK(cudaMemcpyAsync(d_order, order.data(), sizeof(int) * (size_t)cnt, cudaMemcpyHostToDevice, s),
              "vr_sortlast_fold: upload");
    VR_CK(cudaMemcpyAsync(d_count, &cnt, sizeof(int), cudaMemcpyHostToDevice, s), "vr_sortlast_fold: upload");
    SortParams sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.vol = vol_dev(ctx);
    sp.tf = tf_dev(ctx);
    if (!cam_ff(cd, sp.cam)) return fail(ctx, VR_ERR_INVALID_ARG, "vr_sortlast_fold: camera basis is singular");
    sp.mode = mode;
    sp.foot = ctx->dist_foot;
    sp.order = d_order;
    sp.max_layers = 0;
    sp.layer_start = d_count;  // layer_start[max_layers] = the number of ordered partials
    sp.partial = const_cast<float4*>(reinterpret_cast<const float4*>(partial));
    sp.out_rgba = reinterpret_cast<float4*>(out_rgba);
    sp.fold_y0 = y0;
    sp.fold_rows = y1 - y0;
    VR_CK(launch_sortlast_fold(sp, s), "vr_sortlast_fold: fold");
    VR_CK(cudaStreamSynchronize(s), "vr_sortlast_fold: upload");  // host vectors read by the copies
    return VR_OK;
}

const char* vr_last_error(const vr_ctx* ctx) {
    if (!ctx) return "no context";
    return ctx->err.c_str();
}

}  // extern "C"

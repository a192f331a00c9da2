// vr_api.cu -- the C ABI declared in include/vr.h: contexts, volume registry,
// argument checking, device-memory ownership and launch orchestration. Every
// step of the rendering path runs in this library's kernels; this file only
// validates, allocates and enqueues.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "vr_async.cuh"
#include "vr_internal.cuh"

using namespace vr;

namespace {

struct Volume {
    int n[3] = {0, 0, 0};
    int nb[3] = {0, 0, 0};   // skip bricks per axis
    int nsb[3] = {0, 0, 0};  // storage bricks (8^3 cells) per axis
    int bs = 3;              // log2 of the cells per skip-brick edge
    float s[3] = {1, 1, 1};
    long long nvox = 0, nbricks = 0, nsbricks = 0;  // voxels, skip bricks, storage bricks
    float* d_norm = nullptr;
    float* d_bricks = nullptr;
    uint16_t* d_grid = nullptr;
    uint8_t* d_empty = nullptr;
    VolConst* d_vc = nullptr;
    float* d_minmax = nullptr;
    float* d_vessel = nullptr;
    float* d_vbricks = nullptr;
    float* d_dbricks = nullptr;  // derived bricks (voxel-wise I, gradient, Hessian) or nullptr
    uint16_t* d_cellq = nullptr;     // after the morphology precompute: per-cell quantised min/max
    uint32_t* d_cellmask = nullptr;  // and per-cell empty bits under the current transfer function
    float* d_smax = nullptr;  // per-scale max Hessian norm (8 floats)
    float* d_ch2 = nullptr;   // second channel: [0, 2) its I_min, I_max, [4, 8) its VolConst
    bool v_ready = false;     // d_vessel holds a complete second channel (vesselness or a modality)
    float* d_tf = nullptr;
    size_t tf_cap = 0;
    int* d_prefix = nullptr;
    int prefix_cap = 0;
    TissueDev tp{};
    bool morph_ready = false, params_ready = false;
};

struct Batch {
    std::vector<vr_view> views;
    std::vector<ViewDev> table;
    ViewDev* d_views = nullptr;
    int* d_prefix = nullptr;        // 4 packet shapes x n_views
    int n_work[4] = {0, 0, 0, 0};   // packets per packet shape (packet_w = 4, 8, 16, 32)
    bool all_derived = false;       // every view's volume has derived bricks
    int bs = 3;                     // the skip-brick size all views share, 0 when they differ
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;  // (packet_w, warps) -> graph
};

}  // namespace

struct vr_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    std::map<int, Volume*> vols;
    int next_id = 1;
    float* d_partials = nullptr;
    int partials_cap = 0;
    void* d_stage = nullptr;
    size_t stage_cap = 0;
    float* d_scratch = nullptr;   // vesselness scratch (smoothed volume + smoothing pass), prefilter
    size_t scratch_cap = 0;
    float* d_tfgrad = nullptr;    // private copies of a 2D transfer-function gradient
    size_t tfgrad_cap = 0;
    float* d_dgrad = nullptr;     // per-voxel derived-channel gradients (backward on derived bricks)
    size_t dgrad_cap = 0;
    unsigned* d_work = nullptr;   // [0]: staged-kernel work counter, [1]: status word
    int staged_ctas[2][17] = {};   // resident CTAs per SM by (vesselness, warps per block)
    int batch_ctas[2][17] = {};    // resident batch-kernel CTAs per SM by (all derived, warps per block)
    size_t derived_budget = kDerivedBudgetBytes;  // largest derived-brick store precompute builds
    std::map<int, Batch*> batches;
    int next_batch = 1;
    cudaStream_t graph_stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::unordered_map<void*, size_t> allocs;  // device buffers held, with their sizes
    size_t mem_used = 0;                       // sum of allocs
    size_t mem_limit = 0;                      // 0: no limit beyond the device's
    long long fail_after = -1;                 // >= 0: allocations left before an injected failure
};

namespace {

vr_status fail(vr_ctx* c, vr_status s, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
vr_status fail(vr_ctx* c, vr_status s, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

vr_status cuda_fail(vr_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return VR_OK;
    (void)cudaGetLastError();
    return fail(c, e == cudaErrorMemoryAllocation ? VR_ERR_OOM : VR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

// Every device buffer of a context is allocated and freed here, so that the context
// knows what it holds (vr_memory_used), can refuse to grow past a limit
// (vr_set_memory_limit) and can be made to see an allocation fail (vr_debug_fail_alloc).
// A refused allocation returns cudaErrorMemoryAllocation like a failed cudaMalloc.
template <class T>
cudaError_t dalloc(vr_ctx* ctx, T** p, size_t bytes) {
    *p = nullptr;
    if (ctx->fail_after == 0) {
        ctx->fail_after = -1;  // one injected failure, then allocation behaves normally
        return cudaErrorMemoryAllocation;
    }
    if (ctx->fail_after > 0) --ctx->fail_after;
    if (ctx->mem_limit && bytes > ctx->mem_limit - std::min(ctx->mem_limit, ctx->mem_used))
        return cudaErrorMemoryAllocation;
    void* q = nullptr;
    const cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) return e;
    ctx->allocs[q] = bytes;
    ctx->mem_used += bytes;
    *p = static_cast<T*>(q);
    return cudaSuccess;
}

void dfree(vr_ctx* ctx, void* p) {
    if (!p) return;
    auto it = ctx->allocs.find(p);
    if (it != ctx->allocs.end()) {
        ctx->mem_used -= it->second;
        ctx->allocs.erase(it);
    }
    cudaFree(p);
}

void free_volume(vr_ctx* ctx, Volume* v) {
    dfree(ctx, v->d_norm);
    dfree(ctx, v->d_bricks);
    dfree(ctx, v->d_grid);
    dfree(ctx, v->d_empty);
    dfree(ctx, v->d_vc);
    dfree(ctx, v->d_minmax);
    dfree(ctx, v->d_vessel);
    dfree(ctx, v->d_vbricks);
    dfree(ctx, v->d_dbricks);
    dfree(ctx, v->d_cellq);
    dfree(ctx, v->d_cellmask);
    dfree(ctx, v->d_smax);
    dfree(ctx, v->d_ch2);
    dfree(ctx, v->d_tf);
    dfree(ctx, v->d_prefix);
    delete v;
}

Volume* get_vol(vr_ctx* ctx, int id) {
    auto it = ctx->vols.find(id);
    return it == ctx->vols.end() ? nullptr : it->second;
}

cudaError_t ensure_stage(vr_ctx* ctx, size_t bytes) {
    if (ctx->stage_cap >= bytes) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return e;
    dfree(ctx, ctx->d_stage);
    ctx->d_stage = nullptr;
    ctx->stage_cap = 0;
    e = dalloc(ctx, &ctx->d_stage, bytes);
    if (e == cudaSuccess) ctx->stage_cap = bytes;
    return e;
}

// An NVTX range around each public call that enqueues GPU work, so that a trace
// (Nsight Systems or Compute) shows which library call launched each kernel.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Device address of caller data: the data itself (on_device), or a copy of the host
// data in the context's staging buffer, enqueued on the context's stream.
cudaError_t device_input(vr_ctx* ctx, const void* data, int on_device, size_t bytes, const void** raw) {
    *raw = data;
    if (on_device) return cudaSuccess;
    cudaError_t e = ensure_stage(ctx, bytes);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->d_stage, data, bytes, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) *raw = ctx->d_stage;
    return e;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool finite_pos(float x) { return isfinite(x) && x > 0.0f; }

void fill_launch(RenderLaunch& L, const Volume* v, int W, int H, int skip) {
    memset(&L, 0, sizeof L);
    for (int a = 0; a < 3; ++a) {
        L.vol.n[a] = v->n[a];
        L.vol.nb[a] = v->nb[a];
        L.vol.nsb[a] = v->nsb[a];
        L.vol.s[a] = v->s[a];
    }
    L.vol.bs = v->bs;
    L.vol.der_stride = (int)der_brick_floats(v->bs);
    L.vol.bricks = v->d_bricks;
    L.vol.vbricks = (v->tp.tf_mode == 2) ? v->d_vbricks : nullptr;
    L.vol.dbricks = v->d_dbricks;
    L.vol.cellmask = v->d_cellmask;
    L.vol.empty = v->d_empty;
    L.vol.vc = v->d_vc;
    L.tp = v->tp;
    L.tf = v->d_tf;
    L.W = W, L.H = H;
    L.skip = skip ? 1 : 0;
    L.rc = make_ray_consts(W, H, v->s, v->tp.step_vox);
}

vr_status rebuild_bricks(vr_ctx* ctx, Volume* v) {
    CK(launch_make_bricks(v->d_norm, v->n, v->nsb, v->d_bricks, ctx->stream), "bricking");
    CK(launch_brick_minmax(v->d_norm, v->n, v->nb, v->bs, v->d_grid, ctx->stream), "brick min/max");
    if (v->d_dbricks)
        CK(launch_make_derived(v->d_norm, v->n, v->nb, v->bs, v->s, v->d_dbricks, ctx->stream), "derived bricks");
    if (v->d_cellq) CK(launch_cell_minmax(v->d_norm, v->n, v->nb, v->bs, v->d_cellq, ctx->stream), "cell min/max");
    return VR_OK;
}

// Brick skip flags and (once the morphology is precomputed) the per-cell empty bits
// under the volume's current transfer function.
vr_status classify_volume(vr_ctx* ctx, Volume* v) {
    CK(launch_classify(v->d_grid, v->nbricks, v->d_tf, v->tp.tf_w, v->tp.tf_h, v->d_empty, v->d_prefix, ctx->stream),
       "classify");
    if (v->d_cellmask)
        CK(launch_classify_cells(v->d_cellq, v->nbricks, v->bs, v->d_prefix, v->tp.tf_w, v->d_cellmask, ctx->stream),
           "classify cells");
    return VR_OK;
}

}  // namespace

vr_status vr::set_error(vr_ctx* ctx, vr_status status, const char* msg) {
    if (ctx) ctx->err = msg ? msg : "";
    return status;
}

extern "C" {

const char* vr_version(void) { return "vr 1.0 sm_103a"; }

vr_status vr_create(vr_ctx** out, int device, void* cuda_stream) {
    if (!out) return VR_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        (void)cudaGetLastError();
        return VR_ERR_CUDA;
    }
    if (device < 0 || device >= ndev) return VR_ERR_INVALID_ARG;
    vr_ctx* ctx = new vr_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    DeviceGuard g(device);
    cudaError_t e = dalloc(ctx, &ctx->d_work, 64 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_work, 0, 64 * sizeof(unsigned));
    if (e != cudaSuccess) {
        dfree(ctx, ctx->d_work);
        delete ctx;
        (void)cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? VR_ERR_OOM : VR_ERR_CUDA;
    }
    *out = ctx;
    return VR_OK;
}

vr_status vr_destroy(vr_ctx* ctx) {
    if (!ctx) return VR_OK;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto& kv : ctx->batches) {
        for (auto& g : kv.second->graphs) cudaGraphExecDestroy(g.second);
        dfree(ctx, kv.second->d_views);
        dfree(ctx, kv.second->d_prefix);
        delete kv.second;
    }
    for (auto& kv : ctx->vols) free_volume(ctx, kv.second);
    if (ctx->graph_stream) cudaStreamDestroy(ctx->graph_stream);
    if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
    if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
    dfree(ctx, ctx->d_partials);
    dfree(ctx, ctx->d_stage);
    dfree(ctx, ctx->d_scratch);
    dfree(ctx, ctx->d_tfgrad);
    dfree(ctx, ctx->d_dgrad);
    dfree(ctx, ctx->d_work);
    (void)cudaGetLastError();
    delete ctx;
    return VR_OK;
}

vr_status vr_set_stream(vr_ctx* ctx, void* cuda_stream) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    ctx->stream = (cudaStream_t)cuda_stream;
    return VR_OK;
}

vr_status vr_synchronize(vr_ctx* ctx) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    CK(cudaStreamSynchronize(ctx->stream), "stream synchronize");
    CK(cudaGetLastError(), "asynchronous error");
    unsigned status[2] = {0, 0};  // status bits, source line of the first failed index check
    CK(cudaMemcpy(status, ctx->d_work + 1, sizeof status, cudaMemcpyDeviceToHost), "status word");
    if (status[0] || status[1]) {
        CK(cudaMemset(ctx->d_work + 1, 0, sizeof status), "status word reset");
        if (status[0] & kStatusTimeout)
            return fail(ctx, VR_ERR_TIMEOUT, "a bounded device-side wait expired (bulk copy did not complete)");
        if (status[0] & kStatusBounds)
            return fail(ctx, VR_ERR_BOUNDS, "debug build: an index check failed at line %u of a kernel source",
                        status[1]);
    }
    return VR_OK;
}

const char* vr_last_error(vr_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

vr_status vr_reduce_minmax(vr_ctx* ctx, const void* d_data, vr_dtype dtype, long long n, float* d_out2) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    if (!d_data || !d_out2 || n < 1) return fail(ctx, VR_ERR_INVALID_ARG, "reduce_minmax: bad arguments");
    if (dtype != VR_F32 && dtype != VR_U16) return fail(ctx, VR_ERR_INVALID_ARG, "reduce_minmax: bad dtype");
    DeviceGuard g(ctx->device);
    const int nblocks = minmax_blocks(n);
    if (ctx->partials_cap < nblocks) {
        CK(cudaStreamSynchronize(ctx->stream), "reduce_minmax sync");
        dfree(ctx, ctx->d_partials);
        ctx->d_partials = nullptr;
        ctx->partials_cap = 0;
        CK(dalloc(ctx, &ctx->d_partials, sizeof(float) * 2 * nblocks), "reduce_minmax scratch");
        ctx->partials_cap = nblocks;
    }
    CK(launch_minmax_partials(d_data, dtype, n, ctx->d_partials, nblocks, ctx->stream), "minmax partials");
    CK(launch_minmax_final(ctx->d_partials, nblocks, d_out2, ctx->stream), "minmax final");
    return VR_OK;
}

vr_status vr_load_volume(vr_ctx* ctx, const void* data, int on_device, vr_dtype dtype, int nx, int ny, int nz,
                         float sx, float sy, float sz, int* vol_id) {
    NvtxRange range_("vr_load_volume");
    if (!ctx) return VR_ERR_INVALID_ARG;
    if (!data || !vol_id) return fail(ctx, VR_ERR_INVALID_ARG, "load_volume: NULL pointer");
    if (dtype != VR_F32 && dtype != VR_U16) return fail(ctx, VR_ERR_INVALID_ARG, "load_volume: bad dtype");
    if (nx < 2 || ny < 2 || nz < 2 || nx > 2048 || ny > 2048 || nz > 2048)
        return fail(ctx, VR_ERR_INVALID_ARG, "load_volume: dims %d x %d x %d outside [2, 2048]", nx, ny, nz);
    if (!finite_pos(sx) || !finite_pos(sy) || !finite_pos(sz))
        return fail(ctx, VR_ERR_INVALID_ARG, "load_volume: spacing must be finite and > 0");
    DeviceGuard g(ctx->device);
    Volume* v = new Volume();
    v->n[0] = nx, v->n[1] = ny, v->n[2] = nz;
    v->s[0] = sx, v->s[1] = sy, v->s[2] = sz;
    for (int a = 0; a < 3; ++a) {
        v->nb[a] = (v->n[a] - 1 + (1 << v->bs) - 1) >> v->bs;
        v->nsb[a] = (v->n[a] - 1 + kCells - 1) / kCells;
    }
    v->nvox = (long long)nx * ny * nz;
    v->nbricks = (long long)v->nb[0] * v->nb[1] * v->nb[2];
    v->nsbricks = (long long)v->nsb[0] * v->nsb[1] * v->nsb[2];
    const size_t esz = dtype == VR_F32 ? 4 : 2;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = dalloc(ctx, &v->d_norm, sizeof(float) * v->nvox);
    if (e == cudaSuccess) e = dalloc(ctx, &v->d_bricks, (size_t)kBrickBytes * v->nsbricks);
    if (e == cudaSuccess) e = dalloc(ctx, &v->d_grid, sizeof(uint16_t) * 2 * v->nbricks);
    if (e == cudaSuccess) e = dalloc(ctx, &v->d_empty, v->nbricks);
    if (e == cudaSuccess) e = dalloc(ctx, &v->d_vc, sizeof(VolConst));
    if (e == cudaSuccess) e = dalloc(ctx, &v->d_minmax, 2 * sizeof(float));
    if (e == cudaSuccess) e = cudaMemsetAsync(v->d_vc, 0, sizeof(VolConst), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(v->d_empty, 0, v->nbricks, ctx->stream);
    const void* raw = data;
    if (e == cudaSuccess) e = device_input(ctx, data, on_device, esz * v->nvox, &raw);
    if (e != cudaSuccess) {
        free_volume(ctx, v);
        return cuda_fail(ctx, e, "load_volume: allocate/copy");
    }
    vr_status st = vr_reduce_minmax(ctx, raw, dtype, v->nvox, v->d_minmax);
    if (st == VR_OK) {
        e = launch_normalize(raw, dtype, v->nvox, v->d_minmax, v->d_vc, v->d_norm, ctx->stream);
        st = cuda_fail(ctx, e, "normalize");
    }
    if (st == VR_OK) st = rebuild_bricks(ctx, v);
    float mm[2] = {0, 0};
    if (st == VR_OK) {
        e = cudaMemcpyAsync(mm, v->d_minmax, sizeof mm, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        st = cuda_fail(ctx, e, "load_volume: read back I_min/I_max");
    }
    if (st == VR_OK && !(mm[1] > mm[0])) {
        st = fail(ctx, VR_ERR_DEGENERATE, "load_volume: I_max == I_min (%g); Eq. 1 undefined", (double)mm[0]);
    }
    if (st == VR_OK && !(isfinite(mm[0]) && isfinite(mm[1])))
        st = fail(ctx, VR_ERR_INVALID_ARG, "load_volume: non-finite intensities");
    if (st != VR_OK) {
        cudaStreamSynchronize(ctx->stream);
        free_volume(ctx, v);
        return st;
    }
    const int id = ctx->next_id++;
    ctx->vols[id] = v;
    *vol_id = id;
    return VR_OK;
}

vr_status vr_free_volume(vr_ctx* ctx, int vol_id) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    Volume* v = get_vol(ctx, vol_id);
    if (!v) return fail(ctx, VR_ERR_INVALID_ARG, "free_volume: unknown id %d", vol_id);
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    free_volume(ctx, v);
    ctx->vols.erase(vol_id);
    return VR_OK;
}

vr_status vr_precompute_morphology(vr_ctx* ctx, int vol_id, const float* h_sigmas, int n_sigmas) {
    NvtxRange range_("vr_precompute_morphology");
    if (!ctx) return VR_ERR_INVALID_ARG;
    Volume* v = get_vol(ctx, vol_id);
    if (!v) return fail(ctx, VR_ERR_INVALID_ARG, "precompute_morphology: unknown id %d", vol_id);
    if (n_sigmas < 0 || n_sigmas > 8 || (n_sigmas > 0 && !h_sigmas))
        return fail(ctx, VR_ERR_INVALID_ARG, "precompute_morphology: bad sigma list");
    for (int i = 0; i < n_sigmas; ++i)
        if (!(h_sigmas[i] > 0.0f && h_sigmas[i] <= 8.0f))
            return fail(ctx, VR_ERR_INVALID_ARG, "precompute_morphology: sigma %g outside (0, 8]", (double)h_sigmas[i]);
    DeviceGuard g(ctx->device);
    v->morph_ready = false;  // until every step below has been issued
    CK(launch_gmax(v->d_norm, v->n, v->s, v->d_vc, ctx->stream), "gmax");
    // voxel-wise derivatives for the raymarch (Sec. 2.3), within a memory budget
    const size_t dbytes = sizeof(float) * (size_t)der_brick_floats(v->bs) * v->nbricks;
    if (v->d_dbricks && dbytes > ctx->derived_budget) {
        CK(cudaStreamSynchronize(ctx->stream), "precompute_morphology: sync");
        dfree(ctx, v->d_dbricks);
        v->d_dbricks = nullptr;
    }
    if (!v->d_dbricks && dbytes <= ctx->derived_budget) {
        cudaError_t e = dalloc(ctx, &v->d_dbricks, dbytes);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            v->d_dbricks = nullptr;  // fall back to the per-sample stencils
        }
    }
    // per-cell min/max (4 B per cell) and per-cell empty bits, for either path
    if (!v->d_cellq)
        CK(dalloc(ctx, &v->d_cellq, (sizeof(uint16_t) * 2 * (size_t)v->nbricks) << (3 * v->bs)), "cell grid");
    if (!v->d_cellmask)
        CK(dalloc(ctx, &v->d_cellmask, sizeof(uint32_t) * (size_t)cell_words(v->bs) * v->nbricks), "cell flags");
    if (v->d_dbricks)
        CK(launch_make_derived(v->d_norm, v->n, v->nb, v->bs, v->s, v->d_dbricks, ctx->stream), "derived bricks");
    CK(launch_cell_minmax(v->d_norm, v->n, v->nb, v->bs, v->d_cellq, ctx->stream), "cell min/max");
    if (v->params_ready) {
        vr_status cs = classify_volume(ctx, v);
        if (cs != VR_OK) return cs;
    }
    if (n_sigmas > 0) {
        v->v_ready = false;
        if (v->params_ready && v->tp.tf_mode == 2) v->params_ready = false;  // its V channel is being replaced
        if (!v->d_vessel) CK(dalloc(ctx, &v->d_vessel, sizeof(float) * v->nvox), "vesselness volume");
        if (!v->d_vbricks) CK(dalloc(ctx, &v->d_vbricks, (size_t)kBrickBytes * v->nsbricks), "vesselness bricks");
        if (!v->d_smax) CK(dalloc(ctx, &v->d_smax, sizeof(float) * 8), "vesselness scale maxima");
        const size_t need = sizeof(float) * 2 * (size_t)v->nvox;  // smoothed volume + smoothing pass
        if (ctx->scratch_cap < need) {
            CK(cudaStreamSynchronize(ctx->stream), "vesselness scratch sync");
            dfree(ctx, ctx->d_scratch);
            ctx->d_scratch = nullptr;
            ctx->scratch_cap = 0;
            CK(dalloc(ctx, &ctx->d_scratch, need), "vesselness scratch");
            ctx->scratch_cap = need;
        }
        CK(launch_frangi(v->d_norm, v->n, h_sigmas, n_sigmas, ctx->d_scratch, ctx->d_scratch + v->nvox, v->d_smax,
                         v->d_vessel, ctx->stream),
           "vesselness");
        CK(launch_make_bricks(v->d_vessel, v->n, v->nsb, v->d_vbricks, ctx->stream), "vesselness bricks");
        v->v_ready = true;
    }
    v->morph_ready = true;
    return VR_OK;
}

vr_status vr_set_tissue_params(vr_ctx* ctx, int vol_id, const vr_tissue_params* tp) {
    NvtxRange range_("vr_set_tissue_params");
    if (!ctx) return VR_ERR_INVALID_ARG;
    Volume* v = get_vol(ctx, vol_id);
    if (!v) return fail(ctx, VR_ERR_INVALID_ARG, "set_tissue_params: unknown id %d", vol_id);
    if (!tp || !tp->tf) return fail(ctx, VR_ERR_INVALID_ARG, "set_tissue_params: NULL pointer");
    if (tp->tf_mode < 0 || tp->tf_mode > 2) return fail(ctx, VR_ERR_INVALID_ARG, "set_tissue_params: bad tf_mode");
    if (tp->tf_w < 2 || tp->tf_w > 4096) return fail(ctx, VR_ERR_INVALID_ARG, "set_tissue_params: tf_w outside [2, 4096]");
    if (tp->tf_mode == 0 ? tp->tf_h != 1 : (tp->tf_h < 2 || tp->tf_h > 256))
        return fail(ctx, VR_ERR_INVALID_ARG, "set_tissue_params: tf_h %d invalid for mode %d", tp->tf_h, tp->tf_mode);
    if (tp->tf_mode == 2 && !v->v_ready)
        return fail(ctx, VR_ERR_NOT_READY,
                    "set_tissue_params: mode 2 needs precomputed vesselness or a second channel");
    if (!finite_pos(tp->kappa_ref) || !(tp->w_max >= 0.0f) || !isfinite(tp->gamma) || !finite_pos(tp->step_vox) ||
        !(tp->opacity_scale >= 0.0f) || !isfinite(tp->opacity_scale) || !isfinite(tp->et_threshold) ||
        !isfinite(tp->ka) || !isfinite(tp->kd) || !isfinite(tp->ks))
        return fail(ctx, VR_ERR_INVALID_ARG, "set_tissue_params: bad scalar parameter");
    if (!(tp->opacity_ref_step >= 0.0f) || !isfinite(tp->opacity_ref_step))
        return fail(ctx, VR_ERR_INVALID_ARG, "set_tissue_params: opacity_ref_step must be finite and >= 0");
    if (!(tp->step_vox >= 0.01f && tp->step_vox <= 16.0f))
        return fail(ctx, VR_ERR_INVALID_ARG, "set_tissue_params: step_vox %g outside [0.01, 16]", (double)tp->step_vox);
    if ((tp->grad_mod != 0 && tp->grad_mod != 1) || (tp->shading != 0 && tp->shading != 1))
        return fail(ctx, VR_ERR_INVALID_ARG, "set_tissue_params: grad_mod/shading must be 0 or 1");
    DeviceGuard g(ctx->device);
    v->params_ready = false;  // until the table is uploaded and the volume re-classified
    const size_t bytes = sizeof(float) * 4 * (size_t)tp->tf_w * tp->tf_h;
    if (v->tf_cap < bytes) {
        CK(cudaStreamSynchronize(ctx->stream), "set_tissue_params sync");
        dfree(ctx, v->d_tf);
        v->d_tf = nullptr;
        v->tf_cap = 0;
        CK(dalloc(ctx, &v->d_tf, bytes), "transfer function");
        v->tf_cap = bytes;
    }
    if (v->prefix_cap < tp->tf_w + 1) {
        CK(cudaStreamSynchronize(ctx->stream), "set_tissue_params sync");
        dfree(ctx, v->d_prefix);
        v->d_prefix = nullptr;
        v->prefix_cap = 0;
        CK(dalloc(ctx, &v->d_prefix, sizeof(int) * (tp->tf_w + 1)), "classification scratch");
        v->prefix_cap = tp->tf_w + 1;
    }
    CK(cudaMemcpyAsync(v->d_tf, tp->tf, bytes, tp->tf_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       ctx->stream),
       "transfer function copy");
    TissueDev& d = v->tp;
    d.tf_mode = tp->tf_mode, d.tf_w = tp->tf_w, d.tf_h = tp->tf_h;
    d.grad_mod = tp->grad_mod, d.shading = tp->shading;
    d.gamma = tp->gamma, d.kappa_ref = tp->kappa_ref, d.w_max = tp->w_max;
    d.gk = (float)((double)tp->gamma / (double)tp->kappa_ref);
    d.inv_kref = (float)(1.0 / (double)tp->kappa_ref);
    d.ka = tp->ka, d.kd = tp->kd, d.ks = tp->ks;
    d.status = ctx->d_work + 1;
    d.opacity_scale = tp->opacity_scale, d.et_threshold = tp->et_threshold, d.step_vox = tp->step_vox;
    {
        const double smin = fmin((double)v->s[0], fmin((double)v->s[1], (double)v->s[2]));
        d.alpha_exp = tp->opacity_ref_step > 0.0f ? (float)((double)tp->step_vox * smin / (double)tp->opacity_ref_step)
                                                  : 0.0f;
    }
    vr_status cs = classify_volume(ctx, v);
    if (cs != VR_OK) return cs;
    v->params_ready = true;
    return VR_OK;
}

vr_status vr_get_norm(vr_ctx* ctx, int vol_id, float* imin, float* imax, float* gmax) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    Volume* v = get_vol(ctx, vol_id);
    if (!v) return fail(ctx, VR_ERR_INVALID_ARG, "get_norm: unknown id %d", vol_id);
    DeviceGuard g(ctx->device);
    VolConst vc;
    CK(cudaMemcpyAsync(&vc, v->d_vc, sizeof vc, cudaMemcpyDeviceToHost, ctx->stream), "get_norm copy");
    CK(cudaStreamSynchronize(ctx->stream), "get_norm sync");
    if (imin) *imin = vc.imin;
    if (imax) *imax = vc.imax;
    if (gmax) *gmax = vc.gmax;
    return VR_OK;
}

vr_status vr_set_gmax(vr_ctx* ctx, int vol_id, float gmax) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    Volume* v = get_vol(ctx, vol_id);
    if (!v) return fail(ctx, VR_ERR_INVALID_ARG, "set_gmax: unknown id %d", vol_id);
    if (!finite_pos(gmax)) return fail(ctx, VR_ERR_INVALID_ARG, "set_gmax: must be finite and > 0");
    DeviceGuard g(ctx->device);
    static_assert(sizeof(float) == 4, "float");
    // A host value copied on the stream: stage it through a pageable copy (synchronous for the host).
    CK(cudaMemcpyAsync(&v->d_vc->gmax, &gmax, sizeof(float), cudaMemcpyHostToDevice, ctx->stream), "set_gmax copy");
    CK(cudaStreamSynchronize(ctx->stream), "set_gmax sync");
    v->morph_ready = true;
    return VR_OK;
}

vr_status vr_set_normalized(vr_ctx* ctx, int vol_id, const float* d_norm) {
    NvtxRange range_("vr_set_normalized");
    if (!ctx) return VR_ERR_INVALID_ARG;
    Volume* v = get_vol(ctx, vol_id);
    if (!v || !d_norm) return fail(ctx, VR_ERR_INVALID_ARG, "set_normalized: bad arguments");
    DeviceGuard g(ctx->device);
    CK(cudaMemcpyAsync(v->d_norm, d_norm, sizeof(float) * v->nvox, cudaMemcpyDeviceToDevice, ctx->stream),
       "set_normalized copy");
    vr_status st = rebuild_bricks(ctx, v);
    if (st != VR_OK) return st;
    if (v->params_ready) return classify_volume(ctx, v);
    return VR_OK;
}

vr_status vr_load_second_channel(vr_ctx* ctx, int vol_id, const void* data, int on_device, vr_dtype dtype) {
    NvtxRange range_("vr_load_second_channel");
    if (!ctx) return VR_ERR_INVALID_ARG;
    Volume* v = get_vol(ctx, vol_id);
    if (!v) return fail(ctx, VR_ERR_INVALID_ARG, "load_second_channel: unknown id %d", vol_id);
    if (!data) return fail(ctx, VR_ERR_INVALID_ARG, "load_second_channel: NULL pointer");
    if (dtype != VR_F32 && dtype != VR_U16) return fail(ctx, VR_ERR_INVALID_ARG, "load_second_channel: bad dtype");
    DeviceGuard g(ctx->device);
    // until the channel is complete, neither it nor tissue params that render over it are usable
    v->v_ready = false;
    if (v->params_ready && v->tp.tf_mode == 2) v->params_ready = false;
    if (!v->d_vessel) CK(dalloc(ctx, &v->d_vessel, sizeof(float) * v->nvox), "load_second_channel: channel volume");
    if (!v->d_vbricks) CK(dalloc(ctx, &v->d_vbricks, (size_t)kBrickBytes * v->nsbricks), "load_second_channel: bricks");
    if (!v->d_ch2) CK(dalloc(ctx, &v->d_ch2, sizeof(float) * 8), "load_second_channel: normalisation constants");
    const size_t esz = dtype == VR_F32 ? 4 : 2;
    const void* raw = data;
    CK(device_input(ctx, data, on_device, esz * v->nvox, &raw), "load_second_channel: copy");
    // Eq. 1 applied to the channel itself: its own I_min, I_max
    vr_status st = vr_reduce_minmax(ctx, raw, dtype, v->nvox, v->d_ch2);
    if (st != VR_OK) return st;
    CK(launch_normalize(raw, dtype, v->nvox, v->d_ch2, reinterpret_cast<VolConst*>(v->d_ch2 + 4), v->d_vessel,
                        ctx->stream),
       "load_second_channel: normalise");
    CK(launch_make_bricks(v->d_vessel, v->n, v->nsb, v->d_vbricks, ctx->stream), "load_second_channel: bricking");
    float mm[2] = {0, 0};
    CK(cudaMemcpyAsync(mm, v->d_ch2, sizeof mm, cudaMemcpyDeviceToHost, ctx->stream), "load_second_channel: read back");
    CK(cudaStreamSynchronize(ctx->stream), "load_second_channel: sync");
    if (!(isfinite(mm[0]) && isfinite(mm[1])))
        return fail(ctx, VR_ERR_INVALID_ARG, "load_second_channel: non-finite intensities");
    if (!(mm[1] > mm[0]))
        return fail(ctx, VR_ERR_DEGENERATE, "load_second_channel: I_max == I_min (%g); Eq. 1 undefined", (double)mm[0]);
    v->v_ready = true;
    return VR_OK;
}

vr_status vr_get_bricks(vr_ctx* ctx, int vol_id, unsigned short* h_grid, unsigned char* h_empty, int* h_nb) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    Volume* v = get_vol(ctx, vol_id);
    if (!v) return fail(ctx, VR_ERR_INVALID_ARG, "get_bricks: unknown id %d", vol_id);
    DeviceGuard g(ctx->device);
    if (h_grid)
        CK(cudaMemcpyAsync(h_grid, v->d_grid, sizeof(uint16_t) * 2 * v->nbricks, cudaMemcpyDeviceToHost, ctx->stream),
           "get_bricks grid");
    if (h_empty) CK(cudaMemcpyAsync(h_empty, v->d_empty, v->nbricks, cudaMemcpyDeviceToHost, ctx->stream), "get_bricks flags");
    CK(cudaStreamSynchronize(ctx->stream), "get_bricks sync");
    if (h_nb)
        for (int a = 0; a < 3; ++a) h_nb[a] = v->nb[a];
    return VR_OK;
}

vr_status vr_get_layout(vr_ctx* ctx, int vol_id, long long* nbricks, unsigned long long* brick_bytes,
                        unsigned long long* derived_bytes) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    Volume* v = get_vol(ctx, vol_id);
    if (!v) return fail(ctx, VR_ERR_INVALID_ARG, "get_layout: unknown id %d", vol_id);
    if (nbricks) *nbricks = v->nbricks;
    if (brick_bytes) *brick_bytes = (unsigned long long)kBrickBytes * (unsigned long long)v->nsbricks;
    if (derived_bytes)
        *derived_bytes = v->d_dbricks ? sizeof(float) * (unsigned long long)der_brick_floats(v->bs) * v->nbricks : 0ull;
    return VR_OK;
}

vr_status vr_set_brick_size(vr_ctx* ctx, int vol_id, int cells) {
    NvtxRange range_("vr_set_brick_size");
    if (!ctx) return VR_ERR_INVALID_ARG;
    Volume* v = get_vol(ctx, vol_id);
    if (!v) return fail(ctx, VR_ERR_INVALID_ARG, "set_brick_size: unknown id %d", vol_id);
    int bs = -1;
    for (int q = kMinBrickShift; q <= kMaxBrickShift; ++q)
        if (cells == (1 << q)) bs = q;
    if (bs < 0) return fail(ctx, VR_ERR_INVALID_ARG, "set_brick_size: %d cells per brick edge; 4, 8 or 16", cells);
    if (bs == v->bs) return VR_OK;
    DeviceGuard g(ctx->device);
    CK(cudaStreamSynchronize(ctx->stream), "set_brick_size sync");
    // the grid, flags, cells and derived bricks follow the new size; the derived
    // bricks and the cell grid are rebuilt by the next vr_precompute_morphology
    v->morph_ready = false;
    dfree(ctx, v->d_grid);
    dfree(ctx, v->d_empty);
    dfree(ctx, v->d_dbricks);
    dfree(ctx, v->d_cellq);
    dfree(ctx, v->d_cellmask);
    v->d_grid = nullptr, v->d_empty = nullptr, v->d_dbricks = nullptr, v->d_cellq = nullptr, v->d_cellmask = nullptr;
    v->bs = bs;
    for (int a = 0; a < 3; ++a) v->nb[a] = (v->n[a] - 1 + (1 << bs) - 1) >> bs;
    v->nbricks = (long long)v->nb[0] * v->nb[1] * v->nb[2];
    CK(dalloc(ctx, &v->d_grid, sizeof(uint16_t) * 2 * v->nbricks), "set_brick_size: grid");
    CK(dalloc(ctx, &v->d_empty, v->nbricks), "set_brick_size: flags");
    CK(cudaMemsetAsync(v->d_empty, 0, v->nbricks, ctx->stream), "set_brick_size: flags");
    CK(launch_brick_minmax(v->d_norm, v->n, v->nb, v->bs, v->d_grid, ctx->stream), "set_brick_size: brick min/max");
    return VR_OK;
}

vr_status vr_get_vesselness(vr_ctx* ctx, int vol_id, float* out, int out_on_device) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    Volume* v = get_vol(ctx, vol_id);
    if (!v || !out) return fail(ctx, VR_ERR_INVALID_ARG, "get_vesselness: bad arguments");
    if (!v->v_ready) return fail(ctx, VR_ERR_NOT_READY, "get_vesselness: no vesselness or second channel");
    DeviceGuard g(ctx->device);
    CK(cudaMemcpyAsync(out, v->d_vessel, sizeof(float) * v->nvox,
                       out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream),
       "get_vesselness copy");
    if (!out_on_device) CK(cudaStreamSynchronize(ctx->stream), "get_vesselness sync");
    return VR_OK;
}

vr_status vr_get_normalized(vr_ctx* ctx, int vol_id, float* out, int out_on_device) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    Volume* v = get_vol(ctx, vol_id);
    if (!v || !out) return fail(ctx, VR_ERR_INVALID_ARG, "get_normalized: bad arguments");
    DeviceGuard g(ctx->device);
    CK(cudaMemcpyAsync(out, v->d_norm, sizeof(float) * v->nvox,
                       out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream),
       "get_normalized copy");
    if (!out_on_device) CK(cudaStreamSynchronize(ctx->stream), "get_normalized sync");
    return VR_OK;
}

vr_status vr_prefilter(vr_ctx* ctx, int vol_id, int mode, float sigma) {
    NvtxRange range_("vr_prefilter");
    if (!ctx) return VR_ERR_INVALID_ARG;
    Volume* v = get_vol(ctx, vol_id);
    if (!v) return fail(ctx, VR_ERR_INVALID_ARG, "prefilter: unknown id %d", vol_id);
    if (mode != 1 && mode != 2) return fail(ctx, VR_ERR_INVALID_ARG, "prefilter: mode must be 1 (median) or 2 (Gaussian)");
    if (mode == 2 && !(sigma > 0.0f && sigma <= 8.0f))
        return fail(ctx, VR_ERR_INVALID_ARG, "prefilter: sigma %g outside (0, 8]", (double)sigma);
    DeviceGuard g(ctx->device);
    const size_t need = sizeof(float) * 2 * (size_t)v->nvox;
    if (ctx->scratch_cap < need) {
        CK(cudaStreamSynchronize(ctx->stream), "prefilter: scratch sync");
        dfree(ctx, ctx->d_scratch);
        ctx->d_scratch = nullptr;
        ctx->scratch_cap = 0;
        CK(dalloc(ctx, &ctx->d_scratch, need), "prefilter: scratch");
        ctx->scratch_cap = need;
    }
    float* a = ctx->d_scratch;
    if (mode == 1) {
        CK(launch_median3(v->d_norm, a, v->n, ctx->stream), "prefilter: median");
    } else {
        CK(launch_gauss3d(v->d_norm, a, ctx->d_scratch + v->nvox, v->n, sigma, ctx->stream), "prefilter: Gaussian");
    }
    CK(cudaMemcpyAsync(v->d_norm, a, sizeof(float) * v->nvox, cudaMemcpyDeviceToDevice, ctx->stream),
       "prefilter: copy back");
    vr_status st = rebuild_bricks(ctx, v);
    if (st != VR_OK) return st;
    if (v->params_ready) {
        st = classify_volume(ctx, v);
        if (st != VR_OK) return st;
    }
    v->morph_ready = false;  // |grad I|max and vesselness describe the unfiltered volume
    return VR_OK;
}

vr_status vr_tissue_histogram(vr_ctx* ctx, int vol_id, int lo_bin, int hi_bin, unsigned long long* d_hist,
                              int* d_peaks) {
    NvtxRange range_("vr_tissue_histogram");
    if (!ctx) return VR_ERR_INVALID_ARG;
    Volume* v = get_vol(ctx, vol_id);
    if (!v) return fail(ctx, VR_ERR_INVALID_ARG, "tissue_histogram: unknown id %d", vol_id);
    if (!d_hist) return fail(ctx, VR_ERR_INVALID_ARG, "tissue_histogram: NULL histogram");
    if (lo_bin < 0 || hi_bin > 255 || lo_bin > hi_bin)
        return fail(ctx, VR_ERR_INVALID_ARG, "tissue_histogram: bins [%d, %d] outside [0, 255]", lo_bin, hi_bin);
    DeviceGuard g(ctx->device);
    CK(launch_histogram(v->d_norm, v->nvox, d_hist, ctx->stream), "histogram");
    if (d_peaks) CK(launch_tissue_peaks(d_hist, lo_bin, hi_bin, d_peaks, ctx->stream), "tissue peaks");
    return VR_OK;
}

vr_status vr_render(vr_ctx* ctx, int vol_id, const vr_camera* h_cams, int n_cams, int W, int H, float* out_rgba,
                    int out_on_host, const vr_render_opts* opts, vr_counters* d_counters,
                    unsigned int* d_ray_samples) {
    NvtxRange range_("vr_render");
    if (!ctx) return VR_ERR_INVALID_ARG;
    Volume* v = get_vol(ctx, vol_id);
    if (!v) return fail(ctx, VR_ERR_INVALID_ARG, "render: unknown id %d", vol_id);
    if (!h_cams || !out_rgba) return fail(ctx, VR_ERR_INVALID_ARG, "render: NULL pointer");
    if (n_cams < 1 || W < 1 || H < 1 || W > 16384 || H > 16384)
        return fail(ctx, VR_ERR_INVALID_ARG, "render: bad image size %d x %d x %d", n_cams, W, H);
    if (!v->morph_ready) return fail(ctx, VR_ERR_NOT_READY, "render: call vr_precompute_morphology first");
    if (!v->params_ready) return fail(ctx, VR_ERR_NOT_READY, "render: call vr_set_tissue_params first");
    vr_render_opts o{VR_KERNEL_AUTO, 1, 4, 4, nullptr};
    if (opts) o = *opts;
    if (o.kernel < 0 || o.kernel > 4) return fail(ctx, VR_ERR_INVALID_ARG, "render: bad kernel choice");
    const bool staged_der = o.kernel == VR_KERNEL_STAGED_DERIVED;
    if (staged_der) {
        if (!v->d_dbricks)
            return fail(ctx, VR_ERR_INVALID_ARG, "render: the staged derived kernel needs the derived bricks");
        if (v->bs > 3)
            return fail(ctx, VR_ERR_INVALID_ARG, "render: the staged derived kernel stages 4^3- or 8^3-cell bricks");
        if (v->tp.tf_mode == 2)
            return fail(ctx, VR_ERR_INVALID_ARG, "render: the staged derived kernel has no second channel");
        if (o.ray_state) return fail(ctx, VR_ERR_INVALID_ARG, "render: ray_state needs a per-lane kernel");
        if (o.packet_w != 4 && o.packet_w != 8 && o.packet_w != 16 && o.packet_w != 32)
            return fail(ctx, VR_ERR_INVALID_ARG, "render: packet_w must be 4, 8, 16 or 32");
        if (o.warps_per_block < 1 || o.warps_per_block > (v->bs == 2 ? 8 : 6))
            return fail(ctx, VR_ERR_INVALID_ARG, "render: warps_per_block outside the shared memory of a CTA");
    }
    if (o.kernel == VR_KERNEL_STAGED && o.ray_state)
        return fail(ctx, VR_ERR_INVALID_ARG, "render: ray_state needs a per-lane kernel");
    // VR_KERNEL_AUTO picks the per-lane gather kernel: on GB300 the bricked volume stays
    // L1/L2-resident and per-lane marching keeps 91% of lanes busy, while staging one
    // brick per warp idles the lanes outside it (ncu: 58% SIMT efficiency).
    const bool staged = o.kernel == VR_KERNEL_STAGED;
    if (staged && (o.packet_w != 4 && o.packet_w != 8 && o.packet_w != 16 && o.packet_w != 32))
        return fail(ctx, VR_ERR_INVALID_ARG, "render: packet_w must be 4, 8, 16 or 32");
    if (staged && v->bs != 3)
        return fail(ctx, VR_ERR_INVALID_ARG, "render: the staged kernel stages 8^3-cell bricks (vr_set_brick_size 8)");
    if (staged && (o.warps_per_block < 1 || o.warps_per_block > 8))
        return fail(ctx, VR_ERR_INVALID_ARG, "render: warps_per_block must be in [1, 8]");
    if (!staged && !staged_der && o.packet_w != 4 && o.packet_w != 8 && o.packet_w != 16)
        return fail(ctx, VR_ERR_INVALID_ARG, "render: packet_w must be 4, 8 or 16 for the per-lane kernels");
    if (!staged && !staged_der && o.warps_per_block != 2 && o.warps_per_block != 4 && o.warps_per_block != 8)
        return fail(ctx, VR_ERR_INVALID_ARG, "render: warps_per_block must be 2, 4 or 8 for the per-lane kernels");
    DeviceGuard g(ctx->device);
    float* dst = out_rgba;
    const size_t img_bytes = sizeof(float) * 4 * (size_t)n_cams * W * H;
    bool copy_back = false;
    if (out_on_host) {
        // page-locked host memory is mapped into the device's address space: the kernel
        // writes the image there itself, over the host link, while it renders; other
        // host memory goes through a device staging buffer and a copy on the stream
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, out_rgba) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
            pa.devicePointer) {
            dst = static_cast<float*>(pa.devicePointer);
        } else {
            (void)cudaGetLastError();  // an unregistered pointer is not an error here
            CK(ensure_stage(ctx, img_bytes), "render: image staging buffer");
            dst = (float*)ctx->d_stage;
            copy_back = true;
        }
    }
    RenderLaunch L;
    fill_launch(L, v, W, H, o.skip_empty);
    L.out = dst;
    L.counters = d_counters;
    L.ray_samples = d_ray_samples;
    L.ray_state = static_cast<float2*>(o.ray_state);
    if (o.kernel == VR_KERNEL_GATHER_STENCIL) L.vol.dbricks = nullptr;
    L.packet_w = o.packet_w;
    L.packet_h = 32 / (o.packet_w > 0 ? o.packet_w : 8);
    L.work_counter = ctx->d_work;
    L.status = ctx->d_work + 1;
    L.n_packets_x = (W + L.packet_w - 1) / L.packet_w;
    L.n_packets_y = (H + L.packet_h - 1) / L.packet_h;
    int ctas = 0;
    if (staged_der) {
        int per_sm = 0;
        CK(staged_derived_config(o.warps_per_block, v->bs, &per_sm), "render: staged derived kernel configuration");
        if (per_sm < 1) return fail(ctx, VR_ERR_INVALID_ARG, "render: staged derived kernel does not fit on an SM");
        int sms = 0;
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device), "render: SM count");
        ctas = sms * per_sm;
    }
    if (staged) {
        const bool ves = L.vol.vbricks != nullptr;
        int& per_sm = ctx->staged_ctas[ves][o.warps_per_block];
        if (per_sm == 0) CK(staged_config(o.warps_per_block, ves, &per_sm), "render: staged kernel configuration");
        if (per_sm < 1) return fail(ctx, VR_ERR_INVALID_ARG, "render: staged kernel does not fit on an SM");
        int sms = 0;
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device), "render: SM count");
        ctas = sms * per_sm;
    }
    for (int c0 = 0; c0 < n_cams; c0 += kMaxCamsPerLaunch) {
        const int nc = n_cams - c0 < kMaxCamsPerLaunch ? n_cams - c0 : kMaxCamsPerLaunch;
        L.n_cams = nc;
        L.cam_offset = c0;
        memcpy(L.cams, h_cams + c0, sizeof(CamDev) * nc);
        if (staged || staged_der) {
            L.n_work = nc * L.n_packets_x * L.n_packets_y;
            const int need = (L.n_work + o.warps_per_block - 1) / o.warps_per_block;
            CK(cudaMemsetAsync(ctx->d_work, 0, sizeof(unsigned), ctx->stream), "render: reset work counter");
            if (staged_der)
                CK(launch_render_staged_derived(L, o.warps_per_block, ctas < need ? ctas : need, ctx->stream),
                   "render kernel");
            else
                CK(launch_render_staged(L, o.warps_per_block, ctas < need ? ctas : need, ctx->stream),
                   "render kernel");
        } else {
            CK(launch_render_gather(L, o.warps_per_block, ctx->stream), "render kernel");
        }
    }
    if (copy_back)
        CK(cudaMemcpyAsync(out_rgba, dst, img_bytes, cudaMemcpyDeviceToHost, ctx->stream), "render: copy image back");
    return VR_OK;
}

vr_status vr_render_backward(vr_ctx* ctx, int vol_id, const vr_camera* h_cams, int n_cams, int W, int H,
                             const float* d_dl_drgba, float* d_dtf, float* d_dparams, float* d_dvolume,
                             const vr_render_opts* opts) {
    NvtxRange range_("vr_render_backward");
    if (!ctx) return VR_ERR_INVALID_ARG;
    Volume* v = get_vol(ctx, vol_id);
    if (!v) return fail(ctx, VR_ERR_INVALID_ARG, "render_backward: unknown id %d", vol_id);
    if (!h_cams || !d_dl_drgba || !d_dtf)
        return fail(ctx, VR_ERR_INVALID_ARG, "render_backward: NULL pointer");
    if (n_cams < 1 || W < 1 || H < 1 || W > 16384 || H > 16384)
        return fail(ctx, VR_ERR_INVALID_ARG, "render_backward: bad image size %d x %d x %d", n_cams, W, H);
    if (!v->morph_ready) return fail(ctx, VR_ERR_NOT_READY, "render_backward: call vr_precompute_morphology first");
    if (!v->params_ready) return fail(ctx, VR_ERR_NOT_READY, "render_backward: call vr_set_tissue_params first");
    DeviceGuard g(ctx->device);
    const int skip = opts ? opts->skip_empty : 1;
    if (opts && (opts->kernel < 0 || opts->kernel > 3))
        return fail(ctx, VR_ERR_INVALID_ARG, "render_backward: bad kernel choice");
    const size_t ntf = (size_t)v->tp.tf_w * v->tp.tf_h * 4;
    CK(cudaMemsetAsync(d_dtf, 0, sizeof(float) * ntf, ctx->stream), "render_backward: zero dtf");
    if (d_dparams) CK(cudaMemsetAsync(d_dparams, 0, sizeof(float) * 5, ctx->stream), "render_backward: zero dparams");
    BackwardLaunch B;
    memset(&B, 0, sizeof B);
    fill_launch(B.r, v, W, H, skip);
    const bool staged = opts && opts->kernel == VR_KERNEL_STAGED;
    if (staged || (opts && opts->kernel == VR_KERNEL_GATHER_STENCIL)) B.r.vol.dbricks = nullptr;
    B.r.packet_w = opts ? opts->packet_w : 4;
    B.r.ray_state = opts ? static_cast<float2*>(opts->ray_state) : nullptr;
    if (staged && v->bs != 3)
        return fail(ctx, VR_ERR_INVALID_ARG,
                    "render_backward: the staged kernel stages 8^3-cell bricks (vr_set_brick_size 8)");
    if (staged && B.r.ray_state)
        return fail(ctx, VR_ERR_INVALID_ARG, "render_backward: ray_state needs a per-lane kernel");
    if (!staged && B.r.packet_w != 4 && B.r.packet_w != 8 && B.r.packet_w != 16)
        return fail(ctx, VR_ERR_INVALID_ARG, "render_backward: packet_w must be 4, 8 or 16");
    B.r.packet_h = 32 / B.r.packet_w;
    // On the derived bricks, voxel gradients go first to per-voxel channel gradients
    // (vector atomics), then one gather pass applies the channels' stencil transposes.
    const bool channels = d_dvolume && B.r.vol.dbricks;
    if (channels) {
        const size_t need = sizeof(float) * 10 * (size_t)v->nvox;  // three channel planes
        if (ctx->dgrad_cap < need) {
            CK(cudaStreamSynchronize(ctx->stream), "render_backward: scratch sync");
            dfree(ctx, ctx->d_dgrad);
            ctx->d_dgrad = nullptr;
            ctx->dgrad_cap = 0;
            CK(dalloc(ctx, &ctx->d_dgrad, need), "render_backward: channel gradient scratch");
            ctx->dgrad_cap = need;
        }
        CK(cudaMemsetAsync(ctx->d_dgrad, 0, need, ctx->stream), "render_backward: zero channel gradients");
        B.dgrad = ctx->d_dgrad;
    } else if (d_dvolume) {
        CK(cudaMemsetAsync(d_dvolume, 0, sizeof(float) * v->nvox, ctx->stream), "render_backward: zero dvol");
    }
    B.dl_drgba = d_dl_drgba;
    B.dtf = d_dtf;
    B.dparams = d_dparams;
    B.dvol = d_dvolume;
    {
        // private copies of the transfer-function gradient (a 16-float record per
        // lookup cell), summed after the kernels: as many copies as fit 64 MB (so that
        // they stay in L2; 256 MB measured 1 % slower), 8 to 1024: the fewer the table's
        // entries, the more CTAs contend for each, and the cheaper a copy is (a 256x64
        // table: 64 copies of 1 MB)
        const size_t tbytes = sizeof(float) * kTfCellFloats * (size_t)v->tp.tf_w * v->tp.tf_h;
        const int ncopies = (int)std::min<size_t>(1024, std::max<size_t>(8, ((size_t)64 << 20) / tbytes));
        const size_t need = tbytes * ncopies;
        if (ctx->tfgrad_cap < need) {
            CK(cudaStreamSynchronize(ctx->stream), "render_backward: scratch sync");
            dfree(ctx, ctx->d_tfgrad);
            ctx->d_tfgrad = nullptr;
            ctx->tfgrad_cap = 0;
            CK(dalloc(ctx, &ctx->d_tfgrad, need), "render_backward: transfer-function gradient scratch");
            ctx->tfgrad_cap = need;
        }
        CK(cudaMemsetAsync(ctx->d_tfgrad, 0, need, ctx->stream), "render_backward: zero scratch");
        B.dtf_copies = ctx->d_tfgrad;
        B.n_copies = ncopies;
    }
    for (int c0 = 0; c0 < n_cams; c0 += kMaxCamsPerLaunch) {
        const int nc = n_cams - c0 < kMaxCamsPerLaunch ? n_cams - c0 : kMaxCamsPerLaunch;
        B.r.n_cams = nc;
        B.r.cam_offset = c0;
        memcpy(B.r.cams, h_cams + c0, sizeof(CamDev) * nc);
        // per-lane sweep with global voxel atomics by default: at 1080p it measured
        // 46 ms against 84 ms for the brick-synchronous sweep, whose idle lanes and
        // conflicting shared-memory atomics cost more than the global atomics it saves
        CK(launch_render_backward(B, staged, ctx->stream), "render_backward kernel");
    }
    if (channels)
        CK(launch_channels_to_voxels(ctx->d_dgrad, v->n, v->s, d_dvolume, ctx->stream),
           "render_backward: channel gradients to voxels");
    CK(launch_sum_copies(ctx->d_tfgrad, B.n_copies, v->tp.tf_w, v->tp.tf_h, d_dtf, ctx->stream),
       "render_backward: sum gradient copies");
    return VR_OK;
}

namespace {

int shape_index(int packet_w) { return packet_w == 4 ? 0 : packet_w == 8 ? 1 : packet_w == 16 ? 2 : packet_w == 32 ? 3 : -1; }

// Refresh the device view table from the volumes' current state.
vr_status batch_upload(vr_ctx* ctx, Batch* b) {
    const int n = (int)b->views.size();
    b->table.resize(n);
    std::vector<int> prefix(4 * n);
    for (int si = 0; si < 4; ++si) {
        const int pw = 4 << si, ph = 32 / pw;
        int acc = 0;
        for (int i = 0; i < n; ++i) {
            prefix[si * n + i] = acc;
            acc += ((b->views[i].W + pw - 1) / pw) * ((b->views[i].H + ph - 1) / ph);
        }
        b->n_work[si] = acc;
    }
    bool all_derived = true;
    int bs = -1;
    for (int i = 0; i < n; ++i) {
        const vr_view& vw = b->views[i];
        Volume* v = get_vol(ctx, vw.vol_id);
        if (!v) return fail(ctx, VR_ERR_INVALID_ARG, "batch: view %d names unknown volume %d", i, vw.vol_id);
        if (!v->morph_ready || !v->params_ready)
            return fail(ctx, VR_ERR_NOT_READY, "batch: volume %d lacks morphology or tissue params", vw.vol_id);
        RenderLaunch L;
        fill_launch(L, v, vw.W, vw.H, 1);
        ViewDev& d = b->table[i];
        d.vol = L.vol;
        d.tp = L.tp;
        d.tf = L.tf;
        memcpy(&d.cam, &vw.cam, sizeof(CamDev));
        d.out = vw.d_out;
        d.W = vw.W;
        d.H = vw.H;
        d.rc = L.rc;
        all_derived = all_derived && L.vol.dbricks != nullptr;
        bs = (bs < 0 || bs == v->bs) ? v->bs : 0;
    }
    if (all_derived != b->all_derived || bs != b->bs) {
        // the captured graphs launch another kernel variant
        if (ctx->graph_stream) CK(cudaStreamSynchronize(ctx->graph_stream), "batch: graph sync");
        for (auto& gx : b->graphs) cudaGraphExecDestroy(gx.second);
        b->graphs.clear();
        b->all_derived = all_derived;
        b->bs = bs;
    }
    CK(cudaMemcpyAsync(b->d_views, b->table.data(), sizeof(ViewDev) * n, cudaMemcpyHostToDevice, ctx->stream),
       "batch: upload views");
    CK(cudaMemcpyAsync(b->d_prefix, prefix.data(), sizeof(int) * 4 * n, cudaMemcpyHostToDevice, ctx->stream),
       "batch: upload packet table");
    CK(cudaStreamSynchronize(ctx->stream), "batch: upload sync");
    return VR_OK;
}

// Enqueue one batched launch on `st` (no host synchronisation, no allocation).
vr_status batch_enqueue(vr_ctx* ctx, Batch* b, const vr_render_opts& o, vr_counters* ctr, cudaStream_t st) {
    const int si = shape_index(o.packet_w);
    int& per_sm = ctx->batch_ctas[b->all_derived][o.warps_per_block];
    if (per_sm == 0) CK(batch_ctas_per_sm(o.warps_per_block, b->all_derived, &per_sm), "batch: occupancy");
    if (per_sm < 1) return fail(ctx, VR_ERR_INVALID_ARG, "batch: kernel does not fit on an SM");
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device), "batch: SM count");
    BatchLaunch B;
    memset(&B, 0, sizeof B);
    B.views = b->d_views;
    B.packet_prefix = b->d_prefix + si * (int)b->views.size();
    B.n_views = (int)b->views.size();
    B.n_work = b->n_work[si];
    B.packet_w = o.packet_w;
    B.packet_h = 32 / o.packet_w;
    B.work_counter = ctx->d_work + 2;
    B.counters = ctr;
    B.skip = o.skip_empty ? 1 : 0;
    const int need = (B.n_work + o.warps_per_block - 1) / o.warps_per_block;
    int ctas = sms * per_sm;
    if (ctas > need) ctas = need;
    if (ctas < 1) ctas = 1;
    CK(cudaMemsetAsync(ctx->d_work + 2, 0, sizeof(unsigned), st), "batch: reset work counter");
    CK(launch_render_batch(B, o.warps_per_block, ctas, b->all_derived, b->bs, st), "batch kernel");
    return VR_OK;
}

vr_status batch_opts(vr_ctx* ctx, const vr_render_opts* opts, vr_render_opts* o) {
    *o = vr_render_opts{VR_KERNEL_AUTO, 1, 8, 8, nullptr};
    if (opts) *o = *opts;
    if (shape_index(o->packet_w) < 0) return fail(ctx, VR_ERR_INVALID_ARG, "batch: packet_w must be 4, 8, 16 or 32");
    if (o->warps_per_block < 1 || o->warps_per_block > 8)
        return fail(ctx, VR_ERR_INVALID_ARG, "batch: warps_per_block must be in [1, 8]");
    return VR_OK;
}

}  // namespace

vr_status vr_batch_create(vr_ctx* ctx, const vr_view* views, int n_views, int* batch_id) {
    NvtxRange range_("vr_batch_create");
    if (!ctx) return VR_ERR_INVALID_ARG;
    if (!views || !batch_id || n_views < 1 || n_views > (1 << 20))
        return fail(ctx, VR_ERR_INVALID_ARG, "batch_create: bad arguments");
    long long packets = 0;
    for (int i = 0; i < n_views; ++i) {
        if (!views[i].d_out || views[i].W < 1 || views[i].H < 1 || views[i].W > 16384 || views[i].H > 16384)
            return fail(ctx, VR_ERR_INVALID_ARG, "batch_create: view %d has a bad output or size", i);
        packets += ((long long)(views[i].W + 3) / 4) * ((views[i].H + 7) / 8);
    }
    if (packets >= (1LL << 31)) return fail(ctx, VR_ERR_INVALID_ARG, "batch_create: too many rays");
    DeviceGuard g(ctx->device);
    Batch* b = new Batch();
    b->views.assign(views, views + n_views);
    cudaError_t e = dalloc(ctx, &b->d_views, sizeof(ViewDev) * n_views);
    if (e == cudaSuccess) e = dalloc(ctx, &b->d_prefix, sizeof(int) * 4 * n_views);
    if (e != cudaSuccess) {
        dfree(ctx, b->d_views);
        delete b;
        return cuda_fail(ctx, e, "batch_create: allocate");
    }
    vr_status st = batch_upload(ctx, b);
    if (st != VR_OK) {
        dfree(ctx, b->d_views);
        dfree(ctx, b->d_prefix);
        delete b;
        return st;
    }
    const int id = ctx->next_batch++;
    ctx->batches[id] = b;
    *batch_id = id;
    return VR_OK;
}

vr_status vr_batch_update(vr_ctx* ctx, int batch_id) {
    NvtxRange range_("vr_batch_update");
    if (!ctx) return VR_ERR_INVALID_ARG;
    auto it = ctx->batches.find(batch_id);
    if (it == ctx->batches.end()) return fail(ctx, VR_ERR_INVALID_ARG, "batch_update: unknown batch %d", batch_id);
    DeviceGuard g(ctx->device);
    return batch_upload(ctx, it->second);
}

vr_status vr_batch_render(vr_ctx* ctx, int batch_id, const vr_render_opts* opts, vr_counters* d_counters) {
    NvtxRange range_("vr_batch_render");
    if (!ctx) return VR_ERR_INVALID_ARG;
    auto it = ctx->batches.find(batch_id);
    if (it == ctx->batches.end()) return fail(ctx, VR_ERR_INVALID_ARG, "batch_render: unknown batch %d", batch_id);
    vr_render_opts o;
    vr_status st = batch_opts(ctx, opts, &o);
    if (st != VR_OK) return st;
    DeviceGuard g(ctx->device);
    return batch_enqueue(ctx, it->second, o, d_counters, ctx->stream);
}

vr_status vr_batch_render_graph(vr_ctx* ctx, int batch_id, const vr_render_opts* opts) {
    NvtxRange range_("vr_batch_render_graph");
    if (!ctx) return VR_ERR_INVALID_ARG;
    auto it = ctx->batches.find(batch_id);
    if (it == ctx->batches.end())
        return fail(ctx, VR_ERR_INVALID_ARG, "batch_render_graph: unknown batch %d", batch_id);
    vr_render_opts o;
    vr_status st = batch_opts(ctx, opts, &o);
    if (st != VR_OK) return st;
    DeviceGuard g(ctx->device);
    Batch* b = it->second;
    if (!ctx->graph_stream) {
        CK(cudaStreamCreateWithFlags(&ctx->graph_stream, cudaStreamNonBlocking), "graph stream");
        CK(cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming), "graph event");
        CK(cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming), "graph event");
    }
    const auto key = std::make_pair(o.packet_w, o.warps_per_block * 2 + (o.skip_empty ? 1 : 0));
    auto git = b->graphs.find(key);
    if (git == b->graphs.end()) {
        // occupancy and SM count are queried outside the capture
        int& per_sm = ctx->batch_ctas[b->all_derived][o.warps_per_block];
        if (per_sm == 0) CK(batch_ctas_per_sm(o.warps_per_block, b->all_derived, &per_sm), "batch: occupancy");
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(ctx->graph_stream, cudaStreamCaptureModeThreadLocal), "graph capture begin");
        vr_status es = batch_enqueue(ctx, b, o, nullptr, ctx->graph_stream);
        cudaError_t e2 = cudaStreamEndCapture(ctx->graph_stream, &graph);
        if (es != VR_OK) {
            if (graph) cudaGraphDestroy(graph);
            return es;
        }
        CK(e2, "graph capture end");
        cudaGraphExec_t exec = nullptr;
        cudaError_t e3 = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        CK(e3, "graph instantiate");
        git = b->graphs.emplace(key, exec).first;
    }
    CK(cudaEventRecord(ctx->ev_in, ctx->stream), "graph fence in");
    CK(cudaStreamWaitEvent(ctx->graph_stream, ctx->ev_in, 0), "graph fence in wait");
    CK(cudaGraphLaunch(git->second, ctx->graph_stream), "graph launch");
    CK(cudaEventRecord(ctx->ev_out, ctx->graph_stream), "graph fence out");
    CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_out, 0), "graph fence out wait");
    return VR_OK;
}

vr_status vr_batch_free(vr_ctx* ctx, int batch_id) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    auto it = ctx->batches.find(batch_id);
    if (it == ctx->batches.end()) return fail(ctx, VR_ERR_INVALID_ARG, "batch_free: unknown batch %d", batch_id);
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->graph_stream) cudaStreamSynchronize(ctx->graph_stream);
    for (auto& gx : it->second->graphs) cudaGraphExecDestroy(gx.second);
    dfree(ctx, it->second->d_views);
    dfree(ctx, it->second->d_prefix);
    delete it->second;
    ctx->batches.erase(it);
    return VR_OK;
}

vr_status vr_fma_peak(vr_ctx* ctx, int blocks, int iters, int reps, float* h_ms, double* h_flops) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    if (!h_ms || !h_flops || blocks < 1 || blocks > (1 << 20) || iters < 1 || iters > (1 << 20) || reps < 1 ||
        reps > 64)
        return fail(ctx, VR_ERR_INVALID_ARG, "fma_peak: bad arguments");
    DeviceGuard g(ctx->device);
    float* out = nullptr;
    CK(dalloc(ctx, &out, sizeof(float) * 256 * (size_t)blocks), "fma_peak scratch");
    cudaEvent_t ev[2 * 64 + 2];
    int made = 0;
    cudaError_t e = cudaSuccess;
    for (; made < 2 * reps && e == cudaSuccess; ++made) e = cudaEventCreate(&ev[made]);
    if (e == cudaSuccess) e = launch_fma_peak(out, blocks, iters, ctx->stream);  // warm-up
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        e = cudaEventRecord(ev[2 * r], ctx->stream);
        if (e == cudaSuccess) e = launch_fma_peak(out, blocks, iters, ctx->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2 * r + 1], ctx->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    std::vector<float> ms;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        float t = 0.0f;
        e = cudaEventElapsedTime(&t, ev[2 * r], ev[2 * r + 1]);
        ms.push_back(t);
    }
    for (int q = 0; q < made; ++q) cudaEventDestroy(ev[q]);
    dfree(ctx, out);
    if (e != cudaSuccess) return fail(ctx, VR_ERR_CUDA, "fma_peak: %s", cudaGetErrorString(e));
    std::sort(ms.begin(), ms.end());
    *h_ms = ms[ms.size() / 2];
    *h_flops = (double)blocks * 256.0 * (double)iters * 16.0 * 8.0 * 2.0;
    return VR_OK;
}

vr_status vr_set_derived_budget(vr_ctx* ctx, unsigned long long bytes) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    ctx->derived_budget = (size_t)bytes;
    return VR_OK;
}

int vr_debug_build(void) {
#ifdef VR_DEBUG
    return 1;
#else
    return 0;
#endif
}

vr_status vr_debug_check_probe(vr_ctx* ctx) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    CK(launch_check_probe(ctx->d_work + 1, ctx->stream), "index-check probe");
    return VR_OK;
}

vr_status vr_set_memory_limit(vr_ctx* ctx, unsigned long long bytes) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    ctx->mem_limit = (size_t)bytes;
    return VR_OK;
}

vr_status vr_memory_used(vr_ctx* ctx, unsigned long long* bytes) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    if (!bytes) return fail(ctx, VR_ERR_INVALID_ARG, "memory_used: NULL pointer");
    *bytes = (unsigned long long)ctx->mem_used;
    return VR_OK;
}

vr_status vr_debug_fail_alloc(vr_ctx* ctx, long long n_ok, long long* pending) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    if (n_ok < -1) return fail(ctx, VR_ERR_INVALID_ARG, "debug_fail_alloc: n_ok must be >= -1");
    if (pending) *pending = ctx->fail_after;
    ctx->fail_after = n_ok;
    return VR_OK;
}

vr_status vr_probe_bounded_wait(vr_ctx* ctx, long long budget_cycles) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    if (budget_cycles < 1 || budget_cycles > (1LL << 31))
        return fail(ctx, VR_ERR_INVALID_ARG, "probe_bounded_wait: budget outside [1, 2^31] cycles");
    DeviceGuard g(ctx->device);
    CK(launch_wait_probe(ctx->d_work + 1, budget_cycles, ctx->stream), "bounded-wait probe");
    return VR_OK;
}

}  // extern "C"

// vr_internal.cuh -- declarations shared by the library's translation units.
//
// Volume storage. Interpolation cell i0 spans voxels i0 and i0+1 along each axis;
// a sample whose clamped coordinate u_c has floor cell i0 = min(floor(u_c), N-2)
// lies in that cell. Two brick grids cut the cells:
//  * storage bricks of 8^3 cells hold the intensities (and the second channel)
//    for the per-sample stencils: a dense 12^3 float32 block of voxels
//    [8b-1, 8b+11) per axis with clamp-to-edge values outside the volume, so the
//    4-tap stencils of a cell (voxels i0-1 .. i0+2) fall inside it; 6912 bytes
//    (a multiple of 16), one bulk copy moves it;
//  * skip bricks of B^3 cells (B = 2^bs, 4, 8 or 16; 8 by default) carry the
//    quantised min/max grid, the empty flags, the per-cell empty bits and the
//    derived bricks of the voxel-wise derivatives, (B+1)^3 corners each.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vr.h"
#include "vr_async.cuh"
#include "vr_df.cuh"

namespace vr {

constexpr int kCells = 8;                          // interpolation cells per brick edge
constexpr int kEdge = 12;                          // stored brick edge (1 low + 8 + 3 high apron)
constexpr int kBrickVox = kEdge * kEdge * kEdge;   // 1728 floats
constexpr int kBrickBytes = kBrickVox * 4;         // 6912 bytes
constexpr int kMaxCamsPerLaunch = 64;

// Derived bricks: per skip brick the (B+1)^3 corner voxels [Bb, Bb+B] (clamped) of
// its cells, each as 12 floats = I, gx, gy, gz, Hxx, Hyy, Hzz, Hxy, Hxz, Hyz (mm
// units), 0, 0: the voxel-wise derivatives of Sec. 2.3, three 16-byte loads per
// corner (B = 8: 9^3 corners, 34,992 B).
constexpr int kDerFloats = 12;
constexpr int kMinBrickShift = 2, kMaxBrickShift = 4;  // skip bricks of 4^3 .. 16^3 cells

__host__ __device__ __forceinline__ int der_edge(int bs) { return (1 << bs) + 1; }
__host__ __device__ __forceinline__ long long der_brick_floats(int bs) {
    const long long e = der_edge(bs);
    return e * e * e * kDerFloats;
}
// Per-cell empty bits of a skip brick: B^3 bits, in 32-bit words.
__host__ __device__ __forceinline__ int cell_words(int bs) { return (1 << (3 * bs)) >> 5; }
constexpr size_t kDerivedBudgetBytes = (size_t)16 << 30;  // default: built only up to this size

struct CamDev {
    float eye[3], fwd[3], right[3], up[3];
};

struct TissueDev {
    int tf_mode, tf_w, tf_h, grad_mod, shading;
    float gamma, kappa_ref, w_max, ka, kd, ks, opacity_scale, et_threshold, step_vox;
    float alpha_exp;  // dt / opacity_ref_step for the step-size opacity correction; 0 = off
    float gk, inv_kref;  // gamma / kappa_ref and 1 / kappa_ref (rounded from double on the host)
    unsigned* status;    // the context's device status word (debug builds report failed index checks there)
};

// Index checks of the debug library (VR_DEBUG): VR_CHECK(status, cond) is cond,
// and when cond is false it also sets kStatusBounds in status[0] and records the
// source line of the first failed check in status[1]; the caller skips the access.
// Without VR_DEBUG it is the constant true and the check compiles away.
#ifdef VR_DEBUG
__device__ __forceinline__ bool debug_check(bool ok, unsigned* status, int line) {
    if (!ok && status) {
        atomicOr(status, kStatusBounds);
        atomicCAS(status + 1, 0u, (unsigned)line);
    }
    return ok;
}
#define VR_CHECK(status, cond) ::vr::debug_check((cond), (status), __LINE__)
#else
#define VR_CHECK(status, cond) true
#endif

// Per-volume constants that kernels read from device memory (so that host code
// never waits for the reductions that produce them).
struct VolConst {
    float imin, imax, range, gmax;
};

struct VolumeDev {
    int n[3];       // voxels per axis
    int nb[3];      // skip bricks per axis = ceil((n-1)/B)
    int nsb[3];     // storage bricks per axis = ceil((n-1)/8)
    int bs;         // log2 B, cells per skip-brick edge
    int der_stride; // floats per derived brick, der_brick_floats(bs)
    float s[3];     // spacing (mm)
    const float* bricks;     // storage bricks x kBrickVox
    const float* vbricks;    // vesselness storage bricks (same layout) or nullptr
    const float* dbricks;    // derived skip bricks or nullptr (then the per-sample stencils are used)
    const uint8_t* empty;    // skip-brick flags, 1 = skip
    const uint32_t* cellmask;  // skip bricks x cell_words(bs) words, bit (lz*B+ly)*B+lx set when that
                               // cell is empty under the current transfer function (nullptr before
                               // the precompute)
    const VolConst* vc;
};

// Per-launch constants of the ray setup, computed once on the host in FP64 and
// passed as double-floats (hi + lo).
struct RayConsts {
    dfloat_h two_over_w, two_over_h;  // 2/W, 2/H
    dfloat_h inv_s[3];                // 1/spacing
    dfloat_h dt;                      // sample spacing step_vox * min(s)
    float inv_dt;                     // 1/dt (only for the sample-count estimate)
};

inline RayConsts make_ray_consts(int W, int H, const float s[3], float step_vox) {
    RayConsts c;
    c.two_over_w = df_split(2.0 / (double)W);
    c.two_over_h = df_split(2.0 / (double)H);
    for (int q = 0; q < 3; ++q) c.inv_s[q] = df_split(1.0 / (double)s[q]);
    const float smin = s[0] < s[1] ? (s[0] < s[2] ? s[0] : s[2]) : (s[1] < s[2] ? s[1] : s[2]);
    const double dt = (double)step_vox * (double)smin;
    c.dt = df_split(dt);
    c.inv_dt = (float)(1.0 / dt);
    return c;
}

struct RenderLaunch {
    VolumeDev vol;
    TissueDev tp;
    RayConsts rc;
    const float* tf;           // [tf_h][tf_w][4]
    float* out;                // [n_cams][H][W][4]
    vr_counters* counters;     // nullable
    unsigned* ray_samples;     // nullable, [n_cams][H][W][2]
    float2* ray_state;         // nullable, [n_cams][H][W]: (last sample index as int bits, transmittance before it)
    int W, H, n_cams, cam_offset;
    int skip;
    int packet_w, packet_h;    // ray packet of a warp (packet_w * packet_h == 32); per-lane kernels: 4, 8 or 16 wide
    int tile_w, tile_h;        // per-lane kernels: CTA tile in pixels (tile_packets_x packets across)
    int tile_sx;               // log2 of the packets across the tile
    unsigned* work_counter;    // staged kernel work queue (zeroed before launch)
    unsigned* status;          // device status word (kStatusTimeout on an expired wait)
    int n_packets_x, n_packets_y, n_work;
    CamDev cams[kMaxCamsPerLaunch];
};

// CTA tile of a per-lane kernel: `warps` warp packets of packet_w x (32 / packet_w)
// rays (packet_w in {4, 8, 16}), min(warps, 16 / packet_w) packets across and the
// rest down: 4 warps give 16 x 8 pixels for every packet shape, 2 warps 8 x 8 or
// 16 x 4, 8 warps 16 x 16.
__host__ __device__ __forceinline__ int tile_packets_x(int packet_w, int warps) {
    return warps < 16 / packet_w ? warps : 16 / packet_w;
}

// Pixel offset (di, dj) of lane l of warp w within that tile (2^sx packets across).
__device__ __forceinline__ void tile_pixel(int packet_w, int sx, int w, int l, int& di, int& dj) {
    const int pl = __ffs(packet_w) - 1;  // log2 packet_w
    const int wx = w & ((1 << sx) - 1), wy = w >> sx;
    di = (wx << pl) + (l & (packet_w - 1));
    dj = wy * (32 >> pl) + (l >> pl);
}

// floats per lookup cell in a private copy of the transfer-function gradient
constexpr int kTfCellFloats = 16;

struct BackwardLaunch {
    RenderLaunch r;
    const float* dl_drgba;  // [n_cams][H][W][4] upstream gradient
    float* dtf;             // [tf_h][tf_w][4], zeroed by the caller
    float* dparams;         // gamma, ka, kd, ks, opacity_scale, zeroed by the caller
    float* dvol;            // nvox or nullptr, zeroed by the caller
    float* dtf_copies;      // n_copies zeroed private copies of the transfer-function gradient, one
                            // 16-float record per lookup cell (TfGradSink); CTA c adds into copy c % n_copies
    int n_copies;
    float* dgrad;           // derived-brick path with dvol: zeroed channel gradients (10 floats per voxel
                            // in three planes, chan_index), else nullptr
};

// One view of a batched render (device-resident table).
struct ViewDev {
    VolumeDev vol;
    TissueDev tp;
    RayConsts rc;
    const float* tf;
    CamDev cam;
    float* out;     // [H][W][4]
    int W, H;
};

struct BatchLaunch {
    const ViewDev* views;
    const int* packet_prefix;  // n_views entries: first packet of each view
    int n_views, n_work;
    int packet_w, packet_h;
    unsigned* work_counter;    // zeroed before every launch
    vr_counters* counters;     // nullable
    int skip;
};

// Record `msg` as the context's last error and return `status`.
vr_status set_error(vr_ctx* ctx, vr_status status, const char* msg);

// ---------------------------------------------------------------- launchers
// All return cudaSuccess or the launch error; all enqueue on `st`.
cudaError_t launch_minmax_partials(const void* data, vr_dtype dt, long long n, float* partials, int nblocks,
                                   cudaStream_t st);
cudaError_t launch_minmax_final(const float* partials, int nblocks, float* out2, cudaStream_t st);
int minmax_blocks(long long n);

cudaError_t launch_normalize(const void* raw, vr_dtype dt, long long n, const float* minmax2, VolConst* vc,
                             float* norm, cudaStream_t st);
// Storage bricks (8^3 cells) of `nb` storage bricks per axis.
cudaError_t launch_make_bricks(const float* norm, const int n[3], const int nb[3], float* bricks, cudaStream_t st);
// Skip bricks of 2^bs cells per edge, `nb` per axis.
cudaError_t launch_brick_minmax(const float* norm, const int n[3], const int nb[3], int bs, uint16_t* grid,
                                cudaStream_t st);
cudaError_t launch_make_derived(const float* norm, const int n[3], const int nb[3], int bs, const float s[3],
                                float* dbricks, cudaStream_t st);
cudaError_t launch_gmax(const float* norm, const int n[3], const float s[3], VolConst* vc, cudaStream_t st);
cudaError_t launch_classify(const uint16_t* grid, long long nbricks, const float* tf, int tf_w, int tf_h,
                            uint8_t* empty, int* prefix_scratch /* tf_w + 1 ints */, cudaStream_t st);
cudaError_t launch_cell_minmax(const float* norm, const int n[3], const int nb[3], int bs, uint16_t* cellq,
                               cudaStream_t st);
cudaError_t launch_classify_cells(const uint16_t* cellq, long long nbricks, int bs, const int* prefix, int tf_w,
                                  uint32_t* cellmask, cudaStream_t st);

// Multi-scale vesselness of `norm` into V (both nvox floats); tmp_a and tmp_b are
// nvox floats of scratch each, smax receives each scale's max Hessian norm.
cudaError_t launch_frangi(const float* norm, const int n[3], const float* sigmas, int n_sigmas, float* tmp_a,
                          float* tmp_b, float* smax, float* V, cudaStream_t st);

// 256-bin histogram of the normalised volume (zeroes hist first) and its three tissue peaks
// (peaks4 = three ascending bins, -1 padded, then the count).
cudaError_t launch_histogram(const float* norm, long long n, unsigned long long* hist, cudaStream_t st);
cudaError_t launch_tissue_peaks(const unsigned long long* hist, int lo, int hi, int* peaks4, cudaStream_t st);

// Pre-filters: 3x3x3 median; separable Gaussian (out = G * in, tmp is scratch; in != out).
cudaError_t launch_median3(const float* in, float* out, const int n[3], cudaStream_t st);
cudaError_t launch_gauss3d(const float* in, float* out, float* tmp, const int n[3], float sigma, cudaStream_t st);

// warps: warps per CTA (2, 4 or 8), tiled by tile_pixel.
cudaError_t launch_render_gather(const RenderLaunch& L, int warps, cudaStream_t st);
cudaError_t launch_render_backward(const BackwardLaunch& B, bool staged, cudaStream_t st);
// dtf += the entries' shares of the cell records of every copy
cudaError_t launch_sum_copies(const float* copies, int n_copies, int tf_w, int tf_h, float* dtf, cudaStream_t st);
cudaError_t launch_fma_peak(float* out, int blocks, int iters, cudaStream_t st);
cudaError_t launch_wait_probe(unsigned* status, long long budget_cycles, cudaStream_t st);
// One thread fails one index check (debug builds record it; release builds do nothing).
cudaError_t launch_check_probe(unsigned* status, cudaStream_t st);
cudaError_t launch_channels_to_voxels(const float* dgrad, const int n[3], const float s[3], float* dvol,
                                      cudaStream_t st);
// bs: the skip-brick size (log2 cells) every view shares, or 0 when they differ.
cudaError_t launch_render_batch(const BatchLaunch& B, int warps_per_block, int ctas, bool all_derived, int bs,
                                cudaStream_t st);
cudaError_t batch_ctas_per_sm(int warps_per_block, bool all_derived, int* per_sm);
cudaError_t launch_render_staged(const RenderLaunch& L, int warps_per_block, int ctas, cudaStream_t st);
// The staged design on the derived bricks (skip bricks of 4^3 or 8^3 cells, bs 2 or 3).
cudaError_t launch_render_staged_derived(const RenderLaunch& L, int warps_per_block, int ctas, cudaStream_t st);
int staged_derived_smem_bytes(int warps_per_block, int bs);
cudaError_t staged_derived_config(int warps_per_block, int bs, int* ctas_per_sm);
int staged_smem_bytes(int warps_per_block, bool vessel);
// Set the kernel's dynamic shared-memory limit and report resident CTAs per SM.
cudaError_t staged_config(int warps_per_block, bool vessel, int* ctas_per_sm);

}  // namespace vr

/*
 * vr.h -- C ABI of the GB300 direct-volume-rendering library (libvr.so).
 *
 * The calls follow the problem statement of Beckley, "Decentralized Direct
 * Volume Rendering: A Browser-Native GPU Architecture for MRI Digital Twins"
 * (arXiv 2605.19737): a volume is loaded with its dims and spacing and
 * min-max normalised (Sec. 2.2, Eq. 1); its morphology is precomputed once
 * (Sec. 2.3; the multi-scale Hessian vesselness of Sec. 1); tissue windows and
 * transfer-function uniforms change without recomputation (abstract, Sec. 4,
 * Sec. 5.4); a single-pass front-to-back raymarch turns a camera into an RGBA
 * image (Sec. 2.4, Eqs. 4-6); and an adjoint raymarch returns gradients of a
 * loss on that image.
 *
 * Conventions shared by every call:
 *   - Volumes are dense, x fastest: voxel (i,j,k) at (k*ny + j)*nx + i, its
 *     centre at ((i+.5)sx, (j+.5)sy, (k+.5)sz) in mm; the volume fills the box
 *     [0, nx sx] x [0, ny sy] x [0, nz sz]. 2 <= nx, ny, nz <= 2048.
 *   - Images are premultiplied RGBA float32, [n_cams][H][W][4], row 0 = top,
 *     black transparent background.
 *   - Ownership: the caller owns every buffer it passes; the library copies
 *     what it keeps (volume, transfer function) into device memory it owns
 *     and frees in vr_free_volume / vr_destroy.
 *   - Pointers named d_* are device pointers on the context's device; h_* are
 *     host pointers; others say which in their comment.
 *   - Asynchrony: work is enqueued on the context's CUDA stream. Argument
 *     errors return at once; errors raised by kernels surface at the next
 *     vr_synchronize (or at a call that must read results back).
 *   - No call aborts, throws or prints. On failure the returned status is
 *     non-zero and vr_last_error(ctx) describes it.
 *   - One context per host thread; a context is not thread-safe.
 */
#ifndef VR_H
#define VR_H

#ifdef __cplusplus
extern "C" {
#endif

#define VR_ABI_VERSION 1

typedef struct vr_ctx vr_ctx;

typedef enum {
    VR_OK = 0,
    VR_ERR_INVALID_ARG = 1, /* bad pointer, size, id or parameter value */
    VR_ERR_NOT_READY = 2,   /* a required earlier call has not been made */
    VR_ERR_CUDA = 3,        /* a CUDA runtime call or a kernel failed */
    VR_ERR_OOM = 4,         /* device allocation failed */
    VR_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    VR_ERR_DEGENERATE = 6,  /* I_max == I_min: Eq. 1 is undefined */
    VR_ERR_BOUNDS = 7       /* debug library only: a kernel's index check failed */
} vr_status;

typedef enum { VR_F32 = 0, VR_U16 = 1 } vr_dtype;

/* A pinhole camera. fwd is the unit viewing direction; right and up are
 * pre-scaled by tan(fov/2)*aspect and tan(fov/2), so pixel (i, j) looks along
 * normalize(fwd + a*right + b*up), a = 2(i+1/2)/W - 1, b = 1 - 2(j+1/2)/H. */
typedef struct {
    float eye[3];
    float fwd[3];
    float right[3];
    float up[3];
} vr_camera;

typedef enum {
    VR_TF_1D = 0,        /* opacity/colour over I_norm (tf_h == 1) */
    VR_TF_2D_GRAD = 1,   /* over (I_norm, |grad I| / |grad I|_max) */
    VR_TF_2D_VESSEL = 2  /* over (I_norm, V): the vesselness, or a second channel
                            (vr_load_second_channel); needs one of them */
} vr_tf_mode;

/* Tissue and transfer-function uniforms (Sec. 2.4, Eq. 4; Table 2 windows are
 * encoded in the table). Per sample at normalised intensity I:
 *   (r,g,b,a) = tf(I [, second axis])         piecewise-linear lookup
 *   m_g       = grad_mod ? min(|g|/|g|max, 1) : 1
 *   w(kappa)  = clamp(1 + gamma*kappa/kappa_ref, 0, w_max),  kappa = g^T H g/|g|^2
 *   alpha     = clamp(opacity_scale * a * m_g * w, 0, 1)     (Eq. 4)
 *   colour    = shading ? rgb*(ka + kd*d) + ks*d^16 : rgb,   d = |g/|g| . dir|
 * Samples are spaced step_vox * min(s) mm apart (step_vox in [0.01, 16]); a ray stops after the first
 * sample whose accumulated opacity reaches et_threshold (> 1 disables). */
typedef struct {
    int tf_mode;        /* vr_tf_mode */
    int tf_w;           /* entries along I_norm, 2..4096 (256 typical) */
    int tf_h;           /* entries along the second axis: 1 for 1D, 2..256 for 2D */
    const float* tf;    /* [tf_h][tf_w][4] RGBA float32; host or device (tf_on_device) */
    int tf_on_device;
    int grad_mod;       /* 0 or 1 */
    int shading;        /* 0 or 1 */
    float gamma, kappa_ref, w_max;
    float ka, kd, ks;
    float opacity_scale, et_threshold, step_vox;
    float opacity_ref_step; /* mm; > 0: alpha' = 1 - (1 - alpha)^(dt / opacity_ref_step)
                               makes the image independent of the sample spacing dt;
                               0 (default): Eqs. 5-6 as printed */
} vr_tissue_params;

/* Device-side counters a render may add into (zero them yourself first). */
typedef struct {
    unsigned long long rays;              /* rays that hit the volume box */
    unsigned long long dense_samples;     /* sample points up to each ray's stop */
    unsigned long long evaluated_samples; /* of those, not in skipped bricks */
    unsigned long long bricks_staged;     /* brick copies into shared memory */
    unsigned long long shaded_samples;    /* of the evaluated, those whose transfer-function
                                             opacity was non-zero, so that the Hessian, Eq. 4
                                             and the shading were computed (the others add
                                             nothing; all of them for the stencil kernels) */
    unsigned long long interpolated_samples; /* of the evaluated, those whose field was read:
                                             all but the ones in cells classified empty (the
                                             per-lane kernels skip those cells, bit-neutral) */
} vr_counters;

typedef enum {
    VR_KERNEL_AUTO = 0,    /* the fastest measured on GB300 (gather) */
    VR_KERNEL_GATHER = 1,  /* per-lane reads of the bricked volume through L1: the voxel-wise
                              derivatives precomputed by vr_precompute_morphology (8 corners per
                              sample) when they fit the memory budget, else as GATHER_STENCIL */
    VR_KERNEL_STAGED = 2,  /* warp-cooperative brick staging in shared memory, per-sample stencils */
    VR_KERNEL_GATHER_STENCIL = 3, /* per-lane reads, per-sample stencils over the 56 weighted voxels
                                     of the cell's 4x4x4 neighbourhood (no derived data) */
    VR_KERNEL_STAGED_DERIVED = 4  /* warp-cooperative staging of derived skip bricks (4^3 or 8^3
                                     cells) in shared memory by bulk copy; no second channel */
} vr_kernel;

typedef struct {
    int kernel;         /* vr_kernel */
    int skip_empty;     /* 1: skip bricks classified empty (bit-neutral) */
    int packet_w;       /* rays per warp packet along x (packet = 32 rays): 4, 8 or 16 for the
                           per-lane kernels (default 4), also 32 for the staged and batched ones */
    int warps_per_block;/* warps per CTA: the per-lane kernels 2, 4 (default) or 8 -- their CTA
                           tile is min(warps, 16/packet_w) packets across and the rest down
                           (4 warps: 16 x 8 pixels); a render that records ray_state runs
                           at most 4 (8 is taken as 4: the image is the same); the staged
                           kernel 1..8 */
    void* ray_state;    /* NULL, or device memory of n_cams*H*W x 8 bytes (per-lane kernels
                           only): vr_render writes, per pixel, the index of the ray's last
                           sample (int32; -1 for none) and the transmittance in front of it
                           (float32); vr_render_backward with the same volume, tissue
                           parameters, cameras and size reads it instead of re-marching each
                           ray forward. Zero it when constructing the struct. */
} vr_render_opts;

/* ------------------------------------------------------------------ context */

/* Library version string, e.g. "vr 1.0 sm_103a". Never NULL. */
const char* vr_version(void);

/* Create a context on CUDA device `device` that enqueues its work on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).
 * *out receives the context. Errors: INVALID_ARG (out NULL, bad device), CUDA. */
vr_status vr_create(vr_ctx** out, int device, void* cuda_stream);

/* Synchronise, free every buffer the context owns, destroy it. NULL is a no-op. */
vr_status vr_destroy(vr_ctx* ctx);

/* Switch the stream later calls enqueue on. */
vr_status vr_set_stream(vr_ctx* ctx, void* cuda_stream);

/* Wait for the context's stream; report asynchronous kernel errors and the
 * device status word (TIMEOUT if a bounded wait expired). */
vr_status vr_synchronize(vr_ctx* ctx);

/* Message for the last non-OK status of this context ("" if none). */
const char* vr_last_error(vr_ctx* ctx);

/* ------------------------------------------------------------------ volumes */

/* Load a volume (Sec. 2.1 ingestion, Sec. 2.2 Eq. 1).
 *   data: nx*ny*nz values of `dtype`, x fastest; on the device if on_device,
 *         else in host memory (pinned memory makes the copy asynchronous).
 * The library copies the data, computes I_min/I_max with a parallel
 * reduction, writes the normalised volume and its 8^3-cell bricks (stored
 * 12^3 with a clamp-to-edge apron) and the quantised per-brick min/max grid.
 * *vol_id receives the volume's id. Synchronises once to check Eq. 1.
 * Errors: INVALID_ARG (dims outside [2, 2048], spacing <= 0 or not finite,
 * NULL pointers), DEGENERATE (I_max == I_min), OOM, CUDA. */
vr_status vr_load_volume(vr_ctx* ctx, const void* data, int on_device, vr_dtype dtype, int nx, int ny, int nz,
                         float sx, float sy, float sz, int* vol_id);

/* Load a single-file NIfTI-1 volume (.nii, either byte order; Sec. 2.1 ingests
 * NIfTI-1): the first 3D volume of dim[1..3], datatypes uint8, int8, int16,
 * uint16, int32, uint32, float32, float64; scl_slope/scl_inter applied when
 * the slope is non-zero; spacing |pixdim[1..3]| converted to mm from the
 * xyzt_units. uint16 data without scaling is loaded as VR_U16, everything else
 * as VR_F32, then as vr_load_volume. Errors: INVALID_ARG (unreadable file,
 * not NIfTI-1, unsupported datatype, dims outside [2, 2048]) and those of
 * vr_load_volume. */
vr_status vr_load_nifti(vr_ctx* ctx, const char* path, int* vol_id);

/* Header only, no context or GPU needed: dims (3 ints), spacing in mm
 * (3 floats) and the NIfTI datatype code; any output may be NULL. */
vr_status vr_nifti_info(const char* path, int* h_dims, float* h_spacing, int* h_datatype);

/* Free a volume and everything derived from it. */
vr_status vr_free_volume(vr_ctx* ctx, int vol_id);

/* Per-volume morphology (Sec. 2.3 and Sec. 1), run once per volume:
 * |grad I|_max over voxels (Eq. 4's normaliser, a parallel reduction); the
 * voxel-wise I, gradient and Hessian stored per brick for the raymarch (the
 * "derived bricks", 12 floats per corner voxel, within the context's derived
 * budget -- see vr_set_derived_budget) with each cell's quantised min/max; and,
 * when n_sigmas > 0, the multi-scale Frangi vesselness V = max over
 * h_sigmas[0..n_sigmas-1] (voxel units, each in (0, 8]) of the bright-vessel
 * response of the sigma^2-scaled Hessian of the Gaussian-smoothed volume,
 * alpha = beta = 0.5, c = half the largest Hessian norm at that scale.
 * Errors: INVALID_ARG, OOM, CUDA. */
vr_status vr_precompute_morphology(vr_ctx* ctx, int vol_id, const float* h_sigmas, int n_sigmas);

/* Second channel of a loaded volume: a co-registered scalar volume of the same
 * dims (a second MRI contrast or another modality, Sec. 5.4's multi-parametric
 * extension), normalised by its own I_min, I_max (Eq. 1) and bricked like the
 * first. It takes the place of the vesselness channel: VR_TF_2D_VESSEL then
 * renders over (I_norm, second channel), and whichever of this call and a
 * vr_precompute_morphology with n_sigmas > 0 ran last defines that channel.
 * data: nx*ny*nz values of `dtype`, x fastest, host or device (on_device);
 * copied. Reads I_min/I_max back (synchronises). Tissue params in mode 2 must be
 * set again afterwards. Errors: INVALID_ARG, DEGENERATE (a constant channel),
 * OOM, CUDA; after an error mode 2 is NOT_READY until a channel is loaded. */
vr_status vr_load_second_channel(vr_ctx* ctx, int vol_id, const void* data, int on_device, vr_dtype dtype);

/* Set transfer-function and tissue uniforms (copied), then re-classify the
 * bricks (and, with derived bricks, the cells) for empty-space skipping: two
 * small kernels, tens of microseconds. Nothing else is recomputed (the uniform
 * buffers of the abstract and Sec. 4). Errors: INVALID_ARG (bad sizes or
 * values), NOT_READY (mode 2 without vesselness or a second channel), OOM, CUDA.
 * Argument errors change nothing; after an OOM or CUDA error the volume is
 * NOT_READY for rendering until a call succeeds. */
vr_status vr_set_tissue_params(vr_ctx* ctx, int vol_id, const vr_tissue_params* tp);

/* I_min, I_max (Eq. 1) and |grad I|_max (Eq. 4) of a volume; any pointer may be
 * NULL. Reads back from the device (synchronises). gmax is 0 before
 * vr_precompute_morphology. */
vr_status vr_get_norm(vr_ctx* ctx, int vol_id, float* imin, float* imax, float* gmax);

/* Override |grad I|_max (e.g. to hold it fixed while a test perturbs voxels). */
vr_status vr_set_gmax(vr_ctx* ctx, int vol_id, float gmax);

/* Overwrite the normalised intensities of a loaded volume with
 * d_norm[nx*ny*nz] (device, float32, x fastest) and rebuild its bricks, derived
 * bricks (when built) and min/max grid; I_min/I_max and |grad I|_max are kept. Used to render or
 * differentiate a volume given directly in I_norm units. */
vr_status vr_set_normalized(vr_ctx* ctx, int vol_id, const float* d_norm);

/* Copy derived data to host memory (synchronises):
 *   h_grid: nbx*nby*nbz*2 uint16 (qlo, qhi) per brick, nb = ceil((n-1)/8);
 *   h_empty: nbx*nby*nbz bytes, 1 = brick skipped under the current params;
 *   h_nb: 3 ints (nbx, nby, nbz). Any of them may be NULL. */
vr_status vr_get_bricks(vr_ctx* ctx, int vol_id, unsigned short* h_grid, unsigned char* h_empty, int* h_nb);

/* Edge of the skip bricks of a volume, in interpolation cells: 4, 8 (the default)
 * or 16. The brick min/max grid, the empty-brick flags, the per-cell empty bits and
 * the derived bricks of the voxel-wise derivatives are kept per skip brick; empty
 * skip bricks are jumped a brick at a time. Rebuilds the grid at once; the volume
 * then needs vr_precompute_morphology again (NOT_READY until then), which also
 * re-classifies under the current tissue parameters. The images do not depend on
 * the size (skipping is bit-neutral); the evaluated-sample counter does. The
 * staged kernels (VR_KERNEL_STAGED) need 8. Synchronises.
 * Errors: INVALID_ARG (unknown volume, other sizes), OOM, CUDA. */
vr_status vr_set_brick_size(vr_ctx* ctx, int vol_id, int cells);

/* Storage layout of a volume (no GPU work; any pointer may be NULL):
 *   nbricks:       skip bricks (vr_set_brick_size), nbx*nby*nbz;
 *   brick_bytes:   the intensity brick store (8^3-cell storage bricks, 12^3 float32 each);
 *   derived_bytes: the derived-brick store of the voxel-wise derivatives built by
 *                  vr_precompute_morphology (0 when it is not built).
 * Errors: INVALID_ARG (unknown volume). */
vr_status vr_get_layout(vr_ctx* ctx, int vol_id, long long* nbricks, unsigned long long* brick_bytes,
                        unsigned long long* derived_bytes);

/* Copy the second channel -- the vesselness volume, or the normalised channel of
 * vr_load_second_channel -- (nx*ny*nz float32) to `out` (device if
 * out_on_device, else host; synchronises for host). NOT_READY without it. */
vr_status vr_get_vesselness(vr_ctx* ctx, int vol_id, float* out, int out_on_device);

/* Copy the normalised volume (nx*ny*nz float32) to `out` (as above). */
vr_status vr_get_normalized(vr_ctx* ctx, int vol_id, float* out, int out_on_device);

/* Optional pre-filter of the normalised volume (the light smoothing or median
 * passes proposed in Sec. 5.3 against low SNR and impulsive artefacts):
 * mode 1 = 3x3x3 median (clamp-to-edge; exact order statistic), mode 2 =
 * separable Gaussian with sampled normalised weights on [-ceil(4 sigma),
 * ceil(4 sigma)] voxels, sigma in (0, 8]. The filtered intensities replace the
 * volume's I_norm (I_min/I_max of Eq. 1 are kept), bricks and the brick grid are
 * rebuilt and re-classified; morphology (|grad I|max, vesselness) must be
 * recomputed with vr_precompute_morphology before the next render.
 * Errors: INVALID_ARG, OOM, CUDA. */
vr_status vr_prefilter(vr_ctx* ctx, int vol_id, int mode, float sigma);

/* The 256-bin density analysis of Sec. 2.2: d_hist[256] (device, uint64) receives
 * the counts of bin min(floor(I_norm * 256), 255) over all voxels (I_norm in
 * float32 as stored for the volume). When d_peaks (device, 4 ints) is not NULL,
 * the tri-modal tissue peaks behind Tables 1-2 are extracted too: the histogram
 * is smoothed with the integer binomial kernel [1 4 6 4 1] (clamp at the ends), a
 * bin j in [max(lo_bin, 1), min(hi_bin, 254)] is a peak when s[j] > s[j-1] and
 * s[j] >= s[j+1], the three largest peaks (ties to the lower bin) are written in
 * ascending order to d_peaks[0..2] (-1 where fewer exist) and their count to
 * d_peaks[3]. The bin of peak p covers I_norm in [p/256, (p+1)/256). Choose
 * [lo_bin, hi_bin] to exclude the background and fat modes. Asynchronous.
 * Errors: INVALID_ARG (unknown volume, NULL histogram, bins outside [0, 255]). */
vr_status vr_tissue_histogram(vr_ctx* ctx, int vol_id, int lo_bin, int hi_bin, unsigned long long* d_hist,
                              int* d_peaks);

/* Global min and max of n values (the parallel reduction of Sec. 4 applied to
 * Eq. 1's I_min, I_max): d_data holds n values of `dtype` on the device;
 * d_out2[0] = min, d_out2[1] = max as float32 (device). Asynchronous; uses
 * partial results in scratch memory the context owns (allocated on first
 * use, grown as needed). Errors: INVALID_ARG (n < 1, NULL), OOM, CUDA. */
vr_status vr_reduce_minmax(vr_ctx* ctx, const void* d_data, vr_dtype dtype, long long n, float* d_out2);

/* ---------------------------------------------------------------- rendering */

/* Render n_cams images (Sec. 2.4): per pixel one ray, samples at
 * t_near + (k+1/2) dt, per sample the trilinear field and its gradient and
 * Hessian (Eqs. 2-3), opacity by Eq. 4, front-to-back compositing by
 * Eqs. 5-6, early termination, and empty-space skipping.
 *   h_cams: n_cams cameras in host memory (copied at launch).
 *   out_rgba: n_cams*H*W*4 float32 -- device memory, or host memory when
 *             out_on_host: page-locked (pinned) host memory is written by the
 *             kernel itself through its device mapping, other host memory through
 *             a device staging buffer and a copy back on the stream. Either way
 *             the image is complete after the next vr_synchronize.
 *   opts: NULL for defaults (fastest kernel, skipping on).
 *   d_counters: NULL or device vr_counters to add into.
 *   d_ray_samples: NULL or device uint32 [n_cams][H][W][2] receiving each
 *             ray's dense and evaluated sample counts.
 * Errors: INVALID_ARG (n_cams < 1, W or H outside [1, 16384], a ray_state with
 * the staged kernel), NOT_READY
 * (no vr_precompute_morphology or vr_set_tissue_params yet), OOM, CUDA. */
vr_status vr_render(vr_ctx* ctx, int vol_id, const vr_camera* h_cams, int n_cams, int W, int H, float* out_rgba,
                    int out_on_host, const vr_render_opts* opts, vr_counters* d_counters,
                    unsigned int* d_ray_samples);

/* Adjoint of vr_render (the paper renders; differentiating the same
 * Eqs. 2-6 turns its interactive tissue-parameter tuning into fitting those
 * parameters to a target view). For a loss L with image gradient
 * d_dl_drgba = dL/dRGBA ([n_cams][H][W][4] float32, device) of the image
 * vr_render would produce for the same cameras and uniforms, writes
 *   d_dtf:     dL/d(transfer-function entries), [tf_h][tf_w][4] float32;
 *   d_dparams: NULL or dL/d(gamma, ka, kd, ks, opacity_scale), 5 float32 (NULL:
 *              not computed; without a curvature term, gamma = 0, the Hessian
 *              then enters no output and is not read);
 *   d_dvolume: NULL or dL/d(normalised voxel intensity), nx*ny*nz float32.
 * All outputs are device memory and are overwritten. I_min, I_max,
 * |grad I|_max, the vesselness volume and each ray's stopping sample are
 * held fixed. Per ray the kernel re-marches forward, then sweeps back to front
 * rebuilding the transmittance by division (accurate while et_threshold stays
 * at or below ~0.999), re-evaluating each sample instead of storing it. The
 * reverse sweep visits every sample, empty bricks included: a zero-opacity
 * sample still gives the opacity entries it reads a gradient.
 * opts: NULL or as vr_render: skip_empty applies to the forward re-march only,
 * where it is exact; a non-NULL ray_state (written by the vr_render of this image)
 * replaces the re-march: each ray's reverse sweep starts from its recorded last
 * sample and transmittance (per-lane kernels only); kernel VR_KERNEL_STAGED sweeps brick by brick and sums voxel
 * gradients in shared memory before global atomics (per-sample stencils), any
 * other value (default) sweeps each lane independently and adds voxel gradients
 * with global atomics, evaluating samples from the derived bricks when they exist
 * except under VR_KERNEL_GATHER_STENCIL (same sample field up to rounding; the
 * default is the faster one measured). The voxel gradient is always the exact
 * transpose of the per-sample stencils. Errors as vr_render; a kernel value
 * outside 0..3 is VR_ERR_INVALID_ARG. */
vr_status vr_render_backward(vr_ctx* ctx, int vol_id, const vr_camera* h_cams, int n_cams, int W, int H,
                             const float* d_dl_drgba, float* d_dtf, float* d_dparams, float* d_dvolume,
                             const vr_render_opts* opts);

/* Allocation-free variant of the brick classification that vr_set_tissue_params
 * runs. The paper has no counterpart; it exists for callers that cannot allocate
 * device memory when they re-classify (a fixed pre-reserved memory budget, a
 * real-time thread that must stay out of the allocator). No context is needed and
 * nothing is allocated: the kernels' scratch (tf_w + 1 prefix counts) lives in a
 * 16 KB static device array built into the library, which every GPU that loads
 * the library holds until the process exits.
 *   d_grid:  nbricks x (qlo, qhi) uint16, as vr_get_bricks returns (device);
 *   d_tf:    [tf_h][tf_w][4] float32 transfer function (device);
 *   d_empty: nbricks bytes out, 1 = brick skippable (device), identical to the
 *            flags vr_set_tissue_params computes for the same grid and table;
 *   cuda_stream: stream to enqueue on (NULL = legacy default stream), on the
 *            current CUDA device;
 *   h_msg/msg_len: NULL or a host buffer that receives a message on failure.
 * The first call on a device looks up the static array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture. The
 * address is kept per device together with the id of the CUDA context it was
 * taken in: after the context is destroyed and re-created (cudaDeviceReset), the
 * next call sees the new context and looks the address up again, so that call
 * too should come before any capture.
 * All calls share the one array per device, so calls that overlap on the GPU
 * (e.g. on two streams) race; every call rewrites all the entries it reads.
 * Errors: INVALID_ARG (NULL pointers, nbricks outside [1, 2^31], tf_w outside
 * [2, 4096] -- the most the static scratch holds -- or tf_h outside [1, 256]),
 * CUDA. Asynchronous otherwise. */
vr_status vr_classify_bricks_noalloc(const unsigned short* d_grid, long long nbricks, const float* d_tf, int tf_w,
                                     int tf_h, unsigned char* d_empty, void* cuda_stream, char* h_msg, int msg_len);

/* ------------------------------------------------------- batched rendering */

/* One view of a batch: a camera on a loaded volume, rendered into its own
 * device image d_out ([H][W][4] float32, caller-owned). */
typedef struct {
    int vol_id;
    vr_camera cam;
    float* d_out;
    int W, H;
} vr_view;

/* Register a batch of views (any mix of volumes, cameras and image sizes).
 * The view table -- each volume's bricks, skip flags, transfer-function buffer
 * and uniforms at this moment, plus the cameras and outputs -- is uploaded once
 * to device memory (synchronises). Re-upload with vr_batch_update after
 * vr_set_tissue_params, and after a vr_precompute_morphology that adds or drops
 * a member volume's derived bricks (vr_set_derived_budget); vr_free_volume of a
 * member volume invalidates the batch. Errors: INVALID_ARG (unknown volume, bad size or output), NOT_READY
 * (a volume without morphology or tissue params), OOM, CUDA. */
vr_status vr_batch_create(vr_ctx* ctx, const vr_view* views, int n_views, int* batch_id);
vr_status vr_batch_update(vr_ctx* ctx, int batch_id);
vr_status vr_batch_free(vr_ctx* ctx, int batch_id);

/* Render every view of the batch in one persistent launch: warps pull
 * 32-ray packets (opts->packet_w x 32/packet_w pixels, packet_w in {4, 8, 16, 32})
 * from a single work queue spanning all views; opts->warps_per_block in [1, 8]
 * (NULL opts: 8 x 4 packets, 8 warps per CTA). The grid is sized to the SMs
 * times the resident CTAs per SM. Enqueues one memset and one kernel, with no
 * host synchronisation or allocation, so it may be captured into a CUDA graph
 * (capture of the legacy default stream is not possible). Results equal
 * vr_render of each view bit for bit. */
vr_status vr_batch_render(vr_ctx* ctx, int batch_id, const vr_render_opts* opts, vr_counters* d_counters);

/* As vr_batch_render, from a CUDA graph that the library captures once per
 * (batch, packet shape, warps, skip) on a private stream and replays; ordered
 * after earlier work on the context's stream and before later work. */
vr_status vr_batch_render_graph(vr_ctx* ctx, int batch_id, const vr_render_opts* opts);

/* Memory budget for the derived bricks (per-voxel I, gradient and Hessian, 12
 * floats per corner voxel of each brick: about 5x the intensity bricks) that
 * vr_precompute_morphology builds for the raymarch. A volume whose derived store
 * would exceed `bytes` gets none -- its renders and gradients evaluate the
 * per-sample stencils of the intensity bricks instead (same field up to
 * rounding) -- and a later vr_precompute_morphology frees one it already has.
 * Default 16 GiB; 0 disables derived bricks. Applies to subsequent
 * vr_precompute_morphology calls of this context. Errors: INVALID_ARG (NULL ctx). */
vr_status vr_set_derived_budget(vr_ctx* ctx, unsigned long long bytes);

/* Exercise the timeout path of the bounded device-side waits without faulting or
 * hanging the GPU (the paper has no counterpart). Launches, on the context's
 * stream, one CTA whose thread waits on an mbarrier phase that nothing completes,
 * giving up after budget_cycles SM clocks (1..2^31; ~2^31 is about a second), and
 * records the expired wait in the context's device status word exactly as a
 * bulk copy that never landed would: the next vr_synchronize returns
 * VR_ERR_TIMEOUT and clears the word, and the context stays usable.
 * Errors: INVALID_ARG (budget out of range), CUDA. Asynchronous. */
vr_status vr_probe_bounded_wait(vr_ctx* ctx, long long budget_cycles);

/* 1 in the debug library (libvr_debug.so, built with VR_DEBUG), 0 in libvr.so.
 * The debug library checks the indices of the raymarch kernels' memory accesses
 * (brick coordinates, transfer-function cells, voxel and image offsets, the
 * staged kernel's shared-memory slots, batch view ids); a failed check skips the
 * access, sets a bit in the context's device status word and records the source
 * line, and the next vr_synchronize returns VR_ERR_BOUNDS with that line in
 * vr_last_error. It computes the same images as libvr.so; libvr.so compiles the
 * checks away. */
int vr_debug_build(void);

/* Exercise the debug library's index-check reporting: one thread fails one check
 * (no memory is accessed either way), so the next vr_synchronize returns
 * VR_ERR_BOUNDS in the debug library and VR_OK in libvr.so. Asynchronous.
 * Errors: CUDA. */
vr_status vr_debug_check_probe(vr_ctx* ctx);

/* Device memory held by the context: every buffer the library allocates for it
 * (volumes, derived bricks, cell grids, vesselness, batches, scratch) is counted
 * in *bytes; caller-owned buffers (images, counters, ray state) are not. */
vr_status vr_memory_used(vr_ctx* ctx, unsigned long long* bytes);

/* Cap on vr_memory_used (0, the default: no cap beyond the device's memory). An
 * allocation that would take the context past the cap fails as a cudaMalloc
 * would: the call that needed it returns VR_ERR_OOM and releases nothing it did
 * not allocate. Derived bricks are optional: a precompute that cannot get them
 * under the cap renders from the per-sample stencils instead (same images within
 * rounding). Lowering the cap below the current use frees nothing. */
vr_status vr_set_memory_limit(vr_ctx* ctx, unsigned long long bytes);

/* Fault injection for the out-of-memory paths (host side; nothing faults on the
 * GPU): the next n_ok device allocations of the context succeed and the one
 * after them fails as out of memory, once; n_ok = -1 cancels. *pending (may be
 * NULL) receives the setting this call replaces: the allocations that were still
 * to succeed before the injected failure, or -1 once it has happened (or when
 * none was set). After a failed
 * call the context and its other objects stay usable: a vr_load_volume that
 * failed leaves no volume behind; a vr_precompute_morphology or
 * vr_set_tissue_params that failed leaves the volume NOT_READY for rendering
 * until the call is repeated successfully; a failed backward or batch call
 * changes nothing. Errors: INVALID_ARG (n_ok < -1). */
vr_status vr_debug_fail_alloc(vr_ctx* ctx, long long n_ok, long long* pending);

/* Measure the device's FP32 FMA throughput (the paper has no counterpart; it is
 * the roof the raymarch's arithmetic is reported against, since the raymarch is
 * bound by the FP32 pipe and L1 rather than HBM). Launches, on the context's
 * stream, `blocks` CTAs of 256 threads that each run 8 independent FMA chains for
 * iters x 16 steps, `reps` times after one warm-up launch, timing each with CUDA
 * events; synchronises. Writes the median launch time (ms) and the FLOPs of one
 * launch (blocks * 256 * iters * 256). Allocates and frees a scratch output.
 * Errors: INVALID_ARG (NULL pointers, blocks outside [1, 2^20], iters outside
 * [1, 2^20], reps outside [1, 64]), OOM, CUDA. */
vr_status vr_fma_peak(vr_ctx* ctx, int blocks, int iters, int reps, float* h_ms, double* h_flops);

#ifdef __cplusplus
}
#endif
#endif /* VR_H */

/*
 * hm.h -- C ABI of the B300-native hybrid mesh-Gaussian renderer.
 *
 * The library renders the hybrid representation of "Hybrid Mesh-Gaussian
 * Representation for Efficient Indoor Scene Reconstruction" (arXiv
 * 2506.06988): an opaque textured triangle mesh gives per-pixel colour I_m and
 * depth D_m (Sec. 3.4 "Joint rasterization"); 3D Gaussians (Eq. 1, with
 * Sigma = R S S^T R^T and the EWA projection Sigma' = J W Sigma W^T J^T of
 * Sec. 3.1) are alpha-blended front to back (Eq. 2) only while they lie in
 * front of the mesh (D_gs < D_m), and the remaining transmittance T weights
 * the mesh colour, or the background I_bg where no triangle covers the pixel:
 *     I_h = I_gs + T * I_m   (triangle)      I_h = I_gs + T * I_bg   (none).
 * The texture map is optimisable (Sec. 3.4): the backward pass returns
 * gradients for the texels as well as for the Gaussian parameters.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every array argument is a DEVICE pointer owned by the caller, except
 *    `cams` and `opt`, which are HOST pointers read during the call.  The
 *    library allocates nothing; scratch memory is a caller-provided workspace
 *    of at least the size returned by the matching *_workspace_size query.
 *  - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *    NULL = legacy default stream) and capturable into a CUDA graph.
 *  - Return value: host-side status (argument validation, launch errors).
 *    Errors found on the device (pair capacity exceeded, a bounded wait that
 *    gave up) are OR-ed into the caller's device word `d_status` (HM_DEV_*
 *    bits), to be read after the stream is synchronised.
 *  - Camera k renders into a contiguous block of pixels starting at the sum
 *    of the previous cameras' width*height; per-pixel outputs are float32 or
 *    uint32 in row-major order; colour images are planar per camera
 *    ([3][height][width] at 3x the pixel offset).  Per-tile outputs start at
 *    the sum of the previous cameras' tile counts, tiles row-major.
 *  - Gaussian data of camera k, Gaussian i lives at record index k*n + i.
 *  - Parameters are the activated values: scales = exp(log-scale),
 *    opacity = sigmoid(logit); quaternions (w,x,y,z) need not be normalised.
 *  - A pixel (x,y) is sampled at its centre (x+1/2, y+1/2).
 */
#ifndef HM_H
#define HM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t hm_status;

/* host-side return codes */
#define HM_OK 0
#define HM_ERR_INVALID_ARG 1   /* bad size, null required pointer, unsupported option */
#define HM_ERR_CUDA 2          /* a CUDA launch or runtime call failed */
#define HM_ERR_WORKSPACE 3     /* ws_bytes smaller than the *_workspace_size query */

/* device status bits (OR-ed into *d_status) */
#define HM_DEV_CAPACITY 1      /* more (Gaussian,tile) or (face,tile) pairs than capacity */
#define HM_DEV_TIMEOUT 2       /* a bounded wait (inter-CTA look-back, or a bulk copy's
                                  barrier) gave up; outputs are invalid */
#define HM_DEV_BAD_INDEX 4     /* a pair list held a record index >= n_views*n (a list
                                  left invalid by an earlier error); record 0 was read
                                  in its place and the outputs are invalid */

#define HM_MAX_VIEWS 32        /* cameras per call */
#define HM_MAX_PAIRS 0x3FFFFFFF /* pair capacities must stay below 2^30 */

/* texture formats */
#define HM_TEX_RGB8 0          /* [tex_h][tex_w][3] uint8, value/255 */
#define HM_TEX_RGBF32 1        /* [tex_h][tex_w][3] float32 */

/* SH storage formats */
#define HM_SH_F32 0
#define HM_SH_F16 1            /* IEEE binary16, widened in-kernel */

/* Pinhole camera, world -> camera: p_cam = R p_world + t (R row-major);
 * OpenCV axes (+x right, +y down, +z forward); u = fx X/Z + cx. */
typedef struct hm_camera {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height;
} hm_camera;

typedef struct hm_options {
    int32_t tile_w, tile_h;  /* screen tile: 16x16, 32x8 or 8x8 */
    int32_t batch;           /* list entries staged in shared memory per round by the
                                blend kernels (forward; the backward stages at most
                                64): 1 .. tile pixels; the results do not depend on it */
    int32_t mesh_cull;       /* 1: drop (Gaussian, tile) pairs at or behind the tile's
                                farthest mesh depth (result-preserving) */
    float near_gauss;        /* Gaussians with FP32 view depth <= this are culled (0.2) */
    float near_mesh;         /* faces with a vertex at view z <= this are culled (0.01) */
    float bg[3];             /* I_bg */
    int32_t bwd_stages;      /* hm_blend_backward parts to run (HM_BWD_* bits; 0 = all) */
    int32_t ellipse_cull;    /* 1: bin a Gaussian only into tiles whose pixel-centre
                                rectangle its 3-sigma ellipse reaches (result-preserving) */
    float kernel_2d;         /* variance (px^2) added to the projected covariance: 0.3 the
                                3DGS dilation, 0.1 the 2D Mip filter of Mip-Splatting */
    int32_t antialias;       /* 1: scale each opacity by sqrt(det Sigma2D / det(Sigma2D +
                                kernel_2d I)) (Mip-Splatting's 2D Mip filter) */
    int32_t persistent;      /* 1: the blend kernels run as one persistent grid of resident
                                CTAs that claim (view, tile) work items of all cameras from
                                a counter (hm_blend_forward's `work`, the backward's
                                workspace); 0: one CTA per tile.  Same results. */
} hm_options;

/* hm_blend_backward parts.  HM_BWD_PROJECT consumes the per-record partials
 * that HM_BWD_BLEND leaves in the workspace, so a caller splitting the pass
 * runs BLEND before PROJECT on the same workspace. */
#define HM_BWD_TEXTURE 1       /* texel gradients */
#define HM_BWD_BLEND 2         /* blend replay -> per-record partials (workspace) */
#define HM_BWD_PROJECT 4       /* partials -> Gaussian parameter gradients */

/* Fill `opt` with the defaults: 16x16 tiles, batch 128, mesh_cull 1,
 * ellipse_cull 1, near planes 0.2 / 0.01, black background, all backward
 * parts, the 3DGS screen-space kernel (kernel_2d 0.3, antialias 0). */
void hm_default_options(hm_options *opt);

/* Thread-local text of the last host-side error. */
const char *hm_last_error(void);

/* ------------------------------------------------------------------------ */
/* hm_rasterize_mesh -- Sec. 3.1 "Textured mesh" and the I_m, D_m of Sec. 3.4.
 *
 * Per pixel: the nearest covering triangle (two-sided; vertices projected in
 * FP64, snapped to 1/256 px, exact integer edge functions, top-left fill
 * rule; faces with a vertex at z <= near_mesh or beyond +-2^21 px culled),
 * its view depth D_m (the view z of the snapped face at the pixel centre).
 * 1/z is affine in screen space; the depth is evaluated in FP32 as
 * 1 / fma(a, U, fma(b, V, 1/z0)), (U,V) the pixel centre minus the snapped
 * vertex 0 in pixels and a, b, 1/z0 the face's coefficients computed in
 * FP64 and rounded once to FP32 (the face with the largest FP32 1/z wins,
 * ties to the lower face index; the depth is the correctly rounded FP32
 * reciprocal of that 1/z) -- within a few FP32 ulps of the FP64 depth (the band is
 * 3 + 3 kappa ulps, kappa the condition number of that evaluation);
 * perspective-correct UVs and a bilinear,
 * clamp-to-edge texture fetch (texel centres at half-integers, row 0 at v=0).
 *
 *  verts [n_verts][3], uvs [n_verts][2] float32; faces [n_faces][3] int32.
 *  tex   texture in `tex_format` layout.
 *  Outputs (per pixel of all cameras): tri_id int32 (-1 none), depth float32
 *  (+inf none), rgb planar float32 (I_m, or opt->bg where none), uv planar
 *  [2] float32 (0 where none); per tile: tile_max_depth float32 = the
 *  largest depth of the tile's in-image pixels, +inf if any has no triangle.
 *  item_capacity: (face, tile) work items the workspace holds; if exceeded,
 *  HM_DEV_CAPACITY is set, *n_items_out (device int64) gets the need and the
 *  outputs are invalid.  Any of rgb/uv may be NULL.
 */
size_t hm_rasterize_mesh_workspace_size(const hm_camera *cams, int32_t n_views, int32_t n_verts,
                                        int32_t n_faces, int64_t item_capacity,
                                        const hm_options *opt);
hm_status hm_rasterize_mesh(const hm_camera *cams, int32_t n_views, const float *verts,
                            const float *uvs, int32_t n_verts, const int32_t *faces,
                            int32_t n_faces, const void *tex, int32_t tex_w, int32_t tex_h,
                            int32_t tex_format, const hm_options *opt, int32_t *tri_id,
                            float *depth, float *rgb, float *uv, float *tile_max_depth,
                            int64_t item_capacity, int64_t *n_items_out, int32_t *d_status,
                            void *ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------ */
/* hm_project_gaussians -- Eq. 1 and Sec. 3.1: per (camera, Gaussian) the
 * 48-byte record consumed by hm_bin_sort / hm_blend_*:
 *   mean2d (FP32 pixels), conic = Sigma'^-1 (xx, xy, yy) with
 *   Sigma' = J W R S S^T R^T W^T J^T + kernel_2d I (J: affine Jacobian with the
 *   view x/z, y/z clamped to 1.3 x the half field of view), opacity, depth key
 *   z = fp32(fma(R20,x,fma(R21,y,fma(R22,z,t2)))) in FP64, colour
 *   max(0, 0.5 + SH(normalised mean - camera centre)) and the tile rectangle
 *   covering the 3-sigma ellipse d^2 <= 9.  Culled (z <= near_gauss, or no
 *   tile) records carry an empty rectangle; the colour is evaluated only for
 *   records with tiles (0 in the others, which no list holds).
 *  filter_3d [n] float32 >= 0 or NULL: the per-Gaussian variance v of
 *   Mip-Splatting's 3D smoothing filter (hm_mip_filter_3d): the covariance
 *   becomes R (S^2 + v I) R^T and the opacity is scaled by
 *   prod_k s_k / sqrt(s_k^2 + v).  With opt->antialias the opacity is also
 *   scaled by sqrt(det Sigma2D / det Sigma') (Mip-Splatting's 2D Mip filter,
 *   kernel_2d 0.1).  The paper pairs the mesh with this back-end (Tab. 1).
 *  sh [n][(sh_degree+1)^2][3] in sh_format; sh_degree 0..3.
 *  records: n_views*n*48 bytes, 16-byte aligned.
 */
hm_status hm_project_gaussians(const hm_camera *cams, int32_t n_views, int32_t n,
                               const float *means, const float *scales, const float *quats,
                               const float *opacity, const float *filter_3d, const void *sh,
                               int32_t sh_degree, int32_t sh_format, const hm_options *opt,
                               void *records, void *stream);

/* ------------------------------------------------------------------------ */
/* hm_mip_filter_3d -- the variance of Mip-Splatting's 3D smoothing filter per
 * Gaussian (Yu et al., CVPR 2024; the second back-end of Tab. 1):
 *   v_i = s2 / nu_i^2,  nu_i = max over the cameras that see mean i of f / z,
 * f = max(fx, fy), z the FP32 view depth; a camera sees the mean iff
 * z > near_z and the projected mean lies in [0, W] x [0, H].  A Gaussian no
 * camera sees gets v = 0.  s2 > 0 is the filter size in squared sampling
 * intervals (Mip-Splatting: 0.2).  The cameras are the training views; the
 * result is a constant of the projection (no gradient flows into it).
 *  means [n][3] float32 (device); filter_3d [n] float32 (device, written).
 *  Errors: HM_ERR_INVALID_ARG (cameras, n < 0, s2 <= 0, null pointers),
 *  HM_ERR_CUDA.  Launches only.
 */
hm_status hm_mip_filter_3d(const hm_camera *cams, int32_t n_views, int32_t n, const float *means,
                           float s2, float near_z, float *filter_3d, void *stream);

/* ------------------------------------------------------------------------ */
/* hm_bin_sort -- the tile-wise sort the paper's rasteriser relies on (Sec. 1:
 * tile-wise sorting and pixel-wise blending are the cost that grows with the
 * number of Gaussians).  Emits one (tile, depth) key per (record, tile) pair
 * whose tile the record's rectangle covers (minus pairs at or behind the
 * tile's farthest mesh depth when opt->mesh_cull and tile_max_depth are
 * given, and, with opt->ellipse_cull, tiles whose pixel centres all lie
 * outside the 3-sigma ellipse), and sorts them by (tile, FP32 depth, Gaussian index) with an LSD
 * device radix sort.  Outputs: pair_vals[capacity] uint32 record indices in
 * sorted order, *n_pairs_out (device int64) the pair count, tile_ranges
 * [total_tiles][2] uint32 [begin, end) into pair_vals.  If the count exceeds
 * `capacity` (<= HM_MAX_PAIRS), HM_DEV_CAPACITY is set, *n_pairs_out holds
 * the need and the other outputs are invalid.
 */
size_t hm_bin_sort_workspace_size(const hm_camera *cams, int32_t n_views, int32_t n,
                                  int64_t capacity, const hm_options *opt);
hm_status hm_bin_sort(const hm_camera *cams, int32_t n_views, int32_t n, const void *records,
                      const float *tile_max_depth, const hm_options *opt, uint32_t *pair_vals,
                      int64_t capacity, int64_t *n_pairs_out, uint32_t *tile_ranges,
                      int32_t *d_status, void *ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------ */
/* hm_blend_forward -- Eq. 2 with the joint-rasterisation cut-off of Sec. 3.4.
 * Per pixel, front to back over its tile's sorted list: stop at the first
 * Gaussian with depth >= D_m (mesh_depth finite); skip it unless
 * d^2 = D^T conic D <= 9; alpha = min(0.99, o exp(-d^2/2)); skip if
 * alpha < 1/255; stop before a Gaussian that would drop T below 1e-4;
 * C += alpha T c, T *= 1 - alpha.  Finally I_h = C + T * back, with back =
 * mesh_rgb (I_m, or I_bg where no triangle) or opt->bg if mesh_rgb is NULL.
 *  mesh_depth, mesh_rgb: hm_rasterize_mesh outputs, or NULL (no mesh).
 *  Outputs: out_rgb planar, out_T, n_contrib (Gaussians blended), last_idx
 *  (1 + position in pair_vals of the last blended Gaussian, 0 if none; used
 *  by the backward pass; may be NULL).
 *  eval_stats (device uint64[2], may be NULL): when given, [0] += the number
 *  of (pixel, Gaussian) pairs whose alpha was evaluated (inside the 3-sigma
 *  ellipse, before the pixel stopped) and [1] += the list entries examined.
 *  d_status (device int32, may be NULL): HM_DEV_TIMEOUT / HM_DEV_BAD_INDEX.
 *  work (device uint32, 4-byte aligned): the tile counter of the persistent
 *  launch (opt->persistent = 1; zeroed by the call, so concurrent calls need
 *  their own); may be NULL otherwise.
 *  Records are staged into shared memory by bulk asynchronous copies (TMA),
 *  opt->batch list entries per round, double buffered.
 */
hm_status hm_blend_forward(const hm_camera *cams, int32_t n_views, int32_t n, const void *records,
                           const uint32_t *pair_vals, const uint32_t *tile_ranges,
                           const float *mesh_depth, const float *mesh_rgb, const hm_options *opt,
                           float *out_rgb, float *out_T, uint32_t *n_contrib, uint32_t *last_idx,
                           unsigned long long *eval_stats, int32_t *d_status, uint32_t *work,
                           void *stream);

/* ------------------------------------------------------------------------ */
/* hm_blend_backward -- gradients of a loss L through hm_blend_forward and
 * hm_project_gaussians (and, if d_tex is given, through the bilinear texture
 * fetch of hm_rasterize_mesh: dL/dtexel = sum over pixels of
 * T * bilinear weight * dL/dI_h on pixels with a triangle).  Discrete
 * decisions (the blended set, clamps, the mesh hit) carry no gradient; vertex
 * positions and UVs get none.
 *  Inputs: the forward's parameters (with the same filter_3d and options:
 *  the gradients follow the Mip-Splatting filters' opacity factors and the
 *  3D filter's effective scales; v itself is a constant), records, sorted
 *  pairs and ranges, mesh outputs (depth, rgb, uv; NULL for no mesh), out_T
 *  and last_idx, and dL_drgb (planar, like out_rgb) and dL_dT (per pixel,
 *  may be NULL).
 *  dL_dmesh (planar, may be NULL): the gradient of a loss on the mesh colour
 *  I_m itself (such as the texture loss of hm_hybrid_loss), added to the
 *  T * dL/dI_h the texels receive through the composite.
 *  Outputs, ACCUMULATED into caller-zeroed buffers: d_means [n][3],
 *  d_scales [n][3], d_quats [n][4], d_opacity [n], d_sh [n][K][3] float32
 *  (also for F16 SH storage), d_tex [tex_h][tex_w][3] float32 (may be NULL).
 *  d_status (device int32, may be NULL): as for hm_blend_forward.
 */
size_t hm_blend_backward_workspace_size(int32_t n_views, int32_t n);
hm_status hm_blend_backward(const hm_camera *cams, int32_t n_views, int32_t n, const float *means,
                            const float *scales, const float *quats, const float *opacity,
                            const float *filter_3d, const void *sh, int32_t sh_degree,
                            int32_t sh_format,
                            const void *records, const uint32_t *pair_vals,
                            const uint32_t *tile_ranges, const float *mesh_depth,
                            const float *mesh_rgb, const float *mesh_uv, int32_t tex_w,
                            int32_t tex_h, const hm_options *opt, const float *out_T,
                            const uint32_t *last_idx, const float *dL_drgb, const float *dL_dT,
                            const float *dL_dmesh, float *d_means, float *d_scales, float *d_quats,
                            float *d_opacity, float *d_sh, float *d_tex, int32_t *d_status, void *ws,
                            size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------ */
/* hm_blend_backward_noalloc -- hm_blend_backward for callers that cannot
 * allocate device memory: code running inside a CUDA stream capture, a
 * host whose allocator is owned by someone else (a plug-in, an embedded
 * runtime), or a real-time loop that must not allocate.  The paper has no
 * counterpart; it is a convenience of this library.
 *
 * Same arguments (dL_dmesh included) and results as hm_blend_backward,
 * without ws/ws_bytes: the scratch is a library-owned static device array of
 * HM_BWD_NOALLOC_BYTES bytes (16 MiB), which every GPU that loads the library
 * holds until the process exits.  Problems needing more
 * (hm_blend_backward_workspace_size: 44 bytes per record, so n above
 * 381,294 for one view) are rejected with
 * HM_ERR_INVALID_ARG and a message.  The array's device address belongs to the current context: a
 * call outside a stream capture looks it up again (with the caller's device
 * current), a call under capture uses the address the last uncaptured call
 * on that device found.  So the first call on a device -- and the first
 * after a context reset (cudaDeviceReset) -- must come before any stream
 * capture; otherwise the call returns HM_ERR_INVALID_ARG.  Every call shares
 * the one array, which keeps the last call's contents (the call clears what
 * it needs): calls that overlap on the GPU -- on two streams, or a
 * HM_BWD_PROJECT-only call after another call's HM_BWD_BLEND -- race and
 * give wrong gradients.  No allocation happens in this call. */
#define HM_BWD_NOALLOC_BYTES (16u << 20)
hm_status hm_blend_backward_noalloc(const hm_camera *cams, int32_t n_views, int32_t n,
                                    const float *means, const float *scales, const float *quats,
                                    const float *opacity, const float *filter_3d, const void *sh,
                                    int32_t sh_degree, int32_t sh_format, const void *records,
                                    const uint32_t *pair_vals, const uint32_t *tile_ranges,
                                    const float *mesh_depth, const float *mesh_rgb,
                                    const float *mesh_uv, int32_t tex_w, int32_t tex_h,
                                    const hm_options *opt, const float *out_T,
                                    const uint32_t *last_idx, const float *dL_drgb,
                                    const float *dL_dT, const float *dL_dmesh, float *d_means,
                                    float *d_scales, float *d_quats, float *d_opacity, float *d_sh,
                                    float *d_tex, int32_t *d_status, void *stream);

/* Number of tiles of all cameras for the tile shape in `opt`. */
int64_t hm_total_tiles(const hm_camera *cams, int32_t n_views, const hm_options *opt);

/* ------------------------------------------------------------------------ */
/* hm_hybrid_loss -- the joint-optimisation loss of the hybrid representation
 * and its gradients (Sec. 3.4; Eq. 3, Eq. 5, Eq. 6, Eq. 7):
 *   L   = (1 - lambda_ssim) L1(I, I_h) + lambda_ssim (1 - SSIM(I, I_h)) + lambda_t L_t
 *   L_t = M_T * ||I~ - I~_m||^2,  M_T = 1 / (1 + exp(-k (T - 0.5)))
 * where I~, I~_m are the target and the mesh colour on pixels with a
 * triangle (mesh_depth finite) and 0 elsewhere.  Every term is a mean over
 * all pixel-channel elements of all cameras; SSIM uses an 11 x 11 Gaussian
 * window (sigma 1.5, zero outside the image), C1 = 0.01^2, C2 = 0.03^2;
 * M_T is a mask (no gradient to T).
 *  out_rgb (I_h), target (I): planar per camera like hm_blend_forward's
 *  output.  mesh_rgb, out_T, mesh_depth, dL_dmesh: all NULL (no texture
 *  loss) or all given.
 *  Outputs: loss_out (device double[4]: L1, mean SSIM, L_t, L), dL_drgb
 *  (dL/dI_h, planar, written), dL_dmesh (lambda_t dL_t/dI_m, planar,
 *  written; pass it to hm_blend_backward).  The partial sums are reduced in
 *  a fixed order, so equal inputs give bitwise-equal results.  With
 *  lambda_ssim == 0 the SSIM term is not evaluated: one pointwise pass,
 *  dL/dI_h = sign(I_h - I) / N (0 on ties), and loss_out[1] is 0.
 *  ws: hm_hybrid_loss_workspace_size(cams, n_views) bytes of device memory.
 *  Errors: HM_ERR_INVALID_ARG (bad cameras, null pointers, an incomplete
 *  mesh set, lambda_ssim outside [0, 1] or lambda_t < 0), HM_ERR_WORKSPACE
 *  (ws too small), HM_ERR_CUDA (launch failure).  Launches only; runs on
 *  `stream` and never synchronises.
 */
typedef struct hm_loss_params {
    float lambda_ssim;       /* weight of D-SSIM in the photometric loss (0.2) */
    float lambda_t;          /* weight of the texture loss (0.1; 0 in the warm-up) */
    float k;                 /* slope of the transmittance mask (20) */
} hm_loss_params;

/* hm_decode_u8 -- 8-bit image codes to the [0, 1] intensities the loss
 * compares against: dst[i] = src[i] / 255 (correctly rounded FP32), for
 * loading a target image.  src (n bytes) and dst (n floats) are device
 * memory, 16-byte aligned.  Errors: HM_ERR_INVALID_ARG (n < 0, null or
 * misaligned pointers), HM_ERR_CUDA.  Launches only. */
hm_status hm_decode_u8(const uint8_t *src, int64_t n, float *dst, void *stream);

void hm_default_loss_params(hm_loss_params *p);
size_t hm_hybrid_loss_workspace_size(const hm_camera *cams, int32_t n_views);
hm_status hm_hybrid_loss(const hm_camera *cams, int32_t n_views, const float *out_rgb,
                         const float *target, const float *mesh_rgb, const float *out_T,
                         const float *mesh_depth, const hm_loss_params *p, double *loss_out,
                         float *dL_drgb, float *dL_dmesh, void *ws, size_t ws_bytes, void *stream);

/* hm_hybrid_loss_u8 -- hm_hybrid_loss with the target given as 8-bit codes
 * (device uint8, planar like out_rgb): every kernel reads a code c as c / 255
 * (correctly rounded FP32), so the results equal hm_hybrid_loss on the image
 * hm_decode_u8 writes, bit for bit, without that pass or its float image.
 * Same arguments, workspace, outputs and errors as hm_hybrid_loss. */
hm_status hm_hybrid_loss_u8(const hm_camera *cams, int32_t n_views, const float *out_rgb,
                            const uint8_t *target, const float *mesh_rgb, const float *out_T,
                            const float *mesh_depth, const hm_loss_params *p, double *loss_out,
                            float *dL_drgb, float *dL_dmesh, void *ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------ */
/* hm_checked_status -- the index checks of the checked build.  The library
 * built with HM_CHECKED (libhm_checked.so; same entry points) checks every
 * index a kernel reads from a device buffer -- pair and item list entries,
 * bucket and tile-range bounds, tile ids, slots, the backward's stop
 * positions and gradient list -- against the bound it must respect before
 * using it; a failed check skips the access and is recorded instead of
 * faulting the GPU.  The paper has no counterpart: it is a debugging aid
 * for corrupt inputs.
 *  *bits: HM_DEV_BAD_INDEX if a check failed since the last reset, else 0;
 *  reset != 0 clears the record.  Synchronises the device.
 *  Errors: HM_ERR_INVALID_ARG (null bits; or the default library, which has
 *  no checks), HM_ERR_CUDA. */
hm_status hm_checked_status(int32_t *bits, int32_t reset);

/* ------------------------------------------------------------------------ */
/* hm_adam_update -- one Adam step (Kingma and Ba, 2015) on n float32 values
 * in place, for optimised buffers such as the texture map in the texture-only
 * optimisation that initialises it from the images (Sec. 3.3):
 *   m <- beta1 m + (1 - beta1) g,  v <- beta2 v + (1 - beta2) g^2,
 *   p <- p - lr (m / (1 - beta1^step)) / (sqrt(v / (1 - beta2^step)) + eps).
 *  param, m, v (device, updated), grad (device); step >= 1 counts from 1.
 *  Errors: HM_ERR_INVALID_ARG (n < 0, step < 1, betas outside [0, 1),
 *  eps or lr < 0, null pointers), HM_ERR_CUDA.  Launches only.
 */
hm_status hm_adam_update(float *param, const float *grad, float *m, float *v, int64_t n, float lr,
                         float beta1, float beta2, float eps, int32_t step, void *stream);

/* hm_adam_update_dev -- the same update with the bias corrections read from
 * device memory, d_rc[2] = (1 / (1 - beta1^t), 1 / (1 - beta2^t)) as kept by
 * hm_adam_advance, so that a training step can be captured in a CUDA graph
 * once and replayed.  d_status (device int32, may be NULL): when nonzero (a
 * stage of the step reported an error, e.g. a capacity overflow) the update
 * is skipped.  Errors as hm_adam_update.
 * hm_adam_advance -- ++*d_step and d_rc for the new step, skipped when
 * *d_status is nonzero.  d_step (device int32, 0 before the first step). */
hm_status hm_adam_update_dev(float *param, const float *grad, float *m, float *v, int64_t n, float lr,
                             float beta1, float beta2, float eps, const float *d_rc,
                             const int32_t *d_status, void *stream);
hm_status hm_adam_advance(int32_t *d_step, float beta1, float beta2, float *d_rc,
                          const int32_t *d_status, void *stream);

/* ------------------------------------------------------------------------ */
/* hm_activate / hm_activate_backward -- the 3DGS parameterisation the joint
 * optimisation (Sec. 3.4) trains: scales = exp(log_scales) [n][3],
 * opacity = 1 / (1 + exp(-logit)) [n]; and the chain rule back,
 * d_log_scales = d_scales * scales, d_logit = d_opacity * opacity (1 - opacity)
 * (written, not accumulated).  Device pointers; launches only. */
hm_status hm_activate(int64_t n, const float *log_scales, const float *logit, float *scales,
                      float *opacity, void *stream);
hm_status hm_activate_backward(int64_t n, const float *scales, const float *opacity,
                               const float *d_scales, const float *d_opacity, float *d_log_scales,
                               float *d_logit, void *stream);

/* ------------------------------------------------------------------------ */
/* hm_mesh_prune -- the mesh-pruning metrics of Sec. 3.3 / Algorithm 1
 * (stage 1), which prepare the mesh before the joint optimisation.  Per
 * triangle (bits of flags[f]; flags[f] == 0 keeps it):
 *   HM_PRUNE_NORMAL  per view, the floor(alpha_normal % of the covered pixels)
 *                    ranking first by (total variation of the prior normal
 *                    map descending, pixel index ascending) mark the triangle
 *                    tri_id names there.  TV(x,y) = sum_c |N_c(x+1,y) -
 *                    N_c(x,y)| + |N_c(x,y+1) - N_c(x,y)| in FP32 (absent
 *                    neighbours 0), channel by channel in that order;
 *   HM_PRUNE_ANGLE   a triangle sharing an edge has a normal more than
 *                    angle_deg away: n_f . n_g < cos(angle) sqrt(|n_f|^2 |n_g|^2),
 *                    n = (v1 - v0) x (v2 - v0) in FP64 (winding as given;
 *                    zero-area triangles take no part);
 *   HM_PRUNE_AREA    the floor(alpha_area % of F) first by (|n|^2, index);
 *   HM_PRUNE_GROUP   triangles no metric above removed, in edge-connected
 *                    pieces of those triangles with fewer than alpha_group.
 * The metrics are keep masks combined with && (the paper's M_N && M_A && M_S).
 * Hole closing and smoothing (later steps of stage 1) are not part of it.
 *  cams[n_views] give the image sizes of tri_id (hm_rasterize_mesh output,
 *  per pixel of all views) and normals (planar [3][H][W] per view, float32);
 *  with n_views == 0 or either NULL the normal metric is skipped.
 *  verts [n_verts][3] float32, faces [n_faces][3] int32 (device).
 *  Outputs: flags [n_faces] uint8; label [n_faces] int32 (may be NULL): the
 *  smallest triangle index of the piece, -1 where a metric removed it.
 *  Errors: HM_ERR_INVALID_ARG (sizes, parameters, a face index or tri_id out
 *  of range), HM_ERR_WORKSPACE, HM_ERR_CUDA.  SYNCHRONISES `stream` (the
 *  piece labelling iterates until no label changes, at most 64 rounds).
 */
#define HM_PRUNE_NORMAL 1
#define HM_PRUNE_ANGLE 2
#define HM_PRUNE_AREA 4
#define HM_PRUNE_GROUP 8
typedef struct hm_prune_params {
    float alpha_normal;      /* percent of covered pixels per view (20) */
    float alpha_area;        /* percent of triangles (50) */
    float angle_deg;         /* adjacent-angle limit (45) */
    int32_t alpha_group;     /* smallest piece kept, in triangles (100) */
} hm_prune_params;

void hm_default_prune_params(hm_prune_params *p);
size_t hm_mesh_prune_workspace_size(const hm_camera *cams, int32_t n_views, int32_t n_verts,
                                    int32_t n_faces);
hm_status hm_mesh_prune(const hm_camera *cams, int32_t n_views, const float *verts, int32_t n_verts,
                        const int32_t *faces, int32_t n_faces, const int32_t *tri_id,
                        const float *normals, const hm_prune_params *p, uint8_t *flags,
                        int32_t *label, void *ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------ */
/* hm_selftest_bounded_waits -- failure detection without a fault: one thread
 * runs the library's two bounded waits (the scans' look-back wait and the
 * blend kernels' mbarrier wait) on a slot that is never published
 * (d_zero_slot: device uint64, zero) and an mbarrier nothing arrives at.
 * Each gives up after its poll limit (well under a second in total), ORs
 * HM_DEV_TIMEOUT into *d_status and the kernel returns, leaving the context
 * usable.  d_out[2] (device int32): 1 where a wait completed (expected 0, 0).
 * Launches only. */
hm_status hm_selftest_bounded_waits(const unsigned long long *d_zero_slot, int32_t *d_status,
                                    int32_t *d_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* HM_H */

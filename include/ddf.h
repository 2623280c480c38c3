/*
 * ddf.h -- C ABI of the GB300 Directed Distance Field query library (libddf.so).
 *
 * The library evaluates a Directed Distance Field f(x, d) = (t, xi)
 * (Sec. 3.1, Eq. 1): for a ray with origin x and unit direction d, t is the
 * distance to the first surface along d and xi the probability that the ray
 * hits anything. The field is the "first DDF" of Sec. 4.3 / Table 2: a
 * sinusoidal encoding of (x, d) followed by a wide ReLU MLP; the two outputs
 * are t = softplus(z0) and xi = sigmoid(z1), and a ray counts as a hit when
 * z1 > 0. Every query is one network evaluation (Sec. 3.3).
 *
 * Conventions shared by every entry point
 *  - Every call returns a ddf_status and never aborts the process. Arguments
 *    are checked before anything is launched; on failure nothing is launched
 *    and ddf_last_error() describes the problem.
 *  - Ray batches are a structure of arrays: rays[0..5] point to n float32
 *    values each (ox, oy, oz, dx, dy, dz), 4-byte aligned, caller-owned.
 *    Directions are used as given (no renormalisation).
 *  - "device" pointers are CUDA device (or managed) memory on the handle's
 *    device; "host" pointers are ordinary host memory. Calls that take a
 *    stream are asynchronous with respect to the host: results are valid once
 *    the stream has reached the call; the caller keeps inputs alive until then.
 *  - stream is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream. One handle must not be used from two host threads at once, and
 *    two in-flight calls on different streams must not share one handle (they
 *    share its workspace).
 *  - The library owns the weights, their reduced-precision copies, the
 *    workspace and any CUDA graphs; ddf_destroy frees all of it.
 *  - Device kernels bound every wait; a wait that runs out makes the kernel
 *    give up cleanly (no trap, the context stays usable) and sets a bit in the
 *    handle's device status word, which ddf_check_status reads and clears.
 *    Results of a launch that gave up are undefined.
 */
#ifndef DDF_H_
#define DDF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ddf_s* ddf_handle;

typedef enum {
  DDF_OK = 0,
  DDF_ERR_INVALID_ARG = 1,  /* null pointer, bad size, bad alignment, bad config */
  DDF_ERR_CUDA = 2,         /* a CUDA runtime call failed (message in ddf_last_error) */
  DDF_ERR_OOM = 3,          /* device or pinned allocation failed */
  DDF_ERR_BAD_WEIGHTS = 4,  /* blob size mismatch, non-finite values, no weights loaded */
  DDF_ERR_UNSUPPORTED = 5,  /* valid request the library does not support (e.g. width) */
  DDF_ERR_TIMEOUT = 6       /* a device-side bounded wait ran out (see header notes) */
} ddf_status;

typedef enum {
  DDF_FP32 = 0,      /* plain FP32 on CUDA cores (no TF32) */
  DDF_BF16 = 1,      /* bf16 operands, FP32 accumulation on tcgen05 tensor cores */
  DDF_FP8_E4M3 = 2   /* e4m3 operands (layers 2..H), FP32 accumulation on tcgen05 */
} ddf_precision;

/* Network shape and precision (Sec. 4.3: sinusoidal encoding + wide MLP).
 *   octaves        L >= 0 bands per coordinate; encoded width D_in = 6 + 12 L
 *                  laid out as [ox,oy,oz,dx,dy,dz, then for each coordinate c
 *                  and band k: sin(pi 2^k e_c), cos(pi 2^k e_c)], L <= 16
 *   width          hidden width W; tensor-core precisions need W % 128 == 0
 *                  and W <= 2048
 *   hidden_layers  H >= 1 ReLU layers (D_in -> W, then H-1 times W -> W)
 *   precision      a ddf_precision value
 *   device         CUDA device ordinal the handle lives on
 *   kind           DDF_KIND_RAY: the directed distance field of a ray (as
 *                  above, 2 outputs); DDF_KIND_SDF: a signed distance field of
 *                  a point p (the sphere-tracing baseline of Sec. 4.4): input
 *                  [px,py,pz, per coordinate and band sin(pi 2^k p_c),
 *                  cos(pi 2^k p_c)] (D_in = 3 + 6 L), one raw output; bf16 only;
 *                  DDF_KIND_HASHGRID: the paper's final field (Sec. 3.4), a
 *                  ray field whose origin is encoded by a multiresolution hash
 *                  grid (16 levels x 2 features, 2^19 entries per level, base
 *                  resolution 16, growth 1.5, over the box [-1,1]^3, origins
 *                  clamped into it) and whose direction by `octaves` = 4
 *                  sinusoidal bands; code = [level 0..15 features, d, per
 *                  coordinate and band sin, cos] (59 values); `width` = 64,
 *                  1..4 hidden layers; bf16 (bf16 table and MLP on tensor
 *                  cores, FP32 head) or FP32. Level l has N = floor(16 1.5^l)
 *                  cells per axis; it stores every vertex (i + (N+1)(j +
 *                  (N+1) k)) while (N+1)^3 <= 2^19, else 2^19 entries indexed
 *                  by (i xor j * 2654435761 xor k * 805459861) mod 2^19; a
 *                  point reads the trilinear interpolation of its cell's 8
 *                  corners. Ray queries (ddf_query_*) and the training
 *                  calls (ddf_compute_grad, ddf_train_step, ddf_forward_train
 *                  / ddf_backward, ddf_distill, ddf_distill_pool; FP32 on the
 *                  master weights) accept it; tiles and FP8 do not. */
typedef enum { DDF_KIND_RAY = 0, DDF_KIND_SDF = 1, DDF_KIND_HASHGRID = 2 } ddf_kind;

typedef struct {
  int32_t octaves;
  int32_t width;
  int32_t hidden_layers;
  int32_t precision;
  int32_t device;
  int32_t kind;
} ddf_config;

/* Number of floats in the weight blob of cfg (0 if cfg is invalid).
 * Blob layout: for each layer in order, W[out][in] row-major then b[out];
 * layers are D_in->W, (H-1) x W->W, then the head W->2 whose row 0 feeds
 * t = softplus(z0) and row 1 feeds xi = sigmoid(z1). A hash-grid field puts
 * its level tables first (level 0..15, entry-major, the 2 features of an
 * entry adjacent; 13,058,044 floats), then the MLP laid out as above with
 * D_in = 59. */
size_t ddf_param_count(const ddf_config* cfg);

/* Creates a handle on cfg->device. *out receives the handle (NULL on error).
 * Allocates only small bookkeeping; weights arrive with ddf_load_weights. */
ddf_status ddf_create(const ddf_config* cfg, ddf_handle* out);

/* Frees everything the handle owns (synchronises its device first).
 * Passing NULL is a no-op returning DDF_OK. */
ddf_status ddf_destroy(ddf_handle h);

/* Message of the last failing call on this host thread ("" if none).
 * The string stays valid until the next call on the same thread. */
const char* ddf_last_error(void);

/* Copies n_floats = ddf_param_count() FP32 master weights from host memory,
 * then derives the precision-specific device copies (bf16 casts, or e4m3
 * codes with per-output-channel scales s_n = amax_n / 448). Synchronous.
 * DDF_ERR_BAD_WEIGHTS on a size mismatch or a non-finite value. */
ddf_status ddf_load_weights(ddf_handle h, const float* host_blob, size_t n_floats);

/* Copies the current FP32 master weights (after any training steps) into
 * host_blob (n_floats = ddf_param_count()). Synchronous: a checkpoint. */
ddf_status ddf_get_weights(ddf_handle h, float* host_blob, size_t n_floats);

/* FP8 only: per-tensor activation scales s_1..s_{H-1} for the e4m3 inputs of
 * layers 2..H (n = H-1 host floats, each a positive power of two). Layer l+1
 * reads the code e4m3(h_l / s_l). Required before an FP8 query. */
ddf_status ddf_set_act_scales(ddf_handle h, const float* host_scales, int32_t n);

/* One DDF evaluation per ray (Sec. 3.3, primary and bounce rays):
 * out_t[i] = softplus(z0), out_vis[i] = sigmoid(z1) for ray i, i < n.
 * rays: 6 device pointers (SoA, see above); out_t, out_vis: n device floats.
 * n == 0 is a no-op. Asynchronous on stream. */
ddf_status ddf_query_rays(ddf_handle h, const float* const rays[6], int64_t n,
                          float* out_t, float* out_vis, void* stream);

/* Shadow query (Sec. 3.3): as ddf_query_rays, plus out_occluded[i] = 1 when
 * the field reports a hit (z1 > 0) closer than the light, i.e.
 * t < |light - origin_i|, else 0. light: 3 host floats. out_occluded: n
 * device bytes. Asynchronous on stream. */
ddf_status ddf_query_shadow(ddf_handle h, const float* const rays[6], int64_t n,
                            const float light[3], float* out_t, float* out_vis,
                            uint8_t* out_occluded, void* stream);

/* Same as ddf_query_rays with every buffer in HOST memory: the library copies
 * the rays in, evaluates them and copies t and vis back, overlapping the copies
 * of one chunk with the evaluation of the next on its own streams. Returns
 * once the results are in out_t / out_vis (synchronous). Page-locked host
 * buffers give the fastest copies; pageable ones work. */
ddf_status ddf_query_rays_host(ddf_handle h, const float* const rays[6], int64_t n,
                               float* out_t, float* out_vis);

/* Shadow query with every buffer in HOST memory (light: 3 host floats,
 * out_occluded: n host bytes); pipelined and synchronous like
 * ddf_query_rays_host. */
ddf_status ddf_query_shadow_host(ddf_handle h, const float* const rays[6], int64_t n,
                                 const float light[3], float* out_t, float* out_vis,
                                 uint8_t* out_occluded);

/* Allocation-free query (the paper has no counterpart; this is a library
 * service). Same arguments, results and stream semantics as ddf_query_rays,
 * but the scratch the kernels need comes from one static 32 MiB device array
 * that every GPU loading the library reserves until exit, so the call itself
 * never calls cudaMalloc/cudaFree. For callers that cannot allocate mid-work:
 * a renderer's per-frame callback (cudaMalloc may synchronise the device and
 * stall the frame) or a host framework whose pool owns all device memory.
 *  - n must fit the scratch in one pass (about 6,190 rays for 126->1280x8
 *    bf16, about 49,300 for 78->128x4); larger n returns DDF_ERR_INVALID_ARG
 *    with the limit in the message. Hash-grid fields run one fused kernel
 *    with no scratch, so their batches have no such limit.
 *  - The first call on a device looks up the scratch address there; make it
 *    before any stream capture.
 *  - All calls (all handles) share the array and leave their data in it; no
 *    part of it needs to start zeroed. Calls that overlap on the GPU race. */
ddf_status ddf_query_rays_noalloc(ddf_handle h, const float* const rays[6], int64_t n,
                                  float* out_t, float* out_vis, void* stream);

/* Ragged ambient occlusion (Sec. 3.3: evaluate the field along a set of
 * hemisphere directions and average the hit flag). Point p owns the rays
 * offsets[p] .. offsets[p+1]-1 of the n_rays-ray batch (SoA as above);
 * offsets: n_points + 1 device int32, non-decreasing, offsets[0] = 0,
 * offsets[n_points] = n_rays (n_rays < 2^31). Writes
 *   out_hard[p] = 1 - (number of rays with z1 > 0) / count
 *   out_soft[p] = 1 - (sum of vis) / count        (out_soft nullable)
 * and 1 for points with no rays. Device pointers, asynchronous on stream.
 * Keeps a per-ray scratch of 5 bytes x n_rays inside the handle. */
ddf_status ddf_query_ao(ddf_handle h, const float* const rays[6], int64_t n_rays,
                        const int32_t* offsets, int64_t n_points, float* out_hard,
                        float* out_soft, void* stream);

/* Mixed batch (Sec. 3.3: a frame of the application asks, per shading
 * point, one shadow ray and a ragged set of hemisphere rays; both are single
 * field evaluations). Evaluates n_shadow shadow rays (SoA shadow_rays, light
 * and outputs as ddf_query_shadow) and a ragged AO batch (ao_rays, offsets,
 * n_points, out_hard, out_soft as ddf_query_ao) as ONE batch of
 * n_shadow + n_ao_rays rows: rows below n_shadow come from shadow_rays, the
 * rest from ao_rays, and every layer launch covers both kinds, so the ragged
 * sets share the persistent tiles with the shadow rays instead of running a
 * second pass. The results equal those of the two separate queries. In
 * graph mode the whole sequence (all chunks, all layers, the shadow decision
 * and the segmented AO reduce) is one graph replay. Either part may be
 * empty (its pointers may then be NULL); n_ao_rays < 2^31. Device pointers,
 * asynchronous on stream; keeps 5 bytes x n_ao_rays of scratch inside the
 * handle, like ddf_query_ao. */
ddf_status ddf_query_mixed(ddf_handle h, const float* const shadow_rays[6], int64_t n_shadow,
                           const float light[3], float* out_t, float* out_vis,
                           uint8_t* out_occluded, const float* const ao_rays[6], int64_t n_ao_rays,
                           const int32_t* offsets, int64_t n_points, float* out_hard,
                           float* out_soft, void* stream);

/* Graph mode. When on, ddf_query_rays, ddf_query_shadow, ddf_query_ao and
 * ddf_query_mixed record their whole launch sequence (all chunks and layers)
 * into a CUDA
 * graph the first time they see a given set of pointers, sizes and light,
 * and afterwards replay that graph with one cudaGraphLaunch on the caller's
 * stream; the data behind the pointers may change between calls. Up to 8
 * graphs are cached per handle; changing tiles, chunk size, timeout or
 * activation scales, or growing a workspace, drops them. Turning the mode off
 * drops them too. */
ddf_status ddf_set_graph_mode(ddf_handle h, int32_t on);

/* FP8 handles: calibrates the per-tensor activation scales on n rays (device
 * SoA; a representative batch). Runs layers 1..H-1 in bf16 on the same weights,
 * records amax_l = max over the batch of the layer-l output h_l (after ReLU),
 * and sets s_l = the smallest power of two with amax_l / s_l <= 448, as
 * ddf_set_act_scales would. amax_out and scales_out (nullable, H-1 host
 * floats) receive both. Synchronous; allocates 4 (H-1) bytes while it runs. */
ddf_status ddf_calibrate_fp8(ddf_handle h, const float* const rays[6], int64_t n, float* amax_out,
                             float* scales_out, void* stream);

/* ---- distillation (Sec. 3.2 / 3.4) ----
 * One batch of rays with targets: t_target (device float[batch], the exact
 * first-hit distance; ignored where hit_target is 0, may be +inf there) and
 * hit_target (device uint8[batch], 1 = the ray hits the scene). The loss is
 *   L = (1/max(1, N_hit)) sum_{hit} |min(t, 4) - min(t*, 4)|
 *       + 0.3 (1/B) sum_i [softplus(z1) - y z1],     t = softplus(z0).
 * Sinusoidal ray fields (bf16 handles only): bf16 activations, FP32 head and
 * loss, gradients from bf16 operands with FP32 accumulation; the handle keeps
 * every hidden activation (2 W bytes per ray and layer, fewer with
 * ddf_set_recompute), each layer's ReLU pattern as bits (W/8 bytes per ray
 * and layer) and two input-gradient buffers (2 W bytes per ray each); the
 * weight-gradient GEMMs read the stored activations as they lie, so no
 * transposed copy is made. Hash-grid fields (bf16 or FP32 handles):
 * forward and backward in FP32 on the master weights; the level tables'
 * gradient is a scatter of each ray's feature gradient into its 8 corner
 * entries per level (atomic adds, so its last bits may vary from run to run);
 * a bf16 handle's query copies are refreshed after each Adam step.
 * batch: positive multiple of 8, below 2^31. out_loss: device float,
 * nullable. Asynchronous on stream. */

/* Gradient of the batch loss w.r.t. every weight and bias, kept in the
 * handle (read it with ddf_get_grad); the weights do not change. */
ddf_status ddf_compute_grad(ddf_handle h, const float* const rays[6], const float* t_target,
                            const uint8_t* hit_target, int64_t batch, float* out_loss,
                            void* stream);

/* ddf_compute_grad, then one Adam step (beta 0.9 / 0.999, eps 1e-8,
 * bias-corrected, no weight decay; lr > 0) on the FP32 master weights, after
 * which every query on the handle uses the new weights. */
ddf_status ddf_train_step(ddf_handle h, const float* const rays[6], const float* t_target,
                          const uint8_t* hit_target, int64_t batch, float lr, float* out_loss,
                          void* stream);

/* The two halves of ddf_compute_grad, for a loss written elsewhere (the
 * Python binding wraps them in a torch.autograd.Function):
 * ddf_forward_train runs the training forward on a bf16 handle (same batch
 * rules as ddf_compute_grad; inputs = 6 ray arrays, or 3 point arrays for an
 * SDF field), keeps every activation in the handle and writes the head
 * outputs before softplus / sigmoid to out_z (device float, batch x 2 row
 * pairs (z0, z1) for a ray field, batch values for an SDF field).
 * ddf_backward takes dL/dz in the same layout (device float) and computes
 * the gradient of every weight and bias into the handle (ddf_get_grad,
 * ddf_copy_grad). It needs the activations of a ddf_forward_train of the same
 * batch with no training call, weight load or Adam step in between, and
 * fails with DDF_ERR_INVALID_ARG otherwise. Both asynchronous on stream. */
ddf_status ddf_forward_train(ddf_handle h, const float* const inputs[6], int64_t batch,
                             float* out_z, void* stream);
ddf_status ddf_backward(ddf_handle h, const float* dz, int64_t batch, void* stream);

/* Copies the last computed gradient (blob layout) to device memory dev_grad
 * (ddf_param_count floats). Asynchronous on stream. */
ddf_status ddf_copy_grad(ddf_handle h, float* dev_grad, size_t n_floats, void* stream);

/* Replaces the FP32 master weights of a loaded bf16 handle from a device blob
 * (same layout and size as ddf_load_weights; values are not checked for
 * finiteness) and refreshes the bf16 copies every query and training step
 * uses. Asynchronous on stream; the blob may be reused once the stream has
 * passed this call. */
ddf_status ddf_load_weights_device(ddf_handle h, const float* dev_blob, size_t n_floats,
                                   void* stream);

/* ---- the distillation schedule (Sec. 3.2 / 3.4) ----
 * ddf_sample_rays: n training rays into rays_out (6 device float arrays): a
 * fraction surface_frac anchored on the scene (a point uniform by area over
 * the primitives' surfaces, offset 1e-3 along the normal, a direction
 * uniform on the sphere: the "rays that start on the surface and point in
 * all directions" of Sec. 3.2), the rest camera rays (origin uniform on a
 * face of the box [-1,1]^3, aimed at a point uniform in [-0.9,0.9]^3). The
 * surface element (a sphere or one box face) is drawn with an integer weight
 * floor(area 2^24), the area a float32 product clamped to [0, 2^16]; a
 * scene of zero total area gives camera rays only. Counter-based
 * SplitMix64: (seed, step, i) fixes ray i. Primitive arrays as
 * ddf_cast_scene, at most 1024 spheres and 1024 boxes (else
 * DDF_ERR_INVALID_ARG). Asynchronous.
 * ddf_shift_rays: the ray-march shifted points of Sec. 3.2: every ray
 * i in [first, n) with hit[i] moves forward by s = u t[i] (u uniform in
 * [0, 1), from (seed, step, i)) and t[i] becomes t[i] - s. Asynchronous.
 * ddf_distill: `steps` steps of `batch` rays on h (a ray or hash-grid field):
 * sample (surface_frac surface-anchored), cast exact targets, shift the last
 * round(shift_frac batch) rays, ddf_train_step with lr following a cosine
 * from lr0 to 0.05 lr0 (Sec. 3.4: 3e-3, batch 16,384, 30 % shifted).
 * losses: host float[steps] or NULL. Allocates its batch buffers for the
 * call; synchronous. */
ddf_status ddf_sample_rays(const float* spheres, int32_t n_spheres, const float* boxes,
                           int32_t n_boxes, uint64_t seed, uint64_t step, int64_t n,
                           float surface_frac, float* const rays_out[6], void* stream);
ddf_status ddf_shift_rays(float* const rays[6], float* t, const uint8_t* hit, int64_t n,
                          int64_t first, uint64_t seed, uint64_t step, void* stream);
ddf_status ddf_distill(ddf_handle h, const float* spheres, int32_t n_spheres, const float* boxes,
                       int32_t n_boxes, int64_t steps, int64_t batch, float lr0,
                       float surface_frac, float shift_frac, uint64_t seed, float* losses,
                       void* stream);

/* ---- shadow and ambient-occlusion images (the application, Sec. 3.3) ----
 * For a pinhole camera (camera = eye[3], target[3], up[3], fov_y in radians;
 * pixel (x, y), row 0 at the top, looks along f + sx r + sy u with
 * sx = (2 (x + 0.5) / width - 1) tan(fov_y / 2) width / height,
 * sy = (1 - 2 (y + 0.5) / height) tan(fov_y / 2), f = (target - eye)/|.|,
 * r = f x up / |.|, u = r x f): the exact primary hit on the analytic scene,
 * its shading point 1e-3 off the surface along the normal (facing the eye),
 * one shadow ray toward `light` and `ao_samples` cosine-weighted hemisphere
 * rays (Malley's method in the Duff et al. basis; uniforms from SplitMix64
 * per (seed, pixel, sample)). The secondary rays are answered by the field h
 * (occluded iff z1 > 0 and t below the light distance; a hemisphere ray
 * counts when z1 > 0), or by the exact caster when h is NULL (the reference
 * image). out_shadow (device float[height x width], nullable): 1 lit, 0 in
 * shadow; out_ao (nullable): 1 - mean hit flag; background pixels -1.
 * Allocates its ray buffers for the call; synchronous. */
ddf_status ddf_render_gi(ddf_handle h, const float* spheres, int32_t n_spheres,
                         const float* boxes, int32_t n_boxes, const float camera[10],
                         int32_t width, int32_t height, const float light[3], int32_t ao_samples,
                         uint64_t seed, float* out_shadow, float* out_ao, void* stream);

/* ---- Gaussian-rendered depth: the supervision source of Sec. 3.2 that the
 * study of Sec. 4.2 finds too blurry for thin parts ----
 * ddf_render_gs_depth: depth images of n 3D Gaussians (means: device float
 * n x 3; covs: device float n x 6 = (xx, xy, xz, yy, yz, zz) of each
 * world-space covariance; opacities: device float[n]) in n_views pinhole
 * views (cameras: host float n_views x 10, each as for ddf_render_gi), by the
 * 3DGS depth composite: screen covariance J V C V^T J^T + 0.3 I (EWA, V the
 * view rotation, J the projection's Jacobian at the mean; square pixels, the
 * pixel centres of ddf_render_gi); Gaussians with view depth z <= 0.05
 * culled; per pixel front to back by z (equal z: lower index first)
 * alpha = min(0.99, o exp(-q / 2)), q the Mahalanobis distance of the pixel
 * centre in the screen covariance, contributions with alpha < 1/255 skipped,
 * D += T alpha z, A += T alpha, T *= 1 - alpha from T = 1, stopping once
 * T < 1e-4. Writes out_t (device float n_views x height x width, view-major,
 * row 0 at the top): the expected distance along the pixel ray,
 * (D / A) / (d . f), or +inf where A = 0; out_hit (device uint8, same
 * layout): A > 0.5. n <= 2^31; at most 2^31 pixels over all views.
 * Allocates its tile lists for the call; synchronous.
 * ddf_camera_rays: the pixel-centre rays of the same views (origins = eye,
 * unit directions) into 6 device float arrays of n_views x height x width
 * rows, in the layout of out_t. Synchronous.
 * ddf_distill_pool: like ddf_distill, but each step's batch is drawn with
 * replacement from a fixed pool of supervised rays (pool: 6 device float
 * arrays of n_pool rows; pool_t: device float[n_pool], read where pool_hit
 * is set; pool_hit: device uint8[n_pool]): batch row i copies pool row
 * floor(u n_pool), u 32 uniform bits of (seed, step, i); then the shift of
 * ddf_shift_rays on the last round(shift_frac batch) rows and ddf_train_step
 * with the cosine rate of ddf_distill. The pool is not modified.
 * 1 <= n_pool <= 2^31. Synchronous. */
/* ddf_enter_box: a field encodes ray origins inside the box [-1, 1]^3 (the
 * box that bounds the normalised object, Sec. 3.4), so a ray from a camera
 * outside it is first moved to where it enters the box: for n rays (6 device
 * float arrays, updated in place) the slab-test entry distance e (0 when the
 * origin is inside or the ray misses the box [-half_extent, half_extent]^3)
 * moves the origin to o + e d; t (device float[n], nullable) becomes
 * max(t - e, 0) where finite; out_t_in (device float[n], nullable) receives
 * e. Asynchronous. */
ddf_status ddf_enter_box(float* const rays[6], float* t, float* out_t_in, int64_t n,
                         float half_extent, void* stream);
ddf_status ddf_render_gs_depth(const float* means, const float* covs, const float* opacities,
                               int64_t n, const float* cameras, int32_t n_views, int32_t width,
                               int32_t height, float* out_t, uint8_t* out_hit, void* stream);
ddf_status ddf_camera_rays(const float* cameras, int32_t n_views, int32_t width, int32_t height,
                           float* const rays_out[6], void* stream);
ddf_status ddf_distill_pool(ddf_handle h, const float* const pool[6], const float* pool_t,
                            const uint8_t* pool_hit, int64_t n_pool, int64_t steps,
                            int64_t batch, float lr0, float shift_frac, uint64_t seed,
                            float* losses, void* stream);

/* Copies the last computed gradient (weight-blob layout, ddf_param_count
 * floats) to host memory. Synchronous. */
ddf_status ddf_get_grad(ddf_handle h, float* host_grad, size_t n_floats);

/* Activation checkpointing for training sinusoidal ray and SDF fields
 * (the recomputation of activations "where memory asks for it"): segment
 * <= 1 keeps every layer's output for the backward (the default). Segment
 * k >= 2 keeps the outputs of layers k-1, 2k-1, ... and of the last layer.
 * The backward then recomputes each run of dropped layers from the kept
 * layer below it, just before it needs them. Gradients are bitwise those of
 * segment 1: the forward GEMMs are deterministic. Activation memory falls
 * from H buffers of batch x width bf16 to about H/k + k - 1 of them, at the
 * cost of recomputing the dropped layers once per step. The training
 * buffers are laid out anew by the next training call, and activations kept
 * by ddf_forward_train are dropped. Synchronises the device.
 * DDF_ERR_UNSUPPORTED on hash-grid fields. */
ddf_status ddf_set_recompute(ddf_handle h, int32_t segment);

/* Bytes of device memory the activation buffers of the last training batch
 * occupy (0 before the first training call). */
ddf_status ddf_get_train_activation_bytes(ddf_handle h, size_t* out);

/* Training checkpoints (resume a distillation run): ddf_save_checkpoint
 * writes to `path` the field's configuration, its FP32 master weights and,
 * once it has taken an Adam step, the Adam moments and step count, guarded
 * by a CRC-32 (the ISO-HDLC / zlib definition) of everything after the
 * 64-byte header. Layout, little-endian: "DDFCKPT\0", u32 version 1, u32
 * flags (bit 0: optimizer state), the ddf_config, u64 parameter count, i64
 * step, u32 CRC, u32 0, then the weights [, m, v] as float arrays in the
 * blob layout. ddf_load_checkpoint reads one into a handle of the same
 * configuration (the device field aside): the weights as ddf_load_weights
 * would, then the optimizer state (or a reset one), so that k steps, a save,
 * a load into a fresh handle and n - k more steps give the weights of n
 * steps bit for bit (hash-grid fields: up to the atomics of their table
 * gradient). Errors: DDF_ERR_INVALID_ARG for a file that cannot be opened,
 * is not a checkpoint of this version or holds another configuration;
 * DDF_ERR_BAD_WEIGHTS for a wrong size or CRC (the handle is left as it
 * was). Synchronous. */
ddf_status ddf_save_checkpoint(ddf_handle h, const char* path);
ddf_status ddf_load_checkpoint(ddf_handle h, const char* path);

/* Test hook for the out-of-memory paths: the (after + 1)-th device
 * allocation the library makes for a handle from now on (weights,
 * workspaces, training buffers; process-wide count) fails as if the device
 * were full, and the hook switches itself off; after < 0 switches it off at
 * once. The failing call returns DDF_ERR_OOM and releases what it had
 * allocated, so the handle can repeat the call once memory is available. */
ddf_status ddf_debug_fail_allocation(int64_t after);

/* Zeroes the Adam moments and step count. */
ddf_status ddf_reset_optimizer(ddf_handle h);

/* Exact first-hit distance of n rays against a union of spheres and
 * axis-aligned boxes (the exact-cast supervision of Sec. 3.2 with analytic
 * primitives): spheres = n_spheres x (cx, cy, cz, r), boxes = n_boxes x
 * (lox, loy, loz, hix, hiy, hiz), device floats, at most 1024 of each. For
 * each ray the smallest positive root over all primitives (surfaces, not
 * CSG; tangent rays hit; slabs are closed): out_t (device float[n], +inf on a
 * miss) and out_hit (device uint8[n]). No handle needed. Asynchronous. */
ddf_status ddf_cast_scene(const float* spheres, int32_t n_spheres, const float* boxes,
                          int32_t n_boxes, const float* const rays[6], int64_t n, float* out_t,
                          uint8_t* out_hit, void* stream);

/* ---- SDF fields (kind DDF_KIND_SDF): the sphere-tracing baseline ----
 * Blob layout as for ray fields but with a 1-row head (W weights, 1 bias);
 * the output is the raw value s = z0. Ray-field entry points reject SDF
 * handles and the other way round. */

/* out_s[i] = SDF(p_i) for n points (points: 3 device float arrays). Async. */
ddf_status ddf_sdf_eval(ddf_handle h, const float* const points[3], int64_t n, float* out_s,
                        void* stream);

/* Sphere tracing (Sec. 4.4): per ray t = 0, then up to max_steps times
 * s = SDF(o + t d); s < eps: hit at t; else t += s, and the ray stops as a
 * miss once t > t_max. Every step is one full network evaluation of the rays
 * still active, compacted on the device (no host round trip). Writes out_t
 * (device float[n]: t at the hit, else where the ray stopped), out_hit
 * (device uint8[n]) and out_steps (device int32[n], nullable: evaluations
 * used). n <= the chunk size (ddf_set_chunk_rays); max_steps >= 1, eps > 0
 * and t_max >= 0 finite (t_max 0: a ray that does not hit at t = 0 is a miss
 * after its first step). Asynchronous. */
ddf_status ddf_sphere_trace(ddf_handle h, const float* const rays[6], int64_t n, int32_t max_steps,
                            float eps, float t_max, float* out_t, uint8_t* out_hit,
                            int32_t* out_steps, void* stream);

/* SDF regression (distils the baseline network): L = mean |s(p) - s*| over
 * the batch (points: 3 device float arrays, s_target: device float[batch]);
 * gradient into the handle (ddf_get_grad) or followed by one Adam step. Same
 * batch rules and optimiser as ddf_compute_grad / ddf_train_step. */
ddf_status ddf_sdf_compute_grad(ddf_handle h, const float* const points[3], const float* s_target,
                                int64_t batch, float* out_loss, void* stream);
ddf_status ddf_sdf_train_step(ddf_handle h, const float* const points[3], const float* s_target,
                              int64_t batch, float lr, float* out_loss, void* stream);

/* Closed-form signed distance to a union of spheres and boxes (same
 * primitive arrays as ddf_cast_scene) at n points; no handle. Async. */
ddf_status ddf_union_sdf(const float* spheres, int32_t n_spheres, const float* boxes,
                         int32_t n_boxes, const float* const points[3], int64_t n, float* out_s,
                         void* stream);

/* Device status word of the handle: bit 0 = a pipeline wait timed out,
 * bit 1 = a scheduler wait timed out. Synchronises the device, stores the
 * word in *out and clears it. */
ddf_status ddf_check_status(ddf_handle h, uint32_t* out);

/* Wait limit, in nanoseconds, for every device-side wait of later launches
 * (default 2e9). Setting 0 makes any wait that does not succeed at once give
 * up, which exercises the timeout path without faulting the device. */
ddf_status ddf_set_timeout_ns(ddf_handle h, uint64_t ns);

/* Rays per internal chunk of a query (default 1,048,576; minimum 128). Sets
 * the workspace size: about chunk * (4 W + D_in) bytes at bf16/fp8 and twice
 * that at FP32. */
ddf_status ddf_set_chunk_rays(ddf_handle h, int64_t chunk);

/* Tensor-core tile of the layer kernel.
 *   bn         N tile, 128 or 256 (256 needs width % 256 == 0)
 *   epi_warps  epilogue warps draining the TMEM accumulator: 4, or 8 (two per
 *              TMEM lane quarter, each draining half the columns)
 *   cta_pair   1: the 256 x 256 tile a cluster of two CTAs computes with one
 *              pair MMA (needs bn 256)
 *   staged     1: activations leave through shared memory as whole 128-byte
 *              lines instead of per-thread 16-byte pieces (pair tile, or the
 *              fused layer-1 tile)
 *   fused_encode
 *              1: layer 1 only (which = 1). The kernel builds the encoded
 *              rays (Sec. 4.3) in shared memory from the ray arrays instead
 *              of reading an encoded copy from device memory, and keeps each
 *              128-ray block for all its column tiles. Needs bn 256, no pair,
 *              staged 1, 6 + 12 octaves <= 128, width % 256 == 0, more than
 *              one hidden layer and a ray (DDF) field. Results are bitwise
 *              those of the unfused layer 1 with the same epilogue. */
typedef struct {
  int32_t bn;
  int32_t epi_warps;
  int32_t cta_pair;
  int32_t staged;
  int32_t fused_encode;
} ddf_tile;

/* Tile of layer 1 (which = 1) or of layers 2..H (which = 0). Results agree
 * across tiles up to FP32 rounding of the head sums. Default: bn 256 where
 * possible, 4 warps, no pair, not staged, for both. Synchronises the device
 * when weights are loaded. */
ddf_status ddf_set_tile(ddf_handle h, int32_t which, const ddf_tile* tile);
ddf_status ddf_get_tile(ddf_handle h, int32_t which, ddf_tile* tile);

/* Autotuner over the 9 candidate tiles {256,4,0,0,0}, {256,8,0,0,0},
 * {128,4,0,0,0}, {128,8,0,0,0}, {256,4,1,0,0}, {256,4,1,1,0},
 * {256,8,1,1,0}, {256,4,0,1,1}, {256,8,0,1,1} on n rays (device SoA,
 * 1 <= n <= 2^24) on stream. Phase 1 uses one of the first 7 for every layer
 * and keeps the fastest for layers 2..H; phase 2 keeps that and tries all 9
 * for layer 1 (the last two fuse the encoding into it). Every configuration must give t
 * and vis within 1e-3 (relative to max(1, |ref|)) of the first configuration
 * tried before it is timed. The passing candidates are then timed round-robin
 * over 3 rounds, one query each, and keep their best round (so a clock that
 * drifts under the power cap affects all alike): phase 1 times every launch
 * of the query, phase 2 the encoding and layer-1 launches only (CUDA events
 * around each launch). ms_out (nullable,
 * n_out >= 18) receives the per-query ms of phase 1 in [0..8] (7, 8 unused)
 * and of phase 2 in [9..17], -1 where a candidate was skipped or rejected.
 * Synchronous; allocates 16 n bytes of device memory while it runs. A no-op
 * on FP32 handles. */
ddf_status ddf_autotune(ddf_handle h, const float* const rays[6], int64_t n, void* stream,
                        double* ms_out, int32_t n_out);

/* Kernel timing. When on, the library brackets every launch with CUDA events
 * on the launching stream, grouped by kernel class:
 *   0 encode, 1 hidden-layer GEMM (layers 2..H), 2 head/finish, 3 first-layer GEMM.
 * ddf_profile_read synchronises, then stores per class the summed device time
 * in milliseconds (ms[4]) and launch counts (launches[4]), and resets them. */
ddf_status ddf_profile_enable(ddf_handle h, int32_t on);
ddf_status ddf_profile_read(ddf_handle h, double ms[4], int64_t launches[4]);

#ifdef __cplusplus
}
#endif
#endif /* DDF_H_ */

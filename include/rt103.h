/*
 * rt103.h -- C ABI of librt103, a GB300 (sm_103a) implementation of the
 * data-parallel hot path of differentiable radio ray tracing as described in
 * Hoydis et al., "Learning Radio Environments by Differentiable Ray Tracing"
 * (arXiv 2311.18558):
 *
 *   specular path tracing (shoot-and-bounce candidates, image method,
 *   visibility; Sec. II-F)  ->  path coefficients a_i and delays tau_i
 *   (Eq. cfr_cont, Sec. II-C/D)  ->  CFR H[n] = sum_i a_i exp(-j2pi f_n tau_i)
 *   (Sec. II-A), with adjoints of the field and CFR steps for gradient-based
 *   calibration (Sec. III, Algorithm 1) and a neural-material MLP (Sec. III-D).
 *
 * Conventions shared by every call
 *   - Units are SI (m, s, Hz, S/m).  Complex numbers are interleaved {re, im}
 *     float32 pairs ("complex64").  The time convention is exp(+j omega t), so a
 *     delay tau contributes exp(-j 2 pi f tau) and eta = eps_r - j sigma/(eps0 omega).
 *   - Pointers named *_dev are device pointers owned by the caller; *_host are
 *     host pointers read during the call only.  Opaque handles (rt_ctx,
 *     rt_scene, rt_paths) are owned by the library and released with the
 *     matching *_free / rt_destroy call.  A paths object refers to its scene:
 *     free the paths before the scene.
 *   - Every call is ordered on the context's CUDA stream (rt_create /
 *     rt_set_stream) and returns before the GPU work finishes, except where a
 *     call says it synchronises.  Device buffers must stay valid until then.
 *   - Every call returns an rt_status.  Invalid arguments are rejected on the
 *     host before any launch.  Kernels never trap: a device-side problem (a
 *     bounded loop that ran out, a full buffer) sets a sticky status word that
 *     rt_status_word reads.  rt_last_error gives a message for the last failure
 *     of a context (valid until the next call on that context).
 *   - A context is not thread-safe; use one per host thread.
 */
#ifndef RT103_H
#define RT103_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rt_ctx rt_ctx;
typedef struct rt_scene rt_scene;
typedef struct rt_paths rt_paths;

typedef enum {
    RT_OK = 0,
    RT_ERR_INVALID_ARG = 1,     /* rejected on the host, nothing launched           */
    RT_ERR_CUDA = 2,            /* a CUDA runtime call failed                        */
    RT_ERR_OOM = 3,             /* device allocation failed                          */
    RT_ERR_CAPACITY = 4,        /* an internal buffer overflowed (see message)       */
    RT_ERR_STACK_OVERFLOW = 5,  /* BVH traversal stack overflow (device status)      */
    RT_ERR_ITER_LIMIT = 6,      /* a bounded device loop ran out (device status)     */
    RT_ERR_TIMEOUT = 7,         /* a bounded device wait ran out (device status)     */
    RT_ERR_NUMERIC = 8,         /* NaN/Inf or out-of-domain input                    */
    RT_ERR_UNSUPPORTED = 9      /* valid but not supported by this build             */
} rt_status;

/* ------------------------------------------------------------------ context */

/* Create a context on CUDA device `device`, ordering work on `cuda_stream`
 * (a cudaStream_t; NULL = legacy default stream).  *out receives the handle. */
rt_status rt_create(int device, void* cuda_stream, rt_ctx** out);
rt_status rt_destroy(rt_ctx* ctx);
/* Change the stream subsequent calls are ordered on. */
rt_status rt_set_stream(rt_ctx* ctx, void* cuda_stream);
/* Message of the last failed call on ctx (never NULL; "" if none). */
const char* rt_last_error(const rt_ctx* ctx);
/* Synchronises the stream, writes the sticky device status word (an
 * rt_status value, RT_OK if none) to *device_error and clears it. */
rt_status rt_status_word(rt_ctx* ctx, int32_t* device_error);
/* Library version string. */
const char* rt_version(void);

/* Instrumentation (no counterpart in the paper; used by the benchmark).
 * flags bit 0: time the stages of rt_trace_paths with CUDA events (recorded on
 * the stream; the trace does not wait for them, rt_profile_read does);
 * flags bit 1: count BVH node visits and triangle tests in the tracing kernels
 * (adds atomics; leave off when timing). */
rt_status rt_set_profiling(rt_ctx* ctx, int32_t flags);
/* Reads the instrumentation of ctx (any pointer may be NULL):
 *   launches      number of kernels this context launched so far
 *   stage_ms[8]   last trace (waits for its last stage event if not read yet;
 *                 a trace not read before the next one starts is dropped):
 *                 SBR, dedup+sort, image method, visibility,
 *                 emission+records, total, then within SBR the shoot-and-bounce
 *                 kernel alone and the FP64 re-trace (bit 0 set, else zeros)
 *   counters[8]   since the last rt_set_profiling: SBR node visits, SBR triangle
 *                 tests, SBR closest-hit queries, FP64 re-traced rays,
 *                 visibility node visits, visibility triangle tests, visibility
 *                 segments, (candidate, receiver) pairs tested */
rt_status rt_profile_read(rt_ctx* ctx, int64_t* launches, double* stage_ms, int64_t* counters);

/* ------------------------------------------------------------------ scene */

/* Upload a triangle mesh (Sec. II-F: the scene is a set of triangles, each
 * belonging to an object with a material, Sec. II-D) and build its BVH.
 *   verts_host       n_verts x 3 float32 positions [m]
 *   tris_host        n_tris x 3 int32 vertex indices; the geometric normal is
 *                    (v1-v0) x (v2-v0); reflection is two-sided
 *   tri_material_host n_tris int32 material index in [0, n_materials)
 *   material_is_pec_host n_materials uint8, 1 = perfect electric conductor
 *                    (r_perp = -1, r_par = +1, the |eta| -> inf limit of
 *                    Eq. fresnel-1/2)
 * Limits: 1 <= n_tris <= 65535 (triangle sequences are packed in 16-bit
 * fields), finite coordinates, non-degenerate triangles.  Synchronises. */
rt_status rt_scene_upload(rt_ctx* ctx, const float* verts_host, int32_t n_verts,
                          const int32_t* tris_host, int32_t n_tris,
                          const int32_t* tri_material_host, int32_t n_materials,
                          const uint8_t* material_is_pec_host, rt_scene** out);
rt_status rt_scene_free(rt_scene* scene);
/* n_tris, BVH node count and bounding-box diagonal [m] of a scene. */
rt_status rt_scene_info(const rt_scene* scene, int32_t* n_tris, int32_t* n_nodes, double* diag);

/* ------------------------------------------------------------------ tracing */

/* Specular path tracing, Sec. II-F: n_rays rays leave the transmitter along a
 * Fibonacci lattice (direction i: z = 1-(2i+1)/N, r = sqrt(1-z^2),
 * phi = 2 pi frac(i (sqrt5-1)/2), evaluated in FP64 and rounded to FP32) and
 * bounce specularly up to max_depth times (k_r = k_i - 2 (k_i.n) n, Sec. II-D);
 * every prefix of every ray's triangle sequence, plus the empty sequence (line
 * of sight), is a candidate; duplicates are removed; the image method turns each
 * (candidate, receiver) pair into an exact specular chain or rejects it; every
 * segment of a surviving chain must be unobstructed.  Paths whose reflection
 * points coincide on coplanar triangles are kept once (lowest triangle
 * sequence).
 *   tx_host    transmitter position, 3 doubles [m]
 *   rx_dev     n_rx x 3 doubles, receiver positions [m]
 *   1 <= max_depth <= 4, 1 <= n_rays <= 2^31-1, 1 <= n_rx <= 2^24
 * *out receives the paths, grouped by receiver and, within a receiver, ordered
 * by (depth, triangle sequence).  Synchronises (the number of candidates and
 * paths sizes the outputs). */
rt_status rt_trace_paths(rt_ctx* ctx, const rt_scene* scene, const double* tx_host,
                         const double* rx_dev, int32_t n_rx, int64_t n_rays,
                         int32_t max_depth, rt_paths** out);

/* Build a paths object from externally supplied chains (e.g. another tracer):
 *   rx_dev n_paths int32 receiver index in [0, n_rx), non-decreasing
 *   depth_dev n_paths int32 in [0, max_depth]
 *   tri_seq_dev n_paths x max_depth int32 triangle indices (-1 padded)
 *   points_dev n_paths x (max_depth+2) x 3 doubles: Tx, s_1..s_q, Rx, padding.
 * The per-path geometry records (delays, angles, basis changes) are derived on
 * the device exactly as for traced paths. */
rt_status rt_paths_import(rt_ctx* ctx, const rt_scene* scene, int64_t n_paths, int32_t max_depth,
                          int32_t n_rx, const int32_t* rx_dev, const int32_t* depth_dev,
                          const int32_t* tri_seq_dev, const double* points_dev, rt_paths** out);
/* Number of paths and of deduplicated candidates (0 for imported paths). */
rt_status rt_paths_count(const rt_paths* paths, int64_t* n_paths, int64_t* n_candidates);
/* Copies the n_rx+1 int64 path offsets per receiver to rx_offsets_dev. */
rt_status rt_paths_rx_offsets(const rt_paths* paths, int64_t* rx_offsets_dev);
/* Copies path data into caller buffers (any pointer may be NULL to skip):
 * tri_seq n_paths x max_depth int32 (-1 padded), depth n_paths int32,
 * rx n_paths int32, tau n_paths double [s] = path length / c (Eq.
 * transfer_function), points n_paths x (max_depth+2) x 3 double. */
rt_status rt_paths_export(const rt_paths* paths, int32_t* tri_seq_dev, int32_t* depth_dev,
                          int32_t* rx_dev, double* tau_dev, double* points_dev);
/* Copies the candidate list, n_candidates x max_depth int32 (-1 padded), in
 * (length, lexicographic) order; candidate 0 is the empty sequence. */
rt_status rt_paths_candidates(const rt_paths* paths, int32_t* seq_dev);
/* Read-only device views of the paths' own arrays, without a copy: rx_offsets
 * (n_rx + 1 int64) and tau (n_paths double [s]).  They stay valid until
 * rt_paths_free; the caller must not write through them.  Either output may
 * be NULL. */
rt_status rt_paths_device_views(const rt_paths* paths, const int64_t** rx_offsets_dev, const double** tau_dev);
rt_status rt_paths_free(rt_paths* paths);

/* Batched tracing of n_scenes scenes (Sec. II-F, as rt_trace_paths for each
 * scene) in one pipeline: the shoot-and-bounce stage of all scenes runs as one
 * persistent launch whose warps take rays of any scene, and every later stage is
 * one launch over all scenes.  No counterpart in the paper (a batching of its
 * path tracing).
 *   scenes        n_scenes traceable scenes sharing one material table
 *   tx_host       n_scenes x 3 doubles
 *   rx_dev        all receivers, scene after scene (sum of rx_counts x 3 doubles)
 *   rx_counts_host n_scenes int32, each >= 1
 *   n_rays, max_depth  as rt_trace_paths, for every scene
 * *out receives ONE paths object over all receivers (in that order); triangle
 * ids in it are offset per scene (rt_paths_batch_info), and its materials are
 * the shared table.  Per scene the paths equal those of rt_trace_paths.
 * Synchronises. */
rt_status rt_trace_batch(rt_ctx* ctx, const rt_scene* const* scenes, int32_t n_scenes, const double* tx_host,
                         const double* rx_dev, const int32_t* rx_counts_host, int64_t n_rays, int32_t max_depth,
                         rt_paths** out);
/* Scenes of a batch output: receiver offsets and triangle-id offsets per scene
 * (each n_scenes + 1 int64, host memory).  *n_scenes = 1 for a single trace. */
rt_status rt_paths_batch_info(const rt_paths* paths, int32_t* n_scenes, int64_t* scene_rx_offsets_host,
                              int64_t* scene_tri_offsets_host);
/* Launch shapes of the tracing kernels (blocks per SM of the SBR, image-method
 * and visibility kernels, each in [1, 64]). */
rt_status rt_set_tuning(rt_ctx* ctx, int32_t sbr_blocks_per_sm, int32_t pairs_blocks_per_sm,
                        int32_t vis_blocks_per_sm);
/* Autotuner: times rt_trace_paths on the given workload for a set of launch
 * shapes (coordinate descent, each knob judged by its own stage time), applies
 * the fastest to ctx and writes it to chosen[3]; *best_ms (may be NULL) gets the
 * summed stage times (0 when the choice came from the per-process cache keyed by
 * device, scene size, rays, depth and receivers).  Synchronises. */
rt_status rt_autotune_trace(rt_ctx* ctx, const rt_scene* scene, const double* tx_host, const double* rx_dev,
                            int32_t n_rx, int64_t n_rays, int32_t max_depth, int32_t* chosen, double* best_ms);

/* ------------------------------------------------------------------ fields */

/* Path coefficients a_i of Eq. cfr_cont for every path:
 *   a_i = lambda/(4 pi) * sqrt(g_T g_R) / L_i * C_R^T D_{Q+1} G_Q D_Q ... G_1 D_1 C_T
 * with the basis changes D_j of Eq. basis_transform, G_j = diag(r_perp, r_par)
 * from Eq. fresnel-1/2 at eta = eps_r - j sigma/(eps0 2 pi freq), spreading of
 * a spherical wave about the image source (product 1/L over the path), S = 0,
 * and vertically polarised isotropic antennas (Eq. polarization_model, zeta=0).
 *   eps_r_dev, sigma_dev  float32, indexed by material (per_triangle = 0, length
 *                         n_materials) or by triangle (per_triangle = 1, n_tris)
 *   freq_hz              frequency of lambda and eta (> 0)
 *   gain_tx, gain_rx     antenna gains g_T, g_R (> 0)
 *   a_dev                n_paths complex64 output
 *   tau_dev              n_paths double output (may be NULL) */
rt_status rt_eval_fields(rt_ctx* ctx, const rt_paths* paths, const float* eps_r_dev,
                         const float* sigma_dev, int32_t per_triangle, double freq_hz,
                         float gain_tx, float gain_rx, void* a_dev, double* tau_dev);
/* Adjoint of rt_eval_fields with the geometry held fixed (Sec. II-F): given
 * grad_a = dL/dRe a + j dL/dIm a (complex64, n_paths), ACCUMULATES (+=)
 *   grad_eps_r[m] += sum Re(conj(g) da/deps_r),  grad_sigma[m] += sum Re(conj(g) da/dsigma)
 * (da/dsigma = -j/(eps0 omega) da/deta), and grad_gain[0..1] += dL/dg_T, dL/dg_R.
 * Any of the three gradient pointers may be NULL. */
rt_status rt_eval_fields_backward(rt_ctx* ctx, const rt_paths* paths, const float* eps_r_dev,
                                  const float* sigma_dev, int32_t per_triangle, double freq_hz,
                                  float gain_tx, float gain_rx, const void* grad_a_dev,
                                  float* grad_eps_r_dev, float* grad_sigma_dev,
                                  float* grad_gain_dev);

/* ------------------------------------------------------------------ CFR */
/* Arithmetic of the CFR calls: FP32 throughout, phases reduced per path in FP64.
 * With N in {256, 512, 1024, 2048, 4096} and the tensor cores selected (the
 * default, rt_set_cfr_tensor_cores), the products run as three TF32 products
 * on tcgen05.  A receiver with more than 4096 paths (up to 4096 such receivers
 * per call) is then evaluated by a non-uniform FFT instead: an exponential-of-
 * semicircle kernel 8 cells wide on a 2N-cell grid, deconvolved per subcarrier.
 * Its approximation error per entry is at most about 4e-7 of sum_i |a_i| (a
 * lone path; far less when many paths' errors average), on top of FP32
 * rounding.  Its segments add into the grid with float atomics, so the rounding
 * of those receivers (not their value) may differ between runs. */

/* Discrete CFR (Sec. II-A): H[r, n] = sum_{i in r} a_i exp(-j 2 pi (f_c + n df) tau_i),
 * n = -N/2 .. N/2-1, written to column n + N/2 of row r.
 *   rx_offsets_dev  n_rx+1 int64, paths of receiver r are [off[r], off[r+1])
 *   a_dev           complex64 per path;  tau_dev double per path [s]
 *   n_sub           N, even (or 1: a single frequency f_c), N <= 4096
 *   H_dev           n_rx x N complex64 output */
rt_status rt_cfr(rt_ctx* ctx, const int64_t* rx_offsets_dev, int32_t n_rx, const void* a_dev,
                 const double* tau_dev, double f_center_hz, double delta_f_hz, int32_t n_sub,
                 void* H_dev);
/* Adjoint of rt_cfr: grad_a[i] = sum_n grad_H[r(i), n] conj(exp(-j 2 pi f_n tau_i))
 * (overwrites grad_a_dev, complex64 per path). */
rt_status rt_cfr_backward(rt_ctx* ctx, const int64_t* rx_offsets_dev, int32_t n_rx,
                          const double* tau_dev, double f_center_hz, double delta_f_hz,
                          int32_t n_sub, const void* grad_H_dev, void* grad_a_dev);
/* CFR, power loss and CFR adjoint in one launch:
 *   L = 1/(n_rx N) sum_{r,n} (w_r (|H[r,n]|^2 - P*[r,n]))^2
 * (an MSE on CFR power; the paper's Algorithm 1 admits any differentiable loss,
 * Sec. III-E), then grad_a = adjoint of rt_cfr applied to dL/dH.
 *   target_power_dev n_rx x N float32 P*;  rx_weight_dev n_rx float32 w_r
 *   loss_dev  one float32 (overwritten);  grad_a_dev complex64 per path (overwritten)
 *   H_dev     n_rx x N complex64 output, or NULL not to store H */
rt_status rt_cfr_power_mse_fused(rt_ctx* ctx, const int64_t* rx_offsets_dev, int32_t n_rx,
                                 const void* a_dev, const double* tau_dev, double f_center_hz,
                                 double delta_f_hz, int32_t n_sub, const float* target_power_dev,
                                 const float* rx_weight_dev, float* loss_dev, void* grad_a_dev,
                                 void* H_dev);
/* With enable = 1, rt_trace_paths returns without waiting for the GPU: its
 * buffers are sized from the counts of the scene's last trace that did wait (the
 * scene's first trace waits in any case), every stage reads the previous stage's
 * counts on the device, and the paths object holds as many slots as were sized:
 * rt_paths_count gives the slots and the receiver offsets give the real layout.
 * rt_eval_fields, rt_eval_fields_backward, the CFR calls and
 * rt_paths_device_views / rt_paths_rx_offsets accept such paths;
 * rt_paths_export, rt_paths_candidates, rt_antenna_apply*, rt_specular_reduction*
 * and rt_trace_diffraction need rt_paths_resolve first.  A capacity that
 * overflowed sets RT_ERR_CAPACITY in the status word (the results of that trace
 * are then invalid; trace again with enable = 0).  With enable = 0 (the default)
 * rt_trace_paths waits once, at its end, and retries with more room on overflow.
 * The paper has no counterpart: this is a property of the library. */
rt_status rt_set_trace_async(rt_ctx* ctx, int32_t enable);
/* Waits for a trace that returned without waiting and fixes its path count on
 * the host (rt_paths_count then gives the paths); RT_ERR_CAPACITY if one of its
 * capacities overflowed.  A no-op on other paths. */
rt_status rt_paths_resolve(rt_paths* paths);

/* Arithmetic of rt_cfr, rt_cfr_backward and rt_cfr_power_mse_fused (and its
 * allocation-free variant): with enable = 1 (the default) and n_sub in {256, 512,
 * 1024, 2048, 4096} the contraction over the paths runs on the tensor cores
 * (tcgen05, TF32 operands split hi + lo, three products per term, FP32
 * accumulation); otherwise, and with enable = 0, on the FP32 SIMT units.  Both
 * compute the same quantities to FP32 accuracy.  A bounded device wait that runs
 * out sets RT_ERR_TIMEOUT in the status word. */
rt_status rt_set_cfr_tensor_cores(rt_ctx* ctx, int32_t enable);
/* Poll limit of the waits in which one CTA of the CFR calls waits for work of
 * another (the receivers of more than 4096 paths, split over CTAs: waits for
 * their classification, publication and finished forward sums).  polls = 0
 * restores the default, 2^22 polls; 1 <= polls <= 2^22 sets it.  A wait that
 * runs out sets RT_ERR_TIMEOUT in the status word, the kernel finishes without
 * the work it waited for (outputs of that call are then undefined) and later
 * calls are unaffected.  The waits of a CTA on its own tensor-core products keep
 * their fixed bound.  The paper has no counterpart: this exists so that the
 * time-out path can be exercised with a short limit.  polls outside [0, 2^22]
 * returns RT_ERR_INVALID_ARG. */
rt_status rt_set_wait_limit(rt_ctx* ctx, int32_t polls);

/* ------------------------------------------------------------------ antenna patterns */

/* Trainable antenna patterns (Sec. III-B, Eq. polarization_model with zeta = 0):
 * the directional gain is a mixture of M spherical Gaussians,
 *   G(r) = 4 pi eta sum_m w_m exp(lambda_m mu_m . r) / a_m,
 *   a_m = (2 pi / lambda_m) (exp(lambda_m) - exp(-lambda_m)),
 * whose integral over the sphere is 4 pi eta (the factor 4 pi is the reading
 * that matches the paper's normalisation), and a path's coefficient scales by
 * sqrt(G_T(k_1) G_R(-k_{q+1})) with k_1 its departure direction and -k_{q+1}
 * its arrival direction seen from the receiver (from the path records).
 *   *_pattern_dev  1 + 5 M floats {eta, then per lobe w, lambda (> 0), mu_x, mu_y,
 *                  mu_z (unit)}, or NULL for a unit gain on that side; 1 <= M <= 8
 *   a_dev          complex64 per path (e.g. from rt_eval_fields with unit gains)
 *   a_out_dev      complex64 per path, a sqrt(G_T G_R) (may alias a_dev)
 *   gain_*_dev     per-path G_T and G_R (float32; may be NULL when not needed) */
rt_status rt_antenna_apply(rt_ctx* ctx, const rt_paths* paths, const float* tx_pattern_dev, int32_t tx_lobes,
                           const float* rx_pattern_dev, int32_t rx_lobes, const void* a_dev, void* a_out_dev,
                           float* gain_tx_dev, float* gain_rx_dev);
/* Adjoint of rt_antenna_apply given dL/da_out (PyTorch convention):
 *   grad_a_dev    dL/da = sqrt(G_T G_R) dL/da_out (overwritten; may be NULL)
 *   grad_*_dev    dL/d(eta, w, lambda, mu) of each given pattern, same packing,
 *                 ACCUMULATED (+=); mu is treated as a free 3-vector.
 * a_out_dev and gain_*_dev are the outputs of the forward call. */
rt_status rt_antenna_apply_backward(rt_ctx* ctx, const rt_paths* paths, const float* tx_pattern_dev,
                                    int32_t tx_lobes, const float* rx_pattern_dev, int32_t rx_lobes,
                                    const void* a_out_dev, const float* gain_tx_dev, const float* gain_rx_dev,
                                    const void* grad_out_dev, void* grad_a_dev, float* grad_tx_dev,
                                    float* grad_rx_dev);

/* ------------------------------------------------------------------ diffuse reflection */

/* Diffuse reflection found by next-event estimation (Sec. II-F; the diffuse
 * reflection model of Sec. II-D, Eq. scattered_field).  n_rays rays leave the
 * transmitter along the same Fibonacci lattice as rt_trace_paths and bounce
 * specularly up to max_depth times (closest hits decided in FP64); at each hit
 * s_j the ray is scattered towards every receiver strictly on the side of t_j's
 * plane it came from that sees s_j (nothing but t_j on the segment for
 * t in (eps, len - eps), eps = 1e-6 scene diagonal), giving the path
 * Tx -> s_1 .. s_{j-1} (specular) -> s_j (diffuse) -> Rx of depth j.
 *   tx_host  3 doubles;  rx_dev  n_rx x 3 doubles [m]
 *   1 <= max_depth <= 4, 1 <= n_rays, n_rays * max_depth < 2^31, 1 <= n_rx <= 2^24,
 *   and n_rx * n_rays * max_depth / 32 <= 2^31 (the visibility bitmask)
 * *out receives a paths object of the diffuse kind, grouped by receiver and
 * ordered by (launch ray, j) within a receiver; rt_paths_count,
 * rt_paths_rx_offsets, rt_paths_export (points Tx, s_1..s_j, Rx; tau =
 * path length / c), rt_antenna_apply and rt_paths_free accept it; rt_eval_fields
 * rejects it.  Synchronises (the path count sizes the outputs). */
rt_status rt_trace_diffuse(rt_ctx* ctx, const rt_scene* scene, const double* tx_host, const double* rx_dev,
                           int32_t n_rx, int64_t n_rays, int32_t max_depth, rt_paths** out);

/* Coefficients of diffuse paths (Eq. scattered_field; chi_1 = chi_2 = 0 unless
 * phases were attached with rt_set_diffuse_phases):
 * the specular prefix as rt_eval_fields with R = sqrt(1 - S^2) per bounce
 * (Eq. specular_reflection), then at s_j
 *   |E_s| = sqrt(4 pi / n_rays) S sqrt(f_s) |diag(r_perp, r_par) v|
 * (v the incident field in the incidence basis without the spreading 1/l_j,
 * which cancels against cos(theta_i) dA = 4 pi l_j^2 / n_rays: each launch ray
 * samples the solid angle 4 pi / n_rays), the polarisation [sqrt(1 - K_x) e^{j chi_1},
 * sqrt(K_x) e^{j chi_2}] in the basis e_perp = k_s x n / |k_s x n|,
 * e_par = e_perp x k_s, and
 *   a = lambda / (4 pi) sqrt(g_T g_R) |E_s| / d_last (D_last row 0 . pol),
 * which is real when chi = 0.  f_s is the trainable scattering pattern of Sec. III-C:
 *   f_s = w_1 / pi (k_s . n) + w_2 g(lambda_2, -k_i . k_s) + w_3 g(lambda_3, k_r . k_s),
 *   g(lambda, c) = exp(lambda c) / a(lambda, cos theta_i), a = s U + (1 - s) L
 * with U = 2 pi / lambda (e^lambda - 1), L = 2 pi / lambda (1 - e^-lambda) and the
 * smooth step s(t(lambda), cos theta_i) of Sec. III-C.
 *   eps_r_dev, sigma_dev  float32 per material (n_materials)
 *   scat_dev              n_materials x 8 float32: S, K_x, w_1, w_2, w_3, lambda_2,
 *                         lambda_3, unused; 0 <= S <= 1, 0 <= K_x <= 1, lambda > 0
 *   a_dev                 n_paths complex64 output;  tau_dev  n_paths double (may be NULL) */
rt_status rt_eval_fields_diffuse(rt_ctx* ctx, const rt_paths* paths, const float* eps_r_dev, const float* sigma_dev,
                                 const float* scat_dev, double freq_hz, float gain_tx, float gain_rx, void* a_dev,
                                 double* tau_dev);
/* Adjoint of rt_eval_fields_diffuse, geometry held fixed: given grad_a (complex64),
 * ACCUMULATES (+=) dL/d eps_r, dL/d sigma (per material) and dL/d scat
 * (n_materials x 8, the last column untouched).  Gradient pointers may be NULL. */
rt_status rt_eval_fields_diffuse_backward(rt_ctx* ctx, const rt_paths* paths, const float* eps_r_dev,
                                          const float* sigma_dev, const float* scat_dev, double freq_hz,
                                          float gain_tx, float gain_rx, const void* grad_a_dev,
                                          float* grad_eps_r_dev, float* grad_sigma_dev, float* grad_scat_dev);

/* Attaches the random phases chi_1, chi_2 of Eq. scattered_field to a diffuse
 * paths object: chi_dev holds n_paths x 2 float32 (radians, in path order) and
 * stays owned by the caller, who keeps it alive and unchanged while the paths
 * are evaluated; NULL restores chi = 0.  rt_eval_fields_diffuse and its adjoint
 * read it. */
rt_status rt_set_diffuse_phases(rt_ctx* ctx, rt_paths* paths, const float* chi_dev);

/* Specular share of the reflected energy (Sec. II-D, Eq. specular_reflection):
 * a_out[i] = a[i] prod_b sqrt(1 - S_b^2) over the bounces of specular path i,
 * S_b = scat_dev[8 m_b] of the bounce's material.  a_out may alias a. */
rt_status rt_specular_reduction(rt_ctx* ctx, const rt_paths* paths, const float* scat_dev, const void* a_dev,
                                void* a_out_dev);
/* Adjoint: grad_a = prod_b R_b grad_out (may be NULL); ACCUMULATES
 * dL/dS_m = sum Re(conj(g) a_out) sum_{b: m_b = m} (-S_m / (1 - S_m^2)) into
 * grad_scat_dev[8 m] (may be NULL; needs a_out_dev). */
rt_status rt_specular_reduction_backward(rt_ctx* ctx, const rt_paths* paths, const float* scat_dev,
                                         const void* a_out_dev, const void* grad_out_dev, void* grad_a_dev,
                                         float* grad_scat_dev);

/* ------------------------------------------------------------------ diffraction */

/* Wedges of the scene's mesh for first-order diffraction (Sec. II-D Eq.
 * diffraction: infinitely long wedges whose two faces may have different
 * materials).  Two triangles sharing two vertex positions form an edge; the edge
 * is a wedge when its exterior angle n pi, measured outside the solid with the
 * triangles' winding normals taken as outward, has 1 < n <= 2 (n = 2: two
 * coincident faces back to back, a screen).  Flat pairs, concave pairs (n < 1),
 * border edges, edges of three or more triangles and pairs of inconsistent
 * winding are not wedges.  The table is built on the host at the first call that
 * needs it (one copy of the triangles to the host) and kept with the scene.
 *   n_wedges    out: number of wedges
 *   faces_host  2 x n_wedges int32 (face 0 < face n, ordered by (face 0, face n)), or NULL
 *   n_host      n_wedges double, n of each wedge, or NULL */
rt_status rt_scene_wedges(rt_ctx* ctx, const rt_scene* scene, int32_t* n_wedges, int32_t* faces_host,
                          double* n_host);

/* First-order diffraction paths Tx -> Q -> Rx (Sec. II-D Eq. diffraction;
 * Sec. II-F: candidate edges identified during shoot-and-bounce, the point of
 * diffraction by Keller's principle of the shortest path).
 *   specular  a specular trace (rt_trace_paths) of the same scene and transmitter:
 *             the wedges with a face among its depth-1 candidates (the triangles
 *             the launch rays hit first) are the candidate wedges.
 * For every (candidate wedge, receiver): Q is the point of the edge line that
 * minimises |Tx - Q| + |Q - Rx| (FP64); the path is valid when Tx and Rx are off
 * the edge line by more than 1e-6 of the scene diagonal (eps), Q lies on the edge
 * piece (half-open: 0 <= x < length from its start vertex), Tx and Rx are strictly
 * in the wedge's exterior, both segments are longer than eps and no triangle other
 * than the two faces cuts them for t in (eps, len - eps).  Output: a paths object
 * of the diffraction kind, grouped by receiver and ordered by wedge within a
 * receiver; rt_paths_export gives depth 1, the two faces as the triangle
 * sequence (the incidence face, i.e. the face on the transmitter's side, first),
 * the points Tx, Q, Rx, (0, 0, 0) and tau = (|Q - Tx| + |Rx - Q|) / c.
 * rt_eval_fields_diffraction, rt_antenna_apply, rt_paths_rx_offsets and
 * rt_paths_free accept it; rt_eval_fields rejects it.  Synchronises twice (the
 * candidate and path counts size the outputs). */
rt_status rt_trace_diffraction(rt_ctx* ctx, const rt_scene* scene, const rt_paths* specular, const double* tx_host,
                               const double* rx_dev, int32_t n_rx, rt_paths** out);

/* Coefficients of diffraction paths: the uniform theory of diffraction
 * (Kouyoumjian and Pathak, Proc. IEEE 1974) with Luebbers' face coefficients
 * (IEEE Trans. AP 1984), the model the paper names for Q, in the edge-fixed frame:
 *   D_{s,h} = -e^{-j pi/4} / (2 n sqrt(2 pi k) sin beta_0) [T1 + T2 + R_0 T3 + R_n T4],
 *   T_i = cot(eps_i / 2n) F(2 k L sin^2(eps_i / 2)) for the reduced angles eps_i of
 *   pi + (phi - phi'), pi - (phi - phi'), pi - (phi + phi'), pi + (phi + phi'),
 *   F(X) = 2 j sqrt(X) e^{jX} int_{sqrt X}^inf e^{-j t^2} dt,
 *   R_0, R_n the Fresnel coefficients (Eq. fresnel-1/2; r_perp for D_s, r_par for
 *   D_h, -1 / +1 for a perfect conductor) of the incidence face at
 *   cos theta = |sin beta_0 sin phi'| and of the other face at
 *   |sin beta_0 sin(n pi - phi)|,
 *   a = lambda / (4 pi) sqrt(g_T g_R) sqrt(s' / (s (s + s'))) / s'
 *       (D_s b_in b_out + D_h p_in p_out),   L = s s' sin^2 beta_0 / (s + s'),
 * with phi', phi the angles of Tx and Rx about the edge from the incidence face,
 * beta_0 the angle between the edge and the incident ray, s' = |Q - Tx|,
 * s = |Rx - Q|, and b_in, p_in (b_out, p_out) the projections of the transmit
 * (receive) polarisation theta_hat on the edge-fixed bases (beta', phi') of the
 * incident and (beta, phi) of the diffracted ray.  Arguments as rt_eval_fields:
 * per_triangle = 0 indexes eps_r_dev / sigma_dev by material, 1 by triangle
 * (perfect conductors are flagged per material in both cases).
 *   a_dev  n_paths complex64 output;  tau_dev  n_paths double (may be NULL) */
rt_status rt_eval_fields_diffraction(rt_ctx* ctx, const rt_paths* paths, const float* eps_r_dev,
                                     const float* sigma_dev, int32_t per_triangle, double freq_hz, float gain_tx,
                                     float gain_rx, void* a_dev, double* tau_dev);
/* Adjoint of rt_eval_fields_diffraction with the geometry held fixed: given
 * grad_a (complex64), ACCUMULATES (+=) dL/d eps_r and dL/d sigma of both faces'
 * materials (dL/dx = Re(conj(g) da/dx), da/dsigma = -j/(eps0 omega) da/deta) and
 * dL/d(g_T, g_R) into grad_gain_dev (2 floats, may be NULL). */
rt_status rt_eval_fields_diffraction_backward(rt_ctx* ctx, const rt_paths* paths, const float* eps_r_dev,
                                              const float* sigma_dev, int32_t per_triangle, double freq_hz,
                                              float gain_tx, float gain_rx, const void* grad_a_dev,
                                              float* grad_eps_r_dev, float* grad_sigma_dev, float* grad_gain_dev);

/* Per-receiver concatenation of two path lists (8-byte elements: complex64
 * coefficients or double delays), so that specular and diffuse paths go through
 * one CFR: dst holds receiver r's elements of src1 ([off1[r], off1[r+1])) followed
 * by its elements of src2; off_out (n_rx + 1 int64, may be NULL) = off1 + off2.
 * rt_rx_split is its adjoint (either destination may be NULL). */
rt_status rt_rx_merge(rt_ctx* ctx, int32_t n_rx, const int64_t* off1_dev, const int64_t* off2_dev,
                      const void* src1_dev, const void* src2_dev, void* dst_dev, int64_t* off_out_dev);
rt_status rt_rx_split(rt_ctx* ctx, int32_t n_rx, const int64_t* off1_dev, const int64_t* off2_dev,
                      const void* src_dev, void* dst1_dev, void* dst2_dev);

/* ------------------------------------------------------------------ CIR, loss and metrics */

/* CIR by N-point IDFT (Sec. II-A): h[r, l + N/2] = N^-1/2 sum_n H[r, n + N/2]
 * exp(+j 2 pi n l / N), n, l = -N/2 .. N/2-1.
 *   H_dev, h_dev  n_rx x N complex64 (distinct buffers);  N a power of two in [2, 4096] */
rt_status rt_cir(rt_ctx* ctx, const void* H_dev, int32_t n_rx, int32_t n_sub, void* h_dev);
/* Per receiver, from its CFR: total channel gain P = sum_l |h[l]|^2 (Eq. channel_gain)
 * and RMS delay spread tau_RMS [s] (Eq. delay_spread, W = N delta_f); tau_RMS = 0
 * where P = 0.  Either output may be NULL. */
rt_status rt_cir_stats(rt_ctx* ctx, const void* H_dev, int32_t n_rx, int32_t n_sub, double delta_f_hz,
                       float* P_dev, float* tau_rms_dev);
/* Power scale of the measurements (Eq. alpha_hat, scaling_param): alpha^ =
 * sum P_meas P_pred / sum P_meas^2 over the n entries, then
 * alpha <- decay alpha + (1 - decay) alpha^ (alpha <- alpha^ on the first call).
 *   state_dev  2 floats {alpha, initialised}, device, updated in place; set to
 *              {0, 0} before the first call.  decay in [0, 1). */
rt_status rt_power_scale_ema(rt_ctx* ctx, const float* P_meas_dev, const float* P_pred_dev, int32_t n,
                             float decay, float* state_dev);
/* The paper's loss (Eq. loss, Eq. smape) averaged over the batch:
 *   L = 1/n_rx sum_r [ SMAPE(tau_meas_r, tau^_r) + SMAPE(alpha P_meas_r, P^_r) ],
 * SMAPE(x, y) = |x - y| / (x + y) (0 for x = y = 0), with P^, tau^ the statistics
 * of rt_cir_stats for H and alpha = alpha_state_dev[0] (1 if NULL; no gradient).
 *   loss_dev    one float (overwritten)
 *   grad_H_dev  n_rx x N complex64, dL/dRe H + j dL/dIm H (overwritten); a CIR
 *               with P^ = 0 or tau^ = 0 passes no gradient through its delay term
 *   P_pred_dev, tau_pred_dev  per-receiver P^ and tau^ (may be NULL) */
rt_status rt_delay_spread_power_loss(rt_ctx* ctx, const void* H_dev, int32_t n_rx, int32_t n_sub,
                                     double delta_f_hz, const float* P_meas_dev, const float* tau_meas_dev,
                                     const float* alpha_state_dev, float* loss_dev, void* grad_H_dev,
                                     float* P_pred_dev, float* tau_pred_dev);
/* Evaluation metrics per receiver (Sec. IV-C): ALE = |10 log10(alpha P_meas) -
 * 10 log10 P_pred| [dB] and RAE = |tau_meas - tau_pred| / tau_meas; alpha from
 * alpha_state_dev[0] (1 if NULL).  Either output may be NULL. */
rt_status rt_cir_metrics(rt_ctx* ctx, const float* P_meas_dev, const float* tau_meas_dev,
                         const float* P_pred_dev, const float* tau_pred_dev, int32_t n,
                         const float* alpha_state_dev, float* ale_dev, float* rae_dev);

/* ------------------------------------------------------------------ neural materials */

/* Neural materials, Sec. III-D: an MLP evaluated at every triangle's centroid c.
 * The centroid is normalised to the unit cube, p = (c - b) / Delta_b with b the
 * centre and Delta_b the longest edge of the scene's bounding box, and encoded
 * as [p, sin(2^k pi p), cos(2^k pi p) for k = 1..6] (Eq. pos_encoding; per k the
 * three sines then the three cosines; 39 features, padded with one zero to 40);
 * then 40 -> 128 -> 128 -> 128 -> 2 with ReLU on the hidden layers, and
 * sigma = exp(o_1), eps_r = 1 + exp(o_2) (Eq. trainable_materials_1/2).
 * Weights are BF16, row major [in][out], packed W1 (40 x 128, row 39 unused),
 * W2, W3 (128 x 128), W4 (128 x 2): 38144 values, 16-byte aligned.  Biases are
 * float32 packed b1, b2, b3 (128 each), b4 (2): 386 values.  Every layer input is
 * rounded to BF16, products are summed in FP32.
 *   eps_r_dev, sigma_dev  n_tris float32 outputs (indexed by triangle)
 *   act_dev   n_tris x 424 BF16: the inputs of layers 1..4 saved for the
 *             backward pass (may be NULL if no backward pass follows). */
rt_status rt_mlp_forward(rt_ctx* ctx, const rt_scene* scene, const uint16_t* weights_bf16_dev,
                         const float* bias_dev, float* eps_r_dev, float* sigma_dev, uint16_t* act_dev);
/* Adjoint of rt_mlp_forward given dL/deps_r and dL/dsigma per triangle (e.g. from
 * rt_eval_fields_backward with per_triangle = 1): ACCUMULATES (+=) dL/dW into
 * grad_weights_dev (38144 float32, same packing as the weights) and dL/db into
 * grad_bias_dev (386 float32).  dz_work_dev: n_tris x 384 float32 scratch owned
 * by the caller (overwritten).  act_dev, eps_r_dev, sigma_dev come from the
 * forward call with the same weights. */
rt_status rt_mlp_backward(rt_ctx* ctx, const rt_scene* scene, const uint16_t* weights_bf16_dev,
                          const uint16_t* act_dev, const float* eps_r_dev, const float* sigma_dev,
                          const float* grad_eps_r_dev, const float* grad_sigma_dev, float* dz_work_dev,
                          float* grad_weights_dev, float* grad_bias_dev);

/* The loss, its gradient and H of rt_cfr_power_mse_fused (same inputs, outputs
 * and errors), for callers that cannot allocate device memory during the call
 * (for example a loop that reserved its whole memory budget in advance, or a host
 * program whose own memory manager forbids other code from calling the CUDA
 * allocator).  The paper has no counterpart: this is a property of the library,
 * not of the method.
 *   - A receiver of more than 4096 paths is summed exactly, by one CTA, where
 *     rt_cfr_power_mse_fused splits it over CTAs and uses the non-uniform FFT of
 *     its approximation (at most ~4e-7 of sum |a_i| per entry of H).  Results for
 *     such receivers therefore differ from the regular call within that error,
 *     and they take longer (the whole P x N sum on one CTA).  Other receivers get
 *     the same arithmetic as the regular call.
 *   - Allocates nothing: its working memory is one fixed array inside the
 *     library (512 KiB + 256 B) that every GPU loading the library keeps until
 *     the process exits.
 *   - n_rx must be <= 65536; larger values return RT_ERR_INVALID_ARG with a
 *     message, nothing launched.
 *   - The first call on a device looks up that array's device address; make the
 *     first call on each device before any stream capture (a first call inside a
 *     capture returns RT_ERR_INVALID_ARG).  Later calls outside a capture look
 *     it up again.
 *   - All calls share the array: sequential calls are independent (the call
 *     resets what must start at zero), but calls that overlap on the GPU, e.g. on
 *     two streams at once, race on it. */
rt_status rt_cfr_power_mse_fused_noalloc(rt_ctx* ctx, const int64_t* rx_offsets_dev, int32_t n_rx,
                                         const void* a_dev, const double* tau_dev, double f_center_hz,
                                         double delta_f_hz, int32_t n_sub, const float* target_power_dev,
                                         const float* rx_weight_dev, float* loss_dev, void* grad_a_dev,
                                         void* H_dev);

#ifdef __cplusplus
}
#endif

#endif /* RT103_H */

/*
 * bp.h - C ABI of libbp: voxel-driven circular cone-beam back-projection
 * (FDK) on one GB300 GPU (sm_103a).
 *
 * Method: Chen et al., "Performance Portable Back-projection Algorithms on
 * CPUs", ICS '21. Back-projection follows Listing 1 (Section 2.1.2) with the
 * bilinear sampling of Listing 2; the z-invariance of u and w used by every
 * kernel here is the hoisting of Section 3.1.2 / Algorithm 1; projections
 * are staged per view batch like Algorithm 2. The projection matrix is the
 * 3x4 pinhole matrix of Section 2.1.1.
 *
 * Conventions shared by every call
 *   - Array layouts are C row-major. Projections: [batch][np][nv][nu]
 *     (u, the detector column, fastest; nu = the paper's nw, nv = nh).
 *     Volumes: [batch][nz][ny][nx] (x fastest).
 *   - Pointers named "device" must point to CUDA device memory of the
 *     current device, 16-byte aligned; the caller owns them. Host pointers
 *     are only read during the call.
 *   - Calls that take a stream are asynchronous on that stream (NULL means
 *     the legacy default stream). They never allocate and never synchronise;
 *     all device memory the context needs is allocated by bp_create*.
 *   - Every call returns a bp_status; on failure it also stores a message
 *     retrievable with bp_last_error. No call aborts, traps or throws.
 *     Errors raised inside a kernel (a bounded wait that ran out, a staged
 *     tile that would not fit) are recorded in a device word and reported
 *     by bp_device_status.
 *   - Threading: one context may be used from one host thread at a time.
 */
#ifndef BP_H
#define BP_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BP_OK = 0,
    BP_ERR_INVALID_ARG = 1,   /* bad size, pointer, alignment or geometry  */
    BP_ERR_UNSUPPORTED = 2,   /* valid request this context cannot serve   */
    BP_ERR_OOM = 3,           /* device or host allocation failed          */
    BP_ERR_CUDA = 4,          /* a CUDA runtime/driver call failed         */
    BP_ERR_TIMEOUT = 5,       /* a kernel's bounded wait ran out           */
    BP_ERR_DEVICE = 6         /* a kernel recorded another internal error  */
} bp_status;

typedef enum { BP_F32 = 0, BP_F16 = 1 } bp_dtype;

/*
 * Circular cone-beam geometry (Section 2.1.1: source-to-axis distance d,
 * source-to-detector distance D, detector nw x nh, volume nx x ny x nz).
 * Lengths in mm, angles in radians, all FP64.
 *   source at sid*(cos t, sin t, 0); flat detector normal to that direction
 *   at distance sdd from the source; detector u axis (-sin t, cos t, 0),
 *   v axis = z; pixel (r, c) centre at ((c-cu)*du, (r-cv)*dv) with
 *   cu = (nu-1)/2 + u_off_px, cv = (nv-1)/2 + v_off_px;
 *   voxel (i, j, k) centre at ((i-(nx-1)/2)*sx + ox, (j-(ny-1)/2)*sy + oy,
 *   (k-(nz-1)/2)*sz + oz).
 * angles may be NULL, meaning 2*pi*s/n_views for s = 0..n_views-1.
 * Requirements: 0 < sid < sdd; all sizes >= 1; pitches and spacings > 0;
 * every voxel strictly in front of the source in every view.
 */
typedef struct {
    double sid, sdd;
    int n_views;
    const double *angles;          /* host, n_views entries, copied; may be NULL */
    int nu, nv;
    double du, dv, u_off_px, v_off_px;
    int nx, ny, nz;
    double sx, sy, sz, ox, oy, oz;
} bp_geometry;

typedef struct bp_ctx bp_ctx;      /* opaque; owned by the library */

/*
 * Create a context from a circular geometry: builds the FP64 projection
 * matrices (Section 2.1.1; explicit form above), the ramp-filter spectrum
 * and the launch plan, and allocates all device memory the calls need on
 * the current device. *out is set only on BP_OK.
 */
bp_status bp_create(const bp_geometry *g, bp_ctx **out);

/*
 * Create a context from explicit projection matrices P (host, FP64,
 * [n_views][3][4], acting on (i, j, k, 1); row 2 is the depth w, rows 0 and
 * 1 give u*w and v*w in pixels). When every view has P[0][2] = P[2][2] = 0
 * (u and w independent of k, Section 3.1.2) the z-column kernels run;
 * otherwise a per-voxel kernel does. bp_filter is unavailable
 * (BP_ERR_UNSUPPORTED) because the filter needs the physical geometry.
 */
bp_status bp_create_from_matrices(const double *P, int n_views, int nu, int nv,
                                  int nx, int ny, int nz, bp_ctx **out);

/*
 * FDK pre-filtering (Section 2.1.2 assumes filtered projections; the
 * formula is: cosine weight sdd/sqrt(sdd^2+u^2+v^2), then a linear
 * convolution along u with the discrete Ram-Lak kernel on the isocenter
 * pitch dp = du*sid/sdd, h[0] = 1/(4 dp^2), h[odd n] = -1/(pi^2 n^2 dp^2),
 * h[even n != 0] = 0, times dp).
 *   proj  device, FP32 [batch][np][nv][nu]
 *   out   device, [batch][np][nv][nu] of out_t (FP32, or FP16 rounded to
 *         nearest even); may not alias proj when out_t is BP_F16.
 */
bp_status bp_filter(bp_ctx *ctx, const float *proj, void *out, bp_dtype out_t,
                    int batch, void *stream);

/*
 * As bp_filter, for a block of n_views consecutive views of one scan
 * ([batch][n_views][nv][nu], contiguous). The filter acts on each detector
 * row on its own, so which views the block holds does not matter.
 */
bp_status bp_filter_views(bp_ctx *ctx, const float *proj, void *out, bp_dtype out_t,
                          int n_views, int batch, void *stream);

/*
 * Back-projection (Listing 1): for every voxel and view s,
 *   vol += scale * bilinear(proj_s, u, v) / w^2
 * with (u*w, v*w, w) = P_s (i, j, k, 1), floor-based bilinear sampling and
 * zero outside the detector. FP32 arithmetic and accumulation; each voxel
 * is written once per call.
 *   proj        device, [batch][np][nv][nu] of type t (FP32 or FP16)
 *   vol         device, FP32 [batch][nz][ny][nx]
 *   scale       pi/np for FDK, 1 for the plain adjoint of fp_project
 *   accumulate  0: vol = result; 1: vol += result
 */
bp_status bp_backproject(bp_ctx *ctx, const void *proj, bp_dtype t, float *vol,
                         int batch, float scale, int accumulate, void *stream);

/*
 * As bp_backproject, over views view0 .. view0+n_views-1 only. proj points
 * at the first of those views: [batch][n_views][nv][nu] with batch stride
 * proj_batch_stride elements (0 means n_views*nv*nu). Used to overlap the
 * host-to-device copy of later views with the back-projection of earlier
 * ones (call with accumulate = 1 after the first chunk).
 */
bp_status bp_backproject_views(bp_ctx *ctx, const void *proj, bp_dtype t, int view0,
                               int n_views, long long proj_batch_stride, float *vol,
                               int batch, float scale, int accumulate, void *stream);

/*
 * As bp_backproject_views, for the slices z0 .. z0+nz_slab-1 only; every
 * other voxel of vol is left as it is. With mirror != 0 the call also
 * computes the mirrored slices nz-z0-nz_slab .. nz-1-z0 (the middle slice
 * of an odd nz once), in one pass of the mid-plane symmetric kernel
 * (Section 3.1.2, Algorithm 1) where the geometry has the symmetry and the
 * projections are FP32; this needs z0 + nz_slab <= (nz + 1) / 2. vol still
 * points at the whole [batch][nz][ny][nx] volume. A volume computed slab by
 * slab (the same views each time) equals the one-call result to FP32
 * rounding, and bit for bit when nz, z0 and nz_slab are multiples of 64
 * (the slabs then cut along the kernels' z-tiles).
 * Used to copy finished slabs back to the host while later ones are
 * computed, and the unit a z-slab split over GPUs would give each GPU.
 * Errors: BP_ERR_INVALID_ARG for a slice range outside the volume or a
 * mirrored slab reaching past the lower half; otherwise those of
 * bp_backproject_views.
 */
bp_status bp_backproject_slab(bp_ctx *ctx, const void *proj, bp_dtype t, int view0, int n_views,
                              long long proj_batch_stride, int z0, int nz_slab, int mirror,
                              float *vol, int batch, float scale, int accumulate, void *stream);

/*
 * Matched forward projector: the exact transpose of bp_backproject with the
 * same scale (same taps, same bilinear weights, same 1/w^2), so that
 * <bp_backproject(q), x> = <q, fp_project(x)> up to FP32 rounding.
 *   vol   device, FP32 [batch][nz][ny][nx]
 *   proj  device, FP32 [batch][np][nv][nu]; overwritten
 */
bp_status fp_project(bp_ctx *ctx, const float *vol, float *proj, int batch,
                     float scale, void *stream);

/*
 * Analytic line integrals of an ellipsoid phantom (input data for tests,
 * benchmarks and training; not part of the method). ell: host, FP64
 * [n_ell][16] rows of cx, cy, cz, ax, ay, az, R (3x3 body->world,
 * row-major), rho; overlapping ellipsoids add. proj: device FP32
 * [np][nv][nu], overwritten. Needs a context made by bp_create.
 * At most 256 ellipsoids. Unlike the method's calls, this one synchronises
 * the stream once (after uploading the per-view coefficients it derives
 * from ell in FP64) and uses a coefficient buffer of the context, so two
 * calls on one context must not run concurrently on different streams.
 */
bp_status bp_phantom_project(bp_ctx *ctx, const double *ell, int n_ell, float *proj,
                             void *stream);

/* Copy the FP64 projection matrices ([np][3][4]) to host memory P_out. */
bp_status bp_get_matrices(const bp_ctx *ctx, double *P_out);

/* Sizes of the context: any pointer may be NULL. */
bp_status bp_get_dims(const bp_ctx *ctx, int *n_views, int *nu, int *nv,
                      int *nx, int *ny, int *nz);

/*
 * Synchronise the stream, then read and clear the context's device error
 * word: BP_OK, BP_ERR_TIMEOUT or BP_ERR_DEVICE (message in bp_last_error).
 */
bp_status bp_device_status(bp_ctx *ctx, void *stream);

/*
 * Tuning and testing (no counterpart in the paper).
 *   bp_set_tuning      voxels per thread along z in the z-column kernels
 *                      (32 or 64) and, for 32, the CTAs per SM the kernel's
 *                      register budget targets (2 or 3); re-derives the
 *                      staged box sizes.
 *   bp_set_pipeline_depth
 *                      views the staging producer of the back-projector keeps
 *                      in flight (1..8, default 4; BP_ERR_INVALID_ARG when the
 *                      boxes of that many views exceed shared memory). When
 *                      the default does not fit, the plan lowers it (to 2 at
 *                      least) before falling back to direct global loads. The
 *                      GPU counterpart of the paper's view batching and
 *                      prefetching depth (Section 3.1.3, Algorithm 2).
 *   bp_set_symmetry    FP32 back-projection with the mid-plane symmetry of
 *                      Section 3.1.2 / Algorithm 1: a thread owns voxels k
 *                      and nz-1-k and computes v, its floor and fraction
 *                      once for both. 1 (default): used whenever
 *                      v(nz-1-k) = nv-1-v(k) holds for the context's matrices
 *                      (v_off = 0, volume centred on the central plane) and
 *                      the boxes fit shared memory; asking for it explicitly
 *                      on other matrices returns BP_ERR_UNSUPPORTED (and
 *                      leaves it off). 0: always the plain z-column kernel.
 *   bp_set_timeout     limit of every bounded wait inside the kernels
 *                      (seconds, (0, 60]; default 2).
 *   bp_test_drop_view  test hook: the staging producer skips the load of
 *                      this view (-1 = off), so the consumers' bounded wait
 *                      runs out and bp_device_status reports BP_ERR_TIMEOUT.
 *   bp_test_live_allocations  test hook: device allocations held by all
 *                      live contexts of this process. With the environment
 *                      variable BP_TEST_FAIL_ALLOC=n set, the n-th device
 *                      allocation of every bp_create* fails as an
 *                      out-of-memory cudaMalloc would (BP_ERR_OOM, message in
 *                      bp_last_error(NULL)); the count shows that the
 *                      allocations made before it were released.
 *   bp_get_plan        the launch plan: voxels per thread along z, the
 *                      staged box (FP32 width, FP16 width, rows; a width of
 *                      -1 means that element type uses direct global loads),
 *                      the pipeline depth in use and whether FP32 calls use
 *                      the mid-plane symmetry. Any pointer may be NULL.
 */
bp_status bp_set_tuning(bp_ctx *ctx, int tk, int ctas_per_sm);
bp_status bp_set_pipeline_depth(bp_ctx *ctx, int stages);
bp_status bp_set_symmetry(bp_ctx *ctx, int enable);
bp_status bp_set_timeout(bp_ctx *ctx, double seconds);
bp_status bp_test_drop_view(bp_ctx *ctx, int view);
int bp_test_live_allocations(void);
bp_status bp_get_plan(const bp_ctx *ctx, int *tk, int *bu32, int *bu16, int *bv, int *stages,
                      int *symmetric);

/* Message of the last failed call on ctx (never NULL; "" after success).
 * With ctx == NULL: the last failure of bp_create* in this thread. */
const char *bp_last_error(const bp_ctx *ctx);

/* Release the context and its device memory. NULL-safe. */
void bp_destroy(bp_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* BP_H */

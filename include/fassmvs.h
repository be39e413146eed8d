/*
 * fassmvs.h -- C ABI of the B300 (sm_103a) implementation of the FaSS-MVS hot
 * path: plane-sweep census cost volume, surface-aware semi-global matching,
 * winner-takes-all with sub-plane refinement, normal and confidence maps,
 * coarse-to-fine over an image pyramid (Ruf, Weinmann, Hinz, arXiv 2112.00821).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All image, map and volume pointers are DEVICE pointers on the device the
 *    context was created for; the caller owns them.  Camera and plane
 *    parameters are HOST values (copied during the call).
 *  - Layouts are row-major and unpadded unless a pitch or slot stride is given:
 *      image  uint8  [H][W]            census uint64 [H][W]
 *      volume uint16 [H][W][Ds]        slot s of pixel p holds plane lo_p + s,
 *                                      s < D; Ds >= D is the slot stride
 *      lo     int32  [H][W]            first plane of the window of each pixel
 *                                      (NULL: lo_p = 0 everywhere)
 *      dI     int8   [8][H][W]         per-path index jumps (surface-normal SGM)
 *      depth  float  [H][W]            normal float [H][W][3]  conf float [H][W]
 *  - Cameras: K is the 3x3 intrinsic matrix (row-major); neighbour k maps a
 *    point X of the reference camera frame to its own frame as
 *    X_k = R_k X + t_k (R_k row-major 3x3, t_k 3-vector), the relative pose of
 *    Sec. 2.1 / Eq. homography.  side[k] = -1 for a view left of the
 *    reference (k < ref), +1 for a view right of it.
 *  - Planes: n^T X + delta = 0 in the reference frame; the finest list is
 *    uniform in inverse distance, 1/delta_g = rho_far + g * drho, g = 0 the
 *    farthest (Sec. 2.2.3).  Level l uses every 2^l-th plane.
 *  - Path order of the aggregation (and of dI): r = (1,0) (-1,0) (0,1) (0,-1)
 *    (1,1) (-1,-1) (1,-1) (-1,1); the predecessor of p on path r is p - r;
 *    4-path aggregation uses the first four.
 *  - Every call is asynchronous on `stream` (a cudaStream_t, NULL = legacy
 *    default stream).  The returned status covers argument validation and
 *    launch errors; device-side failures surface at fassmvs_sync.  Nothing
 *    throws or aborts across this boundary.  A context is not thread-safe;
 *    use one context per host thread.
 */
#ifndef FASSMVS_H
#define FASSMVS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FASSMVS_API __attribute__((visibility("default")))
#else
#define FASSMVS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fassmvs_ctx fassmvs_ctx; /* opaque, owned by the library */

typedef enum {
    FASSMVS_OK = 0,
    FASSMVS_EINVAL = 1,    /* bad argument: sizes, pointers, limits */
    FASSMVS_ENOMEM = 2,    /* scratch would exceed the context memory budget */
    FASSMVS_EBUSY = 3,     /* no room for the request right now (serving) */
    FASSMVS_ETIMEOUT = 4,  /* a bounded device wait gave up */
    FASSMVS_ECUDA = 5,     /* a CUDA runtime call failed */
    FASSMVS_EINTERNAL = 6, /* a kernel reported an inconsistency */
    FASSMVS_ECANCELED = 7  /* a queued request was withdrawn (serving) */
} fassmvs_status;

/* Sweep planes (Sec. 2.2): normal n (unit, reference frame) and the inverse
 * distances of the finest list. */
typedef struct {
    double n[3];
    double rho_far;  /* 1/delta of plane 0, the farthest */
    double drho;     /* inverse-distance step of the finest list */
    int32_t G0;      /* number of planes of the finest list */
} fassmvs_planes;

/* Estimation settings (Sec. 2.1-2.5 and Sec. 3.2-3.5). */
typedef struct {
    int32_t levels;        /* pyramid levels n, 1..8 (Sec. 2.1) */
    int32_t D[8];          /* plane window per level below the top; the top
                              level sweeps its whole list (<= 256 planes) */
    int32_t paths;         /* 8 or 4 aggregation paths (Sec. 3.5) */
    int32_t variant;       /* 0 plane-wise, 1 surface normal, 2 path gradient
                              (Eq. sgm-smooth-fp / -sn / -pg) */
    int32_t p1;            /* phi1 for one image per subset; multiplied by
                              n_max = max(n_left, n_right) (Sec. 2.3.3) */
    int32_t p2;            /* phi2 (x n_max) when adaptive_p2 == 0 */
    int32_t adaptive_p2;   /* 1: phi2 = phi1 (1 + alpha exp(-dI / beta)) */
    float alpha, beta;     /* Eq. p2-grad, 8 and 10 in the paper */
    int32_t median5;       /* 5x5 median on the refined depth (Sec. 2.1) */
    int32_t normal_radius; /* smoothing window radius; sigma = radius (Sec. 2.4) */
    float normal_beta;     /* beta of Eq. normal-smooth, 10 in the paper */
    float rho_deg;         /* critical angle of Eq. weight-normal, 60 */
    int32_t dmax;          /* clamp of the sn / pg index jumps */
    int32_t cost;          /* matching cost (Sec. 2.2.1): 0 census 9x7 Hamming (at most 62 per
                              view), 1 NCC 5x5, negated, truncated at zero correlation and
                              scaled to 255 (the paper's phi1 for it is 100) */
} fassmvs_config;

/* SGM parameters of one aggregation (Eq. xsgm ... Eq. p2-grad). */
typedef struct {
    int32_t paths;         /* 8 or 4 */
    int32_t variant;       /* 0, 1, 2 as above */
    int32_t p1;            /* phi1, already multiplied by n_max */
    int32_t p2;            /* phi2, already multiplied, used when p2_lut == NULL */
    int32_t dmax;          /* clamp of the index jumps */
    const uint16_t* p2_lut;/* HOST table of 256 phi2 values indexed by |I(p) -
                              I(p-r)|, or NULL for the fixed p2 */
} fassmvs_sgm_params;

/* Fills the paper's defaults: 1 level, D = 256, 8 paths, plane-wise,
 * p1 = 24 (census 9x7, Sec. 3.4), adaptive phi2 with alpha = 8, beta = 10,
 * median on, radius 2, beta 10, rho 60 deg, dmax 8. */
FASSMVS_API fassmvs_status fassmvs_config_default(fassmvs_config* cfg);

/* Creates a context on `device`.  Scratch (pyramids, census, cost and
 * aggregated volumes, per-level maps) is allocated lazily and kept; its total
 * never exceeds mem_budget bytes (0 = no limit), else FASSMVS_ENOMEM. */
FASSMVS_API fassmvs_status fassmvs_create(const fassmvs_config* cfg, int device, size_t mem_budget,
                              fassmvs_ctx** out);
FASSMVS_API void fassmvs_destroy(fassmvs_ctx* ctx);

/* Replaces the configuration (same validation as fassmvs_create). */
FASSMVS_API fassmvs_status fassmvs_set_config(fassmvs_ctx* ctx, const fassmvs_config* cfg);

/* Stores the calibration of the next estimates (host arrays, copied):
 * K 3x3, R n_nb x 3 x 3, t n_nb x 3, side n_nb (Sec. 2.1). */
FASSMVS_API fassmvs_status fassmvs_set_cameras(fassmvs_ctx* ctx, const double K[9], int n_nb,
                                   const double* R, const double* t, const int8_t* side);

/* Full hierarchical estimate of one reference frame (Sec. 2.1, Fig. overview):
 * ref and nbrs[k] are W x H uint8 images with row pitch `pitch` bytes
 * (nbrs is a HOST array of n_nb device pointers, n_nb equal to the count
 * given to fassmvs_set_cameras); depth (W*H floats), normal (W*H*3) and conf
 * (W*H) receive the level-0 maps.  Depth is the z distance in the reference
 * frame; normals face the camera; confidence is in [0, 1]. */
FASSMVS_API fassmvs_status fassmvs_estimate(fassmvs_ctx* ctx, const uint8_t* ref, int W, int H, int pitch,
                                const uint8_t* const* nbrs, int n_nb, const fassmvs_planes* planes,
                                float* depth, float* normal, float* conf, void* stream);

/* The same estimate from HOST images to HOST maps: ref and nbrs[k] (a HOST
 * array of n_nb HOST pointers) are W x H uint8 images in host memory with row
 * pitch `pitch` bytes (>= W); depth (W*H floats), normal (W*H*3) and conf
 * (W*H) are host buffers.  The call copies the images into one of two device
 * slots that the context owns (rows padded to 16 bytes, so that the cost
 * kernel can stage them; allocated on the first call of a size, within the
 * context budget: FASSMVS_ENOMEM beyond it) on a copy stream, runs
 * fassmvs_estimate on `stream` and copies the maps back on a second copy
 * stream; it returns once the maps are in the host buffers.  Page-locked
 * host memory makes the copies DMA transfers; pageable memory works and is
 * staged by the driver.  Results equal those of fassmvs_estimate on device
 * copies of the same images, bit for bit. */
FASSMVS_API fassmvs_status fassmvs_estimate_host(fassmvs_ctx* ctx, const uint8_t* ref, int W, int H, int pitch,
                                                 const uint8_t* const* nbrs, int n_nb,
                                                 const fassmvs_planes* planes, float* depth, float* normal,
                                                 float* conf, void* stream);

/* The same call for a sequence of frames: it returns once the images have
 * been copied to the device (the host image buffers may then be reused), with
 * the estimate and the copy of the maps still running, so that one frame's
 * copies overlap the kernels of the frames next to it (two slots: a call
 * waits, on the device, for the slot's use two calls before).  The maps of a
 * call are in its host buffers, which must stay valid until then, once
 * fassmvs_sync or a later fassmvs_estimate_host returns.  A call whose image
 * size differs from the previous call's first waits for every earlier call. */
FASSMVS_API fassmvs_status fassmvs_estimate_host_async(fassmvs_ctx* ctx, const uint8_t* ref, int W, int H,
                                                       int pitch, const uint8_t* const* nbrs, int n_nb,
                                                       const fassmvs_planes* planes, float* depth, float* normal,
                                                       float* conf, void* stream);

/* ---- batched form ------------------------------------------------------- */

/* One reference frame of a batch (all pointers as for fassmvs_estimate; the
 * camera and plane parameters are HOST arrays read during the call). */
typedef struct {
    const uint8_t* ref;           /* device, W x H, row pitch `pitch` */
    const uint8_t* const* nbrs;   /* HOST array of n_nb device pointers, same layout */
    int32_t W, H, pitch, n_nb;
    const double* K;              /* 3x3 */
    const double* R;              /* n_nb x 3 x 3, reference -> neighbour */
    const double* t;              /* n_nb x 3 */
    const int8_t* side;           /* n_nb: -1 left, +1 right */
    fassmvs_planes planes;
    float* depth;                 /* device W*H */
    float* normal;                /* device W*H*3 */
    float* conf;                  /* device W*H */
} fassmvs_frame;

/* Estimates n (1..64) frames of mixed size, view count and plane count with
 * the context's configuration (Sec. 2.1 applied to every frame).  Per level
 * the frames share launches: the cost volumes of all frames come from one
 * persistent kernel pulling (frame, tile, plane chunk) work items from an
 * atomic counter, and the aggregation runs several directions of all frames
 * per launch, each into its own partial sum (see fassmvs_tuning), which the
 * winner-take-all step adds.  Results equal those of n separate
 * fassmvs_estimate calls, bit for bit, for every tuning.  Scratch for every
 * frame of the batch is held at once: per frame and level about
 * W*H*Ds*2*(1 + parts) bytes for the cost volume and the partial sums (Ds =
 * window planes rounded up to 8), within the context budget (FASSMVS_ENOMEM
 * beyond it).  The per-call argument blocks go through two pinned staging
 * halves; a call waits until the call two before it has finished on the
 * device.  Calls on one context must be ordered (one stream, or synchronised
 * between streams): frames of concurrent calls would share scratch.
 * With graphs enabled (fassmvs_set_graph) and a non-default stream, a batch
 * whose shapes were seen before is captured and launched as one CUDA graph,
 * the executable graph of that shape being updated in place each call; the
 * first call of a shape runs eagerly and allocates. */
FASSMVS_API fassmvs_status fassmvs_estimate_batch(fassmvs_ctx* ctx, const fassmvs_frame* frames, int n,
                                                  void* stream);
FASSMVS_API fassmvs_status fassmvs_set_graph(fassmvs_ctx* ctx, int on);

/* Work decomposition of the batched form; no setting changes any result.
 *   chunk_planes  planes per work item of the persistent cost kernel, 1..256,
 *                 or 0: automatic, at least about three waves of items
 *                 (chunks >= 8 planes), the count up to twice that whose
 *                 items fill their last wave best
 *   ctas_per_sm   persistent cost CTAs per SM, 1 or 2, or 0: one short-lived
 *                 CTA per work item (lets stream priorities act per CTA)
 *   sgm_parts     the form of the aggregation.  1, 2, 4 or 8 (at most the
 *                 path count): one launch per group of directions over path
 *                 lines, with that many partial sums (P directions run
 *                 concurrently in each of paths/P launches), then the
 *                 winner-takes-all; 0 (default): one partial sum per path.
 *                 -1: the two-pass wavefront form -- pass A runs the paths
 *                 from the left and from above, top row first, and stores
 *                 their sum; pass B runs the other paths from the bottom
 *                 right, adds that sum and takes the winner, the parabola
 *                 and the depth in place (8 bytes of DRAM traffic per voxel,
 *                 no aggregate stored, no separate winner-takes-all);
 *                 it needs cooperative launches, without them -1 means 0.
 *                 Every form gives the same bits.
 *   no_staging    0: the cost kernel stages the view images in shared memory
 *                 by TMA where their rows are 16-byte aligned (default);
 *                 1: it reads them from global memory. */
typedef struct {
    int32_t chunk_planes, ctas_per_sm, sgm_parts, no_staging;
} fassmvs_tuning;

/* fassmvs_autotune times a set of candidate tunings on the given batch
 * (running it once per candidate, outputs written each time) and keeps the
 * fastest for later batches of the same shapes; the choice is returned in
 * *chosen (may be NULL) and appended as one JSON line to the file named by the
 * FASSMVS_TUNE_FILE environment variable, when set.  fassmvs_set_tuning sets
 * the context default and forgets earlier choices. */
FASSMVS_API fassmvs_status fassmvs_set_tuning(fassmvs_ctx* ctx, const fassmvs_tuning* tuning);
FASSMVS_API fassmvs_status fassmvs_autotune(fassmvs_ctx* ctx, const fassmvs_frame* frames, int n,
                                            void* stream, fassmvs_tuning* chosen);

/* ---- serving form -------------------------------------------------------- */

/* A server keeps the frames of a video stream resident on the device, each
 * with its image pyramid built once on arrival, and runs keyframe requests
 * (reference frame + neighbour frames + plane list) through the same
 * coarse-to-fine estimate as fassmvs_estimate_batch.  Device memory for the
 * resident frames and for every admitted request's scratch comes from one
 * reservation of mem_budget bytes made at creation; a request is admitted, in
 * submission order, once its scratch fits next to what is in use.  A worker
 * thread batches admitted requests continuously: an idle lane (a stream with
 * its own context) takes up to max_batch admitted requests at once; under a
 * backlog (overlap_queue) it does so while batches on other lanes are still
 * running, so their work overlaps on the device, the older batch on a stream
 * of higher priority.  A request's results are independent of what it was batched
 * with.  The paper has no serving form (its estimates run one keyframe at a
 * time); this is the deployment shape of the same computation. */
typedef struct fassmvs_server fassmvs_server;

typedef struct {
    int32_t lanes;            /* batches in flight at once, 1..4 */
    int32_t max_batch;        /* requests per batch, 1..32 */
    size_t mem_budget;        /* device bytes reserved for frames + request scratch */
    int32_t deadline_ms;      /* a request not admitted within this fails with ETIMEOUT; 0: no limit */
    int32_t overlap_queue;    /* a batch starts next to running ones only while at least this many
                                 admitted requests wait (0 or 1: whenever a lane is idle) */
    fassmvs_tuning tuning;    /* work decomposition of a batch that starts alone */
    fassmvs_tuning tuning_overlap;   /* ... of one that starts next to running batches (same
                                        sgm_parts; ctas_per_sm 0 keeps the older batch first) */
} fassmvs_server_config;

typedef struct {
    int64_t id;               /* caller's tag, returned in the result */
    int64_t ref;              /* reference frame id */
    const int64_t* nbrs;      /* HOST array of n_nb neighbour frame ids (copied) */
    int32_t n_nb;             /* 1..16; a neighbour with a smaller id is a left view */
    fassmvs_planes planes;
    float* depth;             /* W*H, W*H*3, W*H outputs of the reference size: */
    float* normal;            /* pinned host memory when host_outputs (copied */
    float* conf;              /* back by the server), else device memory */
    int32_t host_outputs;
    /* post-filters of Sec. 2.6, run on the device before the outputs are
     * returned (0: none); FASSMVS_POST_* flags: */
    int32_t postfilter;
    int32_t geo_n;            /* FASSMVS_POST_GEO: 1..4 earlier requests ... */
    int64_t geo_ids[4];       /* ... whose estimated depth maps were kept */
    double geo_eta_r;         /* reprojection threshold in pixels (Alg. 4) */
    int32_t geo_eta_h;        /* minimum number of consistent maps (Alg. 4) */
} fassmvs_request;

/* DoG texture mask (Alg. 3) of the reference image applied to the outputs */
#define FASSMVS_POST_DOG 1
/* geometric consistency (Alg. 4) against the kept depth maps geo_ids (same
 * size and intrinsics; their reference poses give the relative poses) */
#define FASSMVS_POST_GEO 2
/* keep this request's estimated depth map (before any post-filter) on the
 * device, inside the memory budget, for later requests' consistency checks,
 * until fassmvs_server_release_depth */
#define FASSMVS_POST_KEEP 4

typedef struct {
    int64_t id;
    int32_t status;           /* FASSMVS_OK, FASSMVS_ETIMEOUT (not admitted in time), FASSMVS_ENOMEM
                                 (cannot fit even with nothing else in flight), FASSMVS_ECUDA ... */
    int32_t batch_size;       /* requests in the batch it ran in (0: never ran) */
    int64_t t_submit_ns, t_admit_ns, t_launch_ns, t_done_ns;   /* steady clock */
} fassmvs_result;

typedef struct {
    int64_t capacity, bytes_in_use, peak_bytes;
    int64_t frames, resident_frames;
    int64_t submitted, completed, failed, queued;
    int64_t batches, max_batch_seen, overlapped;
} fassmvs_server_stats;

FASSMVS_API void fassmvs_server_config_default(fassmvs_server_config* cfg);
/* Reserves mem_budget device bytes (FASSMVS_ENOMEM when the device cannot)
 * and starts the worker thread. */
FASSMVS_API fassmvs_status fassmvs_server_create(const fassmvs_config* cfg, const fassmvs_server_config* scfg,
                                                 int device, fassmvs_server** out);
/* Finishes every admissible request, then stops the worker and frees all. */
FASSMVS_API void fassmvs_server_destroy(fassmvs_server* srv);
/* Uploads a W x H uint8 frame from HOST memory (row pitch `pitch`) and builds
 * its pyramid on the device; K (3x3) and the world -> camera pose
 * X_cam = R X_world + t are HOST arrays.  FASSMVS_EBUSY when the budget has
 * no room for it now (retry once requests complete). */
FASSMVS_API fassmvs_status fassmvs_server_push_frame(fassmvs_server* srv, int64_t id, const uint8_t* img, int W,
                                                     int H, int pitch, const double K[9], const double R[9],
                                                     const double t[3]);
/* The producer will name the frame in no further request; its memory returns
 * once the requests naming it have completed. */
FASSMVS_API fassmvs_status fassmvs_server_release_frame(fassmvs_server* srv, int64_t id);
/* Queues a request; all its frames must be resident and share the reference's
 * size and intrinsics.  FASSMVS_ENOMEM when its scratch exceeds the whole
 * budget (it could never be admitted). */
FASSMVS_API fassmvs_status fassmvs_server_submit(fassmvs_server* srv, const fassmvs_request* req);
/* Withdraws a request that has not been launched yet (waiting for memory or
 * for a lane): it completes at once with status FASSMVS_ECANCELED and its
 * reserved memory and frame references are given back.  FASSMVS_EBUSY when it
 * is already running (it then completes normally); FASSMVS_EINVAL when no
 * queued or running request has that id. */
FASSMVS_API fassmvs_status fassmvs_server_cancel(fassmvs_server* srv, int64_t id);
/* Gives back the depth map kept for request id (FASSMVS_POST_KEEP) once no
 * queued or running request names it; FASSMVS_EINVAL when none is kept. */
FASSMVS_API fassmvs_status fassmvs_server_release_depth(fassmvs_server* srv, int64_t id);
/* Takes up to max completed results (waiting up to timeout_ms for the first);
 * *n_out receives the count.  Outputs of a completed request are in place. */
FASSMVS_API fassmvs_status fassmvs_server_poll(fassmvs_server* srv, fassmvs_result* out, int max, int* n_out,
                                               int timeout_ms);
FASSMVS_API fassmvs_status fassmvs_server_get_stats(fassmvs_server* srv, fassmvs_server_stats* stats);
FASSMVS_API const char* fassmvs_server_last_error(const fassmvs_server* srv);

/* Test hook for failure detection, no fault involved.  mode 1: the cost
 * kernel plans its staging boxes but issues no copies and bounds its waits at
 * about a millisecond, so every staged wait gives up.  The kernel then reads
 * global memory, so results are unchanged, and the next fassmvs_sync reports
 * FASSMVS_ETIMEOUT.  mode 0: off (default). */
FASSMVS_API fassmvs_status fassmvs_debug_inject(fassmvs_ctx* ctx, int mode);

/* Intermediates of one pyramid level of the next estimates (frame 0 of a
 * batch), for parity tests and debugging.  fassmvs_debug_capture(ctx, level)
 * selects the level (-1: off; while on, estimates run eagerly, never from a
 * CUDA graph).  fassmvs_debug_dump copies one intermediate of the last
 * capture into dst (device or host memory, cap bytes; dst NULL: only *bytes
 * and dims) after waiting for the context's last stream; dims (may be NULL)
 * receives W, H, D, Ds, G of the level.  what (layouts row-major): */
#define FASSMVS_DUMP_COST 0       /* uint16 [H][W][Ds]: cost volume, slot s = plane lo_p + s */
#define FASSMVS_DUMP_WINDOW 1     /* int32 [H][W]: window start lo_p (0 at the top level) */
#define FASSMVS_DUMP_DSN 2        /* int8 [8][H][W]: surface-normal index jumps (0 unless sn) */
#define FASSMVS_DUMP_AGG 3        /* uint16 [H][W][Ds]: aggregated costs, all paths summed */
#define FASSMVS_DUMP_ARGMIN 4     /* int32 [H][W]: winning plane of the winner-takes-all */
#define FASSMVS_DUMP_DEPTH_RAW 5  /* float [H][W]: refined depth before the median */
#define FASSMVS_DUMP_DEPTH 6      /* float [H][W]: depth after the 5x5 median */
#define FASSMVS_DUMP_NORMAL 7     /* float [H][W][3]: smoothed unit normals */
#define FASSMVS_DUMP_WARP 8       /* float [H][W]: warped values minus 128 of the (plane, view)
                                     pair set by fassmvs_debug_capture_warp, as the census reads
                                     them (Alg. 1 patch warping); NaN at pixels whose tile did not
                                     sweep that plane */
FASSMVS_API fassmvs_status fassmvs_debug_capture(fassmvs_ctx* ctx, int level);
/* Which (plane of the level's list, neighbour view) the next captures keep
 * the warped values of (FASSMVS_DUMP_WARP); -1, -1: none. */
FASSMVS_API fassmvs_status fassmvs_debug_capture_warp(fassmvs_ctx* ctx, int plane, int view);
FASSMVS_API fassmvs_status fassmvs_debug_dump(fassmvs_ctx* ctx, int level, int what, void* dst, size_t cap,
                                              size_t* bytes, int32_t dims[5]);

/* ---- plane selection (Sec. 2.2.2, Alg. 2; host-side, no device work) ------- */

/* Distances of the bounding planes n^T X + delta = 0 (n unit, reference
 * frame, P_ref = K [I | 0]) of the reference view frustum cut by the fronto
 * near and far planes at depths d_min < d_max (Eq. of the bounding planes):
 * delta_min is the smallest |n^T X| over the four near corners, delta_max the
 * largest over the four far corners (read so that the sweep encloses the
 * frustum; the equation prints min for both).  Corners: the rays through pixel
 * centres (0,0), (W-1,0), (0,H-1), (W-1,H-1).  All arguments on the HOST.
 * FASSMVS_EINVAL when n is not a unit vector or a corner ray does not meet the
 * planes (n^T r >= 0). */
FASSMVS_API fassmvs_status fassmvs_plane_bounds(const double K[9], int W, int H, const double n[3], double d_min,
                                                double d_max, double* delta_min, double* delta_max);

/* Plane distances by the cross-ratio (Alg. 2) for n_cams matching cameras,
 * X_k = R_k X + t_k (R: n_cams x 9 row-major, t: n_cams x 3; HOST).  p_ref and
 * camera k are the image corner and camera with the longest image segment
 * between the projections of the bounding planes; that segment is walked in
 * whole pixels from the far to the near plane, each step's distance following
 * from the cross-ratio of the rays of camera k through the epipole, the two
 * ends and the step, and the walk ends on delta_min (the last step is at most
 * one pixel).  deltas (HOST, max_planes entries, or NULL to count) receives
 * the list far to near, delta_max first; *count its length; *camera (may be
 * NULL) the index of camera k.  `uniform` (may be NULL) receives the sweep
 * the estimate takes: G0 planes uniform in inverse distance from 1/delta_max
 * to 1/delta_min, whose step is at most the smaller of the one-pixel steps of
 * p_ref at the two ends of its segment (its image moves as a projective
 * function of 1/delta, so no step then moves p_ref by more than a pixel).
 * FASSMVS_EINVAL when a camera centre is not in front of Pi_min
 * (n^T C_i + delta_min <= 0), a corner ray misses the planes, no camera sees
 * a segment, or deltas is given and more than max_planes planes are needed
 * (*count is set). */
FASSMVS_API fassmvs_status fassmvs_cross_ratio_planes(const double K[9], int W, int H, int n_cams, const double* R,
                                                      const double* t, const double n[3], double delta_min,
                                                      double delta_max, int max_planes, double* deltas, int* count,
                                                      int* camera, fassmvs_planes* uniform);

/* ---- post-filters (Sec. 2.6) ---------------------------------------------- */

/* Difference-of-Gaussian texture mask (Alg. 3) of the reference image (W x H
 * uint8, row pitch `pitch`, device): 7x7 Gaussian of sigma 1.4 (integer
 * weights summing to 256 per axis, clamp-to-edge), |I - I_smooth| > 0.5 grey
 * level marks texture, 4-connected marked areas below 7 pixels are dropped,
 * a 3x3 dilation, unmarked areas below 21 pixels are filled.  `mask` (device
 * W*H bytes, may be NULL) receives the mask (1 = enough texture); depth,
 * normal (x3) and conf (device, all or none) are set to 0 where it is 0
 * (read as the algorithm's purpose: its last step names the value 1).  A
 * labelling walk that reaches its bound is reported by fassmvs_sync
 * (FASSMVS_EINTERNAL); it cannot happen on a valid image. */
FASSMVS_API fassmvs_status fassmvs_dog_filter(fassmvs_ctx* ctx, const uint8_t* ref, int W, int H, int pitch,
                                              float* depth, float* normal, float* conf, uint8_t* mask,
                                              void* stream);

/* Geometric consistency by mutual reprojection (Alg. 4): every pixel of the
 * reference depth map (z depth, device, W x H) is lifted with its depth,
 * moved into each of the n (0..16) neighbour depth maps (device pointers in
 * the HOST array `depths`, same size and K; R (n x 9), t (n x 3) HOST arrays,
 * reference -> map k) and projected; the depth of map k at the nearest pixel
 * lifts that point back into the reference, and the reprojection error is
 * the distance to the pixel.  Fewer than eta_h maps within eta_r pixels (the
 * paper: 3 and 10) set depth, normal and conf (normal / conf may be NULL) to
 * 0.  FP64 throughout.  `hits` (device W*H bytes, may be NULL) receives the
 * counts. */
FASSMVS_API fassmvs_status fassmvs_geo_filter(fassmvs_ctx* ctx, float* depth, float* normal, float* conf, int W,
                                              int H, const double K[9], int n, const float* const* depths,
                                              const double* R, const double* t, double eta_r, int eta_h,
                                              uint8_t* hits, void* stream);

/* ---- stages of the hot path (used by the estimate and by parity tests) ---- */

/* Sec. 2.1 pyramid level: 3x3 Gaussian (sigma 1, integer weights 70/116/70
 * per axis) then decimation, out[y][x] = blur(in)(2x, 2y), size
 * ceil(W/2) x ceil(H/2), clamp-to-edge, rounded half up. */
FASSMVS_API fassmvs_status fassmvs_pyramid_down(fassmvs_ctx* ctx, const uint8_t* in, int W, int H,
                                    uint8_t* out, void* stream);

/* Census 9x7 (Sec. 2.2.1 / Sec. 3.4): bit (dy+3)*9 + (dx+4) = [I(q) < I(p)],
 * clamp-to-edge, centre bit 0. */
FASSMVS_API fassmvs_status fassmvs_census(fassmvs_ctx* ctx, const uint8_t* img, int W, int H, uint64_t* out,
                              void* stream);

/* Plane-sweep cost volume of one level (Alg. 1): for every pixel p and slot
 * s < D (plane g = lo_p + s of a list of G planes with 1/delta_g = rho0 +
 * g * drho), the census-Hamming cost of each neighbour warped by the
 * plane-induced homography H = K (R - t n^T / delta) K^-1, summed over the
 * left and the right views, each sum rescaled to max(n_left, n_right) images
 * (round half up), S = min of the two.  A view whose centre sample leaves the
 * image costs 62.  With the context's cost set to NCC the per-view cost is
 * the NCC 5x5 cost instead (255 for an invalid view or a flat window).  A
 * sample is the bilinear value (lerp form) of the neighbour image at the
 * exact warped position, clamped to the image, not rounded; the census
 * decides every comparison as the FP64 values would (comparisons closer than
 * 2^-14 grey levels are decided again in double-float), so the census cost
 * equals the FP64 reading's.  K, R, t, n are host arrays.  Slots D..Ds-1 are
 * left untouched. */
FASSMVS_API fassmvs_status fassmvs_cost_volume(fassmvs_ctx* ctx, const uint8_t* ref, const uint8_t* const* nbrs,
                                   int n_nb, const int8_t* side, int W, int H, const double K[9],
                                   const double* R, const double* t, const double n[3], double rho0,
                                   double drho, int G, const int32_t* lo, int D, int Ds, uint16_t* S,
                                   void* stream);

/* Surface-aware SGM (Sec. 2.3, Eq. xsgm, sgm-smooth-fp/-sn/-pg, sgm-aggr) in
 * the normalised form L_r(p,s) = S(p,s) + min(L'(s'), L'(s'-1) + P1,
 * L'(s'+1) + P1, M + P2) - M, with s' = s + lo_p - lo_{p-r} + di, M = min L',
 * slots outside the predecessor's window = +inf, P2 = max(P2, P1), L = S at
 * the first pixel of a path.  di: 0 (plane-wise), dI[r][p] (surface normal)
 * or g(p-2r) - g(p-r) with g = lo + argmin L_r (path gradient), clamped to
 * +-dmax.  img (uint8 [H][W]) feeds the adaptive phi2 and may be NULL with a
 * fixed p2.  Sbar receives sum_r L_r; FASSMVS_EINVAL if that sum could
 * exceed 16 bits (paths * (max S + max P2) >= 65536 with max S = 62 * 6). */
FASSMVS_API fassmvs_status fassmvs_sgm_aggregate(fassmvs_ctx* ctx, const uint16_t* S, const int32_t* lo,
                                     const int8_t* dI, const uint8_t* img, int W, int H, int D,
                                     int Ds, const fassmvs_sgm_params* prm, uint16_t* Sbar,
                                     void* stream);

/* Eq. sgm-wta + plane depth (Sec. 2.3.2) + refinement (Sec. 2.3.4): argmin
 * (lowest slot on ties), parabola through the winner and its neighbours at
 * their plane distances (none at a window edge), clamped between them;
 * depth = -delta / (n^T K^-1 (x, y, 1)^T).  gwin (optional, int32 [H][W])
 * receives the winning plane index lo + s.  Every window start must satisfy
 * 0 <= lo_p <= G - D (a start outside that range is clamped into the
 * G-entry plane table, and its result is meaningless). */
FASSMVS_API fassmvs_status fassmvs_wta_refine(fassmvs_ctx* ctx, const uint16_t* Sbar, const int32_t* lo, int W,
                                  int H, int D, int Ds, const double K[9], const double n[3],
                                  double rho0, double drho, int G, float* depth, int32_t* gwin,
                                  void* stream);

/* The same winner-takes-all and refinement as fassmvs_wta_refine, for callers
 * that cannot allocate device memory: loops that must not call cudaMalloc
 * once running (it can synchronize the device and its latency is unbounded),
 * and processes whose device memory is already reserved by another allocator,
 * so that cudaMalloc would fail although the caller's buffers are valid.  It
 * takes no context and allocates nothing.  The plane-distance table it needs
 * lives in one static device array of FASSMVS_NOALLOC_MAX_PLANES floats
 * (16 KB, held by every device that loads the library until the process
 * exits); G beyond that limit returns FASSMVS_EINVAL.  Every call looks up
 * the array's device address (cudaGetSymbolAddress, a host-side lookup that
 * allocates nothing) on the current device; the first call on a device can
 * also load the library's device code there, so make that first call before
 * any stream capture.  Window starts must satisfy 0 <= lo_p <= G - D, as for
 * fassmvs_wta_refine.  All calls
 * share the array and it keeps the last call's table: calls that overlap on
 * the GPU (on different streams) race on it.  Runs on the current device.
 * The paper has no counterpart of this entry point. */
#define FASSMVS_NOALLOC_MAX_PLANES 4096
FASSMVS_API fassmvs_status fassmvs_wta_refine_noalloc(const uint16_t* Sbar, const int32_t* lo, int W,
                                                      int H, int D, int Ds, const double K[9],
                                                      const double n[3], double rho0, double drho,
                                                      int G, float* depth, int32_t* gwin,
                                                      void* stream);

/* 5x5 median (Sec. 2.1), clamp-to-edge. */
FASSMVS_API fassmvs_status fassmvs_median5(fassmvs_ctx* ctx, const float* in, int W, int H, float* out,
                               void* stream);

/* Sec. 2.4 normals: n = h x v of back-projected central differences, turned
 * to face the camera, then the appearance-weighted Gaussian of Eq.
 * normal-smooth (window radius r, sigma = r, beta), normalised; (0,0,0) when
 * undefined.  raw (optional) receives the unsmoothed normals.  When conf is
 * not NULL it also receives Eq. weight-normal (Sec. 2.5) for the plane normal
 * n_plane and critical angle rho_deg, clamped to [0, 1]. */
FASSMVS_API fassmvs_status fassmvs_normals(fassmvs_ctx* ctx, const float* depth, const uint8_t* img, int W,
                               int H, const double K[9], int radius, float beta, float* normal,
                               float* raw, const double n_plane[3], float rho_deg, float* conf,
                               void* stream);

/* Eq. sampling_range / dynamic cost volume: window of D planes centred on the
 * plane through the nearest-neighbour upscaled coarse depth dc (Wc x Hc):
 * lo = clamp(floor(c + 1/2) - D/2, 0, G - D), c = (rho - rho0) / drho, taken
 * in FP32 (see the oracle's statement of the operation order). */
FASSMVS_API fassmvs_status fassmvs_window(fassmvs_ctx* ctx, const float* dc, int Wc, int Hc, int W, int H,
                              const double K[9], const double n[3], double rho0, double drho,
                              int G, int D, int32_t* lo, void* stream);

/* Eq. sgm-smooth-sn index jumps from the upscaled coarse depth dc and normal
 * nc (Wc x Hc) for the sweep normal n: the predecessor ray meets the tangent
 * plane at Q, di = round_half_away((1/delta(Q) - 1/delta(P)) / drho) with
 * delta(X) = -n^T X, clamped to +-dmax, 0 when the tangent plane or the sweep
 * planes do not face the rays (FP32; for n = (0,0,-1) delta is the depth). */
FASSMVS_API fassmvs_status fassmvs_dsn(fassmvs_ctx* ctx, const float* dc, const float* nc, int Wc, int Hc,
                           int W, int H, const double K[9], const double n[3], double drho, int dmax,
                           int8_t* dI, void* stream);

/* Stage timers.  While enabled, the library brackets each stage it launches
 * with CUDA events on the call's stream and accumulates the elapsed time
 * (milliseconds) and launch count per stage; reading waits for the recorded
 * events.  Stages: */
enum {
    FASSMVS_STAGE_PYRAMID = 0, /* pyramid levels of all views */
    FASSMVS_STAGE_CENSUS = 1,  /* reference census + per-level homography tables */
    FASSMVS_STAGE_COST = 2,    /* plane-sweep cost volume kernel */
    FASSMVS_STAGE_SGM = 3,     /* all aggregation paths (two-pass form: with the winner-takes-all) */
    FASSMVS_STAGE_WTA = 4,     /* winner-takes-all + refinement (per-direction form only) */
    FASSMVS_STAGE_MEDIAN = 5,  /* 5x5 median */
    FASSMVS_STAGE_NORMALS = 6, /* normals, smoothing, confidence */
    FASSMVS_STAGE_WINDOW = 7,  /* plane windows + surface-normal jumps */
    FASSMVS_STAGE_RELAYOUT = 8, /* blocked cost volume -> pixel-major layout */
    FASSMVS_NSTAGES = 9
};
FASSMVS_API fassmvs_status fassmvs_profile_enable(fassmvs_ctx* ctx, int on);
/* ms[FASSMVS_NSTAGES], counts[FASSMVS_NSTAGES] (either may be NULL); reset != 0
 * clears the totals after reading. */
FASSMVS_API fassmvs_status fassmvs_profile_read(fassmvs_ctx* ctx, double* ms, uint64_t* counts,
                                                int reset);

/* Waits for the context's last stream and reports deferred device errors. */
FASSMVS_API fassmvs_status fassmvs_sync(fassmvs_ctx* ctx);

/* Human-readable description of the last failure of this context (never
 * NULL; thread-local text for ctx == NULL). */
FASSMVS_API const char* fassmvs_last_error(const fassmvs_ctx* ctx);

/* Number of kernels the library launched since the context was created. */
FASSMVS_API uint64_t fassmvs_launch_count(const fassmvs_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* FASSMVS_H */

/*
 * tigas.h -- C ABI of the B300-native forward 3D Gaussian Splatting renderer.
 *
 * The library turns a GPU-resident Gaussian scene and a client's 6DoF pose
 * into an RGBA8 frame at the resolution the client's ABR controller picks.
 * This is the rendering engine of the paper's GPU backend (Sec. 4.1, Sec. 5.1
 * "Rendering Engine"): scenes stay resident in device memory across requests
 * (Sec. 4.1 "GPU Backend", persistent VRAM residency), every request is an
 * isolated, stateless render task (Sec. 4.2), and requests carry the fields
 * of the paper's POST /render body: azimuth, elevation, camera centre t,
 * fx, fy, cx, cy, W, H (Sec. 5.2 "Client Interface").
 *
 * Conventions shared by every entry point:
 *  - Every call returns a tigas_status.  No call aborts, traps or exits; on
 *    error a message is available from tigas_last_error() (thread-local).
 *  - Pointers that "may be host or device" are classified with
 *    cudaPointerGetAttributes; memory the CUDA runtime does not know is
 *    treated as pageable host memory.
 *  - The library owns scene memory and its internal workspace.  The caller
 *    owns every input array and every output buffer.
 *  - cuda_stream arguments are cudaStream_t values passed as void* (NULL:
 *    the library's own stream).
 *  - Image layout: row-major, top row first, 4 bytes per pixel (R, G, B, A),
 *    A = 1 - T (final transmittance), each channel floor(clamp(x,0,1)*255+0.5).
 */
#ifndef TIGAS_H
#define TIGAS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TIGAS_OK = 0,
    TIGAS_ERR_INVALID = 1,   /* bad argument: null, non-finite, out of range, bad handle */
    TIGAS_ERR_OOM = 2,       /* device or pinned host allocation failed */
    TIGAS_ERR_CUDA = 3,      /* a CUDA runtime call or kernel failed */
    TIGAS_ERR_AGAIN = 4,     /* server: admission full, or request superseded */
    TIGAS_ERR_OVERFLOW = 5,  /* pair count exceeded the fixed pair budget */
    TIGAS_ERR_TIMEOUT = 6,   /* a bounded wait ran out */
    TIGAS_ERR_NOT_FOUND = 7, /* unknown ticket or model identifier */
    TIGAS_ERR_IO = 8         /* a file or folder could not be opened or read */
} tigas_status;

/* Client pose (Sec. 5.1 "Rendering Engine", Sec. 5.2 request body):
 * azimuth theta and elevation phi in radians, camera centre t in world units.
 * Camera rotation R = R_y(theta) R_x(phi); camera axes x right, y down,
 * z forward; world->camera transform T = [R^T, -R^T t; 0, 1]. */
typedef struct {
    double azimuth;
    double elevation;
    double t[3];
} tigas_pose;

/* Pinhole intrinsics in pixels at the requested width x height: u = fx x/z + cx,
 * v = fy y/z + cy (Sec. 5.1 projection).  Pixel (i, j) is sampled at
 * (i + 0.5, j + 0.5).  On an ABR resolution change the caller scales all four
 * with the frame (Sec. 5.3), which keeps the field of view fixed. */
typedef struct {
    double fx, fy, cx, cy;
} tigas_intrinsics;

enum { TIGAS_STORAGE_FP32 = 0, TIGAS_STORAGE_FP16 = 1 };

/* Scene description: raw per-Gaussian attributes as a 3DGS PLY holds them
 * (Sec. 5.1 "PLY Model and Primitives").  All arrays float32, row-major:
 *   means[n][3], log_scales[n][3], quats[n][4] (w,x,y,z; need not be unit),
 *   opacity_logits[n], sh[n][16][3] (coefficients past sh_degree ignored).
 * storage: TIGAS_STORAGE_FP32 keeps activated attributes in FP32 (236 B of
 * payload per Gaussian); TIGAS_STORAGE_FP16 keeps positions in FP32 and
 * opacity, scales, rotation and SH in FP16 (124 B of payload). */
typedef struct {
    uint64_t n;                   /* number of Gaussians, 1 .. 2^27 */
    int sh_degree;                /* 0..3 */
    int storage;                  /* TIGAS_STORAGE_* */
    const float* means;
    const float* log_scales;
    const float* quats;
    const float* opacity_logits;
    const float* sh;
    int inputs_on_device;         /* 1: the five arrays are device pointers */
    float background[3];          /* RGB composited behind the Gaussians */
} tigas_scene_desc;

typedef struct tigas_scene tigas_scene;

/* Upload and activate a scene (Sec. 5.1: scale = exp(s), opacity =
 * sigmoid(logit), q / |q|) into the library's resident device layout.
 * The caller keeps its arrays.  Synchronous.  Errors: INVALID (null, n out of
 * range, sh_degree or storage invalid), OOM, CUDA. */
tigas_status tigas_scene_load(const tigas_scene_desc* desc, tigas_scene** out_scene);

/* Drop the caller's reference.  The scene's memory is released once no
 * render or queued server request uses it (reference counting, Sec. 5.1
 * "Dynamic Multi-Model Runtime").  NULL is INVALID. */
tigas_status tigas_scene_free(tigas_scene* scene);

/* Resident bytes of a scene's attribute storage (the persistent VRAM
 * residency of Sec. 4.1 "GPU Backend"). */
tigas_status tigas_scene_bytes(const tigas_scene* scene, uint64_t* out_bytes);

/* Render one frame: the backend's rendering engine (Sec. 4.1 "Rendering
 * Engine": the tile-based rasterizer that projects the Gaussians onto the
 * image plane, cited to 3DGS), with the camera of Sec. 5.1 "Rendering Engine"
 * (T_{w->c} from the pose, pinhole K) at the resolution the client's ABR asked
 * for (Sec. 4.1: ABR-driven downscaled frames; Sec. 5.3 "Viewport Display":
 * intrinsics scaled with the resolution).  Each call is one isolated,
 * stateless render task (Sec. 4.2).  The hot path: preprocess, scan,
 * duplicate-and-key emit, radix sort, tile ranges, per-tile blend.
 * out_rgba8: width*height*4 bytes, host or device.  Synchronous: returns after
 * the frame is in out_rgba8.  width, height in 1..8192.
 * Errors: INVALID, OOM, CUDA. */
tigas_status tigas_render(tigas_scene* scene, const tigas_pose* pose, const tigas_intrinsics* intr,
                          int width, int height, uint8_t* out_rgba8);

/* Schedules of the same method; all three give the same frame.
 *  DEPTH_FIRST: the (tile | depth) LSD sort with its depth digits sorted once
 *      per Gaussian before duplication and its tile digits per pair; every
 *      tile's full list is built.
 *  FULL64: 64-bit (tile | depth) keys emitted per pair in index order, every
 *      significant digit sorted per pair; every tile's full list is built.
 *  SLICED (what tigas_render, tigas_render_batch and the server use): the
 *      depth-ordered Gaussians are cut into nearest-first slices and each
 *      slice is emitted, sorted and blended only for tiles that still have a
 *      pixel whose transmittance has not stopped; tile lists are never
 *      materialised whole, so tigas_debug_render cannot return them. */
enum {
    TIGAS_SORT_DEPTH_FIRST = 0,
    TIGAS_SORT_FULL64 = 1,
    TIGAS_SORT_SLICED = 2
};

typedef struct {
    uint64_t n_visible;          /* (Gaussian, view) entries kept after culling */
    uint64_t n_pairs;            /* (Gaussian, tile) pairs emitted (SLICED: summed over slices) */
    uint32_t n_tiles;            /* 16x16 tiles in the frame(s) */
    uint32_t sort_passes;        /* radix passes over the pair array */
    uint64_t blend_evals;        /* list entries evaluated, summed over pixels, up to each pixel's stop */
    uint64_t blend_fetched;      /* list entries staged into shared memory by the blend */
    uint64_t blend_contribs;     /* evaluations that blended (alpha >= 1/255, pixel not stopped) */
    uint32_t depth_sort_passes;  /* SLICED: radix passes the depth sort ran (passes whose digit is the
                                    same for every key are skipped); 0 for the other schedules */
    uint32_t depth_sort_near;    /* SLICED: entries the depth sort's passes after the first ran over:
                                    every entry, or, for a launch set of three or more slices with
                                    fixed pair capacities, the nearest ones, at least those before the
                                    last slice (the last slice's pairs are sorted by tile and depth);
                                    0 for the other schedules */
} tigas_frame_stats;

/* tigas_render with options (same passages: Sec. 4.1, 5.1, 4.2).  The float
 * output is the composite before the 8-bit encoding that the frame payload
 * of Sec. 5.1 ("8-bit JPEG payloads") starts from.
 *   out_rgba8:     width*height*4 bytes, host or device, or NULL
 *   out_rgba_f32:  width*height*4 floats (RGB + alpha before 8-bit encoding),
 *                  host or device, or NULL (at least one output is required)
 *   cuda_stream:   stream the work is ordered on; the call still returns only
 *                  after the frame is complete
 *   sort_mode:     TIGAS_SORT_*; both modes give the same tile lists
 *   stats:         filled when non-NULL */
tigas_status tigas_render_ex(tigas_scene* scene, const tigas_pose* pose, const tigas_intrinsics* intr,
                             int width, int height, uint8_t* out_rgba8, float* out_rgba_f32,
                             void* cuda_stream, int sort_mode, tigas_frame_stats* stats);

/* Render n_views (1..64) poses of one scene in one fused launch set
 * (batching): one preprocess pass reads the scene once for all views, one
 * sort orders every view's pairs.  This serves many clients' requests from
 * one shared resident model (Sec. 5.1 "Dynamic Multi-Model Runtime"); each
 * view stays its own stateless task (Sec. 4.2) and is rendered as tigas_render
 * renders it (Sec. 4.1, 5.1); fusing them is this library's, not the paper's.  Views may have different resolutions.
 * outs[v]: widths[v]*heights[v]*4 bytes, host or device.  Each result equals
 * the frame a separate tigas_render call gives.  Synchronous.
 * Errors: INVALID, OOM, CUDA. */
tigas_status tigas_render_batch(tigas_scene* scene, int n_views, const tigas_pose* poses,
                                const tigas_intrinsics* intrs, const int* widths, const int* heights,
                                uint8_t* const* outs, void* cuda_stream);

/* tigas_render_batch with a schedule (TIGAS_SORT_*) and statistics summed
 * over the views (stats may be NULL).  Passages as tigas_render_batch
 * (Sec. 4.1, 4.2, 5.1). */
tigas_status tigas_render_batch_ex(tigas_scene* scene, int n_views, const tigas_pose* poses,
                                   const tigas_intrinsics* intrs, const int* widths, const int* heights,
                                   uint8_t* const* outs, void* cuda_stream, int sort_mode, tigas_frame_stats* stats);

/* Asynchronous tigas_render_batch (SLICED schedule; passages as
 * tigas_render_batch, Sec. 4.1, 4.2, 5.1): enqueue the launch set on
 * cuda_stream (NULL: the own stream of the ticket's render context, so that
 * a launch set queued behind another overlaps it) and return at once with a
 * ticket.  Host outputs (pinned, for the call to stay asynchronous) are
 * copied back on a copy stream of the ticket's own, which overlaps the
 * copies with later launch sets.  tigas_render_wait completes it:
 * waits for the launch set, and if a fixed-capacity launch set outgrew its
 * pair buffers renders it again exactly before returning (the frames are
 * final only then).  Each outstanding ticket holds its own render context,
 * so a caller can keep the next launch set queued behind the current one;
 * output buffers of a ticket must not be reused before its wait returns.
 * Every ticket must be waited on exactly once.  Errors: as
 * tigas_render_batch. */
typedef struct tigas_ticket tigas_ticket;
tigas_status tigas_render_batch_async(tigas_scene* scene, int n_views, const tigas_pose* poses,
                                      const tigas_intrinsics* intrs, const int* widths, const int* heights,
                                      uint8_t* const* outs, void* cuda_stream, tigas_ticket** out_ticket);
tigas_status tigas_render_wait(tigas_ticket* ticket);

/* ------------------------------------------------------------------ debug */

/* Intermediate results of one frame of the tile-based rasterizer (Sec. 4.1
 * "Rendering Engine", cited 3DGS): per-Gaussian projection results, the
 * (tile, depth)-sorted pair list and the tile ranges, for parity tests.
 * Host arrays, all caller-allocated; any may be NULL.
 *   visible[n] (uint8), radius[n] (int32), rect[n*4] (int32: x_lo, y_lo,
 *   x_hi, y_hi, half-open, in tiles), depth[n] (float32 view z),
 *   uv[n*2] (float32), q[n] (float32 3 sqrt(lambda_max)),
 *   values[pair_capacity] (uint32 Gaussian index, sorted by (tile, depth)),
 *   ranges[n_tiles*2] (uint32 [start, end) per row-major tile),
 *   rgba_f32[width*height*4].
 * *out_pairs receives P; values are written only when P <= pair_capacity. */
typedef struct {
    uint8_t* visible;
    int32_t* radius;
    int32_t* rect;
    float* depth;
    float* uv;
    float* q;
    uint32_t* values;
    uint64_t pair_capacity;
    uint32_t* ranges;
    float* rgba_f32;
} tigas_debug_frame;

tigas_status tigas_debug_render(tigas_scene* scene, const tigas_pose* pose, const tigas_intrinsics* intr,
                                int width, int height, int sort_mode, tigas_debug_frame* out,
                                uint64_t* out_pairs);

/* Stable ascending LSD radix sort of n (key, value) pairs on the device (the
 * (tile | depth) key sort of the tile-based rasterizer of Sec. 4.1, cited
 * 3DGS; exposed for testing), sorting key bits
 * [begin_bit, end_bit) (0 <= begin_bit < end_bit <= 64).  keys: uint64,
 * values: uint32; *_in and *_out are distinct device buffers of n elements;
 * inputs are left unchanged.  Library-owned scratch.  Synchronous on
 * cuda_stream.  Errors: INVALID, OOM, CUDA. */
tigas_status tigas_sort_pairs_u64(const uint64_t* keys_in, const uint32_t* values_in, uint64_t* keys_out,
                                  uint32_t* values_out, uint64_t n, int begin_bit, int end_bit,
                                  void* cuda_stream);

/* The same sort for callers that cannot let this library allocate device
 * memory (applications that manage every byte of device memory through their
 * own pools or budgets, or threads that must not take the device-wide
 * synchronisation cudaMalloc/cudaFree can cause).  The paper has no
 * counterpart; this is a library convenience.
 *   - Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 *     Its scratch (ping-pong buffers and digit tables, about 16 MB) is one
 *     fixed device array that every GPU loading this library holds until the
 *     process exits.
 *   - n is limited to 1048576 (2^20) pairs; larger n returns
 *     TIGAS_ERR_INVALID with a message naming the limit.
 *   - The first call on a device looks up that device's scratch address
 *     (cudaGetSymbolAddress) with the device current; make that first call
 *     before any stream capture.  cuda_stream, when not NULL, must belong to
 *     the current device (else TIGAS_ERR_INVALID).
 *   - Asynchronous: returns once the work is queued on cuda_stream (NULL: the
 *     legacy default stream); outputs are ready when the stream gets there.
 *   - All calls on a device share the scratch and it keeps the last call's
 *     contents: calls whose work overlaps on the GPU (different streams or
 *     host threads without ordering between them) race and corrupt each other.
 *   - Being asynchronous, the call cannot return TIGAS_ERR_TIMEOUT: a sort
 *     whose bounded look-back wait ran out (see tigas_debug_sort_wait_timeout)
 *     leaves an untrusted order and records the event in a sticky per-device
 *     word instead.  tigas_sort_noalloc_check reports and clears it.
 * Other arguments, layout and errors as tigas_sort_pairs_u64. */
tigas_status tigas_sort_pairs_u64_noalloc(const uint64_t* keys_in, const uint32_t* values_in, uint64_t* keys_out,
                                          uint32_t* values_out, uint64_t n, int begin_bit, int end_bit,
                                          void* cuda_stream);

/* Completion check of tigas_sort_pairs_u64_noalloc (no counterpart in the
 * paper).  Waits for cuda_stream (NULL: the legacy default stream), then reads
 * and clears the current device's sticky timeout word: TIGAS_ERR_TIMEOUT when
 * a look-back wait of any allocation-free sort since the previous check ran
 * out (those sorts' outputs are not to be trusted), else TIGAS_OK.  Sorts
 * queued on other streams must have completed for the answer to cover them.
 * Allocates nothing.  Errors: INVALID (stream of another device), CUDA. */
tigas_status tigas_sort_noalloc_check(void* cuda_stream);

/* Failure-detection hook for tests (no counterpart in the paper): the probe
 * of tigas_debug_sort_wait_timeout run inside the allocation-free sort's
 * scratch, recording its run-out wait in the sticky word that
 * tigas_sort_noalloc_check reads.  Queued on cuda_stream; it overwrites the
 * scratch like a sort does.  Errors: INVALID (spin_limit not in 1..2^20,
 * stream of another device), CUDA. */
tigas_status tigas_debug_sort_noalloc_wait_timeout(int spin_limit, void* cuda_stream);

/* ---------------------------------------------------------------- serving */

typedef struct {
    uint64_t hbm_budget_bytes;   /* admission budget for in-flight workspace (0: 16 GiB) */
    int max_batch;               /* requests fused into one launch set (1..64, 0: 16) */
    int max_inflight;            /* launch sets in flight on separate streams (1..8, 0: 2) */
    int batch_window_us;         /* how long a partial batch may wait for more requests (0: none) */
} tigas_server_config;

typedef struct tigas_server tigas_server;

typedef struct {
    uint64_t ticket;
    uint64_t client_id;
    int status;                  /* tigas_status of this request */
    int width, height;
    double submit_us;            /* host monotonic clock, microseconds */
    double admit_us;             /* when the request entered a launch set */
    double done_us;              /* when its frame was complete in its buffer */
} tigas_completion;

/* Start a server thread that keeps taking requests while earlier ones render
 * (continuous batching, Sec. 5.1 multi-client runtime).  Errors: INVALID, OOM, CUDA. */
tigas_status tigas_server_create(const tigas_server_config* cfg, tigas_server** out_server);

/* Server lifecycle of the multi-client runtime (Sec. 5.1).
 * Finish queued work (cancel=0) or complete queued requests with
 * TIGAS_ERR_AGAIN (cancel=1), stop the thread and free the server. */
tigas_status tigas_server_destroy(tigas_server* server, int cancel);

/* Queue one render request.  out_rgba8 (host or device, w*h*4 bytes) must stay
 * valid until the ticket completes.  A queued, not yet admitted request of the
 * same client_id is superseded (completes with TIGAS_ERR_AGAIN): the newest
 * pose wins, as each request is a stateless per-frame task (Sec. 4.2).
 * Errors: INVALID, AGAIN (queue full). */
tigas_status tigas_server_submit(tigas_server* server, tigas_scene* scene, const tigas_pose* pose,
                                 const tigas_intrinsics* intr, int width, int height, uint8_t* out_rgba8,
                                 uint64_t client_id, uint64_t* out_ticket);

/* Completions of submitted requests, one per stateless per-frame task
 * (Sec. 4.2), each with its own status so that one failed request does not
 * affect the others.
 * Collect up to max completions, waiting up to timeout_us (0: do not wait)
 * for at least one.  *n_done receives the count (0 on timeout). */
tigas_status tigas_server_poll(tigas_server* server, tigas_completion* out, int max, int timeout_us,
                               int* n_done);

/* ------------------------------------------------------------- profiling */

/* Profiling (a library facility; the paper reports only whole-frame times,
 * Sec. 6 "Results").  Per-stage GPU time, measured with CUDA events recorded on the stream each
 * stage is launched on (a start and a stop event per stage, so host gaps
 * between stages are not charged to any stage).  Stages: 0 preprocess,
 * 1 depth sort, 2 scan, 3 emit, 4 pair sort, 5 ranges, 6 blend, and 7 the
 * whole frame (first stage start to last stage end).  Off by default. */
enum { TIGAS_N_STAGES = 8 };
tigas_status tigas_profile_enable(int enable);

/* Time only the stages in mask (bit s: stage s, s < 7; 0 turns timing off).
 * Each timed stage adds two event records per launch; timing only the stage
 * of interest keeps the rest of the launch set unperturbed.  The whole-frame
 * entry needs stages 0 and 6.  Errors: INVALID (bits 7 and up). */
tigas_status tigas_profile_stages(uint32_t mask);

/* Accumulated milliseconds and recorded launch sets per stage since the last
 * reset (ms[TIGAS_N_STAGES], calls[TIGAS_N_STAGES], either may be NULL);
 * reset=1 clears the accumulators after reading. */
tigas_status tigas_profile_read(double* ms, uint64_t* calls, int reset);

/* ------------------------------------------------------------ scheduling */

/* Scheduling (a library facility with no counterpart in the paper: the
 * paper does not describe how its rasterizer is scheduled on the GPU).
 * Parameters of the depth-sliced schedule of a launch set.  Frames do not
 * depend on them (only the time to render them does).
 *  n_slices:          depth slices, 1..16
 *  first_slice_inv:   the nearest slice holds 1/first_slice_inv of the kept
 *                     entries, later ones grow geometrically to all of them,
 *                     1..4096 (not used when n_slices is 1)
 *  blend_ctas_per_sm: persistent blend CTAs per SM, 0..64; 0 or more than
 *                     fit means as many as fit (default 0)
 *  blend_batch:       list entries a blend warp stages in shared memory at a
 *                     time, 16 or 32 (0 is read as 32; default 32)
 *  views_per_set:     most views a server launch set fuses (the smaller of
 *                     this and the server's max_batch), 0..64, 0 = no cap
 *                     (default 0); read from the schedule of the server's
 *                     max_batch; tigas_render_batch* are not affected
 * Launch sets are grouped by their view count into seven classes (1, 2,
 * 3-4, 5-8, 9-16, 17-32 and 33-64 views), and each class has its own
 * schedule: a slice costs a fixed number of launches, which weigh more in a
 * small launch set, so small ones do better with fewer slices.  Defaults
 * (n_slices / first_slice_inv): 3 / 16 for one view, 4 / 64 for two, 5 / 64
 * for three or four, 6 / 64 for more. */
typedef struct {
    int n_slices;
    int first_slice_inv;
    int blend_ctas_per_sm;
    int blend_batch;
    int views_per_set;
} tigas_schedule;

/* tigas_set_schedule sets the schedule of every class;
 * tigas_set_schedule_for_views that of the class of n_views (1..64) only;
 * tigas_get_schedule reads the schedule of the class of n_views (1..64).
 * Errors: INVALID (out of range; nothing is changed).  Launch sets already in
 * flight keep the schedule they started with. */
tigas_status tigas_set_schedule(const tigas_schedule* schedule);
tigas_status tigas_set_schedule_for_views(int n_views, const tigas_schedule* schedule);
tigas_status tigas_get_schedule(int n_views, tigas_schedule* schedule);

/* Autotuner of the batching step: renders launch sets of n_views views
 * (device RGBA8 outputs, resolutions widths/heights[n_views]), cycling through
 * n_sets (1..1024) pose sets (poses and intrs hold n_sets * n_views entries,
 * set-major) so that the timing covers varying pair counts.
 *  1. Every candidate sliced schedule (slices 1, 2, 3, 4, 5, 6, 7, 8, 12 x
 *     first slice 1/8, 1/16, 1/32, 1/64, 1/128, 1/256 (one candidate for a
 *     single slice) x blend CTAs per SM all or 4 x blend batch 32 or 16):
 *     two untimed launch sets then `iters` (1..100) timed ones each; the four
 *     with the lowest median device time per launch set (CUDA events around
 *     its work on the render stream) run 2 iters + 1 more times each,
 *     interleaved, and the lowest median of those wins.
 *  2. With that schedule, the views per launch set: the n_views views of a
 *     pose set rendered as launch sets of m = n_views, n_views / 2, ... views
 *     (each m that divides n_views, launch sets of m views taking the winner),
 *     two untimed rounds then 2 iters + 1 timed ones each; the m with the
 *     lowest median time per view wins (views_per_set = m).
 * The result becomes the schedule of the class of n_views (and, when m is
 * smaller than n_views, the winner without its views_per_set that of the
 * class of m); the other classes keep theirs.  It is written to *best
 * (best_ms: the winner's median device time per launch set of n_views views
 * in step 1).  Call it while no other render is running.  Errors: INVALID, and
 * those of tigas_render_batch (every class's schedule in force before the
 * call is restored). */
tigas_status tigas_autotune(tigas_scene* scene, int n_sets, int n_views, const tigas_pose* poses,
                            const tigas_intrinsics* intrs, const int* widths, const int* heights,
                            uint8_t* const* outs_rgba8, int iters, tigas_schedule* best, double* best_ms);

/* ---------------------------------------------------------- frame encoder */

/* Baseline JPEG (ITU-T T.81 sequential DCT, Huffman) of one RGBA8 frame in a
 * JFIF file: the payload the backend returns for a pose request (Sec. 4.1,
 * 5.1; Table 1 lists the quality levels 10, 35, 65 and 90).  Alpha is
 * ignored.
 *  Encoding: JFIF YCbCr with 16-bit fixed-point weights, 4:2:0 chroma (the
 *  rounded mean of each 2x2 group; the image extended to whole 16x16 MCUs by
 *  repeating its last column/row), the T.81 FDCT with 13-bit fixed-point
 *  weights, Annex K quantizer tables scaled by the quality (5000/q below 50,
 *  200 - 2q above), nearest rounding, Annex K Huffman tables, a restart
 *  marker every restart_mcus MCUs.
 *   rgba:         width*height*4 bytes, host or device
 *   quality:      1..100;  restart_mcus: 1..65535 (intervals are encoded in
 *                 parallel: small intervals encode faster, each adds 2 bytes)
 *   out:          host or device buffer of out_capacity bytes
 *   *out_len:     the file length (also when it exceeds out_capacity)
 * Synchronous.  Errors: INVALID, OVERFLOW (out_capacity < *out_len), OOM, CUDA. */
tigas_status tigas_jpeg_encode(const uint8_t* rgba, int width, int height, int quality, int restart_mcus,
                               uint8_t* out, uint64_t out_capacity, uint64_t* out_len, void* cuda_stream);

/* ---------------------------------------------------------------- models
 * 3DGS PLY files (Sec. 4.1 and Sec. 5.1 "PLY Model and Primitives").  One
 * vertex per Gaussian with the properties x y z, f_dc_0..2, f_rest_0..(3M-1),
 * opacity, scale_0..2, rot_0..3 in any order (other properties such as
 * nx ny nz are ignored), in binary_little_endian, binary_big_endian or ascii
 * format, each of type char/uchar/short/ushort/int/uint/float/double.  The SH
 * degree d follows from the f_rest count 3M, M = (d+1)^2 - 1 in {0, 3, 8, 15};
 * f_rest is channel-major: f_rest_{c*M + j} is coefficient j + 1 of colour
 * channel c, f_dc_c coefficient 0.  rot_0 is the quaternion's real part.
 * Values are converted to float32 (round to nearest).  Elements other than
 * "vertex" are skipped (in binary files, those before it may not hold lists). */
typedef struct {
    uint64_t n;             /* vertex count, 1 .. 2^27 */
    uint64_t file_bytes;
    uint64_t body_offset;   /* byte offset of the vertex block (binary) */
    int sh_degree;          /* 0..3 */
    int format;             /* 0 binary little endian, 1 binary big endian, 2 ascii */
    uint32_t row_bytes;     /* bytes per binary vertex record */
    uint32_t n_properties;  /* vertex properties in the file */
} tigas_ply_info;

/* Parse a PLY header (and check that a binary body is complete) without
 * reading vertices.  Host only: needs no GPU.  Errors: INVALID (null, bad or
 * unsupported header, missing property, f_rest count not 0/9/24/45,
 * truncated), IO (cannot open). */
tigas_status tigas_ply_probe(const char* path, tigas_ply_info* out);

/* Decode a PLY's vertices into the raw attribute arrays of tigas_scene_desc
 * (means[n][3], log_scales[n][3], quats[n][4], opacity_logits[n],
 * sh[n][16][3], coefficients past the file's degree set to 0), n from
 * tigas_ply_probe.  The body is streamed into device memory and de-interleaved
 * by a kernel; with outputs_on_device = 0 the arrays are host memory and the
 * result is copied back.  Synchronous.  Errors: as tigas_ply_probe, OOM, CUDA. */
tigas_status tigas_ply_decode(const char* path, float* means, float* log_scales, float* quats,
                              float* opacity_logits, float* sh, int outputs_on_device);

/* tigas_ply_probe + decode + tigas_scene_load in one call, with the file's SH
 * degree; the raw arrays never leave the device. */
tigas_status tigas_scene_load_ply(const char* path, int storage, const float background[3],
                                  tigas_scene** out_scene);

/* Model registry (Sec. 4.1; Sec. 5.1 "Dynamic Multi-Model Runtime").  Models
 * in root_dir are (a) each sub-folder holding a PLY -- the highest
 * point_cloud/iteration_<k>/point_cloud.ply, else its first *.ply by name --
 * with identifier and name = the folder name and preview = preview.png|.jpg|
 * .jpeg in it; (b) each top-level <id>.ply without a same-named folder, with
 * preview <id>.png|.jpg|.jpeg beside it.  Files whose header does not parse
 * are skipped.  A model is loaded into HBM on its first acquire and shared
 * by all later acquires; the registry holds one reference while it is
 * loaded.  An eviction pass unloads every model with no outstanding acquire
 * that has been idle for idle_timeout_s seconds.  With resident_budget_bytes
 * > 0 a load first evicts idle models (least recently used first) until it
 * fits, else fails with OOM.  All registry calls are thread-safe. */
typedef struct tigas_registry tigas_registry;

typedef struct {
    char id[128];            /* truncated to 127 bytes */
    char name[128];
    char ply_path[1024];
    char preview_path[1024]; /* "" when the model has no preview image */
    uint64_t n;              /* Gaussians (from the header until loaded) */
    uint64_t file_bytes;
    uint64_t resident_bytes; /* 0 when not loaded */
    uint64_t loads;          /* times loaded since the registry opened */
    double idle_seconds;     /* loaded with no acquire outstanding: time since last use, else 0 */
    int sh_degree;
    int loaded;
    int users;               /* acquires not yet released */
    int reserved;
} tigas_model_info;

/* Open a registry over root_dir and scan it.  storage: TIGAS_STORAGE_*;
 * idle_timeout_s >= 0; background: as in tigas_scene_desc.  Host only until
 * the first acquire.  Errors: INVALID, IO (root_dir is not a readable folder). */
tigas_status tigas_registry_open(const char* root_dir, int storage, double idle_timeout_s,
                                 uint64_t resident_budget_bytes, const float background[3],
                                 tigas_registry** out);
/* Rescan root_dir: new models are added; known ones keep their state; ones
 * whose files are gone are dropped once unloaded.  Outputs may be NULL. */
tigas_status tigas_registry_scan(tigas_registry* reg, int* n_models, int* n_skipped);
tigas_status tigas_registry_count(tigas_registry* reg, int* n_models);
/* Metadata and state of model index (0 .. count-1, ordered by identifier). */
tigas_status tigas_registry_info(tigas_registry* reg, int index, tigas_model_info* out);
/* The model's resident scene, loading it first if needed (Synchronous; other
 * models stay usable meanwhile; concurrent acquires of a model being loaded
 * wait for that load).  *out_scene is a new reference: hand it back with
 * tigas_registry_release (it may be submitted to a server meanwhile).
 * Errors: NOT_FOUND (unknown identifier), OOM (budget or device), IO,
 * INVALID (bad file), CUDA. */
tigas_status tigas_registry_acquire(tigas_registry* reg, const char* model_id, tigas_scene** out_scene);
/* Return an acquired scene.  INVALID if it was not acquired from reg or was
 * already returned. */
tigas_status tigas_registry_release(tigas_registry* reg, tigas_scene* scene);
/* One eviction pass at the registry's current time; *n_evicted may be NULL. */
tigas_status tigas_registry_evict_idle(tigas_registry* reg, int* n_evicted);
/* Run the eviction pass every period_s seconds (> 0) on a background thread
 * until tigas_registry_close. */
tigas_status tigas_registry_start_eviction(tigas_registry* reg, double period_s);
/* Test clock: now_s >= 0 fixes the registry's time in seconds; negative
 * returns to the monotonic clock. */
tigas_status tigas_registry_set_clock(tigas_registry* reg, double now_s);
/* Stop the eviction thread, wait for loads in progress, drop the registry's
 * references and free reg.  Scenes still acquired stay valid until each is
 * freed with tigas_scene_free. */
tigas_status tigas_registry_close(tigas_registry* reg);

/* ------------------------------------------------------ quality metrics
 * Post-session evaluation (Sec. 5.3 "Sampled OPFS Capture and Post-Session
 * Materialization"; the PSNR and SSIM of Sec. 6).  Frames are RGBA8,
 * row-major, host or device memory (detected per pointer). */

/* Bilinear resample src (w x h) to dst (width x height), all four channels.
 * Source coordinate of output pixel d: s = (d + 0.5) * w / width - 0.5, taken
 * in 16.16 fixed point (floor), clamped to [0, w-1]; weights are the top 8
 * fraction bits; each channel is ((a(256-fx) + b fx)(256-fy) + (c(256-fx) +
 * d fx) fy + 2^15) >> 16, so the result is exact integer arithmetic.  Sizes
 * 1..8192.  Synchronous.  Errors: INVALID, OOM, CUDA. */
tigas_status tigas_resample_rgba8(const uint8_t* src, int w, int h, uint8_t* dst, int width, int height,
                                  void* cuda_stream);

/* SSIM (Wang et al., IEEE TIP 2004) and PSNR between frames a and b of
 * width x height (11..8192 each; alpha ignored).  SSIM: per R, G, B channel,
 * 11 x 11 Gaussian window with sigma 1.5 normalised to sum 1, C1 = (0.01 *
 * 255)^2, C2 = (0.03 * 255)^2, at every window position inside the frame;
 * *out_ssim is the mean over positions and channels.  Computed in FP32 with
 * centred samples: within 1e-3 of the exact value per window and 1e-5 on
 * the mean.  out_map (optional, host or device): [height-10][width-10] floats,
 * the per-position SSIM averaged over channels.  *out_psnr = 10 log10(255^2 /
 * MSE) over all pixels and the three channels (exact squared-error sum;
 * +inf when the frames are equal).  Outputs may be NULL.  Synchronous.
 * Errors: INVALID, OOM, CUDA. */
tigas_status tigas_image_quality(const uint8_t* a, const uint8_t* b, int width, int height, float* out_map,
                                 double* out_ssim, double* out_psnr, void* cuda_stream);

/* Launch sets that ran with a fixed pair capacity (graph replay or a shape's
 * first launch set), outgrew it and were rendered again exactly, since load
 * (scheduling facility; no counterpart in the paper). */
uint64_t tigas_exact_rerenders(void);

/* Failure-detection hook for tests (no counterpart in the paper).  Runs one
 * block of the radix sort's scatter pass whose decoupled look-back waits on
 * digit counts of a preceding chunk that no block ever publishes; each wait
 * gives up after spin_limit polls (1..2^20) and the block records the same
 * timeout flag a real sort would.  Returns TIGAS_ERR_TIMEOUT when the flag
 * was recorded (the expected outcome; the device stays usable), TIGAS_OK if
 * it was not, INVALID for a bad limit, OOM/CUDA otherwise.  Synchronous;
 * allocates and frees its own ~140 KB of device memory. */
tigas_status tigas_debug_sort_wait_timeout(int spin_limit);

/* Host-side fault injection for tests (no counterpart in the paper; the
 * failures it stands for are the ones Sec. 5.3 "Viewport Display" shows to
 * the user and Sec. 4.2 confines to one request).  Every device (kind 0) and
 * pinned host (kind 1) allocation the library makes goes through one
 * counter per kind: after this call, allocations nth .. nth + count - 1 of
 * that kind (1 = the next one) fail as if the memory were exhausted, without
 * calling the CUDA allocator, and the calls that made them return
 * TIGAS_ERR_OOM with a message.  nth = 0 clears the kind.  Nothing is asked
 * of the GPU: no fault, trap or hang is involved.  Process-wide.
 * Errors: INVALID (kind not 0/1, nth < 0, count < 1 with nth > 0). */
tigas_status tigas_debug_fail_alloc(int kind, int64_t nth, int64_t count);

/* Free the workspace of every render context that no call is using (device
 * arenas, captured CUDA graphs, output staging, pinned buffers); later calls
 * allocate it again (a library facility, like returning cached memory to the
 * device; no counterpart in the paper).  Scenes, servers and outstanding
 * tickets are not affected.  Always TIGAS_OK. */
tigas_status tigas_release_workspace(void);

/* Scheduling facility (no counterpart in the paper).
 * Launch sets of the sliced schedule are captured as CUDA graphs per shape
 * (scene, view count and resolutions) when a shape appears a second time, and
 * replayed from then on.  A shape's first launch set runs directly with a
 * pair capacity per slice taken from the largest slice seen so far (exactly,
 * with a host round trip per slice, while nothing has been seen); a launch
 * set that outgrows its capacity is rendered again exactly before the call
 * returns.  enable=0 turns graphs off (default on).  Every call also makes the
 * idle render contexts forget their graphs, seen shapes and capacities. */
tigas_status tigas_set_graphs(int enable);

/* ------------------------------------------------------------------ misc */

/* Message of the last failed call on this thread ("" if none): the short
 * text a client shows in place of the frame when a request fails (Sec. 5.3
 * "Viewport Display": errors replace the viewport with a short message). */
const char* tigas_last_error(void);

/* Library version string (no counterpart in the paper). */
const char* tigas_version(void);

/* Kernel launches issued by this process so far (all entry points; no
 * counterpart in the paper). */
uint64_t tigas_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* TIGAS_H */

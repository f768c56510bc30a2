/*
 * pmbs.h - C ABI of the B300 batched push-rollout engine for PMBS (parallel Monte
 * Carlo tree search with batched simulation, arXiv 2207.06649).
 *
 * The engine executes the paper's batch expansion and batch simulation (Sec. IV-C):
 * many environments, each set to one selected tree state (Sec. IV-C, batch expansion
 * sets the simulator's environments to the chosen states and applies all transitions
 * at once), execute a first push action and then further random pushes drawn
 * by the contour action sampler (Sec. IV-B "Speeding up Action Sampling"), with a
 * terminal test after every push (Sec. IV-C "Batch Simulation").  A scene is a set of
 * rigid boxes on a table plane with a designated target (Sec. III-A, state space); an
 * action is a straight push a^p = (x_s, y_s, x_e, y_e) of a kinematic vertical capsule
 * (Sec. III-A, action space); the transition is rigid-body simulation with friction and
 * collisions (Sec. III-A, transition function); the terminal test is a geometric
 * grasp-clearance check in place of the learned grasp classifier (Sec. IV-B "Grasp
 * Evaluation"); the cost-to-go of an environment is the number of pushes until the
 * target is graspable and its reward gamma^(cost-1) (Sec. III-A reward, Sec. V-A gamma).
 *
 * Conventions.  SI units (m, kg, s, rad); z up; the table plane is z = 0; quaternions
 * are (w, x, y, z).  A box state row has 13 floats: x y z qw qx qy qz vx vy vz wx wy wz.
 * All arithmetic is IEEE binary32 on CUDA cores of one GPU (sm_103a).
 *
 * Errors.  Every call returns a pmbs_status; nothing aborts, exits or traps the GPU.
 * CUDA errors map to PMBS_E_CUDA and invalid arguments to PMBS_E_INVALID, with a
 * message in pmbs_last_error().  Device-side waits are bounded.
 *
 * Ownership.  The context owns all device memory it allocates (or the arena handed to
 * pmbs_create_with_arena, which the caller keeps alive until pmbs_destroy).  Host input
 * arrays are copied before a call returns; host output arrays belong to the caller.
 * Pointers documented as "device" must be device-accessible pointers on the context's
 * device; every other pointer is a host pointer.
 *
 * Threads.  pmbs_create / pmbs_destroy are not thread-safe.  Every other call takes the
 * context's lock, so calls from several threads are serialised and safe.
 */
#ifndef PMBS_H
#define PMBS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pmbs_ctx pmbs_ctx; /* opaque, owned by the library */

typedef enum {
    PMBS_OK = 0,
    PMBS_E_INVALID = 1,   /* bad argument or scene (non-finite, non-unit quaternion, ...) */
    PMBS_E_OOM = 2,       /* device arena cannot hold the request (memory admission) */
    PMBS_E_CUDA = 3,      /* a CUDA runtime call failed; see pmbs_last_error */
    PMBS_E_NOT_READY = 4, /* the batch still has substeps to run */
    PMBS_E_TIMEOUT = 5,   /* a bounded device wait gave up */
    PMBS_E_BUSY = 6       /* the resource is in use (e.g. releasing a running batch) */
} pmbs_status;

/* Per-environment result flags (out_flags). */
enum {
    PMBS_FLAG_GRASP_AFTER_PUSH1 = 1, /* target graspable after the first push */
    PMBS_FLAG_INVALID_START = 2,     /* first push starts inside a box: not simulated */
    PMBS_FLAG_OUT_OF_WORKSPACE = 4,  /* a box centre left the table (Sec. V-A boundary) */
    PMBS_FLAG_CONTACT_OVERFLOW = 8,  /* a pair/manifold/point/colour cap dropped contacts */
    PMBS_FLAG_NOOP_PUSH = 16         /* a sampled push found no free start: no-op push */
};

/* Event counters per environment (pmbs_query_events), in this order. */
#define PMBS_NUM_EVENTS 18

/* Phase timers per environment (pmbs_query_phase_cycles), in this order: push set-up
 * (footprints, start check, contour sampler), gravity + frames + broadphase,
 * narrowphase, contact preparation, colouring, contact solve (with the optional warm
 * start), integration, end of push (workspace and grasp tests, child state). */
#define PMBS_NUM_PHASES 8

typedef struct {
    int device;                 /* CUDA device ordinal */
    int max_envs;               /* largest batch accepted by one pmbs_rollout_pushes */
    int max_boxes_per_env;      /* <= 64 */
    size_t mem_budget_bytes;    /* device arena size (scenes + batches + solver scratch) */
    float dt;                   /* substep length, 1/240 s */
    int substeps_per_push;      /* 240 */
    int pgs_iters;              /* 10 projected Gauss-Seidel iterations per substep */
    float gravity[3];           /* 0, 0, -9.81 */
    float table_half[2];        /* workspace half sizes, 0.2 x 0.2 m */
    float table_mu, pusher_mu;  /* 0.5, 0.5 (pair friction = sqrt(mu_a mu_b)) */
    float pusher_radius;        /* 0.01 m */
    float pusher_z0, pusher_z1; /* capsule segment z range, 0.01 .. 0.20 m */
    float pusher_speed;         /* 0.1 m/s */
    float push_length;          /* 0.1 m, length of device-sampled pushes */
    float gamma;                /* 0.8 (Sec. V-A) */
    float grasp_opening;        /* 0.085 m (two-finger gripper, fixed opening, Sec. III-A) */
    float grasp_clearance;      /* 0.002 m */
    float finger_depth;         /* 0.01 m */
    float finger_width;         /* 0.022 m */
    int grasp_angles;           /* 16 jaw angles k*pi/16, <= 32 */
    float margin;               /* 1e-3 m contact margin */
    float slop;                 /* 5e-4 m allowed penetration */
    float baumgarte;            /* 0.2 */
    float sample_clearance;     /* 0.005 m: sampled pushes start this far beyond radius */
    int sample_attempts;        /* 8 tries per sampled push, <= 32 */
    int contour_points;         /* 16 contour points per object (N_a, Sec. IV-B) */
    int contact_cap;            /* 512 contact points per environment */
    int manifold_cap;           /* 256 manifolds per environment (<= 1024) */
    int pair_cap;               /* 1024 box-box broadphase pairs per environment */
    int lanes_per_env;          /* lanes per environment (8, 16 or 32; a warp runs 32 / that
                                   environments); 0 = autotune */
    int warps_per_block;        /* launch shape (1, 2 or 4); 0 = autotune */
    int smem_points;            /* contact point slots (4 per manifold) in shared memory; -1 = auto */
    int smem_manifolds;         /* manifolds kept in shared memory per env (wins); -1 = auto */
    float watchdog_ms;          /* per environment and launch run-time limit (10000 ms, read
                                   as SM clock cycles at 2 GHz); an environment over it
                                   stops after its current substep, keeps its progress,
                                   and pmbs_step / pmbs_query_cost report PMBS_E_TIMEOUT;
                                   the next pmbs_step resumes it */
    float max_initial_penetration; /* 1e-3 m: scenes with deeper box-box overlap are refused
                                      (child states registered by pmbs_query_cost are the
                                      engine's own output and are not re-checked) */
    int warm_start;             /* 0 (default): contact impulses start at zero every substep;
                                   1: a point takes the impulses of the nearest point of the
                                   same body pair in the previous substep (matched within
                                   warm_tolerance in the frame of the pair's first dynamic
                                   body; friction carried as a world vector) */
    float warm_tolerance;       /* 2e-3 m: match distance for warm starting */
    int cylinders;              /* pmbs_rollout_noalloc only: 1 = the records may hold cylinders
                                   (runs the solver built with the cylinder contact paths);
                                   0 (default) = boxes only: an environment with a cylinder
                                   row is refused like one with a bad box count.  The other
                                   entry points decide from the loaded scenes. */
    int phase_timers;           /* 0 (default); 1 = every environment accumulates the SM clock
                                   cycles its warp (or lane group) spends in each phase of
                                   PMBS_NUM_PHASES, read with pmbs_query_phase_cycles.  Costs
                                   a clock read and a shared-memory add per phase and
                                   substep; off, one uniform branch per phase.  Ignored by
                                   pmbs_rollout_noalloc. */
} pmbs_config;

/* Fill *cfg with the defaults listed above.  Never fails. */
void pmbs_default_config(pmbs_config* cfg);

/* Create a context on cfg->device that enqueues all work on cuda_stream (a cudaStream_t;
 * NULL = the legacy default stream).  Allocates a device arena of cfg->mem_budget_bytes.
 * Returns PMBS_E_INVALID for out-of-range fields, PMBS_E_OOM / PMBS_E_CUDA on failure. */
pmbs_status pmbs_create(const pmbs_config* cfg, void* cuda_stream, pmbs_ctx** out);

/* As pmbs_create, but uses the caller's device allocation (e.g. a PyTorch tensor) of
 * arena_bytes bytes at device pointer d_arena (256-byte aligned) instead of allocating. */
pmbs_status pmbs_create_with_arena(const pmbs_config* cfg, void* cuda_stream, void* d_arena,
                                   size_t arena_bytes, pmbs_ctx** out);

/* Synchronise the stream and free everything the context owns.  NULL is a no-op. */
void pmbs_destroy(pmbs_ctx* ctx);

/* Message of the last error on this context (empty string if none).  Valid until the
 * next call on the context. */
const char* pmbs_last_error(const pmbs_ctx* ctx);

/* Load scenes into the device-resident scene store (Sec. IV-C batch expansion loads
 * selected states into environments; a scene here is such a state).  CSR over boxes:
 * scene s owns rows box_offset[s] .. box_offset[s+1]-1 of pose [B][7] (x y z qw qx qy
 * qz), vel [B][6] (linear, angular; NULL = at rest), half_ext [B][3], mass [B], mu [B];
 * target[s] is the local index of its target box.  A half_ext row (r, -r, h) is a
 * cylinder of radius r and half height h whose axis is its body z axis
 * (contact geometry: the right prism over the regular 16-gon inscribed in its circle;
 * inertia: the solid cylinder's); this convention holds in every entry point that takes
 * half extents.  Writes one id per scene to out_scene_ids.  Validation: finite values,
 * | |q| - 1 | <= 1e-3, 1 <= n <= max boxes, positive half extents (or a cylinder row with
 * equal radii) and mass, target in range, no body-body penetration deeper than
 * cfg->max_initial_penetration (separating-axis test on the device) -> else
 * PMBS_E_INVALID; no room in the arena -> PMBS_E_OOM.  Copies synchronously. */
pmbs_status pmbs_load_scenes(pmbs_ctx* ctx, int n_scenes, const int32_t* box_offset,
                             const float* pose, const float* vel, const float* half_ext,
                             const float* mass, const float* mu, const int32_t* target,
                             int32_t* out_scene_ids);

/* Release scenes.  Unknown or already-freed ids -> PMBS_E_INVALID; a scene used by a batch
 * that has not been released -> PMBS_E_BUSY. */
pmbs_status pmbs_free_scenes(pmbs_ctx* ctx, int n, const int32_t* scene_ids);

/* Enqueue a rollout batch (Sec. IV-C batch expansion + batch simulation, Alg. 1
 * Expansion and Simulation): environment e starts from scene scene_ids[e] and executes
 * first_push[e] = (x_s, y_s, x_e, y_e), then depth-1 pushes drawn on the device by the
 * contour sampler keyed by seeds[e].  Several environments may share one scene (leaf
 * parallelisation, Sec. IV-C).  Copies the inputs and returns a batch handle; no
 * substep runs until pmbs_step.  depth in 1..64; n_envs in 0..max_envs. */
pmbs_status pmbs_rollout_pushes(pmbs_ctx* ctx, int n_envs, const int32_t* scene_ids,
                                const float* first_push, int depth, const uint64_t* seeds,
                                int64_t* out_batch);

/* As pmbs_rollout_pushes with device pointers for scene_ids, first_push and seeds (read
 * on the stream before the first pmbs_step of the batch returns control). */
pmbs_status pmbs_rollout_pushes_device(pmbs_ctx* ctx, int n_envs, const int32_t* d_scene_ids,
                                       const float* d_first_push, int depth,
                                       const uint64_t* d_seeds, int64_t* out_batch);

/* Advance every unfinished environment of the batch by up to max_substeps substeps
 * (<= 0: to completion) in one persistent launch on the context's stream.  Returns
 * PMBS_OK when the batch is finished, PMBS_E_NOT_READY when substeps remain.  The call
 * synchronises the stream only when max_substeps > 0 (to report readiness); with
 * max_substeps <= 0 it returns PMBS_OK immediately after enqueueing.  With
 * max_substeps > 0: PMBS_E_TIMEOUT when an environment hit cfg->watchdog_ms in this
 * launch (its progress is kept; call again to resume), PMBS_E_INVALID when the batch names
 * an unknown scene id (device-side ids). */
pmbs_status pmbs_step(pmbs_ctx* ctx, int64_t batch, int max_substeps);

/* Run the batch to completion as a CUDA graph of launches that each advance every
 * unfinished environment by substeps_per_launch substeps (the substep loop captured in a
 * graph; e.g. 240 = one launch per push).  The graph is captured on the first call for a
 * given substeps_per_launch and replayed afterwards; results are bit-identical to
 * pmbs_step.  Enqueues and returns PMBS_OK. */
pmbs_status pmbs_step_graph(pmbs_ctx* ctx, int64_t batch, int substeps_per_launch);

/* Autotuner of the launch shape (batching knobs only, never the arithmetic): builds the
 * given batch once per candidate shape (lanes per environment 32/16/8, warps per block
 * 4/2/1, manifolds per environment kept in shared memory 0/8/16/40), times its first
 * `substeps` substeps (best of two freshly built batches), re-times the five fastest and
 * the default shape (32 lanes, 2 warps per block, 8 manifolds) over the whole rollout, then
 * picks the iteration tiling of the winner (one persistent
 * launch, or launches of one push or a quarter push of substeps each; the same results)
 * with CUDA events, and records the fastest shape for the batch's box-count bucket; later
 * batches in that bucket use it unless a shape is fixed.  Outputs may be NULL.  Blocks
 * until the timings finish. */
pmbs_status pmbs_autotune(pmbs_ctx* ctx, int n_envs, const int32_t* scene_ids, const float* first_push,
                          int depth, const uint64_t* seeds, int substeps, int32_t* out_lanes_per_env,
                          int32_t* out_warps_per_block, int32_t* out_smem_manifolds, float* out_ms,
                          int32_t* out_substeps_per_launch);

/* Results of a finished batch, copied to host arrays of n_envs entries: cost (pushes
 * until graspable, depth+1 if never), reward (gamma^(cost-1) or 0), flags (PMBS_FLAG_*).
 * out_child_states (NULL to skip): [sum of boxes][13] state after push 1, the new tree
 * node of the expansion (Sec. IV-C); out_child_scene_ids (NULL to skip): registers each
 * child state as a new scene and writes its id.  Synchronises the stream.  Any output
 * pointer may be NULL.  PMBS_E_TIMEOUT when environments were stopped by the watchdog
 * (the batch then counts as unfinished again and pmbs_step resumes it); PMBS_E_INVALID
 * when the batch names an unknown scene id. */
pmbs_status pmbs_query_cost(pmbs_ctx* ctx, int64_t batch, int32_t* out_cost, float* out_reward,
                            uint8_t* out_flags, float* out_child_states,
                            int32_t* out_child_scene_ids);

/* As pmbs_query_cost but copies into device buffers asynchronously on the stream (no
 * status check: entries of environments stopped by the watchdog are undefined). */
pmbs_status pmbs_query_cost_device(pmbs_ctx* ctx, int64_t batch, int32_t* d_cost,
                                   float* d_reward, uint8_t* d_flags);

/* Current state of every environment ([sum of boxes][13], rows in env order) and the
 * number of substeps each environment has simulated so far.  Either may be NULL.
 * Synchronises the stream. */
pmbs_status pmbs_query_states(pmbs_ctx* ctx, int64_t batch, float* out_states,
                              int32_t* out_env_steps);

/* Event counters [n_envs][PMBS_NUM_EVENTS] (substeps, box-steps, pair tests, SAT tests,
 * face contacts, edge contacts, plane candidates, pusher candidates, contact points,
 * manifolds, PGS manifold visits, PGS point visits, push evaluations, sampler attempts,
 * clipped vertices, colours, box-box contact points, PGS point visits between two boxes)
 * used to count the algorithmic flops of a launch. */
pmbs_status pmbs_query_events(pmbs_ctx* ctx, int64_t batch, uint64_t* out_events);

/* Status word of the bounds-checked build (libpmbs_checked.so, compiled with
 * -DPMBS_BOUNDS_CHECK=1): out[0] = number of out-of-range indices met by the rollout
 * kernel on ctx's device since the last reset (shared-memory arrays, contact manifolds,
 * environments, state rows, warm-start records), out[1..3] = the first one's array id,
 * index and capacity.  Such an access was redirected to a sink and the kernel carried on
 * (no trap).  reset != 0 clears the word afterwards.  Synchronises the context's stream.
 * The release library returns PMBS_E_INVALID and zeros. */
pmbs_status pmbs_check_status(pmbs_ctx* ctx, uint32_t* out, int reset);

/* Per-phase SM clock cycles of every environment of a batch, [n_envs][PMBS_NUM_PHASES]
 * (order above), summed over its pushes and substeps and over every launch so far; all
 * zero unless the context was created with cfg->phase_timers = 1.  An environment's
 * phases add up to the cycles its warp spent on it outside fetching and loading it; the
 * cycles count while other warps share the SM, so they measure latency under the launch's
 * load, not issue slots.  Synchronises the context's stream.  Unknown batch or NULL
 * output -> PMBS_E_INVALID. */
pmbs_status pmbs_query_phase_cycles(pmbs_ctx* ctx, int64_t batch, uint64_t* out_cycles);

/* Number of environments and boxes in the batch. */
pmbs_status pmbs_batch_info(pmbs_ctx* ctx, int64_t batch, int32_t* out_n_envs,
                            int32_t* out_n_boxes);

/* Free a batch's device memory (synchronises the stream). */
pmbs_status pmbs_release_batch(pmbs_ctx* ctx, int64_t batch);

/* Snapshot evaluation of the bit-exact binary32 predicates, running the same device
 * functions as the rollout kernel, one environment per warp.  Environments are CSR over
 * state rows ([B][13]) and half extents ([B][3]).
 *  pmbs_eval_pairs: broadphase at the given states (Sec. III-A collisions; AABB per box,
 *    box-box pairs in lexicographic order, plane and pusher candidates).  pusher_xy
 *    [n_envs][2] or NULL (no pusher).  Outputs: out_pairs [n_envs][pair_cap][2],
 *    out_n_pairs [n_envs] (capped), out_plane / out_pusher [B] (per env, in CSR rows, the
 *    first out_n_plane[e] / out_n_pusher[e] entries are box indices).
 *  pmbs_eval_grasp: grasp-clearance decision of target[e] (Sec. IV-B grasp evaluation).
 *  pmbs_eval_sample: device-sampled push number k (>= 2) keyed by seeds[e] (Sec. IV-B
 *    contour sampling); out_attempt[e] = accepted attempt or -1 for a no-op push.
 *  pmbs_eval_start_blocked: 1 when a push starting at starts[e] (x, y) would start inside
 *    a box (Sec. IV-B start-pose collision check). */
pmbs_status pmbs_eval_pairs(pmbs_ctx* ctx, int n_envs, const int32_t* box_offset,
                            const float* states, const float* half_ext, const float* pusher_xy,
                            int32_t* out_pairs, int32_t* out_n_pairs, int32_t* out_plane,
                            int32_t* out_n_plane, int32_t* out_pusher, int32_t* out_n_pusher);
pmbs_status pmbs_eval_grasp(pmbs_ctx* ctx, int n_envs, const int32_t* box_offset,
                            const float* states, const float* half_ext, const int32_t* target,
                            uint8_t* out_graspable);
pmbs_status pmbs_eval_sample(pmbs_ctx* ctx, int n_envs, const int32_t* box_offset,
                             const float* states, const float* half_ext, const uint64_t* seeds,
                             int k, float* out_push, int32_t* out_attempt);
pmbs_status pmbs_eval_start_blocked(pmbs_ctx* ctx, int n_envs, const int32_t* box_offset,
                                    const float* states, const float* half_ext,
                                    const float* starts, uint8_t* out_blocked);

/* Top-down heightmaps of the workspace grid (Sec. V-A: the 0.288 m x 0.288 m workspace
 * centred on the table, seen by an overhead orthographic camera as 144 x 144 cells of
 * 2 mm; this depth image is what the paper's grasp classifier reads, Sec. IV-B).
 * out[e][j][i] (row j along y, column i along x, float32) is the height in m of the
 * highest box surface above the cell centre x_i = -0.144 + (i + 0.5) * 0.002 (y_j
 * likewise), or 0 where the table shows.  Each box's top over a cell is found by clipping
 * the vertical line through the cell centre against the box's three slabs; the whole map
 * is defined in binary32 with one rounding per operation in a fixed order, so it is
 * reproducible bit for bit.
 *  pmbs_render_heightmaps: a state snapshot (same arrays as pmbs_eval_pairs; 0..64 boxes
 *    per environment) to the host array out[n_envs][144][144]; synchronous.  Bad sizes
 *    -> PMBS_E_INVALID, no staging room -> PMBS_E_OOM.
 *  pmbs_render_heightmaps_device: the same with device arrays (d_states and d_half hold
 *    the rows of boxes box_offset[0] .. box_offset[n_envs]; box counts above 64 are
 *    clamped); asynchronous on the context's stream; d_out caller-owned and 16-byte
 *    aligned (PMBS_E_INVALID otherwise).
 *  pmbs_query_heightmaps: the current states of a batch's environments (after a finished
 *    batch: the final states) to the host array out[n_envs][144][144]; synchronous. */
pmbs_status pmbs_render_heightmaps(pmbs_ctx* ctx, int n_envs, const int32_t* box_offset, const float* states,
                                   const float* half_ext, float* out);
pmbs_status pmbs_render_heightmaps_device(pmbs_ctx* ctx, int n_envs, const int32_t* d_box_offset,
                                          const float* d_states, const float* d_half, float* d_out);
pmbs_status pmbs_query_heightmaps(pmbs_ctx* ctx, int64_t batch, float* out);

/* Heightmap form of the grasp test (the paper's classifier decides graspability from the
 * overhead depth image, Sec. IV-B; here the heightmap decides by geometry): for each
 * environment of a state snapshot (arrays as pmbs_eval_grasp), the target's heightmap is
 * rendered as above and out[e] = 1 when, for some jaw angle, the opening condition and
 * both finger rectangles of the footprint test hold with the rectangles checked against
 * the map: no cell whose centre lies in a rectangle beyond the target's side is higher
 * than the finger tips, `depth` m below the target's top.  Bit-exact in binary32.  Box
 * counts 1..64, targets in range and depth >= 0, else PMBS_E_INVALID; synchronous. */
pmbs_status pmbs_eval_grasp_heightmap(pmbs_ctx* ctx, int n_envs, const int32_t* box_offset, const float* states,
                                      const float* half_ext, const int32_t* target, float depth, uint8_t* out);

/* Launch shape the context uses for a batch whose largest scene has max_boxes boxes:
 * lanes per environment, warps per block, contact point slots and manifolds kept in
 * shared memory per environment, and shared bytes per block.  Chosen by the tuning rule
 * (or a tuned table, see pmbs_set_launch_shape) unless fixed in the config. */
pmbs_status pmbs_launch_shape(pmbs_ctx* ctx, int max_boxes, int32_t* out_lanes_per_env,
                              int32_t* out_warps_per_block, int32_t* out_smem_points,
                              int32_t* out_smem_manifolds, int32_t* out_smem_bytes);

/* Override the launch shape for subsequent batches (lanes_per_env in {8,16,32}, 0 = auto;
 * warps_per_block in {1,2,4}, 0 = auto; smem points/manifolds >= 0, -1 = auto).  Changes
 * scheduling only: every environment's arithmetic, and so every result, is bit-identical
 * across shapes. */
pmbs_status pmbs_set_launch_shape(pmbs_ctx* ctx, int lanes_per_env, int warps_per_block,
                                  int smem_points, int smem_manifolds);

/* Measured FP32 FMA throughput of the device (TFLOP/s) from a microbenchmark of
 * independent FMA chains at full occupancy; the paper has no counterpart (roofline
 * denominator for the contact solve). */
pmbs_status pmbs_fp32_peak(pmbs_ctx* ctx, double* out_tflops);


/* Serving loop (continuous batching of rollout requests from many concurrent planners;
 * the paper's planners submit one batch per MCTS iteration, Alg. 1, here many planners
 * share one GPU).  pmbs_server_create starts a dispatcher thread on the context with
 * n_streams non-blocking CUDA streams and at most max_inflight batches on the device.
 * Requests are admitted in arrival order whenever the context's arena can hold their
 * batch (memory-based admission: the arena size is the budget); admitted batches run
 * concurrently, each on its own stream with its own scratch.  A request's results are
 * bit-identical to the same request run alone.  The context must not be destroyed
 * before the server.  pmbs_server_destroy waits for batches on the device. */
typedef struct pmbs_server pmbs_server;
pmbs_status pmbs_server_create(pmbs_ctx* ctx, int n_streams, int max_inflight, pmbs_server** out);
/* Thread-safe: copies the request (same arguments as pmbs_rollout_pushes) and returns a
 * ticket at once. */
pmbs_status pmbs_server_submit(pmbs_server* server, int n_envs, const int32_t* scene_ids,
                               const float* first_push, int depth, const uint64_t* seeds,
                               int64_t* out_ticket);
/* Thread-safe: wait up to timeout_ms (< 0: forever; 0: poll) for a ticket; on success the
 * results (n_envs entries each; any pointer may be NULL) and the latency from submission
 * to completion are written and the ticket is released.  PMBS_E_NOT_READY (poll) or
 * PMBS_E_TIMEOUT while the request is still pending; PMBS_E_INVALID for an unknown or
 * cancelled ticket; the request's own error otherwise. */
pmbs_status pmbs_server_wait(pmbs_server* server, int64_t ticket, int timeout_ms, int32_t* out_cost,
                             float* out_reward, uint8_t* out_flags, int32_t* out_steps,
                             double* out_latency_ms);
/* out[11]: completed requests, simulated env-steps, seconds from the first submission to
 * the last completion, p50 and p99 latency (ms), mean latency (ms), peak arena bytes in
 * use, requests pending or on the device, finished results not yet claimed by a wait,
 * relaunches after the watchdog stopped environments (each resumes them where they
 * stopped, so results do not change), arena bytes in use now. */
pmbs_status pmbs_server_stats(pmbs_server* server, double* out);

/* Drop a ticket whose caller will never wait for it (e.g. a planner that gave up): a
 * pending request is removed, one on the device is discarded when it completes, a finished
 * one releases its held results.  Unknown ticket -> PMBS_E_INVALID. */
pmbs_status pmbs_server_cancel(pmbs_server* server, int64_t ticket);
void pmbs_server_destroy(pmbs_server* server);

/* Allocation-free rollout.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory.  Two kinds of caller need it: a planning
 * loop on a robot that, after start-up, must not pay cudaMalloc's device-wide
 * synchronisation and unbounded latency between decisions; and a library embedded in a
 * host process whose device memory is already reserved by another framework's caching
 * allocator, where a fresh allocation fails or fragments that pool.
 *
 * It needs no context.  The caller passes every input and output as device pointers on
 * device cfg->device and the stream cuda_stream (a cudaStream_t, NULL = legacy default):
 *   d_box_offset [n_envs+1] int32, CSR over boxes: environment e owns records
 *   d_box_offset[e] .. d_box_offset[e+1]-1, so the offsets must start at 0, never
 *   decrease, and end at the number of records B (the call cannot see B: an offset past
 *   the end of d_records makes the kernel read outside it); d_records [B][18] floats per
 *   box (x y z qw qx qy qz vx vy vz wx wy wz, half extents x y z, mass, mu); d_target
 *   [n_envs] local target index; d_first_push [n_envs][4]; d_seeds [n_envs] (may be NULL
 *   when depth == 1).  Outputs: d_state_out [B][13] final states, d_cost, d_reward,
 *   d_flags [n_envs] with the meaning of pmbs_query_cost.  Physics constants come from
 *   *cfg; the launch shape is the context entry points' default (one environment per
 *   warp, two warps per block, eight manifolds per environment in shared memory) unless
 *   cfg->lanes_per_env, warps_per_block or smem_manifolds / smem_points set it.
 * The results equal those of pmbs_rollout_pushes + pmbs_step + pmbs_query_cost for the
 * same inputs.  All scratch (descriptors, progress, counters, per-warp contact spill
 * regions) lives in one file-scope device array of 32 MiB that every device loading the
 * library holds until the process exits; at most 16384 environments per call, and
 * cfg->max_boxes_per_env <= 64.  Larger requests return PMBS_E_INVALID before any GPU
 * work.  The first call on a device looks up that array's device address (and sets the
 * kernel's shared-memory limit); make that first call before any stream capture.  The
 * call makes cfg->device current while it runs and puts the caller's current device back
 * before it returns.  It synchronises cuda_stream and returns:
 *   PMBS_OK;
 *   PMBS_E_INVALID for a bad argument, cfg->warm_start set (its caches need memory), or
 *     an environment that fails the per-environment checks -- a box count outside
 *     1..max_boxes_per_env, a negative first offset, a target out of range, a non-finite
 *     first push, or a record that scene loading would refuse (a non-finite value,
 *     | |q| - 1 | > 1e-3, a non-positive half extent or mass, a negative mu, a cylinder
 *     row (r, -r, h) while cfg->cylinders is 0, a cylinder row whose radii differ).
 *     Such environments are not simulated and their outputs are left as they were; the
 *     other environments are simulated as usual.  Unlike pmbs_load_scenes, the call does
 *     not measure initial body-body penetration: overlapping boxes are simulated (the
 *     solver pushes them apart);
 *   PMBS_E_TIMEOUT when the watchdog (cfg->watchdog_ms) stopped environments: their
 *     outputs are undefined and, having no batch to resume, the call cannot continue
 *     them (the context entry points resume such environments on the next pmbs_step);
 *   PMBS_E_CUDA for a CUDA error.
 * Every call shares the one array and starts by clearing what must start at zero; calls
 * whose GPU work overlaps (several threads or streams at once) race on it and must be
 * serialised by the caller.  It allocates no device memory. */
pmbs_status pmbs_rollout_noalloc(const pmbs_config* cfg, void* cuda_stream, int n_envs,
                                 const int32_t* d_box_offset, const float* d_records,
                                 const int32_t* d_target, const float* d_first_push,
                                 const uint64_t* d_seeds, int depth, float* d_state_out,
                                 int32_t* d_cost, float* d_reward, uint8_t* d_flags);

#ifdef __cplusplus
}
#endif

#endif /* PMBS_H */

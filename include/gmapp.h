/*
 * gmapp.h -- C ABI of the B300 (sm_103a) G-MAPP hot path.
 *
 * G-MAPP (arXiv 2606.12579) plans reactive motions by rolling out many
 * virtual point-mass agents through a sphere-world obstacle set built from a
 * depth cloud, then picking the cheapest agent.  This library implements
 * that data-parallel path as hand-written CUDA:
 *
 *   filter_cloud      Sec. IV-B, Sec. V-A   depth cloud -> obstacle set S_W
 *   rollout_agents    Sec. IV-A, Eq. (mfi), Alg. 1
 *                                           N_a agents x N_k steps under
 *                                           F = f_a + f_r (CF/MFI field)
 *   score_and_select  Sec. IV-A (cost, selection)  costs and best agent i*
 *
 * Conventions shared by every call:
 *   - Pointers named "device" point to memory of the context's GPU; "host"
 *     pointers to ordinary CPU memory.  The caller owns every buffer passed
 *     in (inputs, outputs, workspaces); the library owns only the context.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL is the legacy
 *     default stream).  Argument checks are synchronous and return an error
 *     status without launching anything.
 *   - Errors found on the device (capacity overflow, a bounded wait that ran
 *     out) are OR-ed into a device error word of the context; gmapp_sync()
 *     waits for the stream and reports and clears them.
 *   - No call throws, exits or traps.  gmapp_last_error() describes the last
 *     failure on the calling thread.
 *   - Vectors of agents use the layout [3][N_a] (one row per axis, float32),
 *     scalars per agent [N_a].
 */
#ifndef GMAPP_H
#define GMAPP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *gmapp_stream; /* == cudaStream_t */

typedef enum {
    GMAPP_OK = 0,
    GMAPP_ERR_INVALID_ARG = 1, /* a size, pointer, alignment or value is out of range */
    GMAPP_ERR_CAPACITY = 2,    /* an output or workspace is too small; the needed size is reported */
    GMAPP_ERR_CUDA = 3,        /* a CUDA runtime call failed (message in gmapp_last_error) */
    GMAPP_ERR_TIMEOUT = 4,     /* a device-side bounded wait gave up */
    GMAPP_ERR_NOT_READY = 5    /* the object is busy (serving: no free slot) */
} gmapp_status;

/* Device error-word bits (reported by gmapp_sync as the status above). */
#define GMAPP_DEVERR_CAPACITY 0x1u
#define GMAPP_DEVERR_TIMEOUT 0x2u
#define GMAPP_DEVERR_BOUNDS 0x4u

typedef struct gmapp_ctx gmapp_ctx;

/* Create a context on CUDA device `device`: allocates the device error word
 * and reads the device's SM count and cluster limits.  This and
 * gmapp_destroy are the only calls that allocate or free device memory.
 * Returns GMAPP_ERR_CUDA when the device cannot be used. */
gmapp_status gmapp_create(gmapp_ctx **out, int device);
void gmapp_destroy(gmapp_ctx *ctx);

/* Text of the last failure on the calling thread ("" when none). */
const char *gmapp_last_error(void);

/* Wait for `stream`, then read and clear the context's device error word:
 * GMAPP_OK, GMAPP_ERR_CAPACITY, GMAPP_ERR_TIMEOUT, GMAPP_ERR_INVALID_ARG (an
 * input that is only read on the device was out of range, e.g. an agent
 * without a gate in rollout_agents_culled) or GMAPP_ERR_CUDA. */
gmapp_status gmapp_sync(gmapp_ctx *ctx, gmapp_stream stream);

/* Cap on the polls of the grid-exchange waits (launch shapes with
 * exchange = 1) of rollout_agents, rollout_ensemble and their autotuners,
 * for later launches of this context: a wait that gives up sets
 * GMAPP_DEVERR_TIMEOUT, its CTA skips its later waits and every CTA still
 * finishes, so the failure path can be exercised without a hang (polls = 1
 * makes the exchanges give up).  Only these global-memory polls are capped:
 * the mbarrier waits for TMA copies and DSMEM deliveries keep their bound
 * (2^24 polls), since a CTA that stopped waiting for them could leave
 * while data is still in flight into its shared memory.  0 restores the
 * default (2^22 polls of an exchange word). */
gmapp_status gmapp_set_wait_limit(gmapp_ctx *ctx, uint32_t polls);

/* Raw device error word (bit mask of GMAPP_DEVERR_*), read after a stream
 * synchronisation, without clearing it. */
gmapp_status gmapp_peek_device_error(gmapp_ctx *ctx, uint32_t *bits);

/* ------------------------------------------------------------------------ */
/* Perception: filter_cloud (Sec. IV-B "GPU-accelerated Perception",          */
/* Sec. V-A: transform, workspace crop, voxel grid of edge 2 r_O, voxel       */
/* centres form S_W)                                                          */
/* ------------------------------------------------------------------------ */

/* Workspace voxel grid.  The workspace is the box [lo, lo + dims * voxel).
 * Constraints: voxel > 0, 1 <= dims[a] <= 2^24, dims[0]*dims[1]*dims[2]
 * < 2^32 - 1, min_pts >= 1. */
typedef struct {
    float lo[3];     /* world-frame lower corner (m) */
    float voxel;     /* voxel edge (m); the obstacle radius is r_O = voxel / 2 */
    int32_t dims[3]; /* cells per axis */
    int32_t min_pts; /* a voxel is an obstacle when it holds >= min_pts points */
} gmapp_workspace;

/* The sphere world S_W = {(p_Oj, r_O)}: N_O centres in ascending voxel-key
 * order (SoA float32), with per-voxel key, point count and smallest point
 * index.  All arrays are device memory of `cap` elements, 16-byte aligned;
 * `cap` is a multiple of 4.  `n` is ONE device int32 holding N_O (written by
 * filter_cloud; on overflow it holds the needed size).  keys, counts and
 * rep_idx may be NULL for obstacle sets that do not come from filter_cloud. */
typedef struct {
    float *x, *y, *z;
    uint32_t *keys;
    uint32_t *counts;
    uint32_t *rep_idx;
    int32_t *n;
    int64_t cap;
    float r_O; /* obstacle radius (m); filter_cloud sets it to voxel / 2 */
} gmapp_obstacles;

/* Bytes of device workspace filter_cloud needs for `n_raw` points. */
size_t gmapp_filter_workspace_bytes(int64_t n_raw, const gmapp_workspace *ws);

/* Depth cloud -> S_W.
 *   xyz         device, n_raw x 3 float32 AoS camera-frame points, 16-byte
 *               aligned; rows with a non-finite coordinate are dropped.
 *   T           host, 12 float32: row-major 3x4 camera-to-world [R | t].
 *   ws          host, the voxel grid (above).
 *   out         host struct of device buffers (above); out->r_O is set.
 *   workspace   device scratch of at least gmapp_filter_workspace_bytes(),
 *               256-byte aligned; contents need no initialisation.
 * Arithmetic is the exact binary32 sequence (no fused multiply-add):
 *   w_a = ((T[a][0] x + T[a][1] y) + T[a][2] z) + T[a][3]
 *   q_a = (w_a - lo_a) / voxel (IEEE division); kept iff 0 <= q_a < dims_a
 *   i_a = floor(q_a); key = (i_z dims_y + i_y) dims_x + i_x
 *   centre_a = lo_a + ((float) i_a + 0.5) voxel
 * The result is bit-identical from run to run.  When more than out->cap
 * voxels qualify, the first cap (by key) are written, *out->n holds the
 * total and the device error word gets GMAPP_DEVERR_CAPACITY. */
gmapp_status filter_cloud(gmapp_ctx *ctx, const float *xyz, int64_t n_raw,
                          const float T[12], const gmapp_workspace *ws,
                          gmapp_obstacles *out, void *workspace,
                          size_t workspace_bytes, gmapp_stream stream);

/* filter_cloud without any allocation or caller workspace.  The paper has
 * no counterpart: this exists for callers that must not allocate device
 * memory once running (a fixed-memory real-time control loop, a process
 * that may not call cudaMalloc at that point).  Same arguments, arithmetic
 * and results as filter_cloud, but the scratch lives in one fixed 16 MiB
 * array inside the library's device image, held by every GPU that loads the
 * library until the process exits.  No context is needed.
 *   - Sizes whose scratch would exceed 16 MiB (see
 *     gmapp_filter_workspace_bytes) are rejected with GMAPP_ERR_CAPACITY
 *     before anything is launched.
 *   - The call allocates and frees nothing.  Every call looks up the
 *     array's device address (cudaGetSymbolAddress) on the current device;
 *     the first call on a device loads the library's module there, so make
 *     it before any stream capture.
 *   - All calls share the one array (the kernels clear what must start at
 *     zero), so calls whose work overlaps on the GPU -- on different streams
 *     or devices' threads racing on one device -- race with each other;
 *     order them on one stream.
 *   - Output overflow: *out->n > out->cap, and a capacity flag that
 *     filter_cloud_noalloc_status reports (there is no context error word). */
gmapp_status filter_cloud_noalloc(const float *xyz, int64_t n_raw, const float T[12],
                                  const gmapp_workspace *ws, gmapp_obstacles *out,
                                  gmapp_stream stream);

/* Status of the latest filter_cloud_noalloc call on the current device:
 * waits for `stream`, then returns GMAPP_ERR_CAPACITY when that call found
 * more voxels than out->cap, else GMAPP_OK.  Each filter_cloud_noalloc call
 * clears the flag first.  Allocates nothing. */
gmapp_status filter_cloud_noalloc_status(gmapp_stream stream);

/* Batched filter: many clouds (a stream of frames, or several sensors) in
 * waves of jobs whose scratch fits in L2, three launches per wave
 * (Sec. IV-B, Sec. V-A, as filter_cloud).  The jobs are fixed at creation
 * (their device pointers are kept); each run filters every job's cloud into
 * its obstacle buffers with results bit-identical to filter_cloud on the
 * same cloud. */
typedef struct {
    const float *xyz;     /* device, n_raw x 3 float32 AoS, 16-byte aligned */
    int64_t n_raw;        /* >= 0 points */
    float T[12];          /* camera-to-world transform, row-major 3x4 */
    gmapp_workspace ws;   /* voxel grid; min_pts must be 1 */
    gmapp_obstacles out;  /* caller-owned output buffers; out.n receives N_O */
} gmapp_cloud_job;

typedef struct gmapp_filter_batch gmapp_filter_batch;

/* Checks every job (GMAPP_ERR_INVALID_ARG names the first bad one), keeps the
 * job table on the device and allocates the jobs' scratch once (the library
 * owns it; freed by gmapp_filter_batch_destroy).  Scratch: three sets of
 * wave slots, each slot 8 bytes per cell of the largest grid (a point count
 * and a smallest index per cell) plus the bitmap (about 52 MB for a
 * 200x200x160 grid); waves hold fewer jobs when the slot sets would take
 * more than half of the device memory free at creation.  Synchronous. */
gmapp_status gmapp_filter_batch_create(gmapp_ctx *ctx, const gmapp_cloud_job *jobs,
                                       int32_t n_jobs, gmapp_filter_batch **out);
void gmapp_filter_batch_destroy(gmapp_filter_batch *fb);

/* Filters every job's cloud: three launches per wave, the waves going
 * round-robin to `stream` and two streams of the batch that fork from and
 * join back into `stream` (graph-capturable; allocates nothing).  Output overflow of a job sets
 * GMAPP_DEVERR_CAPACITY and its out.n > out.cap. */
gmapp_status filter_cloud_batch(gmapp_filter_batch *fb, gmapp_stream stream);

/* One sensor's cloud for filter_clouds. */
typedef struct {
    const float *xyz; /* device, n_raw x 3 float32 AoS in the sensor's camera frame,
                         16-byte aligned */
    int64_t n_raw;    /* points (>= 0) */
    float T[12];      /* camera -> world, row-major 3x4 [R | t] */
} gmapp_sensor_cloud;

/* Workspace bytes filter_clouds needs for these clouds (0 when invalid). */
size_t gmapp_filter_clouds_workspace_bytes(const gmapp_sensor_cloud *clouds, int32_t n_sensors,
                                           const gmapp_workspace *ws);

/* Several sensors fused into one obstacle set (Sec. IV-B: the clouds of N_S
 * depth sensors, each with its own camera-to-world transform, voxelised
 * into one grid).  Every point of every sensor goes through the exact
 * binary32 sequence of filter_cloud with its sensor's T; a voxel is occupied
 * when any sensor's point falls in it; counts add over the sensors and the
 * smallest index is taken over all of them, point i of sensor s having the
 * index n_0 + ... + n_{s-1} + i (the clouds' concatenation).  clouds: host
 * array [n_sensors] (n_sensors >= 1; n_sensors = 1 is filter_cloud).  Sum of
 * n_raw below 2^32 - 1.  Output, workspace (gmapp_filter_clouds_workspace_
 * bytes) and errors as filter_cloud. */
gmapp_status filter_clouds(gmapp_ctx *ctx, const gmapp_sensor_cloud *clouds, int32_t n_sensors,
                           const gmapp_workspace *ws, gmapp_obstacles *out, void *workspace,
                           size_t workspace_bytes, gmapp_stream stream);

/* ------------------------------------------------------------------------ */
/* Rollout: rollout_agents (Sec. IV-A agent dynamics and agent set;           */
/* Eq. (mfi) circular-field force; Alg. 1 clamp, detection gate, sum)         */
/* ------------------------------------------------------------------------ */

/* Agent set A = {A_1 .. A_Na}; device arrays, float32. */
typedef struct {
    const float *p0; /* [3][n] start positions (m) */
    const float *v0; /* [3][n] initial velocities (m/s) */
    const float *c;  /* [3][n] artificial current vectors (used as given) */
    const float *k_r; /* [n] field gains; k_f = rho * k_r */
    const float *k_a; /* [n] attractive stiffness (K = k_a I_3) */
    const float *r_d; /* [n] detection radii (m); +inf = no gate */
    const float *r_a; /* [n] agent radii (m) */
    int32_t n;        /* N_a >= 1 */
} gmapp_agents;

/* Rollout constants (host struct). */
typedef struct {
    float goal[3];      /* p_goal (m) */
    float dt;           /* delta_t (s), > 0 */
    int32_t n_steps;    /* N_k >= 1 */
    float damping;      /* D = damping * I_3 */
    float inv_mass;     /* inertia tensor = inv_mass * I_3 */
    float rho;          /* repulsive scale (k_f = rho * k_r) */
    float eps;          /* minimum acceptable distance of Alg. 1, > 0 */
    float vel_half;     /* the 1/2 of the velocity update */
    float clear_margin; /* softplus clearance-penalty margin (m) */
    float clear_beta;   /* softplus sharpness (1/m), > 0 */
    int32_t ckpt_every; /* adjoint checkpoint interval (steps); 0 = no checkpoints */
    float cost_radius;  /* r_c of the goal and obstacle terms of the four-term
                           cost (Eq. cost_goal, Eq. cost_obs), > 0 when
                           gmapp_rollout_out.cost_terms is requested */
} gmapp_rollout_params;

/* Rollout outputs: device buffers written by rollout_agents. */
typedef struct {
    float *traj;      /* [n][n_steps+1][3] positions p_0..p_Nk, or NULL */
    float *p_final;   /* [3][n] */
    float *v_final;   /* [3][n] */
    float *path_len;  /* [n] sum_k |p_k+1 - p_k| */
    float *clear_pen; /* [n] sum_k softplus_beta(margin - m_k), or NULL */
    float *min_clear; /* [n] min_k m_k, or NULL */
    float *w_trace;   /* [n][n_steps] W_k (sum of Alg. 1), or NULL */
    float *m_trace;   /* [n][n_steps] clearance m_k, or NULL */
    float *f_trace;   /* [n][n_steps][3] repulsive force f_r at step k, or NULL */
    float *ckpt;      /* [ceil(n_steps/K)][6][n] state (p_k, v_{k-1}) entering steps
                         k = 0, K, 2K, ... with K = ckpt_every (rows: p x,y,z, v x,y,z),
                         for rollout_adjoint; or NULL */
    float *cost_terms; /* [5][n] sums of the four-term cost (Eq. cost_function) over the
                          candidate trajectory xi^(k) = p_{k-1}, k = 1..N_k (the N_k
                          states where the field is evaluated), for score_and_select4;
                          or NULL.  Rows: S_goal = sum_k min(|p_k - goal|, r_c) / r_c;
                          S_obs = sum_k max(r_c - m_k, 0) / r_c; L = sum_{k=1}^{N_k-1}
                          |p_k - p_{k-1}|; J = sum_{k=3}^{N_k-1} |p_k - 3 p_{k-1} +
                          3 p_{k-2} - p_{k-3}|^2, accumulated as (dt h)^2 |F_{k-1} -
                          F_{k-2}|^2 (h = vel_half dt inv_mass), the same quantity by
                          the step rule; d1 = |p_0 - goal|.  Needs cost_radius > 0 and
                          computes the clearance m_k.  rollout_agents and
                          rollout_ensemble only. */
    unsigned long long *heur_pairs; /* device counter, or NULL: the launch adds the number
                          of agent-obstacle pairs (of every heuristic) whose heuristic terms
                          (rsqrt, clamp, reciprocal, accumulation) it evaluated.  Every pair's |d|^2 and
                          gate are evaluated; a warp evaluates the heuristic terms of its
                          block of 64 obstacles only when one of the block's pairs passes
                          an agent's gate (Alg. 1's branch), so this is a multiple of 64
                          and at least the number of pairs within the gates.  For
                          accounting only (results do not depend on it); rollout_agents,
                          rollout_agents_blockcull and rollout_ensemble only (other calls
                          leave it untouched). */
} gmapp_rollout_out;

/* Roll all agents forward N_k steps in ONE launch.  Step k (0-based):
 *   s_j  = max(|p_k - p_Oj| - (r_a + r_O), eps),  W_k = sum_{s_j <= r_d} 1/s_j
 *   m_k  = min_j |p_k - p_Oj| - (r_a + r_O)
 *   g    = (|v|^2 c - v (v . c)) / |v|      (0 when |v|^2 < 1e-30), v = v_{k-1}
 *   F    = k_a (p_goal - p_k) - damping v + rho k_r W_k g
 *   v_k  = v_{k-1} + vel_half dt inv_mass F;  p_{k+1} = p_k + dt v_k
 * N_O is read from obs->n on the device (so the call may follow
 * filter_cloud on the same stream without a host round trip).  Obstacle
 * arrays must be 16-byte aligned with obs->cap a multiple of 4.  If N_O
 * exceeds obs->cap or what the launch can keep on chip, nothing is written
 * and GMAPP_DEVERR_CAPACITY is set.  The clearance m_k is reduced only
 * when clear_pen, min_clear or m_trace is requested.  FP32 arithmetic;
 * results are deterministic for a given launch shape. */
gmapp_status rollout_agents(gmapp_ctx *ctx, const gmapp_obstacles *obs,
                            const gmapp_agents *agents,
                            const gmapp_rollout_params *prm,
                            gmapp_rollout_out *out, gmapp_stream stream);

/* ------------------------------------------------------------------------ */
/* Differentiable rollout: rollout_adjoint (discrete adjoint of the step map  */
/* of Sec. IV-A with the Alg. 1 sum and the cost; the paper states the field  */
/* is C^1, Sec. IV-A; the adjoint itself is an addition to the paper)         */
/* ------------------------------------------------------------------------ */

/* Weights of the plan cost (Sec. IV-A cost; see score_and_select). */
typedef struct {
    float w_path;  /* weight of the path length */
    float w_goal;  /* weight of the final distance to the goal */
    float w_clear; /* weight of the clearance-penalty sum */
} gmapp_cost_weights;

/* Gradients per agent (device, float32). */
typedef struct {
    float *g_v0; /* [3][n] dC/dv0 */
    float *g_kr; /* [n]    dC/dk_r */
    float *g_ka; /* [n]    dC/dk_a */
    float *g_c;  /* [3][n] dC/dc (c used as given, not renormalised) */
    float *cost; /* [n] C_i recomputed by the adjoint pass, or NULL */
} gmapp_adjoint_out;

/* Bytes of device workspace rollout_adjoint needs: one 64-byte record per
 * agent per step of a checkpoint segment (n_agents x ckpt_every x 64). */
size_t gmapp_adjoint_workspace_bytes(int32_t n_agents, const gmapp_rollout_params *prm);

/* dC_i/d(v0, k_r, k_a, c) for C_i = w_path L_i + w_goal |p_i(N_k) - goal|
 * + w_clear sum_k softplus(margin - m_k), scaled per agent by grad_cost[i]
 * (device [n], NULL = 1).  `ckpt` is the checkpoint array written by a
 * rollout_agents call with the same obstacles, agents and parameters and
 * prm->ckpt_every = K >= 1.  The pass recomputes each K-step segment from
 * its checkpoint (last segment first), storing per-step W, grad W and the
 * nearest obstacle, then sweeps the segment backwards.  Derivatives are
 * those of the branch taken: pairs outside the gate or inside the clamp
 * contribute no gradient, and the clearance gradient follows the nearest
 * obstacle.  FP32; deterministic for a given launch. */
gmapp_status rollout_adjoint(gmapp_ctx *ctx, const gmapp_obstacles *obs,
                             const gmapp_agents *agents, const gmapp_rollout_params *prm,
                             const gmapp_cost_weights *w, const float *ckpt,
                             const float *grad_cost, gmapp_adjoint_out *out,
                             void *workspace, size_t workspace_bytes, gmapp_stream stream);

/* Launch shape of the rollout kernel (see rollout_agents_tuned). */
typedef struct {
    int32_t cluster;        /* CTAs per cluster, each holding 1/cluster of S_W: 1..16 */
    int32_t agents_per_cta; /* agents processed together by one cluster: 1..16 */
    int32_t threads;        /* threads of a CTA that evaluate obstacle pairs: 128, 256,
                               384 or 512 (each CTA has one more warp, which
                               exchanges partial sums and integrates) */
    int32_t exchange;       /* how the CTAs of a group combine their partial sums
                               each step: 0 = a thread-block cluster over
                               distributed shared memory; 1 = a cooperative
                               grid (all CTAs co-resident, groups * cluster <=
                               SM count) over tagged words in global memory,
                               which is not bound to the GPU's cluster
                               placement.  Exchange-1 launches of one context
                               use its exchange slots one at a time: the library
                               orders them across streams, except inside CUDA
                               graph capture, where the caller must. */
} gmapp_tuning;

/* Same as rollout_agents with an explicit launch shape (used by the
 * autotuner).  GMAPP_ERR_INVALID_ARG for shapes outside the ranges above or
 * an obstacle shard that does not fit in shared memory for obs->cap. */
gmapp_status rollout_agents_tuned(gmapp_ctx *ctx, const gmapp_obstacles *obs,
                                  const gmapp_agents *agents,
                                  const gmapp_rollout_params *prm,
                                  gmapp_rollout_out *out, const gmapp_tuning *tune,
                                  gmapp_stream stream);

/* rollout_agents with spatial culling over the key-sorted obstacle set
 * (Alg. 1's gate: pairs with s_j > r_d contribute nothing).  Each CTA keeps
 * the bounding box of every block of 128 consecutive obstacles of its
 * shard; each step, a warp visits only the blocks whose box lies within an
 * agent's gate radius r_d + R (widened by 2^-12 for rounding) and evaluates
 * their pairs exactly as rollout_agents does, in the same order.  So W, the
 * forces, the trajectories and the path lengths equal those of
 * rollout_agents at the same launch shape bit for bit.  The clearance m_k
 * is exact when the nearest obstacle lies within the agent's reach r_d + R,
 * else it is the smallest distance among the visited obstacles (>= r_d) or
 * +inf when none was visited.  Obstacles sorted by voxel key (filter_cloud's
 * order) make the blocks compact; any order gives the same results, culling
 * less.  An agent with r_d = inf cannot be culled: its group evaluates
 * every pair.  tune: the launch shape, or NULL for the one rollout_agents
 * would pick.  Arguments, outputs and errors as for rollout_agents. */
gmapp_status rollout_agents_blockcull(gmapp_ctx *ctx, const gmapp_obstacles *obs,
                                      const gmapp_agents *agents,
                                      const gmapp_rollout_params *prm,
                                      gmapp_rollout_out *out, const gmapp_tuning *tune,
                                      gmapp_stream stream);

/* Autotuner of the launch shape (for the batched/served pattern: the shape
 * is picked by measurement).  Ranks every shape that fits obs->cap by the
 * library's cost model (slowest CTA's pair count, co-resident clusters,
 * per-step exchange), runs the best `max_candidates` of them on the
 * caller's own inputs for min(probe_steps, n_steps) steps (CUDA events on
 * `stream`; each candidate once to warm up, once timed), and stores the
 * fastest in the context's cache, so later rollout_agents calls with the
 * same (obs->cap, agents->n, clearance outputs) use it.  Overwrites `out`.
 * Synchronous (waits for the timing events).  best_ms (may be NULL)
 * receives the fastest time scaled to the full n_steps. */
gmapp_status gmapp_autotune_rollout(gmapp_ctx *ctx, const gmapp_obstacles *obs,
                                    const gmapp_agents *agents,
                                    const gmapp_rollout_params *prm,
                                    gmapp_rollout_out *out, int32_t max_candidates,
                                    int32_t probe_steps, gmapp_tuning *best, float *best_ms,
                                    gmapp_stream stream);

/* The launch shape rollout_agents would choose for these sizes (for a
 * rollout that requests no clearance output): the autotuned shape if one
 * is cached, else the cost model's choice. */
gmapp_status gmapp_pick_tuning(gmapp_ctx *ctx, int64_t obs_cap, int32_t n_agents,
                               gmapp_tuning *tune);

/* ------------------------------------------------------------------------ */
/* Heterogeneous ensemble: rollout_ensemble (Sec. IV-A vector-field           */
/* heuristics: Heuristic 1, APF, Eq. (apf); Heuristic 2, MFI, Eq. (mfi);      */
/* "Other Heuristics": agents with different heuristics and large or small    */
/* detection radii form one ensemble; Sec. IV-D: agents grouped by heuristic) */
/* ------------------------------------------------------------------------ */

/* rollout_agents for an ensemble of three heuristics, agents ordered by
 * heuristic: indices 0 .. n - n_proj - n_apf - 1 follow the MFI field above
 * (the agent's own current c); the next n_proj agents MFI with the current
 * projected per obstacle (Eq. (mfi) with the equation after it); the LAST
 * n_apf agents (n - n_apf .. n - 1) the APF heuristic.  Per-agent r_d gives
 * each agent a large or small detection radius.  At step k, with
 * d_j = p_k - p_Oj and R = r_a + r_O:
 *   APF:        rho_j = max(|d_j|, R + eps),
 *               f = sum over j with |d_j| - R < r_d (strict) of
 *               (1/rho_j - 1/r_d) rho_j^-2 d_j / |d_j|   (a pair with d_j = 0 adds 0)
 *   projected:  s_j = max(|d_j| - R, eps), n_j = d_j / |d_j|, d' = -v_{k-1},
 *               c_j = d' - n_j (n_j . d'),
 *               f = sum over j with s_j <= r_d of (1/s_j) (d'/|d'|) x (c_j x d')
 *                 = (|v|^2 S - v B) / |v|,  S = sum a_j d_j,  B = sum a_j (d_j . v),
 *               a_j = (d_j . v) / (s_j |d_j|^2)   (f = 0 when |v|^2 < 1e-30;
 *               a pair with d_j = 0 adds 0)
 *   both:       F = k_a (p_goal - p_k) - damping v_{k-1} + rho k_r f
 * The rest of the step, the outputs and the error behaviour are those of
 * rollout_agents.  For APF and projected agents, w_trace holds |f| and
 * f_trace rho k_r f.  APF agents need r_d > 0 (+inf = no gate).
 * All agents run in ONE launch: the agent groups of the launch are
 * homogeneous (each holds only MFI or only APF agents), with groups shared
 * in proportion to the two counts.  `tune` selects the launch shape as in
 * rollout_agents_tuned (agents_per_cta is an upper bound per group; at most
 * 12 agents per group and 384 threads), or NULL for the library's choice.
 * With tune = NULL the shape is the one gmapp_autotune_ensemble cached
 * for these sizes, else the cost model's choice among ensemble shapes.
 * n_proj = n_apf = 0 is rollout_agents.  GMAPP_ERR_INVALID_ARG for negative
 * counts or n_proj + n_apf > n, for adjoint checkpoints (out->ckpt) in an
 * ensemble, or for a shape that does not fit. */
gmapp_status rollout_ensemble(gmapp_ctx *ctx, const gmapp_obstacles *obs,
                              const gmapp_agents *agents, int32_t n_proj, int32_t n_apf,
                              const gmapp_rollout_params *prm, gmapp_rollout_out *out,
                              const gmapp_tuning *tune, gmapp_stream stream);

/* rollout_ensemble with spatial culling over the key-sorted obstacle blocks,
 * as rollout_agents_blockcull does for MFI agents: every group (MFI, APF,
 * projected current) visits only the blocks of 128 obstacles whose bounding
 * box meets a gate of its agents.  Forces, trajectories and path lengths
 * equal rollout_ensemble's at the same launch shape bit for bit; the
 * clearance is as for rollout_agents_blockcull.  Arguments and errors as for
 * rollout_ensemble. */
gmapp_status rollout_ensemble_blockcull(gmapp_ctx *ctx, const gmapp_obstacles *obs,
                                        const gmapp_agents *agents, int32_t n_proj,
                                        int32_t n_apf, const gmapp_rollout_params *prm,
                                        gmapp_rollout_out *out, const gmapp_tuning *tune,
                                        gmapp_stream stream);

/* gmapp_autotune_rollout for an ensemble (n_proj, n_apf as in
 * rollout_ensemble): ranks the
 * shapes that fit the ensemble (groups split by heuristic), times the best
 * `max_candidates` on the caller's inputs and caches the fastest for later
 * rollout_ensemble calls with tune = NULL and the same (obs->cap,
 * agents->n, n_proj, n_apf, clearance outputs).  Same arguments, errors and
 * synchronous behaviour as gmapp_autotune_rollout; n_proj = n_apf = 0 is
 * that call. */
gmapp_status gmapp_autotune_ensemble(gmapp_ctx *ctx, const gmapp_obstacles *obs,
                                     const gmapp_agents *agents, int32_t n_proj, int32_t n_apf,
                                     const gmapp_rollout_params *prm,
                                     gmapp_rollout_out *out, int32_t max_candidates,
                                     int32_t probe_steps, gmapp_tuning *best, float *best_ms,
                                     gmapp_stream stream);

/* ------------------------------------------------------------------------ */
/* Rollout with spatial culling (Alg. 1's detection gate; the voxel grid of  */
/* Sec. IV-B as a neighbour grid)                                            */
/* ------------------------------------------------------------------------ */

/* Bytes of the neighbour index of a grid: (ceil(cells / 32) + 1) x 4. */
size_t gmapp_grid_index_bytes(const gmapp_workspace *ws);

/* Neighbour index of an obstacle set that filter_cloud (or filter_clouds)
 * built on the grid `ws`: index[w] = the number of obstacles whose key is
 * below 32 w, for w = 0 .. ceil(cells / 32) (device, uint32, written).
 * Reads obs->keys and N_O (obs->n) on the device; asynchronous. */
gmapp_status gmapp_grid_index(gmapp_ctx *ctx, const gmapp_obstacles *obs,
                              const gmapp_workspace *ws, uint32_t *index, size_t index_bytes,
                              gmapp_stream stream);

/* rollout_agents (MFI field) visiting only the obstacles within each
 * agent's reach r_d + r_a + r_O: the grid rows around the agent give index
 * ranges of S_W through `index` (gmapp_grid_index of the same obstacles and
 * grid).  Alg. 1's gate makes every farther pair contribute nothing, so W,
 * the force and the trajectory are those of rollout_agents (FP32 sums in
 * another order).  The clearance m_k is exact when the nearest obstacle is
 * within the reach, else the smallest distance among the visited obstacles
 * (at least r_d) or +inf when none was visited; clear_pen and min_clear
 * follow it.  Every r_d must be finite (an agent without a gate sets
 * GMAPP_DEVERR_BOUNDS and its outputs are not written).  One CTA of 128
 * threads per agent.  traj, p_final, v_final, path_len, clear_pen,
 * min_clear, w_trace, m_trace as in rollout_agents; checkpoints, f_trace
 * and cost_terms must be NULL (GMAPP_ERR_INVALID_ARG). */
gmapp_status rollout_agents_culled(gmapp_ctx *ctx, const gmapp_obstacles *obs,
                                   const gmapp_workspace *ws, const uint32_t *index,
                                   const gmapp_agents *agents, const gmapp_rollout_params *prm,
                                   gmapp_rollout_out *out, gmapp_stream stream);

/* ------------------------------------------------------------------------ */
/* Cost and selection: score_and_select (Sec. IV-A "Cost Functions" and        */
/* "Selection Mechanism"; gmapp_cost_weights is declared above)               */
/* ------------------------------------------------------------------------ */

/* C_i = w_path L_i + w_goal |p_i(N_k) - p_goal| + w_clear pen_i for every
 * agent, then i* = argmin_i C_i with ties to the lowest index.  With a
 * previous best cost (prev_best_cost not NaN) only agents with
 * C_i < alpha * prev_best_cost qualify and i* = -1 when none does (keep the
 * previous path).  Reads ro->p_final, path_len and, when w_clear != 0,
 * clear_pen (device; NULL counts as zero penalty when w_clear == 0).
 *   costs      device [n_agents] float32 (written)
 *   best       device, one int32 (written)
 *   best_traj  device [(n_steps+1) * 3] float32: the selected agent's
 *              trajectory copied from ro->traj (needs ro->traj), or NULL.
 *              Left untouched when i* = -1. */
gmapp_status score_and_select(gmapp_ctx *ctx, const gmapp_rollout_out *ro,
                              int32_t n_agents, const gmapp_rollout_params *prm,
                              const gmapp_cost_weights *w, float prev_best_cost,
                              float alpha, float *costs, int32_t *best,
                              float *best_traj, gmapp_stream stream);

/* Weights of the paper's four-term cost (Eq. cost_function). */
typedef struct {
    float w_goal;   /* w_1: goal distance term, Eq. (cost_goal) */
    float w_obs;    /* w_2: obstacle distance term, Eq. (cost_obs) */
    float w_path;   /* w_3: path length term, Eq. (cost_path) */
    float w_smooth; /* w_4: smoothness term, Eq. (cost_smooth) */
    float a_max;    /* maximum acceleration (m/s^2) normalising the jerk, > 0 */
} gmapp_cost4;

/* The paper's cost C_i = w_1 C_goal + w_2 C_obs + w_3 C_path + w_4 C_smooth
 * (Sec. IV-A "Cost Functions") from the sums a rollout wrote to
 * ro->cost_terms (see gmapp_rollout_out), with N_k = prm->n_steps:
 *   C_goal = S_goal / N_k,  C_obs = S_obs / N_k,
 *   C_path = 1 - d1 / L if L >= d1, else 1 - L / d1 (0 when L = d1 = 0),
 *   C_smooth = min(1, J / (N_k dt^4 a_max^2)),
 * then the selection of "Selection Mechanism": i* = argmin {C_i : C_i <
 * alpha C_best} with ties to the lowest index.  C_best is the cost of the
 * plan currently followed, kept on the device so a re-planning loop needs
 * no host round trip:
 *   c_best     device, one float32, in/out, or NULL.  NaN (or NULL) = no
 *              current plan: plain argmin over the agents with a finite
 *              cost.  When an agent is selected, *c_best becomes its cost;
 *              when none qualifies, *best = -1 and *c_best is unchanged
 *              (the caller keeps following the previous plan).
 *   costs, best, best_traj  as in score_and_select.
 * GMAPP_ERR_INVALID_ARG when ro->cost_terms is NULL, a weight or alpha is
 * not finite, or a_max <= 0. */
gmapp_status score_and_select4(gmapp_ctx *ctx, const gmapp_rollout_out *ro,
                               int32_t n_agents, const gmapp_rollout_params *prm,
                               const gmapp_cost4 *w, float *c_best, float alpha,
                               float *costs, int32_t *best, float *best_traj,
                               gmapp_stream stream);

/* ------------------------------------------------------------------------ */
/* Batched uneven queries: rollout_batch (the perception -> rollout -> select */
/* query of Sec. IV for many scenes at once; the paper launches one force     */
/* kernel per agent per step, Alg. 1 and Sec. IV-D)                           */
/* ------------------------------------------------------------------------ */

/* One planning query: its cloud and grid, its agents and constants, and the
 * device buffers its results go to (all owned by the caller). */
typedef struct {
    const float *xyz;         /* device, n_raw x 3 camera-frame points, 16-byte aligned */
    int64_t n_raw;
    float T[12];              /* camera-to-world, row-major 3x4 */
    gmapp_workspace ws;       /* voxel grid; min_pts must be 1 in a batch */
    gmapp_agents agents;      /* device agent arrays */
    gmapp_rollout_params prm; /* per-query horizon, goal and constants */
    gmapp_cost_weights w;
    gmapp_obstacles obs;      /* S_W buffers of this query (cap >= 4, multiple of 4) */
    gmapp_rollout_out out;    /* p_final, v_final, path_len required; traj,
                                 clear_pen, min_clear, cost_terms optional; traces
                                 and checkpoints are not produced in a batch.  With
                                 cost_terms set, the query is scored by the paper's
                                 four-term cost (as score_and_select4, with w4, alpha
                                 and c_best below; prm.cost_radius > 0) instead of w */
    float *costs;             /* device [N_a] */
    int32_t *best;            /* device [1] */
    float *best_traj;         /* device [(n_steps+1)*3] or NULL */
    gmapp_cost4 w4;           /* four-term weights (with out.cost_terms) */
    float alpha;              /* hysteresis of the four-term selection */
    float *c_best;            /* device float32 C_best of the query's plan (in/out; NaN = none),
                                 or NULL (plain argmin); the queries of one batch are scored
                                 concurrently, so each needs its own word */
} gmapp_query;

typedef struct gmapp_batch gmapp_batch;

/* Prepare a batch of n_q queries: validates every query, uploads a device
 * descriptor table and allocates the queue and the filter scratch of all
 * queries (the only allocations; runs allocate nothing).  The query
 * buffers are bound by address: refill them between runs.  Each work item
 * keeps up to about 18.9k obstacles of its query in one CTA's shared memory;
 * a larger obstacle set has its remainder read from L2 every step.
 * Default tuning: 8 agents per work item, 256 threads. */
gmapp_status gmapp_batch_create(gmapp_ctx *ctx, const gmapp_query *queries, int32_t n_q,
                                gmapp_batch **out);
void gmapp_batch_destroy(gmapp_batch *batch);

/* Work-item size (agents per item: 2, 4, 6, 8, 12 or 16) and threads per CTA
 * (256, 384, 512) of the persistent rollout kernel.  Discards a captured
 * graph. */
gmapp_status gmapp_batch_set_tuning(gmapp_batch *batch, int32_t agents_per_item,
                                    int32_t threads);

/* on != 0: block culling in the persistent rollout kernel -- a work item's
 * agents visit only the resident blocks of 128 obstacles whose bounding box
 * meets one of their gates (as rollout_agents_blockcull); results equal the
 * unculled batch's bit for bit, except the clearance, which then comes from
 * the visited obstacles (as for rollout_agents_blockcull).  Discards a
 * captured graph. */
gmapp_status gmapp_batch_set_culling(gmapp_batch *batch, int32_t on);

/* Enqueue the whole batch on `stream`: batched filter (5 launches over all
 * queries), the planner (N_O of every query, work items ordered by cost,
 * largest first), ONE persistent rollout launch whose CTAs pop
 * (query, agent group) items from a device queue, and a batched
 * score/select (one CTA per query).  Results equal running each query alone
 * with the same work-item size, bit for bit: each item's arithmetic depends
 * only on its own query. */
gmapp_status rollout_batch(gmapp_batch *batch, gmapp_stream stream);

/* Same as rollout_batch through a CUDA graph: the first call captures the
 * sequence on `stream` (which must not be the legacy default stream), later
 * calls replay it. */
gmapp_status gmapp_batch_launch_graph(gmapp_batch *batch, gmapp_stream stream);

/* Autotuner of the work-item size and thread count: times every supported
 * (agents per item, threads) pair on the batch's own inputs (one warm-up
 * and one timed run each, CUDA events on `stream`), keeps the fastest.
 * Synchronous.  best->cluster is 1. */
gmapp_status gmapp_batch_autotune(gmapp_batch *batch, gmapp_stream stream, gmapp_tuning *best,
                                  float *best_ms);

/* ------------------------------------------------------------------------ */
/* Served control loop with continuous batching (the planning thread of       */
/* Sec. V-B answers a query per control cycle; here requests overlap)         */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t max_slots;       /* requests resident at once */
    int32_t max_agents;      /* largest N_a of a request */
    int32_t max_steps;       /* largest N_k of a request */
    int64_t obs_cap;         /* obstacle capacity of one request (multiple of 4) */
    int64_t arena_bytes;     /* device memory for admitted requests (allocated once) */
    int32_t chunk_steps;     /* M: steps every active request advances per tick */
    int32_t agents_per_item; /* work-item size of the chunk kernel: 4, 8 or 16 */
    int32_t threads;         /* threads per CTA: 256, 384 or 512 */
    int32_t culled;          /* 1: every agent visits only the obstacles within its reach
                                r_d + r_a + r_O (the voxel grid as a neighbour grid, as in
                                rollout_agents_culled; one agent per work item, 128 threads;
                                agents_per_item and threads are then unused and every r_d
                                must be finite); 2: block culling in the chunk kernel (a
                                work item's agents visit only the resident blocks of 128
                                obstacles whose bounding box meets a gate, as in
                                rollout_agents_blockcull; results equal culled = 0 bit for
                                bit); 0: all pairs */
    int32_t admit_bypass;    /* aging bound of the admission: 0 admits queued requests in
                                arrival order, stopping at the first that does not fit;
                                k > 0 admits first fit over the whole queue (a request that
                                fits is admitted although an older one does not), but once
                                the oldest queued request has been overtaken k times, no
                                later request is admitted before it */
    int32_t four_term;       /* 1: the chunk kernel also computes the clearance and the
                                sums of the paper's four-term cost (Eq. cost_function), so
                                requests may ask for cost_mode 1 (slower pair loop: the
                                exact distance of every pair); 0: plain cost only.  With
                                culled = 1 or 2 the obstacle term uses the culled clearance
                                (exact within an agent's reach r_d + r_a + r_O) */
    int32_t max_plan_streams; /* with four_term: number of request streams whose current plan
                                cost C_best the server keeps on the device (Sec. IV-A
                                "Selection Mechanism"); 0 = none */
} gmapp_server_config;

/* A request: HOST cloud and agent arrays (kept alive, unmodified, by the
 * caller until the request is done; pinned memory lets the copies run
 * asynchronously), the grid and the rollout constants. */
typedef struct {
    const float *xyz; /* host, n_raw x 3 camera-frame points */
    int64_t n_raw;
    float T[12];
    gmapp_workspace ws;
    const float *p0, *v0, *c;                /* host [3][n_agents] */
    const float *k_r, *k_a, *r_d, *r_a;      /* host [n_agents] */
    int32_t n_agents;
    gmapp_rollout_params prm;
    gmapp_cost_weights w;    /* cost_mode 0: the weighted cost of score_and_select */
    int32_t cost_mode;       /* 0: score_and_select with w (plain argmin); 1: the paper's
                                four-term cost with w4 and the selection against C_best, as
                                score_and_select4 (needs a four_term server and
                                prm.cost_radius > 0) */
    gmapp_cost4 w4;          /* cost_mode 1: weights of the four terms */
    float alpha;             /* cost_mode 1: hysteresis factor of the selection */
    int32_t plan_stream;     /* cost_mode 1: the request stream (0 <= s < max_plan_streams)
                                whose C_best the selection compares against and updates;
                                requests of one stream are scored in the order they were
                                submitted.  -1: no current plan (plain argmin) */
} gmapp_request;

typedef struct {
    int32_t done;
    int32_t best;          /* selected agent i*; -1 when, with cost_mode 1 and a current plan,
                              no agent is cheaper than alpha C_best (keep following the
                              current plan; best_traj is then undefined) */
    float best_cost;
    int32_t n_obs;         /* N_O of the request's S_W */
    const float *best_traj; /* host [(n_steps+1)*3], valid until release */
    const float *costs;     /* host [n_agents], valid until release */
    double t_submit, t_admit, t_done; /* host steady clock, seconds */
} gmapp_result;

typedef struct {
    int32_t active, pending;
    int64_t completed;
    int64_t arena_free_bytes;
    int32_t shard_cap;     /* obstacles one CTA keeps in shared memory */
} gmapp_server_stats_t;

typedef struct gmapp_server gmapp_server;

/* Create a server: one device arena, a compute and a copy stream, a queue of
 * work items and pinned result staging per slot -- all allocated here;
 * submit/tick/poll allocate no device memory. */
gmapp_status gmapp_server_create(gmapp_ctx *ctx, const gmapp_server_config *cfg,
                                 gmapp_server **out);
void gmapp_server_destroy(gmapp_server *server);

/* Queue a request (returns at once with a ticket).  GMAPP_ERR_CAPACITY when
 * the request can never fit the arena. */
gmapp_status gmapp_server_submit(gmapp_server *server, const gmapp_request *req,
                                 int64_t *ticket);

/* One scheduling round: waits for the previous round's chunk, retires
 * requests whose plan reached host memory (freeing their bytes), admits
 * queued requests while their bytes fit (in arrival order, or first fit
 * with the aging bound admit_bypass; H2D copies on the copy stream,
 * filter_cloud on the compute stream), advances every active request by up
 * to chunk_steps steps in ONE persistent launch over (request, agent group)
 * items, and scores the requests that reached their horizon
 * (score_and_select, or score_and_select4 against the request stream's
 * C_best, then D2H of i*, the costs and the chosen trajectory).  *n_active
 * (may be NULL) receives the active count. */
gmapp_status gmapp_server_tick(gmapp_server *server, int32_t *n_active);

/* Result of a request: GMAPP_ERR_NOT_READY until done.  Identical bit for
 * bit whether the request ran alone or together with any others. */
gmapp_status gmapp_server_poll(gmapp_server *server, int64_t ticket, gmapp_result *res);

/* Forget a finished request (its result pointers become invalid). */
gmapp_status gmapp_server_release(gmapp_server *server, int64_t ticket);

gmapp_status gmapp_server_stats(gmapp_server *server, gmapp_server_stats_t *out);

#ifdef __cplusplus
}
#endif

#endif /* GMAPP_H */

// rollout_agents: host side -- argument checks, launch shapes, launch.
// The kernel itself is in rollout_kernel.cuh (Sec. IV-A, Eq. (mfi), Alg. 1).
#include <math.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "rollout_kernel.cuh"

namespace gmapp {

namespace {

// Agent kinds of a heterogeneous ensemble (agents ordered MFI, projected
// current, APF); all zero for a plain MFI rollout.
struct Kinds {
    int n_proj = 0, n_apf = 0;
    // ensemble level of the kernel: 0 MFI only, 1 + APF, 2 + projected current
    int level() const { return n_proj > 0 ? 2 : n_apf > 0 ? 1 : 0; }
};

// A launch shape resolved for concrete sizes.
struct Shape {
    int cluster;   // C: CTAs per group (a cluster, or a grid-exchange group) = obstacle shards
    int groups;    // G: agent groups
    bool grid;     // exchange through global memory in a cooperative grid
    int ag;        // agents per group held in registers (max over groups)
    int threads;   // NT
    bool clear;    // clearance reduction compiled in
    Kinds kinds;   // heterogeneous ensemble (all zero: MFI only)
    int groups_proj, groups_apf;  // groups of projected-current and APF agents
    RolloutKernel fn;
    int32_t shard_cap;
    size_t smem;   // dynamic shared memory bytes
};

int32_t shard_cap_for(int64_t cap, int cluster) {
    // a multiple of 128: the pair loop pads every shard to whole 128-obstacle blocks
    int64_t s = (cap + cluster - 1) / cluster;
    return static_cast<int32_t>((s + 127) & ~int64_t(127));
}

RolloutKernel pick_kernel(int ag, int nt, bool clear, bool grid, int level) {
    if (level == 2) {
        if (grid) return clear ? rollout_kernel_ens3_grid_clear(ag, nt) : rollout_kernel_ens3_grid_noclear(ag, nt);
        return clear ? rollout_kernel_ens3_clear(ag, nt) : rollout_kernel_ens3_noclear(ag, nt);
    }
    if (level == 1) {
        if (grid) return clear ? rollout_kernel_ens_grid_clear(ag, nt) : rollout_kernel_ens_grid_noclear(ag, nt);
        return clear ? rollout_kernel_ens_clear(ag, nt) : rollout_kernel_ens_noclear(ag, nt);
    }
    if (grid) return clear ? rollout_kernel_grid_clear(ag, nt) : rollout_kernel_grid_noclear(ag, nt);
    return clear ? rollout_kernel_clear(ag, nt) : rollout_kernel_noclear(ag, nt);
}

size_t static_smem(RolloutKernel fn) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, reinterpret_cast<const void *>(fn)) != cudaSuccess) return ~size_t(0);
    return fa.sharedSizeBytes;
}

// Groups per kind of an ensemble: in proportion to the agent counts, at
// least one per kind present, the remainder to the kinds with the most
// agents per group; returns the largest number of agents in a group.
int split_groups(const int (&count)[3], int groups, int (&g)[3]) {
    int sum = 0, total = count[0] + count[1] + count[2];
    for (int i = 0; i < 3; ++i) {
        g[i] = count[i] > 0 ? std::max(1, static_cast<int>(static_cast<int64_t>(groups) *
                                                           count[i] / total)) : 0;
        sum += g[i];
    }
    auto per = [&](int i) { return g[i] > 0 ? (count[i] + g[i] - 1) / g[i] : 0; };
    while (sum > groups) {  // only when a small kind got its one group
        int j = -1;
        for (int i = 0; i < 3; ++i)
            if (g[i] > 1 && (j < 0 || per(i) < per(j))) j = i;
        if (j < 0) break;
        --g[j];
        --sum;
    }
    while (sum < groups) {
        int j = -1;
        for (int i = 0; i < 3; ++i)
            if (count[i] > g[i] && (j < 0 || per(i) > per(j))) j = i;
        if (j < 0) break;
        ++g[j];
        ++sum;
    }
    return std::max(per(0), std::max(per(1), per(2)));
}

// Resolve (cluster, agents per group, threads) for N_a agents and an
// obstacle capacity; false when the shape cannot run.  For an ensemble the
// groups are split by heuristic (homogeneous groups; split_groups) and the
// ensemble kernel of the matching level is used.
bool resolve(gmapp_ctx *ctx, int64_t cap, int n_agents, const gmapp_tuning &t, bool clear,
             Shape *s, Kinds kinds = Kinds{}) {
    if (t.cluster < 1 || t.cluster > kMaxCluster || t.agents_per_cta < 1 ||
        t.agents_per_cta > kMaxAgents || t.exchange < 0 || t.exchange > 1)
        return false;
    s->cluster = t.cluster;
    s->grid = t.exchange == 1;
    s->threads = t.threads;
    s->groups = (n_agents + t.agents_per_cta - 1) / t.agents_per_cta;
    s->ag = (n_agents + s->groups - 1) / s->groups;
    s->clear = clear;
    s->kinds = kinds;
    s->groups_proj = s->groups_apf = 0;
    if (kinds.level() > 0) {
        const int count[3] = {n_agents - kinds.n_proj - kinds.n_apf, kinds.n_proj, kinds.n_apf};
        const int present = (count[0] > 0) + (count[1] > 0) + (count[2] > 0);
        if (s->groups < present) s->groups = present;
        int g[3];
        s->ag = split_groups(count, s->groups, g);
        s->groups_proj = g[1];
        s->groups_apf = g[2];
        if (s->ag > kMaxEnsembleAgents) return false;
    }
    s->fn = pick_kernel(s->ag, t.threads, clear, s->grid, kinds.level());
    if (!s->fn) return false;
    // grid exchange: one slot set per CTA, at most one CTA per SM
    if (s->grid && s->groups * s->cluster > ctx->sm_count) return false;
    s->shard_cap = shard_cap_for(cap, t.cluster);
    const int nw = t.threads / 32;
    // shard + per-warp partials [2][NW][AG] + cluster slots [2][2][C][AG] of
    // one record each ((W, min d^2); APF (f, min d^2): 4 floats; projected
    // current (S, B, min d^2, -): 6) + agent positions and velocities [3][AG]
    // each (4 AG floats apart, keeping the 16-byte alignment) + the
    // four-term cost sums [kCostAcc][AG]
    const size_t rec = kinds.level() == 2 ? 6 : kinds.level() == 1 ? 4 : 2;
    // + the per-block bounding boxes of the shard [shard_cap / 128][6]
    s->smem = (static_cast<size_t>(s->shard_cap) * 3 + 2 * rec * nw * s->ag +
               4 * rec * t.cluster * s->ag + static_cast<size_t>(8 + kCostAcc) * s->ag +
               6 * static_cast<size_t>(s->shard_cap / 128)) *
              sizeof(float);
    return s->smem + static_smem(s->fn) <= static_cast<size_t>(ctx->max_smem_optin);
}

gmapp_status prepare(const Shape &s) {
    GMAPP_CHECK_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void *>(s.fn),
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          static_cast<int>(s.smem)));
    if (s.cluster > 8)
        GMAPP_CHECK_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void *>(s.fn),
                                              cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    return GMAPP_OK;
}

cudaLaunchConfig_t config(const Shape &s, cudaLaunchAttribute *attr, gmapp_stream stream) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(s.groups * s.cluster, 1, 1);
    cfg.blockDim = dim3(s.threads + 32 * kExchWarps, 1, 1);  // compute + exchange warps
    cfg.dynamicSmemBytes = s.smem;
    cfg.stream = stream;
    if (s.grid) {
        // every CTA co-resident: groups poll one another
        attr->id = cudaLaunchAttributeCooperative;
        attr->val.cooperative = 1;
    } else {
        attr->id = cudaLaunchAttributeClusterDimension;
        attr->val.clusterDim.x = s.cluster;
        attr->val.clusterDim.y = 1;
        attr->val.clusterDim.z = 1;
    }
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// Co-resident groups of this shape (0 when it cannot be placed).
int max_active_clusters(gmapp_ctx *ctx, const Shape &s) {
    if (prepare(s) != GMAPP_OK) return 0;
    int m = 0;
    if (s.grid) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reinterpret_cast<const void *>(s.fn),
                                                          s.threads + 32 * kExchWarps, s.smem) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return std::min(per_sm, 1) * ctx->sm_count / s.cluster;
    }
    cudaLaunchAttribute attr;
    cudaLaunchConfig_t cfg = config(s, &attr, nullptr);
    if (cudaOccupancyMaxActiveClusters(&m, reinterpret_cast<const void *>(s.fn), &cfg) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return m;
}

// Cost model in SM cycles for one step of the rollout: the slowest CTA
// evaluates ag x shard pairs at ~7 pairs/clk (measured on B300 for 9-10
// agents; fewer with few agents in flight).  The exchange warp hides the
// per-step exchange behind the pair loop of the other agent half, so a step
// costs the larger of the pair loop and the exchange latency chain (~3000
// cycles over DSMEM, ~4700 through L2 for the grid exchange); cluster
// groups beyond the co-resident count run in later waves, a grid-exchange
// launch must fit in one wave (its groups poll one another).
// CTAs that share an SM (when the occupancy allows more than one) share its
// pipes, so the pair loop slows by the number of co-resident CTAs per SM.
// In an ensemble every group runs AG agent slots and the costliest kind sets
// the pace: an APF pair costs ~1.32 MFI pairs (measured on B300, tabletop),
// a projected-current pair ~1.6 (17 FMA-pipe lane-ops and 2 SFU ops).
double model_cost(const Shape &s, int m, int64_t n_obs_est, int sm_count) {
    const double shard = static_cast<double>((n_obs_est + s.cluster - 1) / s.cluster);
    const double rate = std::min(7.0, 1.5 + 1.2 * s.ag) * (s.threads >= 384 ? 1.0 : 0.95) /
                        (s.kinds.n_proj > 0 ? 1.6 : s.kinds.n_apf > 0 ? 1.32 : 1.0);
    const double share =
        std::max(1.0, static_cast<double>(std::min(s.groups, m)) * s.cluster / sm_count);
    const double loop = s.ag * std::max(shard, 64.0) / rate * share;
    const double chain = (s.grid ? 4700.0 : 3000.0) + 20.0 * s.cluster;
    if (s.grid && s.groups > m) return 1e300;
    const int waves = (s.groups + m - 1) / m;
    return waves * (std::max(loop, chain) + 0.1 * std::min(loop, chain));
}

std::mutex g_tune_mu;
// (device, obstacle capacity, N_a, clearance outputs, projected-current and
// APF agents of an ensemble)
std::map<std::tuple<int, int64_t, int, bool, int, int>, gmapp_tuning> g_tune_cache;

}  // namespace

gmapp_status pick_tuning_impl(gmapp_ctx *ctx, int64_t cap, int32_t n_agents, bool clear,
                              gmapp_tuning *best, Kinds kinds = Kinds{}) {
    const auto key = std::make_tuple(ctx->device, cap, n_agents, clear, kinds.n_proj, kinds.n_apf);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *best = it->second;
            return GMAPP_OK;
        }
    }
    double best_cost = 1e300;
    bool found = false;
    const int threads_list[] = {256, 384, 512};
    for (int x = 0; x <= 1; ++x)
        for (int C = 1; C <= kMaxCluster; ++C) {
            for (int nt : threads_list) {
                int last_groups = -1;
                for (int a = 1; a <= kMaxAgents; ++a) {
                    Shape s;
                    if (!resolve(ctx, cap, n_agents, gmapp_tuning{C, a, nt, x}, clear, &s, kinds))
                        continue;
                    if (s.groups == last_groups) continue;
                    last_groups = s.groups;
                    const int m = max_active_clusters(ctx, s);
                    if (m <= 0) continue;
                    const double cost = model_cost(s, m, cap, ctx->sm_count);
                    if (cost < best_cost) {
                        best_cost = cost;
                        *best = gmapp_tuning{C, kinds.level() > 0 ? a : s.ag, nt, x};
                        found = true;
                    }
                }
            }
        }
    if (!found) {
        set_error("rollout_agents: no launch shape fits an obstacle capacity of %lld",
                  (long long)cap);
        return GMAPP_ERR_CAPACITY;
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = *best;
    return GMAPP_OK;
}

namespace {

gmapp_status validate(const gmapp_obstacles *obs, const gmapp_agents *ag,
                      const gmapp_rollout_params *prm, const gmapp_rollout_out *out) {
    if (!obs || !ag || !prm || !out) {
        set_error("rollout_agents: NULL argument");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (!obs->x || !obs->y || !obs->z || !obs->n || obs->cap < 0 || obs->cap % 4 ||
        obs->cap > (int64_t(1) << 30)) {
        set_error("rollout_agents: obstacle arrays must be set, cap a multiple of 4");
        return GMAPP_ERR_INVALID_ARG;
    }
    if ((reinterpret_cast<uintptr_t>(obs->x) | reinterpret_cast<uintptr_t>(obs->y) |
         reinterpret_cast<uintptr_t>(obs->z)) % 16) {
        set_error("rollout_agents: obstacle arrays must be 16-byte aligned");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (!(obs->r_O >= 0.0f) || !isfinite(obs->r_O)) {
        set_error("rollout_agents: r_O must be finite and >= 0");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (ag->n < 1 || !ag->p0 || !ag->v0 || !ag->c || !ag->k_r || !ag->k_a || !ag->r_d || !ag->r_a) {
        set_error("rollout_agents: agent arrays must be set and n >= 1");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (prm->n_steps < 1 || !(prm->dt > 0.0f) || !isfinite(prm->dt) || !(prm->eps > 0.0f) ||
        !isfinite(prm->eps) || !(prm->clear_beta > 0.0f) || !isfinite(prm->damping) ||
        !isfinite(prm->inv_mass) || !isfinite(prm->rho) || !isfinite(prm->vel_half) ||
        !isfinite(prm->clear_margin) || !isfinite(prm->goal[0]) || !isfinite(prm->goal[1]) ||
        !isfinite(prm->goal[2]) || prm->ckpt_every < 0) {
        set_error("rollout_agents: invalid rollout parameters (n_steps >= 1, dt > 0, eps > 0, "
                  "clear_beta > 0, all finite)");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (!out->p_final || !out->v_final || !out->path_len) {
        set_error("rollout_agents: p_final, v_final and path_len are required");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (out->ckpt && prm->ckpt_every < 1) {
        set_error("rollout_agents: checkpoints need ckpt_every >= 1");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (out->cost_terms && !(prm->cost_radius > 0.0f && isfinite(prm->cost_radius))) {
        set_error("rollout_agents: cost_terms need a finite cost_radius > 0");
        return GMAPP_ERR_INVALID_ARG;
    }
    return GMAPP_OK;
}

bool wants_clear(const gmapp_rollout_out *out) {
    return out->clear_pen || out->min_clear || out->m_trace || out->cost_terms;
}

gmapp_status launch(gmapp_ctx *ctx, const gmapp_obstacles *obs, const gmapp_agents *ag,
                    const gmapp_rollout_params *prm, gmapp_rollout_out *out,
                    const gmapp_tuning &t, gmapp_stream stream, Kinds kinds = Kinds{},
                    bool box_cull = false) {
    Shape s;
    if (!resolve(ctx, obs->cap, ag->n, t, wants_clear(out), &s, kinds)) {
        set_error("rollout_agents: launch shape (cluster %d, agents %d, threads %d, exchange %d) "
                  "does not fit an obstacle capacity of %lld",
                  t.cluster, t.agents_per_cta, t.threads, t.exchange, (long long)obs->cap);
        return GMAPP_ERR_INVALID_ARG;
    }
    gmapp_status st = prepare(s);
    if (st != GMAPP_OK) return st;
    RolloutArgs A;
    A.ox = obs->x;
    A.oy = obs->y;
    A.oz = obs->z;
    A.n_obs = obs->n;
    A.cap = obs->cap;
    A.r_O = obs->r_O;
    A.p0 = ag->p0;
    A.v0 = ag->v0;
    A.c = ag->c;
    A.k_r = ag->k_r;
    A.k_a = ag->k_a;
    A.r_d = ag->r_d;
    A.r_a = ag->r_a;
    A.n_agents = ag->n;
    for (int d = 0; d < 3; ++d) A.goal[d] = prm->goal[d];
    A.dt = prm->dt;
    A.n_steps = prm->n_steps;
    A.damping = prm->damping;
    A.inv_mass = prm->inv_mass;
    A.rho = prm->rho;
    A.eps = prm->eps;
    A.vel_half = prm->vel_half;
    A.clear_margin = prm->clear_margin;
    A.clear_beta = prm->clear_beta;
    A.ckpt_every = prm->ckpt_every;
    A.traj = out->traj;
    A.p_final = out->p_final;
    A.v_final = out->v_final;
    A.path_len = out->path_len;
    A.clear_pen = out->clear_pen;
    A.min_clear = out->min_clear;
    A.w_trace = out->w_trace;
    A.m_trace = out->m_trace;
    A.f_trace = out->f_trace;
    A.ckpt = out->ckpt;
    A.cost_terms = out->cost_terms;
    A.heur_pairs = out->heur_pairs;
    A.xbuf_words = static_cast<int64_t>(xbuf_bytes(ctx->sm_count) / sizeof(uint64_t));
    A.box_cull = box_cull ? 1 : 0;
    A.cost_radius = prm->cost_radius;
    A.shard_cap = s.shard_cap;
    A.n_groups = s.groups;
    A.n_apf = s.kinds.n_apf;
    A.n_groups_apf = s.groups_apf;
    A.n_proj = s.kinds.n_proj;
    A.n_groups_proj = s.groups_proj;
    A.group_ctas = s.cluster;
    A.xbuf = ctx->d_xbuf;
    A.xctl = ctx->d_xctl;
    // the test knob caps only the grid-exchange polls (global-memory words,
    // nothing in flight into shared memory when a CTA gives up); mbarrier
    // waits (TMA copies, DSMEM deliveries) keep their full bound
    A.spin_limit = kSpinLimit;
    A.poll_limit = ctx->wait_limit ? ctx->wait_limit : kPollLimit;
    A.err = ctx->d_err;
    cudaLaunchAttribute attr;
    cudaLaunchConfig_t cfg = config(s, &attr, stream);
    if (!s.grid) {
        GMAPP_CHECK_CUDA(cudaLaunchKernelEx(&cfg, s.fn, A));
        return GMAPP_OK;
    }
    // the grid exchange uses the context's slots and epoch
    bool capturing = false;
    st = grid_exchange_begin(ctx, stream, &capturing);
    if (st != GMAPP_OK) return st;
    GMAPP_CHECK_CUDA(cudaLaunchKernelEx(&cfg, s.fn, A));
    return grid_exchange_end(ctx, stream, capturing);
}

}  // namespace
}  // namespace gmapp

using namespace gmapp;

namespace {

// Checks of an ensemble's agent counts (the kinds are ordered MFI,
// projected current, APF; the adjoint covers MFI agents only).
gmapp_status check_kinds(const char *who, const gmapp_agents *agents, int32_t n_proj,
                         int32_t n_apf, const gmapp_rollout_out *out) {
    if (n_proj < 0 || n_apf < 0 || static_cast<int64_t>(n_proj) + n_apf > agents->n) {
        set_error("%s: n_proj, n_apf must be >= 0 with n_proj + n_apf <= n (%d, %d, n %d)", who,
                  n_proj, n_apf, agents->n);
        return GMAPP_ERR_INVALID_ARG;
    }
    if (n_proj + n_apf > 0 && out->ckpt) {
        set_error("%s: adjoint checkpoints cover MFI agents only", who);
        return GMAPP_ERR_INVALID_ARG;
    }
    return GMAPP_OK;
}

// Measured choice of the launch shape (MFI rollout, or an ensemble): rank
// by the model, time the best candidates on the caller's inputs, cache the
// fastest.
gmapp_status autotune_impl(gmapp_ctx *ctx, const gmapp_obstacles *obs, const gmapp_agents *agents,
                           Kinds kinds, const gmapp_rollout_params *prm,
                           gmapp_rollout_out *out, int32_t max_candidates, int32_t probe_steps,
                           gmapp_tuning *best, float *best_ms, gmapp_stream stream) {
    if (!ctx || !best || max_candidates < 1 || probe_steps < 1) {
        set_error("gmapp_autotune_rollout: invalid argument");
        return GMAPP_ERR_INVALID_ARG;
    }
    gmapp_status st = validate(obs, agents, prm, out);
    if (st != GMAPP_OK) return st;
    if ((st = check_kinds("gmapp_autotune_ensemble", agents, kinds.n_proj, kinds.n_apf, out)) !=
        GMAPP_OK)
        return st;
    const bool clear = wants_clear(out);
    // 1. candidates ranked by the model, one per (cluster, groups, threads)
    struct Cand {
        double cost;
        gmapp_tuning t;
    };
    std::vector<Cand> cands;
    const int threads_list[] = {256, 384, 512};
    for (int x = 0; x <= 1; ++x)
        for (int C = 1; C <= kMaxCluster; ++C)
            for (int nt : threads_list) {
                int last_groups = -1;
                for (int a = 1; a <= kMaxAgents; ++a) {
                    Shape s;
                    if (!resolve(ctx, obs->cap, agents->n, gmapp_tuning{C, a, nt, x}, clear, &s,
                                 kinds))
                        continue;
                    if (s.groups == last_groups) continue;
                    last_groups = s.groups;
                    const int m = max_active_clusters(ctx, s);
                    if (m <= 0) continue;
                    const double cost = model_cost(s, m, obs->cap, ctx->sm_count);
                    if (cost < 1e299)
                        cands.push_back({cost, gmapp_tuning{C, kinds.level() > 0 ? a : s.ag, nt, x}});
                }
            }
    if (cands.empty()) {
        set_error("gmapp_autotune_rollout: no launch shape fits an obstacle capacity of %lld",
                  (long long)obs->cap);
        return GMAPP_ERR_CAPACITY;
    }
    std::sort(cands.begin(), cands.end(),
              [](const Cand &x, const Cand &y) { return x.cost < y.cost; });
    if (static_cast<int>(cands.size()) > max_candidates) cands.resize(max_candidates);
    // 2. time each on the caller's inputs with a shortened horizon
    gmapp_rollout_params probe = *prm;
    probe.n_steps = std::min(prm->n_steps, probe_steps);
    gmapp_rollout_out probe_out = *out;  // the probes add nothing to the caller's counter
    probe_out.heur_pairs = nullptr;
    cudaEvent_t e0, e1;
    GMAPP_CHECK_CUDA(cudaEventCreate(&e0));
    GMAPP_CHECK_CUDA(cudaEventCreate(&e1));
    float best_t = 1e30f;
    gmapp_status result = GMAPP_OK;
    for (const Cand &c : cands) {
        if ((st = launch(ctx, obs, agents, &probe, &probe_out, c.t, stream, kinds)) != GMAPP_OK)
            continue;
        // the faster of two timed launches (a single one is noisy enough to
        // swap close candidates from call to call)
        float ms = 1e30f;
        for (int rep = 0; rep < 2 && st == GMAPP_OK && result == GMAPP_OK; ++rep) {
            cudaEventRecord(e0, stream);
            st = launch(ctx, obs, agents, &probe, &probe_out, c.t, stream, kinds);
            cudaEventRecord(e1, stream);
            if (st != GMAPP_OK) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                result = cuda_fail(cudaGetLastError(), "gmapp_autotune_rollout");
                break;
            }
            float m = 0.0f;
            cudaEventElapsedTime(&m, e0, e1);
            ms = std::min(ms, m);
        }
        if (result != GMAPP_OK) break;
        if (st != GMAPP_OK) continue;
        if (ms < best_t) {
            best_t = ms;
            *best = c.t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result != GMAPP_OK) return result;
    if (best_t >= 1e30f) {
        set_error("gmapp_autotune_rollout: no candidate launched");
        return GMAPP_ERR_CUDA;
    }
    if (best_ms) *best_ms = best_t * static_cast<float>(prm->n_steps) / probe.n_steps;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[std::make_tuple(ctx->device, obs->cap, agents->n, clear, kinds.n_proj,
                                 kinds.n_apf)] = *best;
    return GMAPP_OK;
}

}  // namespace

extern "C" gmapp_status gmapp_autotune_rollout(gmapp_ctx *ctx, const gmapp_obstacles *obs,
                                               const gmapp_agents *agents,
                                               const gmapp_rollout_params *prm,
                                               gmapp_rollout_out *out, int32_t max_candidates,
                                               int32_t probe_steps, gmapp_tuning *best,
                                               float *best_ms, gmapp_stream stream) {
    return autotune_impl(ctx, obs, agents, Kinds{}, prm, out, max_candidates, probe_steps, best,
                         best_ms, stream);
}

extern "C" gmapp_status gmapp_autotune_ensemble(gmapp_ctx *ctx, const gmapp_obstacles *obs,
                                                const gmapp_agents *agents, int32_t n_proj,
                                                int32_t n_apf,
                                                const gmapp_rollout_params *prm,
                                                gmapp_rollout_out *out, int32_t max_candidates,
                                                int32_t probe_steps, gmapp_tuning *best,
                                                float *best_ms, gmapp_stream stream) {
    return autotune_impl(ctx, obs, agents, Kinds{n_proj, n_apf}, prm, out, max_candidates,
                         probe_steps, best, best_ms, stream);
}

extern "C" gmapp_status gmapp_pick_tuning(gmapp_ctx *ctx, int64_t obs_cap, int32_t n_agents,
                                          gmapp_tuning *tune) {
    if (!ctx || !tune || obs_cap < 0 || n_agents < 1) {
        set_error("gmapp_pick_tuning: invalid argument");
        return GMAPP_ERR_INVALID_ARG;
    }
    return pick_tuning_impl(ctx, obs_cap, n_agents, false, tune);
}

extern "C" gmapp_status rollout_agents_tuned(gmapp_ctx *ctx, const gmapp_obstacles *obs,
                                             const gmapp_agents *agents,
                                             const gmapp_rollout_params *prm,
                                             gmapp_rollout_out *out, const gmapp_tuning *tune,
                                             gmapp_stream stream) {
    if (!ctx || !tune) {
        set_error("rollout_agents_tuned: NULL ctx or tuning");
        return GMAPP_ERR_INVALID_ARG;
    }
    gmapp_status st = validate(obs, agents, prm, out);
    if (st != GMAPP_OK) return st;
    if (!(tune->threads == 128 || tune->threads == 256 || tune->threads == 384 ||
          tune->threads == 512)) {
        set_error("rollout_agents_tuned: threads must be 128, 256, 384 or 512");
        return GMAPP_ERR_INVALID_ARG;
    }
    return launch(ctx, obs, agents, prm, out, *tune, stream);
}

extern "C" gmapp_status rollout_agents(gmapp_ctx *ctx, const gmapp_obstacles *obs,
                                       const gmapp_agents *agents,
                                       const gmapp_rollout_params *prm, gmapp_rollout_out *out,
                                       gmapp_stream stream) {
    if (!ctx) {
        set_error("rollout_agents: NULL ctx");
        return GMAPP_ERR_INVALID_ARG;
    }
    gmapp_status st = validate(obs, agents, prm, out);
    if (st != GMAPP_OK) return st;
    gmapp_tuning t;
    st = pick_tuning_impl(ctx, obs->cap, agents->n, wants_clear(out), &t);
    if (st != GMAPP_OK) return st;
    return launch(ctx, obs, agents, prm, out, t, stream);
}

extern "C" gmapp_status rollout_agents_blockcull(gmapp_ctx *ctx, const gmapp_obstacles *obs,
                                                 const gmapp_agents *agents,
                                                 const gmapp_rollout_params *prm,
                                                 gmapp_rollout_out *out, const gmapp_tuning *tune,
                                                 gmapp_stream stream) {
    if (!ctx) {
        set_error("rollout_agents_blockcull: NULL ctx");
        return GMAPP_ERR_INVALID_ARG;
    }
    gmapp_status st = validate(obs, agents, prm, out);
    if (st != GMAPP_OK) return st;
    gmapp_tuning t;
    if (tune) {
        t = *tune;
    } else if ((st = pick_tuning_impl(ctx, obs->cap, agents->n, wants_clear(out), &t)) != GMAPP_OK) {
        return st;
    }
    return launch(ctx, obs, agents, prm, out, t, stream, Kinds{}, true);
}

namespace {
gmapp_status ensemble_impl(const char *who, gmapp_ctx *ctx, const gmapp_obstacles *obs,
                           const gmapp_agents *agents, int32_t n_proj, int32_t n_apf,
                           const gmapp_rollout_params *prm, gmapp_rollout_out *out,
                           const gmapp_tuning *tune, gmapp_stream stream, bool box_cull) {
    if (!ctx) {
        set_error("%s: NULL ctx", who);
        return GMAPP_ERR_INVALID_ARG;
    }
    gmapp_status st = validate(obs, agents, prm, out);
    if (st != GMAPP_OK) return st;
    if ((st = check_kinds(who, agents, n_proj, n_apf, out)) != GMAPP_OK) return st;
    gmapp_tuning t;
    if (tune) {
        if (!(tune->threads == 128 || tune->threads == 256 || tune->threads == 384 ||
              tune->threads == 512)) {
            set_error("%s: threads must be 128, 256, 384 or 512", who);
            return GMAPP_ERR_INVALID_ARG;
        }
        t = *tune;
    } else {
        st = pick_tuning_impl(ctx, obs->cap, agents->n, wants_clear(out), &t, Kinds{n_proj, n_apf});
        if (st != GMAPP_OK) return st;
    }
    return launch(ctx, obs, agents, prm, out, t, stream, Kinds{n_proj, n_apf}, box_cull);
}
}  // namespace

extern "C" gmapp_status rollout_ensemble(gmapp_ctx *ctx, const gmapp_obstacles *obs,
                                         const gmapp_agents *agents, int32_t n_proj,
                                         int32_t n_apf,
                                         const gmapp_rollout_params *prm, gmapp_rollout_out *out,
                                         const gmapp_tuning *tune, gmapp_stream stream) {
    return ensemble_impl("rollout_ensemble", ctx, obs, agents, n_proj, n_apf, prm, out, tune,
                         stream, false);
}

extern "C" gmapp_status rollout_ensemble_blockcull(gmapp_ctx *ctx, const gmapp_obstacles *obs,
                                                   const gmapp_agents *agents, int32_t n_proj,
                                                   int32_t n_apf,
                                                   const gmapp_rollout_params *prm,
                                                   gmapp_rollout_out *out,
                                                   const gmapp_tuning *tune,
                                                   gmapp_stream stream) {
    return ensemble_impl("rollout_ensemble_blockcull", ctx, obs, agents, n_proj, n_apf, prm, out,
                         tune, stream, true);
}

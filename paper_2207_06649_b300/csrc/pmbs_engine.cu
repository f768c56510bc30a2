// Batched push-rollout engine for PMBS on one B300 (sm_103a): kernels and the C ABI.
//
// A warp runs one environment (a scene copy; Sec. IV-C keeps a fixed pool of N_e parallel
// environments); a persistent grid pulls environments from a device work queue ordered by
// box count, largest first, so that scenes of uneven size share one launch and a warp
// whose environment ends early (target graspable; Sec. IV-C reuses such environments for
// further simulations) takes the next one.  See pmbs.h for the contract of every entry
// point.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <array>
#include <map>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <string>
#include <vector>

#include "../../include/pmbs.h"
#include "pmbs_warp.cuh"

using namespace pmbs;

namespace {

constexpr int kRecFloats = 18;  // scene record per box: state13, half[3], mass, mu
constexpr int kSceneTableCap = 1 << 18;
constexpr int kMaxWarpsPerSM = 32;

// ---- rollout device code begins (the benchmark ties its ncu traffic figure to a hash of
// this section and of the three device headers)
struct SceneDesc {
    const float* rec;
    int n;
    int target;
};

struct EnvIn {
    const float* rec;
    int n;
    int target;
    int box_off;
    int scene;
};

struct EnvProg {
    int k, s, push_ready, done;
    int flags, cost, steps, noop;
    float reward;
    float push[4];
    int pad[3];
};

struct RolloutArgs {
    SimConst C;
    Layout L;
    int G;  // lanes per environment (8, 16 or 32); a warp runs 32 / G environments
    int n_envs, depth, max_substeps, child_on;
    const EnvIn* env;
    const int* order;
    int* queue_head;
    int* done_count;
    const float4* first_push;
    const uint64_t* seeds;
    EnvProg* prog;
    float* state;
    float* child;
    int32_t* cost;
    float* reward;
    uint8_t* flags;
    int32_t* steps;
    unsigned long long* events;
    float4* gscratch;
    int scratch_f4_per_warp;
    long long watchdog_cycles;  // per environment and launch; exceeded -> counters[4] = 1
    int* watchdog_flag;
    float4* warm;               // warm-start caches, warm_f4_per_env per environment (or null)
    size_t warm_f4_per_env;
    unsigned long long* phase;  // [n_envs][kNumPhases] cycles when C.timers (else unused)
    long long n_rows;           // rows of state and child (the bounds-checked build checks row indices)
};

// ------------------------------------------------------------------ device: environments
// Load an environment's state into its group's shared memory (from the scene records when
// it has not started, else from the batch state).  Every lane calls this; groups with
// on = false load nothing.
__device__ __forceinline__ void load_env(const RolloutArgs& a, const WarpMem& W, const EnvIn& ei, bool on,
                                         bool from_scene, const Grp& g) {
    const int NB = W.NB();
    const int n = on ? ei.n : 0;
    for (int i = g.gl; i < n; i += g.G) {
        const float* r = ei.rec + kRecFloats * i;
        const float* s = from_scene ? r : a.state + (size_t)(ei.box_off + i) * 13;
        W.x()[i] = s[0];
        W.x()[NB + i] = s[1];
        W.x()[2 * NB + i] = s[2];
        W.q()[i] = s[3];
        W.q()[NB + i] = s[4];
        W.q()[2 * NB + i] = s[5];
        W.q()[3 * NB + i] = s[6];
        const float h0 = r[13], h1 = r[14], h2 = r[15], m = r[16], mu = r[17];
        W.h()[i] = h0;
        W.h()[NB + i] = h1;
        W.h()[2 * NB + i] = h2;
        W.bv()[i] = make_float4(s[7], s[8], s[9], 1.f / m);
        W.bw()[i] = make_float4(s[10], s[11], s[12], mu);
        const float hx2 = h0 * h0, hy2 = h1 * h1, hz2 = h2 * h2;
        if (h1 < 0.f) {
            // solid cylinder (radius h0, height 2 h2): m (3 r^2 + 4 h^2) / 12 about a
            // diameter, m r^2 / 2 about its axis
            const float id = 1.f / (m * (3.f * hx2 + 4.f * hz2) / 12.f);
            W.ib()[i] = id;
            W.ib()[NB + i] = id;
            W.ib()[2 * NB + i] = 1.f / (m * hx2 / 2.f);
        } else {
            W.ib()[i] = 1.f / (m / 3.f * (hy2 + hz2));
            W.ib()[NB + i] = 1.f / (m / 3.f * (hx2 + hz2));
            W.ib()[2 * NB + i] = 1.f / (m / 3.f * (hx2 + hy2));
        }
    }
    __syncwarp();
}

// Copy an environment's state rows to dst (no collective).
__device__ __forceinline__ void store_state(const WarpMem& W, int n, float* dst, const Grp& g) {
    const int NB = W.NB();
    for (int i = g.gl; i < n; i += g.G) {
        float* s = dst + (size_t)i * 13;
        const float4 v = W.bv()[i], w = W.bw()[i];
        s[0] = W.x()[i];
        s[1] = W.x()[NB + i];
        s[2] = W.x()[2 * NB + i];
        s[3] = W.q()[i];
        s[4] = W.q()[NB + i];
        s[5] = W.q()[2 * NB + i];
        s[6] = W.q()[3 * NB + i];
        s[7] = v.x;
        s[8] = v.y;
        s[9] = v.z;
        s[10] = w.x;
        s[11] = w.y;
        s[12] = w.z;
    }
}

// One substep of the group's environment (on = false: the group only takes part in the
// warp's collectives).  Returns true on a cap overflow.  kWarm compiles the optional warm
// start in (batches without it run an instantiation whose substep body is 15 KB smaller:
// the body is larger than an SM's instruction cache).
template <bool kCyl, bool kWarm>
__device__ __forceinline__ bool substep(const RolloutArgs& a, const WarpMem& W, int n_env, bool on, const Pusher& pu,
                                        int s, const Grp& g, float4* warm, int& warm_n, PhaseClock& pc) {
    const SimConst& C = a.C;
    const int n = on ? n_env : 0;
    const bool tm = C.timers != 0, rec = on && g.gl == 0;
    const int done = s < pu.moving ? s : pu.moving;
    const float travel = (C.pspeed * C.dt) * (float)done;
    const float Px = pu.sx + pu.dx * travel, Py = pu.sy + pu.dy * travel;
    const float3 V = (pu.active && s < pu.moving) ? f3(pu.dx * C.pspeed, pu.dy * C.pspeed, 0.f) : f3(0.f, 0.f, 0.f);
    for (int i = g.gl; i < n; i += g.G) {
        float4 v = W.bv()[i];
        v.x += C.gx * C.dt;
        v.y += C.gy * C.dt;
        v.z += C.gz * C.dt;
        W.bv()[i] = v;
    }
    frames_and_aabb(W, n, g, C.margin);
    __syncwarp();
    bool ovf = broadphase(W, n, g, C.pair_cap, on && pu.active, Px, Py, C);
    pc.mark(tm, W, PH_BROADPHASE, rec);
    {
        NarrowStats st{0, 0, 0, 0, 0, 0, 0};
        ovf |= narrowphase<kCyl>(W, g, on, C, Px, Py, st);
        // count now, so that nothing of the narrowphase stays live through the solve
        if (on && g.gl == 0) {
            const SArr<unsigned long long> ev = W.ev();
            ev[EV_SUBSTEPS] += 1;
            ev[EV_BOX_STEPS] += n;
            ev[EV_PAIR_TESTS] += n * (n - 1) / 2;
            ev[EV_SAT] += st.sat;
            ev[EV_FACE] += st.face;
            ev[EV_EDGE] += st.edge;
            ev[EV_PLANE] += st.plane;
            ev[EV_PUSHER] += st.pusher;
            ev[EV_POINTS] += W.scal()[4];
            ev[EV_MANIFOLDS] += W.scal()[3];
            ev[EV_CLIP_VERTS] += st.clip_verts;
            ev[EV_BB_POINTS] += st.bb_points;
        }
    }
    pc.mark(tm, W, PH_NARROWPHASE, rec);
    prepare(W, g, on, C);
    pc.mark(tm, W, PH_PREP, rec);
    ovf |= colour_manifolds(W, n, g, on);
    pc.mark(tm, W, PH_COLOUR, rec);
    if (kWarm && C.warm && a.warm) warm_start(W, g, on, C, warm, warm_n);
    int bb_visits = 0;
    const int visits = pgs(W, g, on, C.iters, V, bb_visits);
    if (kWarm && C.warm && a.warm) {
        const int m = warm_save(W, g, on, warm);
        if (on) warm_n = m;
    }
    pc.mark(tm, W, PH_SOLVE, rec);
    integrate(W, n, g, C.dt);
    pc.mark(tm, W, PH_INTEGRATE, rec);
    const int v_all = g.sum(visits), v_bb = g.sum(bb_visits);
    if (on && g.gl == 0) {
        const SArr<unsigned long long> ev = W.ev();
        ev[EV_PGS_MAN] += (unsigned long long)C.iters * W.scal()[6];
        ev[EV_PGS_PTS] += v_all;
        ev[EV_COLOURS] += W.scal()[5];
        ev[EV_PGS_BB_POINTS] += v_bb;
    }
    __syncwarp();
    return ovf && on;
}

// The environment slots of one warp: each group pulls environments from the work queue
// (largest first) and runs them push by push; a group whose environment finishes early
// (target graspable; Sec. IV-C hands such environments other work) takes the
// next one while the other groups continue.  Push set-up and end-of-push phases run when
// any group needs them; groups without work take part in the collectives only.
template <bool kCyl, bool kWarm>
__device__ __forceinline__ void run_slots(const RolloutArgs& a, const WarpMem& W, const Grp& g) {
    const SimConst& C = a.C;
    int e = -1;
    bool exhausted = false;
    EnvIn ei{nullptr, 0, 0, 0, -1};
    EnvProg pg;
    memset(&pg, 0, sizeof(pg));
    int budget = 0;
    long long t_start = 0;
    bool ovf = false, timed_out = false;
    const bool tm = C.timers != 0;
    PhaseClock pc;
    for (;;) {
        // 1. fetch
        const bool need = e < 0 && !exhausted;
        int slot = 0;
        if (need && g.gl == 0) slot = atomicAdd(a.queue_head, 1);
        slot = g.bcast(slot, 0);
        bool fresh = false;
        if (need) {
            if (slot < a.n_envs) {
                e = a.order[slot];
#if PMBS_BOUNDS_CHECK
                if (!check_index(CHK_ENV, e, a.n_envs)) e = 0;
#endif
                ei = a.env[e];
                pg = a.prog[e];
#if PMBS_BOUNDS_CHECK
                // every state and child row of the environment lies inside the batch
                if (!check_index(CHK_STATE_ROW, ei.box_off, a.n_rows) ||
                    !check_index(CHK_STATE_ROW, (long long)ei.box_off + ei.n - 1, a.n_rows))
                    pg.done = 1;
#endif
                if (pg.done) e = -1;
                else fresh = true;
            } else {
                exhausted = true;
            }
        }
        load_env(a, W, ei, fresh, pg.k == 0, g);
        if (fresh) {
            if (pg.k == 0) {
                pg.k = 1;
                pg.s = 0;
                pg.push_ready = 0;
            }
            budget = a.max_substeps > 0 ? a.max_substeps : INT_MAX;
            ovf = false;
            timed_out = false;
            t_start = clock64();
            if (g.gl == 0) {
                for (int k = 0; k < kNumEvents; k++) W.ev()[k] = 0ull;
                for (int k = 0; k < kNumPhases; k++) W.ph()[k] = 0ull;
            }
        }
        const bool active = e >= 0;
        if (!__any_sync(kFull, active || !exhausted)) break;
        // 2. push set-up: the first push's start check, or a sampled push
        const bool setup = active && !pg.push_ready;
        pc.start(tm);
        if (__any_sync(kFull, setup)) {
            compute_footprints(W, setup ? ei.n : 0, g);
            const bool first = setup && pg.k == 1;
            const float4 fp = first ? a.first_push[e] : make_float4(0.f, 0.f, 0.f, 0.f);
            const bool blocked = start_blocked(W, first ? ei.n : 0, g, fp.x, fp.y, C.pr);
            const bool samp = setup && pg.k > 1;
            float push[4] = {fp.x, fp.y, fp.z, fp.w};
            const int at = sample_push(W, ei.n, g, samp, samp ? a.seeds[e] : 0ull, pg.k, C, push);
            if (first) {
                if (blocked) {
                    pg.flags |= FLAG_INVALID_START;
                    pg.done = 1;
                    pg.cost = a.depth + 1;
                    pg.reward = 0.f;
                } else {
                    pg.noop = 0;
                }
            }
            if (samp) {
                if (g.gl == 0) W.ev()[EV_SAMPLE_ATTEMPTS] += at < 0 ? C.attempts : at + 1;
                if (at < 0) {
                    pg.noop = 1;
                    pg.flags |= FLAG_NOOP;
                    push[0] = push[1] = push[2] = push[3] = 0.f;
                } else {
                    pg.noop = 0;
                }
            }
            if (setup && !pg.done) {
                for (int i = 0; i < 4; i++) pg.push[i] = push[i];
                pg.push_ready = 1;
            }
        }
        pc.mark(tm, W, PH_PUSH_SETUP, setup && g.gl == 0);
        // 3. one substep
        const bool run = active && !pg.done && pg.s < C.substeps && budget > 0;
        const Pusher pu = make_pusher(C, pg.push, pg.noop != 0);
        ovf |= substep<kCyl, kWarm>(a, W, ei.n, run, pu, pg.s, g, a.warm ? a.warm + (size_t)(e < 0 ? 0 : e) * a.warm_f4_per_env : nullptr,
                       pg.pad[0], pc);
        // bounded run time per environment and launch (the shuffle runs in every lane)
        const bool late = g.bcast((int)(clock64() - t_start > a.watchdog_cycles), 0) != 0;
        if (run) {
            pg.s++;
            pg.steps++;
            budget--;
            timed_out = late;
        }
        // 4. end of push: workspace, grasp test, cost and reward
        const bool endp = active && !pg.done && !timed_out && pg.s == C.substeps;
        if (__any_sync(kFull, endp)) {
            if (endp && pg.k == 1 && a.child_on) store_state(W, ei.n, a.child + (size_t)ei.box_off * 13, g);
            bool out = false;
            for (int i = g.gl; endp && i < ei.n; i += g.G)
                out = out || fabsf(W.x()[i]) > C.table_hx || fabsf(W.x()[W.NB() + i]) > C.table_hy;
            out = g.any(out);
            const bool test = endp && !out;
            compute_footprints(W, test ? ei.n : 0, g);
            const bool graspable = grasp_check(W, ei.n, ei.target, g, test, C);
            if (endp) {
                if (g.gl == 0) W.ev()[EV_PUSH_EVALS] += 1;
                if (out) {
                    pg.flags |= FLAG_OUT_OF_WS;
                    pg.done = 1;
                    pg.cost = a.depth + 1;
                    pg.reward = 0.f;
                } else if (graspable) {
                    pg.done = 1;
                    pg.cost = pg.k;
                    pg.reward = powf(C.gamma, (float)(pg.k - 1));
                    if (pg.k == 1) pg.flags |= FLAG_GRASP1;
                } else if (pg.k >= a.depth) {
                    pg.done = 1;
                    pg.cost = a.depth + 1;
                    pg.reward = 0.f;
                } else {
                    pg.k++;
                    pg.s = 0;
                    pg.push_ready = 0;
                }
            }
        }
        pc.mark(tm, W, PH_PUSH_END, endp && g.gl == 0);
        // 5. retire: write the environment back and free the slot
        const bool fin = active && (pg.done || budget <= 0 || timed_out);
        if (fin) {
            if (ovf) pg.flags |= FLAG_OVERFLOW;
            store_state(W, ei.n, a.state + (size_t)ei.box_off * 13, g);
            if (g.gl == 0) {
                a.prog[e] = pg;
                unsigned long long* ev = a.events + (size_t)e * kNumEvents;
                for (int k = 0; k < kNumEvents; k++) ev[k] += W.ev()[k];
                if (tm) {
                    unsigned long long* ph = a.phase + (size_t)e * kNumPhases;
                    for (int k = 0; k < kNumPhases; k++) ph[k] += W.ph()[k];
                }
                a.steps[e] = pg.steps;
                if (pg.done) {
                    a.cost[e] = pg.cost;
                    a.reward[e] = pg.reward;
                    a.flags[e] = (uint8_t)pg.flags;
                    atomicAdd(a.done_count, 1);
                }
                if (timed_out) atomicExch(a.watchdog_flag, 1);
            }
            e = -1;
        }
        __syncwarp();
    }
}

// 128 threads (up to four warps) per block and a register budget for three blocks per SM
// (two with the cylinder contact paths, whose general separating-axis test and clipping
// stay in registers): the solver keeps its working set in registers without spilling.
template <bool kCyl, bool kWarm>
__global__ void __launch_bounds__(128, kCyl ? 2 : 3) rollout_kernel(const __grid_constant__ RolloutArgs a) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const Grp g(a.G, lane);
    const int per_warp = 32 / a.G;
    const int slot = wib * per_warp + (lane / a.G);
    const size_t gslot = (size_t)blockIdx.x * (blockDim.x >> 5) * per_warp + slot;
    const WarpMem W = bind_mem(a.L, (uint32_t)slot * (uint32_t)a.L.bytes, a.gscratch + gslot * a.scratch_f4_per_warp);
    run_slots<kCyl, kWarm>(a, W, g);
}

// The instantiation for a batch: cylinder contact paths and warm start compiled in only
// when the batch needs them.
using RolloutFn = void (*)(RolloutArgs);
inline RolloutFn rollout_fn(bool cyl, bool warm) {
    return cyl ? (warm ? rollout_kernel<true, true> : rollout_kernel<true, false>)
               : (warm ? rollout_kernel<false, true> : rollout_kernel<false, false>);
}
// ---- rollout device code ends

// Batch set-up: per-env scene descriptor and box offset (block-wide scan), processing
// order by descending box count (bucket sort), totals.  One block of 1024 threads.
__global__ void __launch_bounds__(1024) prepare_batch_kernel(int n_envs, const int32_t* scene_ids,
                                                             const SceneDesc* table, int table_cap, EnvIn* env,
                                                             int* order, int* counters) {
    __shared__ int hist[kMaxBoxes + 2];
    __shared__ int warp_sums[32];
    __shared__ int carry;
    const int t = threadIdx.x;
    if (t < kMaxBoxes + 2) hist[t] = 0;
    if (t == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n_envs; base += 1024) {
        const int e = base + t;
        int n = 0;
        SceneDesc d{nullptr, 0, 0};
        int sid = -1;
        if (e < n_envs) {
            sid = scene_ids[e];
            if (sid >= 0 && sid < table_cap) d = table[sid];
            if (d.n <= 0 || d.rec == nullptr) atomicOr(counters + 1, 1);
            n = d.n > 0 ? d.n : 0;
        }
        // block exclusive scan of n
        int v = n;
        const int lane = t & 31, w = t >> 5;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (lane == 31) warp_sums[w] = v;
        __syncthreads();
        if (w == 0) {
            int s = warp_sums[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += u;
            }
            warp_sums[lane] = s;
        }
        __syncthreads();
        const int excl = carry + (w ? warp_sums[w - 1] : 0) + v - n;
        if (e < n_envs) {
            env[e] = EnvIn{d.rec, n, d.target, excl, sid};
            atomicAdd(&hist[kMaxBoxes - min(n, kMaxBoxes)], 1);
        }
        __syncthreads();
        if (t == 0) carry += warp_sums[31];
        __syncthreads();
    }
    if (t == 0) {
        counters[0] = carry;
        int acc = 0;
        for (int b = 0; b <= kMaxBoxes; b++) {
            const int c = hist[b];
            hist[b] = acc;
            acc += c;
        }
    }
    __syncthreads();
    for (int e = t; e < n_envs; e += 1024) {
        const int b = kMaxBoxes - min(env[e].n, kMaxBoxes);
        const int pos = atomicAdd(&hist[b], 1);
        order[pos] = e;
    }
}

// Deepest box-box penetration of each scene (one warp per scene, one lane per pair, the
// rollout engine's separating-axis test); out[s] = max(0, -separation).
__global__ void __launch_bounds__(128) penetration_kernel(int n_scenes, const int32_t* box_offset,
                                                          const float* rec, float* out) {
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (s >= n_scenes) return;
    const int b0 = box_offset[s] - box_offset[0], n = box_offset[s + 1] - box_offset[s];
    const int T = n * (n - 1) / 2;
    float worst = 0.f;
    for (int t = lane; t < T; t += 32) {
        int i, j;
        pair_of_index(t, n, i, j);
        CBox A, B;
        const float* ra = rec + (size_t)kRecFloats * (b0 + i);
        const float* rb = rec + (size_t)kRecFloats * (b0 + j);
        A.c = f3(ra[0], ra[1], ra[2]);
        B.c = f3(rb[0], rb[1], rb[2]);
        quat_to_R_exact(ra[3], ra[4], ra[5], ra[6], A.R);
        quat_to_R_exact(rb[3], rb[4], rb[5], rb[6], B.R);
        for (int k = 0; k < 3; k++) {
            A.h[k] = fabsf(ra[13 + k]);
            B.h[k] = fabsf(rb[13 + k]);
        }
        A.cyl = ra[14] < 0.f;
        B.cyl = rb[14] < 0.f;
        CManifold cm;
        int clip = 0;
        if (A.cyl || B.cyl) {
            float sep = 0.f;
            if (collide_convex(A, B, 0.f, cm, clip, &sep)) worst = fmaxf(worst, -sep);
        } else if (collide_box_box(A, B, 0.f, cm, clip)) {
            for (int p = 0; p < cm.np; p++) worst = fmaxf(worst, -cm.d[p]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, o));
    if (lane == 0) out[s] = worst;
}

// ------------------------------------------------------------------ heightmaps
// Top-down heightmap of the workspace grid (Sec. V-A: 0.288 m x 0.288 m seen from above,
// 144 x 144 cells of 2 mm; the depth image the grasp classifier of Sec. IV-B reads):
// cell (i, j) holds the height of the highest box surface above its centre, or 0.  For
// each box the vertical line through the cell centre is written in the box frame
// (a_k + b_k s with s = z - c_z) and clipped against the three slabs |.| <= h_k (a
// cylinder: nine slabs, its cap axis and the 16-gon's side normal directions) (slab
// ends -(a_k / b_k) -+ h_k / b_k, with 1 / b_k and h_k / b_k rounded once per box and each
// end one fused multiply-add); a non-empty interval puts the box's top at c_z + s_hi.  Every operation is an explicitly
// rounded binary32 intrinsic in a fixed order, so the map is defined bit for bit.  A
// box is only tested for cells inside its footprint's bounding square grown by 1 mm (the
// line misses the box there by at least 1 mm, far beyond any rounding).
struct HMCsr {  // state snapshot: CSR box ranges, 13-float states, half extents
    const int32_t* box_offset;
    const float* states;
    const float* half;
    __device__ __forceinline__ int n(int e) const { return box_offset[e + 1] - box_offset[e]; }
    __device__ __forceinline__ const float* st(int e, int i) const {
        return states + (size_t)(box_offset[e] - box_offset[0] + i) * 13;
    }
    __device__ __forceinline__ const float* h(int e, int i) const {
        return half + (size_t)(box_offset[e] - box_offset[0] + i) * 3;
    }
};
struct HMBatch {  // a rollout batch's current states (half extents from the scene records)
    const EnvIn* env;
    const float* state;
    __device__ __forceinline__ int n(int e) const { return env[e].n; }
    __device__ __forceinline__ const float* st(int e, int i) const {
        return state + (size_t)(env[e].box_off + i) * 13;
    }
    __device__ __forceinline__ const float* h(int e, int i) const { return env[e].rec + (size_t)kRecFloats * i + 13; }
};

constexpr int kHMCells = 144;
constexpr float kHMCell = 0.002f, kHMOrigin = -0.144f;

// One block of 512 threads per environment.  Each box visits only the cells of its grown
// footprint square (threads laid out 32 x 16 over it) and raises a shared-memory map with
// an integer atomicMax on the bit pattern: the heights written are positive floats,
// whose bit patterns order like their values, so the map is the exact maximum whatever
// the order.  The finished map leaves in 16-byte stores.  Dynamic shared memory:
// kHMCells^2 words.
constexpr size_t kHMSmem = sizeof(unsigned int) * kHMCells * kHMCells;

template <class Src>
__global__ void __launch_bounds__(512) heightmap_kernel(const Src src, int n_envs, float* out) {
    // per body its slabs: world normal (x, y, z components), half thickness, 1 / z and
    // half / z (a box: its three axes; a cylinder: its cap axis and 8 side normals)
    __shared__ float sw[kMaxBoxes][9][4], srb[kMaxBoxes][9], shr[kMaxBoxes][9];
    __shared__ float sc[kMaxBoxes][3], sbox[kMaxBoxes][4];
    __shared__ int srect[kMaxBoxes][4], sns[kMaxBoxes];
    unsigned int* map = reinterpret_cast<unsigned int*>(pmbs_smem);
    const int e = blockIdx.x;
    if (e >= n_envs) return;
    const int n = min(src.n(e), kMaxBoxes);
    uint4* m4 = reinterpret_cast<uint4*>(map);
    for (int c = threadIdx.x; c < kHMCells * kHMCells / 4; c += blockDim.x) m4[c] = make_uint4(0u, 0u, 0u, 0u);
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
        const float* s = src.st(e, b);
        const float* hh = src.h(e, b);
        float R[9];
        quat_to_R_exact(s[3], s[4], s[5], s[6], R);
        for (int k = 0; k < 3; k++) sc[b][k] = s[k];
        auto slab = [&](int k, float wx, float wy, float wz, float half) {
            sw[b][k][0] = wx;
            sw[b][k][1] = wy;
            sw[b][k][2] = wz;
            sw[b][k][3] = half;
            srb[b][k] = wz == 0.f ? 0.f : __frcp_rn(wz);  // 1 / b_k, rounded once
            shr[b][k] = __fmul_rn(half, srb[b][k]);      // h_k / b_k
        };
        if (hh[1] < 0.f) {
            slab(0, R[2], R[5], R[8], hh[2]);
            const float apo = __fmul_rn(hh[0], kGonApo);
            for (int k = 0; k < 8; k++)
                slab(1 + k, xa(xm(kGonFC[k], R[0]), xm(kGonFS[k], R[1])), xa(xm(kGonFC[k], R[3]), xm(kGonFS[k], R[4])),
                     xa(xm(kGonFC[k], R[6]), xm(kGonFS[k], R[7])), apo);
            sns[b] = 9;
        } else {
            for (int k = 0; k < 3; k++) slab(k, R[k], R[3 + k], R[6 + k], hh[k]);
            sns[b] = 3;
        }
        const float ex = aabb_half_exact(R, hh[0], hh[1], hh[2]) + 1e-3f;      // row 0: x
        const float ey = aabb_half_exact(R + 3, hh[0], hh[1], hh[2]) + 1e-3f;  // row 1: y
        sbox[b][0] = s[0] - ex;
        sbox[b][1] = s[0] + ex;
        sbox[b][2] = s[1] - ey;
        sbox[b][3] = s[1] + ey;
        // cells whose centres can fall inside the square, one cell of slack on each side
        // (the exact test below decides; the range only bounds the work)
        const float inv = 1.f / kHMCell;
        auto cell_of = [&](float v) {  // clamped before the conversion to int
            return (int)floorf(fminf(fmaxf((v - kHMOrigin) * inv, -4.f), (float)kHMCells + 4.f));
        };
        srect[b][0] = max(0, cell_of(sbox[b][0]) - 1);
        srect[b][1] = min(kHMCells - 1, cell_of(sbox[b][1]) + 1);
        srect[b][2] = max(0, cell_of(sbox[b][2]) - 1);
        srect[b][3] = min(kHMCells - 1, cell_of(sbox[b][3]) + 1);
    }
    __syncthreads();
    // work items: every (body, cell) of every body's cell rectangle, numbered body by body
    // and row by row; the block's threads take consecutive items, so small rectangles do
    // not leave lanes idle
    __shared__ int sstart[kMaxBoxes + 1];
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int b = 0; b < n; b++) {
            sstart[b] = acc;
            acc += max(0, srect[b][1] - srect[b][0] + 1) * max(0, srect[b][3] - srect[b][2] + 1);
        }
        sstart[n] = acc;
    }
    __syncthreads();
    const int total = sstart[n];
    int b = 0;
    for (int item = threadIdx.x; item < total; item += blockDim.x) {
        while (item >= sstart[b + 1]) b++;
        {
            const int w = srect[b][1] - srect[b][0] + 1;
            const int o = item - sstart[b];
            const int jr = o / w;
            const int i = srect[b][0] + (o - jr * w), j = srect[b][2] + jr;
            {
                const float xc = __fadd_rn(kHMOrigin, __fmul_rn(__fadd_rn((float)i, 0.5f), kHMCell));
                const float yc = __fadd_rn(kHMOrigin, __fmul_rn(__fadd_rn((float)j, 0.5f), kHMCell));
                if (xc < sbox[b][0] || xc > sbox[b][1] || yc < sbox[b][2] || yc > sbox[b][3]) continue;
                const float dx = __fsub_rn(xc, sc[b][0]), dy = __fsub_rn(yc, sc[b][1]);
                float s_lo = -INFINITY, s_hi = INFINITY;
                bool hit = true;
                auto clip = [&](int k) {
                    const float a = __fmaf_rn(sw[b][k][0], dx, __fmul_rn(sw[b][k][1], dy));
                    const float bk = sw[b][k][2];
                    if (bk == 0.f) {
                        if (!(fabsf(a) <= sw[b][k][3])) hit = false;
                        return;
                    }
                    const float r = srb[b][k];
                    float t0 = __fmaf_rn(-a, r, -shr[b][k]), t1 = __fmaf_rn(-a, r, shr[b][k]);
                    if (bk < 0.f) {
                        const float tt = t0;
                        t0 = t1;
                        t1 = tt;
                    }
                    if (t0 > s_lo) s_lo = t0;
                    if (t1 < s_hi) s_hi = t1;
                };
                if (sns[b] == 3) {
#pragma unroll
                    for (int k = 0; k < 3; k++) clip(k);
                } else {
                    for (int k = 0; k < 9 && hit; k++) clip(k);
                }
                if (hit && s_lo <= s_hi) {
                    const float z = __fadd_rn(sc[b][2], s_hi);
                    if (z > 0.f) atomicMax(&map[j * kHMCells + i], __float_as_uint(z));
                }
            }
        }
    }
    __syncthreads();
    float4* o = reinterpret_cast<float4*>(out + (size_t)e * kHMCells * kHMCells);
    for (int c = threadIdx.x; c < kHMCells * kHMCells / 4; c += blockDim.x) {
        const uint4 v = m4[c];
        o[c] = make_float4(__uint_as_float(v.x), __uint_as_float(v.y), __uint_as_float(v.z), __uint_as_float(v.w));
    }
}

// Heightmap form of the grasp test, one warp per environment, one (angle, side) pair per
// lane: the jaw angles, the opening condition and the finger rectangles of the footprint
// test; a rectangle is clear when no map cell whose centre lies in it beyond the target's
// side is higher than the finger tips, `depth` below the target's top.  Cells are visited
// over the rectangle's bounding square with one cell of slack; the membership test, in
// fixed-order binary32, decides.
__global__ void __launch_bounds__(128) grasp_hm_kernel(const HMCsr src, const int32_t* target, const float* maps,
                                                       int n_envs, SimConst C, float depth, uint8_t* out) {
    const int lane = threadIdx.x & 31;
    const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (e >= n_envs) return;
    const int t = target[e];
    const float* s = src.st(e, t);
    const float* hh = src.h(e, t);
    float R[9];
    quat_to_R_exact(s[3], s[4], s[5], s[6], R);
    const Foot ft = footprint_exact(s[0], s[1], R, hh[0], hh[1], hh[2]);
    const float z_tip = xs(xa(s[2], vertical_half_exact(R, hh[0], hh[1], hh[2])), depth);
    const float halfW = xm(C.grasp_W, 0.5f), hfw = xm(C.grasp_fw, 0.5f);
    const float* map = maps + (size_t)e * kHMCells * kHMCells;
    bool any = false;
    for (int sb = 0; sb < 2 * C.grasp_K; sb += 32) {
        const int slot = sb + lane;
        const int k = slot >> 1;
        const float sg = (slot & 1) ? -1.f : 1.f;
        bool ok = false;
        if (k < C.grasp_K) {
            const float ax = C.gcos[k], ay = C.gsin[k];
            const float bx = -ay, by = ax;
            const float wa = xa(xm(fabsf(xdot2(ft.ux, ft.uy, ax, ay)), ft.su), xm(fabsf(xdot2(ft.vx, ft.vy, ax, ay)), ft.sv));
            if (xm(xa(wa, C.grasp_c), 2.f) <= C.grasp_W) {
                const float off = xm(xa(xa(wa, halfW), C.grasp_f), 0.5f);
                const float hl = xm(xs(xa(halfW, C.grasp_f), wa), 0.5f);
                const float sax = sg * ax, say = sg * ay;
                const float fcx = xa(ft.cx, xm(sax, off)), fcy = xa(ft.cy, xm(say, off));
                const float rx = fabsf(sax) * hl + fabsf(bx) * hfw, ry = fabsf(say) * hl + fabsf(by) * hfw;
                auto cell_of = [](float v) {  // clamped before the conversion to int
                    return (int)floorf(fminf(fmaxf((v - kHMOrigin) / kHMCell, -4.f), (float)kHMCells + 4.f));
                };
                const int i0 = max(0, cell_of(fcx - rx) - 1), i1 = min(kHMCells - 1, cell_of(fcx + rx) + 1);
                const int j0 = max(0, cell_of(fcy - ry) - 1), j1 = min(kHMCells - 1, cell_of(fcy + ry) + 1);
                ok = true;
                for (int j = j0; j <= j1 && ok; j++) {
                    const float py = xs(xa(kHMOrigin, xm(xa((float)j, 0.5f), kHMCell)), fcy);
                    for (int i = i0; i <= i1; i++) {
                        const float px = xs(xa(kHMOrigin, xm(xa((float)i, 0.5f), kHMCell)), fcx);
                        const float pa = xa(xm(px, sax), xm(py, say)), pb = xa(xm(px, bx), xm(py, by));
                        if (pa > -hl && pa <= hl && fabsf(pb) <= hfw && map[j * kHMCells + i] > z_tip) {
                            ok = false;
                            break;
                        }
                    }
                }
            }
        }
        // both sides of one angle sit on neighbouring lanes
        const bool partner = __shfl_xor_sync(0xffffffffu, ok, 1) != 0;
        any = any || __any_sync(0xffffffffu, ok && partner);
    }
    if (lane == 0) out[e] = any ? 1 : 0;
}

// Scene table update: table[ids[i]] = desc[i].
__global__ void scatter_desc_kernel(int n, const int32_t* ids, const SceneDesc* desc, SceneDesc* table) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) table[ids[i]] = desc[i];
}

// ------------------------------------------------------------------ snapshot evaluation
struct EvalArgs {
    SimConst C;
    Layout L;
    int n_envs, mode, k;
    const int32_t* box_offset;
    const float* states;
    const float* half;
    const float* pusher_xy;
    const int32_t* target;
    const uint64_t* seeds;
    const float* starts;
    int32_t* out_pairs;
    int32_t* out_n_pairs;
    int32_t* out_plane;
    int32_t* out_n_plane;
    int32_t* out_pusher;
    int32_t* out_n_pusher;
    uint8_t* out_u8;
    float* out_push;
    int32_t* out_attempt;
};

__global__ void __launch_bounds__(128) eval_kernel(const __grid_constant__ EvalArgs a) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nw = gridDim.x * (blockDim.x >> 5);
    const WarpMem W = bind_mem(a.L, (uint32_t)wib * (uint32_t)a.L.bytes, nullptr);
    const Grp g(32, lane);
    const int NB = W.NB();
    for (int e = blockIdx.x * (blockDim.x >> 5) + wib; e < a.n_envs; e += nw) {
        const int b0 = a.box_offset[e], n = a.box_offset[e + 1] - b0;
        for (int i = lane; i < n; i += 32) {
            const float* s = a.states + (size_t)(b0 + i) * 13;
            const float* h = a.half + (size_t)(b0 + i) * 3;
            W.x()[i] = s[0]; W.x()[NB + i] = s[1]; W.x()[2 * NB + i] = s[2];
            W.q()[i] = s[3]; W.q()[NB + i] = s[4]; W.q()[2 * NB + i] = s[5]; W.q()[3 * NB + i] = s[6];
            W.h()[i] = h[0]; W.h()[NB + i] = h[1]; W.h()[2 * NB + i] = h[2];
            W.ib()[i] = 1.f; W.ib()[NB + i] = 1.f; W.ib()[2 * NB + i] = 1.f;
        }
        __syncwarp();
        if (a.mode == 0) {
            frames_and_aabb(W, n, g, a.C.margin);
            __syncwarp();
            const bool on = a.pusher_xy != nullptr;
            const float px = on ? a.pusher_xy[2 * e] : 0.f, py = on ? a.pusher_xy[2 * e + 1] : 0.f;
            broadphase(W, n, g, a.C.pair_cap, on, px, py, a.C);
            const int np = W.scal()[0], npl = W.scal()[1], npu = W.scal()[2];
            for (int k = lane; k < np; k += 32) {
                a.out_pairs[((size_t)e * a.C.pair_cap + k) * 2] = W.pairs()[k] & 255;
                a.out_pairs[((size_t)e * a.C.pair_cap + k) * 2 + 1] = W.pairs()[k] >> 8;
            }
            for (int k = lane; k < npl; k += 32) a.out_plane[b0 + k] = W.plane()[k];
            for (int k = lane; k < npu; k += 32) a.out_pusher[b0 + k] = W.pusher()[k];
            if (lane == 0) {
                a.out_n_pairs[e] = np;
                a.out_n_plane[e] = npl;
                a.out_n_pusher[e] = npu;
            }
        } else {
            compute_footprints(W, n, g);
            if (a.mode == 1) {
                const bool ok = grasp_check(W, n, a.target[e], g, true, a.C);
                if (lane == 0) a.out_u8[e] = ok ? 1 : 0;
            } else if (a.mode == 2) {
                float push[4] = {0.f, 0.f, 0.f, 0.f};
                const int at = sample_push(W, n, g, true, a.seeds[e], a.k, a.C, push);
                if (lane == 0) {
                    a.out_attempt[e] = at;
                    for (int i = 0; i < 4; i++) a.out_push[4 * e + i] = at < 0 ? 0.f : push[i];
                }
            } else {
                const bool b = start_blocked(W, n, g, a.starts[2 * e], a.starts[2 * e + 1], a.C.pr);
                if (lane == 0) a.out_u8[e] = b ? 1 : 0;
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ FP32 peak probe
__global__ void __launch_bounds__(256) fma_peak_kernel(float* out, int iters, float seed) {
    float a0 = seed + threadIdx.x, a1 = a0 + 1.f, a2 = a0 + 2.f, a3 = a0 + 3.f;
    float a4 = a0 + 4.f, a5 = a0 + 5.f, a6 = a0 + 6.f, a7 = a0 + 7.f;
    const float m = 0.999999f, c = 1e-7f;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < 16; u++) {
            a0 = fmaf(a0, m, c); a1 = fmaf(a1, m, c); a2 = fmaf(a2, m, c); a3 = fmaf(a3, m, c);
            a4 = fmaf(a4, m, c); a5 = fmaf(a5, m, c); a6 = fmaf(a6, m, c); a7 = fmaf(a7, m, c);
        }
    }
    const float s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
    if (s == 12345.678f) out[blockIdx.x] = s;
}

// ------------------------------------------------------------------ host side
struct Arena {
    char* base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_;  // offset -> bytes
    size_t used = 0;
    void init(char* b, size_t s) {
        base = b;
        size = s;
        free_.clear();
        free_[0] = s;
        used = 0;
    }
    // first fit, 256-byte aligned; returns SIZE_MAX if full
    size_t alloc(size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        if (bytes == 0) bytes = 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, rem = it->second - bytes;
                free_.erase(it);
                if (rem) free_[off + bytes] = rem;
                used += bytes;
                return off;
            }
        }
        return SIZE_MAX;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        if (bytes == 0) bytes = 256;
        used -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct SceneRec {
    bool live = false;
    size_t block = 0;             // arena block holding this scene's records
    size_t rec_off = 0;           // byte offset of its records inside the arena
    int n = 0, target = 0;
    int uses = 0;                 // batches referencing it (host-submitted ids only)
    bool cyl = false;             // holds a cylinder
    std::vector<float> host;      // records, kRecFloats per box
};

struct SceneBlock {
    size_t bytes = 0;
    int live = 0;                 // scenes of this block not yet freed
};

struct Batch {
    int n_envs = 0, depth = 0, nb = 0;
    size_t state_boxes = 0;
    bool host_ids = false;
    std::vector<int> scene_ids;   // for use counts (host submissions)
    size_t off = 0, bytes = 0;
    EnvIn* env = nullptr;
    int* order = nullptr;
    int* counters = nullptr;      // [0] total boxes, [1] bad id, [2] queue head, [3] done count
    float4* first_push = nullptr;
    uint64_t* seeds = nullptr;
    int32_t* ids = nullptr;
    EnvProg* prog = nullptr;
    float* state = nullptr;
    float* child = nullptr;
    int32_t* cost = nullptr;
    float* reward = nullptr;
    uint8_t* flags = nullptr;
    int32_t* steps = nullptr;
    unsigned long long* events = nullptr;
    unsigned long long* phase = nullptr;  // per-phase cycles (cfg.phase_timers)
    float4* warm = nullptr;         // warm-start caches (cfg.warm_start), one per environment
    bool finished = false;
    int G = 32, wpb = 4, Ms = 0;
    int tile = 0;  // substeps per launch when run to completion (0: one persistent launch)
    bool cyl = false;  // may hold cylinders: run the kernel with the cylinder contact paths
    cudaStream_t stream = nullptr;  // stream of this batch's launches (the context's by default)
    bool own_scratch = false;       // contact spill scratch of its own (batches that may overlap)
    size_t scr_off = 0, scr_bytes = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_k = 0;
};

}  // namespace

struct pmbs_ctx {
    pmbs_config cfg;
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0;
    bool own_arena = false;
    Arena arena;
    std::vector<SceneRec> scenes;
    std::map<size_t, SceneBlock> blocks;
    std::vector<int> free_ids;
    SceneDesc* d_table = nullptr;
    size_t table_off = 0;
    std::map<int64_t, Batch> batches;
    int64_t next_batch = 1;
    std::string err;
    std::mutex mu;
    float4* gscratch = nullptr;
    size_t gscratch_off = 0, gscratch_bytes = 0;
    int fixed_wpb = 0, fixed_Ps = -1, fixed_Ms = -1, fixed_G = 0;
    int fixed_tile = -1;  // substeps per launch forced by the autotuner while it times (-1: none)
    std::map<int, std::array<int, 3>> tuned;  // box-count bucket -> {G, wpb, Ms} from pmbs_autotune
    std::map<int, int> tuned_tile;            // box-count bucket -> substeps per launch (0: persistent)
    SimConst C;
};

namespace {

// NVTX range over a host call (visible in a profiler's timeline; free without one).  A
// push runs inside the persistent kernel, so ranges mark the calls and the server's
// launches, not individual pushes.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

pmbs_status fail(pmbs_ctx* c, pmbs_status s, const std::string& m) {
    c->err = m;
    return s;
}

#define CU(call)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(ctx, PMBS_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

void fill_const(const pmbs_config& c, SimConst& C) {
    C.dt = c.dt;
    C.gx = c.gravity[0];
    C.gy = c.gravity[1];
    C.gz = c.gravity[2];
    C.table_hx = c.table_half[0];
    C.table_hy = c.table_half[1];
    C.table_mu = c.table_mu;
    C.pusher_mu = c.pusher_mu;
    C.pr = c.pusher_radius;
    C.pz0 = c.pusher_z0;
    C.pz1 = c.pusher_z1;
    C.pspeed = c.pusher_speed;
    C.plen = c.push_length;
    C.gamma = c.gamma;
    C.grasp_W = c.grasp_opening;
    C.grasp_c = c.grasp_clearance;
    C.grasp_f = c.finger_depth;
    C.grasp_fw = c.finger_width;
    C.margin = c.margin;
    C.slop = c.slop;
    C.baumgarte = c.baumgarte;
    C.sample_clear = c.sample_clearance;
    C.substeps = c.substeps_per_push;
    C.iters = c.pgs_iters;
    C.warm = c.warm_start ? 1 : 0;
    C.warm_tol2 = c.warm_tolerance * c.warm_tolerance;
    C.grasp_K = c.grasp_angles;
    C.attempts = c.sample_attempts;
    C.npts = c.contour_points;
    C.Pcap = c.contact_cap;
    C.Mcap = c.manifold_cap;
    C.pair_cap = c.pair_cap;
    C.timers = c.phase_timers ? 1 : 0;
    for (int k = 0; k < 32; k++) {
        const double th = k < c.grasp_angles ? k * M_PI / c.grasp_angles : 0.0;
        C.gcos[k] = (float)std::cos(th);
        C.gsin[k] = (float)std::sin(th);
    }
}

bool finite(float x) { return std::isfinite(x); }

void* arena_ptr(pmbs_ctx* ctx, size_t off) { return ctx->arena.base + off; }

// Launch shape for environments of up to nb boxes: lanes per environment G (a warp runs
// 32 / G environments), warps per block, and the number of contact manifolds (with their
// four point slots) kept in shared memory per environment.  Default: one environment per
// warp (measured fastest on the uneven workload: the solve is latency-bound per warp and
// packing stretches the largest colour over more passes), about 18 KB of shared memory
// per environment slot.  smem_points (if set) counts
// point slots, four per manifold; smem_manifolds takes precedence.
int shape_bucket(int nb) { return nb <= 8 ? 8 : nb <= 16 ? 16 : nb <= 24 ? 24 : nb <= 32 ? 32 : nb <= 40 ? 40 : 64; }

void choose_shape(pmbs_ctx* ctx, int nb, int& G, int& wpb, int& Ms) {
    const pmbs_config& c = ctx->cfg;
    const auto tuned = ctx->tuned.find(shape_bucket(nb));
    if (tuned != ctx->tuned.end() && ctx->fixed_G == 0 && ctx->fixed_wpb == 0 && ctx->fixed_Ms < 0 &&
        ctx->fixed_Ps < 0 && c.lanes_per_env == 0 && c.warps_per_block == 0 && c.smem_points < 0 &&
        c.smem_manifolds < 0) {
        const int pairS = std::min(c.pair_cap, std::max(1, nb * (nb - 1) / 2));
        G = tuned->second[0];
        wpb = tuned->second[1];
        Ms = tuned->second[2];
        const int K = 32 / G;
        while (Ms > 0 && (size_t)K * make_layout(nb, pairS, Ms, c.manifold_cap).bytes > 227 * 1024) Ms /= 2;
        while (wpb > 1 && (size_t)wpb * K * make_layout(nb, pairS, Ms, c.manifold_cap).bytes > 227 * 1024) wpb >>= 1;
        return;
    }
    const int pairS = std::min(c.pair_cap, std::max(1, nb * (nb - 1) / 2));
    G = ctx->fixed_G > 0 ? ctx->fixed_G : (c.lanes_per_env > 0 ? c.lanes_per_env : 32);
    wpb = ctx->fixed_wpb > 0 ? ctx->fixed_wpb : (c.warps_per_block > 0 ? c.warps_per_block : 2);
    wpb = std::min(wpb, 4);
    const int K = 32 / G;
    // A few manifolds in shared memory, the rest in the L1-cached scratch: shared memory
    // and L1 share one array per SM, and a large shared carve-out starves L1 of the room
    // the contact scratch and the per-thread clip polygons need (measured: 8 manifolds
    // per environment beat 27 by 15 % on the 4096-environment uneven workload).
    int ms = 8;
    if (K > 1) ms = 0;  // several environments per warp: contacts in L1-cached scratch
    if (c.smem_points >= 0) ms = c.smem_points / 4;
    if (c.smem_manifolds >= 0) ms = c.smem_manifolds;
    if (ctx->fixed_Ps >= 0) ms = ctx->fixed_Ps / 4;
    if (ctx->fixed_Ms >= 0) ms = ctx->fixed_Ms;
    Ms = std::min(ms, c.manifold_cap);
    // keep one block within the 227 KB opt-in limit
    while (Ms > 0 && (size_t)K * make_layout(nb, pairS, Ms, c.manifold_cap).bytes > 227 * 1024) Ms /= 2;
    while (wpb > 1 && (size_t)wpb * K * make_layout(nb, pairS, Ms, c.manifold_cap).bytes > 227 * 1024) wpb >>= 1;
}

pmbs_status ensure_scratch(pmbs_ctx* ctx, size_t warps) {
    const size_t per = (size_t)scratch_f4_per_warp(ctx->cfg.manifold_cap) * sizeof(float4);
    const size_t need = warps * per;
    if (need <= ctx->gscratch_bytes) return PMBS_OK;
    if (ctx->gscratch) ctx->arena.release(ctx->gscratch_off, ctx->gscratch_bytes);
    ctx->gscratch = nullptr;
    ctx->gscratch_bytes = 0;
    const size_t off = ctx->arena.alloc(need);
    if (off == SIZE_MAX) return fail(ctx, PMBS_E_OOM, "solver scratch does not fit in the arena");
    ctx->gscratch_off = off;
    ctx->gscratch_bytes = need;
    ctx->gscratch = (float4*)arena_ptr(ctx, off);
    return PMBS_OK;
}

pmbs_status create_common(const pmbs_config* cfg, void* stream, void* d_arena, size_t arena_bytes, pmbs_ctx** out) {
    if (!cfg || !out) return PMBS_E_INVALID;
    *out = nullptr;
    const pmbs_config& c = *cfg;
    if (c.max_boxes_per_env < 1 || c.max_boxes_per_env > kMaxBoxes || c.max_envs < 0 || c.substeps_per_push < 1 ||
        c.pgs_iters < 0 || !(c.dt > 0) || c.grasp_angles < 1 || c.grasp_angles > 32 || c.sample_attempts < 1 ||
        c.sample_attempts > 32 || c.contour_points < 1 || c.contact_cap < 4 || c.manifold_cap < 1 ||
        c.manifold_cap > 1024 || c.pair_cap < 1 || c.pair_cap > 4096 || !(c.pusher_speed > 0) ||
        !(c.pusher_radius > 0) || !(c.watchdog_ms > 0) || !(c.max_initial_penetration >= 0) ||
        !(c.warm_start == 0 || c.warm_start == 1) || !(c.warm_tolerance >= 0) ||
        !(c.lanes_per_env == 0 || c.lanes_per_env == 8 || c.lanes_per_env == 16 ||
                                    c.lanes_per_env == 32))
        return PMBS_E_INVALID;
    pmbs_ctx* ctx = new pmbs_ctx();
    ctx->cfg = c;
    ctx->stream = (cudaStream_t)stream;
    ctx->device = c.device;
    fill_const(c, ctx->C);
    cudaError_t e = cudaSetDevice(c.device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, c.device);
    if (e != cudaSuccess) {
        delete ctx;
        return PMBS_E_CUDA;
    }
    char* base = (char*)d_arena;
    size_t bytes = arena_bytes;
    if (!base) {
        bytes = c.mem_budget_bytes;
        if (bytes < (size_t)64 << 20) bytes = (size_t)64 << 20;
        e = cudaMalloc((void**)&base, bytes);
        if (e != cudaSuccess) {
            delete ctx;
            return PMBS_E_OOM;
        }
        ctx->own_arena = true;
    } else if (((uintptr_t)base & 255) != 0) {
        delete ctx;
        return PMBS_E_INVALID;
    }
    ctx->arena.init(base, bytes);
    ctx->table_off = ctx->arena.alloc(sizeof(SceneDesc) * kSceneTableCap);
    if (ctx->table_off == SIZE_MAX) {
        if (ctx->own_arena) cudaFree(base);
        delete ctx;
        return PMBS_E_OOM;
    }
    ctx->d_table = (SceneDesc*)(base + ctx->table_off);
    e = cudaMemsetAsync(ctx->d_table, 0, sizeof(SceneDesc) * kSceneTableCap, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    for (int k = 0; k < 4 && e == cudaSuccess; k++)
        e = cudaFuncSetAttribute(rollout_fn(k & 1, k & 2), cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(eval_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(heightmap_kernel<HMCsr>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHMSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(heightmap_kernel<HMBatch>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHMSmem);

    if (e != cudaSuccess) {
        if (ctx->own_arena) cudaFree(base);
        delete ctx;
        return PMBS_E_CUDA;
    }
    *out = ctx;
    return PMBS_OK;
}

void release_batch_mem(pmbs_ctx* ctx, Batch& b) {
    if (b.graph) cudaGraphExecDestroy(b.graph);
    b.graph = nullptr;
    if (b.scr_bytes) ctx->arena.release(b.scr_off, b.scr_bytes);
    b.scr_bytes = 0;
    if (b.bytes) ctx->arena.release(b.off, b.bytes);
    b.bytes = 0;
    for (int s : b.scene_ids)
        if (s >= 0 && s < (int)ctx->scenes.size()) ctx->scenes[s].uses--;
    b.scene_ids.clear();
}

pmbs_status rollout_common(pmbs_ctx* ctx, int n_envs, const int32_t* scene_ids, const float* first_push, int depth,
                           const uint64_t* seeds, bool device_ptrs, int64_t* out_batch) {
    const pmbs_config& c = ctx->cfg;
    if (!out_batch || n_envs < 0 || n_envs > c.max_envs || depth < 1 || depth > 64)
        return fail(ctx, PMBS_E_INVALID, "bad batch size or depth");
    if (n_envs > 0 && (!scene_ids || !first_push || (!seeds && depth > 1)))
        return fail(ctx, PMBS_E_INVALID, "missing input array");
    Batch b;
    b.n_envs = n_envs;
    b.depth = depth;
    b.host_ids = !device_ptrs;
    size_t boxes = 0;
    int nb = 1;
    if (!device_ptrs) {
        for (int e = 0; e < n_envs; e++) {
            const int s = scene_ids[e];
            if (s < 0 || s >= (int)ctx->scenes.size() || !ctx->scenes[s].live)
                return fail(ctx, PMBS_E_INVALID, "unknown scene id " + std::to_string(s));
            boxes += ctx->scenes[s].n;
            nb = std::max(nb, ctx->scenes[s].n);
            b.cyl = b.cyl || ctx->scenes[s].cyl;
            const float* p = first_push + 4 * e;
            if (!finite(p[0]) || !finite(p[1]) || !finite(p[2]) || !finite(p[3]))
                return fail(ctx, PMBS_E_INVALID, "non-finite push");
        }
    } else {
        for (const SceneRec& r : ctx->scenes)
            if (r.live) {
                nb = std::max(nb, r.n);
                b.cyl = b.cyl || r.cyl;
            }
        boxes = (size_t)n_envs * nb;
    }
    b.nb = nb;
    b.state_boxes = boxes;
    const size_t ne = (size_t)std::max(n_envs, 1);
    size_t sz = 0;
    auto take = [&](size_t bytes) {
        const size_t o = sz;
        sz += (bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_env = take(sizeof(EnvIn) * ne), o_order = take(sizeof(int) * ne), o_cnt = take(sizeof(int) * 8),
                 o_fp = take(sizeof(float4) * ne), o_seed = take(sizeof(uint64_t) * ne),
                 o_ids = take(sizeof(int32_t) * ne), o_prog = take(sizeof(EnvProg) * ne),
                 o_state = take(sizeof(float) * 13 * std::max(boxes, (size_t)1)),
                 o_child = take(sizeof(float) * 13 * std::max(boxes, (size_t)1)), o_cost = take(sizeof(int32_t) * ne),
                 o_rew = take(sizeof(float) * ne), o_flags = take(ne), o_steps = take(sizeof(int32_t) * ne),
                 o_ev = take(sizeof(unsigned long long) * kNumEvents * ne),
                 o_ph = take(sizeof(unsigned long long) * kNumPhases * ne);
    const size_t warm_f4 = (size_t)kWarmF4 * ctx->cfg.manifold_cap;
    const size_t o_warm = ctx->cfg.warm_start ? take(sizeof(float4) * warm_f4 * ne) : 0;
    b.off = ctx->arena.alloc(sz);
    if (b.off == SIZE_MAX) return fail(ctx, PMBS_E_OOM, "batch does not fit in the device arena");
    b.bytes = sz;
    char* base = (char*)arena_ptr(ctx, b.off);
    b.env = (EnvIn*)(base + o_env);
    b.order = (int*)(base + o_order);
    b.counters = (int*)(base + o_cnt);
    b.first_push = (float4*)(base + o_fp);
    b.seeds = (uint64_t*)(base + o_seed);
    b.ids = (int32_t*)(base + o_ids);
    b.prog = (EnvProg*)(base + o_prog);
    b.state = (float*)(base + o_state);
    b.child = (float*)(base + o_child);
    b.cost = (int32_t*)(base + o_cost);
    b.reward = (float*)(base + o_rew);
    b.flags = (uint8_t*)(base + o_flags);
    b.steps = (int32_t*)(base + o_steps);
    b.events = (unsigned long long*)(base + o_ev);
    b.phase = (unsigned long long*)(base + o_ph);
    b.warm = ctx->cfg.warm_start ? (float4*)(base + o_warm) : nullptr;
    auto bail = [&](const char* what, cudaError_t e) {
        ctx->arena.release(b.off, b.bytes);
        return fail(ctx, PMBS_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    };
    cudaError_t e = cudaMemsetAsync(base + o_cnt, 0, sizeof(int) * 8, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.prog, 0, sizeof(EnvProg) * ne, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.events, 0, sizeof(unsigned long long) * kNumEvents * ne, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.phase, 0, sizeof(unsigned long long) * kNumPhases * ne, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.steps, 0, sizeof(int32_t) * ne, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.seeds, 0, sizeof(uint64_t) * ne, ctx->stream);
    if (n_envs > 0 && e == cudaSuccess) {
        const cudaMemcpyKind k = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        e = cudaMemcpyAsync(b.ids, scene_ids, sizeof(int32_t) * n_envs, k, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b.first_push, first_push, sizeof(float4) * n_envs, k, ctx->stream);
        if (e == cudaSuccess && seeds) e = cudaMemcpyAsync(b.seeds, seeds, sizeof(uint64_t) * n_envs, k, ctx->stream);
        if (e == cudaSuccess) {
            prepare_batch_kernel<<<1, 1024, 0, ctx->stream>>>(n_envs, b.ids, ctx->d_table, kSceneTableCap, b.env,
                                                              b.order, b.counters);
            e = cudaGetLastError();
        }
        // host-submitted ids: the copies read pageable memory, so wait for them here
        if (e == cudaSuccess && !device_ptrs) e = cudaStreamSynchronize(ctx->stream);
    }
    if (e != cudaSuccess) return bail("batch set-up", e);
    if (!device_ptrs) {
        b.scene_ids.assign(scene_ids, scene_ids + n_envs);
        for (int s : b.scene_ids) ctx->scenes[s].uses++;
    }
    b.finished = n_envs == 0;
    b.stream = ctx->stream;
    choose_shape(ctx, nb, b.G, b.wpb, b.Ms);
    {
        const auto t = ctx->tuned_tile.find(shape_bucket(nb));
        b.tile = ctx->fixed_tile >= 0 ? ctx->fixed_tile : (t != ctx->tuned_tile.end() ? t->second : 0);
    }
    const int64_t id = ctx->next_batch++;
    ctx->batches[id] = b;
    *out_batch = id;
    return PMBS_OK;
}

pmbs_status launch_rollout_once(pmbs_ctx* ctx, Batch& b, int max_substeps, cudaStream_t stream);

// A launch of the whole rollout (max_substeps <= 0) follows the batch's iteration tiling:
// one persistent launch, or launches of `tile` substeps each (every environment advances
// by up to `tile` substeps per launch; results are the same either way).
pmbs_status launch_rollout(pmbs_ctx* ctx, Batch& b, int max_substeps, cudaStream_t stream) {
    if (max_substeps > 0 || b.tile <= 0) return launch_rollout_once(ctx, b, max_substeps, stream);
    const long total = (long)b.depth * ctx->cfg.substeps_per_push;
    const long launches = (total + b.tile - 1) / b.tile;
    for (long i = 0; i < launches; i++) {
        const pmbs_status st = launch_rollout_once(ctx, b, b.tile, stream);
        if (st != PMBS_OK) return st;
    }
    return PMBS_OK;
}

pmbs_status launch_rollout_once(pmbs_ctx* ctx, Batch& b, int max_substeps, cudaStream_t stream) {
    const pmbs_config& c = ctx->cfg;
    const int nb = b.nb;
    const int pairS = std::min(c.pair_cap, std::max(1, nb * (nb - 1) / 2));
    const Layout L = make_layout(nb, pairS, b.Ms, c.manifold_cap);
    const int K = 32 / b.G;
    const int threads = 32 * b.wpb;
    const size_t smem = (size_t)L.bytes * b.wpb * K;
    int per_sm = 0;
    const RolloutFn kern = rollout_fn(b.cyl, b.warm != nullptr);
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern,
                                                     threads, smem));
    if (per_sm < 1) return fail(ctx, PMBS_E_INVALID, "launch shape does not fit on an SM");
    per_sm = std::min(per_sm, kMaxWarpsPerSM / b.wpb);
    const int per_block = b.wpb * K;
    const int blocks = std::max(1, std::min((b.n_envs + per_block - 1) / per_block, per_sm * ctx->num_sms));
    const size_t slot_bytes = (size_t)scratch_f4_per_warp(c.manifold_cap) * sizeof(float4);
    float4* scratch = nullptr;
    if (b.own_scratch) {
        const size_t need = (size_t)blocks * per_block * slot_bytes;
        if (need > b.scr_bytes) {
            if (b.scr_bytes) ctx->arena.release(b.scr_off, b.scr_bytes);
            b.scr_bytes = 0;
            const size_t off = ctx->arena.alloc(need);
            if (off == SIZE_MAX) return fail(ctx, PMBS_E_OOM, "batch scratch does not fit in the arena");
            b.scr_off = off;
            b.scr_bytes = need;
        }
        scratch = (float4*)arena_ptr(ctx, b.scr_off);
    } else {
        const pmbs_status st = ensure_scratch(ctx, (size_t)blocks * per_block);
        if (st != PMBS_OK) return st;
        scratch = ctx->gscratch;
    }
    RolloutArgs a;
    a.C = ctx->C;
    a.L = L;
    a.G = b.G;
    a.n_envs = b.n_envs;
    a.depth = b.depth;
    a.max_substeps = max_substeps;
    a.child_on = 1;
    a.env = b.env;
    a.order = b.order;
    a.queue_head = b.counters + 2;
    a.done_count = b.counters + 3;
    a.first_push = b.first_push;
    a.seeds = b.seeds;
    a.prog = b.prog;
    a.state = b.state;
    a.child = b.child;
    a.cost = b.cost;
    a.reward = b.reward;
    a.flags = b.flags;
    a.steps = b.steps;
    a.events = b.events;
    a.gscratch = scratch;
    a.scratch_f4_per_warp = scratch_f4_per_warp(c.manifold_cap);
    a.watchdog_cycles = (long long)((double)c.watchdog_ms * 2.0e6);  // SM cycles at up to 2 GHz
    a.watchdog_flag = b.counters + 4;
    a.warm = b.warm;
    a.warm_f4_per_env = (size_t)kWarmF4 * c.manifold_cap;
    a.phase = b.phase;
    a.n_rows = (long long)b.state_boxes;
    CU(cudaMemsetAsync(b.counters + 2, 0, sizeof(int), stream));
    kern<<<blocks, threads, smem, stream>>>(a);
    CU(cudaGetLastError());
    return PMBS_OK;
}

Batch* find_batch(pmbs_ctx* ctx, int64_t id) {
    auto it = ctx->batches.find(id);
    return it == ctx->batches.end() ? nullptr : &it->second;
}

// Copy the records of n_scenes scenes into one arena block, validate them (deepest initial
// box-box penetration, on the device) when asked, then assign ids and publish the
// descriptors to the device scene table (one copy of the records, one scatter).
pmbs_status register_scenes(pmbs_ctx* ctx, int n_scenes, const int32_t* box_offset, const float* rec_host,
                            const int32_t* target, int32_t* out_ids, bool check_penetration) {
    const int total = box_offset[n_scenes] - box_offset[0];
    const size_t rec_bytes = sizeof(float) * kRecFloats * (size_t)std::max(total, 1);
    const size_t meta = sizeof(int32_t) * n_scenes, meta_al = (meta + 255) & ~(size_t)255;
    const size_t desc_bytes = sizeof(SceneDesc) * n_scenes;
    const size_t pen_bytes = sizeof(float) * n_scenes, pen_al = (pen_bytes + 255) & ~(size_t)255;
    const size_t rec_al = (rec_bytes + 255) & ~(size_t)255;
    // block layout: records | staging ids (also the CSR offsets for validation) | staging
    // descriptors | penetration per scene (staging is reused per call)
    const size_t off_bytes = sizeof(int32_t) * (n_scenes + 1), off_al = (off_bytes + 255) & ~(size_t)255;
    const size_t stage = std::max(meta_al, off_al);
    const size_t bytes = rec_al + stage + ((desc_bytes + 255) & ~(size_t)255) + pen_al;
    const size_t off = ctx->arena.alloc(bytes);
    if (off == SIZE_MAX) return fail(ctx, PMBS_E_OOM, "scene store is full");
    char* base = (char*)arena_ptr(ctx, off);
    char* stage_p = base + rec_al;
    char* desc_p = stage_p + stage;
    float* pen_p = (float*)(desc_p + ((desc_bytes + 255) & ~(size_t)255));
    cudaError_t e = cudaMemcpyAsync(base, rec_host, sizeof(float) * kRecFloats * (size_t)total,
                                    cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess && check_penetration && n_scenes > 0) {
        std::vector<float> pen(n_scenes, 0.f);
        e = cudaMemcpyAsync(stage_p, box_offset, off_bytes, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) {
            penetration_kernel<<<(n_scenes + 3) / 4, 128, 0, ctx->stream>>>(n_scenes, (const int32_t*)stage_p,
                                                                           (const float*)base, pen_p);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(pen.data(), pen_p, pen_bytes, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e == cudaSuccess)
            for (int s = 0; s < n_scenes; s++)
                if (pen[s] > ctx->cfg.max_initial_penetration) {
                    ctx->arena.release(off, bytes);
                    return fail(ctx, PMBS_E_INVALID, "scene " + std::to_string(s) + " starts with box-box penetration " +
                                                         std::to_string(pen[s]) + " m");
                }
    }
    if (e != cudaSuccess) {
        cudaStreamSynchronize(ctx->stream);
        ctx->arena.release(off, bytes);
        return fail(ctx, PMBS_E_CUDA, std::string("scene upload: ") + cudaGetErrorString(e));
    }
    std::vector<int> ids(n_scenes);
    for (int s = 0; s < n_scenes; s++) {
        int id;
        if (!ctx->free_ids.empty()) {
            id = ctx->free_ids.back();
            ctx->free_ids.pop_back();
        } else {
            id = (int)ctx->scenes.size();
            if (id >= kSceneTableCap) {
                for (int t = 0; t < s; t++) ctx->free_ids.push_back(ids[t]);
                cudaStreamSynchronize(ctx->stream);
                ctx->arena.release(off, bytes);
                return fail(ctx, PMBS_E_OOM, "scene table full");
            }
            ctx->scenes.emplace_back();
        }
        ids[s] = id;
    }
    std::vector<SceneDesc> desc(n_scenes);
    for (int s = 0; s < n_scenes; s++) {
        SceneRec& r = ctx->scenes[ids[s]];
        r.n = box_offset[s + 1] - box_offset[s];
        r.target = target[s];
        r.block = off;
        r.rec_off = off + sizeof(float) * kRecFloats * (size_t)(box_offset[s] - box_offset[0]);
        r.host.assign(rec_host + (size_t)kRecFloats * (box_offset[s] - box_offset[0]),
                      rec_host + (size_t)kRecFloats * (box_offset[s + 1] - box_offset[0]));
        r.live = true;
        r.uses = 0;
        r.cyl = false;
        for (int i = 0; i < r.n; i++) r.cyl = r.cyl || r.host[(size_t)kRecFloats * i + 14] < 0.f;
        desc[s] = SceneDesc{(const float*)arena_ptr(ctx, r.rec_off), r.n, r.target};
    }
    SceneBlock blk;
    blk.bytes = bytes;
    blk.live = n_scenes;
    ctx->blocks[off] = blk;
    CU(cudaMemcpyAsync(stage_p, ids.data(), meta, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(desc_p, desc.data(), desc_bytes, cudaMemcpyHostToDevice, ctx->stream));
    scatter_desc_kernel<<<(n_scenes + 255) / 256, 256, 0, ctx->stream>>>(n_scenes, (const int32_t*)stage_p,
                                                                         (const SceneDesc*)desc_p, ctx->d_table);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(ctx->stream));
    for (int s = 0; s < n_scenes; s++) out_ids[s] = ids[s];
    return PMBS_OK;
}

pmbs_status eval_common(pmbs_ctx* ctx, int mode, int n_envs, const int32_t* box_offset, const float* states,
                        const float* half, const float* pusher_xy, const int32_t* target, const uint64_t* seeds,
                        int k, const float* starts, int32_t* out_pairs, int32_t* out_n_pairs, int32_t* out_plane,
                        int32_t* out_n_plane, int32_t* out_pusher, int32_t* out_n_pusher, uint8_t* out_u8,
                        float* out_push, int32_t* out_attempt) {
    if (n_envs < 0 || !box_offset || !states || !half) return fail(ctx, PMBS_E_INVALID, "bad arguments");
    if (n_envs == 0) return PMBS_OK;
    int nb = 1;
    for (int e = 0; e < n_envs; e++) {
        const int n = box_offset[e + 1] - box_offset[e];
        if (n < 1 || n > kMaxBoxes) return fail(ctx, PMBS_E_INVALID, "box count out of range");
        nb = std::max(nb, n);
    }
    const int B = box_offset[n_envs] - box_offset[0];
    const pmbs_config& c = ctx->cfg;
    std::vector<int32_t> off(box_offset, box_offset + n_envs + 1);
    for (auto& o : off) o -= box_offset[0];
    // device staging in one arena block
    size_t sz = 0;
    auto take = [&](size_t bytes) {
        const size_t o = sz;
        sz += (bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_off = take(sizeof(int32_t) * (n_envs + 1)), o_st = take(sizeof(float) * 13 * B),
                 o_h = take(sizeof(float) * 3 * B), o_pxy = take(sizeof(float) * 2 * n_envs),
                 o_t = take(sizeof(int32_t) * n_envs), o_seed = take(sizeof(uint64_t) * n_envs),
                 o_st2 = take(sizeof(float) * 2 * n_envs),
                 o_pairs = take(sizeof(int32_t) * 2 * (size_t)c.pair_cap * n_envs),
                 o_np = take(sizeof(int32_t) * 3 * n_envs), o_pl = take(sizeof(int32_t) * 2 * B),
                 o_u8 = take(n_envs), o_push = take(sizeof(float) * 4 * n_envs), o_at = take(sizeof(int32_t) * n_envs);
    const size_t boff = ctx->arena.alloc(sz);
    if (boff == SIZE_MAX) return fail(ctx, PMBS_E_OOM, "evaluation staging does not fit");
    char* base = (char*)arena_ptr(ctx, boff);
    auto h2d = [&](size_t o, const void* src, size_t bytes) {
        return cudaMemcpyAsync(base + o, src, bytes, cudaMemcpyHostToDevice, ctx->stream);
    };
    cudaError_t e = h2d(o_off, off.data(), sizeof(int32_t) * (n_envs + 1));
    if (e == cudaSuccess) e = h2d(o_st, states, sizeof(float) * 13 * B);
    if (e == cudaSuccess) e = h2d(o_h, half, sizeof(float) * 3 * B);
    if (e == cudaSuccess && pusher_xy) e = h2d(o_pxy, pusher_xy, sizeof(float) * 2 * n_envs);
    if (e == cudaSuccess && target) e = h2d(o_t, target, sizeof(int32_t) * n_envs);
    if (e == cudaSuccess && seeds) e = h2d(o_seed, seeds, sizeof(uint64_t) * n_envs);
    if (e == cudaSuccess && starts) e = h2d(o_st2, starts, sizeof(float) * 2 * n_envs);
    EvalArgs a;
    a.C = ctx->C;
    a.L = make_layout(nb, c.pair_cap, 0, 1);
    a.n_envs = n_envs;
    a.mode = mode;
    a.k = k;
    a.box_offset = (int32_t*)(base + o_off);
    a.states = (float*)(base + o_st);
    a.half = (float*)(base + o_h);
    a.pusher_xy = pusher_xy ? (float*)(base + o_pxy) : nullptr;
    a.target = (int32_t*)(base + o_t);
    a.seeds = (uint64_t*)(base + o_seed);
    a.starts = (float*)(base + o_st2);
    a.out_pairs = (int32_t*)(base + o_pairs);
    a.out_n_pairs = (int32_t*)(base + o_np);
    a.out_n_plane = a.out_n_pairs + n_envs;
    a.out_n_pusher = a.out_n_pairs + 2 * n_envs;
    a.out_plane = (int32_t*)(base + o_pl);
    a.out_pusher = a.out_plane + B;
    a.out_u8 = (uint8_t*)(base + o_u8);
    a.out_push = (float*)(base + o_push);
    a.out_attempt = (int32_t*)(base + o_at);
    if (e == cudaSuccess) {
        const int wpb = 4;
        const int blocks = std::min((n_envs + wpb - 1) / wpb, 4 * ctx->num_sms);
        eval_kernel<<<blocks, 32 * wpb, (size_t)a.L.bytes * wpb, ctx->stream>>>(a);
        e = cudaGetLastError();
    }
    auto d2h = [&](void* dst, size_t o, size_t bytes) {
        return cudaMemcpyAsync(dst, base + o, bytes, cudaMemcpyDeviceToHost, ctx->stream);
    };
    if (e == cudaSuccess && mode == 0) {
        if (out_pairs) e = d2h(out_pairs, o_pairs, sizeof(int32_t) * 2 * (size_t)c.pair_cap * n_envs);
        if (e == cudaSuccess && out_n_pairs) e = d2h(out_n_pairs, o_np, sizeof(int32_t) * n_envs);
        if (e == cudaSuccess && out_n_plane) e = d2h(out_n_plane, o_np + sizeof(int32_t) * n_envs, sizeof(int32_t) * n_envs);
        if (e == cudaSuccess && out_n_pusher)
            e = d2h(out_n_pusher, o_np + 2 * sizeof(int32_t) * n_envs, sizeof(int32_t) * n_envs);
        if (e == cudaSuccess && out_plane) e = d2h(out_plane, o_pl, sizeof(int32_t) * B);
        if (e == cudaSuccess && out_pusher) e = d2h(out_pusher, o_pl + sizeof(int32_t) * B, sizeof(int32_t) * B);
    } else if (e == cudaSuccess && (mode == 1 || mode == 3)) {
        if (out_u8) e = d2h(out_u8, o_u8, n_envs);
    } else if (e == cudaSuccess && mode == 2) {
        if (out_push) e = d2h(out_push, o_push, sizeof(float) * 4 * n_envs);
        if (e == cudaSuccess && out_attempt) e = d2h(out_attempt, o_at, sizeof(int32_t) * n_envs);
    }
    const cudaError_t es = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = es;
    ctx->arena.release(boff, sz);
    if (e != cudaSuccess) return fail(ctx, PMBS_E_CUDA, std::string("evaluation: ") + cudaGetErrorString(e));
    return PMBS_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

void pmbs_default_config(pmbs_config* c) {
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->device = 0;
    c->max_envs = 1 << 16;
    c->max_boxes_per_env = 64;
    c->mem_budget_bytes = (size_t)4 << 30;
    c->dt = 1.f / 240.f;
    c->substeps_per_push = 240;
    c->pgs_iters = 10;
    c->gravity[0] = 0.f;
    c->gravity[1] = 0.f;
    c->gravity[2] = -9.81f;
    c->table_half[0] = 0.2f;
    c->table_half[1] = 0.2f;
    c->table_mu = 0.5f;
    c->pusher_mu = 0.5f;
    c->pusher_radius = 0.01f;
    c->pusher_z0 = 0.01f;
    c->pusher_z1 = 0.20f;
    c->pusher_speed = 0.1f;
    c->push_length = 0.1f;
    c->gamma = 0.8f;
    c->grasp_opening = 0.085f;
    c->grasp_clearance = 0.002f;
    c->finger_depth = 0.01f;
    c->finger_width = 0.022f;
    c->grasp_angles = 16;
    c->margin = 1e-3f;
    c->slop = 5e-4f;
    c->baumgarte = 0.2f;
    c->sample_clearance = 0.005f;
    c->sample_attempts = 8;
    c->contour_points = 16;
    c->contact_cap = 512;
    c->manifold_cap = 256;
    c->pair_cap = 1024;
    c->lanes_per_env = 0;
    c->warps_per_block = 0;
    c->smem_points = -1;
    c->smem_manifolds = -1;
    c->watchdog_ms = 10000.f;
    c->max_initial_penetration = 1e-3f;
    c->warm_start = 0;
    c->warm_tolerance = 2e-3f;
}

pmbs_status pmbs_create(const pmbs_config* cfg, void* cuda_stream, pmbs_ctx** out) {
    return create_common(cfg, cuda_stream, nullptr, 0, out);
}

pmbs_status pmbs_create_with_arena(const pmbs_config* cfg, void* cuda_stream, void* d_arena, size_t arena_bytes,
                                   pmbs_ctx** out) {
    if (!d_arena || arena_bytes < ((size_t)32 << 20)) return PMBS_E_INVALID;
    return create_common(cfg, cuda_stream, d_arena, arena_bytes, out);
}

void pmbs_destroy(pmbs_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto& kv : ctx->batches)
        if (kv.second.graph) cudaGraphExecDestroy(kv.second.graph);
    if (ctx->own_arena && ctx->arena.base) cudaFree(ctx->arena.base);
    delete ctx;
}

const char* pmbs_last_error(const pmbs_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

pmbs_status pmbs_load_scenes(pmbs_ctx* ctx, int n_scenes, const int32_t* box_offset, const float* pose,
                             const float* vel, const float* half_ext, const float* mass, const float* mu,
                             const int32_t* target, int32_t* out_scene_ids) {
    NvtxRange nvtx_("pmbs_load_scenes");
    if (!ctx) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    if (n_scenes < 0 || (n_scenes > 0 && (!box_offset || !pose || !half_ext || !mass || !mu || !target || !out_scene_ids)))
        return fail(ctx, PMBS_E_INVALID, "missing scene array");
    if (n_scenes == 0) return PMBS_OK;
    CU(cudaSetDevice(ctx->device));
    const int b0 = box_offset[0];
    for (int s = 0; s < n_scenes; s++) {
        const int n = box_offset[s + 1] - box_offset[s];
        if (n < 1 || n > ctx->cfg.max_boxes_per_env)
            return fail(ctx, PMBS_E_INVALID, "scene " + std::to_string(s) + " has " + std::to_string(n) + " boxes");
        if (target[s] < 0 || target[s] >= n) return fail(ctx, PMBS_E_INVALID, "target out of range");
    }
    const int total = box_offset[n_scenes] - b0;
    std::vector<float> rec((size_t)kRecFloats * total);
    for (int i = 0; i < total; i++) {
        const float* p = pose + 7 * (size_t)(b0 + i);
        const float* h = half_ext + 3 * (size_t)(b0 + i);
        float* r = rec.data() + (size_t)kRecFloats * i;
        for (int k = 0; k < 7; k++) r[k] = p[k];
        for (int k = 0; k < 6; k++) r[7 + k] = vel ? vel[6 * (size_t)(b0 + i) + k] : 0.f;
        r[13] = h[0];
        r[14] = h[1];
        r[15] = h[2];
        r[16] = mass[b0 + i];
        r[17] = mu[b0 + i];
        for (int k = 0; k < kRecFloats; k++)
            if (!finite(r[k])) return fail(ctx, PMBS_E_INVALID, "non-finite scene value");
        const double qn = std::sqrt((double)r[3] * r[3] + (double)r[4] * r[4] + (double)r[5] * r[5] + (double)r[6] * r[6]);
        if (std::fabs(qn - 1.0) > 1e-3) return fail(ctx, PMBS_E_INVALID, "quaternion is not unit length");
        // a box has three positive half extents; a cylinder of radius r and half height h
        // is the row (r, -r, h)
        const bool cyl = h[1] < 0 && h[1] == -h[0];
        if (!(h[0] > 0 && (h[1] > 0 || cyl) && h[2] > 0) || !(r[16] > 0) || !(r[17] >= 0))
            return fail(ctx, PMBS_E_INVALID, "non-positive half extent or mass, or negative friction");
    }
    return register_scenes(ctx, n_scenes, box_offset, rec.data(), target, out_scene_ids, true);
}

pmbs_status pmbs_free_scenes(pmbs_ctx* ctx, int n, const int32_t* scene_ids) {
    if (!ctx) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    if (n < 0 || (n > 0 && !scene_ids)) return fail(ctx, PMBS_E_INVALID, "bad arguments");
    for (int i = 0; i < n; i++) {
        const int s = scene_ids[i];
        if (s < 0 || s >= (int)ctx->scenes.size() || !ctx->scenes[s].live)
            return fail(ctx, PMBS_E_INVALID, "unknown scene id " + std::to_string(s));
        if (ctx->scenes[s].uses > 0) return fail(ctx, PMBS_E_BUSY, "scene in use by a batch");
    }
    CU(cudaSetDevice(ctx->device));
    CU(cudaStreamSynchronize(ctx->stream));
    std::vector<int32_t> ids;
    for (int i = 0; i < n; i++) {
        SceneRec& r = ctx->scenes[scene_ids[i]];
        if (!r.live) continue;
        r.live = false;
        r.host.clear();
        r.host.shrink_to_fit();
        ids.push_back(scene_ids[i]);
        auto it = ctx->blocks.find(r.block);
        if (it != ctx->blocks.end() && --it->second.live == 0) {
            ctx->arena.release(it->first, it->second.bytes);
            ctx->blocks.erase(it);
        }
    }
    if (!ids.empty()) {
        const size_t nb = ids.size();
        const size_t meta_al = (sizeof(int32_t) * nb + 255) & ~(size_t)255;
        const size_t off = ctx->arena.alloc(meta_al + sizeof(SceneDesc) * nb);
        if (off == SIZE_MAX) return fail(ctx, PMBS_E_OOM, "no room to update the scene table");
        char* base = (char*)arena_ptr(ctx, off);
        std::vector<SceneDesc> z(nb, SceneDesc{nullptr, 0, 0});
        cudaError_t e = cudaMemcpyAsync(base, ids.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(base + meta_al, z.data(), sizeof(SceneDesc) * nb, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) {
            scatter_desc_kernel<<<(int)((nb + 255) / 256), 256, 0, ctx->stream>>>((int)nb, (const int32_t*)base,
                                                                                 (const SceneDesc*)(base + meta_al),
                                                                                 ctx->d_table);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        ctx->arena.release(off, meta_al + sizeof(SceneDesc) * nb);
        if (e != cudaSuccess) return fail(ctx, PMBS_E_CUDA, std::string("free scenes: ") + cudaGetErrorString(e));
        for (int32_t id : ids) ctx->free_ids.push_back(id);
    }
    return PMBS_OK;
}

pmbs_status pmbs_rollout_pushes(pmbs_ctx* ctx, int n_envs, const int32_t* scene_ids, const float* first_push,
                                int depth, const uint64_t* seeds, int64_t* out_batch) {
    NvtxRange nvtx_("pmbs_rollout_pushes");
    if (!ctx) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    CU(cudaSetDevice(ctx->device));
    return rollout_common(ctx, n_envs, scene_ids, first_push, depth, seeds, false, out_batch);
}

pmbs_status pmbs_rollout_pushes_device(pmbs_ctx* ctx, int n_envs, const int32_t* d_scene_ids,
                                       const float* d_first_push, int depth, const uint64_t* d_seeds,
                                       int64_t* out_batch) {
    if (!ctx) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    CU(cudaSetDevice(ctx->device));
    return rollout_common(ctx, n_envs, d_scene_ids, d_first_push, depth, d_seeds, true, out_batch);
}

pmbs_status pmbs_step(pmbs_ctx* ctx, int64_t batch, int max_substeps) {
    NvtxRange nvtx_("pmbs_step");
    if (!ctx) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    Batch* b = find_batch(ctx, batch);
    if (!b) return fail(ctx, PMBS_E_INVALID, "unknown batch");
    if (b->finished) return PMBS_OK;
    CU(cudaSetDevice(ctx->device));
    const pmbs_status st = launch_rollout(ctx, *b, max_substeps, b->stream);
    if (st != PMBS_OK) return st;
    if (max_substeps <= 0) {
        b->finished = true;
        return PMBS_OK;
    }
    int cnt[5] = {0, 0, 0, 0, 0};
    CU(cudaMemcpyAsync(cnt, b->counters, sizeof(cnt), cudaMemcpyDeviceToHost, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    if (cnt[1]) return fail(ctx, PMBS_E_INVALID, "the batch names an unknown scene id");
    if (cnt[4]) {
        // the stopped environments kept their progress: clear the flag so that the next
        // call resumes them
        CU(cudaMemsetAsync(b->counters + 4, 0, sizeof(int), b->stream));
        return fail(ctx, PMBS_E_TIMEOUT, "an environment exceeded the per-launch time limit");
    }
    const int done = cnt[3];
    if (done >= b->n_envs) {
        b->finished = true;
        return PMBS_OK;
    }
    return PMBS_E_NOT_READY;
}

pmbs_status pmbs_step_graph(pmbs_ctx* ctx, int64_t batch, int substeps_per_launch) {
    NvtxRange nvtx_("pmbs_step_graph");
    if (!ctx) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    Batch* b = find_batch(ctx, batch);
    if (!b) return fail(ctx, PMBS_E_INVALID, "unknown batch");
    if (substeps_per_launch < 1) return fail(ctx, PMBS_E_INVALID, "substeps_per_launch must be >= 1");
    if (b->finished) return PMBS_OK;
    CU(cudaSetDevice(ctx->device));
    if (!b->graph || b->graph_k != substeps_per_launch) {
        if (b->graph) cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        // capture on a private stream (the legacy default stream cannot be captured)
        cudaStream_t cs;
        CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        const long total = (long)b->depth * ctx->cfg.substeps_per_push;
        const long launches = (total + substeps_per_launch - 1) / substeps_per_launch;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        pmbs_status st = PMBS_OK;
        for (long i = 0; i < launches && e == cudaSuccess && st == PMBS_OK; i++)
            st = launch_rollout(ctx, *b, substeps_per_launch, cs);
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess && st == PMBS_OK) e = cudaGraphInstantiate(&b->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        if (st != PMBS_OK) return st;
        if (e != cudaSuccess) return fail(ctx, PMBS_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        b->graph_k = substeps_per_launch;
    }
    CU(cudaGraphLaunch(b->graph, b->stream));
    b->finished = true;
    return PMBS_OK;
}

pmbs_status pmbs_autotune(pmbs_ctx* ctx, int n_envs, const int32_t* scene_ids, const float* first_push, int depth,
                          const uint64_t* seeds, int substeps, int32_t* out_lanes_per_env, int32_t* out_warps_per_block,
                          int32_t* out_smem_manifolds, float* out_ms, int32_t* out_substeps_per_launch) {
    NvtxRange nvtx_("pmbs_autotune");
    if (!ctx) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    if (n_envs < 1 || substeps < 1) return fail(ctx, PMBS_E_INVALID, "need environments and substeps to time");
    CU(cudaSetDevice(ctx->device));
    int nb = 1;
    for (int e = 0; e < n_envs; e++) {
        const int sid = scene_ids[e];
        if (sid < 0 || sid >= (int)ctx->scenes.size() || !ctx->scenes[sid].live)
            return fail(ctx, PMBS_E_INVALID, "unknown scene id");
        nb = std::max(nb, ctx->scenes[sid].n);
    }
    const int saved[4] = {ctx->fixed_G, ctx->fixed_wpb, ctx->fixed_Ps, ctx->fixed_Ms};
    ctx->tuned.erase(shape_bucket(nb));
    ctx->tuned_tile.erase(shape_bucket(nb));
    const int Gs[3] = {32, 16, 8}, Ws[3] = {4, 2, 1}, Mss[4] = {0, 8, 16, 40};
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    pmbs_status result = PMBS_OK;
    // time one candidate: best of two freshly built batches (identical work), advancing
    // every environment by up to `steps` substeps (0: the whole rollout)
    auto time_shape = [&](int G, int wpb, int Ms, int steps, float& ms, int& used_Ms) {
        ctx->fixed_G = G;
        ctx->fixed_wpb = wpb;
        ctx->fixed_Ps = -1;
        ctx->fixed_Ms = Ms;
        ms = 1e30f;
        cudaError_t e = cudaSuccess;
        for (int rep = 0; rep < 2 && e == cudaSuccess && result == PMBS_OK; rep++) {
            int64_t id = 0;
            result = rollout_common(ctx, n_envs, scene_ids, first_push, depth, seeds, false, &id);
            if (result != PMBS_OK) break;
            Batch& b = ctx->batches[id];
            float t = 0.f;
            e = cudaEventRecord(e0, b.stream);
            if (e == cudaSuccess) result = launch_rollout(ctx, b, steps, b.stream);
            if (e == cudaSuccess && result == PMBS_OK) e = cudaEventRecord(e1, b.stream);
            if (e == cudaSuccess && result == PMBS_OK) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess && result == PMBS_OK) e = cudaEventElapsedTime(&t, e0, e1);
            used_Ms = b.Ms;
            release_batch_mem(ctx, b);
            ctx->batches.erase(id);
            ms = std::min(ms, t);
        }
        if (e != cudaSuccess) result = fail(ctx, PMBS_E_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
    };
    // screening on the first `substeps` substeps, then the fastest shapes timed over
    // the whole rollout (a batch's time follows its longest environments, which the first
    // push alone does not rank reliably)
    std::vector<std::pair<float, std::array<int, 3>>> screen;
    for (int gi = 0; gi < 3 && result == PMBS_OK; gi++)
        for (int wi = 0; wi < 3 && result == PMBS_OK; wi++)
            for (int mi = 0; mi < 4 && result == PMBS_OK; mi++) {
                float ms = 0.f;
                int used = -1;
                time_shape(Gs[gi], Ws[wi], Mss[mi], substeps, ms, used);
                if (result == PMBS_OK) screen.push_back({ms, {Gs[gi], Ws[wi], used}});
            }
    std::sort(screen.begin(), screen.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
    // whole-rollout finalists: the five fastest screened shapes and the default shape (one
    // environment per warp, two warps per block, eight shared manifolds), which the
    // screening has been seen to rank too low
    std::vector<std::array<int, 3>> finalists;
    for (size_t k = 0; k < std::min<size_t>(5, screen.size()); k++) finalists.push_back(screen[k].second);
    const std::array<int, 3> dflt = {32, 2, 8};
    if (std::find(finalists.begin(), finalists.end(), dflt) == finalists.end()) finalists.push_back(dflt);
    float best_ms = 1e30f;
    std::array<int, 3> best = {32, 4, -1};
    const int saved_tile = ctx->fixed_tile;
    ctx->fixed_tile = 0;
    for (size_t k = 0; k < finalists.size() && result == PMBS_OK; k++) {
        float ms = 0.f;
        int used = -1;
        const auto& sh = finalists[k];
        time_shape(sh[0], sh[1], sh[2], 0, ms, used);
        if (result == PMBS_OK && ms < best_ms) {
            best_ms = ms;
            best = {sh[0], sh[1], used};
        }
    }
    // iteration tiling of the chosen shape: one persistent launch, or launches of one push
    // or a quarter push each
    int best_tile = 0;
    const int tiles[2] = {ctx->cfg.substeps_per_push, std::max(1, ctx->cfg.substeps_per_push / 4)};
    for (int k = 0; k < 2 && result == PMBS_OK; k++) {
        ctx->fixed_tile = tiles[k];
        float ms = 0.f;
        int used = -1;
        time_shape(best[0], best[1], best[2], 0, ms, used);
        if (result == PMBS_OK && ms < best_ms) {
            best_ms = ms;
            best_tile = tiles[k];
        }
    }
    ctx->fixed_tile = saved_tile;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->fixed_G = saved[0];
    ctx->fixed_wpb = saved[1];
    ctx->fixed_Ps = saved[2];
    ctx->fixed_Ms = saved[3];
    if (result != PMBS_OK) return result;
    ctx->tuned[shape_bucket(nb)] = best;
    ctx->tuned_tile[shape_bucket(nb)] = best_tile;
    if (out_lanes_per_env) *out_lanes_per_env = best[0];
    if (out_warps_per_block) *out_warps_per_block = best[1];
    if (out_smem_manifolds) *out_smem_manifolds = best[2];
    if (out_ms) *out_ms = best_ms;
    if (out_substeps_per_launch) *out_substeps_per_launch = best_tile;
    return PMBS_OK;
}

pmbs_status pmbs_query_cost(pmbs_ctx* ctx, int64_t batch, int32_t* out_cost, float* out_reward, uint8_t* out_flags,
                            float* out_child_states, int32_t* out_child_scene_ids) {
    NvtxRange nvtx_("pmbs_query_cost");
    if (!ctx) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    Batch* b = find_batch(ctx, batch);
    if (!b) return fail(ctx, PMBS_E_INVALID, "unknown batch");
    CU(cudaSetDevice(ctx->device));
    CU(cudaStreamSynchronize(ctx->stream));
    if (!b->finished) return fail(ctx, PMBS_E_NOT_READY, "batch not finished");
    const int n = b->n_envs;
    if (n == 0) return PMBS_OK;
    int cnt[5] = {0, 0, 0, 0, 0};
    CU(cudaMemcpyAsync(cnt, b->counters, sizeof(cnt), cudaMemcpyDeviceToHost, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    if (cnt[1]) return fail(ctx, PMBS_E_INVALID, "the batch names an unknown scene id");
    if (cnt[3] < n) {
        // environments stopped by the watchdog kept their progress; pmbs_step resumes them
        b->finished = false;
        CU(cudaMemsetAsync(b->counters + 4, 0, sizeof(int), b->stream));
        return fail(ctx, PMBS_E_TIMEOUT, std::to_string(n - cnt[3]) + " environments exceeded the per-launch time limit");
    }
    if (out_cost) CU(cudaMemcpyAsync(out_cost, b->cost, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, ctx->stream));
    if (out_reward) CU(cudaMemcpyAsync(out_reward, b->reward, sizeof(float) * n, cudaMemcpyDeviceToHost, ctx->stream));
    if (out_flags) CU(cudaMemcpyAsync(out_flags, b->flags, n, cudaMemcpyDeviceToHost, ctx->stream));
    std::vector<float> child;
    std::vector<EnvIn> env;
    if (out_child_states || out_child_scene_ids) {
        env.resize(n);
        CU(cudaMemcpyAsync(env.data(), b->env, sizeof(EnvIn) * n, cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        int total = 0;
        for (const EnvIn& e : env) total += e.n;
        child.resize((size_t)13 * std::max(total, 1));
        CU(cudaMemcpyAsync(child.data(), b->child, sizeof(float) * 13 * total, cudaMemcpyDeviceToHost, ctx->stream));
    }
    CU(cudaStreamSynchronize(ctx->stream));
    if (out_child_states && !child.empty()) std::memcpy(out_child_states, child.data(), sizeof(float) * (child.size()));
    if (out_child_scene_ids) {
        // register each env's state after push 1 as a new scene (statics from the parent)
        std::vector<int32_t> off(n + 1, 0), tgt(n);
        for (int e = 0; e < n; e++) {
            off[e + 1] = off[e] + env[e].n;
            tgt[e] = env[e].target;
        }
        std::vector<float> rec((size_t)kRecFloats * off[n]);
        for (int e = 0; e < n; e++) {
            const SceneRec* parent = (env[e].scene >= 0 && env[e].scene < (int)ctx->scenes.size())
                                         ? &ctx->scenes[env[e].scene] : nullptr;
            for (int i = 0; i < env[e].n; i++) {
                float* r = rec.data() + (size_t)kRecFloats * (off[e] + i);
                const float* s = child.data() + (size_t)13 * (env[e].box_off + i);
                for (int k = 0; k < 13; k++) r[k] = s[k];
                for (int k = 13; k < kRecFloats; k++)
                    r[k] = (parent && parent->live) ? parent->host[(size_t)kRecFloats * i + k] : 1.f;
            }
        }
        // child states come out of the solver and may rest within the contact slop
        const pmbs_status st = register_scenes(ctx, n, off.data(), rec.data(), tgt.data(), out_child_scene_ids, false);
        if (st != PMBS_OK) return st;
    }
    return PMBS_OK;
}

pmbs_status pmbs_query_cost_device(pmbs_ctx* ctx, int64_t batch, int32_t* d_cost, float* d_reward, uint8_t* d_flags) {
    if (!ctx) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    Batch* b = find_batch(ctx, batch);
    if (!b) return fail(ctx, PMBS_E_INVALID, "unknown batch");
    if (!b->finished) return fail(ctx, PMBS_E_NOT_READY, "batch not finished");
    const int n = b->n_envs;
    if (n == 0) return PMBS_OK;
    CU(cudaSetDevice(ctx->device));
    if (d_cost) CU(cudaMemcpyAsync(d_cost, b->cost, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    if (d_reward) CU(cudaMemcpyAsync(d_reward, b->reward, sizeof(float) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    if (d_flags) CU(cudaMemcpyAsync(d_flags, b->flags, n, cudaMemcpyDeviceToDevice, ctx->stream));
    return PMBS_OK;
}

pmbs_status pmbs_query_states(pmbs_ctx* ctx, int64_t batch, float* out_states, int32_t* out_env_steps) {
    if (!ctx) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    Batch* b = find_batch(ctx, batch);
    if (!b) return fail(ctx, PMBS_E_INVALID, "unknown batch");
    CU(cudaSetDevice(ctx->device));
    const int n = b->n_envs;
    if (n == 0) return PMBS_OK;
    int total = 0;
    CU(cudaMemcpyAsync(&total, b->counters, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    // environments that have not started yet still hold their scene's initial state
    std::vector<EnvProg> prog(n);
    std::vector<EnvIn> env(n);
    CU(cudaMemcpyAsync(prog.data(), b->prog, sizeof(EnvProg) * n, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(env.data(), b->env, sizeof(EnvIn) * n, cudaMemcpyDeviceToHost, ctx->stream));
    if (out_env_steps) CU(cudaMemcpyAsync(out_env_steps, b->steps, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, ctx->stream));
    if (out_states) CU(cudaMemcpyAsync(out_states, b->state, sizeof(float) * 13 * total, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (out_states) {
        for (int e = 0; e < n; e++) {
            if (prog[e].k != 0) continue;
            const SceneRec* r = (env[e].scene >= 0 && env[e].scene < (int)ctx->scenes.size()) ? &ctx->scenes[env[e].scene] : nullptr;
            if (!r || !r->live) continue;
            for (int i = 0; i < env[e].n; i++)
                for (int k = 0; k < 13; k++)
                    out_states[(size_t)13 * (env[e].box_off + i) + k] = r->host[(size_t)kRecFloats * i + k];
        }
    }
    return PMBS_OK;
}

pmbs_status pmbs_query_events(pmbs_ctx* ctx, int64_t batch, uint64_t* out_events) {
    if (!ctx) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    Batch* b = find_batch(ctx, batch);
    if (!b || !out_events) return fail(ctx, PMBS_E_INVALID, "unknown batch or null output");
    if (b->n_envs == 0) return PMBS_OK;
    CU(cudaSetDevice(ctx->device));
    CU(cudaMemcpyAsync(out_events, b->events, sizeof(uint64_t) * kNumEvents * b->n_envs, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return PMBS_OK;
}

pmbs_status pmbs_query_phase_cycles(pmbs_ctx* ctx, int64_t batch, uint64_t* out_cycles) {
    if (!ctx) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    Batch* b = find_batch(ctx, batch);
    if (!b || !out_cycles) return fail(ctx, PMBS_E_INVALID, "unknown batch or null output");
    if (b->n_envs == 0) return PMBS_OK;
    CU(cudaSetDevice(ctx->device));
    CU(cudaMemcpyAsync(out_cycles, b->phase, sizeof(uint64_t) * kNumPhases * b->n_envs, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return PMBS_OK;
}

pmbs_status pmbs_batch_info(pmbs_ctx* ctx, int64_t batch, int32_t* out_n_envs, int32_t* out_n_boxes) {
    if (!ctx) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    Batch* b = find_batch(ctx, batch);
    if (!b) return fail(ctx, PMBS_E_INVALID, "unknown batch");
    if (out_n_envs) *out_n_envs = b->n_envs;
    if (out_n_boxes) {
        int total = 0;
        if (b->n_envs > 0) {
            CU(cudaSetDevice(ctx->device));
            CU(cudaMemcpyAsync(&total, b->counters, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
            CU(cudaStreamSynchronize(ctx->stream));
        }
        *out_n_boxes = total;
    }
    return PMBS_OK;
}

pmbs_status pmbs_release_batch(pmbs_ctx* ctx, int64_t batch) {
    if (!ctx) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    auto it = ctx->batches.find(batch);
    if (it == ctx->batches.end()) return fail(ctx, PMBS_E_INVALID, "unknown batch");
    CU(cudaSetDevice(ctx->device));
    CU(cudaStreamSynchronize(ctx->stream));
    release_batch_mem(ctx, it->second);
    ctx->batches.erase(it);
    return PMBS_OK;
}

pmbs_status pmbs_eval_pairs(pmbs_ctx* ctx, int n_envs, const int32_t* box_offset, const float* states,
                            const float* half_ext, const float* pusher_xy, int32_t* out_pairs, int32_t* out_n_pairs,
                            int32_t* out_plane, int32_t* out_n_plane, int32_t* out_pusher, int32_t* out_n_pusher) {
    if (!ctx) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    CU(cudaSetDevice(ctx->device));
    return eval_common(ctx, 0, n_envs, box_offset, states, half_ext, pusher_xy, nullptr, nullptr, 0, nullptr, out_pairs,
                       out_n_pairs, out_plane, out_n_plane, out_pusher, out_n_pusher, nullptr, nullptr, nullptr);
}

pmbs_status pmbs_eval_grasp(pmbs_ctx* ctx, int n_envs, const int32_t* box_offset, const float* states,
                            const float* half_ext, const int32_t* target, uint8_t* out_graspable) {
    if (!ctx) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    if (n_envs > 0 && !target) return fail(ctx, PMBS_E_INVALID, "missing targets");
    for (int e = 0; e < n_envs; e++)
        if (target[e] < 0 || target[e] >= box_offset[e + 1] - box_offset[e])
            return fail(ctx, PMBS_E_INVALID, "target out of range");
    CU(cudaSetDevice(ctx->device));
    return eval_common(ctx, 1, n_envs, box_offset, states, half_ext, nullptr, target, nullptr, 0, nullptr, nullptr,
                       nullptr, nullptr, nullptr, nullptr, nullptr, out_graspable, nullptr, nullptr);
}

pmbs_status pmbs_eval_sample(pmbs_ctx* ctx, int n_envs, const int32_t* box_offset, const float* states,
                             const float* half_ext, const uint64_t* seeds, int k, float* out_push,
                             int32_t* out_attempt) {
    if (!ctx) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    if (k < 2 || (n_envs > 0 && !seeds)) return fail(ctx, PMBS_E_INVALID, "k must be >= 2 and seeds given");
    CU(cudaSetDevice(ctx->device));
    return eval_common(ctx, 2, n_envs, box_offset, states, half_ext, nullptr, nullptr, seeds, k, nullptr, nullptr,
                       nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, out_push, out_attempt);
}

pmbs_status pmbs_eval_start_blocked(pmbs_ctx* ctx, int n_envs, const int32_t* box_offset, const float* states,
                                    const float* half_ext, const float* starts, uint8_t* out_blocked) {
    if (!ctx) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    if (n_envs > 0 && !starts) return fail(ctx, PMBS_E_INVALID, "missing starts");
    CU(cudaSetDevice(ctx->device));
    return eval_common(ctx, 3, n_envs, box_offset, states, half_ext, nullptr, nullptr, nullptr, 0, starts, nullptr,
                       nullptr, nullptr, nullptr, nullptr, nullptr, out_blocked, nullptr, nullptr);
}

pmbs_status pmbs_render_heightmaps_device(pmbs_ctx* ctx, int n_envs, const int32_t* d_box_offset,
                                          const float* d_states, const float* d_half, float* d_out) {
    if (!ctx) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    if (n_envs < 0 || (n_envs > 0 && (!d_box_offset || !d_states || !d_half || !d_out)))
        return fail(ctx, PMBS_E_INVALID, "bad arguments");
    if (reinterpret_cast<uintptr_t>(d_out) % 16 != 0) return fail(ctx, PMBS_E_INVALID, "d_out must be 16-byte aligned");
    if (n_envs == 0) return PMBS_OK;
    CU(cudaSetDevice(ctx->device));
    heightmap_kernel<HMCsr><<<n_envs, 512, kHMSmem, ctx->stream>>>(HMCsr{d_box_offset, d_states, d_half}, n_envs, d_out);
    CU(cudaGetLastError());
    return PMBS_OK;
}

pmbs_status pmbs_render_heightmaps(pmbs_ctx* ctx, int n_envs, const int32_t* box_offset, const float* states,
                                   const float* half_ext, float* out) {
    if (!ctx) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    if (n_envs < 0 || (n_envs > 0 && (!box_offset || !states || !half_ext || !out)))
        return fail(ctx, PMBS_E_INVALID, "bad arguments");
    if (n_envs == 0) return PMBS_OK;
    for (int e = 0; e < n_envs; e++) {
        const int n = box_offset[e + 1] - box_offset[e];
        if (n < 0 || n > kMaxBoxes) return fail(ctx, PMBS_E_INVALID, "box count out of range");
    }
    CU(cudaSetDevice(ctx->device));
    const int B = box_offset[n_envs] - box_offset[0];
    const size_t map_bytes = sizeof(float) * kHMCells * kHMCells * (size_t)n_envs;
    const size_t o_off = 0, o_st = (sizeof(int32_t) * (n_envs + 1) + 255) & ~(size_t)255;
    const size_t o_h = o_st + ((sizeof(float) * 13 * std::max(B, 1) + 255) & ~(size_t)255);
    const size_t o_map = o_h + ((sizeof(float) * 3 * std::max(B, 1) + 255) & ~(size_t)255);
    const size_t sz = o_map + map_bytes;
    const size_t boff = ctx->arena.alloc(sz);
    if (boff == SIZE_MAX) return fail(ctx, PMBS_E_OOM, "heightmap staging does not fit");
    char* base = (char*)arena_ptr(ctx, boff);
    cudaError_t e = cudaMemcpyAsync(base + o_off, box_offset, sizeof(int32_t) * (n_envs + 1), cudaMemcpyHostToDevice,
                                    ctx->stream);
    if (e == cudaSuccess && B > 0)
        e = cudaMemcpyAsync(base + o_st, states + (size_t)13 * box_offset[0], sizeof(float) * 13 * B,
                            cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess && B > 0)
        e = cudaMemcpyAsync(base + o_h, half_ext + (size_t)3 * box_offset[0], sizeof(float) * 3 * B,
                            cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) {
        heightmap_kernel<HMCsr><<<n_envs, 512, kHMSmem, ctx->stream>>>(
            HMCsr{(const int32_t*)(base + o_off), (const float*)(base + o_st), (const float*)(base + o_h)}, n_envs,
            (float*)(base + o_map));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, base + o_map, map_bytes, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    else cudaStreamSynchronize(ctx->stream);
    ctx->arena.release(boff, sz);
    if (e != cudaSuccess) return fail(ctx, PMBS_E_CUDA, std::string("heightmaps: ") + cudaGetErrorString(e));
    return PMBS_OK;
}

pmbs_status pmbs_eval_grasp_heightmap(pmbs_ctx* ctx, int n_envs, const int32_t* box_offset, const float* states,
                                      const float* half_ext, const int32_t* target, float depth, uint8_t* out) {
    if (!ctx) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    if (n_envs < 0 || (n_envs > 0 && (!box_offset || !states || !half_ext || !target || !out)) || !(depth >= 0.f))
        return fail(ctx, PMBS_E_INVALID, "bad arguments");
    if (n_envs == 0) return PMBS_OK;
    for (int e = 0; e < n_envs; e++) {
        const int n = box_offset[e + 1] - box_offset[e];
        if (n < 1 || n > kMaxBoxes) return fail(ctx, PMBS_E_INVALID, "box count out of range");
        if (target[e] < 0 || target[e] >= n) return fail(ctx, PMBS_E_INVALID, "target out of range");
    }
    CU(cudaSetDevice(ctx->device));
    const int B = box_offset[n_envs] - box_offset[0];
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t o_off = 0, o_st = al(sizeof(int32_t) * (n_envs + 1)), o_h = o_st + al(sizeof(float) * 13 * B);
    const size_t o_t = o_h + al(sizeof(float) * 3 * B), o_map = o_t + al(sizeof(int32_t) * n_envs);
    const size_t o_out = o_map + al(sizeof(float) * kHMCells * kHMCells * (size_t)n_envs);
    const size_t sz = o_out + al(n_envs);
    const size_t boff = ctx->arena.alloc(sz);
    if (boff == SIZE_MAX) return fail(ctx, PMBS_E_OOM, "grasp staging does not fit");
    char* base = (char*)arena_ptr(ctx, boff);
    cudaError_t e = cudaMemcpyAsync(base + o_off, box_offset, sizeof(int32_t) * (n_envs + 1), cudaMemcpyHostToDevice,
                                    ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + o_st, states + (size_t)13 * box_offset[0], sizeof(float) * 13 * B,
                            cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + o_h, half_ext + (size_t)3 * box_offset[0], sizeof(float) * 3 * B,
                            cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + o_t, target, sizeof(int32_t) * n_envs, cudaMemcpyHostToDevice, ctx->stream);
    const HMCsr src{(const int32_t*)(base + o_off), (const float*)(base + o_st), (const float*)(base + o_h)};
    if (e == cudaSuccess) {
        heightmap_kernel<HMCsr><<<n_envs, 512, kHMSmem, ctx->stream>>>(src, n_envs, (float*)(base + o_map));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        grasp_hm_kernel<<<(n_envs + 3) / 4, 128, 0, ctx->stream>>>(src, (const int32_t*)(base + o_t),
                                                                   (const float*)(base + o_map), n_envs, ctx->C, depth,
                                                                   (uint8_t*)(base + o_out));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, base + o_out, n_envs, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    else cudaStreamSynchronize(ctx->stream);
    ctx->arena.release(boff, sz);
    if (e != cudaSuccess) return fail(ctx, PMBS_E_CUDA, std::string("grasp heightmap: ") + cudaGetErrorString(e));
    return PMBS_OK;
}

pmbs_status pmbs_query_heightmaps(pmbs_ctx* ctx, int64_t batch, float* out) {
    if (!ctx || !out) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    Batch* b = find_batch(ctx, batch);
    if (!b) return fail(ctx, PMBS_E_INVALID, "unknown batch");
    if (b->n_envs == 0) return PMBS_OK;
    CU(cudaSetDevice(ctx->device));
    const size_t map_bytes = sizeof(float) * kHMCells * kHMCells * (size_t)b->n_envs;
    const size_t boff = ctx->arena.alloc(map_bytes);
    if (boff == SIZE_MAX) return fail(ctx, PMBS_E_OOM, "heightmap staging does not fit");
    float* d_map = (float*)arena_ptr(ctx, boff);
    heightmap_kernel<HMBatch><<<b->n_envs, 512, kHMSmem, b->stream>>>(HMBatch{b->env, b->state}, b->n_envs, d_map);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_map, map_bytes, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    else cudaStreamSynchronize(b->stream);
    ctx->arena.release(boff, map_bytes);
    if (e != cudaSuccess) return fail(ctx, PMBS_E_CUDA, std::string("heightmaps: ") + cudaGetErrorString(e));
    return PMBS_OK;
}

pmbs_status pmbs_launch_shape(pmbs_ctx* ctx, int max_boxes, int32_t* out_lanes, int32_t* out_wpb, int32_t* out_Ps,
                              int32_t* out_Ms, int32_t* out_smem) {
    if (!ctx || max_boxes < 1 || max_boxes > kMaxBoxes) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    int G, wpb, Ms;
    choose_shape(ctx, max_boxes, G, wpb, Ms);
    if (out_lanes) *out_lanes = G;
    const int pairS = std::min(ctx->cfg.pair_cap, std::max(1, max_boxes * (max_boxes - 1) / 2));
    if (out_wpb) *out_wpb = wpb;
    if (out_Ps) *out_Ps = 4 * Ms;
    if (out_Ms) *out_Ms = Ms;
    if (out_smem) *out_smem = make_layout(max_boxes, pairS, Ms, ctx->cfg.manifold_cap).bytes * wpb * (32 / G);
    return PMBS_OK;
}

pmbs_status pmbs_set_launch_shape(pmbs_ctx* ctx, int lanes_per_env, int warps_per_block, int smem_points,
                                  int smem_manifolds) {
    if (!ctx) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!(lanes_per_env == 0 || lanes_per_env == 8 || lanes_per_env == 16 || lanes_per_env == 32))
        return fail(ctx, PMBS_E_INVALID, "lanes_per_env must be 0, 8, 16 or 32");
    ctx->fixed_G = lanes_per_env;
    if (!(warps_per_block == 0 || warps_per_block == 1 || warps_per_block == 2 || warps_per_block == 4))
        return fail(ctx, PMBS_E_INVALID, "warps_per_block must be 0, 1, 2 or 4");
    ctx->fixed_wpb = warps_per_block;
    ctx->fixed_Ps = smem_points;
    ctx->fixed_Ms = smem_manifolds;
    return PMBS_OK;
}

pmbs_status pmbs_check_status(pmbs_ctx* ctx, uint32_t* out, int reset) {
    if (!ctx || !out) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    for (int k = 0; k < 4; k++) out[k] = 0u;
#if PMBS_BOUNDS_CHECK
    CU(cudaSetDevice(ctx->device));
    CU(cudaStreamSynchronize(ctx->stream));
    CU(cudaMemcpyFromSymbol(out, g_check_status, sizeof(uint32_t) * 4));
    if (reset) {
        const uint32_t zero[4] = {0u, 0u, 0u, 0u};
        CU(cudaMemcpyToSymbol(g_check_status, zero, sizeof(zero)));
    }
    return PMBS_OK;
#else
    (void)reset;
    return fail(ctx, PMBS_E_INVALID, "library built without bounds checks (build with PMBS_BOUNDS_CHECK=1)");
#endif
}

pmbs_status pmbs_fp32_peak(pmbs_ctx* ctx, double* out_tflops) {
    if (!ctx || !out_tflops) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    CU(cudaSetDevice(ctx->device));
    const size_t off = ctx->arena.alloc(sizeof(float) * 65536);
    if (off == SIZE_MAX) return fail(ctx, PMBS_E_OOM, "no room for the probe");
    float* out = (float*)arena_ptr(ctx, off);
    const int blocks = ctx->num_sms * 8, threads = 256, iters = 4096;
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    fma_peak_kernel<<<blocks, threads, 0, ctx->stream>>>(out, iters / 8, 1.f);
    CU(cudaEventRecord(e0, ctx->stream));
    fma_peak_kernel<<<blocks, threads, 0, ctx->stream>>>(out, iters, 1.f);
    CU(cudaEventRecord(e1, ctx->stream));
    CU(cudaEventSynchronize(e1));
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->arena.release(off, sizeof(float) * 65536);
    const double flops = (double)blocks * threads * iters * 16.0 * 8.0 * 2.0;
    *out_tflops = flops / (ms * 1e-3) / 1e12;
    return PMBS_OK;
}

}  // extern "C"


// ====================================================================== serving loop
// Continuous batching of rollout requests from many concurrent planners: submit() copies
// a request and returns a ticket; a dispatcher thread admits pending requests in arrival
// order whenever the device arena can hold them (memory-based admission), launches each
// on one of several non-blocking streams with its own contact scratch so that admitted
// batches overlap on the device, and retires them as their completion events fire.  A
// request's result does not depend on what else is running: every environment's
// arithmetic is independent of scheduling.
namespace {

struct Request {
    int64_t ticket = 0;
    int n_envs = 0, depth = 1;
    std::vector<int32_t> scene_ids;
    std::vector<float> first_push;
    std::vector<uint64_t> seeds;
    std::chrono::steady_clock::time_point t_submit, t_done;
    int64_t batch = 0;
    int stream = -1;
    cudaEvent_t done_ev = nullptr;
    bool finished = false;
    bool abandoned = false;  // cancelled while on the device: dropped when it retires
    int resumes = 0;         // relaunches after the watchdog stopped environments
    pmbs_status status = PMBS_OK;
    std::vector<int32_t> cost, steps;
    std::vector<float> reward;
    std::vector<uint8_t> flags;
};

}  // namespace

struct pmbs_server {
    pmbs_ctx* ctx = nullptr;
    std::vector<cudaStream_t> streams;
    int max_inflight = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<int64_t> pending;
    std::vector<int64_t> inflight;
    std::map<int64_t, Request> reqs;
    int64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    int next_stream = 0;
    // statistics
    std::vector<double> latencies_ms;
    double env_steps = 0.0;
    int64_t completed = 0;
    size_t peak_used = 0;
    int64_t resumes = 0;
    int64_t admitting = 0;  // ticket being admitted with the server lock released
    std::chrono::steady_clock::time_point t_first, t_last;
    bool any = false;
};

namespace {

// Admit one pending request: create its batch (host ids: copies and set-up finish before
// return), give it its own stream and scratch, launch it.  Returns PMBS_E_OOM when the
// arena cannot hold it now.
pmbs_status server_admit(pmbs_server* sv, Request& r) {
    NvtxRange nvtx_("pmbs_server_admit");
    pmbs_ctx* ctx = sv->ctx;
    std::lock_guard<std::mutex> lk(ctx->mu);
    int64_t id = 0;
    pmbs_status st = rollout_common(ctx, r.n_envs, r.scene_ids.data(), r.first_push.data(), r.depth,
                                    r.seeds.data(), false, &id);
    if (st != PMBS_OK) return st;
    Batch& b = ctx->batches[id];
    r.stream = sv->next_stream;
    sv->next_stream = (sv->next_stream + 1) % (int)sv->streams.size();
    b.stream = sv->streams[r.stream];
    b.own_scratch = true;
    if (b.n_envs > 0) {
        st = launch_rollout(ctx, b, 0, b.stream);
        if (st != PMBS_OK) {
            release_batch_mem(ctx, b);
            ctx->batches.erase(id);
            return st;
        }
    }
    b.finished = true;
    r.batch = id;
    if (cudaEventCreateWithFlags(&r.done_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(r.done_ev, b.stream) != cudaSuccess) {
        // leave the batch to be retired by a synchronous wait
        r.done_ev = nullptr;
    }
    sv->peak_used = std::max(sv->peak_used, ctx->arena.used);
    return PMBS_OK;
}

// A request's launch has completed.  When the watchdog stopped some of its environments
// (they keep their progress), clear the flag and relaunch the batch on its stream, which
// resumes them, and return false.  Otherwise copy the results back, free the batch and
// return true.
bool server_retire(pmbs_server* sv, Request& r) {
    pmbs_ctx* ctx = sv->ctx;
    std::lock_guard<std::mutex> lk(ctx->mu);
    Batch* b = find_batch(ctx, r.batch);
    const int n = r.n_envs;
    cudaError_t e = cudaSuccess;
    int cnt[5] = {0, 0, 0, 0, 0};
    if (b && n > 0) {
        e = cudaMemcpyAsync(cnt, b->counters, sizeof(cnt), cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e == cudaSuccess && cnt[4] && !cnt[1]) {
            e = cudaMemsetAsync(b->counters + 4, 0, sizeof(int), b->stream);
            if (e == cudaSuccess && launch_rollout(ctx, *b, 0, b->stream) == PMBS_OK &&
                (!r.done_ev || cudaEventRecord(r.done_ev, b->stream) == cudaSuccess)) {
                r.resumes++;
                return false;
            }
            if (e == cudaSuccess) e = cudaErrorLaunchFailure;
        }
    }
    r.cost.assign(n, 0);
    r.reward.assign(n, 0.f);
    r.flags.assign(n, 0);
    r.steps.assign(n, 0);
    if (b && n > 0 && e == cudaSuccess) {
        e = cudaMemcpyAsync(r.cost.data(), b->cost, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(r.reward.data(), b->reward, sizeof(float) * n, cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(r.flags.data(), b->flags, n, cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(r.steps.data(), b->steps, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    } else if (b) {
        cudaStreamSynchronize(b->stream);
    }
    if (b) {
        release_batch_mem(ctx, *b);
        ctx->batches.erase(r.batch);
    }
    if (r.done_ev) cudaEventDestroy(r.done_ev);
    r.done_ev = nullptr;
    r.status = e != cudaSuccess ? PMBS_E_CUDA : (cnt[1] ? PMBS_E_INVALID : PMBS_OK);
    r.t_done = std::chrono::steady_clock::now();
    // r.finished is set by the caller under the server lock
    return true;
}

void server_loop(pmbs_server* sv) {
    cudaSetDevice(sv->ctx->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    while (!sv->stop) {
        bool progressed = false;
        // admit in arrival order while memory and the in-flight limit allow
        while (!sv->pending.empty() && (int)sv->inflight.size() < sv->max_inflight) {
            const int64_t t = sv->pending.front();
            Request& r = sv->reqs[t];
            sv->admitting = t;  // a cancel now only marks the request
            lk.unlock();
            const pmbs_status st = server_admit(sv, r);
            lk.lock();
            sv->admitting = 0;
            if (st == PMBS_E_OOM && !sv->inflight.empty() && !r.abandoned) break;  // wait for memory to free up
            sv->pending.pop_front();
            progressed = true;
            if (r.abandoned && st != PMBS_OK) {
                sv->reqs.erase(t);
                continue;
            }
            if (st != PMBS_OK) {
                r.status = st;
                r.finished = true;
                r.t_done = std::chrono::steady_clock::now();
                sv->cv_done.notify_all();
                continue;
            }
            sv->inflight.push_back(r.ticket);
        }
        // retire finished batches
        for (size_t i = 0; i < sv->inflight.size();) {
            Request& r = sv->reqs[sv->inflight[i]];
            const bool ready = !r.done_ev || cudaEventQuery(r.done_ev) != cudaErrorNotReady;
            if (!ready) {
                i++;
                continue;
            }
            lk.unlock();
            const bool retired = server_retire(sv, r);
            lk.lock();
            progressed = true;
            if (!retired) {
                i++;
                continue;
            }
            const double ms = std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count();
            sv->latencies_ms.push_back(ms);
            for (int32_t s : r.steps) sv->env_steps += s;
            sv->completed++;
            sv->resumes += r.resumes;
            sv->t_last = r.t_done;
            r.finished = true;
            const int64_t t = sv->inflight[i];
            sv->inflight.erase(sv->inflight.begin() + (long)i);
            if (r.abandoned) sv->reqs.erase(t);
            sv->cv_done.notify_all();
        }
        if (!progressed) {
            if (sv->inflight.empty() && sv->pending.empty())
                sv->cv_work.wait(lk, [sv] { return sv->stop || !sv->pending.empty(); });
            else
                sv->cv_work.wait_for(lk, std::chrono::microseconds(50));
        }
    }
}

double percentile(std::vector<double> v, double p) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = p * (double)(v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - (double)i;
    return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" {

pmbs_status pmbs_server_create(pmbs_ctx* ctx, int n_streams, int max_inflight, pmbs_server** out) {
    if (!ctx || !out || n_streams < 1 || n_streams > 64 || max_inflight < 1) return PMBS_E_INVALID;
    *out = nullptr;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return PMBS_E_CUDA;
    pmbs_server* sv = new pmbs_server();
    sv->ctx = ctx;
    sv->max_inflight = max_inflight;
    for (int i = 0; i < n_streams; i++) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t x : sv->streams) cudaStreamDestroy(x);
            delete sv;
            return PMBS_E_CUDA;
        }
        sv->streams.push_back(st);
    }
    sv->worker = std::thread(server_loop, sv);
    *out = sv;
    return PMBS_OK;
}

pmbs_status pmbs_server_submit(pmbs_server* sv, int n_envs, const int32_t* scene_ids, const float* first_push, int depth,
                               const uint64_t* seeds, int64_t* out_ticket) {
    if (!sv || !out_ticket || n_envs < 0 || depth < 1 || depth > 64) return PMBS_E_INVALID;
    if (n_envs > 0 && (!scene_ids || !first_push || (!seeds && depth > 1))) return PMBS_E_INVALID;
    Request r;
    r.n_envs = n_envs;
    r.depth = depth;
    r.scene_ids.assign(scene_ids, scene_ids + n_envs);
    r.first_push.assign(first_push, first_push + 4 * (size_t)n_envs);
    r.seeds.assign((size_t)n_envs, 0ull);
    if (seeds) r.seeds.assign(seeds, seeds + n_envs);
    r.t_submit = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        r.ticket = sv->next_ticket++;
        if (!sv->any) {
            sv->any = true;
            sv->t_first = r.t_submit;
        }
        *out_ticket = r.ticket;
        sv->pending.push_back(r.ticket);
        sv->reqs[r.ticket] = std::move(r);
    }
    sv->cv_work.notify_one();
    return PMBS_OK;
}

pmbs_status pmbs_server_wait(pmbs_server* sv, int64_t ticket, int timeout_ms, int32_t* out_cost, float* out_reward,
                             uint8_t* out_flags, int32_t* out_steps, double* out_latency_ms) {
    if (!sv) return PMBS_E_INVALID;
    std::unique_lock<std::mutex> lk(sv->mu);
    if (sv->reqs.find(ticket) == sv->reqs.end()) return PMBS_E_INVALID;
    // look the ticket up afresh after every wake-up: a cancel may have dropped it
    const auto pred = [&] {
        auto j = sv->reqs.find(ticket);
        return j == sv->reqs.end() || j->second.finished || j->second.abandoned;
    };
    if (timeout_ms < 0) sv->cv_done.wait(lk, pred);
    else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred))
        return timeout_ms == 0 ? PMBS_E_NOT_READY : PMBS_E_TIMEOUT;
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end() || it->second.abandoned) return PMBS_E_INVALID;
    Request& r = it->second;
    const pmbs_status st = r.status;
    const int n = r.n_envs;
    if (st == PMBS_OK) {
        if (out_cost) std::memcpy(out_cost, r.cost.data(), sizeof(int32_t) * n);
        if (out_reward) std::memcpy(out_reward, r.reward.data(), sizeof(float) * n);
        if (out_flags) std::memcpy(out_flags, r.flags.data(), n);
        if (out_steps) std::memcpy(out_steps, r.steps.data(), sizeof(int32_t) * n);
    }
    if (out_latency_ms) *out_latency_ms = std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count();
    sv->reqs.erase(it);
    return st;
}

pmbs_status pmbs_server_stats(pmbs_server* sv, double* out) {
    if (!sv || !out) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(sv->mu);
    const double span = sv->completed ? std::chrono::duration<double>(sv->t_last - sv->t_first).count() : 0.0;
    out[0] = (double)sv->completed;
    out[1] = sv->env_steps;
    out[2] = span;
    out[3] = percentile(sv->latencies_ms, 0.50);
    out[4] = percentile(sv->latencies_ms, 0.99);
    double mean = 0.0;
    for (double x : sv->latencies_ms) mean += x;
    out[5] = sv->latencies_ms.empty() ? 0.0 : mean / (double)sv->latencies_ms.size();
    out[6] = (double)sv->peak_used;
    out[7] = (double)(sv->pending.size() + sv->inflight.size());
    size_t held = 0;
    for (const auto& kv : sv->reqs) held += kv.second.finished ? 1 : 0;
    out[8] = (double)held;
    out[9] = (double)sv->resumes;
    {
        std::lock_guard<std::mutex> lk2(sv->ctx->mu);
        out[10] = (double)sv->ctx->arena.used;
    }
    return PMBS_OK;
}

pmbs_status pmbs_server_cancel(pmbs_server* sv, int64_t ticket) {
    if (!sv) return PMBS_E_INVALID;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return PMBS_E_INVALID;
    Request& r = it->second;
    auto p = std::find(sv->pending.begin(), sv->pending.end(), ticket);
    if (ticket == sv->admitting) {
        r.abandoned = true;
    } else if (p != sv->pending.end()) {
        sv->pending.erase(p);
        sv->reqs.erase(it);
    } else if (r.finished) {
        sv->reqs.erase(it);
    } else {
        r.abandoned = true;
    }
    sv->cv_done.notify_all();
    return PMBS_OK;
}

void pmbs_server_destroy(pmbs_server* sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    cudaSetDevice(sv->ctx->device);
    for (auto& kv : sv->reqs) {
        Request& r = kv.second;
        if (r.batch && !r.finished) {
            do {
                if (r.stream >= 0) cudaStreamSynchronize(sv->streams[r.stream]);
            } while (!server_retire(sv, r));
            r.finished = true;
        }
    }
    for (cudaStream_t st : sv->streams) cudaStreamDestroy(st);
    delete sv;
}

}  // extern "C"

// ====================================================================== allocation-free entry
// pmbs_rollout_noalloc runs the same rollout kernel without any device allocation: every
// piece of scratch it needs (environment descriptors, progress records, work order,
// counters, event counters, step counts and the per-warp contact spill regions) lives in
// one file-scope device array of fixed size, shared by all calls on a device.
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;  // 32 MiB on every device that loads the library
constexpr int kNoAllocMaxEnvs = 16384;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct NoAllocDevice {
    bool ready = false;
    unsigned char* scratch = nullptr;  // device address of g_noalloc_scratch on that device
    int num_sms = 0;
};
NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];
std::mutex g_noalloc_mu;

// Descriptors, order and cleared per-call state for caller-provided environments.
// Environment e owns records box_offset[e] .. box_offset[e+1]-1 (18 floats each: state13,
// half extents, mass, mu).  An environment is not simulated (counters[1] records that)
// when its box count is outside [1, max_boxes], its first record offset is negative, its
// target is out of range, its first push is not finite, or one of its rows fails the
// checks scene loading applies: every value finite, | |q| - 1 | <= 1e-3, positive half
// extents (a cylinder row (r, -r, h) only with the cylinder solver), mass > 0, mu >= 0.
__device__ __forceinline__ bool noalloc_row_ok(const float* r, int allow_cyl) {
    for (int k = 0; k < kRecFloats; k++)
        if (!isfinite(r[k])) return false;
    const double qn = sqrt((double)r[3] * r[3] + (double)r[4] * r[4] + (double)r[5] * r[5] + (double)r[6] * r[6]);
    if (fabs(qn - 1.0) > 1e-3) return false;
    const float* h = r + 13;
    const bool cyl = h[1] < 0.f;
    if (cyl && (!allow_cyl || h[1] != -h[0])) return false;
    return h[0] > 0.f && (h[1] > 0.f || cyl) && h[2] > 0.f && r[16] > 0.f && r[17] >= 0.f;
}

__global__ void __launch_bounds__(1024) noalloc_setup_kernel(int n_envs, int max_boxes, int allow_cyl,
                                                             const int32_t* box_offset, const float* records,
                                                             const int32_t* target, const float4* first_push,
                                                             EnvIn* env, int* order, EnvProg* prog, int* counters,
                                                             unsigned long long* events, int32_t* steps) {
    __shared__ int hist[kMaxBoxes + 2];
    const int t = threadIdx.x;
    if (t < kMaxBoxes + 2) hist[t] = 0;
    if (t < 8) counters[t] = 0;
    __syncthreads();
    for (int e = t; e < n_envs; e += 1024) {
        const int b0 = box_offset[e];
        int n = box_offset[e + 1] - b0;
        const int tg = target[e];
        const float4 fp = first_push[e];
        EnvProg p;
        memset(&p, 0, sizeof(p));
        bool bad = b0 < 0 || n < 1 || n > max_boxes || tg < 0 || tg >= n || !isfinite(fp.x) || !isfinite(fp.y) ||
                   !isfinite(fp.z) || !isfinite(fp.w);
        for (int i = 0; !bad && i < n; i++) bad = !noalloc_row_ok(records + (size_t)kRecFloats * (b0 + i), allow_cyl);
        if (bad) {
            atomicOr(counters + 1, 1);
            p.done = 1;  // not simulated
            n = 0;
        }
        prog[e] = p;
        env[e] = EnvIn{bad ? records : records + (size_t)kRecFloats * b0, n, tg, bad ? 0 : b0, -1};
        for (int k = 0; k < kNumEvents; k++) events[(size_t)e * kNumEvents + k] = 0ull;
        steps[e] = 0;
        atomicAdd(&hist[kMaxBoxes - min(n, kMaxBoxes)], 1);
    }
    __syncthreads();
    if (t == 0) {
        int acc = 0;
        for (int b = 0; b <= kMaxBoxes; b++) {
            const int c = hist[b];
            hist[b] = acc;
            acc += c;
        }
    }
    __syncthreads();
    for (int e = t; e < n_envs; e += 1024) {
        const int pos = atomicAdd(&hist[kMaxBoxes - min(env[e].n, kMaxBoxes)], 1);
        order[pos] = e;
    }
}

}  // namespace

namespace {

pmbs_status noalloc_run(const pmbs_config& c, cudaStream_t stream, int n_envs, const int32_t* d_box_offset,
                        const float* d_records, const int32_t* d_target, const float* d_first_push,
                        const uint64_t* d_seeds, int depth, float* d_state_out, int32_t* d_cost, float* d_reward,
                        uint8_t* d_flags) {
    if (cudaSetDevice(c.device) != cudaSuccess) return PMBS_E_CUDA;
    NoAllocDevice& dv = g_noalloc_dev[c.device];
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!dv.ready) {
            // once per device, with that device current: the device address of the scratch
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return PMBS_E_CUDA;
            int sms = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device) != cudaSuccess) return PMBS_E_CUDA;
            if (cudaFuncSetAttribute(rollout_fn(false, false), cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) !=
                    cudaSuccess ||
                cudaFuncSetAttribute(rollout_fn(true, false), cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) !=
                    cudaSuccess)
                return PMBS_E_CUDA;
            dv.scratch = (unsigned char*)p;
            dv.num_sms = sms;
            dv.ready = true;
        }
    }
    // scratch layout: per-environment records, then per-warp contact spill regions
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t ne = (size_t)n_envs;
    const size_t o_env = take(sizeof(EnvIn) * ne), o_order = take(sizeof(int) * ne), o_prog = take(sizeof(EnvProg) * ne),
                 o_cnt = take(sizeof(int) * 8), o_ev = take(sizeof(unsigned long long) * kNumEvents * ne),
                 o_steps = take(sizeof(int32_t) * ne);
    const int f4_per_warp = scratch_f4_per_warp(c.manifold_cap);
    const size_t warp_bytes = sizeof(float4) * (size_t)f4_per_warp;
    if (off >= kNoAllocScratchBytes || (kNoAllocScratchBytes - off) / warp_bytes < 4) return PMBS_E_INVALID;
    const int max_warps = (int)std::min<size_t>((kNoAllocScratchBytes - off) / warp_bytes, 1 << 20);
    unsigned char* S = dv.scratch;
    EnvIn* env = (EnvIn*)(S + o_env);
    int* order = (int*)(S + o_order);
    EnvProg* prog = (EnvProg*)(S + o_prog);
    int* counters = (int*)(S + o_cnt);
    unsigned long long* events = (unsigned long long*)(S + o_ev);
    int32_t* steps = (int32_t*)(S + o_steps);
    float4* spill = (float4*)(S + off);

    // the context entry points' default shape: one environment per warp, two warps per
    // block, eight manifolds per environment in shared memory (the rest in the spill
    // regions); cfg->lanes_per_env, warps_per_block and smem_manifolds / smem_points
    // override it as they do there
    const int nb = c.max_boxes_per_env;
    const int G = (c.lanes_per_env == 8 || c.lanes_per_env == 16 || c.lanes_per_env == 32) ? c.lanes_per_env : 32;
    const int K = 32 / G;
    int wpb = std::min(c.warps_per_block > 0 ? c.warps_per_block : 2, 4);
    const int pairS = std::min(c.pair_cap, std::max(1, nb * (nb - 1) / 2));
    int Ms = K > 1 ? 0 : 8;
    if (c.smem_points >= 0) Ms = c.smem_points / 4;
    if (c.smem_manifolds >= 0) Ms = c.smem_manifolds;
    Ms = std::min(Ms, c.manifold_cap);
    while (Ms > 0 && (size_t)K * make_layout(nb, pairS, Ms, c.manifold_cap).bytes > 227 * 1024) Ms /= 2;
    while (wpb > 1 && (size_t)wpb * K * make_layout(nb, pairS, Ms, c.manifold_cap).bytes > 227 * 1024) wpb >>= 1;
    const Layout L = make_layout(nb, pairS, Ms, c.manifold_cap);
    const size_t smem = (size_t)L.bytes * wpb * K;
    if (smem > 227 * 1024) return PMBS_E_INVALID;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rollout_fn(c.cylinders != 0, false),
                                                      32 * wpb, smem) != cudaSuccess)
        return PMBS_E_CUDA;
    if (per_sm < 1) return PMBS_E_INVALID;
    per_sm = std::min(per_sm, kMaxWarpsPerSM / wpb);
    const int per_block = wpb * K;
    if (max_warps < per_block) return PMBS_E_INVALID;
    const int blocks = std::max(1, std::min({(n_envs + per_block - 1) / per_block, per_sm * dv.num_sms,
                                             max_warps / per_block}));

    noalloc_setup_kernel<<<1, 1024, 0, stream>>>(n_envs, nb, c.cylinders ? 1 : 0, d_box_offset, d_records, d_target,
                                                 (const float4*)d_first_push, env, order, prog, counters, events,
                                                 steps);
    if (cudaGetLastError() != cudaSuccess) return PMBS_E_CUDA;
    RolloutArgs a;
    fill_const(c, a.C);
    a.L = L;
    a.G = G;
    a.n_envs = n_envs;
    a.depth = depth;
    a.max_substeps = 0;
    a.child_on = 0;
    a.env = env;
    a.order = order;
    a.queue_head = counters + 2;
    a.done_count = counters + 3;
    a.first_push = (const float4*)d_first_push;
    a.seeds = d_seeds ? d_seeds : (const uint64_t*)(S + o_ev);  // unread when depth == 1
    a.prog = prog;
    a.state = d_state_out;
    a.child = nullptr;
    a.cost = d_cost;
    a.reward = d_reward;
    a.flags = d_flags;
    a.steps = steps;
    a.events = events;
    a.gscratch = spill;
    a.scratch_f4_per_warp = f4_per_warp;
    a.watchdog_cycles = (long long)((double)c.watchdog_ms * 2.0e6);
    a.watchdog_flag = counters + 4;
    a.warm = nullptr;  // no room for caches in the fixed scratch: warm start is refused
    a.warm_f4_per_env = 0;
    a.C.timers = 0;    // phase timers have no output here
    a.phase = nullptr;
    a.n_rows = LLONG_MAX;  // the record count is the caller's (not passed)
    rollout_fn(c.cylinders != 0, false)<<<blocks, 32 * wpb, smem, stream>>>(a);
    if (cudaGetLastError() != cudaSuccess) return PMBS_E_CUDA;
    int host_cnt[8];
    if (cudaMemcpyAsync(host_cnt, counters, sizeof(host_cnt), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return PMBS_E_CUDA;
    if (host_cnt[4]) return PMBS_E_TIMEOUT;
    if (host_cnt[1]) return PMBS_E_INVALID;
    return PMBS_OK;
}

}  // namespace

extern "C" pmbs_status pmbs_rollout_noalloc(const pmbs_config* cfg, void* cuda_stream, int n_envs,
                                            const int32_t* d_box_offset, const float* d_records,
                                            const int32_t* d_target, const float* d_first_push,
                                            const uint64_t* d_seeds, int depth, float* d_state_out,
                                            int32_t* d_cost, float* d_reward, uint8_t* d_flags) {
    if (!cfg) return PMBS_E_INVALID;
    const pmbs_config& c = *cfg;
    if (n_envs < 0 || n_envs > kNoAllocMaxEnvs || depth < 1 || depth > 64 || c.max_boxes_per_env < 1 ||
        c.max_boxes_per_env > kMaxBoxes || c.device < 0 || c.device >= kNoAllocMaxDevices || c.grasp_angles < 1 ||
        c.grasp_angles > 32 || c.sample_attempts < 1 || c.sample_attempts > 32 || c.contact_cap < 4 ||
        c.manifold_cap < 1 || c.manifold_cap > 1024 || c.pair_cap < 1 || c.pair_cap > 4096 || c.warm_start)
        return PMBS_E_INVALID;
    if (n_envs == 0) return PMBS_OK;
    if (!d_box_offset || !d_records || !d_target || !d_first_push || (!d_seeds && depth > 1) || !d_state_out ||
        !d_cost || !d_reward || !d_flags)
        return PMBS_E_INVALID;
    // the caller's current device is put back on every return
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return PMBS_E_CUDA;
    const pmbs_status st = noalloc_run(c, (cudaStream_t)cuda_stream, n_envs, d_box_offset, d_records, d_target,
                                       d_first_push, d_seeds, depth, d_state_out, d_cost, d_reward, d_flags);
    if (cudaSetDevice(prev) != cudaSuccess && st == PMBS_OK) return PMBS_E_CUDA;
    return st;
}

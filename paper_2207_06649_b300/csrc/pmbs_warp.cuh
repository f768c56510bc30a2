// Warp-level environment solver: one warp advances one environment through whole
// pushes.  Bodies live in shared memory; contact manifolds and points live in shared
// memory up to a per-launch capacity and in a per-warp global scratch region beyond it
// (addressed through generic pointers, so the solver code is the same either way).
//
// Substep (dt), following the transition of Sec. III-A as read by this library:
//   pusher kinematics -> gravity -> frames + AABB -> broadphase (pairs, plane, pusher)
//   -> narrowphase + ordered emission -> contact preparation -> greedy colouring
//   -> projected Gauss-Seidel over colours -> semi-implicit integration.
// Within one colour the manifolds touch disjoint dynamic bodies, so the lanes solve
// them concurrently and the result equals the sequential order exactly.
#pragma once
#include <cstdint>

#include "pmbs_collide.cuh"
#include "pmbs_exact.cuh"

namespace pmbs {

constexpr int kMaxBoxes = 64;
constexpr int kMaxColours = 32;
constexpr int kPlane = 255;   // body id of the table plane (static)
constexpr int kPusher = 254;  // body id of the kinematic pusher
constexpr int kNumEvents = 18;
enum {
    EV_SUBSTEPS = 0, EV_BOX_STEPS, EV_PAIR_TESTS, EV_SAT, EV_FACE, EV_EDGE, EV_PLANE, EV_PUSHER,
    EV_POINTS, EV_MANIFOLDS, EV_PGS_MAN, EV_PGS_PTS, EV_PUSH_EVALS, EV_SAMPLE_ATTEMPTS,
    EV_CLIP_VERTS, EV_COLOURS, EV_BB_POINTS, EV_PGS_BB_POINTS
};
// Phase timers (SimConst::timers): SM clock cycles an environment's group spends in each
// part of its work, summed over its substeps and pushes.
constexpr int kNumPhases = 8;
enum {
    PH_PUSH_SETUP = 0, PH_BROADPHASE, PH_NARROWPHASE, PH_PREP, PH_COLOUR, PH_SOLVE, PH_INTEGRATE, PH_PUSH_END
};
enum { FLAG_GRASP1 = 1, FLAG_INVALID_START = 2, FLAG_OUT_OF_WS = 4, FLAG_OVERFLOW = 8, FLAG_NOOP = 16 };

// Physical and algorithmic constants of a launch.
struct SimConst {
    float dt, gx, gy, gz;
    float table_hx, table_hy, table_mu, pusher_mu;
    float pr, pz0, pz1, pspeed, plen, gamma;
    float grasp_W, grasp_c, grasp_f, grasp_fw;
    float margin, slop, baumgarte, sample_clear;
    int substeps, iters, grasp_K, attempts, npts;
    int warm;         // carry contact impulses over substeps
    float warm_tol2;  // squared match distance
    int Pcap, Mcap, pair_cap;
    int timers;       // accumulate per-phase clock cycles (off: one uniform branch per phase)
    float gcos[32], gsin[32];
};

// Per-warp shared-memory layout (sizes fixed per launch).
//
// Contact storage is manifold-major with one array per 16-byte field: header fields
// H0 = (n, mu), H1 = (t1, A | B << 8 | np << 16), H2 = (t2, -) and, for each of the four
// point slots j, F0 = (rA, 1/k_n), F1 = (rB, target normal velocity), F2 = (lambda_n,
// lambda_t1, lambda_t2, 1/k_t1), F3 = (1/k_t2, depth, -, -).  Field k of manifold m sits
// at base[k * stride + m], so lanes working on different manifolds touch different banks.
// Manifolds below Ms live in shared memory (stride Ms), the rest in the warp's global
// scratch (stride Mcap).
constexpr int kConFields = 3 + 4 * 4;

struct Layout {
    int NB;        // boxes per environment capacity
    int pairS;     // broadphase pair capacity (<= pair_cap)
    int Ms;        // manifolds kept in shared memory
    int Mcap;      // manifold capacity (lists, global scratch stride)
    int bytes;     // total bytes per warp
    int o_bv, o_bw, o_bI0, o_bI1, o_con, o_x, o_q, o_h, o_ib, o_R, o_lo, o_hi, o_mask, o_plane, o_pusher,
        o_pairs, o_mAB, o_mcol, o_order, o_cstart, o_scal, o_ev;
};

__host__ __device__ inline int align_up(int x, int a) { return (x + a - 1) / a * a; }

__host__ __device__ inline Layout make_layout(int NB, int pairS, int Ms, int Mcap) {
    Layout L;
    L.NB = NB;
    L.pairS = pairS;
    L.Ms = Ms;
    L.Mcap = Mcap;
    int o = 0;
    L.o_bv = o; o += 16 * NB;
    L.o_bw = o; o += 16 * NB;
    L.o_bI0 = o; o += 16 * NB;
    L.o_bI1 = o; o += 16 * NB;
    L.o_con = o; o += 16 * kConFields * Ms;
    L.o_x = o; o += 12 * NB;
    L.o_q = o; o += 16 * NB;
    L.o_h = o; o += 12 * NB;
    L.o_ib = o; o += 12 * NB;
    L.o_R = o; o += 36 * NB;
    L.o_lo = o; o += 12 * NB;
    L.o_hi = o; o += 12 * NB;
    L.o_mask = o; o += 4 * NB;
    L.o_scal = o; o += 4 * 16;
    o = align_up(o, 8);
    L.o_ev = o; o += 8 * (kNumEvents + kNumPhases);  // event counters and phase cycles of the running environment (8-byte aligned)
    L.o_mAB = o; o += 2 * Mcap;
    L.o_order = o; o += 2 * Mcap;
    L.o_cstart = o; o += 2 * (kMaxColours + 2);
    o = align_up(o, 4);
    L.o_pairs = o; o += 2 * pairS;
    L.o_mcol = o; o += Mcap;
    L.o_plane = o; o += NB;
    L.o_pusher = o; o += NB;
    L.bytes = align_up(o, 16);
    return L;
}

// Global scratch per warp, in float4 units.
__host__ __device__ inline int scratch_f4_per_warp(int Mcap) { return kConFields * Mcap; }

// Pointers into one warp's shared region and its global scratch.
// The block's dynamic shared memory; every kernel that binds warp regions uses it.
extern __shared__ __align__(16) unsigned char pmbs_smem[];

// Bounds-checked build (compiled with -DPMBS_BOUNDS_CHECK=1 into a library of its own):
// every shared-memory array index, every contact manifold index and every global row or
// environment index of the rollout kernel is checked against its capacity.  An index out
// of range is recorded in a status word -- violations, then the first one's array id,
// index and capacity -- and the access is redirected to a sink (a load reads the sink, a
// store lands there), so the kernel carries on and ends normally: no trap, no fault.
#ifndef PMBS_BOUNDS_CHECK
#define PMBS_BOUNDS_CHECK 0
#endif
#if PMBS_BOUNDS_CHECK
enum {
    CHK_BV = 1, CHK_BW, CHK_BI0, CHK_BI1, CHK_X, CHK_Q, CHK_H, CHK_IB, CHK_R, CHK_LO, CHK_HI, CHK_MASK, CHK_SCAL,
    CHK_EV, CHK_PH, CHK_MAB, CHK_ORDER, CHK_CSTART, CHK_PAIRS, CHK_MCOL, CHK_PLANE, CHK_PUSHER, CHK_MANIFOLD,
    CHK_STATE_ROW, CHK_ENV, CHK_WARM
};
__device__ unsigned int g_check_status[4];
__device__ float4 g_check_sink[8];
__device__ __noinline__ void check_fail(uint32_t id, long long i, long long cap) {
    if (atomicAdd(&g_check_status[0], 1u) == 0u) {
        g_check_status[1] = id;
        g_check_status[2] = (unsigned int)i;
        g_check_status[3] = (unsigned int)cap;
    }
}
// true when 0 <= i < cap; otherwise records the violation
__device__ __forceinline__ bool check_index(uint32_t id, long long i, long long cap) {
    if (i >= 0 && i < cap) return true;
    check_fail(id, i, cap);
    return false;
}
#endif

// An array in the block's dynamic shared memory held as a 32-bit byte offset: one
// register per array, and accesses compile to shared-memory loads and stores.
template <class T>
struct SArr {
    uint32_t off;
#if PMBS_BOUNDS_CHECK
    uint32_t cap, id;
    __device__ __forceinline__ T& operator[](int i) const {
        if (!check_index(id, i, cap)) return *reinterpret_cast<T*>(g_check_sink);
        return reinterpret_cast<T*>(pmbs_smem + off)[i];
    }
#else
    __device__ __forceinline__ T& operator[](int i) const { return reinterpret_cast<T*>(pmbs_smem + off)[i]; }
#endif
};

#if PMBS_BOUNDS_CHECK
#define PMBS_SARR(o, n, tag) {base + (uint32_t)(o), (uint32_t)(n), (uint32_t)(tag)}
#else
#define PMBS_SARR(o, n, tag) {base + (uint32_t)(o)}
#endif

// One warp's region: its byte offset in the block's dynamic shared memory, the launch's
// layout (a kernel parameter, so field offsets are read from the parameter bank instead
// of being held in registers) and the warp's global contact scratch.  Capacities (used by
// the bounds-checked build only) are those of make_layout.
struct WarpMem {
    uint32_t base;
    const Layout* L;
    float4* con_g;
    __device__ __forceinline__ SArr<float4> bv() const { return PMBS_SARR(L->o_bv, L->NB, CHK_BV); }     // v, 1/m
    __device__ __forceinline__ SArr<float4> bw() const { return PMBS_SARR(L->o_bw, L->NB, CHK_BW); }     // w, mu
    __device__ __forceinline__ SArr<float4> bI0() const { return PMBS_SARR(L->o_bI0, L->NB, CHK_BI0); }  // I^-1 00 01 02 11
    __device__ __forceinline__ SArr<float4> bI1() const { return PMBS_SARR(L->o_bI1, L->NB, CHK_BI1); }  // I^-1 12 22
    __device__ __forceinline__ SArr<float> x() const { return PMBS_SARR(L->o_x, 3 * L->NB, CHK_X); }  // SoA, stride NB
    __device__ __forceinline__ SArr<float> q() const { return PMBS_SARR(L->o_q, 4 * L->NB, CHK_Q); }  // 4 rows
    __device__ __forceinline__ SArr<float> h() const { return PMBS_SARR(L->o_h, 3 * L->NB, CHK_H); }
    __device__ __forceinline__ SArr<float> ib() const { return PMBS_SARR(L->o_ib, 3 * L->NB, CHK_IB); }
    __device__ __forceinline__ SArr<float> R() const { return PMBS_SARR(L->o_R, 9 * L->NB, CHK_R); }  // 9 rows
    __device__ __forceinline__ SArr<float> lo() const { return PMBS_SARR(L->o_lo, 3 * L->NB, CHK_LO); }
    __device__ __forceinline__ SArr<float> hi() const { return PMBS_SARR(L->o_hi, 3 * L->NB, CHK_HI); }
    __device__ __forceinline__ SArr<uint32_t> mask() const { return PMBS_SARR(L->o_mask, L->NB, CHK_MASK); }
    __device__ __forceinline__ SArr<int> scal() const { return PMBS_SARR(L->o_scal, 16, CHK_SCAL); }
    // event counters, written by the group's first lane only
    __device__ __forceinline__ SArr<unsigned long long> ev() const { return PMBS_SARR(L->o_ev, kNumEvents, CHK_EV); }
    // phase cycle counters (kNumPhases), after the event counters
    __device__ __forceinline__ SArr<unsigned long long> ph() const {
        return PMBS_SARR(L->o_ev + 8 * kNumEvents, kNumPhases, CHK_PH);
    }
    __device__ __forceinline__ SArr<uint16_t> mAB() const { return PMBS_SARR(L->o_mAB, L->Mcap, CHK_MAB); }
    __device__ __forceinline__ SArr<uint16_t> order() const { return PMBS_SARR(L->o_order, L->Mcap, CHK_ORDER); }
    __device__ __forceinline__ SArr<uint16_t> cstart() const {
        return PMBS_SARR(L->o_cstart, kMaxColours + 2, CHK_CSTART);
    }
    __device__ __forceinline__ SArr<uint16_t> pairs() const { return PMBS_SARR(L->o_pairs, L->pairS, CHK_PAIRS); }
    __device__ __forceinline__ SArr<uint8_t> mcol() const { return PMBS_SARR(L->o_mcol, L->Mcap, CHK_MCOL); }
    __device__ __forceinline__ SArr<uint8_t> plane() const { return PMBS_SARR(L->o_plane, L->NB, CHK_PLANE); }
    __device__ __forceinline__ SArr<uint8_t> pusher() const { return PMBS_SARR(L->o_pusher, L->NB, CHK_PUSHER); }
    // contacts: shared memory below Ms, global scratch above
    __device__ __forceinline__ float4* con_s() const { return reinterpret_cast<float4*>(pmbs_smem + base + L->o_con); }
    __device__ __forceinline__ int NB() const { return L->NB; }
    __device__ __forceinline__ int Ms() const { return L->Ms; }
    __device__ __forceinline__ int Mcap() const { return L->Mcap; }
    __device__ __forceinline__ int pairS() const { return L->pairS; }
};

// base: the warp region's byte offset in the block's dynamic shared memory; L must be a
// kernel parameter.
__device__ __forceinline__ WarpMem bind_mem(const Layout& L, uint32_t base, float4* gscratch) {
    WarpMem W;
    W.base = base;
    W.L = &L;
    W.con_g = gscratch;
    return W;
}

// Field access for manifold m: field k at ref.p[k * ref.stride].
struct CRef {
    float4* p;
    int stride;
    __device__ __forceinline__ float4& f(int k) const { return p[k * stride]; }
    __device__ __forceinline__ float4& pt(int slot, int k) const { return p[(3 + 4 * slot + k) * stride]; }
};

__device__ __forceinline__ CRef cref(const WarpMem& W, int m) {
    CRef r;
#if PMBS_BOUNDS_CHECK
    if (!check_index(CHK_MANIFOLD, m, W.Mcap())) {
        r.p = g_check_sink;  // every field of a bad manifold index lands on the sink
        r.stride = 0;
        return r;
    }
#endif
    if (m < W.Ms()) {
        r.p = W.con_s() + m;
        r.stride = W.Ms();
    } else {
        r.p = W.con_g + m;
        r.stride = W.Mcap();
    }
    return r;
}

// A group of G consecutive lanes (G = 8, 16 or 32) works on one environment; a warp
// holds 32 / G environments.  Every warp collective is issued by all 32 lanes at the same
// point; the helpers below restrict its result to the calling lane's group.
constexpr unsigned kFull = 0xffffffffu;

struct Grp {
    int G;          // lanes per environment
    int gl;         // lane index inside the group
    int shift;      // warp lane of the group's first lane
    unsigned bits;  // the group's lanes as a warp lane mask
    __device__ __forceinline__ Grp(int G_, int lane) : G(G_), gl(lane & (G_ - 1)), shift(lane & ~(G_ - 1)) {
        bits = (G_ == 32) ? kFull : (((1u << G_) - 1u) << shift);
    }
    // ballot restricted to the group, bit i = group lane i
    __device__ __forceinline__ unsigned ballot(bool p) const { return (__ballot_sync(kFull, p) & bits) >> shift; }
    __device__ __forceinline__ bool any(bool p) const { return (__ballot_sync(kFull, p) & bits) != 0u; }
    __device__ __forceinline__ unsigned lt() const { return (1u << gl) - 1u; }
    __device__ __forceinline__ int excl_scan(int v, int& total) const {
        int s = v;
        for (int o = 1; o < G; o <<= 1) {
            const int t = __shfl_up_sync(kFull, s, o, G);
            if (gl >= o) s += t;
        }
        total = __shfl_sync(kFull, s, G - 1, G);
        return s - v;
    }
    __device__ __forceinline__ int sum(int v) const {
        for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o, G);
        return v;
    }
    __device__ __forceinline__ int vmax(int v) const {
        for (int o = G >> 1; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(kFull, v, o, G));
        return v;
    }
    __device__ __forceinline__ int bcast(int v, int src) const { return __shfl_sync(kFull, v, src, G); }
    __device__ __forceinline__ float bcast(float v, int src) const { return __shfl_sync(kFull, v, src, G); }
};

// Phase clock of a group: on a mark, the group's first lane adds the cycles since the
// previous mark to phase k of its environment (when `rec`).  en = SimConst::timers, a
// launch-uniform value, so a launch without timers pays one branch per mark.
struct PhaseClock {
    long long t = 0;
    __device__ __forceinline__ void start(bool en) {
        if (en) t = clock64();
    }
    __device__ __forceinline__ void mark(bool en, const WarpMem& W, int k, bool rec) {
        if (en) {
            const long long now = clock64();
            if (rec) W.ph()[k] += (unsigned long long)(now - t);
            t = now;
        }
    }
};

// Warp-uniform loop bound: the largest per-group bound.
__device__ __forceinline__ int wmax(int v) { return __reduce_max_sync(kFull, v); }

__device__ __forceinline__ CBox load_cbox(const WarpMem& W, int i) {
    const int NB = W.NB();
    CBox b;
    b.c = f3(W.x()[i], W.x()[NB + i], W.x()[2 * NB + i]);
#pragma unroll
    for (int k = 0; k < 9; k++) b.R[k] = W.R()[k * NB + i];
    b.h[0] = W.h()[i];
    const float h1 = W.h()[NB + i];  // negative: a cylinder of radius h0
    b.h[1] = fabsf(h1);
    b.h[2] = W.h()[2 * NB + i];
    b.cyl = h1 < 0.f;
    return b;
}

// Per-push pusher state (uniform within a group).
struct Pusher {
    bool active;
    float sx, sy, dx, dy;
    int moving;
};

__device__ __forceinline__ Pusher make_pusher(const SimConst& C, const float* push, bool noop) {
    Pusher p;
    const float dx = push[2] - push[0], dy = push[3] - push[1];
    const float L = sqrtf(dx * dx + dy * dy);
    p.active = !noop && (L > 1e-9f);
    p.sx = push[0];
    p.sy = push[1];
    p.dx = p.active ? dx / L : 0.f;
    p.dy = p.active ? dy / L : 0.f;
    long mv = p.active ? lroundf(L / (C.pspeed * C.dt)) : 0;
    if (mv > C.substeps) mv = C.substeps;
    if (mv < 0) mv = 0;
    p.moving = (int)mv;
    return p;
}

// ------------------------------------------------------------------ frames + broadphase
// Per box: rotation (exact), world inverse inertia, AABB (exact).  n = 0 for a group
// without work in this phase (every function below accepts that).
__device__ __forceinline__ void frames_and_aabb(const WarpMem& W, int n, const Grp& g, float margin) {
    const int NB = W.NB();
    for (int i = g.gl; i < n; i += g.G) {
        float R[9];
        quat_to_R_exact(W.q()[i], W.q()[NB + i], W.q()[2 * NB + i], W.q()[3 * NB + i], R);
#pragma unroll
        for (int k = 0; k < 9; k++) W.R()[k * NB + i] = R[k];
        const float i0 = W.ib()[i], i1 = W.ib()[NB + i], i2 = W.ib()[2 * NB + i];
        // R diag(ib) R^T
        const float I00 = R[0] * i0 * R[0] + R[1] * i1 * R[1] + R[2] * i2 * R[2];
        const float I01 = R[0] * i0 * R[3] + R[1] * i1 * R[4] + R[2] * i2 * R[5];
        const float I02 = R[0] * i0 * R[6] + R[1] * i1 * R[7] + R[2] * i2 * R[8];
        const float I11 = R[3] * i0 * R[3] + R[4] * i1 * R[4] + R[5] * i2 * R[5];
        const float I12 = R[3] * i0 * R[6] + R[4] * i1 * R[7] + R[5] * i2 * R[8];
        const float I22 = R[6] * i0 * R[6] + R[7] * i1 * R[7] + R[8] * i2 * R[8];
        W.bI0()[i] = make_float4(I00, I01, I02, I11);
        W.bI1()[i] = make_float4(I12, I22, 0.f, 0.f);
        const float h0 = W.h()[i], h1 = W.h()[NB + i], h2 = W.h()[2 * NB + i];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const float e = aabb_half_exact(R + 3 * k, h0, h1, h2);
            const float c = W.x()[k * NB + i];
            W.lo()[k * NB + i] = xs(xs(c, e), margin);
            W.hi()[k * NB + i] = xa(xa(c, e), margin);
        }
    }
}

// Pair (i, j), i < j, of lexicographic index t among n boxes.
__device__ __forceinline__ void pair_of_index(int t, int n, int& i, int& j) {
    const float b = (float)(2 * n - 1);
    int r = (int)((b - sqrtf(fmaxf(b * b - 8.f * (float)t, 0.f))) * 0.5f);
    r = max(0, min(r, n - 2));
    auto start = [n](int a) { return a * (2 * n - a - 1) / 2; };
    while (r > 0 && start(r) > t) r--;
    while (r < n - 2 && start(r + 1) <= t) r++;
    i = r;
    j = t - start(r) + r + 1;
}

// Pair lists at the current AABBs: box-box pairs (i<j, lexicographic, capped), boxes
// reaching below the plane, boxes meeting the pusher's AABB.  Writes counts to scal[0..2]
// and returns true if the pair cap dropped pairs.
__device__ __forceinline__ bool broadphase(const WarpMem& W, int n, const Grp& g, int pair_cap, bool pusher_on,
                                           float Px, float Py, const SimConst& C) {
    const int NB = W.NB();
    const int cap = min(pair_cap, W.pairS());
    // Row by row: the lane of row i tests every j > i (neighbouring lanes read
    // neighbouring boxes, so the shared loads do not conflict) and keeps a bit mask; rows
    // are emitted in order and bits in ascending j, which is the lexicographic pair order.
    const int rw = wmax(n);
    int np = 0;
    bool overflow = false;
    for (int base = 0; base < rw; base += g.G) {
        const int i = base + g.gl;
        unsigned long long mask = 0ull;
        if (i < n) {
            const float lx = W.lo()[i], hx = W.hi()[i], ly = W.lo()[NB + i], hy = W.hi()[NB + i];
            const float lz = W.lo()[2 * NB + i], hz = W.hi()[2 * NB + i];
            // all six bounds loaded, then combined without short-circuits: one load latency
            // per candidate instead of six dependent load-compare-branch steps
            for (int j = i + 1; j < n; j++) {
                const float hxj = W.hi()[j], lxj = W.lo()[j], hyj = W.hi()[NB + j], lyj = W.lo()[NB + j];
                const float hzj = W.hi()[2 * NB + j], lzj = W.lo()[2 * NB + j];
                const bool ov = (lx <= hxj) & (lxj <= hx) & (ly <= hyj) & (lyj <= hy) & (lz <= hzj) & (lzj <= hz);
                mask |= (unsigned long long)ov << j;
            }
        }
        int total;
        const int pos0 = np + g.excl_scan(__popcll(mask), total);
        int pos = pos0;
        while (mask) {
            const int j = __ffsll((long long)mask) - 1;
            mask &= mask - 1ull;
            if (pos < cap) W.pairs()[pos] = (uint16_t)(i | (j << 8));
            else overflow = true;
            pos++;
        }
        np += total;
    }
    overflow = g.any(overflow);
    int npl = 0, npu = 0;
    const float rm = xa(C.pr, C.margin);
    const float plo0 = xs(Px, rm), plo1 = xs(Py, rm), plo2 = xs(C.pz0, rm);
    const float phi0 = xa(Px, rm), phi1 = xa(Py, rm), phi2 = xa(C.pz1, rm);
    const int nw = wmax(n);
    for (int b = 0; b < nw; b += g.G) {
        const int i = b + g.gl;
        const bool pl = i < n && W.lo()[2 * NB + i] < 0.f;
        bool pu = false;
        if (pusher_on && i < n)
            pu = W.lo()[i] <= phi0 && plo0 <= W.hi()[i] && W.lo()[NB + i] <= phi1 && plo1 <= W.hi()[NB + i] &&
                 W.lo()[2 * NB + i] <= phi2 && plo2 <= W.hi()[2 * NB + i];
        const unsigned mp = g.ballot(pl);
        const unsigned mu = g.ballot(pu);
        if (pl) W.plane()[npl + __popc(mp & g.lt())] = (uint8_t)i;
        if (pu) W.pusher()[npu + __popc(mu & g.lt())] = (uint8_t)i;
        npl += __popc(mp);
        npu += __popc(mu);
    }
    if (g.gl == 0) {
        W.scal()[0] = min(np, cap);
        W.scal()[1] = npl;
        W.scal()[2] = npu;
    }
    __syncwarp();
    return overflow;
}

// ------------------------------------------------------------------ narrowphase + emission
struct NarrowStats {
    int sat, face, edge, plane, pusher, clip_verts, bb_points;
};

// Running emission state: manifolds M and points P emitted so far; stop once a manifold
// did not fit (it and every later one are dropped).
struct Emit {
    int M, P;
    bool stop;
};

// Emit one chunk of candidates (one per group lane) in lane order, honouring the caps.
// kind: 0 box-box (p = world point), 1 plane (p = offset from the box centre),
// 2 pusher (p = world point on the box).  Returns the number of points emitted by the
// chunk's box-box candidates (for the event counters).
__device__ __forceinline__ int emit_chunk(const WarpMem& W, const Grp& g, const SimConst& C, Emit& E,
                                          const CManifold& cm, int A, int B, float mu, int kind, float3 cA,
                                          float3 cB) {
    const bool has = cm.np > 0;
    const unsigned hm = g.ballot(has);
    const int mpre = __popc(hm & g.lt());
    int ptot;
    const int ppre = g.excl_scan(cm.np, ptot);
    const bool fits = !E.stop && (E.M + mpre + 1 <= C.Mcap) && (E.P + ppre + cm.np <= C.Pcap);
    const unsigned viol = g.ballot(has && !fits);
    const int first = viol ? __ffs(viol) - 1 : 32;
    const bool ok = has && g.gl < first;
    if (ok) {
        const int mi = E.M + mpre;
        const CRef r = cref(W, mi);
        r.f(0) = make_float4(cm.n.x, cm.n.y, cm.n.z, mu);
        r.f(1) = make_float4(0.f, 0.f, 0.f, __int_as_float(A | (B << 8) | (cm.np << 16)));
        r.f(2) = make_float4(0.f, 0.f, 0.f, 0.f);
        W.mAB()[mi] = (uint16_t)(A | (B << 8));
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (k >= cm.np) break;
            float3 rA, rB;
            if (kind == 1) {
                rA = f3(0.f, 0.f, 0.f);
                rB = cm.p[k];
            } else if (kind == 2) {
                rA = cm.p[k] - cA;
                rB = f3(0.f, 0.f, 0.f);
            } else {
                rA = cm.p[k] - cA;
                rB = cm.p[k] - cB;
            }
            r.pt(k, 0) = make_float4(rA.x, rA.y, rA.z, 0.f);
            r.pt(k, 1) = make_float4(rB.x, rB.y, rB.z, 0.f);
            r.pt(k, 3) = make_float4(0.f, cm.d[k], 0.f, 0.f);
        }
    }
    const unsigned okm = g.ballot(ok);
    int pemit;
    g.excl_scan(ok ? cm.np : 0, pemit);
    E.M += __popc(okm);
    E.P += pemit;
    if (viol) E.stop = true;
    return g.sum((ok && kind == 0) ? cm.np : 0);
}

// Candidates in order (box-box pairs, plane, pusher), one pass per kind; each yields at
// most four points sharing a normal.  Manifolds are emitted in candidate order until the
// manifold or point capacity would be exceeded; that manifold and every later one are
// dropped.  Writes M, P to scal[3], scal[4] and the box-box manifold count to scal[7],
// plane manifolds to scal[8]; returns true on overflow.  kCyl compiles the cylinder
// contact paths in (batches without cylinders run the instantiation without them).
template <bool kCyl>
__device__ __forceinline__ bool narrowphase(const WarpMem& W, const Grp& g, bool on, const SimConst& C, float Px,
                                            float Py, NarrowStats& st) {
    const int npairs = on ? W.scal()[0] : 0, nplane = on ? W.scal()[1] : 0, npush = on ? W.scal()[2] : 0;
    Emit E{0, 0, false};
    int sat = 0, face = 0, edge = 0, clipv = 0;
    const int pw = wmax(npairs);
    for (int base = 0; base < pw; base += g.G) {
        const int c = base + g.gl;
        CManifold cm;
        cm.np = 0;
        int A = 0, B = 0;
        float mu = 0.f;
        float3 cA = f3(0.f, 0.f, 0.f), cB = cA;
        if (c < npairs && !E.stop) {
            const int pr = W.pairs()[c];
            A = pr & 255;
            B = pr >> 8;
            const CBox a = load_cbox(W, A), b = load_cbox(W, B);
            sat++;
            // with the cylinder paths compiled in, box pairs go through the general convex
            // routine too (the same axes, thresholds and tie rules as the box-box routine):
            // the lanes of a warp stay in one routine and the code stays smaller
            const int kd = kCyl ? collide_convex(a, b, C.margin, cm, clipv) : collide_box_box(a, b, C.margin, cm, clipv);
            if (kd == 1) face++;
            if (kd == 2) edge++;
            mu = sqrtf(W.bw()[A].w * W.bw()[B].w);
            cA = a.c;
            cB = b.c;
        }
        st.bb_points += emit_chunk(W, g, C, E, cm, A, B, mu, 0, cA, cB);
    }
    const int Mbb = E.M;
    const int lw = wmax(nplane);
    for (int base = 0; base < lw; base += g.G) {
        const int c = base + g.gl;
        CManifold cm;
        cm.np = 0;
        int B = 0;
        float mu = 0.f;
        float3 cB = f3(0.f, 0.f, 0.f);
        if (c < nplane && !E.stop) {
            B = W.plane()[c];
            const CBox b = load_cbox(W, B);
            if (kCyl && b.cyl) collide_cyl_plane(b, C.margin, cm);
            else collide_box_plane(b, C.margin, cm);
            mu = sqrtf(W.bw()[B].w * C.table_mu);
            cB = b.c;
        }
        emit_chunk(W, g, C, E, cm, kPlane, B, mu, 1, f3(0.f, 0.f, 0.f), cB);
    }
    const int Mpl = E.M - Mbb;
    const int uw = wmax(npush);
    for (int base = 0; base < uw; base += g.G) {
        const int c = base + g.gl;
        CManifold cm;
        cm.np = 0;
        int A = 0;
        float mu = 0.f;
        float3 cA = f3(0.f, 0.f, 0.f);
        if (c < npush && !E.stop) {
            A = W.pusher()[c];
            const CBox a = load_cbox(W, A);
            if (kCyl && a.cyl) collide_capsule_cyl(a, Px, Py, C.pz0, C.pz1, C.pr, C.margin, cm);
            else collide_capsule_box(a, Px, Py, C.pz0, C.pz1, C.pr, C.margin, cm);
            mu = sqrtf(W.bw()[A].w * C.pusher_mu);
            cA = a.c;
        }
        emit_chunk(W, g, C, E, cm, A, kPusher, mu, 2, cA, f3(0.f, 0.f, 0.f));
    }
    st.sat += g.sum(sat);
    st.face += g.sum(face);
    st.edge += g.sum(edge);
    st.clip_verts += g.sum(clipv);
    st.plane += nplane;
    st.pusher += npush;
    if (g.gl == 0 && on) {
        W.scal()[3] = E.M;
        W.scal()[4] = E.P;
        W.scal()[7] = Mbb;
        W.scal()[8] = Mpl;
    }
    __syncwarp();
    return E.stop;
}

// ------------------------------------------------------------------ contact preparation
__device__ __forceinline__ float3 sym_mul(float4 I0, float4 I1, float3 v) {
    return f3(I0.x * v.x + I0.y * v.y + I0.z * v.z, I0.y * v.x + I0.w * v.y + I1.x * v.z,
              I0.z * v.x + I1.x * v.y + I1.y * v.z);
}

// Tangent basis from the world axis least aligned with n; inverse effective masses along
// n, t1, t2; target normal velocity (speculative -d/dt when separated, Baumgarte
// beta/dt * max(-d - slop, 0) when penetrating); impulses start at zero.
__device__ __forceinline__ void prepare(const WarpMem& W, const Grp& g, bool on, const SimConst& C) {
    const int M = on ? W.scal()[3] : 0;
    for (int m = g.gl; m < M; m += g.G) {
        const CRef r = cref(W, m);
        const float4 h0 = r.f(0), h1 = r.f(1);
        const float3 n = f3(h0.x, h0.y, h0.z);
        const int ids = __float_as_int(h1.w);
        const int A = ids & 255, B = (ids >> 8) & 255, np = (ids >> 16) & 255;
        const float an0 = fabsf(n.x), an1 = fabsf(n.y), an2 = fabsf(n.z);
        int k = 0;
        float amin = an0;
        if (an1 < amin) { k = 1; amin = an1; }
        if (an2 < amin) k = 2;
        const float3 e = f3(k == 0 ? 1.f : 0.f, k == 1 ? 1.f : 0.f, k == 2 ? 1.f : 0.f);
        float3 t1 = cross3(n, e);
        t1 = t1 * rsqrtf(dot3(t1, t1));
        const float3 t2 = cross3(n, t1);
        r.f(1) = make_float4(t1.x, t1.y, t1.z, h1.w);
        r.f(2) = make_float4(t2.x, t2.y, t2.z, 0.f);
        const bool dA = A < kPusher, dB = B < kPusher;
        float4 IA0 = make_float4(0.f, 0.f, 0.f, 0.f), IA1 = IA0, IB0 = IA0, IB1 = IA0;
        float imA = 0.f, imB = 0.f;
        if (dA) { IA0 = W.bI0()[A]; IA1 = W.bI1()[A]; imA = W.bv()[A].w; }
        if (dB) { IB0 = W.bI0()[B]; IB1 = W.bI1()[B]; imB = W.bv()[B].w; }
        for (int p = 0; p < np; p++) {
            const float4 q0 = r.pt(p, 0), q1 = r.pt(p, 1), q3 = r.pt(p, 3);
            const float3 rA = f3(q0.x, q0.y, q0.z), rB = f3(q1.x, q1.y, q1.z);
            const float d = q3.y;
            float kk[3];
            const float3 dirs[3] = {n, t1, t2};
#pragma unroll
            for (int j = 0; j < 3; j++) {
                float s = 0.f;
                if (dA) {
                    const float3 rn = cross3(rA, dirs[j]);
                    s += imA + dot3(rn, sym_mul(IA0, IA1, rn));
                }
                if (dB) {
                    const float3 rn = cross3(rB, dirs[j]);
                    s += imB + dot3(rn, sym_mul(IB0, IB1, rn));
                }
                kk[j] = __fdividef(1.f, s);
            }
            const float bias = d > 0.f ? __fdividef(-d, C.dt) : __fdividef(C.baumgarte, C.dt) * fmaxf(-d - C.slop, 0.f);
            r.pt(p, 0) = make_float4(rA.x, rA.y, rA.z, kk[0]);
            r.pt(p, 1) = make_float4(rB.x, rB.y, rB.z, bias);
            r.pt(p, 2) = make_float4(0.f, 0.f, 0.f, kk[1]);
            r.pt(p, 3) = make_float4(kk[2], d, 0.f, 0.f);
        }
    }
    __syncwarp();
}

// ------------------------------------------------------------------ colouring
// Greedy colouring in manifold order: each manifold takes the smallest colour (< 32) not
// used by an earlier manifold on a shared dynamic body.  Box-box manifolds come first and
// are walked in order by the group's first lane; every plane manifold is the only one of
// its box among the plane manifolds and follows all box-box manifolds, and likewise every
// pusher manifold follows all plane manifolds, so both groups are coloured lane-parallel
// from the box masks with exactly the sequential result.  Then a stable bucket sort of
// manifold ids by colour.  Returns true on colour overflow (manifold dropped).  Writes the
// colour count to scal[5] and the number of coloured manifolds to scal[6].
__device__ __forceinline__ bool colour_manifolds(const WarpMem& W, int n, const Grp& g, bool on) {
    const int M = on ? W.scal()[3] : 0, Mbb = on ? W.scal()[7] : 0, Mpl = on ? W.scal()[8] : 0;
    for (int i = g.gl; i < n; i += g.G) W.mask()[i] = 0u;
    __syncwarp();
    bool overflow = false;
    int cmax = -1;
    if (g.gl == 0) {
        for (int m = 0; m < Mbb; m++) {
            const int ab = W.mAB()[m];
            const int A = ab & 255, B = ab >> 8;
            const uint32_t u = W.mask()[A] | W.mask()[B];
            if (u == 0xffffffffu) {
                W.mcol()[m] = 255;
                overflow = true;
                continue;
            }
            const int c = __ffs(~u) - 1;
            W.mcol()[m] = (uint8_t)c;
            W.mask()[A] = W.mask()[A] | (1u << c);
            W.mask()[B] = W.mask()[B] | (1u << c);
            cmax = max(cmax, c);
        }
    }
    __syncwarp();
    // plane manifolds (body B is the box), then pusher manifolds (body A is the box)
    for (int grp = 0; grp < 2; grp++) {
        const int lo = grp == 0 ? Mbb : Mbb + Mpl, hi = grp == 0 ? Mbb + Mpl : M;
        for (int m = lo + g.gl; m < hi; m += g.G) {
            const int ab = W.mAB()[m];
            const int box = grp == 0 ? (ab >> 8) : (ab & 255);
            const uint32_t u = W.mask()[box];
            if (u == 0xffffffffu) {
                W.mcol()[m] = 255;
                overflow = true;
                continue;
            }
            const int c = __ffs(~u) - 1;
            W.mcol()[m] = (uint8_t)c;
            W.mask()[box] = u | (1u << c);
            cmax = max(cmax, c);
        }
        __syncwarp();
    }
    const int ncol = g.vmax(cmax + 1);
    const int cw = wmax(ncol), mw = wmax(M);
    int pos = 0;
    for (int c = 0; c < cw; c++) {
        if (g.gl == 0 && c < ncol) W.cstart()[c] = (uint16_t)pos;
        for (int base = 0; base < mw; base += g.G) {
            const int m = base + g.gl;
            const bool is = c < ncol && m < M && W.mcol()[m] == c;
            const unsigned bal = g.ballot(is);
            if (is) W.order()[pos + __popc(bal & g.lt())] = (uint16_t)m;
            pos += __popc(bal);
        }
    }
    if (g.gl == 0 && on) {
        W.cstart()[ncol] = (uint16_t)pos;
        W.scal()[5] = ncol;
        W.scal()[6] = pos;
    }
    __syncwarp();
    return g.any(overflow);
}

// ------------------------------------------------------------------ PGS
// One manifold's Gauss-Seidel update: all normal rows, then all friction pairs.  Returns
// the number of points; bb_pts gets them too when both bodies are dynamic.
__device__ __forceinline__ int solve_manifold(const WarpMem& W, int m, float3 pusherV, int& bb_pts) {
    const CRef r = cref(W, m);
    const float4 h0 = r.f(0), h1 = r.f(1), h2 = r.f(2);
    const float3 n = f3(h0.x, h0.y, h0.z), t1 = f3(h1.x, h1.y, h1.z), t2 = f3(h2.x, h2.y, h2.z);
    const float mu = h0.w;
    const int ids = __float_as_int(h1.w);
    const int A = ids & 255, B = (ids >> 8) & 255, np = (ids >> 16) & 255;
    const bool dA = A < kPusher, dB = B < kPusher;
    float3 vA = f3(0.f, 0.f, 0.f), wA = vA, vB = vA, wB = vA;
    float imA = 0.f, imB = 0.f, muA = 0.f, muB = 0.f;
    float4 IA0 = make_float4(0.f, 0.f, 0.f, 0.f), IA1 = IA0, IB0 = IA0, IB1 = IA0;
    if (dA) {
        const float4 a = W.bv()[A], b = W.bw()[A];
        vA = f3(a.x, a.y, a.z);
        imA = a.w;
        wA = f3(b.x, b.y, b.z);
        muA = b.w;
        IA0 = W.bI0()[A];
        IA1 = W.bI1()[A];
    }
    if (dB) {
        const float4 a = W.bv()[B], b = W.bw()[B];
        vB = f3(a.x, a.y, a.z);
        imB = a.w;
        wB = f3(b.x, b.y, b.z);
        muB = b.w;
        IB0 = W.bI0()[B];
        IB1 = W.bI1()[B];
    } else if (B == kPusher) {
        vB = pusherV;
    }
    for (int p = 0; p < np; p++) {
        const float4 q0 = r.pt(p, 0), q1 = r.pt(p, 1);
        float4 q2 = r.pt(p, 2);
        const float3 rA = f3(q0.x, q0.y, q0.z), rB = f3(q1.x, q1.y, q1.z);
        const float3 vr = (vB + cross3(wB, rB)) - (vA + cross3(wA, rA));
        const float vn = dot3(n, vr);
        const float delta = -(vn - q1.w) * q0.w;
        const float l = fmaxf(q2.x + delta, 0.f);
        const float dl = l - q2.x;
        q2.x = l;
        r.pt(p, 2) = q2;
        const float3 P = n * dl;
        vA = vA - P * imA;
        wA = wA - sym_mul(IA0, IA1, cross3(rA, P));
        vB = vB + P * imB;
        wB = wB + sym_mul(IB0, IB1, cross3(rB, P));
    }
    for (int p = 0; p < np; p++) {
        const float4 q0 = r.pt(p, 0), q1 = r.pt(p, 1), q3 = r.pt(p, 3);
        float4 q2 = r.pt(p, 2);
        const float3 rA = f3(q0.x, q0.y, q0.z), rB = f3(q1.x, q1.y, q1.z);
        const float3 vr = (vB + cross3(wB, rB)) - (vA + cross3(wA, rA));
        const float vt1 = dot3(t1, vr), vt2 = dot3(t2, vr);
        float c1 = q2.y - vt1 * q2.w;
        float c2 = q2.z - vt2 * q3.x;
        const float lim = mu * q2.x;
        const float l2 = c1 * c1 + c2 * c2;
        if (l2 > lim * lim) {
            const float sc = lim * rsqrtf(l2);
            c1 *= sc;
            c2 *= sc;
        }
        const float d1 = c1 - q2.y, d2 = c2 - q2.z;
        q2.y = c1;
        q2.z = c2;
        r.pt(p, 2) = q2;
        const float3 P = t1 * d1 + t2 * d2;
        vA = vA - P * imA;
        wA = wA - sym_mul(IA0, IA1, cross3(rA, P));
        vB = vB + P * imB;
        wB = wB + sym_mul(IB0, IB1, cross3(rB, P));
    }
    if (dA) {
        W.bv()[A] = make_float4(vA.x, vA.y, vA.z, imA);
        W.bw()[A] = make_float4(wA.x, wA.y, wA.z, muA);
    }
    if (dB) {
        W.bv()[B] = make_float4(vB.x, vB.y, vB.z, imB);
        W.bw()[B] = make_float4(wB.x, wB.y, wB.z, muB);
    }
    if (dA && dB) bb_pts += np;
    return np;
}

// Returns the number of point visits (normal + friction row pairs) of this lane, and
// in bb_visits those of manifolds between two dynamic bodies.
__device__ __forceinline__ int pgs(const WarpMem& W, const Grp& g, bool on, int iters, float3 pusherV,
                                   int& bb_visits) {
    const int ncol = on ? W.scal()[5] : 0;
    const int cw = wmax(ncol);
    int visits = 0;
    for (int it = 0; it < iters; it++) {
        for (int c = 0; c < cw; c++) {
            const int a = c < ncol ? (int)W.cstart()[c] : 0, b = c < ncol ? (int)W.cstart()[c + 1] : 0;
            for (int k = a + g.gl; k < b; k += g.G) visits += solve_manifold(W, W.order()[k], pusherV, bb_visits);
            __syncwarp();
        }
    }
    return visits;
}

// ------------------------------------------------------------------ warm start (option)
// Cache record of one manifold (kWarmF4 float4 in global memory, per environment):
// [0] = (body-pair key A | B << 8, np, -, -) as integer bits; point p: [1 + 2p] =
// (offset in the key body's frame, lambda_n), [2 + 2p] = (world friction impulse, -).
// The key body is A when dynamic, else B.
constexpr int kWarmF4 = 9;

__device__ __forceinline__ float3 key_local(const WarpMem& W, int kb, float3 r) {
    const int NB = W.NB();
    const SArr<float> R = W.R();
    return f3(R[kb] * r.x + R[3 * NB + kb] * r.y + R[6 * NB + kb] * r.z,
              R[NB + kb] * r.x + R[4 * NB + kb] * r.y + R[7 * NB + kb] * r.z,
              R[2 * NB + kb] * r.x + R[5 * NB + kb] * r.y + R[8 * NB + kb] * r.z);
}

// A new point takes the impulses of the nearest unused point of the same body pair in the
// previous substep's cache within the tolerance (new points in order; the friction
// vector is projected on the new tangents); then the carried impulses are applied to the
// bodies, colour by colour (within a colour the manifolds share no dynamic body).
__device__ __forceinline__ void warm_start(const WarpMem& W, const Grp& g, bool on, const SimConst& C,
                                           const float4* cache, int Mold) {
    const int M = on ? W.scal()[3] : 0;
#if PMBS_BOUNDS_CHECK
    if (!check_index(CHK_WARM, Mold, W.Mcap() + 1)) Mold = 0;
#endif
    for (int m = g.gl; m < M; m += g.G) {
        if (W.mcol()[m] == 255) continue;
        const CRef r = cref(W, m);
        const float4 h1 = r.f(1), h2 = r.f(2);
        const float3 t1 = f3(h1.x, h1.y, h1.z), t2 = f3(h2.x, h2.y, h2.z);
        const int ids = __float_as_int(h1.w);
        const int A = ids & 255, B = (ids >> 8) & 255, np = (ids >> 16) & 255;
        const int key = A | (B << 8);
        int om = -1;
        for (int q = 0; q < Mold; q++)
            if (__float_as_int(cache[(size_t)q * kWarmF4].x) == key) {
                om = q;
                break;
            }
        if (om < 0) continue;
        const float4* rec = cache + (size_t)om * kWarmF4;
        const int onp = __float_as_int(rec[0].y);
        const bool kA = A < kPusher;
        const int kb = kA ? A : B;
        unsigned used = 0u;
        for (int p = 0; p < np; p++) {
            const float4 q = kA ? r.pt(p, 0) : r.pt(p, 1);
            const float3 loc = key_local(W, kb, f3(q.x, q.y, q.z));
            int best = -1;
            float bd = C.warm_tol2;
            for (int o = 0; o < onp; o++) {
                if (used >> o & 1u) continue;
                const float4 ol = rec[1 + 2 * o];
                const float3 d = loc - f3(ol.x, ol.y, ol.z);
                const float d2 = dot3(d, d);
                if (d2 <= bd) {
                    bd = d2;
                    best = o;
                }
            }
            if (best < 0) continue;
            used |= 1u << best;
            const float4 ol = rec[1 + 2 * best], op = rec[2 + 2 * best];
            const float3 Pt = f3(op.x, op.y, op.z);
            float4 q2 = r.pt(p, 2);
            q2.x = ol.w;
            q2.y = dot3(Pt, t1);
            q2.z = dot3(Pt, t2);
            r.pt(p, 2) = q2;
        }
    }
    __syncwarp();
    const int ncol = on ? W.scal()[5] : 0;
    const int cw = wmax(ncol);
    for (int c = 0; c < cw; c++) {
        const int a = c < ncol ? (int)W.cstart()[c] : 0, b = c < ncol ? (int)W.cstart()[c + 1] : 0;
        for (int k = a + g.gl; k < b; k += g.G) {
            const CRef r = cref(W, W.order()[k]);
            const float4 h0 = r.f(0), h1 = r.f(1), h2 = r.f(2);
            const float3 n = f3(h0.x, h0.y, h0.z), t1 = f3(h1.x, h1.y, h1.z), t2 = f3(h2.x, h2.y, h2.z);
            const int ids = __float_as_int(h1.w);
            const int A = ids & 255, B = (ids >> 8) & 255, np = (ids >> 16) & 255;
            float3 PA = f3(0.f, 0.f, 0.f), LA = PA, LB = PA;
            for (int p = 0; p < np; p++) {
                const float4 q0 = r.pt(p, 0), q1 = r.pt(p, 1), q2 = r.pt(p, 2);
                const float3 P = (n * q2.x + t1 * q2.y) + t2 * q2.z;
                PA = PA + P;
                LA = LA + cross3(f3(q0.x, q0.y, q0.z), P);
                LB = LB + cross3(f3(q1.x, q1.y, q1.z), P);
            }
            if (A < kPusher) {
                const float4 v = W.bv()[A], w = W.bw()[A];
                const float3 nv = f3(v.x, v.y, v.z) - PA * v.w;
                const float3 nw = f3(w.x, w.y, w.z) - sym_mul(W.bI0()[A], W.bI1()[A], LA);
                W.bv()[A] = make_float4(nv.x, nv.y, nv.z, v.w);
                W.bw()[A] = make_float4(nw.x, nw.y, nw.z, w.w);
            }
            if (B < kPusher) {
                const float4 v = W.bv()[B], w = W.bw()[B];
                const float3 nv = f3(v.x, v.y, v.z) + PA * v.w;
                const float3 nw = f3(w.x, w.y, w.z) + sym_mul(W.bI0()[B], W.bI1()[B], LB);
                W.bv()[B] = make_float4(nv.x, nv.y, nv.z, v.w);
                W.bw()[B] = make_float4(nw.x, nw.y, nw.z, w.w);
            }
        }
        __syncwarp();
    }
}

// Cache this substep's manifolds (before integration, so offsets are taken in the frames
// the next substep's contacts will be compared in after their own update).  Returns the
// number of records (manifolds dropped by the colour cap are recorded with no points).
__device__ __forceinline__ int warm_save(const WarpMem& W, const Grp& g, bool on, float4* cache) {
    int M = on ? W.scal()[3] : 0;
#if PMBS_BOUNDS_CHECK
    if (!check_index(CHK_WARM, M, W.Mcap() + 1)) M = 0;
#endif
    for (int m = g.gl; m < M; m += g.G) {
        const CRef r = cref(W, m);
        const float4 h1 = r.f(1), h2 = r.f(2);
        const float3 t1 = f3(h1.x, h1.y, h1.z), t2 = f3(h2.x, h2.y, h2.z);
        const int ids = __float_as_int(h1.w);
        const int A = ids & 255, B = (ids >> 8) & 255;
        const int np = W.mcol()[m] == 255 ? 0 : (ids >> 16) & 255;
        float4* rec = cache + (size_t)m * kWarmF4;
        rec[0] = make_float4(__int_as_float(A | (B << 8)), __int_as_float(np), 0.f, 0.f);
        const bool kA = A < kPusher;
        const int kb = kA ? A : B;
        for (int p = 0; p < np; p++) {
            const float4 q = kA ? r.pt(p, 0) : r.pt(p, 1), q2 = r.pt(p, 2);
            const float3 loc = key_local(W, kb, f3(q.x, q.y, q.z));
            const float3 Pt = t1 * q2.y + t2 * q2.z;
            rec[1 + 2 * p] = make_float4(loc.x, loc.y, loc.z, q2.x);
            rec[2 + 2 * p] = make_float4(Pt.x, Pt.y, Pt.z, 0.f);
        }
    }
    __syncwarp();
    return M;
}

// ------------------------------------------------------------------ integration
__device__ __forceinline__ void integrate(const WarpMem& W, int n, const Grp& g, float dt) {
    const int NB = W.NB();
    for (int i = g.gl; i < n; i += g.G) {
        const float4 v = W.bv()[i], w = W.bw()[i];
        W.x()[i] += v.x * dt;
        W.x()[NB + i] += v.y * dt;
        W.x()[2 * NB + i] += v.z * dt;
        const float q0 = W.q()[i], q1 = W.q()[NB + i], q2 = W.q()[2 * NB + i], q3 = W.q()[3 * NB + i];
        const float3 om = f3(w.x, w.y, w.z), qv = f3(q1, q2, q3);
        const float dw = -dot3(om, qv);
        const float3 dv = om * q0 + cross3(om, qv);
        const float hd = 0.5f * dt;
        const float a0 = q0 + hd * dw, a1 = q1 + hd * dv.x, a2 = q2 + hd * dv.y, a3 = q3 + hd * dv.z;
        const float il = rsqrtf(a0 * a0 + a1 * a1 + a2 * a2 + a3 * a3);
        W.q()[i] = a0 * il;
        W.q()[NB + i] = a1 * il;
        W.q()[2 * NB + i] = a2 * il;
        W.q()[3 * NB + i] = a3 * il;
    }
    __syncwarp();
}

// ------------------------------------------------------------------ footprints & tests
// Footprints of every box at the current state into the R area (8 floats per box).
__device__ __forceinline__ void compute_footprints(const WarpMem& W, int n, const Grp& g) {
    const int NB = W.NB();
    for (int i = g.gl; i < n; i += g.G) {
        float R[9];
        quat_to_R_exact(W.q()[i], W.q()[NB + i], W.q()[2 * NB + i], W.q()[3 * NB + i], R);
        const Foot f = footprint_exact(W.x()[i], W.x()[NB + i], R, W.h()[i], W.h()[NB + i], W.h()[2 * NB + i]);
        const SArr<float> o = W.R();
        o[0 * NB + i] = f.cx;
        o[1 * NB + i] = f.cy;
        o[2 * NB + i] = f.ux;
        o[3 * NB + i] = f.uy;
        o[4 * NB + i] = f.vx;
        o[5 * NB + i] = f.vy;
        o[6 * NB + i] = f.su;
        o[7 * NB + i] = f.sv;
    }
    __syncwarp();
}

__device__ __forceinline__ Foot load_foot(const WarpMem& W, int i) {
    const int NB = W.NB();
    const SArr<float> o = W.R();
    Foot f;
    f.cx = o[i];
    f.cy = o[NB + i];
    f.ux = o[2 * NB + i];
    f.uy = o[3 * NB + i];
    f.vx = o[4 * NB + i];
    f.vy = o[5 * NB + i];
    f.su = o[6 * NB + i];
    f.sv = o[7 * NB + i];
    return f;
}

// Grasp-clearance decision on the footprints (Sec. IV-B grasp evaluation stand-in):
// lane pairs (angle k, finger side) test the finger sweep against every other footprint.
// on = false: the group takes no part (result false).
__device__ __forceinline__ bool grasp_check(const WarpMem& W, int n, int t, const Grp& g, bool on,
                                            const SimConst& C) {
    const Foot ft = on ? load_foot(W, t) : Foot{0.f, 0.f, 1.f, 0.f, 0.f, 1.f, 0.f, 0.f};
    const float halfW = xm(C.grasp_W, 0.5f), hfw = xm(C.grasp_fw, 0.5f);
    bool any = false;
    for (int sb = 0; sb < 2 * C.grasp_K; sb += g.G) {
        const int slot = sb + g.gl;
        const int k = slot >> 1;
        const float s = (slot & 1) ? -1.f : 1.f;
        bool ok = false;
        if (on && k < C.grasp_K) {
            const float ax = C.gcos[k], ay = C.gsin[k];
            const float bx = -ay, by = ax;
            const float wa = xa(xm(fabsf(xdot2(ft.ux, ft.uy, ax, ay)), ft.su), xm(fabsf(xdot2(ft.vx, ft.vy, ax, ay)), ft.sv));
            if (xm(xa(wa, C.grasp_c), 2.f) <= C.grasp_W) {
                const float off = xm(xa(xa(wa, halfW), C.grasp_f), 0.5f);
                const float hl = xm(xs(xa(halfW, C.grasp_f), wa), 0.5f);
                const float fcx = xa(ft.cx, s * xm(ax, off));
                const float fcy = xa(ft.cy, s * xm(ay, off));
                ok = true;
                for (int o = 0; o < n; o++) {
                    if (o == t) continue;
                    if (finger_overlaps_exact(load_foot(W, o), fcx, fcy, ax, ay, bx, by, hl, hfw)) {
                        ok = false;
                        break;
                    }
                }
            }
        }
        // every lane executes the collectives (no short-circuit around them)
        const bool partner = __shfl_xor_sync(kFull, ok, 1, g.G) != 0;
        const bool found = g.any(ok && partner);
        any = any || found;
    }
    return any;
}

// Start-pose check of a push starting at (px, py): any footprint within the pusher
// radius (Sec. IV-B: only the start pose is collision-checked).
__device__ __forceinline__ bool start_blocked(const WarpMem& W, int n, const Grp& g, float px, float py, float r) {
    bool hit = false;
    for (int i = g.gl; i < n; i += g.G) hit = hit || disc_hits_foot_exact(load_foot(W, i), px, py, r);
    return g.any(hit);
}

// Contour sampler for push k >= 2 (Sec. IV-B): lane a evaluates attempt a; the lowest
// unblocked attempt wins.  Returns the attempt (or -1) and the push in out[4].  on =
// false: the group takes no part.
__device__ __forceinline__ int sample_push(const WarpMem& W, int n, const Grp& g, bool on, uint64_t seed, int k,
                                           const SimConst& C, float* out) {
    int best = -1;
    for (int ab = 0; ab < C.attempts; ab += g.G) {
        const int a = ab + g.gl;
        float push[4] = {0.f, 0.f, 0.f, 0.f};
        bool good = false;
        if (on && best < 0 && a < C.attempts) {
            int j, p;
            sampler_draws(seed, k, a, n, C.npts, j, p);
            contour_push_exact(load_foot(W, j), p, C.npts, C.pr, C.sample_clear, C.plen, push);
            good = true;
            for (int o = 0; o < n; o++)
                if (disc_hits_foot_exact(load_foot(W, o), push[0], push[1], C.pr)) {
                    good = false;
                    break;
                }
        }
        const unsigned m = g.ballot(good);
        const int src = m ? __ffs(m) - 1 : 0;
        float moved[4];
        for (int i = 0; i < 4; i++) moved[i] = g.bcast(push[i], src);
        if (m && best < 0) {
            best = ab + src;
            for (int i = 0; i < 4; i++) out[i] = moved[i];
        }
    }
    return best;
}

}  // namespace pmbs

// FP64 CPU oracle of the batched push-rollout hot path of PMBS (parallel MCTS with
// batched simulation, Sec. IV-C).  TEST INFRASTRUCTURE ONLY: the product library never
// links, loads or calls this file; only the tests, the smoke check and the timed CPU
// baseline of the benchmark do.
//
// What it computes (Sec. III-A, Sec. IV-B, Sec. IV-C "Batch Simulation"): each
// environment holds boxes and cylinders (right prisms over a 16-gon, with the solid
// cylinder's inertia) on a table plane (z = 0) and a kinematic vertical capsule pusher
// that executes straight push actions a^p = (x_s, y_s, x_e, y_e).  The
// transition function is only described in the paper as quasi-static motion with
// friction and collisions (Sec. III-A, transition function), so every physics rule
// here is a stated reading, written once in plain sequential form:
//   substep = pusher kinematics, gravity, AABB broadphase, narrowphase (box-plane
//   vertices, box-box separating-axis test with face clipping or edge-edge point,
//   capsule-box closest points; pairs with a cylinder through the general convex
//   separating-axis test, cylinder-plane vertices, capsule-cylinder closest points),
//   contact preparation, greedy manifold colouring,
//   projected Gauss-Seidel with disk-clamped Coulomb friction, semi-implicit Euler.
// After each push: workspace bounds, grasp-clearance test standing in for the grasp
// classifier (Sec. IV-B), cost and discounted reward gamma^(k-1) (Sec. III-A, Sec. V-A
// gamma = 0.8).  Pushes after the first are drawn by the contour sampler of Sec. IV-B
// (a fixed number of start points spaced evenly around each object's outline, each push
// aimed inward at the object, only the start pose checked for collision) with SplitMix64
// (Steele, Lea, Flood 2014) as the generator.
//
// Precision: the trajectory runs in double.  The pair-list, grasp and sampler
// predicates are also instantiated in IEEE binary32 (templates below, each operation
// rounded once, compiled with -ffp-contract=off) so that decisions on identical FP32
// state snapshots can be compared bit-for-bit with the GPU.
//
// Flop counter: compiled with -DORACLE_COUNT_FLOPS (a separate library,
// liboracle_flops.so), the double engine's scalar type `real` becomes a counting type:
// every add, subtract, multiply, divide and square root counts 1 into the phase being
// run (compares, abs, min and max count 0; -ffp-contract=off keeps a multiply-add as 2).
// The default build has `real` = double, with the same arithmetic in the same order.
//
// Parity status: every function below is pinned by the CPU tests (closed forms,
// invariants, brute force), except whole multi-contact clutter trajectories, whose
// parity is unpinned (chaotic; FP32 and FP64 diverge).

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

extern "C" {
typedef struct {
    double dt;                 // substep length (s)
    double gravity[3];         // m/s^2
    double table_half[2];      // workspace half sizes (m)
    double table_mu, pusher_mu;
    double pusher_radius, pusher_z0, pusher_z1;  // capsule radius, segment z range
    double pusher_speed, push_length;
    double gamma;              // discount (Sec. V-A: 0.8)
    double grasp_opening, grasp_clearance, finger_depth, finger_width;
    double margin, slop, baumgarte;
    double sample_clearance;   // contour offset beyond the pusher radius
    int32_t substeps_per_push, pgs_iters;
    int32_t point_cap, manifold_cap, pair_cap;
    int32_t grasp_angles, sample_attempts, contour_points;
    int32_t warm_start;        // 0: impulses start at zero every substep; 1: carried over
    double warm_tolerance;     // match distance of a carried-over contact point (m)
} oracle_params;
}

namespace {

using std::fabs;
using std::sqrt;

enum { PLANE = -1, PUSHER = -2 };
enum {
    EV_SUBSTEPS = 0, EV_BOX_STEPS, EV_PAIR_TESTS, EV_SAT, EV_FACE, EV_EDGE, EV_PLANE,
    EV_PUSHER, EV_POINTS, EV_MANIFOLDS, EV_PGS_MAN, EV_PGS_PTS, EV_PUSH_EVALS,
    EV_SAMPLE_ATTEMPTS, EV_CLIP_VERTS, EV_COLOURS, EV_BB_POINTS, EV_PGS_BB_POINTS, NEV
};
enum { F_GRASP1 = 1, F_INVALID_START = 2, F_OUT_OF_WS = 4, F_OVERFLOW = 8, F_NOOP = 16 };
const int MAX_COLOURS = 32;

// ----------------------------------------------------------------------------------
// Precision-generic geometry used by the bit-exact predicates (binary32 twin) and by
// the double trajectory.  Every expression is written in the evaluation order that
// defines the predicate; C++ evaluates left to right and -ffp-contract=off keeps each
// product and sum separately rounded.
// ----------------------------------------------------------------------------------

// Rotation matrix of a unit quaternion (w,x,y,z), row-major R[3*row+col].  Column k
// is the k-th box axis in world coordinates.
template <typename T>
void quat_to_R(const T* q, T* R) {
    const T w = q[0], x = q[1], y = q[2], z = q[3];
    const T xx = x * x, yy = y * y, zz = z * z;
    const T xy = x * y, xz = x * z, yz = y * z;
    const T wx = w * x, wy = w * y, wz = w * z;
    R[0] = T(1) - T(2) * (yy + zz); R[1] = T(2) * (xy - wz);         R[2] = T(2) * (xz + wy);
    R[3] = T(2) * (xy + wz);         R[4] = T(1) - T(2) * (xx + zz); R[5] = T(2) * (yz - wx);
    R[6] = T(2) * (xz - wy);         R[7] = T(2) * (yz + wx);         R[8] = T(1) - T(2) * (xx + yy);
}

// Cylinders.  A row of half extents (r, -r, h) marks a cylinder of radius r and half
// height h about its body z axis; (hx, hy, hz) with all three positive is a box.  For
// contact, footprints and heightmaps a cylinder is the right prism over the regular
// 16-gon inscribed in its circle: vertex k of a cap at angle k pi/8 in the body xy plane,
// side face s with outward normal at angle (2s + 1) pi/16 and apothem r cos(pi/16), cap
// edges of half length r sin(pi/16).  Its mass properties are those of the solid
// cylinder.  Direction tables (cos, sin): vertex directions k = 0..7 (k + 8 is the
// negation) and side normals s = 0..7 (likewise); the values are the closed forms of the
// angles, rounded once to T.
template <typename T>
struct Gon {
    T vc[8], vs[8], fc[8], fs[8];
    T apo, half_edge;  // cos(pi/16), sin(pi/16)
    Gon() {
        const double C1 = std::cos(M_PI / 8), S1 = std::sin(M_PI / 8), H = sqrt(0.5);
        const double D1 = std::cos(M_PI / 16), E1 = std::sin(M_PI / 16);
        const double D3 = std::cos(3 * M_PI / 16), E3 = std::sin(3 * M_PI / 16);
        const double vcd[8] = {1, C1, H, S1, 0, -S1, -H, -C1}, vsd[8] = {0, S1, H, C1, 1, C1, H, S1};
        const double fcd[8] = {D1, D3, E3, E1, -E1, -E3, -D3, -D1}, fsd[8] = {E1, E3, D3, D1, D1, D3, E3, E1};
        for (int k = 0; k < 8; k++) { vc[k] = (T)vcd[k]; vs[k] = (T)vsd[k]; fc[k] = (T)fcd[k]; fs[k] = (T)fsd[k]; }
        apo = (T)D1;
        half_edge = (T)E1;
    }
};
template <typename T>
const Gon<T>& gon() {
    static const Gon<T> g;
    return g;
}
template <typename T>
inline bool is_cyl(const T* h) { return h[1] < T(0); }

// Radial support of the unit-radius 16-gon along the body-plane direction (p0, p1):
// max over the eight vertex directions of |c_k p0 + s_k p1|.
template <typename T>
T gon_support(T p0, T p1) {
    const Gon<T>& G = gon<T>();
    T m = T(0);
    for (int k = 0; k < 8; k++) {
        const T v = fabs(G.vc[k] * p0 + G.vs[k] * p1);
        if (v > m) m = v;
    }
    return m;
}

// World AABB of a box: half-width e_k = (|R_k0| h0 + |R_k1| h1) + |R_k2| h2, grown by
// the contact margin on every side.  A cylinder uses its bounding box (r, r, h).
template <typename T>
void box_aabb(const T* c, const T* R, const T* h, T m, T* lo, T* hi) {
    const T h1 = fabs(h[1]);
    for (int k = 0; k < 3; k++) {
        const T e = (fabs(R[3 * k]) * h[0] + fabs(R[3 * k + 1]) * h1) +
                    fabs(R[3 * k + 2]) * h[2];
        lo[k] = (c[k] - e) - m;
        hi[k] = (c[k] + e) + m;
    }
}

template <typename T>
struct PairList {
    std::vector<int> bb_i, bb_j;  // box-box candidates, lexicographic i<j
    std::vector<int> plane;       // boxes whose AABB reaches below z = 0
    std::vector<int> pusher;      // boxes whose AABB meets the pusher's AABB
    bool overflow = false;
};

// Broadphase at one state (closed interval overlap on all three axes).
template <typename T>
PairList<T> broadphase(int n, const T* x /*[n][3]*/, const T* q /*[n][4]*/, const T* h,
                       T margin, bool pusher_on, const T* P /*xy*/, T pr, T z0, T z1,
                       int pair_cap) {
    PairList<T> out;
    std::vector<T> lo(3 * n), hi(3 * n);
    for (int i = 0; i < n; i++) {
        T R[9];
        quat_to_R(q + 4 * i, R);
        box_aabb(x + 3 * i, R, h + 3 * i, margin, &lo[3 * i], &hi[3 * i]);
    }
    for (int i = 0; i < n; i++)
        for (int j = i + 1; j < n; j++) {
            bool ov = true;
            for (int k = 0; k < 3; k++)
                if (!(lo[3 * i + k] <= hi[3 * j + k] && lo[3 * j + k] <= hi[3 * i + k])) ov = false;
            if (!ov) continue;
            if ((int)out.bb_i.size() >= pair_cap) { out.overflow = true; continue; }
            out.bb_i.push_back(i);
            out.bb_j.push_back(j);
        }
    for (int i = 0; i < n; i++)
        if (lo[3 * i + 2] < T(0)) out.plane.push_back(i);
    if (pusher_on) {
        const T rm = pr + margin;
        const T plo[3] = {P[0] - rm, P[1] - rm, z0 - rm};
        const T phi[3] = {P[0] + rm, P[1] + rm, z1 + rm};
        for (int i = 0; i < n; i++) {
            bool ov = true;
            for (int k = 0; k < 3; k++)
                if (!(lo[3 * i + k] <= phi[k] && plo[k] <= hi[3 * i + k])) ov = false;
            if (ov) out.pusher.push_back(i);
        }
    }
    return out;
}

// Top-down footprint of a box: centre, unit axes u (the horizontal part of the box's
// x axis, or of its y axis when x is vertical) and v = perp(u), and the support
// half-widths of the 3-D box along u and v.  Exact for upright boxes, conservative
// otherwise.  A cylinder's support along u is r times the 16-gon's radial support of
// (u.x_b, u.y_b) plus h |u.z_b| (x_b, y_b, z_b its body axes): the footprint is the
// rectangle bounding the prism's projection along u and v.
template <typename T>
struct Foot { T cx, cy, ux, uy, vx, vy, su, sv; };

template <typename T>
Foot<T> footprint(const T* x, const T* q, const T* h) {
    T R[9];
    quat_to_R(q, R);
    T ex = R[0], ey = R[3];
    T l2 = ex * ex + ey * ey;
    if (l2 < T(1e-12)) { ex = R[1]; ey = R[4]; l2 = ex * ex + ey * ey; }
    const T len = sqrt(l2);
    Foot<T> f;
    f.cx = x[0]; f.cy = x[1];
    f.ux = ex / len; f.uy = ey / len;
    f.vx = -f.uy; f.vy = f.ux;
    if (is_cyl(h)) {
        f.su = gon_support(R[0] * f.ux + R[3] * f.uy, R[1] * f.ux + R[4] * f.uy) * h[0] +
               fabs(R[2] * f.ux + R[5] * f.uy) * h[2];
        f.sv = gon_support(R[0] * f.vx + R[3] * f.vy, R[1] * f.vx + R[4] * f.vy) * h[0] +
               fabs(R[2] * f.vx + R[5] * f.vy) * h[2];
        return f;
    }
    f.su = (fabs(R[0] * f.ux + R[3] * f.uy) * h[0] + fabs(R[1] * f.ux + R[4] * f.uy) * h[1]) +
           fabs(R[2] * f.ux + R[5] * f.uy) * h[2];
    f.sv = (fabs(R[0] * f.vx + R[3] * f.vy) * h[0] + fabs(R[1] * f.vx + R[4] * f.vy) * h[1]) +
           fabs(R[2] * f.vx + R[5] * f.vy) * h[2];
    return f;
}

// Finger rectangle (centre fc, axes a and b, half sizes hl along a and hw along b)
// against a footprint: 2-D separating-axis test over a, b, u_o, v_o.  Projections that
// only touch do not overlap.
template <typename T>
bool finger_overlaps(const Foot<T>& o, T fcx, T fcy, T ax, T ay, T bx, T by, T hl, T hw) {
    const T dx = o.cx - fcx, dy = o.cy - fcy;
    T rO = fabs(o.ux * ax + o.uy * ay) * o.su + fabs(o.vx * ax + o.vy * ay) * o.sv;
    if (fabs(dx * ax + dy * ay) >= hl + rO) return false;
    rO = fabs(o.ux * bx + o.uy * by) * o.su + fabs(o.vx * bx + o.vy * by) * o.sv;
    if (fabs(dx * bx + dy * by) >= hw + rO) return false;
    T rF = fabs(ax * o.ux + ay * o.uy) * hl + fabs(bx * o.ux + by * o.uy) * hw;
    if (fabs(dx * o.ux + dy * o.uy) >= rF + o.su) return false;
    rF = fabs(ax * o.vx + ay * o.vy) * hl + fabs(bx * o.vx + by * o.vy) * hw;
    if (fabs(dx * o.vx + dy * o.vy) >= rF + o.sv) return false;
    return true;
}

// Grasp-clearance test standing in for the learned grasp classifier (Sec. IV-B): a
// parallel-jaw grasp (Sec. III-A, a^g with a fixed opening) centred on the target at
// one of K yaw angles succeeds when (i) the target's width along the closing axis plus
// clearance fits the opening and (ii) neither finger's sweep region overlaps another
// box's footprint.
template <typename T>
bool graspable(int n, const T* x, const T* q, const T* h, int t, const T* ca, const T* sa,
               int K, T W, T c, T f, T fw) {
    std::vector<Foot<T>> F(n);
    for (int i = 0; i < n; i++) F[i] = footprint(x + 3 * i, q + 4 * i, h + 3 * i);
    const Foot<T>& ft = F[t];
    const T halfW = W * T(0.5), hfw = fw * T(0.5);
    for (int k = 0; k < K; k++) {
        const T ax = ca[k], ay = sa[k];
        const T bx = -ay, by = ax;
        const T wa = fabs(ft.ux * ax + ft.uy * ay) * ft.su + fabs(ft.vx * ax + ft.vy * ay) * ft.sv;
        if (!((wa + c) * T(2) <= W)) continue;
        const T off = ((wa + halfW) + f) * T(0.5);
        const T hl = ((halfW + f) - wa) * T(0.5);
        bool clear = true;
        for (int s = 1; s >= -1 && clear; s -= 2) {
            const T fcx = ft.cx + T(s) * (ax * off);
            const T fcy = ft.cy + T(s) * (ay * off);
            for (int o = 0; o < n; o++) {
                if (o == t) continue;
                if (finger_overlaps(F[o], fcx, fcy, ax, ay, bx, by, hl, hfw)) { clear = false; break; }
            }
        }
        if (clear) return true;
    }
    return false;
}

// Start-pose collision check of a push (Sec. IV-B: only the start pose is checked at
// run time): the pusher disc of radius r at (px,py) must keep out of every footprint.
template <typename T>
bool start_blocked(const std::vector<Foot<T>>& F, T px, T py, T r) {
    for (const Foot<T>& o : F) {
        const T ex = px - o.cx, ey = py - o.cy;
        T pu = fabs(ex * o.ux + ey * o.uy) - o.su;
        T pv = fabs(ex * o.vx + ey * o.vy) - o.sv;
        pu = pu > T(0) ? pu : T(0);
        pv = pv > T(0) ? pv : T(0);
        if (pu * pu + pv * pv < r * r) return true;
    }
    return false;
}

// SplitMix64: state += golden gamma, then the variant-13 finaliser.
uint64_t splitmix64_next(uint64_t& s) {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Unbiased multiply-shift draw of an index in [0, count) from the top 32 bits.
int draw_index(uint64_t r, int count) { return (int)(((r >> 32) * (uint64_t)count) >> 32); }

// Contour push sampler (Sec. IV-B and its figure of sampled pushes): for attempt a of push
// k the keyed SplitMix64 stream picks object j and contour point p of N_a points spaced
// evenly by arc length around j's footprint grown by (pusher radius + clearance); the
// push runs from p inward to j's centre for length L.  Returns the
// accepted attempt, or -1 for a no-op push when every attempt's start is blocked.
template <typename T>
int sample_push(int n, const T* x, const T* q, const T* h, uint64_t seed, int k, T r, T clear,
                T L, int attempts, int npts, T* out) {
    std::vector<Foot<T>> F(n);
    for (int i = 0; i < n; i++) F[i] = footprint(x + 3 * i, q + 4 * i, h + 3 * i);
    for (int a = 0; a < attempts; a++) {
        uint64_t st = seed ^ (((uint64_t)(uint32_t)k << 32) | (uint64_t)(uint32_t)a);
        const uint64_t r1 = splitmix64_next(st);
        const uint64_t r2 = splitmix64_next(st);
        const int j = draw_index(r1, n);
        const int p = draw_index(r2, npts);
        const Foot<T>& fj = F[j];
        const T A = (fj.su + r) + clear, B = (fj.sv + r) + clear;
        const T A2 = A * T(2), B2 = B * T(2);
        const T per = (A + B) * T(4);
        T ell = (per * T(p)) / T(npts);
        T lu, lv;
        // walk counter-clockwise from (+A, 0): edge +u, top, edge -u, bottom, back
        if (ell < B) { lu = A; lv = ell; }
        else {
            ell = ell - B;
            if (ell < A2) { lu = A - ell; lv = B; }
            else {
                ell = ell - A2;
                if (ell < B2) { lu = -A; lv = B - ell; }
                else {
                    ell = ell - B2;
                    if (ell < A2) { lu = ell - A; lv = -B; }
                    else { ell = ell - A2; lu = A; lv = ell - B; }
                }
            }
        }
        const T px = (fj.cx + lu * fj.ux) + lv * fj.vx;
        const T py = (fj.cy + lu * fj.uy) + lv * fj.vy;
        const T dx = fj.cx - px, dy = fj.cy - py;
        const T len = sqrt(dx * dx + dy * dy);
        const T dirx = dx / len, diry = dy / len;
        if (start_blocked(F, px, py, r)) continue;
        out[0] = px; out[1] = py;
        out[2] = px + dirx * L; out[3] = py + diry * L;
        return a;
    }
    return -1;
}

// Top-down heightmap of a state (Sec. V-A: the 0.288 m x 0.288 m workspace seen from
// above by an orthographic camera as a 144 x 144 grid; that depth image is what the grasp
// classifier of Sec. IV-B reads).  Cell (i, j) (column i along x, row j along y) takes
// the height of the highest box surface above its centre x_i = x0 + (i + 1/2) cell,
// y_j = y0 + (j + 1/2) cell, or 0 where the table shows.  For a box with centre c,
// rotation R and half extents h, the vertical line through (x, y) written in the box
// frame is a + b s (s = z - c_z) with a_k = R_0k (x - c_x) + R_1k (y - c_y) and
// b_k = R_2k; it is inside the box while |a_k + b_k s| <= h_k for every k, i.e. for s
// in the intersection of [-(a_k r_k) - h_k r_k, -(a_k r_k) + h_k r_k] with r_k = 1 / b_k
// (r_k and h_k r_k rounded once per box; ends swapped when b_k < 0; when b_k = 0 the
// constraint holds for every s if |a_k| <= h_k and for none otherwise).  A non-empty
// intersection [s_lo, s_hi] puts the box's top over the cell at c_z + s_hi.  A cylinder
// is the intersection of nine such slabs (its cap axis and the 16-gon's eight side
// normal directions).  Every
// operation is written in its evaluation order (binary32 twin); fma() is one fused
// multiply-add with a single rounding: a_k = fma(R_0k, x - c_x, R_1k (y - c_y)) and the
// slab ends fma(-a_k, r_k, -+h_k r_k).
template <typename T>
void heightmap(int n, const T* x, const T* q, const T* h, int W, int H, T x0, T y0, T cell, T* out) {
    // Per body its slabs: world normal (wx, wy, wz), half thickness, r = 1/wz and
    // half * r.  A box has its three axes; a cylinder its cap axis and the eight side
    // normal directions of its 16-gon (wx = c_s R_00 + s_s R_01 and so on, half
    // thickness r cos(pi/16) rounded once).
    const Gon<T>& G = gon<T>();
    std::vector<int> first(n + 1, 0);
    std::vector<T> sw;  // 6 per slab
    for (int b = 0; b < n; b++) {
        T R[9];
        quat_to_R(q + 4 * b, R);
        const T* hb = h + 3 * b;
        auto add = [&](T wx, T wy, T wz, T half) {
            const T rb = wz == T(0) ? T(0) : T(1) / wz;
            sw.insert(sw.end(), {wx, wy, wz, half, rb, half * rb});
        };
        if (is_cyl(hb)) {
            add(R[2], R[5], R[8], hb[2]);
            const T apo = hb[0] * G.apo;
            for (int k = 0; k < 8; k++)
                add(G.fc[k] * R[0] + G.fs[k] * R[1], G.fc[k] * R[3] + G.fs[k] * R[4], G.fc[k] * R[6] + G.fs[k] * R[7], apo);
        } else {
            for (int k = 0; k < 3; k++) add(R[k], R[3 + k], R[6 + k], hb[k]);
        }
        first[b + 1] = (int)sw.size() / 6;
    }
    for (int j = 0; j < H; j++)
        for (int i = 0; i < W; i++) {
            const T xc = x0 + ((T)i + T(0.5)) * cell;
            const T yc = y0 + ((T)j + T(0.5)) * cell;
            T top = T(0);
            for (int b = 0; b < n; b++) {
                const T dx = xc - x[3 * b], dy = yc - x[3 * b + 1];
                T s_lo = -INFINITY, s_hi = INFINITY;
                bool hit = true;
                for (int k = first[b]; k < first[b + 1] && hit; k++) {
                    const T* S = &sw[6 * k];
                    const T a = std::fma(S[0], dx, S[1] * dy);
                    const T bk = S[2];
                    if (bk == T(0)) {
                        if (!(fabs(a) <= S[3])) hit = false;
                        continue;
                    }
                    const T r = S[4];
                    T t0 = std::fma(-a, r, -S[5]), t1 = std::fma(-a, r, S[5]);
                    if (bk < T(0)) std::swap(t0, t1);
                    if (t0 > s_lo) s_lo = t0;
                    if (t1 < s_hi) s_hi = t1;
                }
                if (hit && s_lo <= s_hi) {
                    const T z = x[3 * b + 2] + s_hi;
                    if (z > top) top = z;
                }
            }
            out[(size_t)j * W + i] = top;
        }
}

// Heightmap form of the grasp test (the classifier of Sec. IV-B decides from the overhead
// depth image; here the image decides by geometry).  Jaw angles, the opening condition
// (i) and the two finger rectangles are those of the footprint test above.  A finger
// rectangle is clear when no heightmap cell whose centre lies in it beyond the target's
// side -- with p the centre relative to the rectangle centre, off - hl < s p.a <= off + hl
// is replaced by -hl < p.a' <= hl along the rectangle's outward axis a' = s a, and
// |p.b| <= hw -- is higher than the finger tips, which descend to
// z_tip = top_t - depth (top_t = c_z + the target's vertical half extent).  Cells are
// visited over the rectangle's bounding square with one cell of slack; the membership
// test decides.
template <typename T>
bool graspable_hm(const T* map, int cells, T x0, T cellw, int n, const T* x, const T* q, const T* h, int t,
                  const T* ca, const T* sa, int K, T W, T c, T f, T fw, T depth) {
    const Foot<T> ft = footprint(x + 3 * t, q + 4 * t, h + 3 * t);
    T R[9];
    quat_to_R(q + 4 * t, R);
    const T* ht = h + 3 * t;
    const T ez = is_cyl(ht) ? gon_support(R[6], R[7]) * ht[0] + fabs(R[8]) * ht[2]
                            : (fabs(R[6]) * ht[0] + fabs(R[7]) * ht[1]) + fabs(R[8]) * ht[2];
    const T z_tip = (x[3 * t + 2] + ez) - depth;
    const T halfW = W * T(0.5), hfw = fw * T(0.5);
    for (int k = 0; k < K; k++) {
        const T ax = ca[k], ay = sa[k];
        const T bx = -ay, by = ax;
        const T wa = fabs(ft.ux * ax + ft.uy * ay) * ft.su + fabs(ft.vx * ax + ft.vy * ay) * ft.sv;
        if (!((wa + c) * T(2) <= W)) continue;
        const T off = ((wa + halfW) + f) * T(0.5);
        const T hl = ((halfW + f) - wa) * T(0.5);
        bool clear = true;
        for (int s = 1; s >= -1 && clear; s -= 2) {
            const T sax = T(s) * ax, say = T(s) * ay;
            const T fcx = ft.cx + sax * off, fcy = ft.cy + say * off;
            const T rx = fabs(sax) * hl + fabs(bx) * hfw, ry = fabs(say) * hl + fabs(by) * hfw;
            const int i0 = std::max(0, (int)std::floor((fcx - rx - x0) / cellw) - 1);
            const int i1 = std::min(cells - 1, (int)std::floor((fcx + rx - x0) / cellw) + 1);
            const int j0 = std::max(0, (int)std::floor((fcy - ry - x0) / cellw) - 1);
            const int j1 = std::min(cells - 1, (int)std::floor((fcy + ry - x0) / cellw) + 1);
            for (int j = j0; j <= j1 && clear; j++)
                for (int i = i0; i <= i1; i++) {
                    const T px = (x0 + ((T)i + T(0.5)) * cellw) - fcx;
                    const T py = (x0 + ((T)j + T(0.5)) * cellw) - fcy;
                    const T pa = px * sax + py * say, pb = px * bx + py * by;
                    if (pa > -hl && pa <= hl && fabs(pb) <= hfw && map[(size_t)j * cells + i] > z_tip) {
                        clear = false;
                        break;
                    }
                }
        }
        if (clear) return true;
    }
    return false;
}


#ifdef ORACLE_COUNT_FLOPS
// Flop-counting build: every add, subtract, multiply, divide and square root of the
// double engine counts 1 into the current phase (compares, abs, min and max count 0).
thread_local uint64_t g_flops[8];
thread_local int g_phase = 0;
struct real {
    double v;
    real() = default;
    constexpr real(double x) : v(x) {}
    explicit operator double() const { return v; }
};
inline real operator+(real a, real b) { g_flops[g_phase]++; return a.v + b.v; }
inline real operator-(real a, real b) { g_flops[g_phase]++; return a.v - b.v; }
inline real operator*(real a, real b) { g_flops[g_phase]++; return a.v * b.v; }
inline real operator/(real a, real b) { g_flops[g_phase]++; return a.v / b.v; }
inline real operator-(real a) { return -a.v; }
inline real& operator+=(real& a, real b) { a = a + b; return a; }
inline real& operator-=(real& a, real b) { a = a - b; return a; }
inline real& operator*=(real& a, real b) { a = a * b; return a; }
inline real& operator/=(real& a, real b) { a = a / b; return a; }
inline bool operator<(real a, real b) { return a.v < b.v; }
inline bool operator>(real a, real b) { return a.v > b.v; }
inline bool operator<=(real a, real b) { return a.v <= b.v; }
inline bool operator>=(real a, real b) { return a.v >= b.v; }
inline bool operator==(real a, real b) { return a.v == b.v; }
inline bool operator!=(real a, real b) { return a.v != b.v; }
inline real sqrt(real a) { g_flops[g_phase]++; return std::sqrt(a.v); }
inline real fabs(real a) { return std::fabs(a.v); }
inline double as_double(real a) { return a.v; }
// phases: 0 per body (gravity, frames, AABB, integration), 1 narrowphase, 2 contact
// preparation, 3 contact solve, 4 colouring and the rest
inline void set_phase(int k) { g_phase = k; }
#else
typedef double real;
inline double as_double(double a) { return a; }
inline void set_phase(int) {}
#endif

// ----------------------------------------------------------------------------------
// Double-precision engine
// ----------------------------------------------------------------------------------
struct V3 { real x, y, z; };
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(V3 a, real s) { return {a.x * s, a.y * s, a.z * s}; }
inline V3 operator-(V3 a) { return {-a.x, -a.y, -a.z}; }
inline real dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline real norm(V3 a) { return sqrt(dot(a, a)); }

struct Body {
    V3 x, v, w;
    real q[4];
    real h[3], m, invm, mu, invIb[3];  // h = (r, r, half height) for a cylinder
    bool cyl;
    real R[9], invIw[6];   // refreshed every substep
};
inline V3 axis(const Body& b, int k) { return {b.R[k], b.R[3 + k], b.R[6 + k]}; }
inline V3 rot(const real* R, V3 l) {
    return {R[0] * l.x + R[1] * l.y + R[2] * l.z, R[3] * l.x + R[4] * l.y + R[5] * l.z,
            R[6] * l.x + R[7] * l.y + R[8] * l.z};
}
// symmetric 3x3 stored as (00, 01, 02, 11, 12, 22)
inline V3 sym_mul(const real* I, V3 v) {
    return {I[0] * v.x + I[1] * v.y + I[2] * v.z, I[1] * v.x + I[3] * v.y + I[4] * v.z,
            I[2] * v.x + I[4] * v.y + I[5] * v.z};
}

struct Contact {
    V3 p, rA, rB;
    real d;
    real invKn, invKt1, invKt2, bias;
    real ln, lt1, lt2;
};
struct Manifold {
    int A, B;  // A < B for box pairs; PLANE as A; PUSHER as B
    V3 n, t1, t2;
    real mu;
    int np;
    Contact c[4];
    int colour;
};

struct PushState {
    bool active = false;
    real sx = 0, sy = 0, dx = 0, dy = 0;
    int moving = 0;
};

// A contact point carried to the next substep (warm start): its offset in the frame of
// the manifold's key body (A when dynamic, else B), its normal impulse and its friction
// impulse as a world vector (the tangent basis is rebuilt every substep).
struct WarmPoint { V3 loc; real ln; V3 Pt; };
struct WarmManifold { int A, B, np; WarmPoint p[4]; };

struct Env {
    std::vector<Body> b;
    std::vector<WarmManifold> warm;  // last substep's manifolds (warm start only)
    int target = 0;
    PushState push;
    V3 P{0, 0, 0}, V{0, 0, 0};  // pusher position (segment base xy) and velocity
    bool overflow = false;
    uint64_t ev[NEV] = {0};
};

void load_env(Env& E, int n, const real* s13, const float* half, const float* mass, const float* mu) {
    E.b.resize(n);
    for (int i = 0; i < n; i++) {
        Body& b = E.b[i];
        const real* s = s13 + 13 * i;
        b.x = {s[0], s[1], s[2]};
        for (int k = 0; k < 4; k++) b.q[k] = s[3 + k];
        b.v = {s[7], s[8], s[9]};
        b.w = {s[10], s[11], s[12]};
        b.cyl = half[3 * i + 1] < 0.f;
        for (int k = 0; k < 3; k++) b.h[k] = fabs((real)half[3 * i + k]);
        b.m = mass[i];
        b.invm = 1.0 / b.m;
        b.mu = mu[i];
        const real hx2 = b.h[0] * b.h[0], hy2 = b.h[1] * b.h[1], hz2 = b.h[2] * b.h[2];
        if (b.cyl) {
            // solid cylinder of radius r and height 2h: m (3 r^2 + 4 h^2) / 12 about the
            // two diameters, m r^2 / 2 about its axis
            b.invIb[0] = b.invIb[1] = 1.0 / (b.m * (3.0 * hx2 + 4.0 * hz2) / 12.0);
            b.invIb[2] = 1.0 / (b.m * hx2 / 2.0);
        } else {
            // solid box inertia about its centre, from half extents: m/3 (h_j^2 + h_k^2)
            b.invIb[0] = 1.0 / (b.m / 3.0 * (hy2 + hz2));
            b.invIb[1] = 1.0 / (b.m / 3.0 * (hx2 + hz2));
            b.invIb[2] = 1.0 / (b.m / 3.0 * (hx2 + hy2));
        }
    }
}

void store_env(const Env& E, real* s13) {
    for (size_t i = 0; i < E.b.size(); i++) {
        const Body& b = E.b[i];
        real* s = s13 + 13 * i;
        s[0] = b.x.x; s[1] = b.x.y; s[2] = b.x.z;
        for (int k = 0; k < 4; k++) s[3 + k] = b.q[k];
        s[7] = b.v.x; s[8] = b.v.y; s[9] = b.v.z;
        s[10] = b.w.x; s[11] = b.w.y; s[12] = b.w.z;
    }
}

// Pusher kinematics: the tip moves from the start along the unit direction at speed
// v_p for `moving` substeps (the push length over v_p dt, rounded), then rests.
void set_push(Env& E, const oracle_params& P, const real* push) {
    PushState& ps = E.push;
    const real dx = push[2] - push[0], dy = push[3] - push[1];
    const real L = sqrt(dx * dx + dy * dy);
    if (!(L > 1e-9)) { ps.active = false; return; }
    ps.active = true;
    ps.sx = push[0]; ps.sy = push[1];
    ps.dx = dx / L; ps.dy = dy / L;
    const real step = P.pusher_speed * P.dt;
    long mv = std::lround(as_double(L / step));
    if (mv > P.substeps_per_push) mv = P.substeps_per_push;
    if (mv < 0) mv = 0;
    ps.moving = (int)mv;
}

void pusher_at(Env& E, const oracle_params& P, int s) {
    const PushState& ps = E.push;
    const int done = s < ps.moving ? s : ps.moving;
    const real travel = (P.pusher_speed * P.dt) * (real)done;
    E.P = {ps.sx + ps.dx * travel, ps.sy + ps.dy * travel, 0.0};
    if (s < ps.moving) E.V = {ps.dx * P.pusher_speed, ps.dy * P.pusher_speed, 0.0};
    else E.V = {0, 0, 0};
}

// ---- narrowphase -------------------------------------------------------------------

// Box against the table plane: the box vertices lower than the margin, deepest first
// (ties by vertex index), at most four.  Normal +z from the plane (A) to the box (B).
bool box_plane(const Body& b, int bi, const oracle_params& P, Manifold& M) {
    struct Cand { real d; int v; V3 r; };
    Cand c[8];
    int nc = 0;
    for (int v = 0; v < 8; v++) {
        const V3 l = {(v & 1 ? 1.0 : -1.0) * b.h[0], (v & 2 ? 1.0 : -1.0) * b.h[1], (v & 4 ? 1.0 : -1.0) * b.h[2]};
        const V3 r = rot(b.R, l);
        const real d = b.x.z + r.z;
        if (d < P.margin) c[nc++] = {d, v, r};
    }
    if (nc == 0) return false;
    std::sort(c, c + nc, [](const Cand& a, const Cand& b2) { return a.d < b2.d || (a.d == b2.d && a.v < b2.v); });
    M.A = PLANE; M.B = bi;
    M.n = {0, 0, 1};
    M.np = nc < 4 ? nc : 4;
    for (int k = 0; k < M.np; k++) {
        Contact& C = M.c[k];
        C.rB = c[k].r;
        C.p = b.x + c[k].r;
        C.rA = {0, 0, 0};
        C.d = c[k].d;
    }
    return true;
}

// Sutherland-Hodgman clip of a polygon against the half space dot(p - o, a) - h <= 0.
// At most `cap` vertices are kept (eight, the bound for a convex quad clipped four
// times; 32 for faces of cylinders).
std::vector<V3> clip_side(const std::vector<V3>& poly, V3 o, V3 a, real h, size_t cap = 8) {
    std::vector<V3> out;
    const size_t N = poly.size();
    auto add = [&](V3 p) { if (out.size() < cap) out.push_back(p); };
    for (size_t i = 0; i < N; i++) {
        const V3 cur = poly[i], prev = poly[(i + N - 1) % N];
        const real dc = dot(cur - o, a) - h, dp = dot(prev - o, a) - h;
        if (dc <= 0) {
            if (dp > 0) add(prev + (cur - prev) * (dp / (dp - dc)));
            add(cur);
        } else if (dp <= 0) {
            add(prev + (cur - prev) * (dp / (dp - dc)));
        }
    }
    return out;
}

// At most four of the candidate points kp (separations kd) with face normal nref: all
// of them when there are four or fewer; else the deepest (earliest on ties); then the
// farthest from it; then the one spanning the largest triangle with those two; then the
// one adding the largest area outside an edge of that triangle.
int reduce_points(const std::vector<V3>& kp, const std::vector<real>& kd, V3 nref, V3* pts, real* dep) {
    const int nk = (int)kp.size();
    if (nk <= 4) {
        for (int i = 0; i < nk; i++) { pts[i] = kp[i]; dep[i] = kd[i]; }
        return nk;
    }
    std::vector<bool> used(nk, false);
    int sel[4];
    int i1 = 0;
    for (int i = 1; i < nk; i++) if (kd[i] < kd[i1]) i1 = i;
    used[i1] = true;
    int i2 = -1; real b2 = -1;
    for (int i = 0; i < nk; i++) {
        if (used[i]) continue;
        const V3 e = kp[i] - kp[i1];
        const real l = dot(e, e);
        if (i2 < 0 || l > b2) { b2 = l; i2 = i; }
    }
    used[i2] = true;
    auto area = [&](int a, int b, V3 p) { return dot(cross(kp[b] - kp[a], p - kp[a]), nref); };
    int i3 = -1; real b3 = -1;
    for (int i = 0; i < nk; i++) {
        if (used[i]) continue;
        const real A = fabs(area(i1, i2, kp[i]));
        if (i3 < 0 || A > b3) { b3 = A; i3 = i; }
    }
    used[i3] = true;
    const real sgn = area(i1, i2, kp[i3]) < 0 ? -1.0 : 1.0;
    int i4 = -1; real b4 = 0;
    for (int i = 0; i < nk; i++) {
        if (used[i]) continue;
        real A = -sgn * area(i1, i2, kp[i]);
        A = std::max(A, -sgn * area(i2, i3, kp[i]));
        A = std::max(A, -sgn * area(i3, i1, kp[i]));
        if (i4 < 0 || A > b4) { b4 = A; i4 = i; }
    }
    sel[0] = i1; sel[1] = i2; sel[2] = i3; sel[3] = i4;
    for (int i = 0; i < 4; i++) { pts[i] = kp[sel[i]]; dep[i] = kd[sel[i]]; }
    return 4;
}

// Face contact: clip the incident face of box `inc` against the side planes of the
// reference face (outward normal nref, axis index k of box `ref`), keep points within
// the margin of the reference face, reduce to at most four.
int face_contact(const Body& ref, int k, V3 nref, const Body& inc, const oracle_params& P,
                 V3* pts, real* dep, uint64_t* ev) {
    const V3 fc = ref.x + nref * ref.h[k];
    const int k1 = (k == 0) ? 1 : 0, k2 = (k == 2) ? 1 : 2;
    const V3 u = axis(ref, k1), v = axis(ref, k2);
    const real hu = ref.h[k1], hv = ref.h[k2];
    // incident face: the face of `inc` whose outward normal is most anti-parallel to nref
    int best_f = 0;
    real best = 0;
    for (int m = 0; m < 3; m++) {
        const real dm = dot(axis(inc, m), nref);
        if (m == 0 || dm < best) { best = dm; best_f = 2 * m; }
        if (-dm < best) { best = -dm; best_f = 2 * m + 1; }
    }
    const int mi = best_f / 2;
    const real si = (best_f % 2 == 0) ? 1.0 : -1.0;
    const int m1 = (mi == 0) ? 1 : 0, m2 = (mi == 2) ? 1 : 2;
    const V3 fi = inc.x + axis(inc, mi) * (si * inc.h[mi]);
    const V3 e1 = axis(inc, m1) * inc.h[m1], e2 = axis(inc, m2) * inc.h[m2];
    std::vector<V3> poly = {fi + e1 + e2, fi - e1 + e2, fi - e1 - e2, fi + e1 - e2};
    poly = clip_side(poly, fc, u, hu);
    poly = clip_side(poly, fc, -u, hu);
    poly = clip_side(poly, fc, v, hv);
    poly = clip_side(poly, fc, -v, hv);
    ev[EV_CLIP_VERTS] += poly.size();
    std::vector<V3> kp;
    std::vector<real> kd;
    for (const V3& p : poly) {
        const real d = dot(p - fc, nref);
        if (d < P.margin) { kp.push_back(p); kd.push_back(d); }
    }
    return reduce_points(kp, kd, nref, pts, dep);
}

struct SatResult {
    bool touching;
    int axis;      // 0..2 faces of A, 3..5 faces of B, 6..14 edge a*3+b
    real sep;
    V3 n;          // from A to B
};

// Separating-axis test of two boxes over the 15 candidate axes.  Any separation of at
// least the margin means no contact.  Face of B replaces the best face of A only when
// deeper-separated by more than 1e-5 m; an edge axis replaces the chosen face only when
// its separation exceeds the face's by 1e-4 m + 5% of |face separation|.  Earliest axis
// wins exact ties.
SatResult sat(const Body& A, const Body& B, real margin) {
    SatResult r{false, -1, 0, {0, 0, 0}};
    const V3 D = B.x - A.x;
    real C[3][3], aC[3][3];
    for (int k = 0; k < 3; k++)
        for (int m = 0; m < 3; m++) { C[k][m] = dot(axis(A, k), axis(B, m)); aC[k][m] = fabs(C[k][m]); }
    int fa = -1; real sa = 0;
    for (int k = 0; k < 3; k++) {
        const real s = fabs(dot(D, axis(A, k))) - (A.h[k] + (B.h[0] * aC[k][0] + B.h[1] * aC[k][1] + B.h[2] * aC[k][2]));
        if (s >= margin) return r;
        if (fa < 0 || s > sa) { fa = k; sa = s; }
    }
    int fb = -1; real sb = 0;
    for (int m = 0; m < 3; m++) {
        const real s = fabs(dot(D, axis(B, m))) - ((A.h[0] * aC[0][m] + A.h[1] * aC[1][m] + A.h[2] * aC[2][m]) + B.h[m]);
        if (s >= margin) return r;
        if (fb < 0 || s > sb) { fb = m; sb = s; }
    }
    int fe = -1; real se = 0; V3 le{0, 0, 0};
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            const V3 L = cross(axis(A, a), axis(B, b));
            const real l2 = dot(L, L);
            if (l2 < 1e-12) continue;
            const real len = sqrt(l2);
            const real rA = (A.h[0] * fabs(dot(axis(A, 0), L)) + A.h[1] * fabs(dot(axis(A, 1), L))) + A.h[2] * fabs(dot(axis(A, 2), L));
            const real rB = (B.h[0] * fabs(dot(axis(B, 0), L)) + B.h[1] * fabs(dot(axis(B, 1), L))) + B.h[2] * fabs(dot(axis(B, 2), L));
            const real s = (fabs(dot(D, L)) - (rA + rB)) / len;
            if (s >= margin) return r;
            if (fe < 0 || s > se) { fe = 6 + 3 * a + b; se = s; le = L * (1.0 / len); }
        }
    int ax = fa; real s = sa; V3 L = axis(A, fa);
    if (sb > sa + 1e-5) { ax = 3 + fb; s = sb; L = axis(B, fb); }
    if (fe >= 0 && se > s + 1e-4 + 0.05 * fabs(s)) { ax = fe; s = se; L = le; }
    if (dot(L, D) < 0) L = -L;
    r.touching = true; r.axis = ax; r.sep = s; r.n = L;
    return r;
}

// Box-box manifold: face contact by clipping, or one edge-edge point midway between
// the closest points of the two supporting edges.
bool box_box(const Body& A, int ia, const Body& B, int ib, const oracle_params& P, Manifold& M, uint64_t* ev) {
    ev[EV_SAT]++;
    const SatResult s = sat(A, B, P.margin);
    if (!s.touching) return false;
    V3 pts[4];
    real dep[4];
    int np = 0;
    if (s.axis < 3) {
        ev[EV_FACE]++;
        np = face_contact(A, s.axis, s.n, B, P, pts, dep, ev);
    } else if (s.axis < 6) {
        ev[EV_FACE]++;
        np = face_contact(B, s.axis - 3, -s.n, A, P, pts, dep, ev);
    } else {
        ev[EV_EDGE]++;
        const int a = (s.axis - 6) / 3, b = (s.axis - 6) % 3;
        V3 pA = A.x, pB = B.x;
        for (int k = 0; k < 3; k++) {
            if (k == a) continue;
            const real sg = dot(axis(A, k), s.n) < 0 ? -1.0 : 1.0;
            pA = pA + axis(A, k) * (sg * A.h[k]);
        }
        for (int m = 0; m < 3; m++) {
            if (m == b) continue;
            const real sg = dot(axis(B, m), s.n) > 0 ? -1.0 : 1.0;
            pB = pB + axis(B, m) * (sg * B.h[m]);
        }
        const V3 dA = axis(A, a), dB = axis(B, b);
        const V3 r = pA - pB;
        const real bb = dot(dA, dB), c = dot(dA, r), f = dot(dB, r);
        const real den = 1.0 - bb * bb;
        real sa = 0, tb;
        if (den > 1e-12) { sa = (bb * f - c) / den; tb = f + sa * bb; }
        else tb = f;
        sa = std::min(std::max(sa, -A.h[a]), A.h[a]);
        tb = std::min(std::max(tb, -B.h[b]), B.h[b]);
        const V3 qa = pA + dA * sa, qb = pB + dB * tb;
        pts[0] = (qa + qb) * 0.5;
        dep[0] = s.sep;
        np = 1;
    }
    if (np == 0) return false;
    M.A = ia; M.B = ib;
    M.n = s.n;
    M.np = np;
    for (int k = 0; k < np; k++) {
        M.c[k].p = pts[k];
        M.c[k].d = dep[k];
        M.c[k].rA = pts[k] - A.x;
        M.c[k].rB = pts[k] - B.x;
    }
    return true;
}

// Capsule pusher against a box.  The capsule's segment is clipped to the box's vertical
// extent; each end of the clipped range (or its middle when shorter than 1 mm, or the
// nearer segment end when the ranges do not meet) gives one candidate point: the box
// point closest to it.  Candidates closer than radius + margin become contacts; the
// normal (box to pusher) is that of the nearest candidate.
bool capsule_box(const Body& b, int bi, V3 Pp, const oracle_params& P, Manifold& M) {
    const real ez = (fabs(b.R[6]) * b.h[0] + fabs(b.R[7]) * b.h[1]) + fabs(b.R[8]) * b.h[2];
    const real zlo = b.x.z - ez, zhi = b.x.z + ez;
    const real za = std::max<real>(P.pusher_z0, zlo), zb = std::min<real>(P.pusher_z1, zhi);
    real zc[2];
    int nc;
    if (za > zb) { zc[0] = (zhi < P.pusher_z0) ? P.pusher_z0 : P.pusher_z1; nc = 1; }
    else if (zb - za < 1e-3) { zc[0] = (za + zb) * 0.5; nc = 1; }
    else { zc[0] = za; zc[1] = zb; nc = 2; }
    int np = 0;
    real best_d = 0;
    V3 best_n{1, 0, 0};
    for (int i = 0; i < nc; i++) {
        const V3 S = {Pp.x, Pp.y, zc[i]};
        const V3 rel = S - b.x;
        real loc[3], ql[3];
        for (int k = 0; k < 3; k++) {
            loc[k] = dot(axis(b, k), rel);
            ql[k] = std::min(std::max(loc[k], -b.h[k]), b.h[k]);
        }
        const V3 Q = b.x + axis(b, 0) * ql[0] + axis(b, 1) * ql[1] + axis(b, 2) * ql[2];
        const V3 diff = S - Q;
        const real dist = norm(diff);
        V3 nrm;
        real d;
        if (dist > 1e-6) {
            nrm = diff * (1.0 / dist);
            d = dist - P.pusher_radius;
        } else {
            real pen = b.h[0] - fabs(loc[0]);
            for (int k = 1; k < 3; k++) pen = std::min(pen, b.h[k] - fabs(loc[k]));
            d = -pen - P.pusher_radius;
            const V3 w = {S.x - b.x.x, S.y - b.x.y, 0};
            const real lw = norm(w);
            nrm = lw > 1e-9 ? w * (1.0 / lw) : V3{1, 0, 0};
        }
        if (!(d < P.margin)) continue;
        Contact& C = M.c[np];
        C.p = Q;
        C.d = d;
        C.rA = Q - b.x;
        C.rB = {0, 0, 0};
        if (np == 0 || d < best_d) { best_d = d; best_n = nrm; }
        np++;
    }
    if (np == 0) return false;
    M.A = bi; M.B = PUSHER;
    M.n = best_n;
    M.np = np;
    return true;
}

// ---- cylinders (16-gon prisms) ---------------------------------------------------------
// Pairs with a cylinder use the general separating-axis test of two convex polyhedra:
// candidate axes are the face normal directions of A (box: its 3 axes; cylinder: its cap
// axis, then the 8 side normal directions), those of B, and the cross products of an edge
// direction of A with one of B (box: its 3 axes; cylinder: its axis, then the 8 cap edge
// directions), skipped when |cross|^2 < 1e-12.  Separation along a unit axis L is
// |L.(c_B - c_A)| minus the two support half widths; the selection thresholds are those of
// the box-box test.  Contact: the reference face (the selected face, facing the other
// body) clips the other body's incident face (the one whose outward normal is most
// anti-parallel), up to 32 clipped vertices, reduced to four as for boxes; an edge axis
// gives one point midway between the closest points of the two supporting edges.

const Gon<real>& G64() { return gon<real>(); }
// body-plane unit vectors: vertex direction k, side normal s and side tangent s (k, s in 0..15)
inline void gon_vdir(int k, real& c, real& sn) { const real g = k < 8 ? 1 : -1; c = g * G64().vc[k & 7]; sn = g * G64().vs[k & 7]; }
inline void gon_fdir(int s, real& c, real& sn) { const real g = s < 8 ? 1 : -1; c = g * G64().fc[s & 7]; sn = g * G64().fs[s & 7]; }
inline V3 plane_vec(const Body& b, real c, real sn) { return axis(b, 0) * c + axis(b, 1) * sn; }
inline V3 side_normal(const Body& b, int s) { real c, sn; gon_fdir(s, c, sn); return plane_vec(b, c, sn); }
inline V3 side_tangent(const Body& b, int s) { real c, sn; gon_fdir(s, c, sn); return plane_vec(b, -sn, c); }
inline V3 cyl_vertex(const Body& b, int k, real sz) {
    real c, sn;
    gon_vdir(k & 15, c, sn);
    return b.x + plane_vec(b, c * b.h[0], sn * b.h[0]) + axis(b, 2) * (sz * b.h[2]);
}
inline real cyl_apothem(const Body& b) { return b.h[0] * G64().apo; }

real support(const Body& b, V3 L) {
    if (b.cyl) return gon_support(dot(axis(b, 0), L), dot(axis(b, 1), L)) * b.h[0] + fabs(dot(axis(b, 2), L)) * b.h[2];
    return (b.h[0] * fabs(dot(axis(b, 0), L)) + b.h[1] * fabs(dot(axis(b, 1), L))) + b.h[2] * fabs(dot(axis(b, 2), L));
}
inline int n_dirs(const Body& b) { return b.cyl ? 9 : 3; }
inline V3 face_dir(const Body& b, int f) { return !b.cyl ? axis(b, f) : (f == 0 ? axis(b, 2) : side_normal(b, f - 1)); }
inline real face_half(const Body& b, int f) { return !b.cyl ? b.h[f] : (f == 0 ? b.h[2] : cyl_apothem(b)); }
inline V3 edge_dir(const Body& b, int j) { return !b.cyl ? axis(b, j) : (j == 0 ? axis(b, 2) : side_tangent(b, j - 1)); }

struct ConvexSat {
    bool touching;
    int kind;   // 0 face of A, 1 face of B, 2 edge pair
    int i, j;   // face index, or edge of A and edge of B
    real sep;
    V3 n;       // from A to B
};

ConvexSat sat_convex(const Body& A, const Body& B, real margin) {
    ConvexSat r{false, 0, -1, -1, 0, {0, 0, 0}};
    const V3 D = B.x - A.x;
    int fa = -1; real sa = 0;
    for (int f = 0; f < n_dirs(A); f++) {
        const V3 L = face_dir(A, f);
        const real s = fabs(dot(D, L)) - (face_half(A, f) + support(B, L));
        if (s >= margin) return r;
        if (fa < 0 || s > sa) { fa = f; sa = s; }
    }
    int fb = -1; real sb = 0;
    for (int f = 0; f < n_dirs(B); f++) {
        const V3 L = face_dir(B, f);
        const real s = fabs(dot(D, L)) - (support(A, L) + face_half(B, f));
        if (s >= margin) return r;
        if (fb < 0 || s > sb) { fb = f; sb = s; }
    }
    int ea = -1, eb = -1; real se = 0; V3 le{0, 0, 0};
    for (int i = 0; i < n_dirs(A); i++)
        for (int j = 0; j < n_dirs(B); j++) {
            const V3 L = cross(edge_dir(A, i), edge_dir(B, j));
            const real l2 = dot(L, L);
            if (l2 < 1e-12) continue;
            const real len = sqrt(l2);
            const V3 u = L * (1.0 / len);
            const real s = fabs(dot(D, u)) - (support(A, u) + support(B, u));
            if (s >= margin) return r;
            if (ea < 0 || s > se) { ea = i; eb = j; se = s; le = u; }
        }
    int kind = 0, i = fa, j = -1; real s = sa; V3 L = face_dir(A, fa);
    if (sb > sa + 1e-5) { kind = 1; i = fb; s = sb; L = face_dir(B, fb); }
    if (ea >= 0 && se > s + 1e-4 + 0.05 * fabs(s)) { kind = 2; i = ea; j = eb; s = se; L = le; }
    if (dot(L, D) < 0) L = -L;
    r.touching = true; r.kind = kind; r.i = i; r.j = j; r.sep = s; r.n = L;
    return r;
}

// Face contact between convex bodies: reference face f of `ref` with outward normal nref.
int face_contact_convex(const Body& ref, int f, V3 nref, const Body& inc, const oracle_params& P,
                        V3* pts, real* dep, uint64_t* ev) {
    struct Side { V3 a; real h; };
    std::vector<Side> sides;
    V3 fc;
    if (!ref.cyl) {
        fc = ref.x + nref * ref.h[f];
        const int k1 = (f == 0) ? 1 : 0, k2 = (f == 2) ? 1 : 2;
        const V3 u = axis(ref, k1), v = axis(ref, k2);
        sides = {{u, ref.h[k1]}, {-u, ref.h[k1]}, {v, ref.h[k2]}, {-v, ref.h[k2]}};
    } else if (f == 0) {
        fc = ref.x + nref * ref.h[2];
        for (int s = 0; s < 16; s++) sides.push_back({side_normal(ref, s), cyl_apothem(ref)});
    } else {
        const int s = dot(side_normal(ref, f - 1), nref) > 0 ? f - 1 : f + 7;
        fc = ref.x + nref * cyl_apothem(ref);
        const V3 ez = axis(ref, 2), t = side_tangent(ref, s);
        const real w = ref.h[0] * G64().half_edge;
        sides = {{ez, ref.h[2]}, {-ez, ref.h[2]}, {t, w}, {-t, w}};
    }
    std::vector<V3> poly;
    if (!inc.cyl) {
        int best_f = 0;
        real best = 0;
        for (int m = 0; m < 3; m++) {
            const real dm = dot(axis(inc, m), nref);
            if (m == 0 || dm < best) { best = dm; best_f = 2 * m; }
            if (-dm < best) { best = -dm; best_f = 2 * m + 1; }
        }
        const int mi = best_f / 2;
        const real si = (best_f % 2 == 0) ? 1.0 : -1.0;
        const int m1 = (mi == 0) ? 1 : 0, m2 = (mi == 2) ? 1 : 2;
        const V3 fi = inc.x + axis(inc, mi) * (si * inc.h[mi]);
        const V3 e1 = axis(inc, m1) * inc.h[m1], e2 = axis(inc, m2) * inc.h[m2];
        poly = {fi + e1 + e2, fi - e1 + e2, fi - e1 - e2, fi + e1 - e2};
    } else {
        // candidates in order: top cap, bottom cap, sides 0..15
        const real dz = dot(axis(inc, 2), nref);
        int best_c = 0;
        real best = dz;
        if (-dz < best) { best = -dz; best_c = 1; }
        for (int s = 0; s < 16; s++) {
            const real dm = dot(side_normal(inc, s), nref);
            if (dm < best) { best = dm; best_c = 2 + s; }
        }
        if (best_c < 2) {
            const real sz = best_c == 0 ? 1.0 : -1.0;
            for (int k = 0; k < 16; k++) poly.push_back(cyl_vertex(inc, k, sz));
        } else {
            const int s = best_c - 2;
            poly = {cyl_vertex(inc, s, 1.0), cyl_vertex(inc, s + 1, 1.0), cyl_vertex(inc, s + 1, -1.0),
                    cyl_vertex(inc, s, -1.0)};
        }
    }
    for (const Side& sd : sides) poly = clip_side(poly, fc, sd.a, sd.h, 32);
    ev[EV_CLIP_VERTS] += poly.size();
    std::vector<V3> kp;
    std::vector<real> kd;
    for (const V3& p : poly) {
        const real d = dot(p - fc, nref);
        if (d < P.margin) { kp.push_back(p); kd.push_back(d); }
    }
    return reduce_points(kp, kd, nref, pts, dep);
}

// Supporting edge of direction index j of body b toward L: centre, direction, half length.
void support_edge(const Body& b, int j, V3 L, V3& c, V3& d, real& hl) {
    if (!b.cyl) {
        c = b.x;
        for (int k = 0; k < 3; k++) {
            if (k == j) continue;
            const real sg = dot(axis(b, k), L) < 0 ? -1.0 : 1.0;
            c = c + axis(b, k) * (sg * b.h[k]);
        }
        d = axis(b, j);
        hl = b.h[j];
    } else if (j == 0) {
        int kb = 0;
        real best = 0;
        for (int k = 0; k < 16; k++) {
            real vc, vs;
            gon_vdir(k, vc, vs);
            const real v = dot(plane_vec(b, vc, vs), L);
            if (k == 0 || v > best) { best = v; kb = k; }
        }
        c = cyl_vertex(b, kb, 0.0);
        d = axis(b, 2);
        hl = b.h[2];
    } else {
        const int s = dot(side_normal(b, j - 1), L) >= 0 ? j - 1 : j + 7;
        const real sz = dot(axis(b, 2), L) >= 0 ? 1.0 : -1.0;
        c = b.x + side_normal(b, s) * cyl_apothem(b) + axis(b, 2) * (sz * b.h[2]);
        d = side_tangent(b, s);
        hl = b.h[0] * G64().half_edge;
    }
}

bool convex_pair(const Body& A, int ia, const Body& B, int ib, const oracle_params& P, Manifold& M, uint64_t* ev) {
    ev[EV_SAT]++;
    const ConvexSat s = sat_convex(A, B, P.margin);
    if (!s.touching) return false;
    V3 pts[4];
    real dep[4];
    int np = 0;
    if (s.kind == 0) {
        ev[EV_FACE]++;
        np = face_contact_convex(A, s.i, s.n, B, P, pts, dep, ev);
    } else if (s.kind == 1) {
        ev[EV_FACE]++;
        np = face_contact_convex(B, s.i, -s.n, A, P, pts, dep, ev);
    } else {
        ev[EV_EDGE]++;
        V3 pA, pB, dA, dB;
        real ha, hb;
        support_edge(A, s.i, s.n, pA, dA, ha);
        support_edge(B, s.j, -s.n, pB, dB, hb);
        const V3 r = pA - pB;
        const real bb = dot(dA, dB), c = dot(dA, r), f = dot(dB, r);
        const real den = 1.0 - bb * bb;
        real sa = 0, tb;
        if (den > 1e-12) { sa = (bb * f - c) / den; tb = f + sa * bb; }
        else tb = f;
        sa = std::min(std::max(sa, -ha), ha);
        tb = std::min(std::max(tb, -hb), hb);
        const V3 qa = pA + dA * sa, qb = pB + dB * tb;
        pts[0] = (qa + qb) * 0.5;
        dep[0] = s.sep;
        np = 1;
    }
    if (np == 0) return false;
    M.A = ia; M.B = ib;
    M.n = s.n;
    M.np = np;
    for (int k = 0; k < np; k++) {
        M.c[k].p = pts[k];
        M.c[k].d = dep[k];
        M.c[k].rA = pts[k] - A.x;
        M.c[k].rB = pts[k] - B.x;
    }
    return true;
}

// Cylinder against the table plane: its 32 vertices (bottom cap k = 0..15, then top cap)
// lower than the margin; four or fewer are kept deepest first (ties by vertex index),
// more are reduced to four as for face contacts.  Normal +z.
bool cyl_plane(const Body& b, int bi, const oracle_params& P, Manifold& M) {
    std::vector<V3> kp;
    std::vector<real> kd;
    std::vector<int> kv;
    for (int v = 0; v < 32; v++) {
        const V3 r = cyl_vertex(b, v & 15, v < 16 ? -1.0 : 1.0) - b.x;
        const real d = b.x.z + r.z;
        if (d < P.margin) { kp.push_back(r); kd.push_back(d); kv.push_back(v); }
    }
    const int nc = (int)kp.size();
    if (nc == 0) return false;
    V3 pts[4];
    real dep[4];
    int np;
    if (nc <= 4) {
        std::vector<int> o(nc);
        for (int i = 0; i < nc; i++) o[i] = i;
        std::sort(o.begin(), o.end(), [&](int a, int c) { return kd[a] < kd[c] || (kd[a] == kd[c] && kv[a] < kv[c]); });
        for (int i = 0; i < nc; i++) { pts[i] = kp[o[i]]; dep[i] = kd[o[i]]; }
        np = nc;
    } else {
        np = reduce_points(kp, kd, {0, 0, 1}, pts, dep);
    }
    M.A = PLANE; M.B = bi;
    M.n = {0, 0, 1};
    M.np = np;
    for (int k = 0; k < np; k++) {
        Contact& C = M.c[k];
        C.rB = pts[k];
        C.p = b.x + pts[k];
        C.rA = {0, 0, 0};
        C.d = dep[k];
    }
    return true;
}

// Capsule pusher against a cylinder: as against a box, with the cylinder's vertical
// extent h |R_22| + r (16-gon support of (R_20, R_21)) and its closest point to a
// segment point S -- the prism is the 16-gon times [-h, h] in its frame, so the closest
// point is the 16-gon's closest point to S's body-plane coordinates (S's own when
// inside; else the nearest point of the nearest edge, earliest edge on ties) with the
// axial coordinate clamped.  Inside the prism the depth is the smallest distance to a
// face.
bool capsule_cyl(const Body& b, int bi, V3 Pp, const oracle_params& P, Manifold& M) {
    const real ez = gon_support(b.R[6], b.R[7]) * b.h[0] + fabs(b.R[8]) * b.h[2];
    const real zlo = b.x.z - ez, zhi = b.x.z + ez;
    const real za = std::max<real>(P.pusher_z0, zlo), zb = std::min<real>(P.pusher_z1, zhi);
    real zc[2];
    int nc;
    if (za > zb) { zc[0] = (zhi < P.pusher_z0) ? P.pusher_z0 : P.pusher_z1; nc = 1; }
    else if (zb - za < 1e-3) { zc[0] = (za + zb) * 0.5; nc = 1; }
    else { zc[0] = za; zc[1] = zb; nc = 2; }
    const real r = b.h[0], apo = cyl_apothem(b);
    int np = 0;
    real best_d = 0;
    V3 best_n{1, 0, 0};
    for (int i = 0; i < nc; i++) {
        const V3 S = {Pp.x, Pp.y, zc[i]};
        const V3 rel = S - b.x;
        const real lx = dot(axis(b, 0), rel), ly = dot(axis(b, 1), rel), lz = dot(axis(b, 2), rel);
        bool inside = true;
        real pen_side = 1e300;
        for (int s = 0; s < 16; s++) {
            real fcs, fss;
            gon_fdir(s, fcs, fss);
            const real g = apo - (fcs * lx + fss * ly);
            if (g < 0) inside = false;
            pen_side = std::min(pen_side, g);
        }
        real qx = lx, qy = ly;
        if (!inside) {
            real bd = 0;
            for (int s = 0; s < 16; s++) {
                real c0, s0, c1, s1;
                gon_vdir(s, c0, s0);
                gon_vdir((s + 1) & 15, c1, s1);
                const real ax = r * c0, ay = r * s0, ex = r * c1 - ax, ey = r * s1 - ay;
                real t = ((lx - ax) * ex + (ly - ay) * ey) / (ex * ex + ey * ey);
                t = std::min<real>(std::max<real>(t, 0.0), 1.0);
                const real px = ax + ex * t, py = ay + ey * t;
                const real dd = (lx - px) * (lx - px) + (ly - py) * (ly - py);
                if (s == 0 || dd < bd) { bd = dd; qx = px; qy = py; }
            }
        }
        const real qz = std::min(std::max(lz, -b.h[2]), b.h[2]);
        const V3 Q = b.x + axis(b, 0) * qx + axis(b, 1) * qy + axis(b, 2) * qz;
        const V3 diff = S - Q;
        const real dist = norm(diff);
        V3 nrm;
        real d;
        if (dist > 1e-6) {
            nrm = diff * (1.0 / dist);
            d = dist - P.pusher_radius;
        } else {
            const real pen = std::min(b.h[2] - fabs(lz), pen_side);
            d = -pen - P.pusher_radius;
            const V3 w = {S.x - b.x.x, S.y - b.x.y, 0};
            const real lw = norm(w);
            nrm = lw > 1e-9 ? w * (1.0 / lw) : V3{1, 0, 0};
        }
        if (!(d < P.margin)) continue;
        Contact& C = M.c[np];
        C.p = Q;
        C.d = d;
        C.rA = Q - b.x;
        C.rB = {0, 0, 0};
        if (np == 0 || d < best_d) { best_d = d; best_n = nrm; }
        np++;
    }
    if (np == 0) return false;
    M.A = bi; M.B = PUSHER;
    M.n = best_n;
    M.np = np;
    return true;
}

// ---- one substep ---------------------------------------------------------------------

void refresh_body_frames(Env& E) {
    for (Body& b : E.b) {
        quat_to_R(b.q, b.R);
        // world inverse inertia R diag(invIb) R^T
        int idx = 0;
        for (int a = 0; a < 3; a++)
            for (int c = a; c < 3; c++) {
                real s = 0;
                for (int k = 0; k < 3; k++) s += b.R[3 * a + k] * b.invIb[k] * b.R[3 * c + k];
                b.invIw[idx++] = s;
            }
    }
}

void body_vel(const Env& E, int id, V3& v, V3& w) {
    if (id >= 0) { v = E.b[id].v; w = E.b[id].w; }
    else if (id == PUSHER) { v = E.V; w = {0, 0, 0}; }
    else { v = {0, 0, 0}; w = {0, 0, 0}; }
}

std::vector<Manifold> collide(Env& E, const oracle_params& P) {
    const int n = (int)E.b.size();
    std::vector<real> x(3 * n), q(4 * n), h(3 * n);
    for (int i = 0; i < n; i++) {
        x[3 * i] = E.b[i].x.x; x[3 * i + 1] = E.b[i].x.y; x[3 * i + 2] = E.b[i].x.z;
        for (int k = 0; k < 4; k++) q[4 * i + k] = E.b[i].q[k];
        for (int k = 0; k < 3; k++) h[3 * i + k] = E.b[i].h[k];
        if (E.b[i].cyl) h[3 * i + 1] = -h[3 * i + 1];  // keep the cylinder mark
    }
    const real Pxy[2] = {E.P.x, E.P.y};
    set_phase(0);
    PairList<real> pl = broadphase<real>(n, x.data(), q.data(), h.data(), P.margin, E.push.active, Pxy,
                                             P.pusher_radius, P.pusher_z0, P.pusher_z1, P.pair_cap);
    set_phase(1);
    E.ev[EV_PAIR_TESTS] += (uint64_t)n * (n - 1) / 2;
    if (pl.overflow) E.overflow = true;
    std::vector<Manifold> ms;
    int npts = 0;
    bool stop = false;
    auto emit = [&](Manifold& M) {
        if (stop) return;
        if ((int)ms.size() + 1 > P.manifold_cap || npts + M.np > P.point_cap) { stop = true; E.overflow = true; return; }
        M.colour = -1;
        npts += M.np;
        ms.push_back(M);
    };
    for (size_t k = 0; k < pl.bb_i.size() && !stop; k++) {
        Manifold M;
        const int i = pl.bb_i[k], j = pl.bb_j[k];
        const bool hit = (E.b[i].cyl || E.b[j].cyl) ? convex_pair(E.b[i], i, E.b[j], j, P, M, E.ev)
                                                    : box_box(E.b[i], i, E.b[j], j, P, M, E.ev);
        if (hit) {
            const real mu = sqrt(E.b[i].mu * E.b[j].mu);
            M.mu = mu;
            const size_t before = ms.size();
            emit(M);
            if (ms.size() > before) E.ev[EV_BB_POINTS] += M.np;
        }
    }
    for (int i : pl.plane) {
        if (stop) break;
        E.ev[EV_PLANE]++;
        Manifold M;
        if (E.b[i].cyl ? cyl_plane(E.b[i], i, P, M) : box_plane(E.b[i], i, P, M)) { M.mu = sqrt(E.b[i].mu * P.table_mu); emit(M); }
    }
    for (int i : pl.pusher) {
        if (stop) break;
        E.ev[EV_PUSHER]++;
        Manifold M;
        if (E.b[i].cyl ? capsule_cyl(E.b[i], i, E.P, P, M) : capsule_box(E.b[i], i, E.P, P, M)) { M.mu = sqrt(E.b[i].mu * P.pusher_mu); emit(M); }
    }
    E.ev[EV_MANIFOLDS] += ms.size();
    E.ev[EV_POINTS] += npts;
    return ms;
}

// Contact preparation: tangent basis from the world axis least aligned with the
// normal; effective masses along n, t1, t2; target normal velocity (speculative when
// separated, Baumgarte with slop when penetrating); impulses start at zero.
void prepare(Env& E, std::vector<Manifold>& ms, const oracle_params& P) {
    for (Manifold& M : ms) {
        const V3 n = M.n;
        const real an[3] = {fabs(n.x), fabs(n.y), fabs(n.z)};
        int k = 0;
        if (an[1] < an[k]) k = 1;
        if (an[2] < an[k]) k = 2;
        const V3 e = {k == 0 ? 1.0 : 0.0, k == 1 ? 1.0 : 0.0, k == 2 ? 1.0 : 0.0};
        const V3 t = cross(n, e);
        M.t1 = t * (1.0 / norm(t));
        M.t2 = cross(n, M.t1);
        for (int p = 0; p < M.np; p++) {
            Contact& C = M.c[p];
            auto keff = [&](V3 dir) {
                real k2 = 0;
                if (M.A >= 0) {
                    const Body& a = E.b[M.A];
                    const V3 rn = cross(C.rA, dir);
                    k2 += a.invm + dot(rn, sym_mul(a.invIw, rn));
                }
                if (M.B >= 0) {
                    const Body& b = E.b[M.B];
                    const V3 rn = cross(C.rB, dir);
                    k2 += b.invm + dot(rn, sym_mul(b.invIw, rn));
                }
                return k2;
            };
            C.invKn = 1.0 / keff(n);
            C.invKt1 = 1.0 / keff(M.t1);
            C.invKt2 = 1.0 / keff(M.t2);
            if (C.d > 0) C.bias = -C.d / P.dt;
            else C.bias = (P.baumgarte / P.dt) * std::max<real>(-C.d - P.slop, 0.0);
            C.ln = C.lt1 = C.lt2 = 0;
        }
    }
}

// Greedy colouring in manifold order: each manifold takes the smallest colour not yet
// used by a manifold that shares one of its dynamic bodies (plane and pusher are
// static and never conflict).  Returns the number of colours.
int colour_manifolds(Env& E, std::vector<Manifold>& ms) {
    std::vector<uint32_t> used(E.b.size(), 0u);
    int ncol = 0;
    for (Manifold& M : ms) {
        uint32_t u = 0;
        if (M.A >= 0) u |= used[M.A];
        if (M.B >= 0) u |= used[M.B];
        int c = 0;
        while (c < MAX_COLOURS && (u >> c & 1u)) c++;
        if (c >= MAX_COLOURS) { M.colour = -1; E.overflow = true; continue; }
        M.colour = c;
        if (M.A >= 0) used[M.A] |= 1u << c;
        if (M.B >= 0) used[M.B] |= 1u << c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    return ncol;
}

void apply_impulse(Env& E, const Manifold& M, const Contact& C, V3 Pimp) {
    if (M.A >= 0) {
        Body& a = E.b[M.A];
        a.v = a.v - Pimp * a.invm;
        a.w = a.w - sym_mul(a.invIw, cross(C.rA, Pimp));
    }
    if (M.B >= 0) {
        Body& b = E.b[M.B];
        b.v = b.v + Pimp * b.invm;
        b.w = b.w + sym_mul(b.invIw, cross(C.rB, Pimp));
    }
}

V3 rel_vel(const Env& E, const Manifold& M, const Contact& C) {
    V3 va, wa, vb, wb;
    body_vel(E, M.A, va, wa);
    body_vel(E, M.B, vb, wb);
    return (vb + cross(wb, C.rB)) - (va + cross(wa, C.rA));
}

// One manifold's Gauss-Seidel update: all normal rows, then all friction pairs.
void solve_manifold(Env& E, Manifold& M) {
    for (int p = 0; p < M.np; p++) {
        Contact& C = M.c[p];
        const real vn = dot(M.n, rel_vel(E, M, C));
        const real delta = -(vn - C.bias) * C.invKn;
        const real l = std::max<real>(C.ln + delta, 0.0);
        const real dl = l - C.ln;
        C.ln = l;
        apply_impulse(E, M, C, M.n * dl);
    }
    for (int p = 0; p < M.np; p++) {
        Contact& C = M.c[p];
        const V3 vr = rel_vel(E, M, C);
        const real vt1 = dot(M.t1, vr), vt2 = dot(M.t2, vr);
        real c1 = C.lt1 - vt1 * C.invKt1;
        real c2 = C.lt2 - vt2 * C.invKt2;
        const real lim = M.mu * C.ln;
        const real l2 = c1 * c1 + c2 * c2;
        if (l2 > lim * lim) {
            const real s = lim / sqrt(l2);
            c1 *= s;
            c2 *= s;
        }
        const real d1 = c1 - C.lt1, d2 = c2 - C.lt2;
        C.lt1 = c1;
        C.lt2 = c2;
        apply_impulse(E, M, C, M.t1 * d1 + M.t2 * d2);
    }
}

// Projected Gauss-Seidel: iterations, colours in order, manifolds of a colour in
// manifold order (or reversed, for the order-independence check).
void pgs(Env& E, std::vector<Manifold>& ms, int ncol, int iters, bool reverse_within_colour) {
    for (int it = 0; it < iters; it++)
        for (int c = 0; c < ncol; c++) {
            const int N = (int)ms.size();
            for (int k = 0; k < N; k++) {
                Manifold& M = ms[reverse_within_colour ? N - 1 - k : k];
                if (M.colour != c) continue;
                solve_manifold(E, M);
                E.ev[EV_PGS_MAN]++;
                E.ev[EV_PGS_PTS] += M.np;
                if (M.A >= 0 && M.B >= 0) E.ev[EV_PGS_BB_POINTS] += M.np;
            }
        }
}

// Warm start (a reading beyond the paper, off by default): a new contact point takes the
// impulses of the nearest point of the same body pair in the previous substep when the
// two offsets, written in the key body's frame, lie within the tolerance (each old point
// used once, new points in order); the friction part is the old world friction vector
// projected on the new tangents.  The carried impulses are applied to the bodies before
// the first iteration, manifold by manifold in colour order.
inline V3 key_local(const Env& E, const Manifold& M, const Contact& C) {
    const bool a = M.A >= 0;
    const Body& k = E.b[a ? M.A : M.B];
    const V3 r = a ? C.rA : C.rB;
    return {k.R[0] * r.x + k.R[3] * r.y + k.R[6] * r.z, k.R[1] * r.x + k.R[4] * r.y + k.R[7] * r.z,
            k.R[2] * r.x + k.R[5] * r.y + k.R[8] * r.z};
}

void warm_start(Env& E, std::vector<Manifold>& ms, int ncol, const oracle_params& P) {
    for (Manifold& M : ms) {
        const WarmManifold* W = nullptr;
        for (const WarmManifold& w : E.warm)
            if (w.A == M.A && w.B == M.B) { W = &w; break; }
        if (!W) continue;
        bool used[4] = {false, false, false, false};
        for (int p = 0; p < M.np; p++) {
            Contact& C = M.c[p];
            const V3 loc = key_local(E, M, C);
            int best = -1;
            real bd = P.warm_tolerance * P.warm_tolerance;
            for (int q = 0; q < W->np; q++) {
                if (used[q]) continue;
                const V3 d = loc - W->p[q].loc;
                const real d2 = dot(d, d);
                if (d2 <= bd) { bd = d2; best = q; }
            }
            if (best < 0) continue;
            used[best] = true;
            C.ln = W->p[best].ln;
            C.lt1 = dot(W->p[best].Pt, M.t1);
            C.lt2 = dot(W->p[best].Pt, M.t2);
        }
    }
    for (int c = 0; c < ncol; c++)
        for (Manifold& M : ms) {
            if (M.colour != c) continue;
            for (int p = 0; p < M.np; p++) {
                const Contact& C = M.c[p];
                apply_impulse(E, M, C, (M.n * C.ln + M.t1 * C.lt1) + M.t2 * C.lt2);
            }
        }
}

void save_warm(Env& E, const std::vector<Manifold>& ms) {
    E.warm.clear();
    for (const Manifold& M : ms) {
        if (M.colour < 0) continue;
        WarmManifold w;
        w.A = M.A;
        w.B = M.B;
        w.np = M.np;
        for (int p = 0; p < M.np; p++) {
            const Contact& C = M.c[p];
            w.p[p].loc = key_local(E, M, C);
            w.p[p].ln = C.ln;
            w.p[p].Pt = M.t1 * C.lt1 + M.t2 * C.lt2;
        }
        E.warm.push_back(w);
    }
}

// Semi-implicit Euler: x += v dt; q += dt/2 (0, w) (x) q, renormalised.
void integrate(Env& E, const oracle_params& P) {
    const real dt = P.dt;
    for (Body& b : E.b) {
        b.x = b.x + b.v * dt;
        const real w0 = b.q[0];
        const V3 qv = {b.q[1], b.q[2], b.q[3]};
        const real dw = -dot(b.w, qv);
        const V3 dv = b.w * w0 + cross(b.w, qv);
        const real hd = 0.5 * dt;
        real q[4] = {w0 + hd * dw, qv.x + hd * dv.x, qv.y + hd * dv.y, qv.z + hd * dv.z};
        const real l = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        for (int k = 0; k < 4; k++) b.q[k] = q[k] / l;
    }
}

void substep(Env& E, const oracle_params& P, int s, bool reverse_within_colour = false) {
    set_phase(4);
    pusher_at(E, P, s);
    set_phase(0);
    const V3 g = {P.gravity[0], P.gravity[1], P.gravity[2]};
    for (Body& b : E.b) b.v = b.v + g * P.dt;
    refresh_body_frames(E);
    std::vector<Manifold> ms = collide(E, P);
    set_phase(2);
    prepare(E, ms, P);
    set_phase(4);
    const int ncol = colour_manifolds(E, ms);
    E.ev[EV_COLOURS] += ncol;
    set_phase(3);
    if (P.warm_start) warm_start(E, ms, ncol, P);
    pgs(E, ms, ncol, P.pgs_iters, reverse_within_colour);
    if (P.warm_start) save_warm(E, ms);
    set_phase(0);
    integrate(E, P);
    set_phase(4);
    E.ev[EV_SUBSTEPS]++;
    E.ev[EV_BOX_STEPS] += E.b.size();
}

// ---- rollouts ------------------------------------------------------------------------

void grasp_table(int K, std::vector<real>& ca, std::vector<real>& sa) {
    ca.resize(K); sa.resize(K);
    for (int k = 0; k < K; k++) {
        const real th = k * M_PI / K;
        ca[k] = (real)(float)std::cos(as_double(th));   // binary32-rounded table, as in the engine
        sa[k] = (real)(float)std::sin(as_double(th));
    }
}

void env_arrays(const Env& E, std::vector<real>& x, std::vector<real>& q, std::vector<real>& h) {
    const int n = (int)E.b.size();
    x.resize(3 * n); q.resize(4 * n); h.resize(3 * n);
    for (int i = 0; i < n; i++) {
        x[3 * i] = E.b[i].x.x; x[3 * i + 1] = E.b[i].x.y; x[3 * i + 2] = E.b[i].x.z;
        for (int k = 0; k < 4; k++) q[4 * i + k] = E.b[i].q[k];
        for (int k = 0; k < 3; k++) h[3 * i + k] = E.b[i].h[k];
        if (E.b[i].cyl) h[3 * i + 1] = -h[3 * i + 1];  // keep the cylinder mark
    }
}

bool env_graspable(const Env& E, const oracle_params& P) {
    std::vector<real> x, q, h, ca, sa;
    env_arrays(E, x, q, h);
    grasp_table(P.grasp_angles, ca, sa);
    return graspable<real>((int)E.b.size(), x.data(), q.data(), h.data(), E.target, ca.data(), sa.data(),
                             P.grasp_angles, P.grasp_opening, P.grasp_clearance, P.finger_depth, P.finger_width);
}

struct RolloutOut { int32_t cost; float reward; uint8_t flags; int32_t steps; };

// Rollout of one environment (Sec. IV-C, batch expansion then batch simulation): the
// caller's first push, then depth-1 sampled pushes; after each push the workspace and
// grasp tests decide cost k and reward gamma^(k-1), or cost depth+1 and reward 0.
RolloutOut rollout_env(Env& E, const oracle_params& P, const float* first_push, int depth, uint64_t seed,
                       real* child13) {
    RolloutOut r{depth + 1, 0.f, 0, 0};
    for (int k = 1; k <= depth; k++) {
        real push[4];
        if (k == 1) {
            for (int i = 0; i < 4; i++) push[i] = first_push[i];
            std::vector<real> x, q, h;
            env_arrays(E, x, q, h);
            std::vector<Foot<real>> F(E.b.size());
            for (size_t i = 0; i < E.b.size(); i++) F[i] = footprint(&x[3 * i], &q[4 * i], &h[3 * i]);
            if (start_blocked<real>(F, push[0], push[1], P.pusher_radius)) { r.flags |= F_INVALID_START; break; }
        } else {
            std::vector<real> x, q, h;
            env_arrays(E, x, q, h);
            const int a = sample_push<real>((int)E.b.size(), x.data(), q.data(), h.data(), seed, k, P.pusher_radius,
                                              P.sample_clearance, P.push_length, P.sample_attempts, P.contour_points, push);
            E.ev[EV_SAMPLE_ATTEMPTS] += a < 0 ? P.sample_attempts : a + 1;
            if (a < 0) { r.flags |= F_NOOP; push[0] = push[2] = push[1] = push[3] = 0; }
        }
        set_push(E, P, push);
        for (int s = 0; s < P.substeps_per_push; s++) { substep(E, P, s); r.steps++; }
        if (k == 1 && child13) store_env(E, child13);
        E.ev[EV_PUSH_EVALS]++;
        bool out = false;
        for (const Body& b : E.b)
            if (fabs(b.x.x) > P.table_half[0] || fabs(b.x.y) > P.table_half[1]) out = true;
        if (out) { r.flags |= F_OUT_OF_WS; break; }
        if (env_graspable(E, P)) {
            r.cost = k;
            r.reward = (float)std::pow(P.gamma, k - 1);
            if (k == 1) r.flags |= F_GRASP1;
            break;
        }
    }
    if (E.overflow) r.flags |= F_OVERFLOW;
    return r;
}

void to_double(int n, const float* s, real* d) { for (int i = 0; i < 13 * n; i++) d[i] = s[i]; }

}  // namespace

#ifndef ORACLE_COUNT_FLOPS
extern "C" {

int oracle_version(void) { return 1; }
int oracle_num_events(void) { return NEV; }

void oracle_default_params(oracle_params* p) {
    std::memset(p, 0, sizeof(*p));
    p->dt = 1.0 / 240.0;
    p->gravity[0] = 0; p->gravity[1] = 0; p->gravity[2] = -9.81;
    p->table_half[0] = 0.2; p->table_half[1] = 0.2;
    p->table_mu = 0.5; p->pusher_mu = 0.5;
    p->pusher_radius = 0.01; p->pusher_z0 = 0.01; p->pusher_z1 = 0.20;
    p->pusher_speed = 0.1; p->push_length = 0.1;
    p->gamma = 0.8;
    p->grasp_opening = 0.085; p->grasp_clearance = 0.002; p->finger_depth = 0.01; p->finger_width = 0.022;
    p->margin = 1e-3; p->slop = 5e-4; p->baumgarte = 0.2;
    p->sample_clearance = 0.005;
    p->substeps_per_push = 240; p->pgs_iters = 10;
    p->point_cap = 512; p->manifold_cap = 256; p->pair_cap = 1024;
    p->grasp_angles = 16; p->sample_attempts = 8; p->contour_points = 16;
    p->warm_start = 0; p->warm_tolerance = 2e-3;
}

uint64_t oracle_splitmix64(uint64_t* state) { return splitmix64_next(*state); }

// Full rollouts of n_envs environments; env e owns boxes box_offset[e]..box_offset[e+1]
// of the flat arrays.  Threads split the environments.  Returns 0.
int oracle_rollout(const oracle_params* P, int n_envs, const int32_t* box_offset, const float* state13,
                   const float* half, const float* mass, const float* mu, const int32_t* target,
                   const float* first_push, int depth, const uint64_t* seeds, int n_threads,
                   int32_t* out_cost, float* out_reward, uint8_t* out_flags, int32_t* out_steps,
                   double* out_state13, double* out_child13, uint64_t* out_events) {
    std::atomic<int> next(0);
    auto worker = [&]() {
        for (;;) {
            const int e = next.fetch_add(1);
            if (e >= n_envs) break;
            const int a = box_offset[e], n = box_offset[e + 1] - a;
            std::vector<double> s(13 * n);
            to_double(n, state13 + 13 * a, s.data());
            Env E;
            load_env(E, n, s.data(), half + 3 * a, mass + a, mu + a);
            E.target = target[e];
            const RolloutOut r = rollout_env(E, *P, first_push + 4 * e, depth, seeds ? seeds[e] : 0,
                                             out_child13 ? out_child13 + 13 * a : nullptr);
            out_cost[e] = r.cost; out_reward[e] = r.reward; out_flags[e] = r.flags; out_steps[e] = r.steps;
            if (out_state13) store_env(E, out_state13 + 13 * a);
            if (out_events) for (int k = 0; k < NEV; k++) out_events[(size_t)NEV * e + k] = E.ev[k];
        }
    };
    if (n_threads <= 1) worker();
    else {
        std::vector<std::thread> th;
        for (int t = 0; t < n_threads; t++) th.emplace_back(worker);
        for (auto& t : th) t.join();
    }
    return 0;
}

// `count` substeps of one environment (double state in/out) under push `push` (NULL: no
// pusher), starting at substep index s0 of that push.  reverse != 0 processes the
// manifolds of each colour in reverse order.  Returns 1 if a cap overflowed.
int oracle_run_substeps(const oracle_params* P, int n, double* state13, const float* half, const float* mass,
                        const float* mu, const double* push, int s0, int count, int reverse, uint64_t* events) {
    Env E;
    load_env(E, n, state13, half, mass, mu);
    if (push) set_push(E, *P, push);
    for (int s = s0; s < s0 + count; s++) substep(E, *P, s, reverse != 0);
    store_env(E, state13);
    if (events) for (int k = 0; k < NEV; k++) events[k] = E.ev[k];
    return E.overflow ? 1 : 0;
}

// Contact manifolds of one state (after the substep's gravity update), with colours.
// Per manifold: info[m] = {A, B, npts, colour}; normal[m][3]; pts[m][4][4] = p xyz, depth.
int oracle_contacts(const oracle_params* P, int n, const double* state13, const float* half, const float* mass,
                    const float* mu, const double* push, int s, int max_m, int32_t* info, double* normal,
                    double* pts) {
    Env E;
    load_env(E, n, state13, half, mass, mu);
    if (push) set_push(E, *P, push);
    pusher_at(E, *P, s);
    refresh_body_frames(E);
    std::vector<Manifold> ms = collide(E, *P);
    colour_manifolds(E, ms);
    const int nm = (int)ms.size();
    for (int m = 0; m < nm && m < max_m; m++) {
        info[4 * m] = ms[m].A; info[4 * m + 1] = ms[m].B; info[4 * m + 2] = ms[m].np; info[4 * m + 3] = ms[m].colour;
        normal[3 * m] = ms[m].n.x; normal[3 * m + 1] = ms[m].n.y; normal[3 * m + 2] = ms[m].n.z;
        for (int p = 0; p < ms[m].np; p++) {
            double* o = pts + 16 * m + 4 * p;
            o[0] = ms[m].c[p].p.x; o[1] = ms[m].c[p].p.y; o[2] = ms[m].c[p].p.z; o[3] = ms[m].c[p].d;
        }
    }
    return nm;
}

// Separating-axis result for a pair of boxes (state rows of 13): separation, axis id,
// normal A->B, contact points and depths.  Returns the number of contact points, or -1
// when the boxes are farther apart than the margin.  When either body is a cylinder the
// general convex test decides and the axis id is f (face f of A), 100 + f (face f of B)
// or 200 + 9 i + j (edge directions i of A and j of B).
int oracle_box_box(const double* sA, const float* hA, const double* sB, const float* hB, double margin,
                   double* out_sep, int32_t* out_axis, double* out_n, double* out_p, double* out_d) {
    oracle_params P;
    oracle_default_params(&P);
    P.margin = margin;
    Env E;
    double s[26];
    std::memcpy(s, sA, 13 * sizeof(double));
    std::memcpy(s + 13, sB, 13 * sizeof(double));
    const float h[6] = {hA[0], hA[1], hA[2], hB[0], hB[1], hB[2]};
    const float m[2] = {1, 1}, mu[2] = {0.5f, 0.5f};
    load_env(E, 2, s, h, m, mu);
    refresh_body_frames(E);
    if (E.b[0].cyl || E.b[1].cyl) {
        const ConvexSat c = sat_convex(E.b[0], E.b[1], margin);
        if (!c.touching) return -1;
        *out_sep = c.sep;
        *out_axis = c.kind == 2 ? 200 + 9 * c.i + c.j : 100 * c.kind + c.i;
        out_n[0] = c.n.x; out_n[1] = c.n.y; out_n[2] = c.n.z;
        Manifold M;
        if (!convex_pair(E.b[0], 0, E.b[1], 1, P, M, E.ev)) return 0;
        for (int k = 0; k < M.np; k++) {
            out_p[3 * k] = M.c[k].p.x; out_p[3 * k + 1] = M.c[k].p.y; out_p[3 * k + 2] = M.c[k].p.z;
            out_d[k] = M.c[k].d;
        }
        return M.np;
    }
    const SatResult r = sat(E.b[0], E.b[1], margin);
    if (!r.touching) return -1;
    *out_sep = r.sep; *out_axis = r.axis;
    out_n[0] = r.n.x; out_n[1] = r.n.y; out_n[2] = r.n.z;
    Manifold M;
    if (!box_box(E.b[0], 0, E.b[1], 1, P, M, E.ev)) return 0;
    for (int k = 0; k < M.np; k++) {
        out_p[3 * k] = M.c[k].p.x; out_p[3 * k + 1] = M.c[k].p.y; out_p[3 * k + 2] = M.c[k].p.z;
        out_d[k] = M.c[k].d;
    }
    return M.np;
}

// Pair lists in binary32 (f32 != 0) or double.  Output: bb[k] = {i, j}; plane and pusher
// box lists.  pusher_xy NULL: no pusher.  Returns 1 if the pair cap overflowed.
int oracle_pairs(const oracle_params* P, int f32, int n, const float* state13, const float* half,
                 const float* pusher_xy, int32_t* bb, int32_t* n_bb, int32_t* plane, int32_t* n_plane,
                 int32_t* pusher, int32_t* n_pusher) {
    auto run = [&](auto zero) {
        using T = decltype(zero);
        std::vector<T> x(3 * n), q(4 * n), h(3 * n);
        for (int i = 0; i < n; i++) {
            for (int k = 0; k < 3; k++) x[3 * i + k] = (T)state13[13 * i + k];
            for (int k = 0; k < 4; k++) q[4 * i + k] = (T)state13[13 * i + 3 + k];
            for (int k = 0; k < 3; k++) h[3 * i + k] = (T)half[3 * i + k];
        }
        T Pxy[2] = {0, 0};
        if (pusher_xy) { Pxy[0] = (T)pusher_xy[0]; Pxy[1] = (T)pusher_xy[1]; }
        PairList<T> pl = broadphase<T>(n, x.data(), q.data(), h.data(), (T)P->margin, pusher_xy != nullptr, Pxy,
                                       (T)P->pusher_radius, (T)P->pusher_z0, (T)P->pusher_z1, P->pair_cap);
        *n_bb = (int32_t)pl.bb_i.size();
        for (size_t k = 0; k < pl.bb_i.size(); k++) { bb[2 * k] = pl.bb_i[k]; bb[2 * k + 1] = pl.bb_j[k]; }
        *n_plane = (int32_t)pl.plane.size();
        for (size_t k = 0; k < pl.plane.size(); k++) plane[k] = pl.plane[k];
        *n_pusher = (int32_t)pl.pusher.size();
        for (size_t k = 0; k < pl.pusher.size(); k++) pusher[k] = pl.pusher[k];
        return pl.overflow ? 1 : 0;
    };
    return f32 ? run(0.0f) : run(0.0);
}

// Grasp-clearance decision for target t in binary32 (f32 != 0) or double.
int oracle_grasp(const oracle_params* P, int f32, int n, const float* state13, const float* half, int t) {
    auto run = [&](auto zero) {
        using T = decltype(zero);
        std::vector<T> x(3 * n), q(4 * n), h(3 * n), ca(P->grasp_angles), sa(P->grasp_angles);
        for (int i = 0; i < n; i++) {
            for (int k = 0; k < 3; k++) x[3 * i + k] = (T)state13[13 * i + k];
            for (int k = 0; k < 4; k++) q[4 * i + k] = (T)state13[13 * i + 3 + k];
            for (int k = 0; k < 3; k++) h[3 * i + k] = (T)half[3 * i + k];
        }
        for (int k = 0; k < P->grasp_angles; k++) {
            const double th = k * M_PI / P->grasp_angles;
            ca[k] = (T)(float)std::cos(th);
            sa[k] = (T)(float)std::sin(th);
        }
        return graspable<T>(n, x.data(), q.data(), h.data(), t, ca.data(), sa.data(), P->grasp_angles,
                            (T)P->grasp_opening, (T)P->grasp_clearance, (T)P->finger_depth, (T)P->finger_width)
                   ? 1 : 0;
    };
    return f32 ? run(0.0f) : run(0.0);
}

// Contour-sampled push k (>= 2) for a state, in binary32 (f32 != 0) or double.  Returns
// the accepted attempt index or -1 (no-op push).
int oracle_sample_push(const oracle_params* P, int f32, int n, const float* state13, const float* half,
                       uint64_t seed, int k, float* out_push) {
    auto run = [&](auto zero) {
        using T = decltype(zero);
        std::vector<T> x(3 * n), q(4 * n), h(3 * n);
        for (int i = 0; i < n; i++) {
            for (int j = 0; j < 3; j++) x[3 * i + j] = (T)state13[13 * i + j];
            for (int j = 0; j < 4; j++) q[4 * i + j] = (T)state13[13 * i + 3 + j];
            for (int j = 0; j < 3; j++) h[3 * i + j] = (T)half[3 * i + j];
        }
        T out[4] = {0, 0, 0, 0};
        const int a = sample_push<T>(n, x.data(), q.data(), h.data(), seed, k, (T)P->pusher_radius,
                                     (T)P->sample_clearance, (T)P->push_length, P->sample_attempts,
                                     P->contour_points, out);
        for (int j = 0; j < 4; j++) out_push[j] = (float)out[j];
        return a;
    };
    return f32 ? run(0.0f) : run(0.0);
}

// 1 if a push starting at (sx, sy) is blocked by a footprint (binary32 when f32 != 0).
int oracle_start_blocked(const oracle_params* P, int f32, int n, const float* state13, const float* half,
                         float sx, float sy) {
    auto run = [&](auto zero) {
        using T = decltype(zero);
        std::vector<Foot<T>> F(n);
        for (int i = 0; i < n; i++) {
            T x[3], q[4], h[3];
            for (int k = 0; k < 3; k++) x[k] = (T)state13[13 * i + k];
            for (int k = 0; k < 4; k++) q[k] = (T)state13[13 * i + 3 + k];
            for (int k = 0; k < 3; k++) h[k] = (T)half[3 * i + k];
            F[i] = footprint<T>(x, q, h);
        }
        return start_blocked<T>(F, (T)sx, (T)sy, (T)P->pusher_radius) ? 1 : 0;
    };
    return f32 ? run(0.0f) : run(0.0);
}

// Footprints (cx, cy, ux, uy, vx, vy, su, sv) of every box, binary32 or double.
void oracle_footprints(int f32, int n, const float* state13, const float* half, double* out8) {
    for (int i = 0; i < n; i++) {
        if (f32) {
            float x[3], q[4], h[3];
            for (int k = 0; k < 3; k++) x[k] = state13[13 * i + k];
            for (int k = 0; k < 4; k++) q[k] = state13[13 * i + 3 + k];
            for (int k = 0; k < 3; k++) h[k] = half[3 * i + k];
            const Foot<float> f = footprint<float>(x, q, h);
            const float v[8] = {f.cx, f.cy, f.ux, f.uy, f.vx, f.vy, f.su, f.sv};
            for (int k = 0; k < 8; k++) out8[8 * i + k] = v[k];
        } else {
            double x[3], q[4], h[3];
            for (int k = 0; k < 3; k++) x[k] = state13[13 * i + k];
            for (int k = 0; k < 4; k++) q[k] = state13[13 * i + 3 + k];
            for (int k = 0; k < 3; k++) h[k] = half[3 * i + k];
            const Foot<double> f = footprint<double>(x, q, h);
            const double v[8] = {f.cx, f.cy, f.ux, f.uy, f.vx, f.vy, f.su, f.sv};
            for (int k = 0; k < 8; k++) out8[8 * i + k] = v[k];
        }
    }
}

// Heightmap (W x H cells of `cell` m from (x0, y0)) of one state, binary32 (f32 != 0)
// or double; written as float.
void oracle_heightmap(int f32, int n, const float* state13, const float* half, int W, int H, double x0, double y0,
                      double cell, float* out) {
    auto run = [&](auto zero) {
        using T = decltype(zero);
        std::vector<T> x(3 * n), q(4 * n), h(3 * n), o((size_t)W * H);
        for (int i = 0; i < n; i++) {
            for (int k = 0; k < 3; k++) x[3 * i + k] = (T)state13[13 * i + k];
            for (int k = 0; k < 4; k++) q[4 * i + k] = (T)state13[13 * i + 3 + k];
            for (int k = 0; k < 3; k++) h[3 * i + k] = (T)half[3 * i + k];
        }
        heightmap<T>(n, x.data(), q.data(), h.data(), W, H, (T)(float)x0, (T)(float)y0, (T)(float)cell, o.data());
        for (size_t k = 0; k < o.size(); k++) out[k] = (float)o[k];
    };
    if (f32) run(0.0f);
    else run(0.0);
}

// Heightmap grasp decision for target t (binary32 twin when f32 != 0): the state's own
// heightmap on the Sec. V-A grid, then the finger-rectangle test with tips `depth` below
// the target's top.
int oracle_grasp_heightmap(const oracle_params* P, int f32, int n, const float* state13, const float* half, int t,
                           double depth) {
    const int cells = 144;
    auto run = [&](auto zero) {
        using T = decltype(zero);
        std::vector<T> x(3 * n), q(4 * n), h(3 * n), ca(P->grasp_angles), sa(P->grasp_angles), map(cells * cells);
        for (int i = 0; i < n; i++) {
            for (int k = 0; k < 3; k++) x[3 * i + k] = (T)state13[13 * i + k];
            for (int k = 0; k < 4; k++) q[4 * i + k] = (T)state13[13 * i + 3 + k];
            for (int k = 0; k < 3; k++) h[3 * i + k] = (T)half[3 * i + k];
        }
        for (int k = 0; k < P->grasp_angles; k++) {
            const double th = k * M_PI / P->grasp_angles;
            ca[k] = (T)(float)std::cos(th);
            sa[k] = (T)(float)std::sin(th);
        }
        const T x0 = (T)-0.144f, cw = (T)0.002f;
        heightmap<T>(n, x.data(), q.data(), h.data(), cells, cells, x0, x0, cw, map.data());
        return graspable_hm<T>(map.data(), cells, x0, cw, n, x.data(), q.data(), h.data(), t, ca.data(), sa.data(),
                               P->grasp_angles, (T)P->grasp_opening, (T)P->grasp_clearance, (T)P->finger_depth,
                               (T)P->finger_width, (T)(float)depth) ? 1 : 0;
    };
    return f32 ? run(0.0f) : run(0.0);
}

}  // extern "C"
#endif

#ifdef ORACLE_COUNT_FLOPS
extern "C" {
// Flop-counting build only: `count` substeps of one environment from state13 with the
// given push; flops[0..4] = adds, subtracts, multiplies, divides and square roots of the
// double engine by phase (per body, narrowphase, contact preparation, contact solve,
// the rest), events[NEV] = the engine's event counters.
int oracle_count_flops(const oracle_params* P, int n, const double* state13, const float* half, const float* mass,
                       const float* mu, const double* push, int count, uint64_t* flops, uint64_t* events) {
    std::vector<real> s13(state13, state13 + 13 * n);
    std::vector<real> pu(push, push + 4);
    Env E;
    load_env(E, n, s13.data(), half, mass, mu);
    set_push(E, *P, pu.data());
    for (int k = 0; k < 8; k++) g_flops[k] = 0;  // the substeps only, not the set-up
    for (int s = 0; s < count; s++) substep(E, *P, s);
    for (int k = 0; k < 5; k++) flops[k] = g_flops[k];
    for (int k = 0; k < NEV; k++) events[k] = E.ev[k];
    return E.overflow ? 1 : 0;
}
int oracle_num_events(void) { return NEV; }
}
#endif

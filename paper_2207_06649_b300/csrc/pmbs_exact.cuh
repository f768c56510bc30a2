// Bit-exact binary32 predicates of the rollout engine: rotation matrix, AABB, top-down
// footprint, grasp-clearance finger test, start-pose check and contour push sampler.
// Every operation is an explicitly rounded intrinsic (__fmul_rn, __fadd_rn, ...), so the
// compiler cannot fuse or reorder them: the results are defined by IEEE binary32 and the
// evaluation order written here, and decisions taken on identical FP32 states are the
// same on any conforming implementation.
#pragma once
#include <cstdint>

namespace pmbs {

__device__ __forceinline__ float xm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float xa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float xs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float xd(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float xsqrt(float a) { return __fsqrt_rn(a); }
// dot of two 2-vectors: (a0 b0) + (a1 b1)
__device__ __forceinline__ float xdot2(float a0, float a1, float b0, float b1) {
    return xa(xm(a0, b0), xm(a1, b1));
}

// Rotation matrix (row-major) of the unit quaternion (w, x, y, z); column k is box axis k.
__device__ __forceinline__ void quat_to_R_exact(float w, float x, float y, float z, float* R) {
    const float xx = xm(x, x), yy = xm(y, y), zz = xm(z, z);
    const float xy = xm(x, y), xz = xm(x, z), yz = xm(y, z);
    const float wx = xm(w, x), wy = xm(w, y), wz = xm(w, z);
    R[0] = xs(1.f, xm(2.f, xa(yy, zz))); R[1] = xm(2.f, xs(xy, wz)); R[2] = xm(2.f, xa(xz, wy));
    R[3] = xm(2.f, xa(xy, wz)); R[4] = xs(1.f, xm(2.f, xa(xx, zz))); R[5] = xm(2.f, xs(yz, wx));
    R[6] = xm(2.f, xs(xz, wy)); R[7] = xm(2.f, xa(yz, wx)); R[8] = xs(1.f, xm(2.f, xa(xx, yy)));
}

// Cylinders: a half-extent row (r, -r, h) marks a cylinder of radius r and half height h
// about its body z axis.  Its contact, footprint and heightmap shape is the right prism
// over the regular 16-gon inscribed in its circle: cap vertex k at angle k pi/8 in the
// body xy plane, side face s with outward normal at angle (2s + 1) pi/16 and apothem
// r cos(pi/16), cap edges of half length r sin(pi/16).  Direction tables (cos, sin) of
// the vertex directions k = 0..7 and side normals s = 0..7 (k + 8, s + 8: negated), the
// closed forms rounded to binary32.
__constant__ float kGonC[8] = {1.f, 0.923879504f, 0.707106769f, 0.382683426f, 0.f, -0.382683426f, -0.707106769f,
                               -0.923879504f};
__constant__ float kGonS[8] = {0.f, 0.382683426f, 0.707106769f, 0.923879504f, 1.f, 0.923879504f, 0.707106769f,
                               0.382683426f};
__constant__ float kGonFC[8] = {0.980785251f, 0.831469595f, 0.555570245f, 0.195090324f, -0.195090324f,
                                -0.555570245f, -0.831469595f, -0.980785251f};
__constant__ float kGonFS[8] = {0.195090324f, 0.555570245f, 0.831469595f, 0.980785251f, 0.980785251f,
                                0.831469595f, 0.555570245f, 0.195090324f};
constexpr float kGonApo = 0.980785251f;       // cos(pi/16)
constexpr float kGonHalfEdge = 0.195090324f;  // sin(pi/16)

// Radial support of the unit 16-gon along the body-plane direction (p0, p1):
// max_k |c_k p0 + s_k p1| over the eight vertex directions.
__device__ __forceinline__ float gon_support_exact(float p0, float p1) {
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 8; k++) m = fmaxf(m, fabsf(xa(xm(kGonC[k], p0), xm(kGonS[k], p1))));
    return m;
}

// AABB half width along world axis k: (|R_k0| h0 + |R_k1| h1) + |R_k2| h2 (a cylinder's
// bounding box: h1 taken as |h1| = r).
__device__ __forceinline__ float aabb_half_exact(const float* Rrow, float h0, float h1, float h2) {
    return xa(xa(xm(fabsf(Rrow[0]), h0), xm(fabsf(Rrow[1]), fabsf(h1))), xm(fabsf(Rrow[2]), h2));
}

// Vertical half extent (support along z) of a box or cylinder.
__device__ __forceinline__ float vertical_half_exact(const float* R, float h0, float h1, float h2) {
    if (h1 < 0.f) return xa(xm(gon_support_exact(R[6], R[7]), h0), xm(fabsf(R[8]), h2));
    return aabb_half_exact(R + 6, h0, h1, h2);
}

// Footprint: centre, unit axes u, v = perp(u), support half widths su, sv (the rectangle
// bounding the body's projection along u and v).
struct Foot {
    float cx, cy, ux, uy, vx, vy, su, sv;
};

__device__ __forceinline__ Foot footprint_exact(float cx, float cy, const float* R, float h0, float h1,
                                                float h2) {
    float ex = R[0], ey = R[3];
    float l2 = xdot2(ex, ey, ex, ey);
    if (l2 < 1e-12f) {
        ex = R[1];
        ey = R[4];
        l2 = xdot2(ex, ey, ex, ey);
    }
    const float len = xsqrt(l2);
    Foot f;
    f.cx = cx;
    f.cy = cy;
    f.ux = xd(ex, len);
    f.uy = xd(ey, len);
    f.vx = -f.uy;
    f.vy = f.ux;
    if (h1 < 0.f) {
        // cylinder: r times the 16-gon support of (u.x_b, u.y_b), plus h |u.z_b|
        f.su = xa(xm(gon_support_exact(xdot2(R[0], R[3], f.ux, f.uy), xdot2(R[1], R[4], f.ux, f.uy)), h0),
                  xm(fabsf(xdot2(R[2], R[5], f.ux, f.uy)), h2));
        f.sv = xa(xm(gon_support_exact(xdot2(R[0], R[3], f.vx, f.vy), xdot2(R[1], R[4], f.vx, f.vy)), h0),
                  xm(fabsf(xdot2(R[2], R[5], f.vx, f.vy)), h2));
        return f;
    }
    f.su = xa(xa(xm(fabsf(xdot2(R[0], R[3], f.ux, f.uy)), h0), xm(fabsf(xdot2(R[1], R[4], f.ux, f.uy)), h1)),
              xm(fabsf(xdot2(R[2], R[5], f.ux, f.uy)), h2));
    f.sv = xa(xa(xm(fabsf(xdot2(R[0], R[3], f.vx, f.vy)), h0), xm(fabsf(xdot2(R[1], R[4], f.vx, f.vy)), h1)),
              xm(fabsf(xdot2(R[2], R[5], f.vx, f.vy)), h2));
    return f;
}

// Finger rectangle (centre fc, axes a, b; half sizes hl, hw) overlaps footprint o under
// the 2-D separating-axis test; touching projections do not overlap.
__device__ __forceinline__ bool finger_overlaps_exact(const Foot& o, float fcx, float fcy, float ax, float ay,
                                                      float bx, float by, float hl, float hw) {
    const float dx = xs(o.cx, fcx), dy = xs(o.cy, fcy);
    float rO = xa(xm(fabsf(xdot2(o.ux, o.uy, ax, ay)), o.su), xm(fabsf(xdot2(o.vx, o.vy, ax, ay)), o.sv));
    if (fabsf(xdot2(dx, dy, ax, ay)) >= xa(hl, rO)) return false;
    rO = xa(xm(fabsf(xdot2(o.ux, o.uy, bx, by)), o.su), xm(fabsf(xdot2(o.vx, o.vy, bx, by)), o.sv));
    if (fabsf(xdot2(dx, dy, bx, by)) >= xa(hw, rO)) return false;
    float rF = xa(xm(fabsf(xdot2(ax, ay, o.ux, o.uy)), hl), xm(fabsf(xdot2(bx, by, o.ux, o.uy)), hw));
    if (fabsf(xdot2(dx, dy, o.ux, o.uy)) >= xa(rF, o.su)) return false;
    rF = xa(xm(fabsf(xdot2(ax, ay, o.vx, o.vy)), hl), xm(fabsf(xdot2(bx, by, o.vx, o.vy)), hw));
    if (fabsf(xdot2(dx, dy, o.vx, o.vy)) >= xa(rF, o.sv)) return false;
    return true;
}

// Pusher disc of radius r at (px, py) intersects footprint o.
__device__ __forceinline__ bool disc_hits_foot_exact(const Foot& o, float px, float py, float r) {
    const float ex = xs(px, o.cx), ey = xs(py, o.cy);
    float pu = xs(fabsf(xdot2(ex, ey, o.ux, o.uy)), o.su);
    float pv = xs(fabsf(xdot2(ex, ey, o.vx, o.vy)), o.sv);
    pu = pu > 0.f ? pu : 0.f;
    pv = pv > 0.f ? pv : 0.f;
    return xa(xm(pu, pu), xm(pv, pv)) < xm(r, r);
}

// SplitMix64 (Steele, Lea & Flood 2014): advance the state by the golden gamma and
// finalise with the variant-13 mixer.
__device__ __forceinline__ uint64_t splitmix64(uint64_t& s) {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Index in [0, count) from the top 32 bits by multiply-shift.
__device__ __forceinline__ int draw_index(uint64_t r, int count) {
    return (int)(((r >> 32) * (uint64_t)count) >> 32);
}

// Keyed draws of attempt a of push k: object j and contour point p.
__device__ __forceinline__ void sampler_draws(uint64_t seed, int k, int a, int n, int npts, int& j, int& p) {
    uint64_t st = seed ^ (((uint64_t)(uint32_t)k << 32) | (uint64_t)(uint32_t)a);
    const uint64_t r1 = splitmix64(st);
    const uint64_t r2 = splitmix64(st);
    j = draw_index(r1, n);
    p = draw_index(r2, npts);
}

// Contour point p of npts spaced evenly by arc length around footprint f grown by
// (r + clear), counter-clockwise from (+A, 0) in the (u, v) frame; the push runs from it
// toward the footprint centre for length L.  out = (x_s, y_s, x_e, y_e).
__device__ __forceinline__ void contour_push_exact(const Foot& f, int p, int npts, float r, float clear,
                                                   float L, float* out) {
    const float A = xa(xa(f.su, r), clear), B = xa(xa(f.sv, r), clear);
    const float A2 = xm(A, 2.f), B2 = xm(B, 2.f);
    const float per = xm(xa(A, B), 4.f);
    float ell = xd(xm(per, (float)p), (float)npts);
    float lu, lv;
    if (ell < B) {
        lu = A;
        lv = ell;
    } else {
        ell = xs(ell, B);
        if (ell < A2) {
            lu = xs(A, ell);
            lv = B;
        } else {
            ell = xs(ell, A2);
            if (ell < B2) {
                lu = -A;
                lv = xs(B, ell);
            } else {
                ell = xs(ell, B2);
                if (ell < A2) {
                    lu = xs(ell, A);
                    lv = -B;
                } else {
                    ell = xs(ell, A2);
                    lu = A;
                    lv = xs(ell, B);
                }
            }
        }
    }
    const float px = xa(xa(f.cx, xm(lu, f.ux)), xm(lv, f.vx));
    const float py = xa(xa(f.cy, xm(lu, f.uy)), xm(lv, f.vy));
    const float dx = xs(f.cx, px), dy = xs(f.cy, py);
    const float len = xsqrt(xdot2(dx, dy, dx, dy));
    const float dirx = xd(dx, len), diry = xd(dy, len);
    out[0] = px;
    out[1] = py;
    out[2] = xa(px, xm(dirx, L));
    out[3] = xa(py, xm(diry, L));
}

}  // namespace pmbs

// Narrowphase of the rollout engine (FP32, one lane per candidate pair).
//
// The paper specifies the transition only as rigid-body motion with friction and
// collisions (Sec. III-A, transition function); the contact model below is this
// library's reading: box-plane vertex contacts, box-box separating-axis test over 15 axes
// with reference-face clipping (at most four points) or one edge-edge point, and a
// capsule pusher against a box by closest points at the ends of the overlapping height
// range; cylinders (16-gon prisms) take the general convex form of the same rules.
// Separation d < 0 means penetration; contacts are kept while d < margin.
#pragma once
#include <cstdint>

#include "pmbs_exact.cuh"

namespace pmbs {

__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator-(float3 a) { return f3(-a.x, -a.y, -a.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float norm3(float3 a) { return sqrtf(dot3(a, a)); }

// A box (or cylinder) for collision: centre, row-major rotation (columns = axes), half
// extents; a cylinder has cyl set and h = (r, r, half height).
struct CBox {
    float3 c;
    float R[9];
    float h[3];
    bool cyl;
    __device__ __forceinline__ float3 ax(int k) const { return f3(R[k], R[3 + k], R[6 + k]); }
    // runtime index through selects (keeps the box in registers)
    __device__ __forceinline__ float3 axs(int k) const { return k == 0 ? ax(0) : (k == 1 ? ax(1) : ax(2)); }
    __device__ __forceinline__ float hs(int k) const { return k == 0 ? h[0] : (k == 1 ? h[1] : h[2]); }
    __device__ __forceinline__ float3 rot(float3 l) const {
        return f3(R[0] * l.x + R[1] * l.y + R[2] * l.z, R[3] * l.x + R[4] * l.y + R[5] * l.z,
                  R[6] * l.x + R[7] * l.y + R[8] * l.z);
    }
};

// Contact points produced for one candidate: point p (world), separation d; all points
// share one normal n, from body A to body B.
struct CManifold {
    int np;
    float3 n;
    float3 p[4];
    float d[4];
};

// Box against plane z = 0 (A = plane, B = box): vertices below the margin, deepest
// first with ties by vertex index, at most four.  Contact offsets from the box centre
// are returned in p (the world point is c + p).
__device__ __forceinline__ void collide_box_plane(const CBox& b, float margin, CManifold& M) {
    M.np = 0;
    M.n = f3(0.f, 0.f, 1.f);
    // kept rolled: the substep body is larger than an SM's instruction cache, and the
    // rolled loop (8.7 KB less code) runs faster than the unrolled one
#pragma unroll 1
    for (int v = 0; v < 8; v++) {
        const float3 l = f3((v & 1) ? b.h[0] : -b.h[0], (v & 2) ? b.h[1] : -b.h[1], (v & 4) ? b.h[2] : -b.h[2]);
        float3 r = b.rot(l);
        float d = b.c.z + r.z;
        if (!(d < margin)) continue;
        // insertion into the depth-sorted list (stable: equal depths keep vertex order):
        // the new entry goes before the first strictly shallower one, every later entry
        // moves down one slot, and an entry pushed past the fourth slot is dropped
        bool shift = false;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (k < M.np) {
                if (shift || d < M.d[k]) {
                    shift = true;
                    const float td = M.d[k];
                    const float3 tp = M.p[k];
                    M.d[k] = d;
                    M.p[k] = r;
                    d = td;
                    r = tp;
                }
            } else if (k == M.np) {
                M.d[k] = d;
                M.p[k] = r;
            }
        }
        if (M.np < 4) M.np++;
    }
}

// Sutherland-Hodgman clip of poly (n points) against dot(p - o, a) - h <= 0.  A convex
// quad clipped four times has at most eight vertices; rounding on degenerate faces could
// produce more, and vertices beyond the eighth are dropped.
__device__ __forceinline__ int clip_side(const float3* in, int n, float3* out, float3 o, float3 a, float h) {
    int m = 0;
    if (n <= 0) return 0;
    // the previous vertex and its signed distance carried from the last iteration
    float3 prev = in[n - 1];
    float dp = dot3(prev - o, a) - h;
    for (int i = 0; i < n; i++) {
        const float3 cur = in[i];
        const float dc = dot3(cur - o, a) - h;
        if (dc <= 0.f) {
            if (dp > 0.f && m < 8) out[m++] = prev + (cur - prev) * __fdividef(dp, dp - dc);
            if (m < 8) out[m++] = cur;
        } else if (dp <= 0.f) {
            if (m < 8) out[m++] = prev + (cur - prev) * __fdividef(dp, dp - dc);
        }
        prev = cur;
        dp = dc;
    }
    return m;
}

// Clip the incident face of `inc` against the side planes of face k (outward normal
// nref) of `ref`; keep points within the margin; reduce to four points.  Returns the
// number of points in M (p = world point, d = separation from the reference face).
// Box axes and extents are picked by selects so that both boxes stay in registers; only
// the clip polygons live in per-thread memory.
__device__ __forceinline__ int face_contact(const CBox& ref, int k, float3 nref, const CBox& inc, float margin,
                                            CManifold& M, int& clip_verts) {
    const float3 fc = ref.c + nref * ref.hs(k);
    const int k1 = (k == 0) ? 1 : 0, k2 = (k == 2) ? 1 : 2;
    const float3 u = ref.axs(k1), v = ref.axs(k2);
    const float hu = ref.hs(k1), hv = ref.hs(k2);
    int best_f = 0;
    float best = 0.f;
#pragma unroll
    for (int m = 0; m < 3; m++) {
        const float dm = dot3(inc.ax(m), nref);
        if (m == 0 || dm < best) {
            best = dm;
            best_f = 2 * m;
        }
        if (-dm < best) {
            best = -dm;
            best_f = 2 * m + 1;
        }
    }
    const int mi = best_f >> 1;
    const float si = (best_f & 1) ? -1.f : 1.f;
    const int m1 = (mi == 0) ? 1 : 0, m2 = (mi == 2) ? 1 : 2;
    const float3 fi = inc.c + inc.axs(mi) * (si * inc.hs(mi));
    const float3 e1 = inc.axs(m1) * inc.hs(m1), e2 = inc.axs(m2) * inc.hs(m2);
    float3 P[2][8];
    P[0][0] = fi + e1 + e2;
    P[0][1] = fi - e1 + e2;
    P[0][2] = fi - e1 - e2;
    P[0][3] = fi + e1 - e2;
    int n = 4;
    // sides +u, -u, +v, -v; the polygon alternates between the two buffers and ends in P[0]
#pragma unroll 1
    for (int side = 0; side < 4; side++) {
        const float3 a = side < 2 ? u : v;
        n = clip_side(P[side & 1], n, P[(side & 1) ^ 1], fc, (side & 1) ? -a : a, side < 2 ? hu : hv);
    }
    clip_verts += n;
    float3* B = P[1];
    float kd[8];
    int nk = 0;
    for (int i = 0; i < n; i++) {
        const float d = dot3(P[0][i] - fc, nref);
        if (d < margin) {
            B[nk] = P[0][i];
            kd[nk] = d;
            nk++;
        }
    }
    if (nk <= 4) {
#pragma unroll
        for (int i = 0; i < 4; i++)
            if (i < nk) {
                M.p[i] = B[i];
                M.d[i] = kd[i];
            }
        return nk;
    }
    // deepest; farthest from it; largest triangle; largest area added outside an edge
    unsigned used = 0;
    int i1 = 0;
    for (int i = 1; i < nk; i++)
        if (kd[i] < kd[i1]) i1 = i;
    used |= 1u << i1;
    int i2 = -1;
    float b2 = -1.f;
    for (int i = 0; i < nk; i++) {
        if (used >> i & 1u) continue;
        const float3 e = B[i] - B[i1];
        const float l = dot3(e, e);
        if (i2 < 0 || l > b2) {
            b2 = l;
            i2 = i;
        }
    }
    used |= 1u << i2;
    int i3 = -1;
    float b3 = -1.f;
    for (int i = 0; i < nk; i++) {
        if (used >> i & 1u) continue;
        const float a = fabsf(dot3(cross3(B[i2] - B[i1], B[i] - B[i1]), nref));
        if (i3 < 0 || a > b3) {
            b3 = a;
            i3 = i;
        }
    }
    used |= 1u << i3;
    const float sgn = dot3(cross3(B[i2] - B[i1], B[i3] - B[i1]), nref) < 0.f ? -1.f : 1.f;
    int i4 = -1;
    float b4 = 0.f;
    for (int i = 0; i < nk; i++) {
        if (used >> i & 1u) continue;
        float a = -sgn * dot3(cross3(B[i2] - B[i1], B[i] - B[i1]), nref);
        a = fmaxf(a, -sgn * dot3(cross3(B[i3] - B[i2], B[i] - B[i2]), nref));
        a = fmaxf(a, -sgn * dot3(cross3(B[i1] - B[i3], B[i] - B[i3]), nref));
        if (i4 < 0 || a > b4) {
            b4 = a;
            i4 = i;
        }
    }
    M.p[0] = B[i1];
    M.d[0] = kd[i1];
    M.p[1] = B[i2];
    M.d[1] = kd[i2];
    M.p[2] = B[i3];
    M.d[2] = kd[i3];
    M.p[3] = B[i4];
    M.d[3] = kd[i4];
    return 4;
}

// Box-box contact (A = lower index).  Separating axes: 3 faces of A, 3 of B, 9 edge
// crosses (skipped when |cross|^2 < 1e-12).  Any separation >= margin: no contact.  A
// face of B replaces A's best face only when its separation is larger by > 1e-5 m; an
// edge axis replaces the face only when larger by > 1e-4 m + 5% |face separation|;
// earliest axis wins exact ties.  Normal from A to B.  kind: 0 none, 1 face, 2 edge.
__device__ __forceinline__ int collide_box_box(const CBox& A, const CBox& B, float margin, CManifold& M,
                                               int& clip_verts) {
    M.np = 0;
    const float3 D = B.c - A.c;
    float3 a[3] = {A.ax(0), A.ax(1), A.ax(2)};
    float3 b[3] = {B.ax(0), B.ax(1), B.ax(2)};
    float aC[3][3];
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int m = 0; m < 3; m++) aC[k][m] = fabsf(dot3(a[k], b[m]));
    int fa = -1;
    float sa = 0.f;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const float s = fabsf(dot3(D, a[k])) - (A.h[k] + (B.h[0] * aC[k][0] + B.h[1] * aC[k][1] + B.h[2] * aC[k][2]));
        if (s >= margin) return 0;
        if (fa < 0 || s > sa) {
            fa = k;
            sa = s;
        }
    }
    int fb = -1;
    float sb = 0.f;
#pragma unroll
    for (int m = 0; m < 3; m++) {
        const float s = fabsf(dot3(D, b[m])) - ((A.h[0] * aC[0][m] + A.h[1] * aC[1][m] + A.h[2] * aC[2][m]) + B.h[m]);
        if (s >= margin) return 0;
        if (fb < 0 || s > sb) {
            fb = m;
            sb = s;
        }
    }
    int fe = -1;
    float se = 0.f;
    float3 le = f3(0.f, 0.f, 0.f);
    // the nine edge axes in one rolled loop (instruction-cache footprint, as above)
#pragma unroll 1
    for (int ij = 0; ij < 9; ij++) {
        const int i = ij / 3, j = ij - 3 * (ij / 3);
        const float3 ai = i == 0 ? a[0] : (i == 1 ? a[1] : a[2]);
        const float3 bj = j == 0 ? b[0] : (j == 1 ? b[1] : b[2]);
        const float3 L = cross3(ai, bj);
        const float l2 = dot3(L, L);
        if (l2 < 1e-12f) continue;
        const float inv = rsqrtf(l2);
        const float rA = (A.h[0] * fabsf(dot3(a[0], L)) + A.h[1] * fabsf(dot3(a[1], L))) + A.h[2] * fabsf(dot3(a[2], L));
        const float rB = (B.h[0] * fabsf(dot3(b[0], L)) + B.h[1] * fabsf(dot3(b[1], L))) + B.h[2] * fabsf(dot3(b[2], L));
        const float s = (fabsf(dot3(D, L)) - (rA + rB)) * inv;
        if (s >= margin) return 0;
        if (fe < 0 || s > se) {
            fe = 6 + 3 * i + j;
            se = s;
            le = L * inv;
        }
    }
    int axis = fa;
    float s = sa;
    float3 L = A.axs(fa);
    if (sb > sa + 1e-5f) {
        axis = 3 + fb;
        s = sb;
        L = B.axs(fb);
    }
    if (fe >= 0 && se > s + 1e-4f + 0.05f * fabsf(s)) {
        axis = fe;
        s = se;
        L = le;
    }
    if (dot3(L, D) < 0.f) L = -L;
    M.n = L;
    if (axis < 6) {
        // one clipping routine for both reference boxes
        const bool ar = axis < 3;
        const CBox ref = ar ? A : B, inc = ar ? B : A;
        M.np = face_contact(ref, ar ? axis : axis - 3, ar ? L : -L, inc, margin, M, clip_verts);
        return M.np ? 1 : 0;
    }
    const int ea = (axis - 6) / 3, eb = (axis - 6) % 3;
    float3 pA = A.c, pB = B.c;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        if (k == ea) continue;
        const float sg = dot3(a[k], L) < 0.f ? -1.f : 1.f;
        pA = pA + a[k] * (sg * A.h[k]);
    }
#pragma unroll
    for (int m = 0; m < 3; m++) {
        if (m == eb) continue;
        const float sg = dot3(b[m], L) > 0.f ? -1.f : 1.f;
        pB = pB + b[m] * (sg * B.h[m]);
    }
    const float3 dA = A.axs(ea), dB = B.axs(eb);
    const float3 r = pA - pB;
    const float bb = dot3(dA, dB), c = dot3(dA, r), f = dot3(dB, r);
    const float den = 1.f - bb * bb;
    float ta = 0.f, tb;
    if (den > 1e-12f) {
        ta = (bb * f - c) / den;
        tb = f + ta * bb;
    } else {
        tb = f;
    }
    const float ha = A.hs(ea), hb = B.hs(eb);
    ta = fminf(fmaxf(ta, -ha), ha);
    tb = fminf(fmaxf(tb, -hb), hb);
    const float3 qa = pA + dA * ta, qb = pB + dB * tb;
    M.p[0] = (qa + qb) * 0.5f;
    M.d[0] = s;
    M.np = 1;
    return 2;
}

// Vertical capsule (axis through (px, py), z in [z0, z1], radius r) against a box (A =
// box, B = pusher).  The segment is clipped to the box's vertical extent; each end of
// the clipped range (its middle when shorter than 1 mm; the nearer segment end when the
// ranges do not meet) yields the closest box point.  Normal (box to pusher) of the
// nearest candidate.  p = point on the box (world).
__device__ __forceinline__ void collide_capsule_box(const CBox& b, float px, float py, float z0, float z1, float r,
                                                    float margin, CManifold& M) {
    M.np = 0;
    const float ez = (fabsf(b.R[6]) * b.h[0] + fabsf(b.R[7]) * b.h[1]) + fabsf(b.R[8]) * b.h[2];
    const float zlo = b.c.z - ez, zhi = b.c.z + ez;
    const float za = fmaxf(z0, zlo), zb = fminf(z1, zhi);
    float zc0, zc1 = 0.f;
    int nc;
    if (za > zb) {
        zc0 = (zhi < z0) ? z0 : z1;
        nc = 1;
    } else if (zb - za < 1e-3f) {
        zc0 = (za + zb) * 0.5f;
        nc = 1;
    } else {
        zc0 = za;
        zc1 = zb;
        nc = 2;
    }
    float best_d = 0.f;
    float3 best_n = f3(1.f, 0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 2; i++) {
        if (i >= nc) break;
        const float3 S = f3(px, py, i == 0 ? zc0 : zc1);
        const float3 rel = S - b.c;
        float loc[3], ql[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            loc[k] = dot3(b.ax(k), rel);
            ql[k] = fminf(fmaxf(loc[k], -b.h[k]), b.h[k]);
        }
        const float3 Q = b.c + b.ax(0) * ql[0] + b.ax(1) * ql[1] + b.ax(2) * ql[2];
        const float3 diff = S - Q;
        const float dist = norm3(diff);
        float3 nrm;
        float d;
        if (dist > 1e-6f) {
            nrm = diff * (1.f / dist);
            d = dist - r;
        } else {
            float pen = b.h[0] - fabsf(loc[0]);
            pen = fminf(pen, b.h[1] - fabsf(loc[1]));
            pen = fminf(pen, b.h[2] - fabsf(loc[2]));
            d = -pen - r;
            const float3 w = f3(S.x - b.c.x, S.y - b.c.y, 0.f);
            const float lw = norm3(w);
            nrm = lw > 1e-9f ? w * (1.f / lw) : f3(1.f, 0.f, 0.f);
        }
        if (!(d < margin)) continue;
        if (M.np == 0) {
            M.p[0] = Q;
            M.d[0] = d;
        } else {
            M.p[1] = Q;
            M.d[1] = d;
        }
        if (M.np == 0 || d < best_d) {
            best_d = d;
            best_n = nrm;
        }
        M.np++;
    }
    M.n = best_n;
}

// ------------------------------------------------------------------ cylinders
// The loops over the 16 cap vertices or side faces stay rolled: unrolled, they make the
// cylinder instantiation's code larger than the instruction cache holds (measured
// slower).
//
// Pairs with a cylinder (a 16-gon prism, see pmbs_exact.cuh) take the general
// separating-axis test of two convex polyhedra: face normal directions of A (box: its 3
// axes; cylinder: its cap axis, then the 8 side normal directions), those of B, and the
// cross products of an edge direction of A with one of B (box: its 3 axes; cylinder: its
// axis, then the 8 cap edge directions; skipped when |cross|^2 < 1e-12).  Separation along
// a unit axis is |L.D| minus both support half widths; the selection thresholds are the
// box-box test's.  A face axis clips the other body's incident face (most anti-parallel
// outward normal) against the reference face's side planes (at most 32 vertices) and
// reduces to four points; an edge axis gives one point midway between the closest points
// of the two supporting edges.

__device__ __forceinline__ void gon_vdir(int k, float& c, float& s) {
    const float g = k < 8 ? 1.f : -1.f;
    c = g * kGonC[k & 7];
    s = g * kGonS[k & 7];
}
__device__ __forceinline__ void gon_fdir(int k, float& c, float& s) {
    const float g = k < 8 ? 1.f : -1.f;
    c = g * kGonFC[k & 7];
    s = g * kGonFS[k & 7];
}
__device__ __forceinline__ float3 plane_vec(const CBox& b, float c, float s) { return b.ax(0) * c + b.ax(1) * s; }
__device__ __forceinline__ float3 side_normal(const CBox& b, int k) {
    float c, s;
    gon_fdir(k, c, s);
    return plane_vec(b, c, s);
}
__device__ __forceinline__ float3 side_tangent(const CBox& b, int k) {
    float c, s;
    gon_fdir(k, c, s);
    return plane_vec(b, -s, c);
}
__device__ __forceinline__ float3 cyl_vertex(const CBox& b, int k, float sz) {
    float c, s;
    gon_vdir(k & 15, c, s);
    return b.c + plane_vec(b, c * b.h[0], s * b.h[0]) + b.ax(2) * (sz * b.h[2]);
}
// Radial support of the unit 16-gon along (p0, p1): the largest |c_k p0 + s_k p1| over
// the vertex directions.  By the 16-gon's symmetry, with a >= b the magnitudes of the
// components, it is the largest of a, cos(pi/8) a + sin(pi/8) b and (a + b) / sqrt 2 --
// the vertex directions 0, pi/8 and pi/4 that bracket the first octant.
__device__ __forceinline__ float gon_sup(float p0, float p1) {
    const float u = fabsf(p0), v = fabsf(p1);
    const float a = fmaxf(u, v), b = fminf(u, v);
    return fmaxf(a, fmaxf(0.923879504f * a + 0.382683426f * b, 0.707106769f * a + 0.707106769f * b));
}
__device__ __forceinline__ float support(const CBox& b, float3 L) {
    if (b.cyl) return gon_sup(dot3(b.ax(0), L), dot3(b.ax(1), L)) * b.h[0] + fabsf(dot3(b.ax(2), L)) * b.h[2];
    return (b.h[0] * fabsf(dot3(b.ax(0), L)) + b.h[1] * fabsf(dot3(b.ax(1), L))) + b.h[2] * fabsf(dot3(b.ax(2), L));
}
__device__ __forceinline__ int n_dirs(const CBox& b) { return b.cyl ? 9 : 3; }
__device__ __forceinline__ float3 face_dir(const CBox& b, int f) {
    return !b.cyl ? b.axs(f) : (f == 0 ? b.ax(2) : side_normal(b, f - 1));
}
__device__ __forceinline__ float face_half(const CBox& b, int f) {
    return !b.cyl ? b.hs(f) : (f == 0 ? b.h[2] : b.h[0] * kGonApo);
}
__device__ __forceinline__ float3 edge_dir(const CBox& b, int j) {
    return !b.cyl ? b.axs(j) : (j == 0 ? b.ax(2) : side_tangent(b, j - 1));
}

// At most four of nk candidate points B (separations kd, normal nref): all when nk <= 4;
// else the deepest (earliest on ties), the farthest from it, the one spanning the largest
// triangle with those two, the one adding the largest area outside an edge.
__device__ __forceinline__ int reduce_points(const float3* B, const float* kd, int nk, float3 nref, CManifold& M) {
    if (nk <= 4) {
        for (int i = 0; i < nk; i++) {
            M.p[i] = B[i];
            M.d[i] = kd[i];
        }
        return nk;
    }
    unsigned used = 0;
    int i1 = 0;
    for (int i = 1; i < nk; i++)
        if (kd[i] < kd[i1]) i1 = i;
    used |= 1u << i1;
    int i2 = -1;
    float b2 = -1.f;
    for (int i = 0; i < nk; i++) {
        if (used >> i & 1u) continue;
        const float3 e = B[i] - B[i1];
        const float l = dot3(e, e);
        if (i2 < 0 || l > b2) {
            b2 = l;
            i2 = i;
        }
    }
    used |= 1u << i2;
    int i3 = -1;
    float b3 = -1.f;
    for (int i = 0; i < nk; i++) {
        if (used >> i & 1u) continue;
        const float a = fabsf(dot3(cross3(B[i2] - B[i1], B[i] - B[i1]), nref));
        if (i3 < 0 || a > b3) {
            b3 = a;
            i3 = i;
        }
    }
    used |= 1u << i3;
    const float sgn = dot3(cross3(B[i2] - B[i1], B[i3] - B[i1]), nref) < 0.f ? -1.f : 1.f;
    int i4 = -1;
    float b4 = 0.f;
    for (int i = 0; i < nk; i++) {
        if (used >> i & 1u) continue;
        float a = -sgn * dot3(cross3(B[i2] - B[i1], B[i] - B[i1]), nref);
        a = fmaxf(a, -sgn * dot3(cross3(B[i3] - B[i2], B[i] - B[i2]), nref));
        a = fmaxf(a, -sgn * dot3(cross3(B[i1] - B[i3], B[i] - B[i3]), nref));
        if (i4 < 0 || a > b4) {
            b4 = a;
            i4 = i;
        }
    }
    M.p[0] = B[i1];
    M.d[0] = kd[i1];
    M.p[1] = B[i2];
    M.d[1] = kd[i2];
    M.p[2] = B[i3];
    M.d[2] = kd[i3];
    M.p[3] = B[i4];
    M.d[3] = kd[i4];
    return 4;
}

// Sutherland-Hodgman clip against dot(p - o, a) - h <= 0, at most 32 vertices kept.
__device__ __forceinline__ int clip_side32(const float3* in, int n, float3* out, float3 o, float3 a, float h) {
    int m = 0;
    if (n <= 0) return 0;
    // the previous vertex and its signed distance carried from the last iteration
    float3 prev = in[n - 1];
    float dp = dot3(prev - o, a) - h;
    for (int i = 0; i < n; i++) {
        const float3 cur = in[i];
        const float dc = dot3(cur - o, a) - h;
        if (dc <= 0.f) {
            if (dp > 0.f && m < 32) out[m++] = prev + (cur - prev) * __fdividef(dp, dp - dc);
            if (m < 32) out[m++] = cur;
        } else if (dp <= 0.f) {
            if (m < 32) out[m++] = prev + (cur - prev) * __fdividef(dp, dp - dc);
        }
        prev = cur;
        dp = dc;
    }
    return m;
}

// Face contact between convex bodies: reference face f of ref (outward normal nref).
__device__ __forceinline__ int face_contact_convex(const CBox& ref, int f, float3 nref, const CBox& inc, float margin,
                                                CManifold& M, int& clip_verts) {
    // reference face: centre and side planes (origin fc)
    float3 fc;
    int nside, rs = 0;
    if (!ref.cyl) {
        fc = ref.c + nref * ref.hs(f);
        nside = 4;
    } else if (f == 0) {
        fc = ref.c + nref * ref.h[2];
        nside = 16;
    } else {
        rs = dot3(side_normal(ref, f - 1), nref) > 0.f ? f - 1 : f + 7;
        fc = ref.c + nref * (ref.h[0] * kGonApo);
        nside = 4;
    }
    float3 P[2][32];
    int n;
    if (!inc.cyl) {
        int best_f = 0;
        float best = 0.f;
        for (int m = 0; m < 3; m++) {
            const float dm = dot3(inc.axs(m), nref);
            if (m == 0 || dm < best) {
                best = dm;
                best_f = 2 * m;
            }
            if (-dm < best) {
                best = -dm;
                best_f = 2 * m + 1;
            }
        }
        const int mi = best_f >> 1;
        const float si = (best_f & 1) ? -1.f : 1.f;
        const int m1 = (mi == 0) ? 1 : 0, m2 = (mi == 2) ? 1 : 2;
        const float3 fi = inc.c + inc.axs(mi) * (si * inc.hs(mi));
        const float3 e1 = inc.axs(m1) * inc.hs(m1), e2 = inc.axs(m2) * inc.hs(m2);
        P[0][0] = fi + e1 + e2;
        P[0][1] = fi - e1 + e2;
        P[0][2] = fi - e1 - e2;
        P[0][3] = fi + e1 - e2;
        n = 4;
    } else {
        // candidates: top cap, bottom cap, sides 0..15
        const float dz = dot3(inc.ax(2), nref);
        int best_c = 0;
        float best = dz;
        if (-dz < best) {
            best = -dz;
            best_c = 1;
        }
        #pragma unroll 1
        for (int k = 0; k < 16; k++) {
            const float dm = dot3(side_normal(inc, k), nref);
            if (dm < best) {
                best = dm;
                best_c = 2 + k;
            }
        }
        if (best_c < 2) {
            const float sz = best_c == 0 ? 1.f : -1.f;
            #pragma unroll 1
            for (int k = 0; k < 16; k++) P[0][k] = cyl_vertex(inc, k, sz);
            n = 16;
        } else {
            const int k = best_c - 2;
            P[0][0] = cyl_vertex(inc, k, 1.f);
            P[0][1] = cyl_vertex(inc, k + 1, 1.f);
            P[0][2] = cyl_vertex(inc, k + 1, -1.f);
            P[0][3] = cyl_vertex(inc, k, -1.f);
            n = 4;
        }
    }
    // the polygon alternates between the two buffers; an even number of sides ends in P[0]
    for (int i = 0; i < nside; i++) {
        float3 a;
        float h;
        if (!ref.cyl) {
            const int k1 = (f == 0) ? 1 : 0, k2 = (f == 2) ? 1 : 2;
            const int kk = i < 2 ? k1 : k2;
            a = (i & 1) ? -ref.axs(kk) : ref.axs(kk);
            h = ref.hs(kk);
        } else if (f == 0) {
            a = side_normal(ref, i);
            h = ref.h[0] * kGonApo;
        } else {
            const float3 base = i < 2 ? ref.ax(2) : side_tangent(ref, rs);
            a = (i & 1) ? -base : base;
            h = i < 2 ? ref.h[2] : ref.h[0] * kGonHalfEdge;
        }
        n = clip_side32(P[i & 1], n, P[(i & 1) ^ 1], fc, a, h);
    }
    clip_verts += n;
    float kd[32];
    int nk = 0;
    for (int i = 0; i < n; i++) {
        const float d = dot3(P[0][i] - fc, nref);
        if (d < margin) {
            P[1][nk] = P[0][i];
            kd[nk] = d;
            nk++;
        }
    }
    return reduce_points(P[1], kd, nk, nref, M);
}

// Supporting edge of direction index j of b toward L: centre, direction, half length.
__device__ __forceinline__ void support_edge(const CBox& b, int j, float3 L, float3& c, float3& d, float& hl) {
    if (!b.cyl) {
        c = b.c;
        for (int k = 0; k < 3; k++) {
            if (k == j) continue;
            const float sg = dot3(b.axs(k), L) < 0.f ? -1.f : 1.f;
            c = c + b.axs(k) * (sg * b.hs(k));
        }
        d = b.axs(j);
        hl = b.hs(j);
    } else if (j == 0) {
        int kb = 0;
        float best = 0.f;
        #pragma unroll 1
        for (int k = 0; k < 16; k++) {
            float vc, vs;
            gon_vdir(k, vc, vs);
            const float v = dot3(plane_vec(b, vc, vs), L);
            if (k == 0 || v > best) {
                best = v;
                kb = k;
            }
        }
        c = cyl_vertex(b, kb, 0.f);
        d = b.ax(2);
        hl = b.h[2];
    } else {
        const int s = dot3(side_normal(b, j - 1), L) >= 0.f ? j - 1 : j + 7;
        const float sz = dot3(b.ax(2), L) >= 0.f ? 1.f : -1.f;
        c = b.c + side_normal(b, s) * (b.h[0] * kGonApo) + b.ax(2) * (sz * b.h[2]);
        d = side_tangent(b, s);
        hl = b.h[0] * kGonHalfEdge;
    }
}

// Convex pair with a cylinder (A = lower index).  Returns 0 none, 1 face, 2 edge; the
// separation of the chosen axis in *sep_out when given.
__device__ __forceinline__ int collide_convex(const CBox& A, const CBox& B, float margin, CManifold& M, int& clip_verts,
                                           float* sep_out = nullptr) {
    M.np = 0;
    const float3 D = B.c - A.c;
    int fa = -1;
    float sa = 0.f;
    for (int f = 0; f < n_dirs(A); f++) {
        const float3 L = face_dir(A, f);
        const float s = fabsf(dot3(D, L)) - (face_half(A, f) + support(B, L));
        if (s >= margin) return 0;
        if (fa < 0 || s > sa) {
            fa = f;
            sa = s;
        }
    }
    int fb = -1;
    float sb = 0.f;
    for (int f = 0; f < n_dirs(B); f++) {
        const float3 L = face_dir(B, f);
        const float s = fabsf(dot3(D, L)) - (support(A, L) + face_half(B, f));
        if (s >= margin) return 0;
        if (fb < 0 || s > sb) {
            fb = f;
            sb = s;
        }
    }
    int ea = -1, eb = -1;
    float se = 0.f;
    float3 le = f3(0.f, 0.f, 0.f);
    for (int i = 0; i < n_dirs(A); i++) {
        const float3 dA = edge_dir(A, i);
        for (int j = 0; j < n_dirs(B); j++) {
            const float3 L = cross3(dA, edge_dir(B, j));
            const float l2 = dot3(L, L);
            if (l2 < 1e-12f) continue;
            const float3 u = L * rsqrtf(l2);
            const float s = fabsf(dot3(D, u)) - (support(A, u) + support(B, u));
            if (s >= margin) return 0;
            if (ea < 0 || s > se) {
                ea = i;
                eb = j;
                se = s;
                le = u;
            }
        }
    }
    int kind = 0, fi = fa;
    float s = sa;
    float3 L = face_dir(A, fa);
    if (sb > sa + 1e-5f) {
        kind = 1;
        fi = fb;
        s = sb;
        L = face_dir(B, fb);
    }
    if (ea >= 0 && se > s + 1e-4f + 0.05f * fabsf(s)) {
        kind = 2;
        s = se;
        L = le;
    }
    if (dot3(L, D) < 0.f) L = -L;
    M.n = L;
    if (sep_out) *sep_out = s;
    if (kind < 2) {
        const bool ar = kind == 0;
        M.np = face_contact_convex(ar ? A : B, fi, ar ? L : -L, ar ? B : A, margin, M, clip_verts);
        return M.np ? 1 : 0;
    }
    float3 pA, pB, dA, dB;
    float ha, hb;
    support_edge(A, ea, L, pA, dA, ha);
    support_edge(B, eb, -L, pB, dB, hb);
    const float3 r = pA - pB;
    const float bb = dot3(dA, dB), c = dot3(dA, r), f = dot3(dB, r);
    const float den = 1.f - bb * bb;
    float ta = 0.f, tb;
    if (den > 1e-12f) {
        ta = (bb * f - c) / den;
        tb = f + ta * bb;
    } else {
        tb = f;
    }
    ta = fminf(fmaxf(ta, -ha), ha);
    tb = fminf(fmaxf(tb, -hb), hb);
    const float3 qa = pA + dA * ta, qb = pB + dB * tb;
    M.p[0] = (qa + qb) * 0.5f;
    M.d[0] = s;
    M.np = 1;
    return 2;
}

// Offset from the centre of a cylinder's vertex v (v < 16: bottom cap vertex v, else top
// cap vertex v - 16).
__device__ __forceinline__ float3 cyl_offset(const CBox& b, int v) {
    float c, s;
    gon_vdir(v & 15, c, s);
    return plane_vec(b, c * b.h[0], s * b.h[0]) + b.ax(2) * ((v < 16 ? -1.f : 1.f) * b.h[2]);
}

// Cylinder against the plane z = 0 (A = plane, B = cylinder): its 32 vertices (bottom cap
// k = 0..15, then top) below the margin; four or fewer kept deepest first (ties by vertex
// index), more reduced to four as for face contacts (normal +z, so the areas are the z
// components of the cross products).  p = offset from the centre.  The candidates are a
// bit mask and every vertex is recomputed when needed, so nothing leaves registers; a cap
// whose lowest vertex is clear of the margin by more than 1e-6 m (far beyond the
// rounding of that bound) is skipped.  Loops run over vertex indices uniformly across the
// warp, so the direction-table reads are broadcasts.
__device__ __forceinline__ void collide_cyl_plane(const CBox& b, float margin, CManifold& M) {
    M.np = 0;
    M.n = f3(0.f, 0.f, 1.f);
    const float rad = gon_sup(b.R[6], b.R[7]) * b.h[0], ax = b.R[8] * b.h[2];
    const bool bot = b.c.z - ax - rad < margin + 1e-6f, top = b.c.z + ax - rad < margin + 1e-6f;
    const int v0 = bot ? 0 : 16, v1 = top ? 32 : 16;
    unsigned cand = 0u;
    int nk = 0, i1 = -1;
    float d1 = 0.f;
    for (int v = v0; v < v1; v++) {
        const float d = b.c.z + cyl_offset(b, v).z;
        if (d < margin) {
            cand |= 1u << v;
            nk++;
            if (i1 < 0 || d < d1) {
                d1 = d;
                i1 = v;
            }
        }
    }
    if (nk == 0) return;
    if (nk <= 4) {
        // stable insertion by depth, candidates in vertex order
        for (int v = v0; v < v1; v++) {
            if (!(cand >> v & 1u)) continue;
            const float3 r = cyl_offset(b, v);
            const float d = b.c.z + r.z;
            int k = M.np;
            while (k > 0 && d < M.d[k - 1]) {
                M.d[k] = M.d[k - 1];
                M.p[k] = M.p[k - 1];
                k--;
            }
            M.d[k] = d;
            M.p[k] = r;
            M.np++;
        }
        return;
    }
    const float3 p1 = cyl_offset(b, i1);
    unsigned left = cand & ~(1u << i1);
    int i2 = -1;
    float b2 = -1.f;
    for (int v = v0; v < v1; v++) {
        if (!(left >> v & 1u)) continue;
        const float3 e = cyl_offset(b, v) - p1;
        const float l = dot3(e, e);
        if (i2 < 0 || l > b2) {
            b2 = l;
            i2 = v;
        }
    }
    left &= ~(1u << i2);
    const float3 p2 = cyl_offset(b, i2);
    const float3 e2 = p2 - p1;
    auto area = [](float3 e, float3 f) { return e.x * f.y - e.y * f.x; };
    int i3 = -1;
    float b3 = -1.f;
    for (int v = v0; v < v1; v++) {
        if (!(left >> v & 1u)) continue;
        const float a = fabsf(area(e2, cyl_offset(b, v) - p1));
        if (i3 < 0 || a > b3) {
            b3 = a;
            i3 = v;
        }
    }
    left &= ~(1u << i3);
    const float3 p3 = cyl_offset(b, i3);
    const float sgn = area(e2, p3 - p1) < 0.f ? -1.f : 1.f;
    int i4 = -1;
    float b4 = 0.f;
    for (int v = v0; v < v1; v++) {
        if (!(left >> v & 1u)) continue;
        const float3 q = cyl_offset(b, v);
        float a = -sgn * area(e2, q - p1);
        a = fmaxf(a, -sgn * area(p3 - p2, q - p2));
        a = fmaxf(a, -sgn * area(p1 - p3, q - p3));
        if (i4 < 0 || a > b4) {
            b4 = a;
            i4 = v;
        }
    }
    const float3 p4 = cyl_offset(b, i4);
    M.p[0] = p1;
    M.d[0] = b.c.z + p1.z;
    M.p[1] = p2;
    M.d[1] = b.c.z + p2.z;
    M.p[2] = p3;
    M.d[2] = b.c.z + p3.z;
    M.p[3] = p4;
    M.d[3] = b.c.z + p4.z;
    M.np = 4;
}

// Vertical capsule against a cylinder (A = cylinder, B = pusher): as against a box, with
// the cylinder's vertical extent and its closest point to a segment point S (the 16-gon's
// closest point to S's body-plane coordinates -- S's own when inside, else the nearest
// point of the nearest edge, earliest on ties -- with the axial coordinate clamped);
// inside the prism the depth is the smallest distance to a face.
__device__ __forceinline__ void collide_capsule_cyl(const CBox& b, float px, float py, float z0, float z1, float rp,
                                                 float margin, CManifold& M) {
    M.np = 0;
    const float ez = gon_sup(b.R[6], b.R[7]) * b.h[0] + fabsf(b.R[8]) * b.h[2];
    const float zlo = b.c.z - ez, zhi = b.c.z + ez;
    const float za = fmaxf(z0, zlo), zb = fminf(z1, zhi);
    float zc0, zc1 = 0.f;
    int nc;
    if (za > zb) {
        zc0 = (zhi < z0) ? z0 : z1;
        nc = 1;
    } else if (zb - za < 1e-3f) {
        zc0 = (za + zb) * 0.5f;
        nc = 1;
    } else {
        zc0 = za;
        zc1 = zb;
        nc = 2;
    }
    const float r = b.h[0], apo = r * kGonApo;
    float best_d = 0.f;
    float3 best_n = f3(1.f, 0.f, 0.f);
    for (int i = 0; i < nc; i++) {
        const float3 S = f3(px, py, i == 0 ? zc0 : zc1);
        const float3 rel = S - b.c;
        const float lx = dot3(b.ax(0), rel), ly = dot3(b.ax(1), rel), lz = dot3(b.ax(2), rel);
        bool inside = true;
        float pen_side = 3.0e38f;
        #pragma unroll 1
        for (int s = 0; s < 16; s++) {
            float fcs, fss;
            gon_fdir(s, fcs, fss);
            const float gq = apo - (fcs * lx + fss * ly);
            if (gq < 0.f) inside = false;
            pen_side = fminf(pen_side, gq);
        }
        float qx = lx, qy = ly;
        if (!inside) {
            float bd = 0.f;
            #pragma unroll 1
            for (int s = 0; s < 16; s++) {
                float c0, s0, c1, s1;
                gon_vdir(s, c0, s0);
                gon_vdir((s + 1) & 15, c1, s1);
                const float ax = r * c0, ay = r * s0, ex = r * c1 - ax, ey = r * s1 - ay;
                float t = ((lx - ax) * ex + (ly - ay) * ey) / (ex * ex + ey * ey);
                t = fminf(fmaxf(t, 0.f), 1.f);
                const float ppx = ax + ex * t, ppy = ay + ey * t;
                const float dd = (lx - ppx) * (lx - ppx) + (ly - ppy) * (ly - ppy);
                if (s == 0 || dd < bd) {
                    bd = dd;
                    qx = ppx;
                    qy = ppy;
                }
            }
        }
        const float qz = fminf(fmaxf(lz, -b.h[2]), b.h[2]);
        const float3 Q = b.c + b.ax(0) * qx + b.ax(1) * qy + b.ax(2) * qz;
        const float3 diff = S - Q;
        const float dist = norm3(diff);
        float3 nrm;
        float d;
        if (dist > 1e-6f) {
            nrm = diff * (1.f / dist);
            d = dist - rp;
        } else {
            const float pen = fminf(b.h[2] - fabsf(lz), pen_side);
            d = -pen - rp;
            const float3 w = f3(S.x - b.c.x, S.y - b.c.y, 0.f);
            const float lw = norm3(w);
            nrm = lw > 1e-9f ? w * (1.f / lw) : f3(1.f, 0.f, 0.f);
        }
        if (!(d < margin)) continue;
        if (M.np == 0) {
            M.p[0] = Q;
            M.d[0] = d;
        } else {
            M.p[1] = Q;
            M.d[1] = d;
        }
        if (M.np == 0 || d < best_d) {
            best_d = d;
            best_n = nrm;
        }
        M.np++;
    }
    M.n = best_n;
}

}  // namespace pmbs
